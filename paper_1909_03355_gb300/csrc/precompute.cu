// FP64 pre-computation kernels: the pre-computation stage of Fig. 1 (i).
//
//  k_elem_hex / k_elem_tet  element conduction operators (Eq. 12 by 2x2x2 Gauss points for
//                           hexahedra, Eq. 18 for tets), stored as the pair conductances
//                           c_ij = -theta_e K0_e[i][j] (i < j) in the element stream and in an
//                           FP64 copy; shape-function integrals w_ie = int_e N_i dV
//  k_face_share             boundary face area / number of face nodes (nodal lumping)
//  k_node_sums              lumped thermal mass C0_i = sum_e rho c0 w_ie (Section 3.1),
//                           constant nodal loads Q_i = sum_e s_e w_ie + nodal Q, area shares;
//                           fixed-order gathers over node incidence lists (deterministic)
//  k_apply / k_gather       FP64 element operator apply y = sum_e f_k,e K0_e x_e, used by the
//                           power iteration for dt_crit (Section 3.4), the energy balance and
//                           the internal-load query
//  block reductions         fixed-tree FP64 sums (deterministic)
#include <cuda_runtime.h>

#include "fedfem_internal.h"
#include "hexpoint.cuh"
#include "precompute.cuh"

namespace fedfem {

// natural coordinates of the VTK hex nodes
__constant__ signed char c_hex_sign[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                              {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

__device__ __forceinline__ int cond_offset(int p, int lane, int CH, int VW, int rs)
{
    const int v = p / VW, r = p % VW;
    return ((v * CH + lane) * VW + r) * rs;
}

__device__ __forceinline__ void store_cond(uint8_t *chunks, int chunk_bytes, int64_t slot, int CH, int VW,
                                           int precision, int p, double c)
{
    const int64_t chunk = slot / CH;
    const int lane = (int)(slot % CH);
    uint8_t *base = chunks + chunk * (int64_t)chunk_bytes;
    if (precision == 64)
        *reinterpret_cast<double *>(base + cond_offset(p, lane, CH, VW, 8)) = c;
    else
        *reinterpret_cast<float *>(base + cond_offset(p, lane, CH, VW, 4)) = (float)c;
}

__global__ void k_elem_hex(ElemArgs a)
{
    const double g = 0.57735026918962576451;  // 1/sqrt(3)
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.ne; e += (int64_t)gridDim.x * blockDim.x) {
        double x[8][3];
        for (int i = 0; i < 8; ++i) {
            const int64_t n = a.conn[8 * e + i];
            for (int r = 0; r < 3; ++r) x[i][r] = a.xyz[3 * n + r];
        }
        const int m = a.mat ? a.mat[e] : 0;
        const double th = a.kscale ? a.kscale[e] : 1.0;
        double k[9];
        for (int r = 0; r < 9; ++r) k[r] = th * a.mat_k0[9 * m + r];
        double K[28], w[8];
        for (int p = 0; p < 28; ++p) K[p] = 0.0;
        for (int i = 0; i < 8; ++i) w[i] = 0.0;
        bool bad = false;
        // points 0-7: 2x2x2 Gauss (unit weights) for w and, by default, K; point 8: the centre
        // with weight 8 for the one-point conduction matrix of Eq. 17
        const bool centre = a.quad == 1;
        for (int q = 0; q < (centre ? 9 : 8); ++q) {
            const bool is_c = q == 8;
            const double xi = is_c ? 0.0 : g * c_hex_sign[q][0], et = is_c ? 0.0 : g * c_hex_sign[q][1],
                         ze = is_c ? 0.0 : g * c_hex_sign[q][2];
            double N[8], B[8][3], det;
            if (!hex_point(x, xi, et, ze, N, B, det)) {
                bad = true;
                break;
            }
            const bool add_K = centre ? is_c : true;
            const double wk = is_c ? 8.0 * det : det;
            int p = 0;
            for (int i = 0; i < 8; ++i) {
                const double kb0 = k[0] * B[i][0] + k[1] * B[i][1] + k[2] * B[i][2];
                const double kb1 = k[3] * B[i][0] + k[4] * B[i][1] + k[5] * B[i][2];
                const double kb2 = k[6] * B[i][0] + k[7] * B[i][1] + k[8] * B[i][2];
                if (add_K)
                    for (int j = i + 1; j < 8; ++j) {
                        const double t = wk * (B[j][0] * kb0 + B[j][1] * kb1 + B[j][2] * kb2);
                        // the point's own pair conductances (conductivity evaluated at the points)
                        if (a.cond_qp && !is_c) a.cond_qp[(8 * e + q) * 28 + p] = -t;
                        K[p++] += t;
                    }
                if (!is_c) w[i] += det * N[i];
            }
        }
        if (bad) {
            atomicOr(a.err, ERRBIT_MESH);
            atomicMin(a.bad_elem, (unsigned long long)e);
            continue;
        }
        const int64_t slot = a.slot_of_elem[e];
        for (int p = 0; p < 28; ++p) {
            a.cond64[28 * e + p] = -K[p];
            store_cond(a.chunks, a.chunk_bytes, slot, a.CH, a.VW, a.precision, p, -K[p]);
        }
        for (int i = 0; i < 8; ++i) a.W[8 * e + i] = w[i];
    }
}

__global__ void k_elem_tet(ElemArgs a)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.ne; e += (int64_t)gridDim.x * blockDim.x) {
        double x[4][3];
        for (int i = 0; i < 4; ++i) {
            const int64_t n = a.conn[4 * e + i];
            for (int r = 0; r < 3; ++r) x[i][r] = a.xyz[3 * n + r];
        }
        const int m = a.mat ? a.mat[e] : 0;
        const double th = a.kscale ? a.kscale[e] : 1.0;
        // edge matrix E (columns x_i - x_0); grad N_i (i = 1..3) are the rows of E^{-1}
        double E[3][3];
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) E[r][s] = x[s + 1][r] - x[0][r];
        const double C00 = E[1][1] * E[2][2] - E[1][2] * E[2][1];
        const double C01 = E[1][2] * E[2][0] - E[1][0] * E[2][2];
        const double C02 = E[1][0] * E[2][1] - E[1][1] * E[2][0];
        const double det = E[0][0] * C00 + E[0][1] * C01 + E[0][2] * C02;
        if (!(det > 0.0)) {
            atomicOr(a.err, ERRBIT_MESH);
            atomicMin(a.bad_elem, (unsigned long long)e);
            continue;
        }
        const double C10 = E[0][2] * E[2][1] - E[0][1] * E[2][2];
        const double C11 = E[0][0] * E[2][2] - E[0][2] * E[2][0];
        const double C12 = E[0][1] * E[2][0] - E[0][0] * E[2][1];
        const double C20 = E[0][1] * E[1][2] - E[0][2] * E[1][1];
        const double C21 = E[0][2] * E[1][0] - E[0][0] * E[1][2];
        const double C22 = E[0][0] * E[1][1] - E[0][1] * E[1][0];
        const double id = 1.0 / det;
        double G[4][3];
        // row s of E^{-1} is (C0s, C1s, C2s) / det
        G[1][0] = C00 * id, G[1][1] = C10 * id, G[1][2] = C20 * id;
        G[2][0] = C01 * id, G[2][1] = C11 * id, G[2][2] = C21 * id;
        G[3][0] = C02 * id, G[3][1] = C12 * id, G[3][2] = C22 * id;
        for (int r = 0; r < 3; ++r) G[0][r] = -(G[1][r] + G[2][r] + G[3][r]);
        const double V = det / 6.0;
        double k[9];
        for (int r = 0; r < 9; ++r) k[r] = th * a.mat_k0[9 * m + r];
        const int64_t slot = a.slot_of_elem[e];
        int p = 0;
        for (int i = 0; i < 4; ++i) {
            const double kb0 = k[0] * G[i][0] + k[1] * G[i][1] + k[2] * G[i][2];
            const double kb1 = k[3] * G[i][0] + k[4] * G[i][1] + k[5] * G[i][2];
            const double kb2 = k[6] * G[i][0] + k[7] * G[i][1] + k[8] * G[i][2];
            for (int j = i + 1; j < 4; ++j, ++p) {
                const double c = -V * (G[j][0] * kb0 + G[j][1] * kb1 + G[j][2] * kb2);
                a.cond64[6 * e + p] = c;
                store_cond(a.chunks, a.chunk_bytes, slot, a.CH, a.VW, a.precision, p, c);
            }
            a.W[4 * e + i] = 0.25 * V;
        }
    }
}

// Face area share: area of the face / number of its nodes (bilinear patch for quads by
// 2x2 Gauss points; half cross product for triangles).
__global__ void k_face_share(int64_t nf, int nv, const int32_t *faces, const double *xyz, double *share)
{
    const double g = 0.57735026918962576451;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
        double x[4][3];
        for (int i = 0; i < nv; ++i)
            for (int r = 0; r < 3; ++r) x[i][r] = xyz[3 * (int64_t)faces[nv * f + i] + r];
        double A = 0.0;
        if (nv == 3) {
            const double u0 = x[1][0] - x[0][0], u1 = x[1][1] - x[0][1], u2 = x[1][2] - x[0][2];
            const double v0 = x[2][0] - x[0][0], v1 = x[2][1] - x[0][1], v2 = x[2][2] - x[0][2];
            const double n0 = u1 * v2 - u2 * v1, n1 = u2 * v0 - u0 * v2, n2 = u0 * v1 - u1 * v0;
            A = 0.5 * sqrt(n0 * n0 + n1 * n1 + n2 * n2);
        } else {
            const double sg[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
            for (int q = 0; q < 4; ++q) {
                const double s = g * sg[q][0], t = g * sg[q][1];
                double xs[3] = {0, 0, 0}, xt[3] = {0, 0, 0};
                for (int i = 0; i < 4; ++i) {
                    const double ds = 0.25 * sg[i][0] * (1.0 + t * sg[i][1]);
                    const double dt = 0.25 * sg[i][1] * (1.0 + s * sg[i][0]);
                    for (int r = 0; r < 3; ++r) {
                        xs[r] += ds * x[i][r];
                        xt[r] += dt * x[i][r];
                    }
                }
                const double n0 = xs[1] * xt[2] - xs[2] * xt[1];
                const double n1 = xs[2] * xt[0] - xs[0] * xt[2];
                const double n2 = xs[0] * xt[1] - xs[1] * xt[0];
                A += sqrt(n0 * n0 + n1 * n1 + n2 * n2);
            }
        }
        share[f] = A / nv;
    }
}

__global__ void k_node_sums(NodeArgs a)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < a.nn; g += (int64_t)gridDim.x * blockDim.x) {
        double C = 0.0, Q = 0.0;
        for (int q = a.n2e_ptr[g]; q < a.n2e_ptr[g + 1]; ++q) {
            const int64_t ek = a.n2e[q];
            const int64_t e = ek >> 3;
            const int k = (int)(ek & 7);
            const double w = a.W[a.npe * e + k];
            const int m = a.mat ? a.mat[e] : 0;
            C += a.mat_rhoc[m] * w;
            if (a.source) Q += a.source[e] * w;
        }
        if (a.nodal_Q) Q += a.nodal_Q[a.old_of_new[g]];
        double Ac = 0.0, Ar = 0.0;
        if (a.fc_ptr)
            for (int q = a.fc_ptr[g]; q < a.fc_ptr[g + 1]; ++q) Ac += a.fc_share[a.fc_idx[q]];
        if (a.fr_ptr)
            for (int q = a.fr_ptr[g]; q < a.fr_ptr[g + 1]; ++q) Ar += a.fr_share[a.fr_idx[q]];
        a.C0[g] = C;
        a.Qext64[g] = Q;
        a.Ac64[g] = Ac;
        a.Ar64[g] = Ar;
        if (a.Qext32) {
            a.Qext32[g] = (float)Q;
            a.Ac32[g] = (float)Ac;
            a.Ar32[g] = (float)Ar;
        }
    }
}

// A_i = dt / C0_i (Eq. 14 / 21) in FP64, -0.0 on Dirichlet nodes (a zero whose sign bit tells
// the step kernel that the node's value follows the prescribed-temperature schedule);
// optionally also as the float pair (hi, lo) with hi = fl32(A), lo = fl32(A - hi) used by the
// FP32 form.
__global__ void k_set_A(int64_t nn, double dt, const double *C0, const uint8_t *isdir, double *A, float2 *A2)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        const double v = isdir[g] ? -0.0 : dt / C0[g];
        A[g] = v;
        if (A2) {
            const float hi = (float)v;
            A2[g] = make_float2(hi, (float)(v - (double)hi));
        }
    }
}

// y_e = f_k,e (K0_e x_e) in FP64 with K0_e x = sum_{j != i} c_ij (x_i - x_j); f_k,e from the
// element mean of `Tk` (or 1 when Tk == NULL).
template <int NPE>
__global__ void k_apply(int64_t ne, const int32_t *gconn, const double *cond64, const double *x, const double *Tk,
                        double k_a, double k_lin, int tab, HingeLaw<double> tk, double *Y)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        double xv[NPE], F[NPE];
        double s = 0.0;
        for (int k = 0; k < NPE; ++k) {
            const int g = gconn[NPE * e + k];
            xv[k] = x[g];
            if (Tk) s += tab ? hinge_value(tk, Tk[g]) : Tk[g];
            F[k] = 0.0;
        }
        int p = 0;
        for (int i = 0; i < NPE; ++i)
            for (int j = i + 1; j < NPE; ++j) {
                const double gg = cond64[(NPE * (NPE - 1) / 2) * e + p++] * (xv[i] - xv[j]);
                F[i] += gg;
                F[j] -= gg;
            }
        const double fk = Tk ? (tab ? s / NPE : k_a + k_lin * (s / NPE)) : 1.0;
        for (int k = 0; k < NPE; ++k) Y[NPE * e + k] = fk * F[k];
    }
}

// F_g = sum over the node's incidence list (ascending element order) of Y.
__global__ void k_gather(int64_t nn, int npe, const int32_t *n2e_ptr, const int64_t *n2e, const double *Y, double *F)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = n2e_ptr[g]; q < n2e_ptr[g + 1]; ++q) {
            const int64_t ek = n2e[q];
            s += Y[npe * (ek >> 3) + (ek & 7)];
        }
        F[g] = s;
    }
}

// power iteration helpers (free nodes only): u = x / sqrt(C0)
__global__ void k_scale_free(int64_t nn, const double *x, const double *C0, const uint8_t *isdir, double *u)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x)
        u[g] = isdir[g] ? 0.0 : x[g] / sqrt(C0[g]);
}

template <int BS>
__device__ __forceinline__ void block_sum2(double &a, double &b, double *red)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[2 * w] = a;
        red[2 * w + 1] = b;
    }
    __syncthreads();
    if (w == 0) {
        a = l < BS / 32 ? red[2 * l] : 0.0;
        b = l < BS / 32 ? red[2 * l + 1] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

// z = F / sqrt(C0) on free nodes; per-block partial sums of (x . z, z . z)
__global__ void __launch_bounds__(256) k_power_dots(int64_t nn, const double *x, const double *F, const double *C0,
                                                    const uint8_t *isdir, double *z, double *partial)
{
    __shared__ double red[64];
    double a = 0.0, b = 0.0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        const double v = isdir[g] ? 0.0 : F[g] / sqrt(C0[g]);
        z[g] = v;
        a += x[g] * v;
        b += v * v;
    }
    block_sum2<256>(a, b, red);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

// single-block fixed-order sum of per-block partial pairs
__global__ void __launch_bounds__(256) k_sum_partials(int nblocks, const double *partial, double *out)
{
    __shared__ double red[64];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
        a += partial[2 * i];
        b += partial[2 * i + 1];
    }
    block_sum2<256>(a, b, red);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

__global__ void k_normalize(int64_t nn, const double *z, const double *sums, double *x)
{
    const double inv = 1.0 / sqrt(sums[1]);
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x)
        x[g] = z[g] * inv;
}

// Lanczos steps for the largest eigenvalue of M = C0^-1/2 K0 C0^-1/2 on the free nodes (the
// vectors are zero on Dirichlet nodes).  Step j: w = M v_j - beta_{j-1} v_{j-1},
// alpha_j = w . v_j, w -= alpha_j v_j, beta_j^2 = w . w, v_{j+1} = w / beta_j.  The
// coefficients stay in device memory (read by the next kernels); the host reads them in batches.

// w = C0^-1/2 F - beta_{j-1} v_{j-1} (free nodes), written over F; partial sums of w . v_j
__global__ void __launch_bounds__(256) k_lz_w(int64_t nn, double *F, const double *C0, const uint8_t *isdir,
                                              const double *vprev, const double *beta2_prev, const double *vcur,
                                              double *partial)
{
    __shared__ double red[64];
    const double b = beta2_prev ? sqrt(*beta2_prev) : 0.0;
    double a = 0.0, z = 0.0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        const double w = isdir[g] ? 0.0 : F[g] / sqrt(C0[g]) - (beta2_prev ? b * vprev[g] : 0.0);
        F[g] = w;
        a += w * vcur[g];
    }
    block_sum2<256>(a, z, red);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = 0.0;
    }
}

// w -= alpha_j v_j; partial sums of w . w (alpha == NULL: plain squared norm)
__global__ void __launch_bounds__(256) k_lz_orth(int64_t nn, double *w, const double *vcur, const double *alpha,
                                                 double *partial)
{
    __shared__ double red[64];
    const double al = alpha ? *alpha : 0.0;
    double s = 0.0, z = 0.0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        const double x = alpha ? w[g] - al * vcur[g] : w[g];
        if (alpha) w[g] = x;
        s += x * x;
    }
    block_sum2<256>(s, z, red);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = s;
        partial[2 * blockIdx.x + 1] = 0.0;
    }
}

// v_{j+1} = w / beta_j (zero once beta_j underflows: the Krylov space is exhausted)
__global__ void k_lz_next(int64_t nn, const double *w, const double *beta2, double *vnext)
{
    const double b2 = *beta2;
    const double inv = b2 > 1e-280 ? 1.0 / sqrt(b2) : 0.0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x)
        vnext[g] = w[g] * inv;
}

// per-block (min, max) of x over all nodes
__global__ void __launch_bounds__(256) k_minmax(int64_t nn, const double *x, double *partial)
{
    __shared__ double red[16];
    double lo = 1e300, hi = -1e300;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        lo = fmin(lo, x[g]);
        hi = fmax(hi, x[g]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[2 * (threadIdx.x >> 5)] = lo;
        red[2 * (threadIdx.x >> 5) + 1] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = fmin(lo, red[2 * w]);
            hi = fmax(hi, red[2 * w + 1]);
        }
        partial[2 * blockIdx.x] = fmin(lo, red[0]);
        partial[2 * blockIdx.x + 1] = fmax(hi, red[1]);
    }
}

__global__ void k_init_power(int64_t nn, const uint8_t *isdir, double *x)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x)
        x[g] = isdir[g] ? 0.0 : 1.0 + 0.5 * sin(1.3 * (double)g + 0.2);
}

// Largest linearised surface rate max_i (A^c h + A^r 4 sigma eps r3) / (C0 fc_min) on free nodes
// (per-block maxima in partial[2*b]).
__global__ void __launch_bounds__(256) k_surface_rate(int64_t nn, const double *Ac, const double *Ar,
                                                      const double *C0, const uint8_t *isdir, double h,
                                                      double rad_coef, double fc_min, double *partial)
{
    __shared__ double red[8];
    double m = 0.0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x)
        if (!isdir[g]) m = fmax(m, (Ac[g] * h + Ar[g] * rad_coef) / (C0[g] * fc_min));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        partial[2 * blockIdx.x] = m;
        partial[2 * blockIdx.x + 1] = 0.0;
    }
}

// ---- state conversion (new node order) ----
template <typename R>
__global__ void k_state_to_f64(int64_t nn, const R *T, const float *comp, double *out)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x)
        out[g] = (double)T[g] - (comp ? (double)comp[g] : 0.0);
}
template __global__ void k_state_to_f64<float>(int64_t, const float *, const float *, double *);
template __global__ void k_state_to_f64<double>(int64_t, const double *, const float *, double *);

// old-order FP64 field -> working state (new order); Kahan compensation = T_hi - T0
template <typename R>
__global__ void k_set_state(int64_t nn, const double *T0_old, const int32_t *old_of_new, R *T, float *comp)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        const double v = T0_old[old_of_new[g]];
        const R r = (R)v;
        T[g] = r;
        if (comp) comp[g] = (float)((double)r - v);
    }
}
template __global__ void k_set_state<float>(int64_t, const double *, const int32_t *, float *, float *);
template __global__ void k_set_state<double>(int64_t, const double *, const int32_t *, double *, float *);

__global__ void k_impose_dirichlet(int64_t nd, const int32_t *dir_new, const double *dir_T, double offset,
                                   double *T0_old, const int32_t *old_of_new)
{
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < nd; d += (int64_t)gridDim.x * blockDim.x)
        T0_old[old_of_new[dir_new[d]]] = dir_T[d] + offset;
}

// prescribed values dir_T + offset written into the working state (new order), with the
// compensation of k_set_state
template <typename R>
__global__ void k_impose_dirichlet_state(int64_t nd, const int32_t *dir_new, const double *dir_T, double offset, R *T,
                                         float *comp)
{
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < nd; d += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = dir_new[d];
        const double v = dir_T[d] + offset;
        const R r = (R)v;
        T[g] = r;
        if (comp) comp[g] = (float)((double)r - v);
    }
}

__global__ void k_permute_new_to_old(int64_t nn, const double *x_new, const int32_t *old_of_new, double *x_old)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x)
        x_old[old_of_new[g]] = x_new[g];
}

__global__ void k_permute_old_to_new(int64_t nn, const double *x_old, const int32_t *old_of_new, double *x_new)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x)
        x_new[g] = x_old[old_of_new[g]];
}

// Energy terms of one step (FP64): per block partial sums of
//   S = sum_free C0 f_c(T0) (T1 - T0),  B = dt (sum_free Q(T0) + sum_dir F(T0)).
__global__ void __launch_bounds__(256) k_energy_terms(int64_t nn, const double *T0, const double *T1,
                                                      const double *F, const double *C0, const double *Qext,
                                                      const double *Ac, const double *Ar, const uint8_t *isdir,
                                                      EnergyPhys ph, double *partial)
{
    __shared__ double red[64];
    double S = 0.0, B = 0.0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        if (isdir[g]) {
            B += ph.dt * F[g];
            continue;
        }
        const double t = T0[g];
        const double u = t - ph.T_zero, b = ph.T_amb - ph.T_zero;
        const double Q = ph.qs * Qext[g] - Ac[g] * ph.h * (t - ph.T_inf) - Ar[g] * ph.eps_sigma * ((u - b) * (u + b) * (u * u + b * b));
        S += C0[g] * (ph.tab ? hinge_value(ph.tc, t) : ph.c_a + ph.c_lin * t) * (T1[g] - t);
        B += ph.dt * Q;
    }
    block_sum2<256>(S, B, red);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = S;
        partial[2 * blockIdx.x + 1] = B;
    }
}

// ---- host wrappers ----
static int nblk(int64_t n, int bs = 256, int cap = 4096)
{
    int64_t b = (n + bs - 1) / bs;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

void launch_elem(int npe, const ElemArgs &a, cudaStream_t st)
{
    if (npe == 8)
        k_elem_hex<<<nblk(a.ne, 128), 128, 0, st>>>(a);
    else
        k_elem_tet<<<nblk(a.ne, 128), 128, 0, st>>>(a);
}

void launch_face_share(int64_t nf, int nv, const int32_t *faces, const double *xyz, double *share, cudaStream_t st)
{
    if (nf > 0) k_face_share<<<nblk(nf), 256, 0, st>>>(nf, nv, faces, xyz, share);
}

void launch_node_sums(const NodeArgs &a, cudaStream_t st) { k_node_sums<<<nblk(a.nn), 256, 0, st>>>(a); }

void launch_set_A(int64_t nn, double dt, const double *C0, const uint8_t *isdir, double *A, float2 *A2,
                  cudaStream_t st)
{
    k_set_A<<<nblk(nn), 256, 0, st>>>(nn, dt, C0, isdir, A, A2);
}

void launch_apply(int npe, int64_t ne, int64_t nn, const int32_t *gconn, const double *cond64, const int32_t *n2e_ptr,
                  const int64_t *n2e, const double *x, const double *Tk, double k_a, double k_lin,
                  const HingeLaw<double> *tk, double *Y, double *F, cudaStream_t st)
{
    const int tab = tk != nullptr;
    const HingeLaw<double> law = tk ? *tk : HingeLaw<double>{};
    if (npe == 8)
        k_apply<8><<<nblk(ne), 256, 0, st>>>(ne, gconn, cond64, x, Tk, k_a, k_lin, tab, law, Y);
    else
        k_apply<4><<<nblk(ne), 256, 0, st>>>(ne, gconn, cond64, x, Tk, k_a, k_lin, tab, law, Y);
    k_gather<<<nblk(nn), 256, 0, st>>>(nn, npe, n2e_ptr, n2e, Y, F);
}

int reduce_blocks(int64_t nn) { return nblk(nn, 256, 1024); }

void launch_power_init(int64_t nn, const uint8_t *isdir, double *x, cudaStream_t st)
{
    k_init_power<<<nblk(nn), 256, 0, st>>>(nn, isdir, x);
}

void launch_scale_free(int64_t nn, const double *x, const double *C0, const uint8_t *isdir, double *u, cudaStream_t st)
{
    k_scale_free<<<nblk(nn), 256, 0, st>>>(nn, x, C0, isdir, u);
}

void launch_power_dots(int64_t nn, const double *x, const double *F, const double *C0, const uint8_t *isdir, double *z,
                       double *partial, double *sums, cudaStream_t st)
{
    const int nb = reduce_blocks(nn);
    k_power_dots<<<nb, 256, 0, st>>>(nn, x, F, C0, isdir, z, partial);
    k_sum_partials<<<1, 256, 0, st>>>(nb, partial, sums);
}

void launch_lanczos_start(int64_t nn, const uint8_t *isdir, double *x, double *v0, double *partial, double *norm2,
                          cudaStream_t st)
{
    const int nb = reduce_blocks(nn);
    k_init_power<<<nblk(nn), 256, 0, st>>>(nn, isdir, x);
    k_lz_orth<<<nb, 256, 0, st>>>(nn, x, nullptr, nullptr, partial);
    k_sum_partials<<<1, 256, 0, st>>>(nb, partial, norm2);
    k_lz_next<<<nblk(nn), 256, 0, st>>>(nn, x, norm2, v0);
}

void launch_lanczos_step(int npe, int64_t ne, int64_t nn, const int32_t *gconn, const double *cond64,
                         const int32_t *n2e_ptr, const int64_t *n2e, const double *C0, const uint8_t *isdir,
                         double *vprev, const double *vcur, double *u, double *F, double *Y, const double *beta2_prev,
                         double *coef, double *partial, cudaStream_t st)
{
    const int nb = reduce_blocks(nn);
    k_scale_free<<<nblk(nn), 256, 0, st>>>(nn, vcur, C0, isdir, u);
    launch_apply(npe, ne, nn, gconn, cond64, n2e_ptr, n2e, u, nullptr, 1.0, 0.0, nullptr, Y, F, st);
    k_lz_w<<<nb, 256, 0, st>>>(nn, F, C0, isdir, vprev, beta2_prev, vcur, partial);
    k_sum_partials<<<1, 256, 0, st>>>(nb, partial, coef);  // coef[0] = alpha_j
    k_lz_orth<<<nb, 256, 0, st>>>(nn, F, vcur, coef, partial);
    k_sum_partials<<<1, 256, 0, st>>>(nb, partial, coef + 2);  // coef[2] = beta_j^2
    k_lz_next<<<nblk(nn), 256, 0, st>>>(nn, F, coef + 2, vprev);  // v_{j+1} over v_{j-1}
}

int launch_minmax(int64_t nn, const double *x, double *partial, cudaStream_t st)
{
    const int nb = reduce_blocks(nn);
    k_minmax<<<nb, 256, 0, st>>>(nn, x, partial);
    return nb;
}

void launch_normalize(int64_t nn, const double *z, const double *sums, double *x, cudaStream_t st)
{
    k_normalize<<<nblk(nn), 256, 0, st>>>(nn, z, sums, x);
}

int launch_surface_rate(int64_t nn, const double *Ac, const double *Ar, const double *C0, const uint8_t *isdir, double h,
                        double rad_coef, double fc_min, double *partial, cudaStream_t st)
{
    const int nb = reduce_blocks(nn);
    k_surface_rate<<<nb, 256, 0, st>>>(nn, Ac, Ar, C0, isdir, h, rad_coef, fc_min, partial);
    return nb;
}

void launch_state_to_f64(int precision, int64_t nn, const void *T, const float *comp, double *out, cudaStream_t st)
{
    if (precision == 64)
        k_state_to_f64<double><<<nblk(nn), 256, 0, st>>>(nn, (const double *)T, nullptr, out);
    else
        k_state_to_f64<float><<<nblk(nn), 256, 0, st>>>(nn, (const float *)T, comp, out);
}

void launch_set_state(int precision, int64_t nn, const double *T0_old, const int32_t *old_of_new, void *T, float *comp,
                      cudaStream_t st)
{
    if (precision == 64)
        k_set_state<double><<<nblk(nn), 256, 0, st>>>(nn, T0_old, old_of_new, (double *)T, nullptr);
    else
        k_set_state<float><<<nblk(nn), 256, 0, st>>>(nn, T0_old, old_of_new, (float *)T, comp);
}

void launch_impose_dirichlet(int64_t nd, const int32_t *dir_new, const double *dir_T, double offset, double *T0_old,
                             const int32_t *old_of_new, cudaStream_t st)
{
    if (nd > 0) k_impose_dirichlet<<<nblk(nd), 256, 0, st>>>(nd, dir_new, dir_T, offset, T0_old, old_of_new);
}

void launch_impose_dirichlet_state(int precision, int64_t nd, const int32_t *dir_new, const double *dir_T,
                                   double offset, void *T, float *comp, cudaStream_t st)
{
    if (nd <= 0) return;
    if (precision == 64)
        k_impose_dirichlet_state<double><<<nblk(nd), 256, 0, st>>>(nd, dir_new, dir_T, offset, (double *)T, nullptr);
    else
        k_impose_dirichlet_state<float><<<nblk(nd), 256, 0, st>>>(nd, dir_new, dir_T, offset, (float *)T, comp);
}

void launch_permute_new_to_old(int64_t nn, const double *x_new, const int32_t *old_of_new, double *x_old, cudaStream_t st)
{
    k_permute_new_to_old<<<nblk(nn), 256, 0, st>>>(nn, x_new, old_of_new, x_old);
}

void launch_permute_old_to_new(int64_t nn, const double *x_old, const int32_t *old_of_new, double *x_new, cudaStream_t st)
{
    k_permute_old_to_new<<<nblk(nn), 256, 0, st>>>(nn, x_old, old_of_new, x_new);
}

void launch_energy(int64_t nn, const double *T0, const double *T1, const double *F, const double *C0, const double *Qext,
                   const double *Ac, const double *Ar, const uint8_t *isdir, const EnergyPhys &ph, double *partial,
                   double *sums, cudaStream_t st)
{
    const int nb = reduce_blocks(nn);
    k_energy_terms<<<nb, 256, 0, st>>>(nn, T0, T1, F, C0, Qext, Ac, Ar, isdir, ph, partial);
    k_sum_partials<<<1, 256, 0, st>>>(nb, partial, sums);
}

}  // namespace fedfem
