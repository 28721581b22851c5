// Method variants of the explicit step, run as three plain launches per step.
//
//  conductivity at the quadrature points (kT_eval = 1): Eq. 20 with D(T) inside the integral,
//      F_e = theta_e sum_q f_k(T_q) K_{e,q} T_e,  T_q = sum_i N_i(xi_q) T_i,
//      K_{e,q} the contribution of point q to K0_e (2x2x2 Gauss points of a hexahedron; its
//      centre with the one-point rule of Eq. 17; the centroid of a linear tet, where the
//      gradients are constant).  Each K_{e,q} has zero row sums, so the loads keep the
//      difference form F_i = f_q sum_j c_{q,ij} (T_i - T_j).
//  consistent face integration (face_quadrature = 1): Eq. 4 and Eq. 7 integrated with the face
//      shape functions: convection Q_i -= h sum_j M_ij (T_j - T_inf) with the face mass matrix
//      M_ij = int_f N_i N_j dA, radiation Q_i -= eps sigma sum_p w_p N_i(p) ((T_p - T_z)^4 -
//      (T_amb - T_z)^4) over the face rule (3x3 Gauss-Legendre points on quadrilaterals, Radon's
//      7-point degree-5 rule on triangles).
//
// One step: k_var_elem (one thread per element: element loads into per-element slots),
// k_var_face (one thread per boundary face: face loads into per-face slots), k_var_node (one
// thread per node: the node's element and face loads gathered in ascending element / face
// order, then the update of Eq. 16 with the same Kahan compensation and Dirichlet handling as
// the persistent kernel).  Deterministic; the state lives in the context's arrays (tiling node
// order, step-parity double buffers), so set_T, get_T and the adaptive step are unchanged.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"
#include "hexpoint.cuh"
#include "update.cuh"

#define CK(call, where)                                          \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where);   \
    } while (0)

namespace fedfem {

namespace {

constexpr int kThreads = 128;

int blocks_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 1 << 20)); }

// Natural coordinate of 2x2x2 point q (VTK corner order) along axis d: +-1/sqrt(3).
__device__ __forceinline__ double gauss2(int q, int d) { return 0.57735026918962576451 * hex_sign(q, d); }

// Shape values of the quadrature points: 2x2x2 hexahedron points, or one point (centre /
// centroid) where every N_i = 1 / npe.
template <int NPE>
__device__ __forceinline__ double point_N(int nq, int q, int i)
{
    if (NPE == 8 && nq == 8) {
        double v = 0.125;
        for (int d = 0; d < 3; ++d) v *= 1.0 + hex_sign(i, d) * gauss2(q, d);
        return v;
    }
    return 1.0 / NPE;
}

// Face rule: point p of nfq, shape values N [nv] and the reference weight (quadrilateral:
// weights on [-1,1]^2, summing to 4; triangle: weights summing to 1).
__device__ __forceinline__ void face_point(int nv, int p, double *N, double &w)
{
    if (nv == 4) {
        const double g = 0.77459666924148337704;  // sqrt(3/5)
        const int a = p / 3, b = p % 3;
        const double s = (a - 1) * g, t = (b - 1) * g;
        const double ws = a == 1 ? 8.0 / 9.0 : 5.0 / 9.0, wt = b == 1 ? 8.0 / 9.0 : 5.0 / 9.0;
        const double S[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
        for (int i = 0; i < 4; ++i) N[i] = 0.25 * (1.0 + s * S[i][0]) * (1.0 + t * S[i][1]);
        w = ws * wt;
        return;
    }
    // Radon's degree-5 rule: the centroid and two orbits (a, a, 1 - 2a), a = (6 -+ sqrt 15) / 21
    const double r = 3.87298334620741688698;  // sqrt(15)
    if (p == 0) {
        N[0] = N[1] = N[2] = 1.0 / 3.0;
        w = 9.0 / 40.0;
        return;
    }
    const int orbit = (p - 1) / 3, k = (p - 1) % 3;
    const double a = orbit == 0 ? (6.0 - r) / 21.0 : (6.0 + r) / 21.0;
    for (int i = 0; i < 3; ++i) N[i] = i == k ? 1.0 - 2.0 * a : a;
    w = orbit == 0 ? (155.0 - r) / 1200.0 : (155.0 + r) / 1200.0;
}

// Pair conductances per point into SoA [q * np + p][ne] (FP64 and the working precision): from
// the per-point FP64 values [ne][8][28] of 2x2x2 hexahedra, or (one point) from cond64.
template <typename R>
__global__ void k_var_pack(int64_t ne, int nq, int np, const double *cond_qp64, const double *cond64, double *vq64,
                           R *vq)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x)
        for (int q = 0; q < nq; ++q)
            for (int p = 0; p < np; ++p) {
                const double v = nq > 1 ? cond_qp64[((int64_t)nq * e + q) * np + p] : cond64[(int64_t)np * e + p];
                vq64[(int64_t)(q * np + p) * ne + e] = v;
                vq[(int64_t)(q * np + p) * ne + e] = (R)v;
            }
}

// Face mass matrices of the convection faces and quadrature weights x area Jacobian of the
// radiation faces (FP64 and the working precision).  faces: original node ids.
template <typename R>
__global__ void k_var_faces(int64_t n_conv, int64_t n_rad, int nv, int nfq, const int32_t *conv, const int32_t *rad,
                            const double *xyz, double *Mf64, R *Mf, double *Wf64, R *Wf)
{
    const int64_t nf = n_conv + n_rad;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
        const bool is_conv = f < n_conv;
        const int32_t *v = is_conv ? conv + (int64_t)nv * f : rad + (int64_t)nv * (f - n_conv);
        double x[4][3];
        for (int i = 0; i < nv; ++i)
            for (int r = 0; r < 3; ++r) x[i][r] = xyz[3 * (int64_t)v[i] + r];
        double W[9], Nall[9][4];
        double area_tri = 0.0;
        if (nv == 3) {
            const double a0 = x[1][0] - x[0][0], a1 = x[1][1] - x[0][1], a2 = x[1][2] - x[0][2];
            const double b0 = x[2][0] - x[0][0], b1 = x[2][1] - x[0][1], b2 = x[2][2] - x[0][2];
            const double c0 = a1 * b2 - a2 * b1, c1 = a2 * b0 - a0 * b2, c2 = a0 * b1 - a1 * b0;
            area_tri = 0.5 * sqrt(c0 * c0 + c1 * c1 + c2 * c2);
        }
        for (int p = 0; p < nfq; ++p) {
            double w;
            face_point(nv, p, Nall[p], w);
            if (nv == 3) {
                W[p] = w * area_tri;
                continue;
            }
            // |x_s x x_t| of the bilinear patch at the point
            const double g = 0.77459666924148337704;
            const double s = (p / 3 - 1) * g, t = (p % 3 - 1) * g;
            const double S[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
            double xs[3] = {0, 0, 0}, xt[3] = {0, 0, 0};
            for (int i = 0; i < 4; ++i)
                for (int r = 0; r < 3; ++r) {
                    xs[r] += x[i][r] * S[i][0] * (1.0 + t * S[i][1]) * 0.25;
                    xt[r] += x[i][r] * (1.0 + s * S[i][0]) * S[i][1] * 0.25;
                }
            const double c0 = xs[1] * xt[2] - xs[2] * xt[1], c1 = xs[2] * xt[0] - xs[0] * xt[2],
                         c2 = xs[0] * xt[1] - xs[1] * xt[0];
            W[p] = w * sqrt(c0 * c0 + c1 * c1 + c2 * c2);
        }
        if (is_conv) {
            for (int i = 0; i < nv; ++i)
                for (int j = 0; j < nv; ++j) {
                    double m = 0.0;
                    for (int p = 0; p < nfq; ++p) m += W[p] * Nall[p][i] * Nall[p][j];
                    Mf64[((int64_t)nv * f + i) * nv + j] = m;
                    Mf[((int64_t)nv * f + i) * nv + j] = (R)m;
                }
        } else {
            const int64_t fr = f - n_conv;
            for (int p = 0; p < nfq; ++p) {
                Wf64[(int64_t)nfq * fr + p] = W[p];
                Wf[(int64_t)nfq * fr + p] = (R)W[p];
            }
        }
    }
}

// Conductivity law at a temperature: linear (k_a + k_lin T) or the tabulated hinge form.
template <typename R, bool TAB>
__device__ __forceinline__ R law_at(const HingeLaw<R> &tk, R k_a, R k_lin, R T)
{
    return TAB ? hinge_value(tk, T) : k_a + k_lin * T;
}

// Element loads of one step into Y [ne][NPE]: with qp, f_k at each quadrature point's
// temperature; without (nq = 1), the element mean of the nodal factors of Section 4.2.2.
template <typename R, int NPE, bool TAB>
__global__ void __launch_bounds__(kThreads) k_var_elem(int64_t ne, int nq, int qp, const int32_t *gconn, const R *vq,
                                                        const R *T, R k_a, R k_lin, HingeLaw<R> tk, R *Y)
{
    constexpr int NP = NPE * (NPE - 1) / 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        R Te[NPE], F[NPE];
        R fmean = 0;
        for (int k = 0; k < NPE; ++k) {
            Te[k] = T[gconn[(int64_t)NPE * e + k]];
            F[k] = 0;
            if (!qp) fmean += TAB ? hinge_value(tk, Te[k]) : Te[k];
        }
        fmean = TAB ? fmean * ((R)1 / (R)NPE) : k_a + k_lin * (fmean * ((R)1 / (R)NPE));
        for (int q = 0; q < nq; ++q) {
            R f = fmean;
            if (qp) {
                R Tq = 0;
                for (int i = 0; i < NPE; ++i) Tq += (R)point_N<NPE>(nq, q, i) * Te[i];
                f = law_at<R, TAB>(tk, k_a, k_lin, Tq);
            }
            R Fq[NPE];
            for (int k = 0; k < NPE; ++k) Fq[k] = 0;
            int p = 0;
            for (int i = 0; i < NPE; ++i)
                for (int j = i + 1; j < NPE; ++j, ++p) {
                    const R g = vq[(int64_t)(q * NP + p) * ne + e] * (Te[i] - Te[j]);
                    Fq[i] += g;
                    Fq[j] -= g;
                }
            for (int k = 0; k < NPE; ++k) F[k] += f * Fq[k];
        }
        for (int k = 0; k < NPE; ++k) Y[(int64_t)NPE * e + k] = F[k];
    }
}

// Face loads of one step into Yf [n_conv + n_rad][nv] (faces in the tiling's node ids):
// convection -h M (T - T_inf), radiation -eps sigma sum_p W_p N(p) (u^4 - b^4) with the quartic
// difference factored as (u - b)(u + b)(u^2 + b^2).
template <typename R>
__global__ void __launch_bounds__(kThreads) k_var_face(int64_t n_conv, int64_t n_rad, int nv, int nfq,
                                                        const int32_t *cf, const int32_t *rf, const R *Mf, const R *Wf,
                                                        const R *T, R h, R T_inf, R eps_sigma, R T_amb, R T_zero, R *Yf)
{
    const int64_t nf = n_conv + n_rad;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
        R Tv[4], out[4] = {0, 0, 0, 0};
        if (f < n_conv) {
            for (int i = 0; i < nv; ++i) Tv[i] = T[cf[(int64_t)nv * f + i]] - T_inf;
            for (int i = 0; i < nv; ++i) {
                R acc = 0;
                for (int j = 0; j < nv; ++j) acc += Mf[((int64_t)nv * f + i) * nv + j] * Tv[j];
                out[i] = -h * acc;
            }
        } else {
            const int64_t fr = f - n_conv;
            for (int i = 0; i < nv; ++i) Tv[i] = T[rf[(int64_t)nv * fr + i]];
            const R b = T_amb - T_zero;
            for (int p = 0; p < nfq; ++p) {
                double Nd[4], w;
                face_point(nv, p, Nd, w);
                R Tp = 0;
                for (int j = 0; j < nv; ++j) Tp += (R)Nd[j] * Tv[j];
                const R u = Tp - T_zero;
                const R flux = eps_sigma * ((u - b) * (u + b) * (u * u + b * b));
                const R wf = Wf[(int64_t)nfq * fr + p] * flux;
                for (int i = 0; i < nv; ++i) out[i] -= wf * (R)Nd[i];
            }
        }
        for (int i = 0; i < nv; ++i) Yf[(int64_t)nv * f + i] = out[i];
    }
}

// Load of node g from the face slots of its faces (ascending face order): the slot of g in
// face f is found by its id among the face's nodes.
template <typename R>
__device__ __forceinline__ R face_sum(int g, const int32_t *ptr, const int32_t *idx, const int32_t *faces, int nv,
                                      int64_t slot0, const R *Yf)
{
    R s = 0;
    if (!ptr) return s;
    for (int q = ptr[g]; q < ptr[g + 1]; ++q) {
        const int64_t f = idx[q];
        int k = 0;
        while (k < nv - 1 && faces[(int64_t)nv * f + k] != g) ++k;
        s += Yf[(int64_t)nv * (slot0 + f) + k];
    }
    return s;
}

struct VarFaces {
    const int32_t *fc_ptr, *fc_idx, *fr_ptr, *fr_idx, *cf, *rf;
    int64_t n_conv;
    int nv, consistent;
};

// Node pass of one step: gather the element loads (ascending element order) and, with
// consistent faces, the face loads; then the explicit update of Eq. 16.  Lumped faces use the
// nodal area shares as the persistent kernel does.
template <typename R, bool KAHAN, bool TAB>
__global__ void __launch_bounds__(kThreads) k_var_node(int64_t nn, int npe, const int32_t *n2e_ptr, const int64_t *n2e,
                                                        const R *Y, VarFaces vf, const R *Yf, const R *T, const float *comp,
                                                        const float2 *A2, const double *A, const R *Qext, const R *Ac,
                                                        const R *Ar, PhysParams pp, double qs, double T_inf, double dD,
                                                        HingeLaw<R> tc, R *Tn, float *comp_n, int32_t *err)
{
    Phys<R> ph(pp);
    ph.qs = (R)qs;
    ph.T_inf = (R)T_inf;
    ph.dD = (R)dD;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        R F = 0;
        for (int q = n2e_ptr[g]; q < n2e_ptr[g + 1]; ++q) {
            const int64_t ek = n2e[q];
            F += Y[(int64_t)npe * (ek >> 3) + (ek & 7)];
        }
        const R Tg = T[g];
        R Q = Qext[g] * ph.qs;
        if (vf.consistent) {
            Q += face_sum<R>((int)g, vf.fc_ptr, vf.fc_idx, vf.cf, vf.nv, 0, Yf);
            Q += face_sum<R>((int)g, vf.fr_ptr, vf.fr_idx, vf.rf, vf.nv, vf.n_conv, Yf);
        } else {
            F += surface_outflow<R>(Tg, Ac[g], Ar[g], ph);
        }
        float cn;
        ACoef<R> a;
        if constexpr (sizeof(R) == 4)
            a.v = A2[g];
        else
            a.v = A[g];
        Tn[g] = node_update<R, KAHAN, TAB>(Tg, KAHAN ? comp[g] : 0.0f, a, Q, F, ph.dD, ph, tc, cn, err);
        if (KAHAN) comp_n[g] = cn;
    }
}

// FP64 gathers for load queries: element loads and face loads per node.
__global__ void k_var_gather64(int64_t nn, int npe, const int32_t *n2e_ptr, const int64_t *n2e, const double *Y,
                               VarFaces vf, const double *Yf, const double *Qext, double qs, double *F, double *Qs)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = n2e_ptr[g]; q < n2e_ptr[g + 1]; ++q) {
            const int64_t ek = n2e[q];
            s += Y[(int64_t)npe * (ek >> 3) + (ek & 7)];
        }
        F[g] = s;
        if (Qs)
            Qs[g] = qs * Qext[g] + face_sum<double>((int)g, vf.fc_ptr, vf.fc_idx, vf.cf, vf.nv, 0, Yf) +
                    face_sum<double>((int)g, vf.fr_ptr, vf.fr_idx, vf.rf, vf.nv, vf.n_conv, Yf);
    }
}

}  // namespace

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
namespace {

VarFaces var_faces(const fedfem_ctx *c)
{
    VarFaces vf;
    vf.fc_ptr = c->n_conv ? c->d_fc_ptr : nullptr;
    vf.fc_idx = c->d_fc_idx;
    vf.fr_ptr = c->n_rad ? c->d_fr_ptr : nullptr;
    vf.fr_idx = c->d_fr_idx;
    vf.cf = c->d_cf_new;
    vf.rf = c->d_rf_new;
    vf.n_conv = c->n_conv;
    vf.nv = c->face_nv;
    vf.consistent = c->face_cons;
    return vf;
}

PhysParams phys_of(const fedfem_ctx *c)
{
    return PhysParams{c->k_lin, c->c_lin, c->h, c->T_inf, c->eps * 5.67e-8, c->T_amb, c->T_zero, c->opt.T_guard,
                      c->k_a(), c->c_a()};
}

template <typename R>
HingeLaw<R> law_copy(const HingeLaw<double> &h);
template <>
HingeLaw<double> law_copy<double>(const HingeLaw<double> &h)
{
    return h;
}
template <>
HingeLaw<float> law_copy<float>(const HingeLaw<double> &h)
{
    return hinge_law_f32(h);
}

// One step of the variant path on the context's state (step c->step -> c->step + 1).
template <typename R, int NPE, bool TAB, bool KAHAN>
cudaError_t var_step(fedfem_ctx *c)
{
    const int64_t n0 = c->step;
    const int cur = (int)(n0 & 1), nxt = cur ^ 1;
    const R *T = static_cast<const R *>(c->d_T[cur]);
    const HingeLaw<R> tk = law_copy<R>(c->hk), tc = law_copy<R>(c->hc);
    k_var_elem<R, NPE, TAB><<<blocks_for(c->ne), kThreads, 0, c->stream>>>(
        c->ne, c->nq, c->kT_qp, c->d_gconn, static_cast<const R *>(c->d_vq), T, (R)c->k_a(), (R)c->k_lin, tk,
        static_cast<R *>(c->d_Yv));
    if (c->face_cons && c->n_conv + c->n_rad > 0)
        k_var_face<R><<<blocks_for(c->n_conv + c->n_rad), kThreads, 0, c->stream>>>(
            c->n_conv, c->n_rad, c->face_nv, c->nfq, c->d_cf_new, c->d_rf_new, static_cast<const R *>(c->d_Mf),
            static_cast<const R *>(c->d_Wf), T, (R)c->h, (R)c->Tinf_at(n0), (R)(c->eps * 5.67e-8), (R)c->T_amb,
            (R)c->T_zero, static_cast<R *>(c->d_Yf));
    const double dD = c->Tdir_at(n0 + 1) - c->Tdir_at(n0);
    k_var_node<R, KAHAN, TAB><<<blocks_for(c->nn), kThreads, 0, c->stream>>>(
        c->nn, c->npe, c->d_n2e_ptr, c->d_n2e, static_cast<const R *>(c->d_Yv), var_faces(c),
        static_cast<const R *>(c->d_Yf), T, KAHAN ? c->d_comp[cur] : nullptr, c->d_A2, c->d_A,
        static_cast<const R *>(c->d_Qext), static_cast<const R *>(c->d_Ac), static_cast<const R *>(c->d_Ar), phys_of(c),
        c->qs_at(n0), c->Tinf_at(n0), dD, tc, static_cast<R *>(c->d_T[nxt]), KAHAN ? c->d_comp[nxt] : nullptr,
        c->d_err);
    return cudaGetLastError();
}

template <typename R, bool KAHAN>
cudaError_t var_step_dispatch(fedfem_ctx *c)
{
    const bool tab = c->n_tab > 0;
    if (c->npe == 8) return tab ? var_step<R, 8, true, KAHAN>(c) : var_step<R, 8, false, KAHAN>(c);
    return tab ? var_step<R, 4, true, KAHAN>(c) : var_step<R, 4, false, KAHAN>(c);
}

}  // namespace

fedfem_status variant_init(fedfem_ctx *c)
{
    const int64_t ne = c->ne, npe = c->npe;
    const size_t rs = c->precision == 64 ? 8 : 4;
    const int np = n_pairs(c->npe);
    c->nq = (c->kT_qp && npe == 8 && c->opt.quadrature != 1) ? 8 : 1;
    c->nfq = c->face_cons ? (c->face_nv == 4 ? 9 : 7) : 0;
    if (c->nq == 8) CK(dalloc(c, (void **)&c->d_cond_qp64, (size_t)ne * 8 * 28 * 8), "alloc point conductances");
    CK(dalloc(c, (void **)&c->d_vq64, (size_t)c->nq * np * ne * 8), "alloc point conductances");
    CK(dalloc(c, &c->d_vq, (size_t)c->nq * np * ne * rs), "alloc point conductances");
    CK(dalloc(c, &c->d_Yv, (size_t)ne * npe * rs), "alloc element loads");
    if (c->face_cons) {
        const int nv = c->face_nv;
        for (int pass = 0; pass < 2; ++pass) {
            const std::vector<int32_t> &faces = pass ? c->rad_faces : c->conv_faces;
            std::vector<int32_t> fnew(faces.size());
            for (size_t i = 0; i < faces.size(); ++i) fnew[i] = c->til.new_of_old[faces[i]];
            CK(upload(c, (void **)(pass ? &c->d_rf_new : &c->d_cf_new), fnew.data(), fnew.size() * 4), "upload faces");
        }
        const int64_t nf = c->n_conv + c->n_rad;
        CK(dalloc(c, (void **)&c->d_Mf64, (size_t)std::max<int64_t>(c->n_conv, 1) * nv * nv * 8), "alloc face mass");
        CK(dalloc(c, &c->d_Mf, (size_t)std::max<int64_t>(c->n_conv, 1) * nv * nv * rs), "alloc face mass");
        CK(dalloc(c, (void **)&c->d_Wf64, (size_t)std::max<int64_t>(c->n_rad, 1) * c->nfq * 8), "alloc face weights");
        CK(dalloc(c, &c->d_Wf, (size_t)std::max<int64_t>(c->n_rad, 1) * c->nfq * rs), "alloc face weights");
        CK(dalloc(c, &c->d_Yf, (size_t)std::max<int64_t>(nf, 1) * nv * rs), "alloc face loads");
        CK(dalloc(c, (void **)&c->d_Yf64, (size_t)std::max<int64_t>(nf, 1) * nv * 8), "alloc face loads");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
    }
    return FEDFEM_OK;
}

fedfem_status variant_precompute(fedfem_ctx *c)
{
    const int np = n_pairs(c->npe);
    if (c->precision == 64)
        k_var_pack<double><<<blocks_for(c->ne), kThreads, 0, c->stream>>>(
            c->ne, c->nq, np, c->d_cond_qp64, c->d_cond64, c->d_vq64, static_cast<double *>(c->d_vq));
    else
        k_var_pack<float><<<blocks_for(c->ne), kThreads, 0, c->stream>>>(c->ne, c->nq, np, c->d_cond_qp64, c->d_cond64,
                                                                         c->d_vq64, static_cast<float *>(c->d_vq));
    CK(cudaGetLastError(), "point conductances");
    const int64_t nf = c->n_conv + c->n_rad;
    if (c->face_cons && nf > 0) {
        if (c->precision == 64)
            k_var_faces<double><<<blocks_for(nf), kThreads, 0, c->stream>>>(
                c->n_conv, c->n_rad, c->face_nv, c->nfq, c->d_conv_faces, c->d_rad_faces, c->d_xyz, c->d_Mf64,
                static_cast<double *>(c->d_Mf), c->d_Wf64, static_cast<double *>(c->d_Wf));
        else
            k_var_faces<float><<<blocks_for(nf), kThreads, 0, c->stream>>>(
                c->n_conv, c->n_rad, c->face_nv, c->nfq, c->d_conv_faces, c->d_rad_faces, c->d_xyz, c->d_Mf64,
                static_cast<float *>(c->d_Mf), c->d_Wf64, static_cast<float *>(c->d_Wf));
        CK(cudaGetLastError(), "face integration data");
    }
    return FEDFEM_OK;
}

fedfem_status variant_steps(fedfem_ctx *c, int64_t n)
{
    for (int64_t k = 0; k < n; ++k) {
        cudaError_t e;
        if (c->precision == 64)
            e = var_step_dispatch<double, false>(c);
        else
            e = c->kahan ? var_step_dispatch<float, true>(c) : var_step_dispatch<float, false>(c);
        CK(e, "variant step launch");
        ++c->step;
    }
    return FEDFEM_OK;
}

fedfem_status variant_loads64(fedfem_ctx *c, const double *T_new, int64_t step, double *F_new, double *Qtot_new)
{
    const bool tab = c->n_tab > 0;
    double *Y = c->d_Y;
    if (c->npe == 8) {
        if (tab)
            k_var_elem<double, 8, true><<<blocks_for(c->ne), kThreads, 0, c->stream>>>(
                c->ne, c->nq, c->kT_qp, c->d_gconn, c->d_vq64, T_new, c->k_a(), c->k_lin, c->hk, Y);
        else
            k_var_elem<double, 8, false><<<blocks_for(c->ne), kThreads, 0, c->stream>>>(
                c->ne, c->nq, c->kT_qp, c->d_gconn, c->d_vq64, T_new, c->k_a(), c->k_lin, c->hk, Y);
    } else {
        if (tab)
            k_var_elem<double, 4, true><<<blocks_for(c->ne), kThreads, 0, c->stream>>>(
                c->ne, c->nq, c->kT_qp, c->d_gconn, c->d_vq64, T_new, c->k_a(), c->k_lin, c->hk, Y);
        else
            k_var_elem<double, 4, false><<<blocks_for(c->ne), kThreads, 0, c->stream>>>(
                c->ne, c->nq, c->kT_qp, c->d_gconn, c->d_vq64, T_new, c->k_a(), c->k_lin, c->hk, Y);
    }
    const bool faces = Qtot_new && c->face_cons;
    if (faces && c->n_conv + c->n_rad > 0)
        k_var_face<double><<<blocks_for(c->n_conv + c->n_rad), kThreads, 0, c->stream>>>(
            c->n_conv, c->n_rad, c->face_nv, c->nfq, c->d_cf_new, c->d_rf_new, c->d_Mf64, c->d_Wf64, T_new, c->h,
            c->Tinf_at(step), c->eps * 5.67e-8, c->T_amb, c->T_zero, c->d_Yf64);
    k_var_gather64<<<blocks_for(c->nn), kThreads, 0, c->stream>>>(c->nn, c->npe, c->d_n2e_ptr, c->d_n2e, Y, var_faces(c),
                                                                   c->d_Yf64, c->d_Qext64, c->qs_at(step), F_new,
                                                                   faces ? Qtot_new : nullptr);
    CK(cudaGetLastError(), "variant loads");
    return FEDFEM_OK;
}

}  // namespace fedfem
