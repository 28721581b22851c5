// Reverse-time discrete adjoint of the explicit FED-FEM step (fedfem_forward_record /
// fedfem_adjoint).  The paper has no adjoint; the recursion below is the exact derivative of
// the discrete update of Eq. 16 with the element loads of Eq. 20 (element-mean k(T), Section
// 4.2.2), the nodal c(T) of Eq. 16 and the surface loads of Eq. 4 and 7.
//
// With a_i = A_i / f_c(T_i^n) (zero on Dirichlet nodes, whose A is -0.0), mu_i = a_i lambda_i^{n+1},
// R_i = Q_i - F_i and c_e = theta_e K0_e (the stored pair conductances):
//   lambda_j^n = dL/dT_j^n + lambda_j^{n+1} (1 + d_j) + mu_j dQ_j/dT_j - G_j,
//   d_j = -a_j f_c'(T_j) / f_c(T_j) R_j,
//   G_j = sum_{e∋j} [ f_k,e (c_e mu_e)_j + (mu_e . c_e T_e) f_k'(T_j) / npe ],
// (f' = k_lin, c_lin for the linear laws; the segment slope, 0 where the end values are held,
// for tabulated factors)
//   dL/dtheta_e = -sum_n f_k,e (mu_e . c_e T_e) / theta_e  (the sum first, then the division),
//   dL/ds_e     =  sum_{i in e} w_ie sum_n mu_i^n.
// The forward run keeps checkpoints of the state every K steps; each segment is recomputed
// (bit-identically: the forward is deterministic) with the per-step state recorded, then swept
// backwards, with fixed-order (deterministic) node gathers.  After an FP64 forward run the
// sweep is FP64 throughout.  After an FP32 run (whose states carry FP32 rounding) the per-step
// element and node products, mu and the element slots are FP32, with FP32 conductances; lambda,
// sum mu and the theta gradient are carried in FP64 from step to step.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cstring>
#include <vector>

#include "ctx.h"

using namespace fedfem;

#define CK(call, where)                                          \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where);   \
    } while (0)

namespace {

constexpr double kSigma = 5.67e-8;

struct AdjPhys {
    double k_lin, c_lin, h, T_inf, eps_sigma, T_amb, T_zero;
    double k_a, c_a;  // f_k = k_a + k_lin T, f_c = c_a + c_lin T
    double qs;        // external-load multiplier of the step (time-dependent loads)
    int tab;          // 1: tabulated f_k = tk, f_c = tc instead of the linear laws
    HingeLaw<double> tk, tc;
};

__device__ __forceinline__ double adj_fc(const AdjPhys &ph, double t)
{
    return ph.tab ? hinge_value(ph.tc, t) : ph.c_a + ph.c_lin * t;
}

__device__ __forceinline__ double adj_dfc(const AdjPhys &ph, double t)
{
    return ph.tab ? hinge_slope(ph.tc, t) : ph.c_lin;
}

// f_c, f_k and f_k' in precision P (tabulated laws evaluated in FP64, then rounded)
template <typename P>
__device__ __forceinline__ P adj_fc_p(const AdjPhys &ph, P t)
{
    return ph.tab ? (P)hinge_value(ph.tc, (double)t) : (P)ph.c_a + (P)ph.c_lin * t;
}

template <typename P>
__device__ __forceinline__ P adj_dfk_p(const AdjPhys &ph, P t)
{
    return ph.tab ? (P)hinge_slope(ph.tk, (double)t) : (P)ph.k_lin;
}

int nblk(int64_t n, int bs = 256)
{
    int64_t b = (n + bs - 1) / bs;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 65535));
}

template <typename R>
__global__ void k_gather_sensors(int ns, const int32_t *sens, const R *T, const float *comp, double *out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < ns) {
        const int g = sens[s];
        out[s] = (double)T[g] - (comp ? (double)comp[g] : 0.0);
    }
}

// mu_i = a_i lambda_i, a_i = A_i / f_c(T_i) (A = -0.0 on Dirichlet nodes); musum += mu.
// a_i in precision P, the product with lambda and the sum in FP64; mu is stored in P.
template <typename R, typename P>
__device__ __forceinline__ void adj_mu_one(int64_t g, const R *Tn, const double *A, const double *lam,
                                           const AdjPhys &ph, double qs, P *mu, double *musum)
{
    const P t = (P)Tn[g];
    const double m = (double)((P)A[g] / adj_fc_p<P>(ph, t)) * __ldcg(lam + g);
    mu[g] = (P)m;
    musum[g] += qs * m;  // d Q_g / d s_e = qs w_ge
}

// N consecutive values at src into registers, with 16-byte (else 8-byte) vector loads when N
// values fill them (src aligned accordingly: the per-element rows of the arrays read here are).
template <typename V, int N>
__device__ __forceinline__ void vload(const V *src, V *dst)
{
    if constexpr (sizeof(V) == 4 && N % 4 == 0) {
        using V4 = typename std::conditional<std::is_same<V, float>::value, float4, int4>::type;
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            const V4 v = reinterpret_cast<const V4 *>(src)[i];
            dst[4 * i] = v.x;
            dst[4 * i + 1] = v.y;
            dst[4 * i + 2] = v.z;
            dst[4 * i + 3] = v.w;
        }
    } else if constexpr (N % 2 == 0) {
        using V2 = typename std::conditional<sizeof(V) == 8, double2,
                                             typename std::conditional<std::is_same<V, float>::value, float2,
                                                                       int2>::type>::type;
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const V2 v = reinterpret_cast<const V2 *>(src)[i];
            dst[2 * i] = v.x;
            dst[2 * i + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) dst[i] = src[i];
    }
}

// The same for stores.
template <typename V, int N>
__device__ __forceinline__ void vstore(V *dst, const V *src)
{
    if constexpr (sizeof(V) == 4 && N % 4 == 0) {
        using V4 = typename std::conditional<std::is_same<V, float>::value, float4, int4>::type;
#pragma unroll
        for (int i = 0; i < N / 4; ++i)
            reinterpret_cast<V4 *>(dst)[i] = V4{src[4 * i], src[4 * i + 1], src[4 * i + 2], src[4 * i + 3]};
    } else if constexpr (N % 2 == 0) {
        using V2 = typename std::conditional<sizeof(V) == 8, double2,
                                             typename std::conditional<std::is_same<V, float>::value, float2,
                                                                       int2>::type>::type;
#pragma unroll
        for (int i = 0; i < N / 2; ++i) reinterpret_cast<V2 *>(dst)[i] = V2{src[2 * i], src[2 * i + 1]};
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) dst[i] = src[i];
    }
}

// Element pass of element e: forward loads F_e = f_k (c T_e) and adjoint loads
// G_e = f_k (c mu_e) + (mu_e . c T_e) f_k'(T_j) / npe into per-element slots; theta gradient.
// Everything per element is in precision P (FP64 for an FP64 forward run; FP32 for an FP32
// one, whose states carry FP32 rounding anyway, with FP32 conductances and mu); the theta
// gradient is accumulated in FP64.
template <int NPE, typename R, typename P>
__device__ __forceinline__ void adj_elem_one(int64_t e, const int32_t *gconn, const P *cond, const R *Tn,
                                             const P *mu, const AdjPhys &ph, P *YF, P *YG, double *gtheta)
{
    constexpr int NC = NPE * (NPE - 1) / 2;
    P T[NPE], m[NPE], cT[NPE], cm[NPE];
    P sum = 0;
    int gid[NPE];
    vload<int32_t, NPE>(gconn + NPE * e, gid);
    for (int k = 0; k < NPE; ++k) {
        const int g = gid[k];
        T[k] = (P)Tn[g];
        m[k] = __ldcg(mu + g);
        sum += ph.tab ? (P)hinge_value(ph.tk, (double)T[k]) : T[k];
        cT[k] = 0;
        cm[k] = 0;
    }
    P ce[NC];
    vload<P, NC>(cond + NC * e, ce);
    int p = 0;
    for (int i = 0; i < NPE; ++i)
        for (int j = i + 1; j < NPE; ++j, ++p) {
            const P c = ce[p];
            const P gt = c * (T[i] - T[j]);
            const P gm = c * (m[i] - m[j]);
            cT[i] += gt;
            cT[j] -= gt;
            cm[i] += gm;
            cm[j] -= gm;
        }
    const P fk = ph.tab ? sum / NPE : (P)ph.k_a + (P)ph.k_lin * (sum / NPE);
    P mcT = 0;
    for (int k = 0; k < NPE; ++k) mcT += m[k] * cT[k];
    P yf[NPE], yg[NPE];
    for (int k = 0; k < NPE; ++k) {
        yf[k] = fk * cT[k];
        yg[k] = fk * cm[k] + mcT * adj_dfk_p<P>(ph, T[k]) / NPE;
    }
    vstore<P, NPE>(YF + NPE * e, yf);
    vstore<P, NPE>(YG + NPE * e, yg);
    gtheta[e] += (double)(fk * mcT);  // scaled by -1 / theta_e once, after the sweep
}

// Node pass of node g: gather F and G in fixed (ascending element) order and form lambda^n.
// With Tprev (the state one step earlier) the pass also prepares the next reverse step:
// lambda^n += dL/dT^n at the sensors (dl_next, sensor index per node), mu = A / f_c(T^(n-1))
// lambda^n written over mu (each thread touches only its node), musum += qs_prev mu.
template <typename R, typename P>
__device__ __forceinline__ void adj_node_one(int64_t g, int npe, const int32_t *n2e_ptr, const int64_t *n2e,
                                             const P *YF, const P *YG, const R *Tn, const double *lam, P *mu,
                                             const double *A, const double *Qext, const double *Ac, const double *Ar,
                                             const uint8_t *isdir, const AdjPhys &ph, double *lam_out, const R *Tprev,
                                             const int32_t *sens_idx, const double *dl_next, double qs_prev,
                                             double *musum)
{
    // eight incident elements at a time: their slot indices, then their slots, are loaded
    // together (one round trip each) and added in ascending order
    P F = 0, G = 0;
    const int q0 = n2e_ptr[g], q1 = n2e_ptr[g + 1];
    for (int qb = q0; qb < q1; qb += 8) {
        int64_t sl[8];
        P yf[8], yg[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (qb + j < q1) {
                const int64_t ek = n2e[qb + j];
                sl[j] = npe * (ek >> 3) + (ek & 7);
            }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (qb + j < q1) {
                yf[j] = __ldcg(YF + sl[j]);
                yg[j] = __ldcg(YG + sl[j]);
            }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (qb + j < q1) {
                F += yf[j];
                G += yg[j];
            }
    }
    const double lg = __ldcg(lam + g);
    double l;
    if (isdir[g]) {
        l = lg - (double)G;
    } else {
        // the factors of the recursion in P (FP32 for an FP32 forward run), accumulated in FP64
        const P t = (P)Tn[g];
        const P fc = adj_fc_p<P>(ph, t);
        const P a = (P)A[g] / fc;
        const P u = t - (P)ph.T_zero, b = (P)ph.T_amb - (P)ph.T_zero;
        const P Q = (P)ph.qs * (P)Qext[g] - (P)Ac[g] * (P)ph.h * (t - (P)ph.T_inf) -
                    (P)Ar[g] * (P)ph.eps_sigma * ((u - b) * (u + b) * (u * u + b * b));
        const P dQ = -(P)Ac[g] * (P)ph.h - (P)Ar[g] * (P)ph.eps_sigma * (P)4 * u * u * u;
        const P d = -a * (P)adj_dfc(ph, (double)t) / fc * (Q - F);
        l = lg * (1.0 + (double)d) + (double)(__ldcg(mu + g) * dQ) - (double)G;
    }
    if (Tprev) {
        if (dl_next && sens_idx[g] >= 0) l += dl_next[sens_idx[g]];
        const double m = (double)((P)A[g] / adj_fc_p<P>(ph, (P)Tprev[g])) * l;
        mu[g] = (P)m;
        musum[g] += qs_prev * m;
    }
    lam_out[g] = l;
}

template <typename R>
__global__ void k_adj_mu(int64_t nn, const R *Tn, const double *A, const double *lam, AdjPhys ph, double qs,
                         R *mu, double *musum)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x)
        adj_mu_one<R, R>(g, Tn, A, lam, ph, qs, mu, musum);
}

template <int NPE, typename R>
__global__ void k_adj_elem(int64_t ne, const int32_t *gconn, const R *cond, const R *Tn, const R *mu, AdjPhys ph,
                           R *YF, R *YG, double *gtheta)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x)
        adj_elem_one<NPE, R, R>(e, gconn, cond, Tn, mu, ph, YF, YG, gtheta);
}

template <typename R>
__global__ void k_adj_node(int64_t nn, int npe, const int32_t *n2e_ptr, const int64_t *n2e, const R *YF,
                           const R *YG, const R *Tn, const double *lam, R *mu, const double *A,
                           const double *Qext, const double *Ac, const double *Ar, const uint8_t *isdir, AdjPhys ph,
                           double *lam_out, const R *Tprev, const int32_t *sens_idx, const double *dl_next,
                           double qs_prev, double *musum)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x)
        adj_node_one<R, R>(g, npe, n2e_ptr, n2e, YF, YG, Tn, lam, mu, A, Qext, Ac, Ar, isdir, ph, lam_out, Tprev,
                           sens_idx, dl_next, qs_prev, musum);
}

// Grid-wide barrier of a cooperative launch (all blocks co-resident): a generation counter
// bumped by the last block to arrive.  Bounded: after timeout_ns (or once another block has
// raised an error) a waiting block sets ERRBIT_TIMEOUT and the barrier returns false.
__device__ bool adj_grid_barrier(unsigned int *count, unsigned int *gen, int32_t *err, long long timeout_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned int g;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(gen) : "memory");
        __threadfence();
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            atomicExch(count, 0u);
            __threadfence();
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(gen), "r"(g + 1u) : "memory");
        } else {
            unsigned long long t0;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            for (unsigned spin = 0;; ++spin) {
                unsigned int v;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(gen) : "memory");
                if (v != g) break;
                if ((spin & 15u) == 15u) {
                    unsigned long long t;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                    if (*(volatile int32_t *)err) {
                        ok = 0;
                        break;
                    }
                    if ((long long)(t - t0) > timeout_ns) {
                        atomicOr(err, ERRBIT_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// One checkpoint segment of the reverse sweep in a single cooperative launch: for s = K-1 .. 0
// the element pass and the node pass of the step from T^(n) (n = step0 + s), separated by grid
// barriers; at the segment's first reverse step the sensor injection and mu pass come first.
// The arithmetic per element and node is that of the per-pass kernels above (same order, so
// the same results); only the launches between the passes are replaced by barriers.  Values
// written by other blocks within the launch (mu, lambda, the element slots) are read through
// L2 (ld.cg), never from a possibly stale L1 line.
struct AdjSegArgs {
    int64_t nn, ne;
    int K, ns, se;
    int64_t rel0;                 // record steps before the segment's first state
    const int32_t *gconn, *n2e_ptr, *sens, *sens_idx;
    const int64_t *n2e;
    const double *A, *Qext, *Ac, *Ar, *dl;
    const void *cond;             // pair conductances in the forward precision R
    const uint8_t *isdir;
    const void *rec;              // [K][nn] recorded states of the segment
    const double *step_Tinf, *step_qs;  // per recorded step (index: record step)
    double *lam0, *lam1, *musum, *gth;
    void *mu, *YF, *YG;           // in the forward precision R
    unsigned int *bar_count, *bar_gen;
    int32_t *err;
    long long timeout_ns;
    int cur;                      // lambda buffer holding lambda at the segment's end
};

// threads per block of the one-launch-per-segment sweep (fewer blocks arrive at each grid barrier)
constexpr int kSegThreads = 256;

template <int NPE, typename R>
__global__ void __launch_bounds__(kSegThreads) k_adj_segment(AdjSegArgs a, AdjPhys ph)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const R *rec = static_cast<const R *>(a.rec);
    const R *cond = static_cast<const R *>(a.cond);
    R *mu = static_cast<R *>(a.mu), *YF = static_cast<R *>(a.YF), *YG = static_cast<R *>(a.YG);
    double *lam[2] = {a.lam0, a.lam1};
    int cur = a.cur;
    for (int s = a.K - 1; s >= 0; --s) {
        const int64_t rel = a.rel0 + s + 1;  // record steps up to the state T^{n+1}
        const int64_t ri = a.rel0 + s;       // record index of the step from T^n
        const R *Tn = rec + (size_t)s * a.nn;
        ph.T_inf = a.step_Tinf[ri];
        ph.qs = a.step_qs[ri];
        if (s == a.K - 1) {  // no earlier node pass prepared this step
            if (rel % a.se == 0)
                for (int64_t q = tid0; q < a.ns; q += stride) lam[cur][a.sens[q]] += a.dl[(rel / a.se - 1) * a.ns + q];
            if (!adj_grid_barrier(a.bar_count, a.bar_gen, a.err, a.timeout_ns)) return;
            for (int64_t g = tid0; g < a.nn; g += stride) adj_mu_one<R, R>(g, Tn, a.A, lam[cur], ph, ph.qs, mu, a.musum);
            if (!adj_grid_barrier(a.bar_count, a.bar_gen, a.err, a.timeout_ns)) return;
        }
        for (int64_t e = tid0; e < a.ne; e += stride)
            adj_elem_one<NPE, R, R>(e, a.gconn, cond, Tn, mu, ph, YF, YG, a.gth);
        if (!adj_grid_barrier(a.bar_count, a.bar_gen, a.err, a.timeout_ns)) return;
        const R *Tprev = s > 0 ? rec + (size_t)(s - 1) * a.nn : nullptr;
        const double *dl_next = (s > 0 && (rel - 1) % a.se == 0) ? a.dl + ((rel - 1) / a.se - 1) * a.ns : nullptr;
        const double qs_prev = s > 0 ? a.step_qs[ri - 1] : 0.0;
        for (int64_t g = tid0; g < a.nn; g += stride)
            adj_node_one<R, R>(g, NPE, a.n2e_ptr, a.n2e, YF, YG, Tn, lam[cur], mu, a.A, a.Qext, a.Ac, a.Ar,
                               a.isdir, ph, lam[cur ^ 1], Tprev, a.sens_idx, dl_next, qs_prev, a.musum);
        cur ^= 1;
        if (!adj_grid_barrier(a.bar_count, a.bar_gen, a.err, a.timeout_ns)) return;
    }
}

// FP32 copy of an FP64 array (the pair conductances of an FP32 run's reverse sweep)
__global__ void k_to_f32(int64_t n, const double *x, float *y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

// sens_idx[sensor node] = its index in the sensor list (the array is -1 elsewhere)
__global__ void k_sensor_index(int ns, const int32_t *sens, int32_t *sens_idx)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < ns) sens_idx[sens[s]] = s;
}

__global__ void k_adj_inject(int ns, const int32_t *sens, const double *dl, double *lam)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < ns) lam[sens[s]] += dl[s];  // sensors are distinct nodes
}

// dL/dtheta_e = -(sum over the steps) / theta_e
__global__ void k_adj_theta(int64_t ne, const double *theta, double *gth)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x)
        gth[e] = -gth[e] / theta[e];
}

// dL/ds_e = sum_k w_ek musum[node_k]
template <int NPE>
__global__ void k_adj_source(int64_t ne, const int32_t *gconn, const double *W, const double *musum, double *gs)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < NPE; ++k) s += W[NPE * e + k] * musum[gconn[NPE * e + k]];
        gs[e] = s;
    }
}

cudaError_t adj_alloc(fedfem_ctx *c, void **p, size_t bytes)
{
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) c->adj_allocs.push_back(*p);
    return e;
}

void adj_free(fedfem_ctx *c)
{
    for (void *p : c->adj_allocs) cudaFree(p);
    c->adj_allocs.clear();
    c->recorded = false;
}

size_t state_bytes_dev(fedfem_ctx *c) { return (size_t)c->nn * (c->precision == 64 ? 8 : 4); }

fedfem_status copy_state(fedfem_ctx *c, int64_t step, uint8_t *dst, bool save)
{
    const int b = (int)(step & 1);
    const size_t tb = state_bytes_dev(c);
    uint8_t *T = (uint8_t *)c->d_T[b];
    if (save) {
        CK(cudaMemcpyAsync(dst, T, tb, cudaMemcpyDeviceToDevice, c->stream), "save state");
        if (c->kahan) CK(cudaMemcpyAsync(dst + tb, c->d_comp[b], c->nn * 4, cudaMemcpyDeviceToDevice, c->stream), "save");
    } else {
        CK(cudaMemcpyAsync(T, dst, tb, cudaMemcpyDeviceToDevice, c->stream), "restore state");
        if (c->kahan) CK(cudaMemcpyAsync(c->d_comp[b], dst + tb, c->nn * 4, cudaMemcpyDeviceToDevice, c->stream), "restore");
    }
    return FEDFEM_OK;
}

// One reverse step: mu (only at the first step of a segment; later steps get it from the
// previous node pass), the element pass and the node pass.  Small blocks (64 / 128 threads)
// spread the few warps of small meshes over all SMs (32^3: 94.7 -> 90.8 ms per adjoint).
template <typename R>
void adj_step(fedfem_ctx *c, bool first, const void *Tn, const void *Tprev, const double *dl_next, double qs_prev,
              const AdjPhys &ph, const double *lam_in, double *lam_out, void *mu_, double *musum, const void *cond_,
              void *YF_, void *YG_, double *gth, const int32_t *sens_idx)
{
    const int64_t nn = c->nn, ne = c->ne;
    const int npe = c->npe;
    const R *T = static_cast<const R *>(Tn);
    const R *cond = static_cast<const R *>(cond_);
    R *mu = static_cast<R *>(mu_), *YF = static_cast<R *>(YF_), *YG = static_cast<R *>(YG_);
    if (first)
        k_adj_mu<R><<<nblk(nn, 128), 128, 0, c->stream>>>(nn, T, c->d_A, lam_in, ph, ph.qs, mu, musum);
    if (npe == 8)
        k_adj_elem<8, R><<<nblk(ne, 64), 64, 0, c->stream>>>(ne, c->d_gconn, cond, T, mu, ph, YF, YG, gth);
    else
        k_adj_elem<4, R><<<nblk(ne, 64), 64, 0, c->stream>>>(ne, c->d_gconn, cond, T, mu, ph, YF, YG, gth);
    k_adj_node<R><<<nblk(nn, 128), 128, 0, c->stream>>>(nn, npe, c->d_n2e_ptr, c->d_n2e, YF, YG, T, lam_in, mu, c->d_A,
                                                   c->d_Qext64, c->d_Ac64, c->d_Ar64, c->d_isdir, ph, lam_out,
                                                   static_cast<const R *>(Tprev), sens_idx, dl_next, qs_prev, musum);
}

}  // namespace

static fedfem_status forward_record_impl(fedfem_ctx *c, int64_t n_steps, const int32_t *sensors, int32_t n_sensors,
                                         int32_t sample_every, int32_t ckpt_every, double *trace, bool trace_on_device)
{
    if (!c) return FEDFEM_ERR_ARG;
    if (c->variant())
        return fail(c, FEDFEM_ERR_UNSUPPORTED, "the adjoint covers kT_eval = 0 and face_quadrature = 0 only");
    if (!c->has_dt || !c->has_T) return fail(c, FEDFEM_ERR_STATE, "call fedfem_set_dt and fedfem_set_T first");
    if (n_steps <= 0 || sample_every <= 0 || ckpt_every <= 0 || n_steps % sample_every || n_steps % ckpt_every ||
        ckpt_every % sample_every)
        return fail(c, FEDFEM_ERR_ARG, "n_steps must be a multiple of ckpt_every, which must be a multiple of sample_every");
    if (n_sensors <= 0 || !sensors || !trace) return fail(c, FEDFEM_ERR_ARG, "sensors and trace required");
    std::vector<int32_t> sn(n_sensors);
    std::vector<uint8_t> seen(c->nn, 0);
    for (int s = 0; s < n_sensors; ++s) {
        if (sensors[s] < 0 || sensors[s] >= c->nn) return fail(c, FEDFEM_ERR_ARG, "sensor node out of range");
        sn[s] = c->til.new_of_old[sensors[s]];
        if (seen[sn[s]]++) return fail(c, FEDFEM_ERR_ARG, "sensor nodes must be distinct");
    }
    adj_free(c);
    const int64_t n_ckpt = n_steps / ckpt_every, n_samp = n_steps / sample_every;
    c->ckpt_bytes = state_bytes_dev(c) + (c->kahan ? (size_t)c->nn * 4 : 0);
    c->ckpt_bytes = (c->ckpt_bytes + 255) & ~(size_t)255;
    double *d_trace = nullptr;
    CK(adj_alloc(c, (void **)&c->d_sensors, n_sensors * 4), "alloc sensors");
    CK(adj_alloc(c, &c->d_ckpt, (n_ckpt + 1) * c->ckpt_bytes), "alloc checkpoints");
    CK(adj_alloc(c, (void **)&d_trace, n_samp * n_sensors * 8), "alloc trace");
    CK(cudaMemcpyAsync(c->d_sensors, sn.data(), n_sensors * 4, cudaMemcpyHostToDevice, c->stream), "upload sensors");
    c->rec_step0 = c->step;
    for (int64_t k = 0; k < n_ckpt; ++k) {
        fedfem_status s = copy_state(c, c->step, (uint8_t *)c->d_ckpt + k * c->ckpt_bytes, true);
        if (s != FEDFEM_OK) return s;
        for (int32_t j = 0; j < ckpt_every / sample_every; ++j) {
            s = enqueue_steps(c, sample_every, nullptr, 0);
            if (s != FEDFEM_OK) return s;
            const int64_t samp = (c->step - c->rec_step0) / sample_every - 1;
            const int b = (int)(c->step & 1);
            if (c->precision == 64)
                k_gather_sensors<double><<<nblk(n_sensors), 256, 0, c->stream>>>(
                    n_sensors, c->d_sensors, (const double *)c->d_T[b], nullptr, d_trace + samp * n_sensors);
            else
                k_gather_sensors<float><<<nblk(n_sensors), 256, 0, c->stream>>>(
                    n_sensors, c->d_sensors, (const float *)c->d_T[b], c->kahan ? c->d_comp[b] : nullptr,
                    d_trace + samp * n_sensors);
            CK(cudaGetLastError(), "sensor gather");
        }
    }
    // the end state, restored after the reverse sweep
    fedfem_status s = copy_state(c, c->step, (uint8_t *)c->d_ckpt + n_ckpt * c->ckpt_bytes, true);
    if (s != FEDFEM_OK) return s;
    CK(cudaMemcpyAsync(trace, d_trace, n_samp * n_sensors * 8,
                       trace_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
       "copy trace");
    int32_t bits = 0;
    CK(cudaMemcpyAsync(&bits, c->d_err, 4, cudaMemcpyDeviceToHost, c->stream), "status");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    if (bits) {
        CK(cudaMemset(c->d_err, 0, 4), "clear");
        return fail(c, (bits & ERRBIT_DIVERGED) ? FEDFEM_ERR_DIVERGED : FEDFEM_ERR_TIMEOUT, "forward run failed");
    }
    c->recorded = true;
    c->rec_steps = n_steps;
    c->rec_sample_every = sample_every;
    c->rec_ckpt_every = ckpt_every;
    c->rec_n_sensors = n_sensors;
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_forward_record(fedfem_ctx *c, int64_t n_steps, const int32_t *sensors,
                                               int32_t n_sensors, int32_t sample_every, int32_t ckpt_every,
                                               double *trace)
{
    return forward_record_impl(c, n_steps, sensors, n_sensors, sample_every, ckpt_every, trace, false);
}

extern "C" fedfem_status fedfem_forward_record_device(fedfem_ctx *c, int64_t n_steps, const int32_t *sensors,
                                                      int32_t n_sensors, int32_t sample_every, int32_t ckpt_every,
                                                      double *trace_dev)
{
    return forward_record_impl(c, n_steps, sensors, n_sensors, sample_every, ckpt_every, trace_dev, true);
}

static fedfem_status adjoint_impl(fedfem_ctx *c, const double *dL_dtrace, double *dL_dkscale, double *dL_dsource,
                                  bool on_device)
{
    if (!c) return FEDFEM_ERR_ARG;
    if (!c->recorded) return fail(c, FEDFEM_ERR_STATE, "call fedfem_forward_record first");
    if (!dL_dtrace || !dL_dkscale || !dL_dsource) return fail(c, FEDFEM_ERR_ARG, "NULL array");
    const int64_t nn = c->nn, ne = c->ne;
    const int npe = c->npe;
    const int K = c->rec_ckpt_every, se = c->rec_sample_every, ns = c->rec_n_sensors;
    const int64_t n_ckpt = c->rec_steps / K, n_samp = c->rec_steps / se;
    const size_t rs = c->precision == 64 ? 8 : 4;
    std::vector<void *> tmp;
    auto talloc = [&](void **p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess) tmp.push_back(*p);
        return e;
    };
    auto release = [&]() {
        for (void *p : tmp) cudaFree(p);
        tmp.clear();
    };
    // mu, the element slots and the conductances in the forward precision (rs bytes)
    double *d_dl = nullptr, *lam[2] = {nullptr, nullptr}, *musum = nullptr, *gth = nullptr, *gs = nullptr;
    void *rec = nullptr, *mu = nullptr, *YF = nullptr, *YG = nullptr;
    const void *cond = c->d_cond64;
    const int64_t n_cond = ne * (int64_t)(npe * (npe - 1) / 2);
    cudaError_t e = cudaSuccess;
    if ((e = talloc((void **)&d_dl, n_samp * ns * 8)) != cudaSuccess || (e = talloc(&rec, (size_t)K * nn * rs)) != cudaSuccess ||
        (e = talloc((void **)&lam[0], nn * 8)) != cudaSuccess || (e = talloc((void **)&lam[1], nn * 8)) != cudaSuccess ||
        (e = talloc(&mu, nn * rs)) != cudaSuccess || (e = talloc((void **)&musum, nn * 8)) != cudaSuccess ||
        (e = talloc(&YF, ne * npe * rs)) != cudaSuccess || (e = talloc(&YG, ne * npe * rs)) != cudaSuccess ||
        (e = talloc((void **)&gth, ne * 8)) != cudaSuccess || (e = talloc((void **)&gs, ne * 8)) != cudaSuccess) {
        release();
        return cuda_fail(c, e, "adjoint buffers");
    }
    if (c->precision != 64) {
        float *c32 = nullptr;
        if ((e = talloc((void **)&c32, n_cond * 4)) != cudaSuccess) {
            release();
            return cuda_fail(c, e, "adjoint buffers");
        }
        k_to_f32<<<nblk(n_cond), 256, 0, c->stream>>>(n_cond, c->d_cond64, c32);
        cond = c32;
    }
#define CKR(call, where)                       \
    do {                                       \
        cudaError_t e_ = (call);               \
        if (e_ != cudaSuccess) {               \
            release();                         \
            return cuda_fail(c, e_, where);    \
        }                                      \
    } while (0)
    CKR(cudaMemcpyAsync(d_dl, dL_dtrace, n_samp * ns * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        c->stream),
        "copy dL/dtrace");
    CKR(cudaMemsetAsync(lam[0], 0, nn * 8, c->stream), "memset");
    CKR(cudaMemsetAsync(musum, 0, nn * 8, c->stream), "memset");
    CKR(cudaMemsetAsync(gth, 0, ne * 8, c->stream), "memset");
    // sensor index of every node (-1 elsewhere) for the injections fused into the node pass
    int32_t *sens_idx = nullptr;
    CKR(talloc((void **)&sens_idx, nn * 4), "adjoint buffers");
    CKR(cudaMemsetAsync(sens_idx, 0xFF, nn * 4, c->stream), "memset");
    k_sensor_index<<<nblk(ns), 256, 0, c->stream>>>(ns, c->d_sensors, sens_idx);
    AdjPhys ph{c->k_lin, c->c_lin, c->h,   c->T_inf, c->eps * kSigma, c->T_amb, c->T_zero, c->k_a(), c->c_a(), 1.0,
               c->n_tab > 0, c->hk,    c->hc};
    // per recorded step: convection temperature and load multiplier (schedules), and the grid
    // barrier of the one-launch-per-segment sweep
    double *step_Tinf = nullptr, *step_qs = nullptr;
    unsigned int *bar = nullptr;
    CKR(talloc((void **)&step_Tinf, c->rec_steps * 8), "adjoint buffers");
    CKR(talloc((void **)&step_qs, c->rec_steps * 8), "adjoint buffers");
    CKR(talloc((void **)&bar, 64), "adjoint buffers");
    {
        std::vector<double> ti(c->rec_steps), qs(c->rec_steps);
        for (int64_t i = 0; i < c->rec_steps; ++i) {
            ti[i] = c->Tinf_at(c->rec_step0 + i);
            qs[i] = c->qs_at(c->rec_step0 + i);
        }
        CKR(cudaMemcpyAsync(step_Tinf, ti.data(), ti.size() * 8, cudaMemcpyHostToDevice, c->stream), "upload");
        CKR(cudaMemcpyAsync(step_qs, qs.data(), qs.size() * 8, cudaMemcpyHostToDevice, c->stream), "upload");
        CKR(cudaMemsetAsync(bar, 0, 64, c->stream), "memset");
        CKR(cudaStreamSynchronize(c->stream), "synchronize");
    }
    void *seg_kernel = nullptr;
    if (npe == 8)
        seg_kernel = c->precision == 64 ? (void *)k_adj_segment<8, double> : (void *)k_adj_segment<8, float>;
    else
        seg_kernel = c->precision == 64 ? (void *)k_adj_segment<4, double> : (void *)k_adj_segment<4, float>;
    int seg_grid = 0;
    {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, seg_kernel, kSegThreads, 0) == cudaSuccess &&
            per_sm > 0) {
            const int64_t want = (std::max(nn, ne) + kSegThreads - 1) / kSegThreads;
            seg_grid = (int)std::min<int64_t>((int64_t)per_sm * c->num_sms, want);
        }
    }
    bool persistent = seg_grid > 0;
    int cur = 0;
    for (int64_t k = n_ckpt - 1; k >= 0; --k) {
        // recompute the segment from its checkpoint, recording T^n for every step
        const int64_t step_k = c->rec_step0 + k * K;
        c->step = step_k;
        fedfem_status st = copy_state(c, step_k, (uint8_t *)c->d_ckpt + k * c->ckpt_bytes, false);
        if (st == FEDFEM_OK) st = enqueue_steps(c, K, rec, nn);
        if (st != FEDFEM_OK) {
            release();
            return st;
        }
        if (persistent) {
            AdjSegArgs sa;
            sa.nn = nn;
            sa.ne = ne;
            sa.K = K;
            sa.ns = ns;
            sa.se = se;
            sa.rel0 = k * K;
            sa.gconn = c->d_gconn;
            sa.n2e_ptr = c->d_n2e_ptr;
            sa.sens = c->d_sensors;
            sa.sens_idx = sens_idx;
            sa.n2e = c->d_n2e;
            sa.cond = cond;
            sa.A = c->d_A;
            sa.Qext = c->d_Qext64;
            sa.Ac = c->d_Ac64;
            sa.Ar = c->d_Ar64;
            sa.dl = d_dl;
            sa.isdir = c->d_isdir;
            sa.rec = rec;
            sa.step_Tinf = step_Tinf;
            sa.step_qs = step_qs;
            sa.lam0 = lam[0];
            sa.lam1 = lam[1];
            sa.mu = mu;
            sa.musum = musum;
            sa.YF = YF;
            sa.YG = YG;
            sa.gth = gth;
            sa.bar_count = bar;
            sa.bar_gen = bar + 1;
            sa.err = c->d_err;
            sa.timeout_ns = (long long)(c->opt.barrier_timeout_s * 1e9);
            sa.cur = cur;
            void *params[] = {(void *)&sa, (void *)&ph};
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(seg_grid);
            cfg.blockDim = dim3(kSegThreads);
            cfg.stream = c->stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            const cudaError_t le = cudaLaunchKernelExC(&cfg, seg_kernel, params);
            if (le == cudaSuccess) {
                cur ^= (K & 1);
                continue;
            }
            // a cooperative launch that cannot run (e.g. too few resident blocks): the passes as
            // separate launches from this segment on
            (void)cudaGetLastError();
            persistent = false;
        }
        for (int s = K - 1; s >= 0; --s) {
            const int64_t rel = k * K + s + 1;  // steps after the record start of the state T^{n+1}
            const int64_t n = step_k + s;       // the step from T^n
            const bool first = s == K - 1;      // no earlier node pass prepared this step
            if (first && rel % se == 0)
                k_adj_inject<<<nblk(ns), 256, 0, c->stream>>>(ns, c->d_sensors, d_dl + (rel / se - 1) * ns, lam[cur]);
            const void *Tn = (const uint8_t *)rec + (size_t)s * nn * rs;
            ph.T_inf = c->Tinf_at(n);
            ph.qs = c->qs_at(n);
            // the node pass prepares the next reverse step (the step from T^(n-1)) of this segment
            const void *Tprev = s > 0 ? (const uint8_t *)rec + (size_t)(s - 1) * nn * rs : nullptr;
            const double *dl_next = (s > 0 && (rel - 1) % se == 0) ? d_dl + ((rel - 1) / se - 1) * ns : nullptr;
            const double qs_prev = s > 0 ? c->qs_at(n - 1) : 0.0;
            if (c->precision == 64)
                adj_step<double>(c, first, Tn, Tprev, dl_next, qs_prev, ph, lam[cur], lam[cur ^ 1], mu, musum, cond, YF, YG,
                                 gth, sens_idx);
            else
                adj_step<float>(c, first, Tn, Tprev, dl_next, qs_prev, ph, lam[cur], lam[cur ^ 1], mu, musum, cond, YF, YG,
                                gth, sens_idx);
            cur ^= 1;
        }
        CKR(cudaGetLastError(), "adjoint sweep");
    }
    k_adj_theta<<<nblk(ne), 256, 0, c->stream>>>(ne, c->d_kscale, gth);
    if (npe == 8)
        k_adj_source<8><<<nblk(ne), 256, 0, c->stream>>>(ne, c->d_gconn, c->d_W, musum, gs);
    else
        k_adj_source<4><<<nblk(ne), 256, 0, c->stream>>>(ne, c->d_gconn, c->d_W, musum, gs);
    CKR(cudaGetLastError(), "source gradient");
    const cudaMemcpyKind out_kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CKR(cudaMemcpyAsync(dL_dkscale, gth, ne * 8, out_kind, c->stream), "copy dL/dkscale");
    CKR(cudaMemcpyAsync(dL_dsource, gs, ne * 8, out_kind, c->stream), "copy dL/dsource");
    // leave the context in the state at the end of the recorded run
    c->step = c->rec_step0 + c->rec_steps;
    fedfem_status st = copy_state(c, c->step, (uint8_t *)c->d_ckpt + n_ckpt * c->ckpt_bytes, false);
    int32_t bits = 0;
    CKR(cudaMemcpyAsync(&bits, c->d_err, 4, cudaMemcpyDeviceToHost, c->stream), "status");
    CKR(cudaStreamSynchronize(c->stream), "synchronize");
    release();
    if (st != FEDFEM_OK) return st;
    if (bits) {
        cudaMemset(c->d_err, 0, 4);
        return fail(c, (bits & ERRBIT_DIVERGED) ? FEDFEM_ERR_DIVERGED : FEDFEM_ERR_TIMEOUT, "recomputation failed");
    }
    return FEDFEM_OK;
#undef CKR
}

extern "C" fedfem_status fedfem_adjoint(fedfem_ctx *c, const double *dL_dtrace, double *dL_dkscale, double *dL_dsource)
{
    return adjoint_impl(c, dL_dtrace, dL_dkscale, dL_dsource, false);
}

extern "C" fedfem_status fedfem_adjoint_device(fedfem_ctx *c, const double *dL_dtrace_dev, double *dL_dkscale_dev,
                                               double *dL_dsource_dev)
{
    return adjoint_impl(c, dL_dtrace_dev, dL_dkscale_dev, dL_dsource_dev, true);
}
