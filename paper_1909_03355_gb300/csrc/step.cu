// Persistent FED-FEM time-step kernel for sm_103a: the time-stepping stage of Fig. 1 (iii).
//
// One cooperative launch advances the mesh by `nsteps` explicit steps.  Each CTA owns a fixed
// contiguous run of element tiles.  Per step and tile:
//   load     T^n of the tile's nodes into shared memory; for halo (shared) nodes T^n is
//            finished here from T^{n-1} and the fixed-order sum of last step's halo partials
//            (the owner tile writes it back), so one grid barrier per step suffices;
//   elements the element stream (pair conductances + tile-local node ids) arrives by TMA bulk
//            copies (cp.async.bulk) through a ring of shared-memory stages; each thread forms
//            F_e = f_k,e sum_j c_ij (T_i - T_j) for one element (Eq. 20 with the element-mean
//            conductivity law of Section 4.2.2; theta_e is folded into c_ij) and the CTA adds
//            the element loads into shared-memory accumulators colour by colour, so the
//            per-node summation order is fixed (deterministic);
//   surface  convection and radiation loads of the tile's owned boundary nodes (Eq. 4, 7);
//   update   T^{n+1} = T^n + A / f_c(T^n) (Q - F) for interior nodes (Eq. 16), with a Kahan
//            compensated FP32 accumulator or in FP64; A = dt / C0 is FP64 and 0 on Dirichlet
//            nodes, which therefore stay fixed (Fig. 1 (iii) 2.3);
//   halo     write the tile's partial loads of its shared nodes.
// Then a grid barrier with a deadline.  Every device wait is bounded: on timeout the kernel
// sets an error bit, drains its own copies in flight and returns.
#include <cuda_runtime.h>

#include "fedfem_internal.h"

namespace fedfem {

// ------------------------------------------------------------------------------------------
// PTX helpers (TMA bulk copies, mbarriers, timers)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait on an mbarrier phase; false after `timeout_ns`.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long timeout_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned spin = 1;; ++spin) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((spin & 63u) == 0 && (long long)(global_ns() - t0) > timeout_ns) return false;
    }
}

__device__ __forceinline__ void tma_bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

template <typename R>
__device__ __forceinline__ R ld_cg(const R *p)
{
    return __ldcg(p);
}

// Grid-wide barrier on a monotonically increasing counter with a deadline.  Returns false if
// the deadline passed or another CTA raised an error (every CTA then leaves the kernel).
__device__ bool grid_sync(unsigned int *bar, unsigned int target, int32_t *err, long long timeout_ns,
                          bool withhold)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        if (!withhold) atomicAdd(bar, 1u);
        const unsigned long long t0 = global_ns();
        for (unsigned spin = 0;; ++spin) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            if (*(volatile int32_t *)err) {
                ok = 0;
                break;
            }
            if ((spin & 31u) == 31u && (long long)(global_ns() - t0) > timeout_ns) {
                atomicOr(err, ERRBIT_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(40);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------------------------------------------
// element stream layout
// ------------------------------------------------------------------------------------------
template <typename R, int NPE>
struct Layout;

template <>
struct Layout<float, 8> {  // 28 conductances as 7 x float4, ids as 8 x u16
    static constexpr int NC = 28, VW = 4, NV = 7;
    using V = float4;
    using I = uint4;
};
template <>
struct Layout<float, 4> {  // 6 conductances as 3 x float2, ids as 4 x u16
    static constexpr int NC = 6, VW = 2, NV = 3;
    using V = float2;
    using I = uint2;
};
template <>
struct Layout<double, 8> {
    static constexpr int NC = 28, VW = 2, NV = 14;
    using V = double2;
    using I = uint4;
};
template <>
struct Layout<double, 4> {
    static constexpr int NC = 6, VW = 2, NV = 3;
    using V = double2;
    using I = uint2;
};

template <typename V, typename R>
__device__ __forceinline__ void unpack(const V &v, R *c);
template <>
__device__ __forceinline__ void unpack<float4, float>(const float4 &v, float *c)
{
    c[0] = v.x;
    c[1] = v.y;
    c[2] = v.z;
    c[3] = v.w;
}
template <>
__device__ __forceinline__ void unpack<float2, float>(const float2 &v, float *c)
{
    c[0] = v.x;
    c[1] = v.y;
}
template <>
__device__ __forceinline__ void unpack<double2, double>(const double2 &v, double *c)
{
    c[0] = v.x;
    c[1] = v.y;
}

__device__ __forceinline__ void unpack_ids(const uint4 &v, int *id)
{
    id[0] = v.x & 0xFFFF;
    id[1] = v.x >> 16;
    id[2] = v.y & 0xFFFF;
    id[3] = v.y >> 16;
    id[4] = v.z & 0xFFFF;
    id[5] = v.z >> 16;
    id[6] = v.w & 0xFFFF;
    id[7] = v.w >> 16;
}
__device__ __forceinline__ void unpack_ids(const uint2 &v, int *id)
{
    id[0] = v.x & 0xFFFF;
    id[1] = v.x >> 16;
    id[2] = v.y & 0xFFFF;
    id[3] = v.y >> 16;
}

int chunk_bytes_for(int precision, int npe, int CH)
{
    const int rs = precision == 64 ? 8 : 4;
    return CH * (n_pairs(npe) * rs + npe * 2);
}

// Element conduction loads of the element in lane `lane` of a staged chunk (Eq. 20):
// F_i = f_k,e sum_{j != i} c_ij (T_i - T_j), f_k,e = 1 + k_lin mean_i T_i.
template <typename R, int NPE>
__device__ __forceinline__ void element_loads(const uint8_t *blk, int CH, int lane, const R *Ts, R k_lin,
                                              R *F, int *id)
{
    using L = Layout<R, NPE>;
    const typename L::V *cv = reinterpret_cast<const typename L::V *>(blk);
    const typename L::I *iv = reinterpret_cast<const typename L::I *>(blk + (size_t)L::NV * CH * sizeof(typename L::V));
    unpack_ids(iv[lane], id);
    R T[NPE];
    R sum = 0;
#pragma unroll
    for (int k = 0; k < NPE; ++k) {
        T[k] = Ts[id[k]];
        sum += T[k];
        F[k] = 0;
    }
    R c[L::NC];
#pragma unroll
    for (int v = 0; v < L::NV; ++v) unpack(cv[v * CH + lane], c + v * L::VW);
    int p = 0;
#pragma unroll
    for (int i = 0; i < NPE; ++i)
#pragma unroll
        for (int j = i + 1; j < NPE; ++j) {
            const R g = c[p++] * (T[i] - T[j]);
            F[i] += g;
            F[j] -= g;
        }
    const R fk = (R)1 + k_lin * (sum * ((R)1 / (R)NPE));
#pragma unroll
    for (int k = 0; k < NPE; ++k) F[k] *= fk;
}

// Explicit nodal update (Eq. 16): T' = T + A / f_c(T) (Q - F).
template <typename R, bool KAHAN>
__device__ __forceinline__ R node_update(R T, float comp, double A, R Q, R F, const StepArgs &a, float &comp_out,
                                         int32_t *err)
{
    R Tn;
    if constexpr (KAHAN) {
        const float fc = 1.0f + (float)a.c_lin * T;
        const float r = (float)Q - (float)F;
        const float inc = (float)(A * (double)(r / fc));
        const float y = inc - comp;
        const float t = (float)T + y;
        comp_out = (t - (float)T) - y;
        Tn = t;
    } else if constexpr (sizeof(R) == 4) {
        const float fc = 1.0f + (float)a.c_lin * T;
        Tn = T + (float)(A * (double)((Q - F) / fc));
        comp_out = 0.0f;
    } else {
        const double fc = 1.0 + a.c_lin * (double)T;
        Tn = T + A / fc * ((double)Q - (double)F);
        comp_out = 0.0f;
    }
    if (!(fabs((double)Tn) <= a.T_guard)) atomicOr(err, ERRBIT_DIVERGED);
    return Tn;
}

// Convection + radiation outflow of a boundary node (Eq. 4 and Eq. 7 lumped to the node);
// the quartic difference is evaluated as (a-b)(a+b)(a^2+b^2).
template <typename R>
__device__ __forceinline__ R surface_outflow(R T, R Ac, R Ar, const StepArgs &a)
{
    const R u = T - (R)a.T_zero, b = (R)a.T_amb - (R)a.T_zero;
    const R rad = (R)a.eps_sigma * ((u - b) * (u + b) * (u * u + b * b));
    return Ac * (R)a.h * (T - (R)a.T_inf) + Ar * rad;
}

template <typename R, int NPE, bool KAHAN, int SCATTER>
__global__ void __launch_bounds__(512) fed_step_kernel(const StepArgs a, int max_local)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const int CH = blockDim.x;
    const int tid = threadIdx.x;
    const int S = a.stages;
    uint8_t *ring = smem;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + (size_t)S * a.chunk_bytes);
    R *Ts = reinterpret_cast<R *>(smem + (size_t)S * a.chunk_bytes + 64);
    R *Fs = Ts + ((max_local + 3) & ~3);

    const R *Qext = reinterpret_cast<const R *>(a.Qext);
    const R *Ac = reinterpret_cast<const R *>(a.Ac);
    const R *Ar = reinterpret_cast<const R *>(a.Ar);

    const int t0 = blockIdx.x * a.tiles_per_cta;
    const int t1 = min(t0 + a.tiles_per_cta, a.n_tiles);
    const int cb = t0 < t1 ? a.tiles[t0].chunk_begin : 0;
    const int nch = t0 < t1 ? a.tiles[t1 - 1].chunk_begin + a.tiles[t1 - 1].n_chunks - cb : 0;
    const long long total = (long long)nch * a.nsteps;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&mbar[s], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    long long issued = 0;  // meaningful in thread 0 only
    if (tid == 0) {
        for (; issued < S && issued < total; ++issued) {
            const int slot = (int)issued;
            const int ch = cb + (int)(issued % nch);
            mbar_arrive_expect_tx(&mbar[slot], (uint32_t)a.chunk_bytes);
            tma_bulk_g2s(ring + (size_t)slot * a.chunk_bytes, a.chunks + (size_t)ch * a.chunk_bytes,
                         (uint32_t)a.chunk_bytes, &mbar[slot]);
        }
    }

    long long kc = 0;  // chunks consumed
    bool ok = true;
    unsigned int bar_target = 0;
    for (int s = 0; s < a.nsteps && ok; ++s) {
        const long long n = a.n0 + s;
        const int cur = (int)(n & 1), nxt = cur ^ 1;
        R *Tc = reinterpret_cast<R *>(a.T[cur]);
        R *Tn = reinterpret_cast<R *>(a.T[nxt]);
        for (int t = t0; t < t1 && ok; ++t) {
            const TileInfo ti = a.tiles[t];
            // ---- load T^n
            for (int l = tid; l < ti.n_owned; l += CH) Ts[l] = ld_cg(Tc + ti.node_begin + l);
            __syncthreads();
            for (int q = tid; q < ti.sh_count; q += CH) {
                const int4 sh = a.sh[ti.sh_begin + q];
                R v;
                if (s == 0) {
                    v = ld_cg(Tc + sh.y);
                } else {
                    const int q0 = a.sptr[sh.z], q1 = a.sptr[sh.z + 1];
                    const R *part = reinterpret_cast<const R *>(a.part[nxt]);
                    R F = 0;
                    for (int qq = q0; qq < q1; ++qq) F += ld_cg(part + qq);
                    const float cp = KAHAN ? ld_cg(a.comp[nxt] + sh.y) : 0.0f;
                    float cn;
                    v = node_update<R, KAHAN>(ld_cg(Tn + sh.y), cp, a.A[sh.y], Qext[sh.y], F, a, cn, a.err);
                    if (sh.w == q0) {
                        Tc[sh.y] = v;
                        if (KAHAN) a.comp[cur][sh.y] = cn;
                    }
                }
                Ts[sh.x] = v;
            }
            for (int l = tid; l < ti.n_local; l += CH) Fs[l] = (R)0;
            __syncthreads();
            if (a.rec) {
                R *rec = reinterpret_cast<R *>(a.rec) + (size_t)s * a.rec_stride;
                for (int l = tid; l < ti.n_owned; l += CH) rec[ti.node_begin + l] = Ts[l];
            }
            // ---- element loads, accumulated colour by colour
            for (int c = 0; c < ti.n_chunks; ++c, ++kc) {
                const int slot = (int)(kc % S);
                const uint32_t par = (uint32_t)((kc / S) & 1);
                const int bad = mbar_wait(&mbar[slot], par, a.timeout_ns) ? 0 : 1;
                if (__syncthreads_or(bad)) {
                    if (tid == 0) atomicOr(a.err, ERRBIT_TIMEOUT);
                    ok = false;
                    break;
                }
                const uint8_t *blk = ring + (size_t)slot * a.chunk_bytes;
                const int chunk = ti.chunk_begin + c;
                const int col = a.elem_col[(size_t)chunk * CH + tid];
                R F[NPE];
                int id[NPE];
                element_loads<R, NPE>(blk, CH, tid, Ts, (R)a.k_lin, F, id);
                if (SCATTER == FEDFEM_SCATTER_ATOMIC) {
                    if (col != 0xFF)
#pragma unroll
                        for (int k = 0; k < NPE; ++k) atomicAdd(&Fs[id[k]], F[k]);
                    __syncthreads();
                } else {
                    const int c_lo = a.chunk_col[2 * chunk], c_hi = a.chunk_col[2 * chunk + 1];
                    for (int cc = c_lo; cc <= c_hi; ++cc) {
                        if (col == cc)
#pragma unroll
                            for (int k = 0; k < NPE; ++k) Fs[id[k]] += F[k];
                        __syncthreads();
                    }
                }
                // every thread is done with this stage: refill it
                if (tid == 0 && issued < total) {
                    const int slot2 = (int)(issued % S);
                    const int ch = cb + (int)(issued % nch);
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&mbar[slot2], (uint32_t)a.chunk_bytes);
                    tma_bulk_g2s(ring + (size_t)slot2 * a.chunk_bytes, a.chunks + (size_t)ch * a.chunk_bytes,
                                 (uint32_t)a.chunk_bytes, &mbar[slot2]);
                    ++issued;
                }
            }
            if (!ok) break;
            // ---- surface loads of owned boundary nodes
            for (int q = tid; q < ti.bnd_count; q += CH) {
                const int2 b = a.bnd[ti.bnd_begin + q];
                Fs[b.x] += surface_outflow<R>(Ts[b.x], Ac[b.y], Ar[b.y], a);
            }
            __syncthreads();
            // ---- update interior nodes
            for (int l = tid; l < ti.n_interior; l += CH) {
                const int g = ti.node_begin + l;
                const float cp = KAHAN ? ld_cg(a.comp[cur] + g) : 0.0f;
                float cn;
                const R v = node_update<R, KAHAN>(Ts[l], cp, a.A[g], Qext[g], Fs[l], a, cn, a.err);
                Tn[g] = v;
                if (KAHAN) a.comp[nxt][g] = cn;
            }
            // ---- halo partials
            R *part = reinterpret_cast<R *>(a.part[cur]);
            for (int q = tid; q < ti.sh_count; q += CH) {
                const int4 sh = a.sh[ti.sh_begin + q];
                part[sh.w] = Fs[sh.x];
            }
            __syncthreads();
        }
        if (!ok) break;
        bar_target += gridDim.x;
        const bool withhold = s == 0 && a.withhold > 0 && (int)blockIdx.x == a.withhold - 1;
        if (!grid_sync(a.barrier, bar_target, a.err, a.timeout_ns, withhold)) ok = false;
    }

    if (ok) {
        // finish the owned halo nodes at the final step
        const long long n = a.n0 + a.nsteps;
        const int cur = (int)(n & 1), prv = cur ^ 1;
        R *Tc = reinterpret_cast<R *>(a.T[cur]);
        const R *Tp = reinterpret_cast<const R *>(a.T[prv]);
        const R *part = reinterpret_cast<const R *>(a.part[prv]);
        for (int t = t0; t < t1; ++t) {
            const TileInfo ti = a.tiles[t];
            for (int q = tid; q < ti.sh_count; q += CH) {
                const int4 sh = a.sh[ti.sh_begin + q];
                if (sh.x >= ti.n_owned) continue;
                const int q0 = a.sptr[sh.z], q1 = a.sptr[sh.z + 1];
                R F = 0;
                for (int qq = q0; qq < q1; ++qq) F += ld_cg(part + qq);
                const float cp = KAHAN ? ld_cg(a.comp[prv] + sh.y) : 0.0f;
                float cn;
                const R v = node_update<R, KAHAN>(ld_cg(Tp + sh.y), cp, a.A[sh.y], Qext[sh.y], F, a, cn, a.err);
                Tc[sh.y] = v;
                if (KAHAN) a.comp[cur][sh.y] = cn;
            }
        }
    } else if (tid == 0) {
        // drain this CTA's copies in flight before leaving (bounded)
        for (long long k = kc; k < issued; ++k) mbar_wait(&mbar[k % S], (uint32_t)((k / S) & 1), a.timeout_ns);
    }
}

size_t step_smem_bytes(int precision, int npe, int block, int stages, int max_local)
{
    const size_t rs = precision == 64 ? 8 : 4;
    const size_t nodes = (size_t)((max_local + 3) & ~3) * rs;
    return (size_t)stages * chunk_bytes_for(precision, npe, block) + 64 + 2 * nodes;
}

template <typename R, int NPE, bool KAHAN, int SCATTER>
static void *kernel_ptr()
{
    return (void *)fed_step_kernel<R, NPE, KAHAN, SCATTER>;
}

static void *select_kernel(int precision, int kahan, int npe, int scatter)
{
#define FEDFEM_SEL(R, N, K)                                                                        \
    return scatter == FEDFEM_SCATTER_ATOMIC ? kernel_ptr<R, N, K, FEDFEM_SCATTER_ATOMIC>()         \
                                            : kernel_ptr<R, N, K, FEDFEM_SCATTER_COLOR>()
    if (precision == 64) {
        if (npe == 8) FEDFEM_SEL(double, 8, false);
        FEDFEM_SEL(double, 4, false);
    }
    if (kahan) {
        if (npe == 8) FEDFEM_SEL(float, 8, true);
        FEDFEM_SEL(float, 4, true);
    }
    if (npe == 8) FEDFEM_SEL(float, 8, false);
    FEDFEM_SEL(float, 4, false);
#undef FEDFEM_SEL
}

int step_max_blocks_per_sm(int precision, int kahan, int npe, int block, size_t smem)
{
    void *k = select_kernel(precision, kahan, npe, FEDFEM_SCATTER_COLOR);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_step(const StepArgs &a, int precision, int kahan, int npe, int grid, int block, size_t smem,
                        cudaStream_t st)
{
    void *k = select_kernel(precision, kahan, npe, a.scatter);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int max_local = 0;
    // max_local is recovered from the shared-memory size by the caller's plan
    const size_t rs = precision == 64 ? 8 : 4;
    max_local = (int)((smem - (size_t)a.stages * a.chunk_bytes - 64) / (2 * rs));
    StepArgs args = a;
    void *params[] = {(void *)&args, (void *)&max_local};
    return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(block), params, smem, st);
}

}  // namespace fedfem
