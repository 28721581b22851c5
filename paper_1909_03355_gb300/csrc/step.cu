// Persistent FED-FEM time-step kernel for sm_103a: the time-stepping stage of Fig. 1 (iii).
//
// One cooperative launch advances the mesh by `nsteps` explicit steps.  Each CTA owns a fixed
// contiguous run of element tiles.  Per step and tile:
//   load     T^n of the tile's interior nodes stays in shared memory from the CTA's own update
//            of the previous step (a TMA bulk copy, cp.async.bulk, brings the owned range at a
//            launch's first step or when a CTA takes several tiles); the tile waits until the
//            tiles it shares nodes with have finished the previous step (per-tile progress
//            counters, no grid barrier), then finishes T^n of its halo (shared) nodes from
//            T^{n-1} and the fixed-order sum of last step's halo partials (the owner tile writes
//            it back);
//   elements the element stream (pair conductances, tile-local node ids, colours) arrives by
//            TMA bulk copies through a ring of shared-memory stages; each thread forms
//            F_e = f_k,e sum_j c_ij (T_i - T_j) for one element (Eq. 20 with the element-mean
//            conductivity law of Section 4.2.2; theta_e is folded into c_ij) and the CTA adds
//            the element loads into shared-memory accumulators colour by colour, so the
//            per-node summation order is fixed (deterministic);
//   surface  convection and radiation loads of the tile's owned boundary nodes (Eq. 4, 7);
//   halo     write the tile's partial loads of its shared nodes and publish the step;
//   update   T^{n+1} = T^n + A / f_c(T^n) (Q - F) for interior nodes (Eq. 16), with a Kahan
//            compensated FP32 accumulator or in FP64; A = dt / C0 is FP64 and -0.0 on Dirichlet
//            nodes, which move only by the change of their prescribed value (Fig. 1 (iii) 2.3).
// Every device wait is bounded: on timeout the kernel sets an error bit, drains its own copies
// in flight and returns.
//
// Element chunk layout (CH elements, chunk_bytes = CH (NC rs + 2 npe + 1) + 16):
//   [NV][CH] vectors of conductances | [CH] id vectors (npe x u16) | [CH] u8 colours |
//   16-byte header {u8 first colour, u8 last colour, ...}
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "fedfem_internal.h"
#include "update.cuh"

namespace fedfem {

constexpr int MBAR_BYTES = 1536;  // 2 x 63 ring barriers, the node barrier, 63 slot tags

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

// Bounded wait that also gives up (without reporting a timeout) once any part of the grid has
// raised an error; the error word is polled only while the wait is still pending.
// Returns true when the phase completed.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity, long long timeout_ns,
                                                   int32_t *err)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned spin = 1;; ++spin) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((spin & 63u) == 0) {
            if (*(volatile int32_t *)err) return false;
            if ((long long)(global_ns() - t0) > timeout_ns) {
                atomicOr(err, ERRBIT_TIMEOUT);
                return false;
            }
        }
    }
}

// Wait until stage `slot` holds chunk k: the parity test alone can match the phase of the
// chunk two generations back when this warp runs ahead of the ring, so the slot's tag (written
// by the producer before it arms the barrier) must also name chunk k.
__device__ __forceinline__ bool wait_chunk(uint64_t *bar, volatile int *tag, int k, uint32_t parity,
                                           long long timeout_ns, int32_t *err)
{
    if (mbar_try_wait(bar, parity) && *tag == k) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned spin = 1;; ++spin) {
        if (mbar_try_wait(bar, parity) && *tag == k) return true;
        if ((spin & 63u) == 0) {
            if (*(volatile int32_t *)err) return false;
            if ((long long)(global_ns() - t0) > timeout_ns) {
                atomicOr(err, ERRBIT_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                             uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void l2_prefetch_bulk(const void *src, uint32_t bytes, uint64_t policy)
{
    asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(src), "r"(bytes), "l"(policy)
                 : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_normal()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
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

// Barrier among the NC consumer threads of the CTA (named barrier 1; the producer warp of the
// element ring never takes part).
__device__ __forceinline__ void csync(int nc)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nc) : "memory");
}

__device__ __forceinline__ int csync_or(int nc, int pred)
{
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 p, %2, 0;\n\t"
        "bar.red.or.pred q, 1, %1, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(nc), "r"(pred)
        : "memory");
    return r;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Neighbour synchronisation (in place of a grid barrier).  A tile publishes how many steps it
// has completed, counted from the launch's progress base (the counters only grow from launch to
// launch, so they need no reset between launches); before step s it waits until every tile it
// shares a node with has completed step s - 1.  Neighbours therefore never drift apart by more than one step, which
// is what the step-parity double buffers of T, the compensation and the halo partials allow.
// Entered by the NC consumer threads; thread 0 does the memory operations.
__device__ __forceinline__ void tile_publish(unsigned int *done, int t, unsigned int steps, bool withhold, int nc)
{
    csync(nc);  // every consumer's halo writes precede the release
    if (threadIdx.x == 0) {
        __threadfence();
        if (!withhold) asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(done + t), "r"(steps) : "memory");
    }
}

// Wait (with a deadline) until all neighbours of tile t have completed `steps` steps; the lanes
// of warp 0 poll the neighbours' counters in parallel.  Returns false if the deadline passed or
// another CTA raised an error (every CTA then leaves).
__device__ bool tile_wait(const unsigned int *done, const int32_t *nbr_ptr, const int32_t *nbr, int t,
                          unsigned int steps, int32_t *err, long long timeout_ns, int nc, int *s_ok)
{
    fence_proxy_async_global();  // order this thread's global writes before later TMA reads
    csync(nc);
    if (threadIdx.x < 32) {
        int ok = 1;
        const unsigned long long t0 = global_ns();
        unsigned spin = 0;
        const int q1 = nbr_ptr[t + 1];
        for (int q = nbr_ptr[t] + (int)threadIdx.x; q < q1 && ok; q += 32) {
            const unsigned int *p = done + nbr[q];
            for (;; ++spin) {
                unsigned int v;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
                if (v >= steps) break;
                if ((spin & 15u) == 15u) {
                    if (*(volatile int32_t *)err) {
                        ok = 0;
                        break;
                    }
                    if ((long long)(global_ns() - t0) > timeout_ns) {
                        atomicOr(err, ERRBIT_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(32);
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        __threadfence();
        fence_proxy_async_global();
        if (threadIdx.x == 0) *s_ok = ok;
    }
    csync(nc);
    return *s_ok != 0;
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
    return CH * (n_pairs(npe) * rs + npe * 2 + 1) + 16;
}

int chunk_colour_offset(int precision, int npe, int CH)
{
    const int rs = precision == 64 ? 8 : 4;
    return CH * (n_pairs(npe) * rs + npe * 2);
}

int chunk_header_offset(int precision, int npe, int CH) { return chunk_bytes_for(precision, npe, CH) - 16; }

// Four consecutive node values (16-byte aligned for float, 32-byte for double).
template <typename R>
struct Vec4 {
    R v[4];
};
template <typename R>
__device__ __forceinline__ Vec4<R> load4(const R *p);
template <>
__device__ __forceinline__ Vec4<float> load4<float>(const float *p)
{
    const float4 x = __ldcg(reinterpret_cast<const float4 *>(p));
    return Vec4<float>{{x.x, x.y, x.z, x.w}};
}
template <>
__device__ __forceinline__ Vec4<double> load4<double>(const double *p)
{
    const double2 x = __ldcg(reinterpret_cast<const double2 *>(p));
    const double2 y = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    return Vec4<double>{{x.x, x.y, y.x, y.y}};
}
__device__ __forceinline__ void load4d(const double *p, double *o)
{
    const double2 x = __ldcg(reinterpret_cast<const double2 *>(p));
    const double2 y = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    o[0] = x.x, o[1] = x.y, o[2] = y.x, o[3] = y.y;
}
template <typename R>
__device__ __forceinline__ void store4(R *p, const Vec4<R> &v);
template <>
__device__ __forceinline__ void store4<float>(float *p, const Vec4<float> &v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
}
template <>
__device__ __forceinline__ void store4<double>(double *p, const Vec4<double> &v)
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(v.v[0], v.v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v.v[2], v.v[3]);
}

// Element conduction loads of the element in lane `lane` of a staged chunk (Eq. 20):
// F_i = f_k,e sum_{j != i} c_ij (T_i - T_j), f_k,e = k_a + k_lin mean_i T_i, or with a table
// (TAB) the mean of the tabulated nodal factors (Section 4.2.2).
template <typename R, int NPE, bool TAB, int NH = kHinges>
__device__ __forceinline__ void element_loads(const uint8_t *blk, int CH, int lane, const R *Ts, R k_a, R k_lin,
                                              const HingeLaw<R> &tk, R *F, int *id)
{
    using L = Layout<R, NPE>;
    const typename L::V *cv = reinterpret_cast<const typename L::V *>(blk);
    const typename L::I *iv = reinterpret_cast<const typename L::I *>(blk + (size_t)L::NV * CH * sizeof(typename L::V));
    unpack_ids(iv[lane], id);
    R c[L::NC];
#pragma unroll
    for (int v = 0; v < L::NV; ++v) unpack(cv[v * CH + lane], c + v * L::VW);
    R T[NPE];
    R sum = 0;
#pragma unroll
    for (int k = 0; k < NPE; ++k) {
        T[k] = Ts[id[k]];
        if (!TAB) sum += T[k];
        F[k] = 0;
    }
    int p = 0;
#pragma unroll
    for (int i = 0; i < NPE; ++i)
#pragma unroll
        for (int j = i + 1; j < NPE; ++j) {
            const R g = c[p++] * (T[i] - T[j]);
            F[i] += g;
            F[j] -= g;
        }
    if (TAB) {  // after the pair loop, when the conductances are no longer live
#pragma unroll
        for (int k = 0; k < NPE; ++k) sum += hinge_value<NH>(tk, T[k]);
    }
    const R fk = TAB ? sum * ((R)1 / (R)NPE) : k_a + k_lin * (sum * ((R)1 / (R)NPE));
#pragma unroll
    for (int k = 0; k < NPE; ++k) F[k] *= fk;
}

// Time-dependent loads of global step n: the load multiplier of steps n and n - 1 (the halo
// nodes are finished for step n - 1), the convection ambient temperature of step n and the
// changes d(n + 1) - d(n), d(n) - d(n - 1) of the prescribed-temperature offset d (formed in
// FP64, so the Dirichlet values follow d up to the rounding of the working precision).
template <typename R>
__device__ __forceinline__ void apply_schedule(Phys<R> &ph, const StepArgs &a, long long n)
{
    if (a.sched_len <= 0) return;
    const long long L = a.sched_len - 1;
    const long long i = n < L ? n : L;
    const long long ip = n - 1 < 0 ? 0 : (n - 1 < L ? n - 1 : L);
    const long long in = n + 1 < L ? n + 1 : L;
    if (a.sched_q) {
        ph.qs = (R)a.sched_q[i];
        ph.qs_prev = (R)a.sched_q[ip];
    }
    if (a.sched_Tinf) ph.T_inf = (R)a.sched_Tinf[i];
    if (a.sched_Tdir) {
        ph.dD = (R)(a.sched_Tdir[in] - a.sched_Tdir[i]);
        ph.dD_prev = (R)(a.sched_Tdir[i] - a.sched_Tdir[ip]);
    }
}

template <typename R>
__device__ __forceinline__ ACoef<R> load_A(const StepArgs &a, int g);
// A of the four nodes g .. g + 3 (g a multiple of 4: 16-byte aligned vector loads)
template <typename R>
__device__ __forceinline__ void load_A4(const StepArgs &a, int g, ACoef<R> *out);
template <>
__device__ __forceinline__ void load_A4<float>(const StepArgs &a, int g, ACoef<float> *out)
{
    const float4 x = __ldg(reinterpret_cast<const float4 *>(a.A2 + g));
    const float4 y = __ldg(reinterpret_cast<const float4 *>(a.A2 + g) + 1);
    out[0].v = make_float2(x.x, x.y);
    out[1].v = make_float2(x.z, x.w);
    out[2].v = make_float2(y.x, y.y);
    out[3].v = make_float2(y.z, y.w);
}
template <>
__device__ __forceinline__ void load_A4<double>(const StepArgs &a, int g, ACoef<double> *out)
{
    const double2 x = __ldg(reinterpret_cast<const double2 *>(a.A + g));
    const double2 y = __ldg(reinterpret_cast<const double2 *>(a.A + g) + 1);
    out[0].v = x.x;
    out[1].v = x.y;
    out[2].v = y.x;
    out[3].v = y.y;
}
template <>
__device__ __forceinline__ ACoef<float> load_A<float>(const StepArgs &a, int g)
{
    return ACoef<float>{__ldg(a.A2 + g)};
}
template <>
__device__ __forceinline__ ACoef<double> load_A<double>(const StepArgs &a, int g)
{
    return ACoef<double>{__ldg(a.A + g)};
}

// Store one element's nodal loads into its slot (slot gather accumulation).
template <typename R, int NPE>
__device__ __forceinline__ void store_slot(R *Ys, int slot, const R *F)
{
#pragma unroll
    for (int q = 0; q < NPE; ++q) Ys[slot * NPE + q] = F[q];
}

// Add one element's nodal loads into the tile accumulators.  With colour classes the element's
// nodes are distinct (a tet that lists a node twice has zero volume and is refused by the
// pre-computation) and no other element of the class touches them, so a tet issues all its
// loads before the stores (one shared-memory round trip instead of four in a row); hexahedra
// add node by node (their registers are taken by the element).
template <typename R, int NPE, int SCATTER>
__device__ __forceinline__ void add_loads(R *Fs, const R *F, const int *id)
{
    if (SCATTER == FEDFEM_SCATTER_ATOMIC) {
#pragma unroll
        for (int q = 0; q < NPE; ++q) atomicAdd(&Fs[id[q]], F[q]);
    } else if (NPE == 8) {
#pragma unroll
        for (int q = 0; q < NPE; ++q) Fs[id[q]] += F[q];
    } else {
        R f[NPE];
#pragma unroll
        for (int q = 0; q < NPE; ++q) f[q] = Fs[id[q]];
#pragma unroll
        for (int q = 0; q < NPE; ++q) Fs[id[q]] = f[q] + F[q];
    }
}

// The same for the two elements of a lane in a 64-element chunk (one colour: all their nodes
// are distinct); padding slots (use = false) add nothing.
template <typename R, int NPE>
__device__ __forceinline__ void add_loads2(R *Fs, const R *F0, const int *id0, bool use0, const R *F1,
                                           const int *id1, bool use1)
{
    R f0[NPE], f1[NPE];
#pragma unroll
    for (int q = 0; q < NPE; ++q) {
        if (use0) f0[q] = Fs[id0[q]];
        if (use1) f1[q] = Fs[id1[q]];
    }
#pragma unroll
    for (int q = 0; q < NPE; ++q) {
        if (use0) Fs[id0[q]] = f0[q] + F0[q];
        if (use1) Fs[id1[q]] = f1[q] + F1[q];
    }
}

// Tabulated f_k and f_c in the working precision (kernel parameters).
template <typename R>
__device__ __forceinline__ const HingeLaw<R> &law_k(const StepArgs &a);
template <typename R>
__device__ __forceinline__ const HingeLaw<R> &law_c(const StepArgs &a);
template <>
__device__ __forceinline__ const HingeLaw<float> &law_k<float>(const StepArgs &a)
{
    return a.tk32;
}
template <>
__device__ __forceinline__ const HingeLaw<double> &law_k<double>(const StepArgs &a)
{
    return a.tk64;
}
template <>
__device__ __forceinline__ const HingeLaw<float> &law_c<float>(const StepArgs &a)
{
    return a.tc32;
}
template <>
__device__ __forceinline__ const HingeLaw<double> &law_c<double>(const StepArgs &a)
{
    return a.tc64;
}

// Operands of the update of one halo node: T^{n-1}, its compensation, A, Q and the first four
// halo partials of step n-1.  halo_load issues every load at once (the partial count is not
// known at compile time, so a plain loop would wait for each partial before loading the next);
// halo_finish adds the partials in slot order and applies the update.
// Halo entries per consumer thread whose loads are in flight together.  Two is the most that
// fits the 128-register budget without spilling (measured at 128^3: 2 -> 76.5 us/step,
// 3 -> 79.3 us, 4 -> 85.6 us, all spills going to local memory).
#ifndef HALO_INFLIGHT
#define HALO_INFLIGHT 2
#endif
// Groups of four interior nodes per consumer thread whose loads are in flight together.
#ifndef UPD_INFLIGHT
#define UPD_INFLIGHT 2
#endif

template <typename R>
struct HaloIn {
    R p[2];  // partials of slots z, z + 1 (a shared node has at least two)
    R T, Q;
    float cp;
    ACoef<R> A;
    int cnt, z;
};

template <typename R, bool KAHAN>
__device__ __forceinline__ void halo_load(HaloIn<R> &h, const int4 sh, const R *Tprev, const float *cprev,
                                          const R *part, const R *Qext, const StepArgs &a)
{
    h.cnt = sh.w & 0xFFFF;
    h.z = sh.z;
    h.p[0] = ld_cg(part + sh.z);
    h.p[1] = ld_cg(part + sh.z + 1);
    h.T = ld_cg(Tprev + sh.y);
    h.cp = KAHAN ? ld_cg(cprev + sh.y) : 0.0f;
    h.A = load_A<R>(a, sh.y);
    h.Q = Qext[sh.y];
}

// T^n of a halo node from T^{n-1}, its compensation and the fixed-order sum of the halo
// partials of step n-1.
template <typename R, bool KAHAN, bool TAB, int NH = kHinges>
__device__ __forceinline__ R halo_finish(const HaloIn<R> &h, const R *part, const Phys<R> &ph,
                                         const HingeLaw<R> &tc, float &cn, int32_t *err, R &F)
{
    F = 0;
    F += h.p[0];
    F += h.p[1];
    for (int q = 2; q < h.cnt; ++q) F += ld_cg(part + h.z + q);
    return node_update<R, KAHAN, TAB, NH>(h.T, h.cp, h.A, h.Q * ph.qs_prev, F, ph.dD_prev, ph, tc, cn, err);
}

// Energy audit (an instantiation of the step kernel): every node update adds, in FP64, the
// stored-heat change C0_i f_c(T_i) (T_i' - T_i) of a free node (values with their Kahan
// compensation) and the boundary input dt Q_i (free node) or dt F_i (Dirichlet node), F here
// including the node's surface outflow, which the surface pass subtracts again as -dt outflow;
// shared nodes are counted by their owner tile only.  Sums per thread, per CTA at launch end.
template <bool EN>
struct EnergyAcc {
    double S = 0.0, B = 0.0;
    double c_a = 0.0, c_lin = 0.0;  // capacity law of the current tile's problem (FP64)
    __device__ __forceinline__ void set_law(const PhysParams *pp)
    {
        if constexpr (EN) {
            c_a = pp->c_a;
            c_lin = pp->c_lin;
        }
    }
    template <typename R>
    __device__ __forceinline__ void node(const StepArgs &a, int g, R T, float c, R Tn, float cn, bool dir, R Q, R F)
    {
        if constexpr (EN) {
            const double t0 = (double)T - (double)c, t1 = (double)Tn - (double)cn;
            if (!dir) S += a.C0[g] * (c_a + c_lin * t0) * (t1 - t0);
            B += a.dt * (double)(dir ? F : Q);
        }
    }
    template <typename R>
    __device__ __forceinline__ void outflow(const StepArgs &a, R o)
    {
        if constexpr (EN) B -= a.dt * (double)o;
    }
};

// Shared-memory layout: [stages][chunk_bytes] ring | MBAR_BYTES of mbarriers (full[S], empty[S],
// node) | Ts[ts_cap] | Fs[ts_cap].  Threads [0, NC) are consumers; the last warp is the
// producer of the element ring.  With at most 15 consumer warps + 1 producer warp every SM
// sub-partition holds at most 4 warps, which leaves 128 registers per thread.
template <typename R, int NPE, bool KAHAN, int SCATTER, int TABN, bool EN>
__global__ void __maxnreg__(sizeof(R) == 8 ? 168 : 128) fed_step_kernel(const StepArgs a, int ts_cap)
{
    // TABN: 0 = the linear laws; else tabulated factors with up to TABN hinges evaluated
    constexpr bool TAB = TABN > 0;
    constexpr int NH = TAB ? TABN : kHinges;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_ok;
    // the current tile's record and physics, staged once per tile (kept out of registers)
    __shared__ TileInfo s_ti;
    __shared__ int s_colptr[65];  // the tile's colour-class chunk offsets (at most 64 classes)
    __shared__ Phys<R> s_ph, s_ph0;
    constexpr int ALN = 16 / sizeof(R);  // nodes per 16 bytes
    const int NC = blockDim.x - 32;      // consumer threads
    const int NW = NC / 32;              // consumer warps
    const int CH = a.chunk;              // elements per chunk: 32 or 64
    const int EPT = CH / 32;             // elements per thread and chunk
    const int tid = threadIdx.x;
    const int wid = tid >> 5, lane32 = tid & 31;
    const int S = a.stages;
    constexpr int HU = HALO_INFLIGHT;  // halo entries per thread in flight
    uint8_t *ring = smem;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)S * a.chunk_bytes);
    uint64_t *empty = full + S;
    uint64_t *tbar = empty + S;
    volatile int *tag = reinterpret_cast<volatile int *>(tbar + 1);  // chunk index held by each slot
    R *Ts_raw = reinterpret_cast<R *>(smem + (size_t)S * a.chunk_bytes + MBAR_BYTES);
    R *Fs = Ts_raw + ts_cap;
    R *Ys = Fs + ts_cap;  // slot gather: element load slots of the current tile

    const int t0 = a.cta_tile ? a.cta_tile[blockIdx.x] : blockIdx.x * a.tiles_per_cta;
    const int t1 = a.cta_tile ? a.cta_tile[blockIdx.x + 1] : min(t0 + a.tiles_per_cta, a.n_tiles);
    const int cb = t0 < t1 ? a.tiles[t0].chunk_begin : 0;
    const int nch = t0 < t1 ? a.tiles[t1 - 1].chunk_begin + a.tiles[t1 - 1].n_chunks - cb : 0;
    const long long total = (long long)nch * a.nsteps;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);  // released by the warp that consumed it
        }
        mbar_init(tbar, 1);
        for (int s2 = 0; s2 < S; ++s2) tag[s2] = -1;
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();  // the only CTA-wide barrier (before the roles split)

    // ---------------------------------------------------------------- producer warp
    if (tid >= NC) {
        if (tid == NC) {
            const uint64_t pol = a.l2_stream_policy == 1 ? policy_evict_first() : policy_evict_normal();
            // 32-bit incremental ring bookkeeping (the counts of one launch fit in 32 bits)
            const int tot = (int)total;
            int k = 0, slot = 0, ch = 0;
            uint32_t ephase = 0;  // parity of the empty-barrier phase awaited for this slot
            for (; k < tot; ++k) {
                if (k >= S && !mbar_wait_or_abort(&empty[slot], ephase, a.timeout_ns, a.err)) break;
                tag[slot] = k;  // consumers check the tag after the parity test
                mbar_arrive_expect_tx(&full[slot], (uint32_t)a.chunk_bytes);
                tma_bulk_g2s(ring + (size_t)slot * a.chunk_bytes, a.chunks + (size_t)(cb + ch) * a.chunk_bytes,
                             (uint32_t)a.chunk_bytes, &full[slot], pol);
                if (++ch == nch) ch = 0;
                if (++slot == S) {
                    slot = 0;
                    if (k >= S) ephase ^= 1;
                }
            }
            // wait (bounded) until this CTA's last copies have landed before the warp leaves
            for (int j = k > S ? k - S : 0; j < k; ++j) mbar_wait(&full[j % S], (uint32_t)((j / S) & 1), a.timeout_ns);
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    // Staggered start: CTAs that begin a launch in lockstep stream their elements at the same
    // time and then leave DRAM idle together in their node phases; delaying CTA b by
    // stagger * b / grid (at most a few tens of us, once per launch) spreads the phases from the
    // first step on.  The producer warp starts at once and fills the ring meanwhile.
    if (a.stagger_ns > 0) {
        const long long dl = a.stagger_ns * (long long)blockIdx.x / (long long)gridDim.x;
        const unsigned long long d0 = global_ns();
        while ((long long)(global_ns() - d0) < dl) __nanosleep(256);
    }
    const R *Qext = reinterpret_cast<const R *>(a.Qext);
    const int col_off = a.colour_offset;

    EnergyAcc<EN> en;
    int kc = 0;           // chunks consumed (fits in 32 bits per launch)
    uint32_t tphase = 0;  // phase of the node-load barrier
    bool ok = true;
    for (int s = 0; s < a.nsteps && ok; ++s) {
        const long long n = a.n0 + s;
        const int cur = (int)(n & 1), nxt = cur ^ 1;
        R *Tc = reinterpret_cast<R *>(a.T[cur]);
        R *Tn = reinterpret_cast<R *>(a.T[nxt]);
        for (int t = t0; t < t1 && ok; ++t) {
            if (tid == 0) {
                // a CTA with one tile reads its record and physics once per launch
                if (s == 0 || t1 - t0 > 1) {
                    s_ti = a.tiles[t];
                    s_ph0 = Phys<R>(a.phys[s_ti.scenario]);
                }
                s_ph = s_ph0;
                apply_schedule(s_ph, a, a.n0 + s);
            }
            csync(NC);
            const TileInfo &ti = s_ti;
            const Phys<R> &ph = s_ph;
            if (SCATTER == FEDFEM_SCATTER_COLOR && tid <= ti.n_colors)  // read after the barrier
                s_colptr[tid] = __ldg(a.colptr + ti.col_begin + tid);     // before the elements
            en.set_law(a.phys + ti.scenario);
            const int nb = ti.node_begin;
            const int a0 = nb & ~(ALN - 1);
            const int a1 = (nb + ti.n_owned + ALN - 1) & ~(ALN - 1);
            R *Ts = Ts_raw + (nb - a0);
            // ---- T^n of the interior nodes: a CTA with one tile keeps them in shared memory
            //      from its own update of the previous step; at the first step of a launch, and
            //      when a CTA takes several tiles, the owned range arrives by one bulk copy.
            //      L2 prefetch of the update operands.
            const bool bulk = s == 0 || t1 - t0 > 1;
            if (tid == 0) {
                if (bulk) {
                    mbar_arrive_expect_tx(tbar, (uint32_t)((a1 - a0) * sizeof(R)));
                    tma_bulk_g2s(Ts_raw, Tc + a0, (uint32_t)((a1 - a0) * sizeof(R)), tbar, policy_evict_normal());
                }
                const int i0 = nb & ~3, i1 = (nb + ti.n_interior + 3) & ~3;
                if (i1 > i0) {
                    const uint64_t pk = a.l2_stream_policy == 1 ? policy_evict_last() : policy_evict_normal();
                    if (sizeof(R) == 4)
                        l2_prefetch_bulk(a.A2 + i0, (uint32_t)((i1 - i0) * 8), pk);
                    else
                        l2_prefetch_bulk(a.A + i0, (uint32_t)((i1 - i0) * 8), pk);
                    l2_prefetch_bulk(Qext + i0, (uint32_t)((i1 - i0) * sizeof(R)), pk);
                    if (KAHAN) l2_prefetch_bulk(a.comp[cur] + i0, (uint32_t)((i1 - i0) * 4), pk);
                }
            }
            if (s > 0 && !tile_wait(a.tile_done, a.nbr_ptr, a.nbr, t, a.progress_base + (unsigned)s, a.err,
                                    a.timeout_ns, NC, &s_ok)) {
                ok = false;
                break;
            }
            // ---- halo nodes (local ids [n_interior, n_local)): T^n from T^(n-1) and the halo
            //      partials of step n-1 (the owner writes it back); HU entries per thread in
            //      flight, the next HU entries loaded meanwhile.  The values go straight into Ts,
            //      or into Fs (free until the element phase) while a bulk copy is in flight.
            R *Hs = bulk ? Fs : Ts;
            const int4 *shp = a.sh + ti.sh_begin;
            int4 shn[HU];
#pragma unroll
            for (int u = 0; u < HU; ++u)
                if (tid + u * NC < ti.sh_count) shn[u] = __ldg(shp + tid + u * NC);
            for (int q0 = tid; q0 < ti.sh_count; q0 += HU * NC) {
                int4 sh[HU];
#pragma unroll
                for (int u = 0; u < HU; ++u) {
                    sh[u] = shn[u];
                    if (q0 + (HU + u) * NC < ti.sh_count) shn[u] = __ldg(shp + q0 + (HU + u) * NC);
                }
                const R *pprev = reinterpret_cast<const R *>(a.part[nxt]);
                HaloIn<R> hin[HU];
                if (s > 0) {
#pragma unroll
                    for (int u = 0; u < HU; ++u)
                        if (q0 + u * NC < ti.sh_count)
                            halo_load<R, KAHAN>(hin[u], sh[u], Tn, KAHAN ? a.comp[nxt] : nullptr, pprev, Qext, a);
                }
#pragma unroll
                for (int u = 0; u < HU; ++u) {
                    if (q0 + u * NC >= ti.sh_count) continue;
                    if (s == 0) {
                        Hs[sh[u].x] = ld_cg(Tc + sh[u].y);
                        continue;
                    }
                    float cn;
                    R Fh;
                    const R v = halo_finish<R, KAHAN, TAB, NH>(hin[u], pprev, ph, law_c<R>(a), cn, a.err, Fh);
                    if ((sh[u].w >> 16) == 0) {  // owner writes T^n back
                        Tc[sh[u].y] = v;
                        if (KAHAN) a.comp[cur][sh[u].y] = cn;
                        en.node(a, sh[u].y, hin[u].T, hin[u].cp, v, cn, hin[u].A.dir(), hin[u].Q * ph.qs_prev, Fh);
                    }
                    Hs[sh[u].x] = v;
                }
            }
            if (bulk) {
                const int bad = mbar_wait_or_abort(tbar, tphase, a.timeout_ns, a.err) ? 0 : 1;
                tphase ^= 1;
                if (csync_or(NC, bad)) {
                    ok = false;
                    break;
                }
            }
            // halo values into Ts after a bulk copy; accumulators cleared
            for (int l = tid; l < ti.n_local; l += NC) {
                if (bulk && l >= ti.n_interior) Ts[l] = Fs[l];
                Fs[l] = (R)0;
            }
            if (a.rec) {
                if (!bulk) csync(NC);  // the halo values were written by other threads
                R *rec = reinterpret_cast<R *>(a.rec) + (size_t)s * a.rec_stride;
                for (int l = tid; l < ti.n_owned; l += NC) rec[nb + l] = Ts[l];
            }
            csync(NC);
            // ---- element loads (Eq. 20), colour class by colour class.  Every chunk holds one
            //      colour; chunk u of the tile is consumed by warp (kbase + u) mod NW, which adds
            //      its elements into the shared-memory accumulators with plain read-modify-writes
            //      (elements of one colour share no node).  The CTA synchronises only between
            //      classes, so every node receives its contributions in a fixed order.  The
            //      atomic variant treats the whole tile as one class and adds with atomics.
            {
                const int kbase = kc;
                const int ncls = SCATTER == FEDFEM_SCATTER_COLOR ? ti.n_colors : 1;
                // This warp consumes the tile's chunks k = wk, wk + NW, ... with k = wid (mod NW)
                // (in every class, chunk u goes to warp (kbase + u) mod NW).  For tets (a warp
                // takes about one chunk per class) the ring slot and phase parity of its next
                // chunk advance incrementally; the hexahedral kernels, whose registers are taken
                // by the element, form k / S as the high half of k * ceil(2^64 / S) (exact for
                // k < 2^58).  Either way no integer division per chunk.
                constexpr bool INCR = NPE == 4;
                int wk = kbase + (wid - kbase % NW + NW) % NW;
                int wslot = 0;
                uint32_t wpar = 0;
                if constexpr (INCR) {
                    wslot = wk % S;
                    wpar = (uint32_t)((wk / S) & 1);
                }
                for (int c = 0; c < ncls; ++c) {
                    int u1 = ti.n_chunks;
                    if (SCATTER == FEDFEM_SCATTER_COLOR) u1 = s_colptr[c + 1];
                    const int k1 = kbase + u1;
                    int bad = 0;
                    // the class holds chunks [kbase + u0, k1); this warp's next chunk wk is the
                    // first of them with wk = wid (mod NW), since the previous class ended at u0
                    for (; wk < k1; wk += NW) {
                        const int k = wk;
                        const int u = k - kbase;
                        int slot;
                        uint32_t par;
                        if constexpr (INCR) {
                            slot = wslot;
                            par = wpar;
                            wslot += NW;
                            while (wslot >= S) {
                                wslot -= S;
                                wpar ^= 1u;
                            }
                        } else {
                            const uint64_t q = __umul64hi((uint64_t)k, a.stage_magic);
                            slot = k - (int)q * S;
                            par = (uint32_t)(q & 1);
                        }
                        if (!wait_chunk(&full[slot], tag + slot, k, par, a.timeout_ns, a.err)) {
                            bad = 1;
                            break;
                        }
                        const uint8_t *blk = ring + (size_t)slot * a.chunk_bytes;
                        if (EPT == 1) {
                            R F[NPE];
                            int id[NPE];
                            const int col = blk[col_off + lane32];
                            element_loads<R, NPE, TAB, NH>(blk, CH, lane32, Ts, ph.k_a, ph.k_lin, law_k<R>(a), F, id);
                            __syncwarp();
                            if (lane32 == 0) mbar_arrive(&empty[slot]);  // stage back to the producer
                            if (col != 0xFF) {
                                if (SCATTER == FEDFEM_SCATTER_SLOTS)
                                    store_slot<R, NPE>(Ys, u * CH + lane32, F);
                                else
                                    add_loads<R, NPE, SCATTER>(Fs, F, id);
                            }
                        } else {
                            R F0[NPE], F1[NPE];
                            int id0[NPE], id1[NPE];
                            const int col0 = blk[col_off + lane32], col1 = blk[col_off + lane32 + 32];
                            element_loads<R, NPE, TAB, NH>(blk, CH, lane32, Ts, ph.k_a, ph.k_lin, law_k<R>(a), F0, id0);
                            element_loads<R, NPE, TAB, NH>(blk, CH, lane32 + 32, Ts, ph.k_a, ph.k_lin, law_k<R>(a), F1,
                                                       id1);
                            __syncwarp();
                            if (lane32 == 0) mbar_arrive(&empty[slot]);
                            if (SCATTER == FEDFEM_SCATTER_SLOTS) {
                                if (col0 != 0xFF) store_slot<R, NPE>(Ys, u * CH + lane32, F0);
                                if (col1 != 0xFF) store_slot<R, NPE>(Ys, u * CH + lane32 + 32, F1);
                            } else if (SCATTER == FEDFEM_SCATTER_COLOR && NPE == 4) {
                                add_loads2<R, NPE>(Fs, F0, id0, col0 != 0xFF, F1, id1, col1 != 0xFF);
                            } else {
                                if (col0 != 0xFF) add_loads<R, NPE, SCATTER>(Fs, F0, id0);
                                if (col1 != 0xFF) add_loads<R, NPE, SCATTER>(Fs, F1, id1);
                            }
                        }
                    }
                    if (csync_or(NC, bad)) {
                        ok = false;
                        break;
                    }
                }
                kc += ti.n_chunks;
            }
            if (!ok) break;
            // ---- slot gather: every local node sums the element slots that touch it, in
            //      ascending slot order (after the class barrier above, all slots are written)
            if (SCATTER == FEDFEM_SCATTER_SLOTS) {
                const int32_t *gp = a.gptr + ti.gp_begin;
                for (int l = tid; l < ti.n_local; l += NC) {
                    const int q1 = __ldg(gp + l + 1);
                    R f = 0;
                    for (int q = __ldg(gp + l); q < q1; ++q) f += Ys[__ldg(a.gidx + q)];
                    Fs[l] = f;
                }
                csync(NC);
            }
            // ---- surface loads of owned boundary nodes
            for (int q = tid; q < ti.bnd_count; q += NC) {
                // the entry and its node's areas are independent loads (one round trip)
                using R2 = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
                const int2 b = a.bnd[ti.bnd_begin + q];
                const R2 ar = reinterpret_cast<const R2 *>(a.bnd_area)[ti.bnd_begin + q];
                const R o = surface_outflow<R>(Ts[b.x], ar.x, ar.y, ph);
                Fs[b.x] += o;
                en.outflow(a, o);
            }
            csync(NC);
            // ---- halo partials (the only data other tiles read after the barrier): entry q is
            //      local node n_interior + q; only its (first slot, count | rank) pair is read
            R *part = reinterpret_cast<R *>(a.part[cur]);
            for (int q = tid; q < ti.sh_count; q += NC) {
                const int4 sh = a.sh[ti.sh_begin + q];
                part[sh.z + (sh.w >> 16)] = Fs[sh.x];
            }
            {
                // publish the step: the interior updates below touch only this tile's own nodes
                const bool withhold = a.withhold > 0 && (int)blockIdx.x == a.withhold - 1;
                tile_publish(a.tile_done, t, a.progress_base + (unsigned)(s + 1), withhold, NC);
            }
            // ---- update interior nodes: aligned groups of four consecutive nodes per thread
            //      (vector loads), UG groups in flight; scalar head and tail
            {
                constexpr int UG = UPD_INFLIGHT;
                const int head = min(ti.n_interior, (4 - (nb & 3)) & 3);
                const int ngrp = (ti.n_interior - head) >> 2;
                const int tail0 = head + 4 * ngrp;
                for (int j0 = tid; j0 < ngrp; j0 += UG * NC) {
                    Vec4<R> Qv[UG], cpv[UG];
                    ACoef<R> Av[UG][4];
#pragma unroll
                    for (int u = 0; u < UG; ++u) {
                        const int j = j0 + u * NC;
                        if (j < ngrp) {
                            const int g = nb + head + 4 * j;
                            Qv[u] = load4<R>(Qext + g);
                            load_A4<R>(a, g, Av[u]);
                            if (KAHAN) cpv[u] = load4<R>(reinterpret_cast<const R *>(a.comp[cur] + g));
                        }
                    }
#pragma unroll
                    for (int u = 0; u < UG; ++u) {
                        const int j = j0 + u * NC;
                        if (j < ngrp) {
                            const int l = head + 4 * j;
                            const int g = nb + l;
                            Vec4<R> out, cout;
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                float cn;
                                const R Told = Ts[l + e];
                                out.v[e] = node_update<R, KAHAN, TAB, NH>(Told, KAHAN ? (float)cpv[u].v[e] : 0.0f,
                                                                       Av[u][e], Qv[u].v[e] * ph.qs, Fs[l + e], ph.dD,
                                                                       ph, law_c<R>(a), cn, a.err);
                                en.node(a, g + e, Told, KAHAN ? (float)cpv[u].v[e] : 0.0f, out.v[e], cn,
                                        Av[u][e].dir(), Qv[u].v[e] * ph.qs, Fs[l + e]);
                                cout.v[e] = (R)cn;
                                Ts[l + e] = out.v[e];  // kept for the next step
                            }
                            store4<R>(Tn + g, out);
                            if (KAHAN) store4<R>(reinterpret_cast<R *>(a.comp[nxt] + g), cout);
                        }
                    }
                }
                for (int l = tid; l < ti.n_interior; l += NC) {
                    if (l >= head && l < tail0) continue;
                    const int g = nb + l;
                    float cn;
                    const float c0 = KAHAN ? ld_cg(a.comp[cur] + g) : 0.0f;
                    const ACoef<R> Ag = load_A<R>(a, g);
                    const R v = node_update<R, KAHAN, TAB, NH>(Ts[l], c0, Ag, Qext[g] * ph.qs, Fs[l], ph.dD, ph,
                                                           law_c<R>(a), cn, a.err);
                    en.node(a, g, Ts[l], c0, v, cn, Ag.dir(), Qext[g] * ph.qs, Fs[l]);
                    Tn[g] = v;
                    Ts[l] = v;
                    if (KAHAN) a.comp[nxt][g] = cn;
                }
            }
            if (t1 - t0 > 1) {
                // the next tile's bulk copy (async proxy) reads T written here and overwrites
                // the shared memory written here
                fence_proxy_async_global();
                fence_proxy_async_smem();
            }
            csync(NC);
        }
        if (!ok) break;
    }

    if (ok) {
        // finish the owned halo nodes at the final step
        const long long n = a.n0 + a.nsteps;
        const int cur = (int)(n & 1), prv = cur ^ 1;
        R *Tc = reinterpret_cast<R *>(a.T[cur]);
        const R *Tp = reinterpret_cast<const R *>(a.T[prv]);
        const R *part = reinterpret_cast<const R *>(a.part[prv]);
        for (int t = t0; t < t1 && ok; ++t) {
            if (!tile_wait(a.tile_done, a.nbr_ptr, a.nbr, t, a.progress_base + (unsigned)a.nsteps, a.err, a.timeout_ns,
                           NC, &s_ok)) {
                ok = false;
                break;
            }
            const TileInfo ti = a.tiles[t];
            Phys<R> ph(a.phys[ti.scenario]);
            apply_schedule(ph, a, n);  // qs_prev: the loads of step n - 1
            en.set_law(a.phys + ti.scenario);
            for (int q = tid; q < ti.sh_count; q += NC) {
                const int4 sh = a.sh[ti.sh_begin + q];
                if ((sh.w >> 16) != 0) continue;
                float cn;
                HaloIn<R> h;
                halo_load<R, KAHAN>(h, sh, Tp, KAHAN ? a.comp[prv] : nullptr, part, Qext, a);
                R Fh;
                const R v = halo_finish<R, KAHAN, TAB, NH>(h, part, ph, law_c<R>(a), cn, a.err, Fh);
                Tc[sh.y] = v;
                if (KAHAN) a.comp[cur][sh.y] = cn;
                en.node(a, sh.y, h.T, h.cp, v, cn, h.A.dir(), h.Q * ph.qs_prev, Fh);
            }
        }
    }
    if constexpr (EN) {
        // the CTA's sums in a fixed order: lanes by shuffle, then warps in order; added to the
        // CTA's own running totals.  The node accumulators (Fs, free after the last update and
        // 16-byte aligned) hold the per-warp sums, so the audit adds no shared memory.
        double *e_red = reinterpret_cast<double *>(Fs);
        double eS = en.S, eB = en.B;
        for (int o = 16; o > 0; o >>= 1) {
            eS += __shfl_down_sync(0xffffffffu, eS, o);
            eB += __shfl_down_sync(0xffffffffu, eB, o);
        }
        if (lane32 == 0) {
            e_red[2 * wid] = eS;
            e_red[2 * wid + 1] = eB;
        }
        csync(NC);
        if (tid == 0 && ok) {
            double S = 0.0, B = 0.0;
            for (int w = 0; w < NW; ++w) {
                S += e_red[2 * w];
                B += e_red[2 * w + 1];
            }
            a.energy_acc[2 * blockIdx.x] += S;
            a.energy_acc[2 * blockIdx.x + 1] += B;
        }
    }
}

template <typename R>
__global__ void k_bnd_areas(int64_t n, const int2 *bnd, const R *Ac, const R *Ar, R *out)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int g = bnd[q].y;
        out[2 * q] = Ac[g];
        out[2 * q + 1] = Ar[g];
    }
}

cudaError_t launch_bnd_areas(int precision, int64_t n, const int2 *bnd, const void *Ac, const void *Ar, void *out,
                             cudaStream_t st)
{
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    if (precision == 64)
        k_bnd_areas<double><<<blocks, 256, 0, st>>>(n, bnd, static_cast<const double *>(Ac),
                                                    static_cast<const double *>(Ar), static_cast<double *>(out));
    else
        k_bnd_areas<float><<<blocks, 256, 0, st>>>(n, bnd, static_cast<const float *>(Ac),
                                                   static_cast<const float *>(Ar), static_cast<float *>(out));
    return cudaGetLastError();
}

int step_ts_cap(int precision, int max_local)
{
    const int aln = precision == 64 ? 2 : 4;
    return ((max_local + 2 * aln) + 3) & ~3;
}

size_t step_smem_bytes(int precision, int npe, int chunk, int stages, int max_local, int slot_cap)
{
    const size_t rs = precision == 64 ? 8 : 4;
    return (size_t)stages * chunk_bytes_for(precision, npe, chunk) + MBAR_BYTES +
           2 * (size_t)step_ts_cap(precision, max_local) * rs + (size_t)slot_cap * npe * rs;
}

// table: the number of points of the property tables (0 = the linear laws).  Tables of up to
// five points (at most three hinges) take an instance that evaluates three hinges, larger
// ones all kHinges.
template <typename R, int NPE, bool KAHAN, int SCATTER>
static void *kernel_ptr(int table)
{
    if (table <= 0) return (void *)fed_step_kernel<R, NPE, KAHAN, SCATTER, 0, false>;
    if (table - 2 <= 3) return (void *)fed_step_kernel<R, NPE, KAHAN, SCATTER, 3, false>;
    return (void *)fed_step_kernel<R, NPE, KAHAN, SCATTER, kHinges, false>;
}

template <typename R, int NPE, bool KAHAN>
static void *slots_kernel_ptr(int table)
{
    return kernel_ptr<R, NPE, KAHAN, FEDFEM_SCATTER_SLOTS>(table);
}

// Energy-audit instantiations: colour scatter and the linear laws, FP32 + Kahan or FP64.
static void *select_energy_kernel(int precision, int kahan, int npe)
{
    if (precision == 64)
        return npe == 8 ? (void *)fed_step_kernel<double, 8, false, FEDFEM_SCATTER_COLOR, 0, true>
                        : (void *)fed_step_kernel<double, 4, false, FEDFEM_SCATTER_COLOR, 0, true>;
    if (!kahan) return nullptr;
    return npe == 8 ? (void *)fed_step_kernel<float, 8, true, FEDFEM_SCATTER_COLOR, 0, true>
                    : (void *)fed_step_kernel<float, 4, true, FEDFEM_SCATTER_COLOR, 0, true>;
}

static void *select_kernel(int precision, int kahan, int npe, int scatter, int table)
{
#define FEDFEM_SEL(R, N, K)                                                                        \
    return scatter == FEDFEM_SCATTER_ATOMIC  ? kernel_ptr<R, N, K, FEDFEM_SCATTER_ATOMIC>(table)   \
           : scatter == FEDFEM_SCATTER_SLOTS ? slots_kernel_ptr<R, N, K>(table)                    \
                                             : kernel_ptr<R, N, K, FEDFEM_SCATTER_COLOR>(table)
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
    void *k = select_kernel(precision, kahan, npe, FEDFEM_SCATTER_COLOR, 0);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block + 32, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t prepare_step(int precision, int kahan, int npe, int scatter, int table, size_t smem)
{
    return cudaFuncSetAttribute(select_kernel(precision, kahan, npe, scatter, table),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_step(const StepArgs &a, int precision, int kahan, int npe, int table, int grid, int block,
                        size_t smem, int ts_cap, cudaStream_t st)
{
    void *k = a.energy_acc ? select_energy_kernel(precision, kahan, npe) : select_kernel(precision, kahan, npe, a.scatter, table);
    if (!k) return cudaErrorInvalidValue;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusNone) {  // while capturing, prepare_step has done this
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    StepArgs args = a;
    void *params[] = {(void *)&args, (void *)&ts_cap};
    // block consumer threads plus one producer warp for the element ring; a cooperative launch
    // (all CTAs co-resident, since tiles wait for their neighbours) that can also be captured in a CUDA graph
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block + 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, k, params);
}

}  // namespace fedfem
