// fedfem_energy_terms_noalloc: the energy-balance reduction of fedfem_energy for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits, such as a solver callback
// executed while another library owns the device memory pool, a process working under a hard
// device-memory budget, or a host loop that must not synchronise (cudaMalloc and cudaFree can
// synchronise the device).  The reduction's only temporary storage (one pair of partial sums
// per thread block) therefore lives in a file-scope device array that exists for as long as
// the library is loaded, instead of in memory allocated per call or per context.
//
// Limits and behaviour:
//  - at most kMaxBlocks blocks of kItemsPerBlock nodes, i.e. n_nodes <= 16,777,216; larger
//    sizes are rejected with FEDFEM_ERR_ARG;
//  - every GPU that loads the library holds the 64 KB array until the process exits;
//  - all calls on a device share the array: calls whose work overlaps on the GPU (different
//    streams, or host threads without ordering) race and give wrong sums.  Every call
//    overwrites all the partial sums it reads, so nothing has to be cleared between calls;
//  - the first call on each device looks the array's device address up with
//    cudaGetSymbolAddress (with that device current); make that first call before any stream
//    capture begins.  The address is kept for the life of the process: do not use this entry
//    point on a device after cudaDeviceReset (or any other reset of its primary context),
//    which reloads the library's device code at a possibly different address;
//  - the sums are those of fedfem_energy for the step whose data the caller passes: with a
//    load schedule, Qext must already carry that step's load multiplier and T_inf must be
//    that step's convection temperature.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fedfem.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItemsPerThread = 16;
constexpr int kItemsPerBlock = kThreads * kItemsPerThread;  // 4096 nodes per block
constexpr int kMaxBlocks = 4096;                            // 16,777,216 nodes at most
constexpr int kMaxDevices = 64;

// per-block partial sums (S, B) of the last call on this device
static __device__ __align__(256) double g_partials[2 * kMaxBlocks];

double *g_partials_addr[kMaxDevices];
bool g_partials_ready[kMaxDevices];
std::mutex g_lock;

__device__ __forceinline__ void warp_sum2(double &a, double &b)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
}

// Block b reduces nodes [b * kItemsPerBlock, (b + 1) * kItemsPerBlock) in a fixed order.
__global__ void __launch_bounds__(kThreads) k_energy_blocks(int64_t n, const double *T0, const double *T1,
                                                             const double *F, const double *C0, const double *Qext,
                                                             const double *Ac, const double *Ar, const uint8_t *isdir,
                                                             double dt, double c_lin, double h, double T_inf,
                                                             double eps_sigma, double T_amb, double T_zero,
                                                             double T_ref, double *partials)
{
    __shared__ double red[2 * (kThreads / 32)];
    double S = 0.0, B = 0.0;
    const int64_t base = (int64_t)blockIdx.x * kItemsPerBlock;
    for (int i = 0; i < kItemsPerThread; ++i) {
        const int64_t g = base + (int64_t)i * kThreads + threadIdx.x;
        if (g >= n) break;
        if (isdir[g]) {
            B += dt * F[g];
            continue;
        }
        const double t = T0[g];
        const double u = t - T_zero, b = T_amb - T_zero;
        const double Q = Qext[g] - Ac[g] * h * (t - T_inf) - Ar[g] * eps_sigma * ((u - b) * (u + b) * (u * u + b * b));
        S += C0[g] * (1.0 + c_lin * (t - T_ref)) * (T1[g] - t);
        B += dt * Q;
    }
    warp_sum2(S, B);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[2 * w] = S;
        red[2 * w + 1] = B;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0, bb = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) {
            s += red[2 * k];
            bb += red[2 * k + 1];
        }
        partials[2 * blockIdx.x] = s;
        partials[2 * blockIdx.x + 1] = bb;
    }
}

// One block adds the per-block partials in a fixed order and writes (S, B) to out.
__global__ void __launch_bounds__(kThreads) k_energy_final(int nblocks, const double *partials, double *out)
{
    __shared__ double red[2 * (kThreads / 32)];
    double S = 0.0, B = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += kThreads) {
        S += partials[2 * i];
        B += partials[2 * i + 1];
    }
    warp_sum2(S, B);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[2 * w] = S;
        red[2 * w + 1] = B;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0, bb = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) {
            s += red[2 * k];
            bb += red[2 * k + 1];
        }
        out[0] = s;
        out[1] = bb;
    }
}

// Device address of g_partials on the current device (looked up once per device).
fedfem_status partials_on_current_device(double **ptr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FEDFEM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return FEDFEM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_partials_ready[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || p == nullptr) return FEDFEM_ERR_CUDA;
        g_partials_addr[dev] = static_cast<double *>(p);
        g_partials_ready[dev] = true;
    }
    *ptr = g_partials_addr[dev];
    return FEDFEM_OK;
}

}  // namespace

extern "C" fedfem_status fedfem_energy_terms_noalloc(int64_t n_nodes, const double *T_prev, const double *T_next,
                                                     const double *F, const double *C0, const double *Qext,
                                                     const double *Ac, const double *Ar, const uint8_t *is_dirichlet,
                                                     const fedfem_energy_params *ph, double *out, void *stream)
{
    if (n_nodes <= 0 || n_nodes > (int64_t)kMaxBlocks * kItemsPerBlock) return FEDFEM_ERR_ARG;
    if (!T_prev || !T_next || !F || !C0 || !Qext || !Ac || !Ar || !is_dirichlet || !ph || !out) return FEDFEM_ERR_ARG;
    double *partials = nullptr;
    const fedfem_status st = partials_on_current_device(&partials);
    if (st != FEDFEM_OK) return st;
    const int nblocks = (int)((n_nodes + kItemsPerBlock - 1) / kItemsPerBlock);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // each launch's own return code: an error left behind by unrelated earlier work is neither
    // reported here nor cleared
    double dt = ph->dt, c_lin = ph->c_lin, h = ph->h, T_inf = ph->T_inf, eps_sigma = ph->eps * 5.67e-8,
           T_amb = ph->T_amb, T_zero = ph->T_zero, T_ref = ph->T_ref;
    void *args1[] = {&n_nodes, &T_prev, &T_next, &F, &C0, &Qext, &Ac, &Ar, &is_dirichlet, &dt, &c_lin,
                     &h, &T_inf, &eps_sigma, &T_amb, &T_zero, &T_ref, &partials};
    if (cudaLaunchKernel((const void *)k_energy_blocks, dim3(nblocks), dim3(kThreads), args1, 0, s) != cudaSuccess)
        return FEDFEM_ERR_CUDA;
    int nb = nblocks;
    void *args2[] = {&nb, &partials, &out};
    if (cudaLaunchKernel((const void *)k_energy_final, dim3(1), dim3(kThreads), args2, 0, s) != cudaSuccess)
        return FEDFEM_ERR_CUDA;
    return FEDFEM_OK;
}
