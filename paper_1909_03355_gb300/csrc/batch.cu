// Batched scenarios: many independent FED-FEM problems advanced together (no counterpart in
// the paper).
//
// The scenarios are packed into one mesh, ordered by decreasing step count, and tiled so that
// no tile spans two scenarios.  While the run is between two consecutive distinct step counts
// the set of unfinished scenarios is fixed and, thanks to the ordering, its tiles are a prefix
// of the tile order: each such phase is a sequence of persistent launches of the ordinary step
// kernel over that prefix, with CTA -> tile ranges balanced by element count.  Each tile
// carries its scenario's physical constants (a per-scenario table) and each node its
// scenario's time step (folded into A = dt / C0).  The critical step of every scenario comes
// from FP64 Lanczos segmented by scenario.  The whole launch sequence is captured
// once in a CUDA graph and replayed by fedfem_batch_run; %globaltimer stamps at the phase ends
// give each scenario's completion time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "ctx.h"

using namespace fedfem;

struct fedfem_batch {
    std::string err;
    fedfem_ctx *c = nullptr;
    int S = 0;
    std::vector<int> order;            // packed position -> scenario index
    std::vector<int> pos;              // scenario index -> packed position
    std::vector<int64_t> node_off;     // packed node offsets (original node order of each scenario)
    std::vector<int64_t> steps;        // per packed position
    std::vector<double> dt, dt_crit;   // per scenario index
    std::vector<int> phase_of;         // per packed position: phase in which it finishes
    std::vector<int64_t> phase_end;    // step count at the end of each phase
    double elem_steps = 0.0;
    std::vector<void *> allocs;
    double *d_T0 = nullptr;
    unsigned long long *d_stamp = nullptr;  // [0] start, [1 + j] end of phase j
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
};

namespace {

int nblk(int64_t n, int bs = 256)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + bs - 1) / bs, 65535));
}

__global__ void k_stamp(unsigned long long *t)
{
    unsigned long long v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    *t = v;
}

// A_i = dt_i / C0_i with a per-node time step (-0.0 on Dirichlet nodes), plus the float pair.
__global__ void k_set_A_nodes(int64_t nn, const double *dtn, const double *C0, const uint8_t *isdir, double *A,
                              float2 *A2)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        const double v = isdir[g] ? -0.0 : dtn[g] / C0[g];
        A[g] = v;
        if (A2) {
            const float hi = (float)v;
            A2[g] = make_float2(hi, (float)(v - (double)hi));
        }
    }
}

// Fixed-order sum over a block of 256 threads; the result is valid in thread 0.
__device__ double block_sum1(double a, double *red)
{
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// Lanczos steps for the largest eigenvalue of C0^-1/2 K0 C0^-1/2 of every scenario, one block
// per scenario over its node range (vectors zero on Dirichlet nodes): w = C0^-1/2 F -
// beta_{j-1} v_{j-1} written over F and alpha_j = w . v_j; then w -= alpha_j v_j and
// beta_j^2 = w . w; then v_{j+1} = w / beta_j.  Coefficients per scenario: [p].
__global__ void __launch_bounds__(256) k_seg_lz_w(const int64_t *nr, double *F, const double *C0, const uint8_t *isdir,
                                                  const double *vprev, const double *beta2_prev, const double *vcur,
                                                  double *alpha)
{
    __shared__ double red[8];
    const int p = blockIdx.x;
    const double b = beta2_prev ? sqrt(beta2_prev[p]) : 0.0;
    double a = 0.0;
    for (int64_t g = nr[p] + threadIdx.x; g < nr[p + 1]; g += blockDim.x) {
        const double w = isdir[g] ? 0.0 : F[g] / sqrt(C0[g]) - (beta2_prev ? b * vprev[g] : 0.0);
        F[g] = w;
        a += w * vcur[g];
    }
    a = block_sum1(a, red);
    if (threadIdx.x == 0) alpha[p] = a;
}

// w -= alpha_j v_j (alpha == NULL: w unchanged); beta2 = w . w
__global__ void __launch_bounds__(256) k_seg_lz_orth(const int64_t *nr, double *w, const double *vcur,
                                                     const double *alpha, double *beta2)
{
    __shared__ double red[8];
    const int p = blockIdx.x;
    const double al = alpha ? alpha[p] : 0.0;
    double s = 0.0;
    for (int64_t g = nr[p] + threadIdx.x; g < nr[p + 1]; g += blockDim.x) {
        const double x = alpha ? w[g] - al * vcur[g] : w[g];
        if (alpha) w[g] = x;
        s += x * x;
    }
    s = block_sum1(s, red);
    if (threadIdx.x == 0) beta2[p] = s;
}

// v_{j+1} = w / beta_j (zero once beta_j underflows: that scenario's Krylov space is exhausted)
__global__ void __launch_bounds__(256) k_seg_lz_next(const int64_t *nr, const double *w, const double *beta2,
                                                     double *vnext)
{
    const int p = blockIdx.x;
    const double inv = beta2[p] > 1e-280 ? 1.0 / sqrt(beta2[p]) : 0.0;
    for (int64_t g = nr[p] + threadIdx.x; g < nr[p + 1]; g += blockDim.x) vnext[g] = w[g] * inv;
}

// Largest linearised surface rate per scenario (one block each).
__global__ void __launch_bounds__(256) k_seg_surface(const int64_t *nr, const double *Ac, const double *Ar,
                                                     const double *C0, const uint8_t *isdir, const double *coef,
                                                     double *out)
{
    __shared__ double red[8];
    const int p = blockIdx.x;
    const double h = coef[3 * p], rad = coef[3 * p + 1], fcmin = coef[3 * p + 2];
    double m = 0.0;
    for (int64_t g = nr[p] + threadIdx.x; g < nr[p + 1]; g += blockDim.x)
        if (!isdir[g]) m = fmax(m, (Ac[g] * h + Ar[g] * rad) / (C0[g] * fcmin));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        out[p] = m;
    }
}

fedfem_status bfail(fedfem_batch *b, fedfem_status s, const std::string &m)
{
    b->err = m;
    return s;
}

cudaError_t balloc(fedfem_batch *b, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) b->allocs.push_back(*p);
    return e;
}

#define BCK(call, where)                                                              \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return bfail(b, FEDFEM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" void fedfem_batch_destroy(fedfem_batch *b)
{
    if (!b) return;
    if (b->c) cudaStreamSynchronize(b->c->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (void *p : b->allocs) cudaFree(p);
    if (b->c) fedfem_destroy(b->c);
    delete b;
}

static fedfem_status batch_build(fedfem_batch *b, const fedfem_scenario *sc, int32_t S, const fedfem_options *opt)
{
    // ---- validate and order the scenarios (decreasing step count, stable)
    const int npe = sc[0].mesh.nodes_per_elem;
    for (int s = 0; s < S; ++s) {
        if (sc[s].mesh.nodes_per_elem != npe) return bfail(b, FEDFEM_ERR_ARG, "all scenarios must use one element type");
        if (sc[s].n_steps < 1) return bfail(b, FEDFEM_ERR_ARG, "n_steps must be >= 1");
        if (!(sc[s].dt_scale > 0.0)) return bfail(b, FEDFEM_ERR_ARG, "dt_scale must be > 0");
        if (!(sc[s].T_lo <= sc[s].T_hi)) return bfail(b, FEDFEM_ERR_ARG, "T_lo must be <= T_hi");
        if (!sc[s].T0 || !sc[s].mesh.xyz || !sc[s].mesh.conn) return bfail(b, FEDFEM_ERR_ARG, "NULL scenario array");
        if (sc[s].mesh.elem_mat) return bfail(b, FEDFEM_ERR_UNSUPPORTED, "one material per scenario");
    }
    b->S = S;
    b->order.resize(S);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int x, int y) { return sc[x].n_steps > sc[y].n_steps; });
    b->pos.resize(S);
    for (int p = 0; p < S; ++p) b->pos[b->order[p]] = p;

    // ---- pack
    int face_nv = 0;
    for (int s = 0; s < S; ++s)
        if (sc[s].bcs.n_conv_faces + sc[s].bcs.n_rad_faces > 0) {
            if (face_nv && sc[s].bcs.face_nv != face_nv) return bfail(b, FEDFEM_ERR_ARG, "one face size for all scenarios");
            face_nv = sc[s].bcs.face_nv;
        }
    if (!face_nv) face_nv = npe == 8 ? 4 : 3;
    std::vector<double> xyz, kscale, source, nodalQ, dirT, T0;
    std::vector<int32_t> conn, emat, dirn, conv, rad;
    std::vector<fedfem_material> mats(S);
    std::vector<int64_t> group_elem(1, 0);
    b->node_off.assign(1, 0);
    b->steps.resize(S);
    bool any_k = false, any_s = false, any_q = false;
    for (int s = 0; s < S; ++s) {
        any_k |= sc[s].mesh.elem_kscale != nullptr;
        any_s |= sc[s].bcs.elem_source != nullptr;
        any_q |= sc[s].bcs.nodal_Q != nullptr;
    }
    for (int p = 0; p < S; ++p) {
        const fedfem_scenario &q = sc[b->order[p]];
        const int64_t n0 = b->node_off.back(), nn = q.mesh.n_nodes, ne = q.mesh.n_elems;
        xyz.insert(xyz.end(), q.mesh.xyz, q.mesh.xyz + 3 * nn);
        for (int64_t i = 0; i < ne * npe; ++i) {
            if (q.mesh.conn[i] < 0 || q.mesh.conn[i] >= nn) return bfail(b, FEDFEM_ERR_ARG, "connectivity id out of range");
            conn.push_back((int32_t)(q.mesh.conn[i] + n0));
        }
        emat.insert(emat.end(), ne, p);
        mats[p] = q.mat;
        if (any_k) {
            if (q.mesh.elem_kscale)
                kscale.insert(kscale.end(), q.mesh.elem_kscale, q.mesh.elem_kscale + ne);
            else
                kscale.insert(kscale.end(), ne, 1.0);
        }
        if (any_s) {
            if (q.bcs.elem_source)
                source.insert(source.end(), q.bcs.elem_source, q.bcs.elem_source + ne);
            else
                source.insert(source.end(), ne, 0.0);
        }
        if (any_q) {
            if (q.bcs.nodal_Q)
                nodalQ.insert(nodalQ.end(), q.bcs.nodal_Q, q.bcs.nodal_Q + nn);
            else
                nodalQ.insert(nodalQ.end(), nn, 0.0);
        }
        for (int64_t d = 0; d < q.bcs.n_dir; ++d) {
            dirn.push_back((int32_t)(q.bcs.dir_nodes[d] + n0));
            dirT.push_back(q.bcs.dir_T[d]);
        }
        for (int64_t i = 0; i < q.bcs.n_conv_faces * face_nv; ++i) conv.push_back((int32_t)(q.bcs.conv_faces[i] + n0));
        for (int64_t i = 0; i < q.bcs.n_rad_faces * face_nv; ++i) rad.push_back((int32_t)(q.bcs.rad_faces[i] + n0));
        T0.insert(T0.end(), q.T0, q.T0 + nn);
        b->node_off.push_back(n0 + nn);
        group_elem.push_back(group_elem.back() + ne);
        b->steps[p] = q.n_steps;
        b->elem_steps += (double)ne * (double)q.n_steps;
    }
    fedfem_mesh m{};
    m.nodes_per_elem = npe;
    m.n_nodes = b->node_off.back();
    m.n_elems = group_elem.back();
    m.xyz = xyz.data();
    m.conn = conn.data();
    m.elem_mat = emat.data();
    m.elem_kscale = any_k ? kscale.data() : nullptr;
    fedfem_bcs bc{};
    bc.n_dir = (int64_t)dirn.size();
    bc.dir_nodes = dirn.data();
    bc.dir_T = dirT.data();
    bc.n_conv_faces = (int64_t)conv.size() / face_nv;
    bc.conv_faces = conv.data();
    bc.n_rad_faces = (int64_t)rad.size() / face_nv;
    bc.rad_faces = rad.data();
    bc.face_nv = face_nv;
    bc.T_zero = sc[0].bcs.T_zero;
    bc.nodal_Q = any_q ? nodalQ.data() : nullptr;
    bc.elem_source = any_s ? source.data() : nullptr;
    fedfem_status st = create_ctx(&m, mats.data(), S, &bc, opt, &group_elem, &b->c, b->err);
    if (st != FEDFEM_OK) return st;
    fedfem_ctx *c = b->c;
    const int64_t nn = c->nn;

    // ---- per-scenario physics table (packed order)
    std::vector<PhysParams> phys(S);
    for (int p = 0; p < S; ++p) {
        const fedfem_scenario &q = sc[b->order[p]];
        const double Tz = (q.bcs.T_zero == 0.0 && q.bcs.n_rad_faces == 0) ? -273.15 : q.bcs.T_zero;
        phys[p] = PhysParams{q.mat.k_lin, q.mat.c_lin, q.bcs.h, q.bcs.T_inf, q.bcs.eps * 5.67e-8, q.bcs.T_amb, Tz,
                             c->opt.T_guard, 1.0 - q.mat.k_lin * q.mat.T_ref, 1.0 - q.mat.c_lin * q.mat.T_ref};
    }
    BCK(balloc(b, (void **)&c->d_phys, S * sizeof(PhysParams)), "alloc physics");
    BCK(cudaMemcpy(c->d_phys, phys.data(), S * sizeof(PhysParams), cudaMemcpyHostToDevice), "upload physics");

    // ---- pre-computation: element operators, masses, loads, areas
    st = run_precompute_arrays(c);
    if (st != FEDFEM_OK) return bfail(b, st, c->err);
    c->precomputed = true;

    // node ranges (new numbering) of every packed scenario
    std::vector<int64_t> nr(S + 1, nn);
    {
        std::vector<char> seen(S, 0);
        for (int t = 0; t < c->til.n_tiles; ++t) {
            const int g = c->til.tiles[t].scenario;
            if (!seen[g]) {
                seen[g] = 1;
                nr[g] = c->til.tiles[t].node_begin;
            }
        }
        nr[S] = nn;
    }
    int64_t *d_nr = nullptr;
    BCK(balloc(b, (void **)&d_nr, (S + 1) * 8), "alloc");
    BCK(cudaMemcpy(d_nr, nr.data(), (S + 1) * 8, cudaMemcpyHostToDevice), "upload");

    // ---- critical step of every scenario: Lanczos segmented by scenario; the host takes each
    //      scenario's largest tridiagonal eigenvalue every 16 steps until all have converged
    //      (relative change < tol) or exhausted their Krylov space
    double *vcur = c->d_v[0], *vprev = c->d_v[1], *u = c->d_v[2], *F = c->d_v[3];
    double *surf = nullptr, *coef = nullptr, *lz_a = nullptr, *lz_b = nullptr, *norm2 = nullptr;
    const int max_iter = c->power_max_iter;
    BCK(balloc(b, (void **)&surf, S * 8), "alloc");
    BCK(balloc(b, (void **)&coef, 3 * S * 8), "alloc");
    BCK(balloc(b, (void **)&norm2, S * 8), "alloc");
    BCK(balloc(b, (void **)&lz_a, (size_t)max_iter * S * 8), "alloc");
    BCK(balloc(b, (void **)&lz_b, (size_t)max_iter * S * 8), "alloc");
    cudaStream_t stm = c->stream;
    launch_power_init(nn, c->d_isdir, F, stm);
    k_seg_lz_orth<<<S, 256, 0, stm>>>(d_nr, F, nullptr, nullptr, norm2);
    k_seg_lz_next<<<S, 256, 0, stm>>>(d_nr, F, norm2, vcur);
    std::vector<double> lam(S, 0.0), ha, hb, al, b2;
    std::vector<char> lz_done(S, 0);
    for (int it = 0; it < max_iter; ++it) {
        launch_scale_free(nn, vcur, c->d_C0, c->d_isdir, u, stm);
        launch_apply(c->npe, c->ne, nn, c->d_gconn, c->d_cond64, c->d_n2e_ptr, c->d_n2e, u, nullptr, 1.0, 0.0, nullptr, c->d_Y,
                     F, stm);
        k_seg_lz_w<<<S, 256, 0, stm>>>(d_nr, F, c->d_C0, c->d_isdir, vprev, it ? lz_b + (size_t)(it - 1) * S : nullptr,
                                       vcur, lz_a + (size_t)it * S);
        k_seg_lz_orth<<<S, 256, 0, stm>>>(d_nr, F, vcur, lz_a + (size_t)it * S, lz_b + (size_t)it * S);
        k_seg_lz_next<<<S, 256, 0, stm>>>(d_nr, F, lz_b + (size_t)it * S, vprev);
        std::swap(vprev, vcur);  // v_{j+1} was written over v_{j-1}
        if ((it & 15) == 15 || it == max_iter - 1) {
            const size_t m = (size_t)(it + 1);
            ha.resize(m * S);
            hb.resize(m * S);
            BCK(cudaMemcpyAsync(ha.data(), lz_a, m * S * 8, cudaMemcpyDeviceToHost, stm), "read");
            BCK(cudaMemcpyAsync(hb.data(), lz_b, m * S * 8, cudaMemcpyDeviceToHost, stm), "read");
            BCK(cudaStreamSynchronize(stm), "synchronize");
            bool done = true;
            al.resize(m);
            b2.resize(m);
            for (int p = 0; p < S; ++p) {
                if (lz_done[p]) continue;
                for (size_t j = 0; j < m; ++j) {
                    al[j] = ha[j * S + p];
                    b2[j] = hb[j * S + p];
                }
                const double theta = tridiag_max_eigenvalue(al, b2, (int)m);
                const bool exhausted = !(b2[m - 1] > 1e-28 * theta * theta);
                if (exhausted || (it > 16 && std::fabs(theta - lam[p]) <= c->power_tol * std::fabs(theta)))
                    lz_done[p] = 1;
                else
                    done = false;
                lam[p] = theta;
            }
            if (done) break;
        }
    }
    BCK(cudaGetLastError(), "Lanczos");
    std::vector<double> h_coef(3 * S), fk_max(S), fc_min(S);
    for (int p = 0; p < S; ++p) {
        const fedfem_scenario &q = sc[b->order[p]];
        const double r = q.mat.T_ref;
        const double fk_lo = 1.0 + q.mat.k_lin * (q.T_lo - r), fk_hi = 1.0 + q.mat.k_lin * (q.T_hi - r);
        fk_max[p] = std::max(fk_lo, fk_hi);
        fc_min[p] = std::min(1.0 + q.mat.c_lin * (q.T_lo - r), 1.0 + q.mat.c_lin * (q.T_hi - r));
        if (!(std::min(fk_lo, fk_hi) > 0) || !(fc_min[p] > 0))
            return bfail(b, FEDFEM_ERR_ARG, "material law not positive on [T_lo, T_hi]");
        const double rl = std::fabs(q.T_lo - phys[p].T_zero), rh = std::fabs(q.T_hi - phys[p].T_zero);
        h_coef[3 * p] = q.bcs.h;
        h_coef[3 * p + 1] = 4.0 * 5.67e-8 * q.bcs.eps * std::max(rl * rl * rl, rh * rh * rh);
        h_coef[3 * p + 2] = fc_min[p];
    }
    BCK(cudaMemcpyAsync(coef, h_coef.data(), 3 * S * 8, cudaMemcpyHostToDevice, stm), "upload");
    k_seg_surface<<<S, 256, 0, stm>>>(d_nr, c->d_Ac64, c->d_Ar64, c->d_C0, c->d_isdir, coef, surf);
    std::vector<double> h_surf(S);
    BCK(cudaMemcpyAsync(h_surf.data(), surf, S * 8, cudaMemcpyDeviceToHost, stm), "read");
    BCK(cudaStreamSynchronize(stm), "synchronize");
    b->dt.assign(S, 0.0);
    b->dt_crit.assign(S, 0.0);
    std::vector<double> dtn(nn);
    for (int p = 0; p < S; ++p) {
        const int s = b->order[p];
        b->dt_crit[s] = 2.0 / (lam[p] * fk_max[p] / fc_min[p] + h_surf[p]);
        b->dt[s] = sc[s].dt_scale * b->dt_crit[s];
        for (int64_t g = nr[p]; g < nr[p + 1]; ++g) dtn[g] = b->dt[s];
    }
    BCK(cudaMemcpyAsync(c->d_v[1], dtn.data(), nn * 8, cudaMemcpyHostToDevice, stm), "upload");
    k_set_A_nodes<<<nblk(nn), 256, 0, stm>>>(nn, c->d_v[1], c->d_C0, c->d_isdir, c->d_A, c->d_A2);
    BCK(cudaGetLastError(), "time steps");
    c->has_dt = true;
    c->has_T = true;

    // ---- initial states (packed original order)
    BCK(balloc(b, (void **)&b->d_T0, nn * 8), "alloc");
    BCK(cudaMemcpyAsync(b->d_T0, T0.data(), nn * 8, cudaMemcpyHostToDevice, stm), "upload T0");
    BCK(cudaStreamSynchronize(stm), "synchronize");

    // ---- phases: distinct step counts, active tile prefix, balanced CTA ranges
    std::vector<int64_t> distinct(b->steps.begin(), b->steps.end());
    std::sort(distinct.begin(), distinct.end());
    distinct.erase(std::unique(distinct.begin(), distinct.end()), distinct.end());
    const int J = (int)distinct.size();
    b->phase_end = distinct;
    b->phase_of.assign(S, 0);
    for (int p = 0; p < S; ++p)
        b->phase_of[p] = (int)(std::lower_bound(distinct.begin(), distinct.end(), b->steps[p]) - distinct.begin());
    BCK(balloc(b, (void **)&b->d_stamp, (J + 1) * 8), "alloc");
    const int max_ctas = c->grid;  // co-resident CTAs verified by the launch plan
    std::vector<int32_t *> d_ranges(J, nullptr);
    std::vector<int> grids(J, 0);
    for (int j = 0; j < J; ++j) {
        int P = 0;  // active scenarios: packed prefix with steps >= distinct[j]
        while (P < S && b->steps[P] >= distinct[j]) ++P;
        int A = 0;
        while (A < c->til.n_tiles && c->til.tiles[A].scenario < P) ++A;
        const int G = std::max(1, std::min(max_ctas, A));
        double total = 0.0;
        for (int t = 0; t < A; ++t) total += c->til.tiles[t].n_chunks;
        std::vector<int32_t> rg(1, 0);
        double acc = 0.0;
        for (int t = 0; t < A; ++t) {
            acc += c->til.tiles[t].n_chunks;
            const int left_tiles = A - (t + 1), left_ctas = G - (int)rg.size();
            if ((int)rg.size() < G && (acc >= total * rg.size() / G || left_tiles <= left_ctas) && left_tiles >= left_ctas)
                rg.push_back(t + 1);
        }
        if (rg.back() != A) rg.push_back(A);
        grids[j] = (int)rg.size() - 1;
        BCK(balloc(b, (void **)&d_ranges[j], rg.size() * 4), "alloc");
        BCK(cudaMemcpy(d_ranges[j], rg.data(), rg.size() * 4, cudaMemcpyHostToDevice), "upload");
    }

    // ---- capture the whole run in a CUDA graph
    BCK(prepare_step(c->precision, c->kahan, c->npe, c->scatter_mode, 0, c->smem), "kernel attributes");
    StepArgs a = step_args(c);
    const int64_t spl = c->opt.steps_per_launch > 0 ? c->opt.steps_per_launch : 200;
    // capture on a private stream (the legacy default stream cannot be captured); the graph is
    // later launched on the context's stream
    BCK(cudaStreamSynchronize(stm), "synchronize");
    cudaStream_t cap = nullptr;
    BCK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
    b->cap_stream = cap;
    stm = cap;
    BCK(cudaStreamBeginCapture(stm, cudaStreamCaptureModeThreadLocal), "begin capture");
    k_stamp<<<1, 1, 0, stm>>>(b->d_stamp);
    cudaMemcpyAsync(c->d_v[0], b->d_T0, nn * 8, cudaMemcpyDeviceToDevice, stm);
    launch_impose_dirichlet((int64_t)c->dir_nodes.size(), c->d_dir_new, c->d_dir_T, 0.0, c->d_v[0], c->d_old_of_new, stm);
    launch_set_state(c->precision, nn, c->d_v[0], c->d_old_of_new, c->d_T[0], c->kahan ? c->d_comp[0] : nullptr, stm);
    int64_t n = 0;
    // tile progress counters: reset once per replay, then launch j starts from base n
    cudaMemsetAsync(c->d_tile_done, 0, c->til.n_tiles * sizeof(unsigned int), stm);
    for (int j = 0; j < J; ++j) {
        a.cta_tile = d_ranges[j];
        while (n < distinct[j]) {
            const int64_t k = std::min<int64_t>(spl, distinct[j] - n);
            a.n0 = n;
            a.nsteps = (int32_t)k;
            a.progress_base = (uint32_t)n;
            launch_step(a, c->precision, c->kahan, c->npe, 0, grids[j], c->block, c->smem, c->ts_cap, stm);
            n += k;
        }
        k_stamp<<<1, 1, 0, stm>>>(b->d_stamp + 1 + j);
    }
    cudaError_t ce = cudaStreamEndCapture(stm, &b->graph);
    if (ce != cudaSuccess) return bfail(b, FEDFEM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    BCK(cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate");
    c->step = 0;
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_batch_create(const fedfem_scenario *sc, int32_t n_scenarios, const fedfem_options *opt,
                                             fedfem_batch **out)
{
    if (!out) return FEDFEM_ERR_ARG;
    *out = nullptr;
    fedfem_batch *b = new fedfem_batch();
    if (!sc || n_scenarios < 1) {
        b->err = "no scenarios";
        *out = b;  // the caller reads the message, then destroys it
        return FEDFEM_ERR_ARG;
    }
    const fedfem_status st = batch_build(b, sc, n_scenarios, opt);
    *out = b;
    return st;
}

extern "C" fedfem_status fedfem_batch_run(fedfem_batch *b)
{
    if (!b || !b->exec) return b ? bfail(b, FEDFEM_ERR_STATE, "batch not built") : FEDFEM_ERR_ARG;
    fedfem_ctx *c = b->c;
    const cudaError_t e = cudaGraphLaunch(b->exec, c->stream);
    if (e != cudaSuccess) return bfail(b, FEDFEM_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    const fedfem_status st = check_device(c);
    if (st != FEDFEM_OK) return bfail(b, st, c->err);
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_batch_times(fedfem_batch *b, double *t_done_ns, double *elem_steps_total, double *dt)
{
    if (!b || !b->exec) return b ? bfail(b, FEDFEM_ERR_STATE, "batch not built") : FEDFEM_ERR_ARG;
    const int J = (int)b->phase_end.size();
    std::vector<unsigned long long> st(J + 1);
    if (cudaMemcpy(st.data(), b->d_stamp, (J + 1) * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return bfail(b, FEDFEM_ERR_CUDA, "read stamps");
    for (int s = 0; s < b->S; ++s) {
        if (t_done_ns) t_done_ns[s] = (double)(st[1 + b->phase_of[b->pos[s]]] - st[0]);
        if (dt) dt[s] = b->dt[s];
    }
    if (elem_steps_total) *elem_steps_total = b->elem_steps;
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_batch_get_T(fedfem_batch *b, int32_t s, double *T_host)
{
    if (!b || !b->c || s < 0 || s >= b->S || !T_host) return b ? bfail(b, FEDFEM_ERR_ARG, "bad scenario") : FEDFEM_ERR_ARG;
    fedfem_ctx *c = b->c;
    const int p = b->pos[s];
    fedfem_status st = state_f64_new(c, b->steps[p], c->d_v[0]);
    if (st != FEDFEM_OK) return bfail(b, st, c->err);
    launch_permute_new_to_old(c->nn, c->d_v[0], c->d_old_of_new, c->d_v[1], c->stream);
    const int64_t n0 = b->node_off[p], cnt = b->node_off[p + 1] - n0;
    if (cudaMemcpyAsync(T_host, c->d_v[1] + n0, cnt * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return bfail(b, FEDFEM_ERR_CUDA, "download");
    st = check_device(c);
    return st == FEDFEM_OK ? FEDFEM_OK : bfail(b, st, c->err);
}

extern "C" const char *fedfem_batch_error_string(fedfem_batch *b) { return b ? b->err.c_str() : "NULL batch"; }
