// C ABI of libfedfem.so: contexts, the launch plan, the pre-computation stage and the time
// loop of Fig. 1, state transfer and diagnostics.  All arithmetic of the method runs in the
// kernels of step.cu and precompute.cu; this file validates, lays out and orchestrates.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

using namespace fedfem;

static thread_local std::string g_create_error;

// ------------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------------
namespace fedfem {

fedfem_status fail(fedfem_ctx *c, fedfem_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

fedfem_status cuda_fail(fedfem_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, e == cudaErrorMemoryAllocation ? FEDFEM_ERR_OOM : FEDFEM_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

cudaError_t dalloc(fedfem_ctx *c, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) c->allocs.push_back(*p);
    return e;
}

cudaError_t upload(fedfem_ctx *c, void **p, const void *src, size_t bytes)
{
    cudaError_t e = dalloc(c, p, bytes);
    if (e != cudaSuccess) return e;
    if (bytes) e = cudaMemcpyAsync(*p, src, bytes, cudaMemcpyHostToDevice, c->stream);
    return e;
}

}  // namespace fedfem

#define CK(call, where)                                          \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where);   \
    } while (0)

static std::string status_message(int32_t bits)
{
    std::string m;
    if (bits & ERRBIT_DIVERGED) m += "watchdog: a temperature became non-finite or exceeded T_guard; ";
    if (bits & ERRBIT_TIMEOUT) m += "device wait exceeded its limit (neighbouring tiles' progress or a TMA stage); ";
    if (bits & ERRBIT_MESH) m += "element with non-positive Jacobian; ";
    if (bits & ERRBIT_BOUNDS) m += "index out of bounds; ";
    return m;
}

// Read and clear the device error word (synchronises the stream).
fedfem_status fedfem::check_device(fedfem_ctx *c)
{
    int32_t bits = 0;
    CK(cudaMemcpyAsync(&bits, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream), "read status");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    if (bits) {
        CK(cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), c->stream), "clear status");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        // a divergence can leave secondary timeouts behind: report the root cause first
        const fedfem_status s = (bits & ERRBIT_DIVERGED) ? FEDFEM_ERR_DIVERGED
                                : (bits & ERRBIT_MESH)   ? FEDFEM_ERR_MESH
                                                         : FEDFEM_ERR_TIMEOUT;
        return fail(c, s, status_message(bits));
    }
    return FEDFEM_OK;
}

extern "C" void fedfem_default_options(fedfem_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = FEDFEM_FP32;
    o->kahan = 1;
    o->scatter = FEDFEM_SCATTER_COLOR;
    o->barrier_timeout_s = 1.0;
    o->T_guard = 1e6;
    o->device = -1;
}

// ------------------------------------------------------------------------------------------
// create
// ------------------------------------------------------------------------------------------
static std::string validate(const fedfem_mesh *m, const fedfem_material *mats, int32_t n_mats, const fedfem_bcs *b,
                            bool per_material_laws)
{
    if (!m || !mats || !b) return "NULL mesh, materials or bcs";
    if (m->nodes_per_elem != 8 && m->nodes_per_elem != 4) return "nodes_per_elem must be 8 or 4";
    if (m->n_nodes <= 0 || m->n_elems <= 0) return "empty mesh";
    if (m->n_nodes >= (1LL << 31) || m->n_elems >= (1LL << 31)) return "mesh too large for int32 ids";
    if (!m->xyz || !m->conn) return "NULL xyz or conn";
    if (n_mats < 1) return "n_mats must be >= 1";
    const int npe = m->nodes_per_elem;
    for (int64_t i = 0; i < m->n_elems * npe; ++i)
        if (m->conn[i] < 0 || m->conn[i] >= m->n_nodes) return "connectivity id out of range at " + std::to_string(i);
    for (int64_t i = 0; i < m->n_nodes * 3; ++i)
        if (!std::isfinite(m->xyz[i])) return "non-finite coordinate";
    if (m->elem_mat)
        for (int64_t e = 0; e < m->n_elems; ++e)
            if (m->elem_mat[e] < 0 || m->elem_mat[e] >= n_mats) return "elem_mat out of range";
    if (m->elem_kscale)
        for (int64_t e = 0; e < m->n_elems; ++e)
            if (!(m->elem_kscale[e] > 0) || !std::isfinite(m->elem_kscale[e])) return "elem_kscale must be > 0";
    for (int i = 0; i < n_mats; ++i) {
        if (!(mats[i].rho > 0) || !(mats[i].c0 > 0)) return "rho and c0 must be > 0";
        if (!per_material_laws &&
            (mats[i].k_lin != mats[0].k_lin || mats[i].c_lin != mats[0].c_lin || mats[i].T_ref != mats[0].T_ref))
            return "all materials must share k_lin, c_lin and T_ref";
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s)
                if (mats[i].k0[3 * r + s] != mats[i].k0[3 * s + r]) return "k0 must be symmetric";
    }
    if (b->n_dir < 0 || b->n_conv_faces < 0 || b->n_rad_faces < 0) return "negative boundary counts";
    if (b->n_dir > 0 && (!b->dir_nodes || !b->dir_T)) return "NULL Dirichlet arrays";
    for (int64_t d = 0; d < b->n_dir; ++d)
        if (b->dir_nodes[d] < 0 || b->dir_nodes[d] >= m->n_nodes) return "Dirichlet node out of range";
    const int64_t nf = b->n_conv_faces + b->n_rad_faces;
    if (nf > 0 && b->face_nv != 3 && b->face_nv != 4) return "face_nv must be 3 or 4";
    for (int pass = 0; pass < 2; ++pass) {
        const int64_t n = pass ? b->n_rad_faces : b->n_conv_faces;
        const int32_t *f = pass ? b->rad_faces : b->conv_faces;
        if (n > 0 && !f) return "NULL face array";
        for (int64_t i = 0; i < n * b->face_nv; ++i)
            if (f[i] < 0 || f[i] >= m->n_nodes) return "face node out of range";
    }
    return "";
}

// Elements per chunk: 64 for FP32 tets (two per lane: 64^3 6-tet cube 38.2 -> 35.5 us/step,
// paper-shaped cube 9.15 -> 8.74; the ring depth barely matters there, 38.2 -> 37.4 us from 16
// to 63 stages), else 32 (64^3 hex 18.9 -> 21.7 us/step with 64: fewer stages fit).
static int default_chunk(int precision, int npe)
{
    return precision == 32 && npe == 4 ? 64 : 32;
}

// Shared memory for the element-load slots up to which the default plan takes the slot gather.
static constexpr size_t kSlotBudget = 48 * 1024;

// Deepest element ring the plan tries when the stage count is not given.
static constexpr int kMaxAutoStages = 16;

// Choose tiles, grid, chunking and shared memory; builds c->til.
static fedfem_status make_plan(fedfem_ctx *c, const std::vector<uint8_t> &is_bnd)
{
    const int npe = c->npe;
    // consumer threads per CTA (one producer warp is added at launch); the FP32 default runs
    // two CTAs of 7 consumer warps + 1 producer warp per SM (16 warps, 128 registers each).
    // FP32 hexahedral meshes whose element stream stays in L2 (at most 64 MB) run one CTA of 15
    // consumer warps per SM instead, on tiles twice as large, with fewer halo nodes per element
    // (64^3 hex cube: 16.8 -> 16.4 us/step; the 64^3 tet cube is slower that way, 24.3 ->
    // 32.7, and so is the 128^3 cube, whose node phases then leave the SM's DRAM stream idle)
    const bool small_hex = c->precision == 32 && npe == 8 && c->group_elem.empty() && !c->opt.block &&
                           !c->opt.ctas_per_sm &&
                           (int64_t)c->ne * chunk_bytes_for(32, 8, 32) / 32 <= (64LL << 20);
    const int block = c->opt.block ? c->opt.block : (c->precision == 64 ? 256 : small_hex ? 480 : 224);
    if (block % 32 || block < 64 || block > 480) return fail(c, FEDFEM_ERR_ARG, "block must be a multiple of 32 in [64, 480]");
    const int chunk = c->opt.chunk ? c->opt.chunk : default_chunk(c->precision, npe);
    if (chunk != 32 && chunk != 64) return fail(c, FEDFEM_ERR_ARG, "chunk must be 32 or 64");
    // two CTAs per SM only while (block + 32) threads x 128 registers fit twice per SM
    const int cps = c->opt.ctas_per_sm ? c->opt.ctas_per_sm : (c->precision == 32 && block <= 224 ? 2 : 1);
    if (c->opt.stages && (c->opt.stages < 2 || c->opt.stages > 63))
        return fail(c, FEDFEM_ERR_ARG, "stages must be in [2, 63]");
    // default ring depth: the deepest ring (at most kMaxAutoStages) that keeps cps CTAs per SM;
    // the element stream runs faster with more bytes in flight (128^3 hex, 2 CTAs/SM:
    // 6 stages 76.4 us/step, 9 -> 72.9, 11 -> 72.1)
    int stages = c->opt.stages ? c->opt.stages : kMaxAutoStages;
    int tpc = c->opt.tiles_per_cta ? c->opt.tiles_per_cta : 1;
    const int cb = chunk_bytes_for(c->precision, npe, chunk);
    for (int attempt = 0; attempt < 12; ++attempt) {
        const int64_t n_ctas = (int64_t)c->num_sms * cps;
        int64_t n_tiles = n_ctas * tpc;
        n_tiles = std::min<int64_t>(n_tiles, std::max<int64_t>(1, c->ne / block));
        int grid = (int)((n_tiles + tpc - 1) / tpc);
        std::string e;
        // accumulation: the slot gather when forced; by default when the colour classes pad
        // the tiles to at least 1.5 times the chunks their elements need (many small classes:
        // each class costs a barrier and a padded chunk) and a tile's element loads fit in 48 KB
        bool slots = c->group_elem.empty() && !c->opt.energy_audit && c->opt.scatter == FEDFEM_SCATTER_SLOTS;
        if (c->group_elem.empty()) {
            e = build_tiling(npe, c->ne, c->nn, c->conn.data(), c->xyz.data(), is_bnd.data(), (int)n_tiles, chunk,
                             c->til, slots);
            if (e.empty() && !slots && c->opt.scatter == FEDFEM_SCATTER_COLOR && !c->opt.energy_audit) {
                int64_t need = 0;
                int max_need = 0;
                for (const TileInfo &ti : c->til.tiles) {
                    int64_t m = 0;
                    for (int u = 0; u < ti.n_chunks; ++u)
                        for (int l = 0; l < chunk; ++l)
                            if (c->til.elem_col[(size_t)(ti.chunk_begin + u) * chunk + l] != 0xFF) ++m;
                    const int nc = (int)((m + chunk - 1) / chunk);
                    need += nc;
                    max_need = std::max(max_need, nc);
                }
                const size_t rs_ = c->precision == 64 ? 8 : 4;
                if (2 * (int64_t)c->til.n_chunks >= 3 * need && (size_t)max_need * chunk * npe * rs_ <= kSlotBudget) {
                    slots = true;
                    e = build_tiling(npe, c->ne, c->nn, c->conn.data(), c->xyz.data(), is_bnd.data(), (int)n_tiles,
                                     chunk, c->til, true);
                }
            }
        } else {
            // batched scenarios: tiles of about ne / n_tiles elements, never spanning two scenarios
            const int64_t te = std::max<int64_t>(block, (c->ne + n_tiles - 1) / n_tiles);
            std::vector<int> per;
            for (size_t g = 0; g + 1 < c->group_elem.size(); ++g)
                per.push_back((int)((c->group_elem[g + 1] - c->group_elem[g] + te - 1) / te));
            e = build_tiling_groups(npe, c->ne, c->nn, c->conn.data(), c->xyz.data(), is_bnd.data(), c->group_elem,
                                    per, chunk, c->til);
            grid = (int)std::min<int64_t>(n_ctas, c->til.n_tiles);
        }
        c->scatter_mode = c->opt.scatter == FEDFEM_SCATTER_ATOMIC ? FEDFEM_SCATTER_ATOMIC
                          : slots                                 ? FEDFEM_SCATTER_SLOTS
                                                                  : FEDFEM_SCATTER_COLOR;
        if (!e.empty()) {
            if (e.find("65535") != std::string::npos) {
                tpc *= 2;
                continue;
            }
            return fail(c, FEDFEM_ERR_MESH, e);
        }
        e = validate_tiling(c->til);
        if (!e.empty()) return fail(c, FEDFEM_ERR_MESH, "tiling check failed: " + e);
        // fewer stages before smaller tiles, unless the stage count was given
        int st = stages;
        const int slot_cap = slots ? c->til.max_chunks * chunk : 0;
        size_t smem = step_smem_bytes(c->precision, npe, chunk, st, c->til.max_local, slot_cap);
        auto fits = [&](size_t sm) {
            return sm <= (size_t)c->max_smem && step_max_blocks_per_sm(c->precision, c->kahan, npe, block, sm) >= cps;
        };
        while (!c->opt.stages && st > 4 && !fits(smem)) {
            --st;
            smem = step_smem_bytes(c->precision, npe, chunk, st, c->til.max_local, slot_cap);
        }
        int nb = 0;
        if (smem <= (size_t)c->max_smem) nb = step_max_blocks_per_sm(c->precision, c->kahan, npe, block, smem);
        if (nb >= cps && nb * c->num_sms >= grid) {
            c->block = block;
            c->chunk = chunk;
            c->stages = st;
            c->tpc = tpc;
            c->grid = grid;
            c->smem = smem;
            c->chunk_bytes = cb;
            c->ts_cap = step_ts_cap(c->precision, c->til.max_local);
            // start stagger (off unless given: measured neutral on the 128^3 cube)
            c->stagger_ns = c->opt.start_stagger_us > 0 ? (long long)(std::min(c->opt.start_stagger_us, 1000.0) * 1e3) : 0;
            if (c->opt.verbose)
                std::fprintf(stderr,
                             "fedfem plan: tiles=%d grid=%d block=%d chunk=%d stages=%d tpc=%d max_local=%d "
                             "colours=%d smem=%zu chunks=%d\n",
                             c->til.n_tiles, grid, block, chunk, st, tpc, c->til.max_local, c->til.max_colors, smem,
                             c->til.n_chunks);
            return FEDFEM_OK;
        }
        tpc *= 2;
    }
    return fail(c, FEDFEM_ERR_UNSUPPORTED, "no launch plan fits in shared memory");
}

namespace fedfem {

// Largest eigenvalue of the m x m symmetric tridiagonal matrix with diagonal a and squared
// off-diagonal b2 (b2[i] couples rows i and i + 1) by bisection on the Sturm count of the
// LDL^T pivots (number of eigenvalues below x).
double tridiag_max_eigenvalue(const std::vector<double> &a, const std::vector<double> &b2, int m)
{
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; ++i) {
        const double r = (i > 0 ? std::sqrt(b2[i - 1]) : 0.0) + (i + 1 < m ? std::sqrt(b2[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    const double pad = 1e-12 * std::max(std::fabs(lo), std::fabs(hi)) + 1e-300;
    lo -= pad;
    hi += pad;
    auto below = [&](double x) {
        int n = 0;
        double d = 1.0;
        for (int i = 0; i < m; ++i) {
            d = (a[i] - x) - (i > 0 ? b2[i - 1] / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0.0) ++n;
        }
        return n;
    };
    for (int k = 0; k < 200 && hi - lo > 1e-15 * std::max(std::fabs(hi), std::fabs(lo)); ++k) {
        const double mid = 0.5 * (lo + hi);
        if (below(mid) >= m)
            hi = mid;
        else
            lo = mid;
    }
    return hi;
}

}  // namespace fedfem

namespace fedfem {

// Host copy of the problem and device set-up; group_elem (optional) packs independent meshes
// (batched scenarios) whose tiles must not mix.
fedfem_status create_ctx(const fedfem_mesh *mesh, const fedfem_material *mats, int32_t n_mats, const fedfem_bcs *bcs,
                         const fedfem_options *opt_in, const std::vector<int64_t> *group_elem, fedfem_ctx **out,
                         std::string &err)
{
    *out = nullptr;
    std::string v = validate(mesh, mats, n_mats, bcs, group_elem != nullptr);
    if (!v.empty()) {
        err = v;
        return FEDFEM_ERR_ARG;
    }
    fedfem_ctx *c = new fedfem_ctx();
    fedfem_options o;
    fedfem_default_options(&o);
    if (opt_in) {
        o = *opt_in;
        if (o.precision == 0) o.precision = FEDFEM_FP32;
        if (o.barrier_timeout_s <= 0) o.barrier_timeout_s = 1.0;
        if (o.T_guard <= 0) o.T_guard = 1e6;
    }
    if (o.precision != 32 && o.precision != 64) {
        err = "precision must be 32 or 64";
        delete c;
        return FEDFEM_ERR_ARG;
    }
    if (o.quadrature != 0 && o.quadrature != 1 && o.quadrature != 8) {
        err = "quadrature must be 0, 1 or 8";
        delete c;
        return FEDFEM_ERR_ARG;
    }
    if (o.scatter < FEDFEM_SCATTER_COLOR || o.scatter > FEDFEM_SCATTER_CLASSES) {
        err = "scatter must be FEDFEM_SCATTER_COLOR, _ATOMIC, _SLOTS or _CLASSES";
        delete c;
        return FEDFEM_ERR_ARG;
    }
    if ((o.kT_eval != 0 && o.kT_eval != 1) || (o.face_quadrature != 0 && o.face_quadrature != 1)) {
        err = "kT_eval and face_quadrature must be 0 or 1";
        delete c;
        return FEDFEM_ERR_ARG;
    }
    if (group_elem && (o.kT_eval || o.face_quadrature)) {
        err = "batched scenarios run the persistent kernel only: kT_eval and face_quadrature must be 0";
        delete c;
        return FEDFEM_ERR_UNSUPPORTED;
    }
    c->kT_qp = o.kT_eval;
    c->face_cons = o.face_quadrature;
    if (o.energy_audit && (o.kT_eval || o.face_quadrature || group_elem || o.scatter == FEDFEM_SCATTER_ATOMIC ||
                           o.scatter == FEDFEM_SCATTER_SLOTS ||
                           (o.precision == 32 && !o.kahan))) {
        err = "energy_audit needs the persistent kernel with colour scatter and FP32 + Kahan or FP64";
        delete c;
        return FEDFEM_ERR_UNSUPPORTED;
    }
    c->opt = o;
    c->precision = o.precision;
    c->kahan = (o.precision == 32 && o.kahan) ? 1 : 0;
    c->npe = mesh->nodes_per_elem;
    c->nn = mesh->n_nodes;
    c->ne = mesh->n_elems;
    if (group_elem) c->group_elem = *group_elem;
    const int npe = c->npe;
    c->xyz.assign(mesh->xyz, mesh->xyz + 3 * c->nn);
    c->conn.assign(mesh->conn, mesh->conn + npe * c->ne);
    if (mesh->elem_mat) c->elem_mat.assign(mesh->elem_mat, mesh->elem_mat + c->ne);
    c->kscale.assign(c->ne, 1.0);
    if (mesh->elem_kscale) c->kscale.assign(mesh->elem_kscale, mesh->elem_kscale + c->ne);
    if (bcs->elem_source) c->source.assign(bcs->elem_source, bcs->elem_source + c->ne);
    if (bcs->nodal_Q) c->nodal_Q.assign(bcs->nodal_Q, bcs->nodal_Q + c->nn);
    c->mats.assign(mats, mats + n_mats);
    c->k_lin = mats[0].k_lin;
    c->c_lin = mats[0].c_lin;
    c->T_ref = mats[0].T_ref;
    c->dir_nodes.assign(bcs->dir_nodes, bcs->dir_nodes + bcs->n_dir);
    c->dir_T.assign(bcs->dir_T, bcs->dir_T + bcs->n_dir);
    c->face_nv = bcs->face_nv ? bcs->face_nv : (npe == 8 ? 4 : 3);
    c->n_conv = bcs->n_conv_faces;
    c->n_rad = bcs->n_rad_faces;
    if (c->n_conv) c->conv_faces.assign(bcs->conv_faces, bcs->conv_faces + c->n_conv * c->face_nv);
    if (c->n_rad) c->rad_faces.assign(bcs->rad_faces, bcs->rad_faces + c->n_rad * c->face_nv);
    c->h = bcs->h;
    c->T_inf = bcs->T_inf;
    c->eps = bcs->eps;
    c->T_amb = bcs->T_amb;
    c->T_zero = (bcs->T_zero == 0.0 && bcs->n_rad_faces == 0) ? -273.15 : bcs->T_zero;

    fedfem_status st = fedfem_ctx_init_device(c);
    if (st != FEDFEM_OK) {
        err = c->err;
        fedfem_destroy(c);
        return st;
    }
    *out = c;
    return FEDFEM_OK;
}

}  // namespace fedfem

extern "C" fedfem_status fedfem_create(const fedfem_mesh *mesh, const fedfem_material *mats, int32_t n_mats,
                                       const fedfem_bcs *bcs, const fedfem_options *opt_in, fedfem_ctx **out)
{
    if (!out) return FEDFEM_ERR_ARG;
    g_create_error.clear();
    return create_ctx(mesh, mats, n_mats, bcs, opt_in, nullptr, out, g_create_error);
}

namespace fedfem {

fedfem_status fedfem_ctx_init_device(fedfem_ctx *c)
{
    if (c->opt.device >= 0) CK(cudaSetDevice(c->opt.device), "cudaSetDevice");
    CK(cudaGetDevice(&c->device), "cudaGetDevice");
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, c->device), "cudaGetDeviceProperties");
    c->num_sms = prop.multiProcessorCount;
    c->max_smem = (int)prop.sharedMemPerBlockOptin;
    if (!prop.cooperativeLaunch) return fail(c, FEDFEM_ERR_UNSUPPORTED, "device lacks cooperative launch");
    c->stream = (cudaStream_t)c->opt.stream;

    // boundary node flags (nodes with surface loads) for the tiling
    std::vector<uint8_t> is_bnd(c->nn, 0);
    for (int32_t v : c->conv_faces) is_bnd[v] = 1;
    for (int32_t v : c->rad_faces) is_bnd[v] = 1;
    fedfem_status s = make_plan(c, is_bnd);
    if (s != FEDFEM_OK) return s;
    const Tiling &T = c->til;
    const int64_t nn = c->nn, ne = c->ne;
    const int npe = c->npe;
    const size_t rs = c->precision == 64 ? 8 : 4;

    // element stream: tile-local ids, colours and chunk headers (the conductances are filled
    // in by the pre-computation)
    {
        const int CH = c->chunk;
        std::vector<uint8_t> host((size_t)T.n_chunks * c->chunk_bytes, 0);
        const size_t id_off = (size_t)n_pairs(npe) * rs * CH;
        const size_t col_off = chunk_colour_offset(c->precision, npe, CH);
        const size_t hdr_off = chunk_header_offset(c->precision, npe, CH);
        for (int64_t ch = 0; ch < T.n_chunks; ++ch) {
            uint8_t *blk = host.data() + ch * c->chunk_bytes;
            std::memcpy(blk + id_off, T.lconn.data() + (size_t)ch * CH * npe, (size_t)CH * npe * 2);
            std::memcpy(blk + col_off, T.elem_col.data() + (size_t)ch * CH, CH);
            blk[hdr_off] = T.chunk_col[2 * ch];
            blk[hdr_off + 1] = T.chunk_col[2 * ch + 1];
        }
        CK(upload(c, (void **)&c->d_chunks, host.data(), host.size()), "upload element stream");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
    }
    CK(upload(c, (void **)&c->d_tiles, T.tiles.data(), T.tiles.size() * sizeof(TileInfo)), "upload tiles");
    CK(upload(c, (void **)&c->d_sh, T.sh.data(), T.sh.size() * sizeof(int4)), "upload halo");
    CK(upload(c, (void **)&c->d_sptr, T.sptr.data(), T.sptr.size() * sizeof(int32_t)), "upload halo ptr");
    CK(upload(c, (void **)&c->d_bnd, T.bnd.data(), T.bnd.size() * sizeof(int2)), "upload boundary");
    CK(dalloc(c, &c->d_bnd_area, std::max<size_t>(T.bnd.size(), 1) * 2 * (c->precision == 64 ? 8 : 4)),
       "alloc boundary areas");
    CK(upload(c, (void **)&c->d_colptr, T.colptr.data(), T.colptr.size() * sizeof(int32_t)), "upload colours");
    if (T.single_class) {
        CK(upload(c, (void **)&c->d_gptr, T.gptr.data(), T.gptr.size() * sizeof(int32_t)), "upload gather lists");
        CK(upload(c, (void **)&c->d_gidx, T.gidx.data(), T.gidx.size() * sizeof(int32_t)), "upload gather lists");
    }
    CK(upload(c, (void **)&c->d_nbr_ptr, T.nbr_ptr.data(), T.nbr_ptr.size() * sizeof(int32_t)), "upload neighbours");
    CK(upload(c, (void **)&c->d_nbr, T.nbr.data(), T.nbr.size() * sizeof(int32_t)), "upload neighbours");
    CK(dalloc(c, (void **)&c->d_tile_done, (T.n_tiles + 16) * sizeof(unsigned int)), "alloc tile progress");
    CK(cudaMemsetAsync(c->d_tile_done, 0, (T.n_tiles + 16) * sizeof(unsigned int), c->stream), "memset");
    c->progress_base = 0;
    const size_t n_slots = T.sptr.empty() ? 0 : (size_t)T.sptr.back();
    for (int b = 0; b < 2; ++b) {
        CK(dalloc(c, &c->d_T[b], (nn + NODE_PAD) * rs), "alloc T");
        CK(cudaMemsetAsync(c->d_T[b], 0, (nn + NODE_PAD) * rs, c->stream), "memset");
        CK(dalloc(c, &c->d_part[b], std::max<size_t>(n_slots, 1) * rs), "alloc halo partials");
        if (c->kahan) {
            CK(dalloc(c, (void **)&c->d_comp[b], (nn + NODE_PAD) * sizeof(float)), "alloc comp");
            CK(cudaMemsetAsync(c->d_comp[b], 0, (nn + NODE_PAD) * sizeof(float), c->stream), "memset");
        }
    }
    CK(dalloc(c, (void **)&c->d_A, (nn + NODE_PAD) * 8), "alloc A");
    CK(cudaMemsetAsync(c->d_A, 0, (nn + NODE_PAD) * 8, c->stream), "memset");
    if (c->precision == 32) {
        CK(dalloc(c, (void **)&c->d_A2, (nn + NODE_PAD) * 8), "alloc A2");
        CK(cudaMemsetAsync(c->d_A2, 0, (nn + NODE_PAD) * 8, c->stream), "memset");
    }
    CK(dalloc(c, (void **)&c->d_C0, nn * 8), "alloc C0");
    CK(dalloc(c, (void **)&c->d_Qext64, (nn + NODE_PAD) * 8), "alloc Q");
    CK(dalloc(c, (void **)&c->d_Ac64, nn * 8), "alloc Ac");
    CK(dalloc(c, (void **)&c->d_Ar64, nn * 8), "alloc Ar");
    if (c->precision == 32) {
        CK(dalloc(c, &c->d_Qext, (nn + NODE_PAD) * 4), "alloc Q32");
        CK(dalloc(c, &c->d_Ac, nn * 4), "alloc Ac32");
        CK(dalloc(c, &c->d_Ar, nn * 4), "alloc Ar32");
    } else {
        c->d_Qext = c->d_Qext64;
        c->d_Ac = c->d_Ac64;
        c->d_Ar = c->d_Ar64;
    }
    {
        const PhysParams ph{c->k_lin, c->c_lin, c->h,      c->T_inf, c->eps * 5.67e-8, c->T_amb, c->T_zero,
                            c->opt.T_guard, c->k_a(), c->c_a()};
        CK(upload(c, (void **)&c->d_phys, &ph, sizeof(ph)), "upload physics");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
    }
    if (c->opt.energy_audit) {
        CK(dalloc(c, (void **)&c->d_energy_acc, 2 * (size_t)c->grid * 8), "alloc energy sums");
        CK(cudaMemsetAsync(c->d_energy_acc, 0, 2 * (size_t)c->grid * 8, c->stream), "memset");
    }
    CK(dalloc(c, (void **)&c->d_err, 64), "alloc status");
    CK(cudaMemsetAsync(c->d_err, 0, 64, c->stream), "memset");
    CK(dalloc(c, (void **)&c->d_bad_elem, 8), "alloc");

    // pre-computation inputs
    std::vector<uint8_t> isdir(nn, 0);
    std::vector<int32_t> dir_new(c->dir_nodes.size());
    for (size_t d = 0; d < c->dir_nodes.size(); ++d) {
        isdir[T.new_of_old[c->dir_nodes[d]]] = 1;
        dir_new[d] = T.new_of_old[c->dir_nodes[d]];
    }
    CK(upload(c, (void **)&c->d_isdir, isdir.data(), nn), "upload isdir");
    CK(upload(c, (void **)&c->d_dir_new, dir_new.data(), dir_new.size() * 4), "upload dir");
    CK(upload(c, (void **)&c->d_dir_T, c->dir_T.data(), c->dir_T.size() * 8), "upload dir T");
    CK(upload(c, (void **)&c->d_xyz, c->xyz.data(), c->xyz.size() * 8), "upload xyz");
    CK(upload(c, (void **)&c->d_conn, c->conn.data(), c->conn.size() * 4), "upload conn");
    {
        std::vector<int32_t> g(c->conn.size());
        for (size_t i = 0; i < g.size(); ++i) g[i] = T.new_of_old[c->conn[i]];
        CK(upload(c, (void **)&c->d_gconn, g.data(), g.size() * 4), "upload gconn");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
    }
    if (!c->elem_mat.empty()) CK(upload(c, (void **)&c->d_mat, c->elem_mat.data(), ne * 4), "upload mat");
    {
        std::vector<double> k0(9 * c->mats.size()), rhoc(c->mats.size());
        for (size_t m = 0; m < c->mats.size(); ++m) {
            std::memcpy(&k0[9 * m], c->mats[m].k0, 9 * 8);
            rhoc[m] = c->mats[m].rho * c->mats[m].c0;
        }
        CK(upload(c, (void **)&c->d_matk0, k0.data(), k0.size() * 8), "upload k0");
        CK(upload(c, (void **)&c->d_matrhoc, rhoc.data(), rhoc.size() * 8), "upload rho c");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
    }
    CK(dalloc(c, (void **)&c->d_kscale, ne * 8), "alloc kscale");
    CK(dalloc(c, (void **)&c->d_source, ne * 8), "alloc source");
    CK(cudaMemsetAsync(c->d_source, 0, ne * 8, c->stream), "memset");
    if (!c->nodal_Q.empty()) CK(upload(c, (void **)&c->d_nodalQ, c->nodal_Q.data(), nn * 8), "upload nodal Q");
    CK(upload(c, (void **)&c->d_slot_of_elem, T.slot_of_elem.data(), ne * 8), "upload slots");
    CK(upload(c, (void **)&c->d_old_of_new, T.old_of_new.data(), nn * 4), "upload perm");
    CK(upload(c, (void **)&c->d_n2e_ptr, T.n2e_ptr.data(), (nn + 1) * 4), "upload n2e");
    CK(upload(c, (void **)&c->d_n2e, T.n2e.data(), T.n2e.size() * 8), "upload n2e");
    CK(dalloc(c, (void **)&c->d_cond64, (size_t)ne * n_pairs(npe) * 8), "alloc cond64");
    CK(dalloc(c, (void **)&c->d_W, (size_t)ne * npe * 8), "alloc W");
    for (int pass = 0; pass < 2; ++pass) {
        const int64_t nf = pass ? c->n_rad : c->n_conv;
        const std::vector<int32_t> &faces = pass ? c->rad_faces : c->conv_faces;
        std::vector<int32_t> ptr, idx;
        build_face_csr(nn, T.new_of_old, faces.data(), nf, c->face_nv, ptr, idx);
        int32_t **dp = pass ? &c->d_fr_ptr : &c->d_fc_ptr;
        int32_t **di = pass ? &c->d_fr_idx : &c->d_fc_idx;
        int32_t **df = pass ? &c->d_rad_faces : &c->d_conv_faces;
        double **ds = pass ? &c->d_fr_share : &c->d_fc_share;
        CK(upload(c, (void **)dp, ptr.data(), ptr.size() * 4), "upload face csr");
        CK(upload(c, (void **)di, idx.data(), idx.size() * 4), "upload face csr");
        CK(upload(c, (void **)df, faces.data(), faces.size() * 4), "upload faces");
        CK(dalloc(c, (void **)ds, std::max<int64_t>(nf, 1) * 8), "alloc face share");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
    }
    // FP64 scratch for power iteration / energy / state I/O
    for (int i = 0; i < 4; ++i) CK(dalloc(c, (void **)&c->d_v[i], nn * 8), "alloc scratch");
    CK(dalloc(c, (void **)&c->d_Y, (size_t)ne * npe * 8), "alloc scratch");
    CK(dalloc(c, (void **)&c->d_red, 2 * 1024 * 8 + 64), "alloc scratch");
    CK(dalloc(c, (void **)&c->d_lz, 4 * (size_t)c->power_max_iter * 8), "alloc Lanczos coefficients");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    if (c->variant()) return variant_init(c);
    return FEDFEM_OK;
}

}  // namespace fedfem

// ------------------------------------------------------------------------------------------
// pre-computation
// ------------------------------------------------------------------------------------------
fedfem_status fedfem::run_precompute_arrays(fedfem_ctx *c)
{
    const int npe = c->npe;
    if (!c->params_on_device) {
        CK(cudaMemcpyAsync(c->d_kscale, c->kscale.data(), c->ne * 8, cudaMemcpyHostToDevice, c->stream), "upload kscale");
        if (!c->source.empty())
            CK(cudaMemcpyAsync(c->d_source, c->source.data(), c->ne * 8, cudaMemcpyHostToDevice, c->stream),
               "upload source");
    }
    unsigned long long big = ~0ULL;
    CK(cudaMemcpyAsync(c->d_bad_elem, &big, 8, cudaMemcpyHostToDevice, c->stream), "init");
    ElemArgs ea;
    ea.ne = c->ne;
    ea.xyz = c->d_xyz;
    ea.conn = c->d_conn;
    ea.mat = c->d_mat;
    ea.mat_k0 = c->d_matk0;
    ea.kscale = c->d_kscale;
    ea.slot_of_elem = c->d_slot_of_elem;
    ea.CH = c->chunk;
    ea.VW = (c->precision == 32 && npe == 8) ? 4 : 2;
    ea.precision = c->precision;
    ea.chunk_bytes = c->chunk_bytes;
    ea.chunks = c->d_chunks;
    ea.cond64 = c->d_cond64;
    ea.W = c->d_W;
    ea.quad = c->opt.quadrature == 1 ? 1 : 8;
    ea.cond_qp = c->nq == 8 ? c->d_cond_qp64 : nullptr;
    ea.err = c->d_err;
    ea.bad_elem = c->d_bad_elem;
    launch_elem(npe, ea, c->stream);
    CK(cudaGetLastError(), "element pre-computation");
    launch_face_share(c->n_conv, c->face_nv, c->d_conv_faces, c->d_xyz, c->d_fc_share, c->stream);
    launch_face_share(c->n_rad, c->face_nv, c->d_rad_faces, c->d_xyz, c->d_fr_share, c->stream);
    NodeArgs na;
    na.nn = c->nn;
    na.npe = npe;
    na.n2e_ptr = c->d_n2e_ptr;
    na.n2e = c->d_n2e;
    na.W = c->d_W;
    na.mat = c->d_mat;
    na.mat_rhoc = c->d_matrhoc;
    na.source = (c->source.empty() && !c->params_on_device) ? nullptr : c->d_source;
    na.nodal_Q = c->d_nodalQ;
    na.old_of_new = c->d_old_of_new;
    na.fc_ptr = c->n_conv ? c->d_fc_ptr : nullptr;
    na.fc_idx = c->d_fc_idx;
    na.fr_ptr = c->n_rad ? c->d_fr_ptr : nullptr;
    na.fr_idx = c->d_fr_idx;
    na.fc_share = c->d_fc_share;
    na.fr_share = c->d_fr_share;
    na.C0 = c->d_C0;
    na.Qext64 = c->d_Qext64;
    na.Ac64 = c->d_Ac64;
    na.Ar64 = c->d_Ar64;
    na.Qext32 = c->precision == 32 ? (float *)c->d_Qext : nullptr;
    na.Ac32 = c->precision == 32 ? (float *)c->d_Ac : nullptr;
    na.Ar32 = c->precision == 32 ? (float *)c->d_Ar : nullptr;
    launch_node_sums(na, c->stream);
    if (!c->til.bnd.empty())
        CK(launch_bnd_areas(c->precision, (int64_t)c->til.bnd.size(), c->d_bnd, c->d_Ac, c->d_Ar, c->d_bnd_area,
                            c->stream),
           "boundary areas");    CK(cudaGetLastError(), "node pre-computation");
    int32_t bits = 0;
    unsigned long long bad = 0;
    CK(cudaMemcpyAsync(&bits, c->d_err, 4, cudaMemcpyDeviceToHost, c->stream), "read status");
    CK(cudaMemcpyAsync(&bad, c->d_bad_elem, 8, cudaMemcpyDeviceToHost, c->stream), "read status");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    if (bits & ERRBIT_MESH) {
        CK(cudaMemsetAsync(c->d_err, 0, 4, c->stream), "clear");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        return fail(c, FEDFEM_ERR_MESH, "element " + std::to_string(bad) + " has det J <= 0 (inverted or degenerate)");
    }
    if (c->variant()) {
        const fedfem_status vs = variant_precompute(c);
        if (vs != FEDFEM_OK) return vs;
    }
    if (c->has_dt) launch_set_A(c->nn, c->dt, c->d_C0, c->d_isdir, c->d_A, c->d_A2, c->stream);
    return FEDFEM_OK;
}

// dt_crit of Section 3.4 over [T_lo, T_hi] from the pre-computed lambda_cond: 2 / (lambda_cond
// max f_k / min f_c + the largest linearised surface rate).
static fedfem_status crit_step(fedfem_ctx *c, double T_lo, double T_hi, double *dt_crit)
{
    double fk_max, fk_min, fc_min;
    c->law_extrema(T_lo, T_hi, &fk_max, &fk_min, &fc_min);
    if (!(fc_min > 0) || !(fk_min > 0)) return fail(c, FEDFEM_ERR_ARG, "conductivity or heat law not positive on [T_lo, T_hi]");
    const double rl = std::fabs(T_lo - c->T_zero), rh = std::fabs(T_hi - c->T_zero);
    const double r3 = std::max(rl * rl * rl, rh * rh * rh);
    double *partial = c->d_red;
    const int nb = launch_surface_rate(c->nn, c->d_Ac64, c->d_Ar64, c->d_C0, c->d_isdir, c->h,
                                       4.0 * 5.67e-8 * c->eps * r3, fc_min, partial, c->stream);
    std::vector<double> pr(2 * nb);
    CK(cudaMemcpyAsync(pr.data(), partial, pr.size() * 8, cudaMemcpyDeviceToHost, c->stream), "read");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    double surf = 0.0;
    for (int b = 0; b < nb; ++b) surf = std::max(surf, pr[2 * b]);
    *dt_crit = 2.0 / (c->lambda_cond * fk_max / fc_min + surf);
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_precompute(fedfem_ctx *c, double T_lo, double T_hi, double *dt_crit_out)
{
    if (!c) return FEDFEM_ERR_ARG;
    if (!(T_lo <= T_hi)) return fail(c, FEDFEM_ERR_ARG, "T_lo must be <= T_hi");
    fedfem_status s = run_precompute_arrays(c);
    if (s != FEDFEM_OK) return s;
    // critical time step (Section 3.4): largest eigenvalue of C0^-1/2 K0 C0^-1/2 on the free
    // nodes by Lanczos.  The coefficients stay on the device; every 16 steps the host reads them
    // and takes the largest eigenvalue of the tridiagonal matrix, and stops when it changes by
    // < tol relative or the Krylov space is exhausted.
    const int64_t nn = c->nn;
    double *vcur = c->d_v[0], *vprev = c->d_v[1], *u = c->d_v[2], *F = c->d_v[3];
    double *partial = c->d_red, *norm2 = c->d_red + 2 * 1024;
    const int max_iter = c->power_max_iter;
    const double tol = c->power_tol;
    launch_lanczos_start(nn, c->d_isdir, F, vcur, partial, norm2, c->stream);
    double lam = 0.0;
    int it = 0;
    std::vector<double> coef, alpha, beta2;
    for (it = 0; it < max_iter; ++it) {
        launch_lanczos_step(c->npe, c->ne, nn, c->d_gconn, c->d_cond64, c->d_n2e_ptr, c->d_n2e, c->d_C0, c->d_isdir,
                            vprev, vcur, u, F, c->d_Y, it ? c->d_lz + 4 * (it - 1) + 2 : nullptr, c->d_lz + 4 * it,
                            partial, c->stream);
        std::swap(vprev, vcur);  // v_{j+1} was written over v_{j-1}
        if ((it & 15) == 15 || it == max_iter - 1) {
            coef.resize(4 * (size_t)(it + 1));
            CK(cudaMemcpyAsync(coef.data(), c->d_lz, coef.size() * 8, cudaMemcpyDeviceToHost, c->stream), "read");
            CK(cudaStreamSynchronize(c->stream), "synchronize");
            alpha.resize(it + 1);
            beta2.resize(it + 1);
            for (int j = 0; j <= it; ++j) {
                alpha[j] = coef[4 * j];
                beta2[j] = coef[4 * j + 2];
            }
            const double theta = fedfem::tridiag_max_eigenvalue(alpha, beta2, it + 1);
            const bool exhausted = !(beta2[it] > 1e-28 * theta * theta);
            const bool done = exhausted || (it > 16 && std::fabs(theta - lam) <= tol * std::fabs(theta));
            lam = theta;
            if (done) break;
        }
    }
    CK(cudaGetLastError(), "Lanczos");
    c->lambda_cond = lam;
    c->power_iters = it;
    double dtc = 0.0;
    s = crit_step(c, T_lo, T_hi, &dtc);
    if (s != FEDFEM_OK) return s;
    c->dt_crit = dtc;
    c->T_lo = T_lo;
    c->T_hi = T_hi;
    c->precomputed = true;
    if (dt_crit_out) *dt_crit_out = c->dt_crit;
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_set_dt(fedfem_ctx *c, double dt, int32_t force)
{
    if (!c) return FEDFEM_ERR_ARG;
    if (!c->precomputed) return fail(c, FEDFEM_ERR_STATE, "call fedfem_precompute first");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(c, FEDFEM_ERR_ARG, "dt must be > 0");
    if (dt > c->dt_crit && !force)
        return fail(c, FEDFEM_ERR_UNSTABLE, "dt = " + std::to_string(dt) + " exceeds dt_crit = " + std::to_string(c->dt_crit));
    c->dt = dt;
    c->has_dt = true;
    launch_set_A(c->nn, dt, c->d_C0, c->d_isdir, c->d_A, c->d_A2, c->stream);
    CK(cudaGetLastError(), "set dt");
    return FEDFEM_OK;
}

// ------------------------------------------------------------------------------------------
// state
// ------------------------------------------------------------------------------------------
namespace fedfem {

// Energy-audit totals restart (a new initial state).
fedfem_status reset_energy_totals(fedfem_ctx *c)
{
    c->energy_steps = 0;
    if (c->d_energy_acc) CK(cudaMemsetAsync(c->d_energy_acc, 0, 2 * (size_t)c->grid * 8, c->stream), "memset");
    return FEDFEM_OK;
}

// Install a field given in original node order (device FP64) as the state at step 0.
fedfem_status install_T(fedfem_ctx *c, const double *T0_dev_old)
{
    double *tmp = c->d_v[0];
    CK(cudaMemcpyAsync(tmp, T0_dev_old, c->nn * 8, cudaMemcpyDeviceToDevice, c->stream), "copy T0");
    launch_impose_dirichlet((int64_t)c->dir_nodes.size(), c->d_dir_new, c->d_dir_T, c->Tdir_at(0), tmp, c->d_old_of_new,
                            c->stream);
    launch_set_state(c->precision, c->nn, tmp, c->d_old_of_new, c->d_T[0], c->kahan ? c->d_comp[0] : nullptr, c->stream);
    CK(cudaGetLastError(), "set T");
    c->step = 0;
    c->has_T = true;
    return reset_energy_totals(c);
}

// Current state as FP64 in new node order into dst (device).
fedfem_status state_f64_new(fedfem_ctx *c, int64_t step, double *dst)
{
    const int b = (int)(step & 1);
    launch_state_to_f64(c->precision, c->nn, c->d_T[b], c->kahan ? c->d_comp[b] : nullptr, dst, c->stream);
    CK(cudaGetLastError(), "state");
    return FEDFEM_OK;
}

}  // namespace fedfem

extern "C" fedfem_status fedfem_set_T(fedfem_ctx *c, const double *T0)
{
    if (!c || !T0) return c ? fail(c, FEDFEM_ERR_ARG, "NULL T0") : FEDFEM_ERR_ARG;
    CK(cudaMemcpyAsync(c->d_v[1], T0, c->nn * 8, cudaMemcpyHostToDevice, c->stream), "upload T0");
    return install_T(c, c->d_v[1]);
}

extern "C" fedfem_status fedfem_set_T_device(fedfem_ctx *c, const double *T0_dev)
{
    if (!c || !T0_dev) return c ? fail(c, FEDFEM_ERR_ARG, "NULL T0") : FEDFEM_ERR_ARG;
    return install_T(c, T0_dev);
}

extern "C" fedfem_status fedfem_get_T_device(fedfem_ctx *c, double *T_dev)
{
    if (!c || !T_dev) return c ? fail(c, FEDFEM_ERR_ARG, "NULL output") : FEDFEM_ERR_ARG;
    if (!c->has_T) return fail(c, FEDFEM_ERR_STATE, "no temperature field set");
    fedfem_status s = state_f64_new(c, c->step, c->d_v[0]);
    if (s != FEDFEM_OK) return s;
    launch_permute_new_to_old(c->nn, c->d_v[0], c->d_old_of_new, T_dev, c->stream);
    CK(cudaGetLastError(), "get T");
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_get_T(fedfem_ctx *c, double *T_host)
{
    if (!c || !T_host) return c ? fail(c, FEDFEM_ERR_ARG, "NULL output") : FEDFEM_ERR_ARG;
    fedfem_status s = fedfem_get_T_device(c, c->d_v[1]);
    if (s != FEDFEM_OK) return s;
    CK(cudaMemcpyAsync(T_host, c->d_v[1], c->nn * 8, cudaMemcpyDeviceToHost, c->stream), "download T");
    return check_device(c);
}

extern "C" fedfem_status fedfem_get_step(fedfem_ctx *c, int64_t *step)
{
    if (!c || !step) return FEDFEM_ERR_ARG;
    *step = c->step;
    return FEDFEM_OK;
}

// ------------------------------------------------------------------------------------------
// time stepping
// ------------------------------------------------------------------------------------------
namespace fedfem {

StepArgs step_args(fedfem_ctx *c)
{
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.chunks = c->d_chunks;
    a.tiles = c->d_tiles;
    a.sh = c->d_sh;
    a.sptr = c->d_sptr;
    a.bnd = c->d_bnd;
    a.bnd_area = c->d_bnd_area;
    a.colptr = c->d_colptr;
    a.gptr = c->d_gptr;
    a.gidx = c->d_gidx;
    for (int b = 0; b < 2; ++b) {
        a.T[b] = c->d_T[b];
        a.comp[b] = c->d_comp[b];
        a.part[b] = c->d_part[b];
    }
    a.A = c->d_A;
    a.A2 = c->d_A2;
    a.Qext = c->d_Qext;
    a.Ac = c->d_Ac;
    a.Ar = c->d_Ar;
    a.tile_done = c->d_tile_done;
    a.nbr_ptr = c->d_nbr_ptr;
    a.nbr = c->d_nbr;
    a.err = c->d_err;
    a.phys = c->d_phys;
    a.cta_tile = c->d_cta_tile;
    a.n_tiles = c->til.n_tiles;
    a.tiles_per_cta = c->tpc;
    a.chunk_bytes = c->chunk_bytes;
    a.stages = c->stages;
    a.stage_magic = ~0ULL / (uint64_t)c->stages + 1;
    a.chunk = c->chunk;
    a.colour_offset = chunk_colour_offset(c->precision, c->npe, c->chunk);
    // the element stream is evicted first when it cannot stay resident in L2 (> 64 MB);
    // smaller meshes keep it cached from step to step
    const bool big = (int64_t)c->til.n_chunks * c->chunk_bytes > (64LL << 20);
    a.l2_stream_policy = c->opt.l2_policy == 2 || (c->opt.l2_policy == 0 && big) ? 1 : 0;
    a.sched_q = c->sched_q.empty() ? nullptr : c->d_sched_q;
    a.sched_Tinf = c->sched_Tinf.empty() ? nullptr : c->d_sched_Tinf;
    a.sched_Tdir = c->sched_Tdir.empty() ? nullptr : c->d_sched_Tdir;
    a.sched_len = c->sched_len;
    if (c->n_tab) {
        a.tk64 = c->hk;
        a.tc64 = c->hc;
        a.tk32 = hinge_law_f32(c->hk);
        a.tc32 = hinge_law_f32(c->hc);
    }
    a.scatter = c->scatter_mode;
    a.withhold = c->opt.debug_withhold_barrier;
    a.timeout_ns = (long long)(c->opt.barrier_timeout_s * 1e9);
    a.energy_acc = c->d_energy_acc;
    a.C0 = c->d_C0;
    a.dt = c->dt;
    return a;
}

// Enqueue n steps as persistent launches of at most steps_per_launch steps.
fedfem_status enqueue_steps(fedfem_ctx *c, int64_t n, void *rec, int64_t rec_stride)
{
    if (c->variant()) {
        if (rec) return fail(c, FEDFEM_ERR_UNSUPPORTED, "the adjoint record needs kT_eval = 0 and face_quadrature = 0");
        return variant_steps(c, n);
    }
    StepArgs a = step_args(c);
    int64_t spl = c->opt.steps_per_launch > 0 ? c->opt.steps_per_launch : 200;
    // the kernel counts the chunks of one launch in 32 bits
    int64_t max_chunks = 1;
    for (int t = 0; t < c->til.n_tiles; t += c->tpc) {
        int64_t n = 0;
        for (int u = t; u < std::min(t + c->tpc, c->til.n_tiles); ++u) n += c->til.tiles[u].n_chunks;
        max_chunks = std::max(max_chunks, n);
    }
    spl = std::max<int64_t>(1, std::min<int64_t>(spl, ((int64_t)1 << 30) / max_chunks));
    int64_t done = 0;
    while (done < n) {
        const int64_t k = std::min(spl, n - done);
        a.n0 = c->step;
        a.nsteps = (int32_t)k;
        a.rec = rec ? (uint8_t *)rec + (size_t)done * rec_stride * (c->precision == 64 ? 8 : 4) : nullptr;
        a.rec_stride = rec_stride;
        // the progress counters keep growing from launch to launch (every launch waits for
        // values above its base, which no earlier launch wrote); they restart from 0 only
        // before they would reach 2^31
        if ((uint64_t)c->progress_base + (uint64_t)k >= (1ull << 31)) {
            CK(cudaMemsetAsync(c->d_tile_done, 0, c->til.n_tiles * sizeof(unsigned int), c->stream), "reset tile progress");
            c->progress_base = 0;
        }
        a.progress_base = c->progress_base;
        // staggered start only for launches long enough to amortise it
        a.stagger_ns = k >= 8 ? c->stagger_ns : 0;
        CK(launch_step(a, c->precision, c->kahan, c->npe, c->n_tab, c->grid, c->block, c->smem, c->ts_cap, c->stream),
           "step launch");
        c->progress_base += (uint32_t)k;
        if (c->d_energy_acc) c->energy_steps += k;
        c->step += k;
        done += k;
    }
    return FEDFEM_OK;
}

}  // namespace fedfem

extern "C" fedfem_status fedfem_step_async(fedfem_ctx *c, int64_t n_steps)
{
    if (!c) return FEDFEM_ERR_ARG;
    if (n_steps < 0) return fail(c, FEDFEM_ERR_ARG, "n_steps < 0");
    if (!c->has_dt) return fail(c, FEDFEM_ERR_STATE, "call fedfem_set_dt first");
    if (!c->has_T) return fail(c, FEDFEM_ERR_STATE, "call fedfem_set_T first");
    if (n_steps == 0) return FEDFEM_OK;
    return enqueue_steps(c, n_steps, nullptr, 0);
}

extern "C" fedfem_status fedfem_sync(fedfem_ctx *c)
{
    if (!c) return FEDFEM_ERR_ARG;
    return check_device(c);
}

extern "C" fedfem_status fedfem_step(fedfem_ctx *c, int64_t n_steps)
{
    fedfem_status s = fedfem_step_async(c, n_steps);
    if (s != FEDFEM_OK) return s;
    return check_device(c);
}

extern "C" fedfem_status fedfem_step_adaptive(fedfem_ctx *c, int64_t n_steps, double safety, double margin,
                                              double *t_elapsed)
{
    if (!c) return FEDFEM_ERR_ARG;
    if (n_steps < 0 || !(safety > 0) || !(safety <= 1) || !(margin >= 0) || !std::isfinite(margin))
        return fail(c, FEDFEM_ERR_ARG, "need n_steps >= 0, 0 < safety <= 1, margin >= 0");
    if (!c->precomputed || !c->has_T) return fail(c, FEDFEM_ERR_STATE, "call fedfem_precompute and fedfem_set_T first");
    const int64_t spl = c->opt.steps_per_launch > 0 ? c->opt.steps_per_launch : 200;
    double t = 0.0;
    for (int64_t done = 0; done < n_steps;) {
        const int64_t k = std::min(spl, n_steps - done);
        // temperature range of the current state -> dt_crit over it -> dt for this launch
        fedfem_status s = state_f64_new(c, c->step, c->d_v[0]);
        if (s != FEDFEM_OK) return s;
        const int nb = launch_minmax(c->nn, c->d_v[0], c->d_red, c->stream);
        std::vector<double> pr(2 * nb);
        CK(cudaMemcpyAsync(pr.data(), c->d_red, pr.size() * 8, cudaMemcpyDeviceToHost, c->stream), "read");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        double lo = 1e300, hi = -1e300;
        for (int b = 0; b < nb; ++b) {
            lo = std::min(lo, pr[2 * b]);
            hi = std::max(hi, pr[2 * b + 1]);
        }
        if (!std::isfinite(lo) || !std::isfinite(hi)) return fail(c, FEDFEM_ERR_DIVERGED, "non-finite temperature");
        double dtc = 0.0;
        s = crit_step(c, lo - margin, hi + margin, &dtc);
        if (s != FEDFEM_OK) return s;
        c->dt = safety * dtc;
        c->has_dt = true;
        launch_set_A(c->nn, c->dt, c->d_C0, c->d_isdir, c->d_A, c->d_A2, c->stream);
        s = enqueue_steps(c, k, nullptr, 0);
        if (s != FEDFEM_OK) return s;
        t += (double)k * c->dt;
        done += k;
    }
    if (t_elapsed) *t_elapsed = t;
    return check_device(c);
}

// ------------------------------------------------------------------------------------------
// diagnostics
// ------------------------------------------------------------------------------------------
extern "C" fedfem_status fedfem_internal_loads(fedfem_ctx *c, const double *T_host, double *F_host)
{
    if (!c || !T_host || !F_host) return c ? fail(c, FEDFEM_ERR_ARG, "NULL array") : FEDFEM_ERR_ARG;
    if (!c->precomputed) return fail(c, FEDFEM_ERR_STATE, "call fedfem_precompute first");
    CK(cudaMemcpyAsync(c->d_v[0], T_host, c->nn * 8, cudaMemcpyHostToDevice, c->stream), "upload");
    launch_permute_old_to_new(c->nn, c->d_v[0], c->d_old_of_new, c->d_v[1], c->stream);
    if (c->variant()) {
        const fedfem_status vs = variant_loads64(c, c->d_v[1], c->step, c->d_v[2], nullptr);
        if (vs != FEDFEM_OK) return vs;
    } else {
        launch_apply(c->npe, c->ne, c->nn, c->d_gconn, c->d_cond64, c->d_n2e_ptr, c->d_n2e, c->d_v[1], c->d_v[1], c->k_a(),
                     c->k_lin, c->tk_ptr(), c->d_Y, c->d_v[2], c->stream);
    }
    launch_permute_new_to_old(c->nn, c->d_v[2], c->d_old_of_new, c->d_v[3], c->stream);
    CK(cudaGetLastError(), "internal loads");
    CK(cudaMemcpyAsync(F_host, c->d_v[3], c->nn * 8, cudaMemcpyDeviceToHost, c->stream), "download");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_energy_totals(fedfem_ctx *c, double *stored_change, double *boundary_in,
                                              int64_t *n_steps)
{
    if (!c || !stored_change || !boundary_in || !n_steps) return c ? fail(c, FEDFEM_ERR_ARG, "NULL output") : FEDFEM_ERR_ARG;
    if (!c->d_energy_acc) return fail(c, FEDFEM_ERR_UNSUPPORTED, "create the context with energy_audit = 1");
    std::vector<double> acc(2 * (size_t)c->grid);
    CK(cudaMemcpyAsync(acc.data(), c->d_energy_acc, acc.size() * 8, cudaMemcpyDeviceToHost, c->stream), "read");
    const fedfem_status s = check_device(c);
    if (s != FEDFEM_OK) return s;
    double S = 0.0, B = 0.0;  // CTA order: deterministic
    for (int b = 0; b < c->grid; ++b) {
        S += acc[2 * b];
        B += acc[2 * b + 1];
    }
    *stored_change = S;
    *boundary_in = B;
    *n_steps = c->energy_steps;
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_energy(fedfem_ctx *c, double *stored_change, double *boundary_in)
{
    if (!c || !stored_change || !boundary_in) return c ? fail(c, FEDFEM_ERR_ARG, "NULL output") : FEDFEM_ERR_ARG;
    if (c->step < 1 || !c->has_dt) return fail(c, FEDFEM_ERR_STATE, "no step taken yet");
    double *T0 = c->d_v[0], *T1 = c->d_v[1], *F = c->d_v[2];
    fedfem_status s = state_f64_new(c, c->step - 1, T0);
    if (s != FEDFEM_OK) return s;
    s = state_f64_new(c, c->step, T1);
    if (s != FEDFEM_OK) return s;
    // the step from T^(n-1) to T^n with the loads of step n - 1
    EnergyPhys ph{c->dt,     c->c_lin,  c->h,   c->Tinf_at(c->step - 1), c->eps * 5.67e-8, c->T_amb, c->T_zero, c->c_a(),
                  c->qs_at(c->step - 1), c->n_tab > 0, c->hc};
    const double *Qin = c->d_Qext64;
    if (c->variant()) {
        // element loads of the variant; with consistent faces the whole nodal heat flow (external
        // and surface loads) comes from the face integration, so the lumped surface terms are off
        double *Qtot = c->face_cons ? c->d_v[3] : nullptr;
        s = variant_loads64(c, T0, c->step - 1, F, Qtot);
        if (s != FEDFEM_OK) return s;
        if (Qtot) {
            Qin = Qtot;
            ph.h = 0.0;
            ph.eps_sigma = 0.0;
            ph.qs = 1.0;
        }
    } else {
        launch_apply(c->npe, c->ne, c->nn, c->d_gconn, c->d_cond64, c->d_n2e_ptr, c->d_n2e, T0, T0, c->k_a(), c->k_lin,
                     c->tk_ptr(), c->d_Y, F, c->stream);
    }
    double *partial = c->d_red, *sums = c->d_red + 2 * 1024;
    launch_energy(c->nn, T0, T1, F, c->d_C0, Qin, c->d_Ac64, c->d_Ar64, c->d_isdir, ph, partial, sums, c->stream);
    CK(cudaGetLastError(), "energy");
    double h2[2];
    CK(cudaMemcpyAsync(h2, sums, 16, cudaMemcpyDeviceToHost, c->stream), "read");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    *stored_change = h2[0];
    *boundary_in = h2[1];
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_set_schedule(fedfem_ctx *c, int64_t n_entries, const double *q_scale,
                                             const double *T_inf, const double *T_dir)
{
    if (!c) return FEDFEM_ERR_ARG;
    if (n_entries < 0) return fail(c, FEDFEM_ERR_ARG, "n_entries < 0");
    if (!c->group_elem.empty()) return fail(c, FEDFEM_ERR_UNSUPPORTED, "load schedules are not available for batches");
    if (n_entries > 0 && !q_scale && !T_inf && !T_dir) return fail(c, FEDFEM_ERR_ARG, "no schedule array given");
    for (int64_t i = 0; i < n_entries; ++i)
        if ((q_scale && !std::isfinite(q_scale[i])) || (T_inf && !std::isfinite(T_inf[i])) ||
            (T_dir && !std::isfinite(T_dir[i])))
            return fail(c, FEDFEM_ERR_ARG, "non-finite schedule entry");
    const bool had_Tdir = !c->sched_Tdir.empty();
    if (n_entries > c->sched_cap) {
        CK(dalloc(c, (void **)&c->d_sched_q, n_entries * 8), "alloc schedule");
        CK(dalloc(c, (void **)&c->d_sched_Tinf, n_entries * 8), "alloc schedule");
        CK(dalloc(c, (void **)&c->d_sched_Tdir, n_entries * 8), "alloc schedule");
        c->sched_cap = n_entries;
    }
    // the stream may still run steps that read the previous schedule
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    c->sched_q.clear();
    c->sched_Tinf.clear();
    c->sched_Tdir.clear();
    c->sched_len = 0;
    if (n_entries > 0) {
        if (q_scale) {
            c->sched_q.assign(q_scale, q_scale + n_entries);
            CK(cudaMemcpy(c->d_sched_q, q_scale, n_entries * 8, cudaMemcpyHostToDevice), "upload schedule");
        }
        if (T_inf) {
            c->sched_Tinf.assign(T_inf, T_inf + n_entries);
            CK(cudaMemcpy(c->d_sched_Tinf, T_inf, n_entries * 8, cudaMemcpyHostToDevice), "upload schedule");
        }
        if (T_dir) {
            c->sched_Tdir.assign(T_dir, T_dir + n_entries);
            CK(cudaMemcpy(c->d_sched_Tdir, T_dir, n_entries * 8, cudaMemcpyHostToDevice), "upload schedule");
        }
        c->sched_len = n_entries;
    }
    // a field already installed takes the prescribed values of the current step
    if (c->has_T && (had_Tdir || !c->sched_Tdir.empty())) {
        const int b = (int)(c->step & 1);
        launch_impose_dirichlet_state(c->precision, (int64_t)c->dir_nodes.size(), c->d_dir_new, c->d_dir_T,
                                      c->Tdir_at(c->step), c->d_T[b], c->kahan ? c->d_comp[b] : nullptr, c->stream);
        CK(cudaGetLastError(), "impose Dirichlet values");
    }
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_set_property_table(fedfem_ctx *c, int32_t n_points, const double *T, const double *fk,
                                                   const double *fc)
{
    if (!c) return FEDFEM_ERR_ARG;
    if (!c->group_elem.empty()) return fail(c, FEDFEM_ERR_UNSUPPORTED, "property tables are not available for batches");
    if (c->precomputed) return fail(c, FEDFEM_ERR_STATE, "set the property table before fedfem_precompute");
    if (n_points == 0) {
        c->n_tab = 0;
        c->tab_T.clear();
        c->tab_fk.clear();
        c->tab_fc.clear();
        return FEDFEM_OK;
    }
    if (n_points < 2 || n_points > kMaxTablePoints) return fail(c, FEDFEM_ERR_ARG, "a table has 2 to 8 points");
    if (!T || !fk || !fc) return fail(c, FEDFEM_ERR_ARG, "NULL table array");
    for (int j = 0; j < n_points; ++j) {
        if (!std::isfinite(T[j]) || (j > 0 && !(T[j] > T[j - 1])))
            return fail(c, FEDFEM_ERR_ARG, "table temperatures must be finite and increasing");
        if (!(fk[j] > 0) || !(fc[j] > 0) || !std::isfinite(fk[j]) || !std::isfinite(fc[j]))
            return fail(c, FEDFEM_ERR_ARG, "table factors must be finite and > 0");
    }
    c->n_tab = n_points;
    c->tab_T.assign(T, T + n_points);
    c->tab_fk.assign(fk, fk + n_points);
    c->tab_fc.assign(fc, fc + n_points);
    c->hk = make_hinge_law(n_points, T, fk);
    c->hc = make_hinge_law(n_points, T, fc);
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_set_params(fedfem_ctx *c, const double *kscale, const double *source)
{
    if (!c) return FEDFEM_ERR_ARG;
    if (!c->precomputed) return fail(c, FEDFEM_ERR_STATE, "call fedfem_precompute first");
    if (kscale) {
        for (int64_t e = 0; e < c->ne; ++e)
            if (!(kscale[e] > 0) || !std::isfinite(kscale[e])) return fail(c, FEDFEM_ERR_ARG, "kscale must be > 0");
        c->kscale.assign(kscale, kscale + c->ne);
    }
    if (source) c->source.assign(source, source + c->ne);
    if (c->params_on_device) {
        // the other parameter still lives on the device only: bring it back to the host copy
        if (!kscale) {
            c->kscale.resize(c->ne);
            CK(cudaMemcpyAsync(c->kscale.data(), c->d_kscale, c->ne * 8, cudaMemcpyDeviceToHost, c->stream), "read");
        }
        if (!source) {
            c->source.resize(c->ne);
            CK(cudaMemcpyAsync(c->source.data(), c->d_source, c->ne * 8, cudaMemcpyDeviceToHost, c->stream), "read");
        }
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        c->params_on_device = false;
    }
    return run_precompute_arrays(c);
}

extern "C" fedfem_status fedfem_set_params_device(fedfem_ctx *c, const double *kscale_dev, const double *source_dev)
{
    if (!c) return FEDFEM_ERR_ARG;
    if (!c->precomputed) return fail(c, FEDFEM_ERR_STATE, "call fedfem_precompute first");
    if (!c->params_on_device) {
        // the parameter not given keeps its current value: make the device copies current
        CK(cudaMemcpyAsync(c->d_kscale, c->kscale.data(), c->ne * 8, cudaMemcpyHostToDevice, c->stream), "upload");
        if (c->source.empty())
            CK(cudaMemsetAsync(c->d_source, 0, c->ne * 8, c->stream), "memset");
        else
            CK(cudaMemcpyAsync(c->d_source, c->source.data(), c->ne * 8, cudaMemcpyHostToDevice, c->stream), "upload");
    }
    if (kscale_dev) {
        CK(cudaMemcpyAsync(c->d_kscale, kscale_dev, c->ne * 8, cudaMemcpyDeviceToDevice, c->stream), "copy kscale");
        // every theta_e > 0 and finite: the smallest and largest value, read back (a few partials)
        const int nb = launch_minmax(c->ne, c->d_kscale, c->d_red, c->stream);
        std::vector<double> pr(2 * nb);
        CK(cudaMemcpyAsync(pr.data(), c->d_red, pr.size() * 8, cudaMemcpyDeviceToHost, c->stream), "read");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        for (int b = 0; b < nb; ++b)
            if (!(pr[2 * b] > 0) || !std::isfinite(pr[2 * b + 1])) return fail(c, FEDFEM_ERR_ARG, "kscale must be > 0");
    }
    if (source_dev) CK(cudaMemcpyAsync(c->d_source, source_dev, c->ne * 8, cudaMemcpyDeviceToDevice, c->stream), "copy source");
    c->params_on_device = true;
    return run_precompute_arrays(c);
}

extern "C" fedfem_status fedfem_state_bytes(fedfem_ctx *c, size_t *bytes)
{
    if (!c || !bytes) return FEDFEM_ERR_ARG;
    const size_t rs = c->precision == 64 ? 8 : 4;
    *bytes = 32 + c->nn * rs + (c->kahan ? c->nn * 4 : 0);
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_get_state(fedfem_ctx *c, void *buf)
{
    if (!c || !buf) return FEDFEM_ERR_ARG;
    if (!c->has_T) return fail(c, FEDFEM_ERR_STATE, "no temperature field set");
    const size_t rs = c->precision == 64 ? 8 : 4;
    int64_t hdr[4] = {c->step, c->nn, c->precision, c->kahan};
    std::memcpy(buf, hdr, 32);
    const int b = (int)(c->step & 1);
    uint8_t *p = (uint8_t *)buf + 32;
    CK(cudaMemcpyAsync(p, c->d_T[b], c->nn * rs, cudaMemcpyDeviceToHost, c->stream), "download state");
    if (c->kahan) CK(cudaMemcpyAsync(p + c->nn * rs, c->d_comp[b], c->nn * 4, cudaMemcpyDeviceToHost, c->stream), "download");
    return check_device(c);
}

extern "C" fedfem_status fedfem_set_state(fedfem_ctx *c, const void *buf)
{
    if (!c || !buf) return FEDFEM_ERR_ARG;
    int64_t hdr[4];
    std::memcpy(hdr, buf, 32);
    if (hdr[1] != c->nn || hdr[2] != c->precision || hdr[3] != c->kahan)
        return fail(c, FEDFEM_ERR_ARG, "state blob does not match this context");
    if (hdr[0] < 0) return fail(c, FEDFEM_ERR_ARG, "state blob with a negative step counter");
    const size_t rs = c->precision == 64 ? 8 : 4;
    // the step counter (which selects the ping-pong buffer and indexes the schedules) changes
    // only once the state it describes has arrived
    const int64_t step = hdr[0];
    const int b = (int)(step & 1);
    const uint8_t *p = (const uint8_t *)buf + 32;
    CK(cudaMemcpyAsync(c->d_T[b], p, c->nn * rs, cudaMemcpyHostToDevice, c->stream), "upload state");
    if (c->kahan) CK(cudaMemcpyAsync(c->d_comp[b], p + c->nn * rs, c->nn * 4, cudaMemcpyHostToDevice, c->stream), "upload");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    c->step = step;
    c->has_T = true;
    {
        const fedfem_status es = reset_energy_totals(c);
        if (es != FEDFEM_OK) return es;
    }
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_get_info(fedfem_ctx *c, fedfem_info *info)
{
    if (!c || !info) return FEDFEM_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n_nodes = c->nn;
    info->n_elems = c->ne;
    info->n_tiles = c->til.n_tiles;
    info->grid = c->grid;
    info->block = c->block;
    info->stages = c->stages;
    info->chunk = c->chunk;
    info->scatter = c->scatter_mode;
    info->steps_per_launch = c->opt.steps_per_launch > 0 ? c->opt.steps_per_launch : 200;
    info->max_tile_nodes = c->til.max_local;
    info->n_colors_max = c->til.max_colors;
    info->smem_bytes = (int32_t)c->smem;
    info->n_shared_nodes = c->til.sptr.empty() ? 0 : (int64_t)c->til.sptr.size() - 1;
    info->n_halo_slots = c->til.sptr.empty() ? 0 : c->til.sptr.back();
    info->elem_bytes = (int64_t)c->til.n_chunks * c->chunk_bytes;
    info->dt = c->dt;
    info->dt_crit = c->dt_crit;
    return FEDFEM_OK;
}

extern "C" const char *fedfem_error_string(fedfem_ctx *c) { return c ? c->err.c_str() : "NULL context"; }

extern "C" const char *fedfem_create_error(void) { return g_create_error.c_str(); }

extern "C" fedfem_status fedfem_check_tiling(const fedfem_mesh *mesh, int64_t n_boundary, const int32_t *boundary_nodes,
                                             int32_t n_tiles, int32_t chunk, int32_t single_class,
                                             fedfem_tiling_stats *stats)
{
    g_create_error.clear();
    // the mesh checks of fedfem_create, with a neutral material and no boundary data
    fedfem_material mat;
    std::memset(&mat, 0, sizeof(mat));
    mat.rho = mat.c0 = 1.0;
    mat.k0[0] = mat.k0[4] = mat.k0[8] = 1.0;
    fedfem_bcs bcs;
    std::memset(&bcs, 0, sizeof(bcs));
    std::string e = validate(mesh, &mat, 1, &bcs, false);
    if (e.empty() && (n_tiles < 1 || (chunk != 32 && chunk != 64))) e = "n_tiles must be >= 1 and chunk 32 or 64";
    if (e.empty() && (n_boundary < 0 || (n_boundary > 0 && !boundary_nodes))) e = "bad boundary node list";
    std::vector<uint8_t> is_bnd;
    if (e.empty()) {
        is_bnd.assign(mesh->n_nodes, 0);
        for (int64_t i = 0; i < n_boundary && e.empty(); ++i) {
            if (boundary_nodes[i] < 0 || boundary_nodes[i] >= mesh->n_nodes) e = "boundary node out of range";
            else is_bnd[boundary_nodes[i]] = 1;
        }
    }
    if (!e.empty()) {
        g_create_error = e;
        return FEDFEM_ERR_ARG;
    }
    Tiling T;
    e = build_tiling(mesh->nodes_per_elem, mesh->n_elems, mesh->n_nodes, mesh->conn, mesh->xyz, is_bnd.data(), n_tiles,
                     chunk, T, single_class != 0);
    if (e.empty()) e = validate_tiling(T);
    if (!e.empty()) {
        g_create_error = "tiling: " + e;
        return FEDFEM_ERR_MESH;
    }
    if (stats) {
        stats->n_tiles = T.n_tiles;
        stats->n_chunks = T.n_chunks;
        stats->max_tile_nodes = T.max_local;
        stats->n_colors_max = T.max_colors;
        stats->n_shared_nodes = T.sptr.empty() ? 0 : (int64_t)T.sptr.size() - 1;
        stats->n_halo_slots = T.sptr.empty() ? 0 : T.sptr.back();
        stats->n_padding_slots = (int64_t)T.n_chunks * chunk - mesh->n_elems;
    }
    return FEDFEM_OK;
}

extern "C" void fedfem_destroy(fedfem_ctx *c)
{
    if (!c) return;
    if (c->stream || c->device >= 0) cudaStreamSynchronize(c->stream);
    for (void *p : c->allocs) cudaFree(p);
    for (void *p : c->adj_allocs) cudaFree(p);
    delete c;
}
