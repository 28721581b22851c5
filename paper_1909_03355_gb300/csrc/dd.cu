// Domain decomposition of one mesh into sub-domains with explicit halo buffers.
//
// Section 3 (Eq. 15-16): with the lumped capacitance every nodal equation is independent once
// its element loads are known.  The mesh is cut into slabs (dd_plan.cpp); each sub-domain is a
// full context of its own (tiling, persistent step kernel) over its core elements plus a
// one-element ghost layer, so that every node it owns receives all of its element loads
// locally.  Its ghost nodes (owned by a neighbour) are held fixed like Dirichlet nodes during a
// step.  After every step each owner packs the new values of the nodes its neighbours hold as
// ghosts into a send buffer, the buffers travel to the neighbours' receive buffers (one copy
// per sub-domain pair: the message a multi-process run would send), and every sub-domain
// unpacks them into its ghost slots.  The owned values are computed from the same element
// loads as in the undecomposed mesh; only the order of the floating-point sums differs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"
#include "dd_plan.h"

using namespace fedfem;

struct fedfem_dd {
    DDPlan plan;
    int npe = 8, precision = 32, kahan = 1;
    int64_t nn = 0, ne = 0, step = 0;
    cudaStream_t stream = nullptr;
    std::vector<fedfem_ctx *> sub;
    // exchange entries (grouped by sub-domain pair): source / destination sub-domain and node
    // (context-internal ids) per entry, and the table of the sub-domains' state arrays
    int64_t n_ent = 0;
    int32_t *d_src_sub = nullptr, *d_src_id = nullptr, *d_dst_sub = nullptr, *d_dst_id = nullptr;
    void **d_Tptr = nullptr;   // [n_sub][2] temperature arrays (step parity)
    float **d_cptr = nullptr;  // [n_sub][2] Kahan compensation arrays (NULL without Kahan)
    uint64_t *d_send = nullptr, *d_recv = nullptr;  // halo buffers, 8 bytes per entry
    std::vector<void *> allocs;
    double dt_crit = 0, dt = 0;
    bool precomputed = false, has_dt = false, has_T = false;
    std::string err;
};

static thread_local std::string g_dd_create_error;

namespace {

fedfem_status dd_fail(fedfem_dd *d, fedfem_status s, const std::string &m)
{
    d->err = m;
    return s;
}

fedfem_status dd_sub_fail(fedfem_dd *d, int s, fedfem_status st)
{
    return dd_fail(d, st, "sub-domain " + std::to_string(s) + ": " + fedfem_error_string(d->sub[s]));
}

#define DDCK(x, what)                                                                            \
    do {                                                                                         \
        cudaError_t e_ = (x);                                                                    \
        if (e_ != cudaSuccess) return dd_fail(d, FEDFEM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Pack: entry q takes the state of node src_id[q] of sub-domain src_sub[q] at step parity b
// (FP32 + Kahan: value and compensation as a float pair; FP64: the double).
__global__ void k_dd_pack(int64_t n, int b, int kahan, int fp64, const int32_t *src_sub, const int32_t *src_id,
                          void *const *Tptr, float *const *cptr, uint64_t *send)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int s = src_sub[q], i = src_id[q];
    if (fp64) {
        send[q] = (uint64_t)__double_as_longlong(static_cast<const double *>(Tptr[2 * s + b])[i]);
    } else {
        const float t = static_cast<const float *>(Tptr[2 * s + b])[i];
        const float c = kahan ? cptr[2 * s + b][i] : 0.0f;
        send[q] = (uint64_t)__float_as_uint(t) | ((uint64_t)__float_as_uint(c) << 32);
    }
}

// Unpack: entry q writes its received value into ghost node dst_id[q] of sub-domain dst_sub[q].
__global__ void k_dd_unpack(int64_t n, int b, int kahan, int fp64, const int32_t *dst_sub, const int32_t *dst_id,
                            void *const *Tptr, float *const *cptr, const uint64_t *recv)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int s = dst_sub[q], i = dst_id[q];
    const uint64_t v = recv[q];
    if (fp64) {
        static_cast<double *>(Tptr[2 * s + b])[i] = __longlong_as_double((long long)v);
    } else {
        static_cast<float *>(Tptr[2 * s + b])[i] = __uint_as_float((uint32_t)v);
        if (kahan) cptr[2 * s + b][i] = __uint_as_float((uint32_t)(v >> 32));
    }
}

cudaError_t dd_alloc(fedfem_dd *d, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) d->allocs.push_back(*p);
    return e;
}

// Ghost values of every sub-domain from their owners, at the state of step d->step.
fedfem_status dd_exchange(fedfem_dd *d)
{
    if (d->n_ent == 0) return FEDFEM_OK;
    const int b = (int)(d->step & 1);
    const int th = 256;
    const int nb = (int)((d->n_ent + th - 1) / th);
    const int fp64 = d->precision == 64;
    k_dd_pack<<<nb, th, 0, d->stream>>>(d->n_ent, b, d->kahan, fp64, d->d_src_sub, d->d_src_id, d->d_Tptr, d->d_cptr,
                                       d->d_send);
    DDCK(cudaGetLastError(), "halo pack");
    for (const DDPair &pr : d->plan.pairs)  // one message per sub-domain pair
        DDCK(cudaMemcpyAsync(d->d_recv + pr.begin, d->d_send + pr.begin, (size_t)pr.count * 8, cudaMemcpyDeviceToDevice,
                             d->stream),
             "halo transfer");
    k_dd_unpack<<<nb, th, 0, d->stream>>>(d->n_ent, b, d->kahan, fp64, d->d_dst_sub, d->d_dst_id, d->d_Tptr, d->d_cptr,
                                         d->d_recv);
    DDCK(cudaGetLastError(), "halo unpack");
    return FEDFEM_OK;
}

}  // namespace

extern "C" fedfem_status fedfem_dd_create(const fedfem_mesh *mesh, const fedfem_material *mats, int32_t n_mats,
                                          const fedfem_bcs *bcs, const fedfem_options *opt, int32_t n_sub,
                                          fedfem_dd **out)
{
    g_dd_create_error.clear();
    if (!out) return FEDFEM_ERR_ARG;
    *out = nullptr;
    if (!mesh || !mats || !bcs || !mesh->xyz || !mesh->conn || n_mats < 1) {
        g_dd_create_error = "NULL mesh, materials or boundary conditions";
        return FEDFEM_ERR_ARG;
    }
    const int npe = mesh->nodes_per_elem;
    if (npe != 8 && npe != 4) {
        g_dd_create_error = "nodes_per_elem must be 8 or 4";
        return FEDFEM_ERR_ARG;
    }
    const int64_t nn = mesh->n_nodes, ne = mesh->n_elems;
    if (nn <= 0 || ne <= 0 || n_sub < 1 || n_sub > 64 || ne < n_sub) {
        g_dd_create_error = "need 1 <= n_sub <= 64 sub-domains and at least n_sub elements";
        return FEDFEM_ERR_ARG;
    }
    for (int64_t q = 0; q < ne * npe; ++q)
        if (mesh->conn[q] < 0 || mesh->conn[q] >= nn) {
            g_dd_create_error = "node id out of range in conn";
            return FEDFEM_ERR_MESH;
        }
    fedfem_dd *d = new fedfem_dd();
    d->npe = npe;
    d->nn = nn;
    d->ne = ne;
    fedfem_options o;
    fedfem_default_options(&o);
    if (opt) o = *opt;
    if (o.kT_eval || o.face_quadrature || o.energy_audit) {
        g_dd_create_error = "the decomposed mesh runs the persistent kernel without the energy audit: kT_eval, "
                            "face_quadrature and energy_audit must be 0";
        delete d;
        return FEDFEM_ERR_UNSUPPORTED;
    }
    d->precision = o.precision == 64 ? 64 : 32;
    d->kahan = (d->precision == 32 && o.kahan) ? 1 : 0;
    d->stream = static_cast<cudaStream_t>(o.stream);
    std::string m = build_dd_plan(npe, ne, nn, mesh->conn, mesh->xyz, n_sub, d->plan);
    if (!m.empty()) {
        g_dd_create_error = m;
        delete d;
        return FEDFEM_ERR_ARG;
    }
    const int nvf = bcs->face_nv ? bcs->face_nv : (npe == 8 ? 4 : 3);
    std::vector<uint8_t> isdir(nn, 0);
    std::vector<double> dirT(nn, 0.0);
    for (int64_t q = 0; q < bcs->n_dir; ++q) {
        const int32_t n = bcs->dir_nodes[q];
        if (n < 0 || n >= nn) {
            g_dd_create_error = "Dirichlet node id out of range";
            delete d;
            return FEDFEM_ERR_ARG;
        }
        isdir[n] = 1;
        dirT[n] = bcs->dir_T[q];
    }
    std::vector<int32_t> loc(nn, -1);
    for (int s = 0; s < n_sub; ++s) {
        const DDSub &S = d->plan.sub[s];
        for (size_t l = 0; l < S.nodes.size(); ++l) loc[S.nodes[l]] = (int32_t)l;
        // the sub-mesh in local ids
        std::vector<double> xyz(3 * S.nodes.size());
        for (size_t l = 0; l < S.nodes.size(); ++l)
            for (int r = 0; r < 3; ++r) xyz[3 * l + r] = mesh->xyz[3 * (int64_t)S.nodes[l] + r];
        std::vector<int32_t> conn(S.elems.size() * npe), emat, fconv, frad, dnodes;
        std::vector<double> ks, src, nq, dT;
        for (size_t e = 0; e < S.elems.size(); ++e) {
            const int64_t g = S.elems[e];
            for (int k = 0; k < npe; ++k) conn[npe * e + k] = loc[mesh->conn[npe * g + k]];
            if (mesh->elem_mat) emat.push_back(mesh->elem_mat[g]);
            if (mesh->elem_kscale) ks.push_back(mesh->elem_kscale[g]);
            if (bcs->elem_source) src.push_back(bcs->elem_source[g]);
        }
        // boundary faces whose nodes all belong to the sub-domain (every face at an owned node
        // is one of them)
        auto faces = [&](const int32_t *f, int64_t nf, std::vector<int32_t> &outf) {
            for (int64_t q = 0; q < nf; ++q) {
                bool in = true;
                for (int k = 0; k < nvf; ++k) in = in && f[nvf * q + k] >= 0 && f[nvf * q + k] < nn && loc[f[nvf * q + k]] >= 0;
                if (in)
                    for (int k = 0; k < nvf; ++k) outf.push_back(loc[f[nvf * q + k]]);
            }
        };
        faces(bcs->conv_faces, bcs->n_conv_faces, fconv);
        faces(bcs->rad_faces, bcs->n_rad_faces, frad);
        if (bcs->nodal_Q)
            for (size_t l = 0; l < S.nodes.size(); ++l) nq.push_back(bcs->nodal_Q[S.nodes[l]]);
        // Dirichlet nodes of the problem, and the ghosts (held during a step; their value is
        // written by the exchange, so the prescribed value given here is a placeholder)
        for (size_t l = 0; l < S.nodes.size(); ++l)
            if (isdir[S.nodes[l]] || S.ghost_owner[l] >= 0) {
                dnodes.push_back((int32_t)l);
                dT.push_back(isdir[S.nodes[l]] ? dirT[S.nodes[l]] : 0.0);
            }
        fedfem_mesh sm = *mesh;
        sm.n_nodes = (int64_t)S.nodes.size();
        sm.n_elems = (int64_t)S.elems.size();
        sm.xyz = xyz.data();
        sm.conn = conn.data();
        sm.elem_mat = mesh->elem_mat ? emat.data() : nullptr;
        sm.elem_kscale = mesh->elem_kscale ? ks.data() : nullptr;
        fedfem_bcs sb = *bcs;
        sb.n_dir = (int64_t)dnodes.size();
        sb.dir_nodes = dnodes.data();
        sb.dir_T = dT.data();
        sb.n_conv_faces = (int64_t)(fconv.size() / nvf);
        sb.conv_faces = fconv.data();
        sb.n_rad_faces = (int64_t)(frad.size() / nvf);
        sb.rad_faces = frad.data();
        sb.nodal_Q = bcs->nodal_Q ? nq.data() : nullptr;
        sb.elem_source = bcs->elem_source ? src.data() : nullptr;
        fedfem_ctx *c = nullptr;
        fedfem_status st = fedfem_create(&sm, mats, n_mats, &sb, &o, &c);
        for (size_t l = 0; l < S.nodes.size(); ++l) loc[S.nodes[l]] = -1;
        if (st != FEDFEM_OK) {
            g_dd_create_error = "sub-domain " + std::to_string(s) + ": " + fedfem_create_error();
            fedfem_dd_destroy(d);
            return st;
        }
        d->sub.push_back(c);
    }
    // exchange tables in the contexts' internal node numbering
    const DDPlan &P = d->plan;
    d->n_ent = (int64_t)P.src_local.size();
    std::vector<int32_t> ss(d->n_ent), si(d->n_ent), ds(d->n_ent), di(d->n_ent);
    for (const DDPair &pr : P.pairs)
        for (int64_t q = pr.begin; q < pr.begin + pr.count; ++q) {
            ss[q] = pr.src;
            si[q] = d->sub[pr.src]->til.new_of_old[P.src_local[q]];
            ds[q] = pr.dst;
            di[q] = d->sub[pr.dst]->til.new_of_old[P.dst_local[q]];
        }
    std::vector<void *> tp(2 * n_sub);
    std::vector<float *> cp(2 * n_sub);
    for (int s = 0; s < n_sub; ++s)
        for (int b = 0; b < 2; ++b) {
            tp[2 * s + b] = d->sub[s]->d_T[b];
            cp[2 * s + b] = d->kahan ? d->sub[s]->d_comp[b] : nullptr;
        }
    auto up = [&](void **p, const void *src, size_t bytes) -> cudaError_t {
        cudaError_t e = dd_alloc(d, p, bytes);
        if (e == cudaSuccess && bytes) e = cudaMemcpy(*p, src, bytes, cudaMemcpyHostToDevice);
        return e;
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = up((void **)&d->d_src_sub, ss.data(), ss.size() * 4);
    if (e == cudaSuccess) e = up((void **)&d->d_src_id, si.data(), si.size() * 4);
    if (e == cudaSuccess) e = up((void **)&d->d_dst_sub, ds.data(), ds.size() * 4);
    if (e == cudaSuccess) e = up((void **)&d->d_dst_id, di.data(), di.size() * 4);
    if (e == cudaSuccess) e = up((void **)&d->d_Tptr, tp.data(), tp.size() * sizeof(void *));
    if (e == cudaSuccess) e = up((void **)&d->d_cptr, cp.data(), cp.size() * sizeof(float *));
    if (e == cudaSuccess) e = dd_alloc(d, (void **)&d->d_send, (size_t)d->n_ent * 8);
    if (e == cudaSuccess) e = dd_alloc(d, (void **)&d->d_recv, (size_t)d->n_ent * 8);
    if (e != cudaSuccess) {
        g_dd_create_error = std::string("device allocation: ") + cudaGetErrorString(e);
        fedfem_dd_destroy(d);
        return e == cudaErrorMemoryAllocation ? FEDFEM_ERR_OOM : FEDFEM_ERR_CUDA;
    }
    *out = d;
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_dd_precompute(fedfem_dd *d, double T_lo, double T_hi, double *dt_crit_out)
{
    if (!d) return FEDFEM_ERR_ARG;
    double dtc = INFINITY;
    for (size_t s = 0; s < d->sub.size(); ++s) {
        double x = 0;
        fedfem_status st = fedfem_precompute(d->sub[s], T_lo, T_hi, &x);
        if (st != FEDFEM_OK) return dd_sub_fail(d, (int)s, st);
        // a sub-domain that owns no free node constrains nothing
        if (d->plan.sub[s].n_owned > 0) dtc = std::min(dtc, x);
    }
    d->dt_crit = dtc;
    d->precomputed = true;
    if (dt_crit_out) *dt_crit_out = dtc;
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_dd_set_dt(fedfem_dd *d, double dt, int32_t force)
{
    if (!d) return FEDFEM_ERR_ARG;
    if (!d->precomputed) return dd_fail(d, FEDFEM_ERR_STATE, "call fedfem_dd_precompute first");
    if (!(dt > 0) || !std::isfinite(dt)) return dd_fail(d, FEDFEM_ERR_ARG, "dt must be > 0");
    if (dt > d->dt_crit && !force) return dd_fail(d, FEDFEM_ERR_UNSTABLE, "dt exceeds dt_crit");
    for (size_t s = 0; s < d->sub.size(); ++s) {
        fedfem_status st = fedfem_set_dt(d->sub[s], dt, 1);
        if (st != FEDFEM_OK) return dd_sub_fail(d, (int)s, st);
    }
    d->dt = dt;
    d->has_dt = true;
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_dd_set_T(fedfem_dd *d, const double *T0)
{
    if (!d || !T0) return d ? dd_fail(d, FEDFEM_ERR_ARG, "NULL T0") : FEDFEM_ERR_ARG;
    std::vector<double> loc;
    for (size_t s = 0; s < d->sub.size(); ++s) {
        const DDSub &S = d->plan.sub[s];
        loc.resize(S.nodes.size());
        for (size_t l = 0; l < S.nodes.size(); ++l) loc[l] = T0[S.nodes[l]];
        fedfem_status st = fedfem_set_T(d->sub[s], loc.data());
        if (st != FEDFEM_OK) return dd_sub_fail(d, (int)s, st);
        DDCK(cudaStreamSynchronize(d->stream), "synchronize");  // the upload has read loc
    }
    d->step = 0;
    // ghosts carry placeholder values until their owners' values arrive
    fedfem_status st = dd_exchange(d);
    if (st != FEDFEM_OK) return st;
    d->has_T = true;
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_dd_step(fedfem_dd *d, int64_t n_steps)
{
    if (!d) return FEDFEM_ERR_ARG;
    if (n_steps < 0) return dd_fail(d, FEDFEM_ERR_ARG, "n_steps < 0");
    if (!d->has_dt) return dd_fail(d, FEDFEM_ERR_STATE, "call fedfem_dd_set_dt first");
    if (!d->has_T) return dd_fail(d, FEDFEM_ERR_STATE, "call fedfem_dd_set_T first");
    for (int64_t k = 0; k < n_steps; ++k) {
        // one step of every sub-domain (their own persistent kernel, one step per launch),
        // then the ghost values of the new state
        for (size_t s = 0; s < d->sub.size(); ++s) {
            fedfem_status st = fedfem::enqueue_steps(d->sub[s], 1, nullptr, 0);
            if (st != FEDFEM_OK) return dd_sub_fail(d, (int)s, st);
        }
        ++d->step;
        fedfem_status st = dd_exchange(d);
        if (st != FEDFEM_OK) return st;
    }
    for (size_t s = 0; s < d->sub.size(); ++s) {
        fedfem_status st = fedfem_sync(d->sub[s]);
        if (st != FEDFEM_OK) return dd_sub_fail(d, (int)s, st);
    }
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_dd_get_T(fedfem_dd *d, double *T_host)
{
    if (!d || !T_host) return d ? dd_fail(d, FEDFEM_ERR_ARG, "NULL output") : FEDFEM_ERR_ARG;
    if (!d->has_T) return dd_fail(d, FEDFEM_ERR_STATE, "no temperature field set");
    std::vector<double> loc;
    for (size_t s = 0; s < d->sub.size(); ++s) {
        const DDSub &S = d->plan.sub[s];
        loc.resize(S.nodes.size());
        fedfem_status st = fedfem_get_T(d->sub[s], loc.data());
        if (st != FEDFEM_OK) return dd_sub_fail(d, (int)s, st);
        for (size_t l = 0; l < S.nodes.size(); ++l)
            if (S.ghost_owner[l] < 0) T_host[S.nodes[l]] = loc[l];
    }
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_dd_get_info(fedfem_dd *d, fedfem_dd_info *info)
{
    if (!d || !info) return FEDFEM_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n_sub = d->plan.n_sub;
    info->axis = d->plan.axis;
    info->n_messages = (int32_t)d->plan.pairs.size();
    info->halo_entries = d->n_ent;
    info->halo_bytes_per_step = d->n_ent * (d->precision == 64 ? 8 : (d->kahan ? 8 : 4));
    int64_t ghost_elems = 0;
    for (const DDSub &S : d->plan.sub) ghost_elems += (int64_t)S.elems.size() - S.n_core;
    info->ghost_elements = ghost_elems;
    info->dt_crit = d->dt_crit;
    info->step = d->step;
    return FEDFEM_OK;
}

extern "C" fedfem_status fedfem_dd_subdomain(const fedfem_mesh *mesh, int32_t n_sub, int32_t s, int64_t *n_elems,
                                             int32_t *elems, int64_t *n_nodes, int32_t *nodes, int32_t *ghost_owner)
{
    if (!mesh || !mesh->xyz || !mesh->conn || !n_elems || !n_nodes) return FEDFEM_ERR_ARG;
    const int npe = mesh->nodes_per_elem;
    if ((npe != 8 && npe != 4) || mesh->n_nodes <= 0 || mesh->n_elems <= 0 || s < 0 || s >= n_sub) return FEDFEM_ERR_ARG;
    for (int64_t q = 0; q < mesh->n_elems * npe; ++q)
        if (mesh->conn[q] < 0 || mesh->conn[q] >= mesh->n_nodes) return FEDFEM_ERR_MESH;
    DDPlan P;
    if (!build_dd_plan(npe, mesh->n_elems, mesh->n_nodes, mesh->conn, mesh->xyz, n_sub, P).empty()) return FEDFEM_ERR_ARG;
    const DDSub &S = P.sub[s];
    *n_elems = (int64_t)S.elems.size();
    *n_nodes = (int64_t)S.nodes.size();
    if (elems) std::copy(S.elems.begin(), S.elems.end(), elems);
    if (nodes) std::copy(S.nodes.begin(), S.nodes.end(), nodes);
    if (ghost_owner) std::copy(S.ghost_owner.begin(), S.ghost_owner.end(), ghost_owner);
    return FEDFEM_OK;
}

extern "C" const char *fedfem_dd_error_string(fedfem_dd *d) { return d ? d->err.c_str() : g_dd_create_error.c_str(); }

extern "C" void fedfem_dd_destroy(fedfem_dd *d)
{
    if (!d) return;
    cudaStreamSynchronize(d->stream);
    for (fedfem_ctx *c : d->sub) fedfem_destroy(c);
    for (void *p : d->allocs) cudaFree(p);
    delete d;
}
