// Host-side plan of the domain decomposition (no CUDA): slab partition of the elements, node
// ownership, the one-element ghost layer of each sub-domain and its exchange lists.
//
// The nodal equations of the explicit scheme are independent once the element loads are known
// (Section 3, Eq. 15-16): a node needs the loads of the elements around it and nothing else.
// A sub-domain therefore holds its own (core) elements plus every other element that touches a
// node it owns, so each owned node receives all of its element loads locally; the nodes of
// those extra elements that it does not own are its ghosts, held fixed during a step and
// refreshed from their owners after it.
#include <algorithm>
#include <numeric>

#include "dd_plan.h"

namespace fedfem {

std::string build_dd_plan(int npe, int64_t ne, int64_t nn, const int32_t *conn, const double *xyz, int n_sub,
                          DDPlan &P)
{
    if (n_sub < 1) return "n_sub must be >= 1";
    if (ne < n_sub) return "fewer elements than sub-domains";
    P = DDPlan();
    P.n_sub = n_sub;
    // slab axis: the longest extent of the bounding box
    double lo[3], hi[3];
    for (int r = 0; r < 3; ++r) lo[r] = hi[r] = nn > 0 ? xyz[r] : 0.0;
    for (int64_t i = 0; i < nn; ++i)
        for (int r = 0; r < 3; ++r) {
            lo[r] = std::min(lo[r], xyz[3 * i + r]);
            hi[r] = std::max(hi[r], xyz[3 * i + r]);
        }
    int ax = 0;
    for (int r = 1; r < 3; ++r)
        if (hi[r] - lo[r] > hi[ax] - lo[ax]) ax = r;
    P.axis = ax;
    // elements ordered by centroid along the axis (ties by id), cut into equal-count slabs
    std::vector<double> cz(ne);
    for (int64_t e = 0; e < ne; ++e) {
        double s = 0.0;
        for (int k = 0; k < npe; ++k) s += xyz[3 * (int64_t)conn[npe * e + k] + ax];
        cz[e] = s / npe;
    }
    std::vector<int64_t> order(ne);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cz[a] < cz[b]; });
    P.elem_sub.assign(ne, 0);
    for (int64_t r = 0; r < ne; ++r) P.elem_sub[order[r]] = (int32_t)((r * n_sub) / ne);
    // owner of a node: the lowest sub-domain among the core elements that touch it
    P.node_owner.assign(nn, -1);
    for (int64_t e = 0; e < ne; ++e)
        for (int k = 0; k < npe; ++k) {
            const int32_t n = conn[npe * e + k];
            if (P.node_owner[n] < 0 || P.elem_sub[e] < P.node_owner[n]) P.node_owner[n] = P.elem_sub[e];
        }
    // node -> element incidence
    std::vector<int64_t> ptr(nn + 1, 0), ent((size_t)ne * npe);
    for (int64_t e = 0; e < ne; ++e)
        for (int k = 0; k < npe; ++k) ++ptr[conn[npe * e + k] + 1];
    for (int64_t n = 0; n < nn; ++n) ptr[n + 1] += ptr[n];
    {
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t e = 0; e < ne; ++e)
            for (int k = 0; k < npe; ++k) ent[fill[conn[npe * e + k]]++] = e;
    }
    P.sub.resize(n_sub);
    std::vector<int32_t> mark_e(ne, -1), mark_n(nn, -1);
    for (int s = 0; s < n_sub; ++s) {
        DDSub &S = P.sub[s];
        // elements: the core ones plus every element touching an owned node (ascending ids)
        for (int64_t e = 0; e < ne; ++e)
            if (P.elem_sub[e] == s) mark_e[e] = s;
        for (int64_t n = 0; n < nn; ++n)
            if (P.node_owner[n] == s)
                for (int64_t q = ptr[n]; q < ptr[n + 1]; ++q) mark_e[ent[q]] = s;
        for (int64_t e = 0; e < ne; ++e)
            if (mark_e[e] == s) {
                S.elems.push_back((int32_t)e);
                if (P.elem_sub[e] == s) ++S.n_core;
                for (int k = 0; k < npe; ++k) mark_n[conn[npe * e + k]] = s;
            }
        for (int64_t n = 0; n < nn; ++n)
            if (mark_n[n] == s) {
                S.nodes.push_back((int32_t)n);
                S.ghost_owner.push_back(P.node_owner[n] == s ? -1 : P.node_owner[n]);
                if (P.node_owner[n] == s) ++S.n_owned;
            }
    }
    // every node belongs to some element, and every owner holds its owned nodes
    for (int64_t n = 0; n < nn; ++n)
        if (P.node_owner[n] < 0) return "node " + std::to_string(n) + " belongs to no element";
    // exchange lists: ghost g of sub-domain d gets its value from the owner o = owner(g); the
    // entries are grouped by (o, d) and ordered by global id inside a group
    auto local_id = [&](int s, int32_t g) -> int32_t {
        const std::vector<int32_t> &v = P.sub[s].nodes;
        auto it = std::lower_bound(v.begin(), v.end(), g);
        return (it != v.end() && *it == g) ? (int32_t)(it - v.begin()) : -1;
    };
    for (int o = 0; o < n_sub; ++o)
        for (int d = 0; d < n_sub; ++d) {
            if (o == d) continue;
            DDPair pr;
            pr.src = o;
            pr.dst = d;
            pr.begin = (int64_t)P.src_local.size();
            const DDSub &D = P.sub[d];
            for (size_t l = 0; l < D.nodes.size(); ++l)
                if (D.ghost_owner[l] == o) {
                    const int32_t sl = local_id(o, D.nodes[l]);
                    if (sl < 0) return "ghost node " + std::to_string(D.nodes[l]) + " missing from its owner";
                    P.src_local.push_back(sl);
                    P.dst_local.push_back((int32_t)l);
                }
            pr.count = (int64_t)P.src_local.size() - pr.begin;
            if (pr.count > 0) P.pairs.push_back(pr);
        }
    return "";
}

}  // namespace fedfem
