// Host-side plan of the domain decomposition (shared by dd.cu and the host-only query).
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

namespace fedfem {

// One sub-domain: its elements (core elements of its slab plus the ghost layer, ascending
// global ids) and the nodes they touch (ascending global ids; local id = index), with the
// owner of each node that it does not own (-1 for owned nodes).
struct DDSub {
    std::vector<int32_t> elems, nodes, ghost_owner;
    int64_t n_core = 0, n_owned = 0;
};

// Ghost values sent from sub-domain src to sub-domain dst: entries [begin, begin + count) of
// the exchange lists.
struct DDPair {
    int32_t src = 0, dst = 0;
    int64_t begin = 0, count = 0;
};

struct DDPlan {
    int n_sub = 0, axis = 2;
    std::vector<int32_t> elem_sub;    // [ne] slab (core sub-domain) of each element
    std::vector<int32_t> node_owner;  // [nn] owning sub-domain of each node
    std::vector<DDSub> sub;
    std::vector<DDPair> pairs;
    std::vector<int32_t> src_local, dst_local;  // per exchange entry: local ids in src and dst
};

// Slab partition along the longest axis of the bounding box into n_sub element slabs of equal
// size (by element centroid), owner of a node = lowest sub-domain among its elements, one
// ghost layer.  Returns "" on success, else a message.
std::string build_dd_plan(int npe, int64_t ne, int64_t nn, const int32_t *conn, const double *xyz, int n_sub,
                          DDPlan &P);

}  // namespace fedfem
