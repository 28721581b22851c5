// Host-side data layout for the persistent FED-FEM kernel.
//
// The paper's algorithm (Fig. 1 (iii)) loops over elements and then over nodes; on the GPU the
// element loop is split into tiles that one CTA processes with the tile's node temperatures
// and load accumulators in shared memory.  This pass decides that layout for an arbitrary
// mesh (it uses no structure of the mesh beyond its connectivity and element centroids):
//   1. sort elements along a Morton (Z-order) curve of their centroids and cut the order into
//      tiles of near-equal element counts;
//   2. give every node an owner tile (the lowest tile touching it) and renumber nodes so that
//      each tile owns a contiguous range [interior | owned-shared];
//   3. colour each tile's elements so that elements of one colour share no node (the
//      deterministic shared-memory accumulation runs colour by colour): the lattice parity of
//      structured hexahedral grids (8 colours) where a check proves it proper, else greedy;
//   4. give every (tile, shared node) pair a halo slot; the slots of one node are contiguous
//      and ordered by tile, which fixes the order of the cross-tile sum.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>

#include "fedfem_internal.h"

namespace fedfem {

static uint64_t spread3(uint64_t v)
{
    uint64_t x = v & 0x1fffffULL;
    x = (x | (x << 32)) & 0x1f00000000ffffULL;
    x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}

// Morton (Z-order) sort of elements [e0, e1) by centroid, appended to `order`.
static void morton_sort(int npe, int64_t e0, int64_t e1, const int32_t *conn, const double *xyz,
                        std::vector<int64_t> &order)
{
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t e = e0; e < e1; ++e)
        for (int k = 0; k < npe; ++k)
            for (int r = 0; r < 3; ++r) {
                const double v = xyz[3 * (int64_t)conn[npe * e + k] + r];
                lo[r] = std::min(lo[r], v);
                hi[r] = std::max(hi[r], v);
            }
    // one scale for all three axes (the largest span), so the curve, and the tiles cut from
    // it, stay compact in physical space on elongated domains
    const double span = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    std::vector<std::pair<uint64_t, int64_t>> key(e1 - e0);
    const double q = (double)((1u << 21) - 1);
    for (int64_t e = e0; e < e1; ++e) {
        double c[3] = {0, 0, 0};
        for (int k = 0; k < npe; ++k)
            for (int r = 0; r < 3; ++r) c[r] += xyz[3 * (int64_t)conn[npe * e + k] + r];
        uint64_t m = 0;
        for (int r = 0; r < 3; ++r) {
            double u = span > 0 ? (c[r] / npe - lo[r]) / span : 0.0;
            u = std::min(1.0, std::max(0.0, u));
            m |= spread3((uint64_t)(u * q)) << r;
        }
        key[e - e0] = {m, e};
    }
    std::sort(key.begin(), key.end());
    for (const auto &kv : key) order.push_back(kv.second);
}

// Iterated-greedy passes of the per-tile element colouring.
static constexpr int kColourPasses = 8;

// Lattice parity of the hexahedra of a structured grid, from the connectivity alone (any node
// jitter or anisotropy): crossing a face of local face pair d (VTK order: d = 0 for the faces
// (0,3,7,4) / (1,2,6,5), 1 for (0,1,5,4) / (3,2,6,7), 2 for (0,1,2,3) / (4,5,6,7)) flips bit d,
// assigned breadth-first over face neighbours (two hexahedra share a face when they share two
// opposite corners of it).  Face-connected parts start at 0.  Returns false (bits unusable)
// when the propagation contradicts itself, i.e. the mesh is not a consistently oriented grid.
static bool hex_lattice_parity(int64_t ne, int64_t nn, const int32_t *conn, std::vector<int8_t> &bits)
{
    static const int F[6][4] = {{0, 3, 7, 4}, {1, 2, 6, 5}, {0, 1, 5, 4}, {3, 2, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}};
    std::vector<int64_t> ptr(nn + 1, 0);
    for (int64_t i = 0; i < ne * 8; ++i) ++ptr[conn[i] + 1];
    for (int64_t i = 0; i < nn; ++i) ptr[i + 1] += ptr[i];
    std::vector<int32_t> inc(ptr[nn]);
    {
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t e = 0; e < ne; ++e)
            for (int k = 0; k < 8; ++k) inc[fill[conn[8 * e + k]]++] = (int32_t)e;
    }
    auto has = [&](int64_t e, int32_t n) {
        for (int k = 0; k < 8; ++k)
            if (conn[8 * e + k] == n) return true;
        return false;
    };
    bits.assign(ne, -1);
    std::vector<int64_t> queue;
    queue.reserve(ne);
    for (int64_t s = 0; s < ne; ++s) {
        if (bits[s] >= 0) continue;
        bits[s] = 0;
        queue.clear();
        queue.push_back(s);
        for (size_t qi = 0; qi < queue.size(); ++qi) {
            const int64_t e = queue[qi];
            for (int f = 0; f < 6; ++f) {
                const int32_t a = conn[8 * e + F[f][0]], c = conn[8 * e + F[f][2]];
                for (int64_t q = ptr[a]; q < ptr[a + 1]; ++q) {
                    const int64_t o = inc[q];
                    if (o == e || !has(o, c)) continue;
                    const int8_t want = (int8_t)(bits[e] ^ (1 << (f >> 1)));
                    if (bits[o] < 0) {
                        bits[o] = want;
                        queue.push_back(o);
                    } else if (bits[o] != want) {
                        return false;
                    }
                }
            }
        }
    }
    return true;
}

std::string build_tiling(int npe, int64_t ne, int64_t nn, const int32_t *conn, const double *xyz,
                         const uint8_t *is_bnd, int n_tiles, int CH, Tiling &T, bool single_class)
{
    if (n_tiles < 1) n_tiles = 1;
    if (n_tiles > ne) n_tiles = (int)std::max<int64_t>(1, ne);
    return build_tiling_groups(npe, ne, nn, conn, xyz, is_bnd, {0, ne}, {n_tiles}, CH, T, single_class);
}

std::string build_tiling_groups(int npe, int64_t ne, int64_t nn, const int32_t *conn, const double *xyz,
                                const uint8_t *is_bnd, const std::vector<int64_t> &group_elem,
                                const std::vector<int> &tiles_per_group, int CH, Tiling &T, bool single_class)
{
    T = Tiling();
    T.single_class = single_class;
    T.npe = npe;
    T.ne = ne;
    T.nn = nn;
    T.CH = CH;
    if (ne <= 0 || nn <= 0) return "empty mesh";
    const int G = (int)tiles_per_group.size();
    if ((int)group_elem.size() != G + 1 || group_elem[0] != 0 || group_elem[G] != ne) return "bad element groups";

    // 1. Morton order of element centroids inside each group; each group cut into its tiles
    std::vector<int64_t> order;
    order.reserve(ne);
    std::vector<int64_t> tb(1, 0);
    std::vector<int32_t> tile_group;
    for (int g = 0; g < G; ++g) {
        const int64_t e0 = group_elem[g], e1 = group_elem[g + 1];
        if (e1 <= e0) return "empty element group";
        morton_sort(npe, e0, e1, conn, xyz, order);
        const int nt = std::max<int>(1, (int)std::min<int64_t>(tiles_per_group[g], e1 - e0));
        for (int t = 1; t <= nt; ++t) {
            tb.push_back(e0 + (int64_t)((__int128)(e1 - e0) * t / nt));
            tile_group.push_back(g);
        }
    }
    const int n_tiles = (int)tile_group.size();
    T.n_tiles = n_tiles;

    // 2. node -> tiles (ascending) CSR, owner = first tile
    std::vector<int32_t> last(nn, -1), cnt(nn, 0);
    for (int t = 0; t < n_tiles; ++t)
        for (int64_t p = tb[t]; p < tb[t + 1]; ++p) {
            const int64_t e = order[p];
            for (int k = 0; k < npe; ++k) {
                const int32_t n = conn[npe * e + k];
                if (last[n] != t) {
                    last[n] = t;
                    ++cnt[n];
                }
            }
        }
    for (int64_t i = 0; i < nn; ++i)
        if (cnt[i] == 0) return "node " + std::to_string(i) + " belongs to no element";
    std::vector<int64_t> ntp(nn + 1, 0);
    for (int64_t i = 0; i < nn; ++i) ntp[i + 1] = ntp[i] + cnt[i];
    std::vector<int32_t> ntl(ntp[nn]);
    {
        std::vector<int64_t> fill(ntp.begin(), ntp.end() - 1);
        std::fill(last.begin(), last.end(), -1);
        for (int t = 0; t < n_tiles; ++t)
            for (int64_t p = tb[t]; p < tb[t + 1]; ++p) {
                const int64_t e = order[p];
                for (int k = 0; k < npe; ++k) {
                    const int32_t n = conn[npe * e + k];
                    if (last[n] != t) {
                        last[n] = t;
                        ntl[fill[n]++] = t;
                    }
                }
            }
    }
    auto owner = [&](int32_t n) { return ntl[ntp[n]]; };

    // renumber: per tile, interior nodes then owned-shared nodes, first-touch order
    T.new_of_old.assign(nn, -1);
    T.old_of_new.assign(nn, -1);
    T.tiles.resize(n_tiles);
    int32_t next = 0;
    for (int t = 0; t < n_tiles; ++t) {
        TileInfo &ti = T.tiles[t];
        std::memset(&ti, 0, sizeof(ti));
        ti.scenario = tile_group[t];
        ti.node_begin = next;
        for (int pass = 0; pass < 2; ++pass) {
            for (int64_t p = tb[t]; p < tb[t + 1]; ++p) {
                const int64_t e = order[p];
                for (int k = 0; k < npe; ++k) {
                    const int32_t n = conn[npe * e + k];
                    if (T.new_of_old[n] >= 0 || owner(n) != t) continue;
                    const bool shared = cnt[n] > 1;
                    if ((pass == 0) == shared) continue;
                    T.new_of_old[n] = next;
                    T.old_of_new[next] = n;
                    ++next;
                }
            }
            if (pass == 0) ti.n_interior = next - ti.node_begin;
        }
        ti.n_owned = next - ti.node_begin;
    }
    if (next != nn) return "internal error: renumbering incomplete";

    // shared ids in new-id order, halo slots ordered by tile
    std::vector<int32_t> sid_of_new(nn, -1);
    T.sptr.assign(1, 0);
    for (int32_t g = 0; g < nn; ++g) {
        const int32_t o = T.old_of_new[g];
        if (cnt[o] > 1) {
            sid_of_new[g] = (int32_t)T.sptr.size() - 1;
            T.sptr.push_back(T.sptr.back() + cnt[o]);
        }
    }

    // tile neighbours: tiles that share at least one node (CSR, ascending)
    {
        std::vector<std::vector<int32_t>> nb(n_tiles);
        for (int64_t i = 0; i < nn; ++i) {
            if (cnt[i] < 2) continue;
            for (int64_t a = ntp[i]; a < ntp[i + 1]; ++a)
                for (int64_t b = ntp[i]; b < ntp[i + 1]; ++b)
                    if (a != b) nb[ntl[a]].push_back(ntl[b]);
        }
        T.nbr_ptr.assign(1, 0);
        for (int t = 0; t < n_tiles; ++t) {
            std::sort(nb[t].begin(), nb[t].end());
            nb[t].erase(std::unique(nb[t].begin(), nb[t].end()), nb[t].end());
            T.nbr.insert(T.nbr.end(), nb[t].begin(), nb[t].end());
            T.nbr_ptr.push_back((int32_t)T.nbr.size());
        }
    }

    // lattice parity of structured hexahedral grids (a colouring candidate for every tile)
    std::vector<int8_t> lattice;
    const bool have_lattice = npe == 8 && hex_lattice_parity(ne, nn, conn, lattice);

    // 3./4. per tile: local numbering, colouring, chunks, shared and boundary entries
    std::vector<int32_t> loc(nn, -1);
    std::vector<uint64_t> mask;
    T.max_local = 0;
    T.max_colors = 0;
    int32_t chunk = 0;
    for (int t = 0; t < n_tiles; ++t) {
        TileInfo &ti = T.tiles[t];
        std::vector<int32_t> ghosts;
        for (int64_t p = tb[t]; p < tb[t + 1]; ++p) {
            const int64_t e = order[p];
            for (int k = 0; k < npe; ++k) {
                const int32_t n = conn[npe * e + k];
                const int32_t g = T.new_of_old[n];
                if (loc[n] != -1) continue;
                if (owner(n) == t) {
                    loc[n] = g - ti.node_begin;
                } else {
                    loc[n] = -2;  // ghost, numbered below
                    ghosts.push_back(g);
                }
            }
        }
        std::sort(ghosts.begin(), ghosts.end());
        for (size_t i = 0; i < ghosts.size(); ++i) loc[T.old_of_new[ghosts[i]]] = ti.n_owned + (int32_t)i;
        ti.n_local = ti.n_owned + (int32_t)ghosts.size();
        if (ti.n_local > 65535) return "tile with more than 65535 nodes (use more tiles)";
        T.max_local = std::max(T.max_local, ti.n_local);

        // element colouring (every class costs the step kernel a barrier and a padded chunk):
        // the lattice parity of the connectivity, else the parity pattern of the quantised
        // centroids, when proper (structured hex grids: 8 colours), else the best of greedy
        // colourings from the Morton order, from a raster order, and iterated greedy
        // (Culberson: recolouring class by class, classes in reverse order, never needs more
        // colours)
        const int64_t m = tb[t + 1] - tb[t];
        std::vector<uint8_t> col(m, 0);
        int ncol_best = single_class ? 1 : 0;
        if (single_class) {
            T.max_colors = std::max(T.max_colors, 1);
        } else {
            // raster order of the element centroids quantised to the mean element edge
            std::vector<int64_t> raster(m);
            std::vector<uint8_t> parity(m);  // candidate 8-colouring (validated below)
            {
                double lo[3] = {1e300, 1e300, 1e300};
                std::vector<double> cen(3 * m);
                double hsum = 0;  // sum of the elements' mean bounding-box edges
                for (int64_t p = 0; p < m; ++p) {
                    const int64_t e = order[tb[t] + p];
                    double edge = 0;
                    for (int r = 0; r < 3; ++r) {
                        double c = 0, a = 1e300, b = -1e300;
                        for (int k = 0; k < npe; ++k) {
                            const double v = xyz[3 * (int64_t)conn[npe * e + k] + r];
                            c += v;
                            a = std::min(a, v);
                            b = std::max(b, v);
                        }
                        cen[3 * p + r] = c / npe;
                        lo[r] = std::min(lo[r], cen[3 * p + r]);
                        edge += (b - a) / 3;
                    }
                    hsum += edge;
                }
                const double hsz = std::max(1e-300, hsum / (double)std::max<int64_t>(m, 1));
                std::vector<std::array<int64_t, 3>> q(m);
                for (int64_t p = 0; p < m; ++p)
                    for (int r = 0; r < 3; ++r) q[p][2 - r] = (int64_t)std::floor((cen[3 * p + r] - lo[r]) / hsz + 0.5);
                std::iota(raster.begin(), raster.end(), 0);
                std::stable_sort(raster.begin(), raster.end(), [&](int64_t a, int64_t b) { return q[a] < q[b]; });
                for (int64_t p = 0; p < m; ++p)
                    parity[p] = (uint8_t)((q[p][2] & 1) | ((q[p][1] & 1) << 1) | ((q[p][0] & 1) << 2));
            }
            // the lattice parity of the connectivity and the parity pattern of the quantised
            // centroids are proper colourings on structured hex grids (the latter only while
            // node jitter leaves the centroids on their lattice); a candidate is kept only if no
            // two elements sharing a node got the same colour
            std::vector<uint8_t> lat;
            if (have_lattice) {
                lat.resize(m);
                for (int64_t p = 0; p < m; ++p) lat[p] = (uint8_t)lattice[order[tb[t] + p]];
            }
            for (int cand = have_lattice ? 0 : 1; cand < 2 && ncol_best == 0; ++cand) {
                const std::vector<uint8_t> &cv = cand == 0 ? lat : parity;
                mask.assign(ti.n_local, 0);
                bool proper = true;
                for (int64_t p = 0; p < m && proper; ++p) {
                    const int64_t e = order[tb[t] + p];
                    const uint64_t bit = 1ULL << cv[p];
                    for (int k = 0; k < npe; ++k) {
                        uint64_t &mk = mask[loc[conn[npe * e + k]]];
                        if (mk & bit) proper = false;
                        mk |= bit;
                    }
                }
                if (proper) {
                    col = cv;
                    for (int64_t p = 0; p < m; ++p) ncol_best = std::max(ncol_best, (int)cv[p] + 1);
                }
            }
            // no colouring needs fewer colours than the most elements of the tile on one node
            int deg_max = 0;
            {
                std::vector<int> deg(ti.n_local, 0);
                for (int64_t p = 0; p < m; ++p)
                    for (int k = 0; k < npe; ++k)
                        deg_max = std::max(deg_max, ++deg[loc[conn[npe * order[tb[t] + p] + k]]]);
            }
            std::vector<int64_t> seq(m);
            std::iota(seq.begin(), seq.end(), 0);
            std::vector<uint8_t> trial(m);
            // saturation-degree order (Brelaz's DSATUR): colour next the uncoloured element
            // whose nodes already carry the most distinct colours (ties: the earliest in the
            // tile's element order), with the lowest colour free at its nodes.  Levels of
            // saturation are kept as bit sets over the element positions.
            if (ncol_best != deg_max && m > 0) {
                std::vector<int32_t> nptr(ti.n_local + 1, 0), nlist((size_t)m * npe);
                for (int64_t p = 0; p < m; ++p)
                    for (int k = 0; k < npe; ++k) ++nptr[loc[conn[npe * order[tb[t] + p] + k]] + 1];
                for (int32_t l = 0; l < ti.n_local; ++l) nptr[l + 1] += nptr[l];
                {
                    std::vector<int32_t> fill(nptr.begin(), nptr.end() - 1);
                    for (int64_t p = 0; p < m; ++p)
                        for (int k = 0; k < npe; ++k) nlist[fill[loc[conn[npe * order[tb[t] + p] + k]]]++] = (int32_t)p;
                }
                const int64_t W = (m + 63) / 64;
                std::vector<uint64_t> level((size_t)65 * W, 0);
                std::vector<int64_t> cnt(65, 0);
                std::vector<uint8_t> sat(m, 0), done(m, 0);
                for (int64_t p = 0; p < m; ++p) level[p >> 6] |= 1ULL << (p & 63);
                cnt[0] = m;
                mask.assign(ti.n_local, 0);
                auto seen = [&](int64_t p) {
                    const int64_t e = order[tb[t] + p];
                    uint64_t u = 0;
                    for (int k = 0; k < npe; ++k) u |= mask[loc[conn[npe * e + k]]];
                    return u;
                };
                int top = 0, nc = 0;
                for (int64_t it = 0; it < m; ++it) {
                    while (cnt[top] == 0) --top;
                    int64_t p = -1;
                    for (int64_t w = 0; w < W; ++w) {
                        const uint64_t v = level[(size_t)top * W + w];
                        if (v) {
                            p = w * 64 + __builtin_ctzll(v);
                            break;
                        }
                    }
                    level[(size_t)top * W + (p >> 6)] &= ~(1ULL << (p & 63));
                    --cnt[top];
                    done[p] = 1;
                    const uint64_t used = seen(p);
                    if (~used == 0) return "more than 64 colours needed in a tile";
                    const int c = __builtin_ctzll(~used);
                    trial[p] = (uint8_t)c;
                    nc = std::max(nc, c + 1);
                    const int64_t e = order[tb[t] + p];
                    for (int k = 0; k < npe; ++k) {
                        const int32_t v = loc[conn[npe * e + k]];
                        if (mask[v] & (1ULL << c)) continue;
                        mask[v] |= 1ULL << c;
                        for (int32_t j = nptr[v]; j < nptr[v + 1]; ++j) {
                            const int32_t f = nlist[j];
                            if (done[f]) continue;
                            const int sf = __builtin_popcountll(seen(f));
                            if (sf != sat[f]) {
                                level[(size_t)sat[f] * W + (f >> 6)] &= ~(1ULL << (f & 63));
                                --cnt[sat[f]];
                                sat[f] = (uint8_t)sf;
                                level[(size_t)sf * W + (f >> 6)] |= 1ULL << (f & 63);
                                ++cnt[sf];
                                top = std::max(top, sf);
                            }
                        }
                    }
                }
                if (ncol_best == 0 || nc < ncol_best) {
                    col = trial;
                    ncol_best = nc;
                }
            }
            for (int pass = 0; pass < kColourPasses && ncol_best != deg_max; ++pass) {
                if (pass == 1) seq = raster;
                mask.assign(ti.n_local, 0);
                int nc = 0;
                for (int64_t p : seq) {
                    const int64_t e = order[tb[t] + p];
                    uint64_t used = 0;
                    for (int k = 0; k < npe; ++k) used |= mask[loc[conn[npe * e + k]]];
                    if (~used == 0) return "more than 64 colours needed in a tile";
                    const int c = __builtin_ctzll(~used);
                    trial[p] = (uint8_t)c;
                    nc = std::max(nc, c + 1);
                    for (int k = 0; k < npe; ++k) mask[loc[conn[npe * e + k]]] |= 1ULL << c;
                }
                if (ncol_best == 0 || nc < ncol_best) {
                    col = trial;
                    ncol_best = nc;
                }
                // next order (after the two starting orders): the classes of the best colouring,
                // last class first
                if (pass >= 1)
                    std::stable_sort(seq.begin(), seq.end(), [&](int64_t a, int64_t b) { return col[a] > col[b]; });
            }
            // number the colours in use 0, 1, ... (a candidate may leave a class empty)
            int remap[64];
            for (int c = 0; c < 64; ++c) remap[c] = -1;
            for (int64_t p = 0; p < m; ++p) remap[col[p]] = 0;
            int used = 0;
            for (int c = 0; c < 64; ++c)
                if (remap[c] == 0) remap[c] = used++;
            for (int64_t p = 0; p < m; ++p) col[p] = (uint8_t)remap[col[p]];
            ncol_best = used;
            T.max_colors = std::max(T.max_colors, ncol_best);
        }
        std::vector<int64_t> perm(m);
        std::iota(perm.begin(), perm.end(), 0);
        std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) { return col[a] < col[b]; });

        // chunks: every colour class starts a new chunk (padding slots have colour 0xFF), so
        // each chunk holds elements of a single colour
        int ncol = 0;
        for (int64_t p = 0; p < m; ++p) ncol = std::max(ncol, (int)col[p] + 1);
        std::vector<int64_t> cnt_c(ncol, 0);
        for (int64_t p = 0; p < m; ++p) ++cnt_c[col[p]];
        ti.chunk_begin = chunk;
        ti.col_begin = (int32_t)T.colptr.size();
        ti.n_colors = ncol;
        int32_t nchk = 0;
        for (int c = 0; c < ncol; ++c) {
            T.colptr.push_back(nchk);
            nchk += (int32_t)((cnt_c[c] + CH - 1) / CH);
        }
        T.colptr.push_back(nchk);
        ti.n_chunks = nchk;
        chunk += nchk;
        const size_t slots = (size_t)chunk * CH;
        T.elem_of_slot.resize(slots, -1);
        T.elem_col.resize(slots, 0xFF);
        T.lconn.resize(slots * npe, 0);
        {
            int64_t p = 0;
            for (int c = 0; c < ncol; ++c) {
                const int64_t base = ((int64_t)ti.chunk_begin + T.colptr[ti.col_begin + c]) * CH;
                for (int64_t i = 0; i < cnt_c[c]; ++i, ++p) {
                    const int64_t e = order[tb[t] + perm[p]];
                    const int64_t s = base + i;
                    T.elem_of_slot[s] = (int32_t)e;
                    T.elem_col[s] = col[perm[p]];
                    for (int k = 0; k < npe; ++k) T.lconn[s * npe + k] = (uint16_t)loc[conn[npe * e + k]];
                }
            }
        }

        // slot gather lists: for every local node the slots (and node positions) that touch it,
        // in ascending slot order
        if (single_class) {
            T.max_chunks = std::max(T.max_chunks, ti.n_chunks);
            ti.gp_begin = (int32_t)T.gptr.size();
            std::vector<int32_t> cntl(ti.n_local + 1, 0);
            const int64_t s0 = (int64_t)ti.chunk_begin * CH, s1 = (int64_t)(ti.chunk_begin + ti.n_chunks) * CH;
            for (int64_t s = s0; s < s1; ++s)
                if (T.elem_of_slot[s] >= 0)
                    for (int k = 0; k < npe; ++k) ++cntl[T.lconn[s * npe + k] + 1];
            if (T.gidx.size() + (size_t)m * npe > (size_t)INT32_MAX) return "too many slot gather entries";
            const int32_t base = (int32_t)T.gidx.size();
            for (int32_t l = 0; l < ti.n_local; ++l) cntl[l + 1] += cntl[l];
            for (int32_t l = 0; l <= ti.n_local; ++l) T.gptr.push_back(base + cntl[l]);
            T.gidx.resize(T.gidx.size() + (size_t)cntl[ti.n_local]);
            std::vector<int32_t> fill(cntl.begin(), cntl.end() - 1);
            for (int64_t s = s0; s < s1; ++s)
                if (T.elem_of_slot[s] >= 0)
                    for (int k = 0; k < npe; ++k) {
                        const int l = T.lconn[s * npe + k];
                        T.gidx[base + fill[l]++] = (int32_t)((s - s0) * npe + k);
                    }
        }

        // shared entries: owned-shared then ghosts
        ti.sh_begin = (int32_t)T.sh.size();
        for (int32_t l = ti.n_interior; l < ti.n_local; ++l) {
            const int32_t g = l < ti.n_owned ? ti.node_begin + l : ghosts[l - ti.n_owned];
            const int32_t o = T.old_of_new[g];
            const int32_t sid = sid_of_new[g];
            int32_t rank = 0;
            while (ntl[ntp[o] + rank] != t) ++rank;
            T.sh.push_back(make_int4(l, g, T.sptr[sid], (T.sptr[sid + 1] - T.sptr[sid]) | (rank << 16)));
        }
        ti.sh_count = (int32_t)T.sh.size() - ti.sh_begin;

        // owned boundary nodes
        ti.bnd_begin = (int32_t)T.bnd.size();
        if (is_bnd)
            for (int32_t l = 0; l < ti.n_owned; ++l) {
                const int32_t g = ti.node_begin + l;
                if (is_bnd[T.old_of_new[g]]) T.bnd.push_back(make_int2(l, g));
            }
        ti.bnd_count = (int32_t)T.bnd.size() - ti.bnd_begin;

        // reset the local map
        for (int64_t p = tb[t]; p < tb[t + 1]; ++p) {
            const int64_t e = order[p];
            for (int k = 0; k < npe; ++k) loc[conn[npe * e + k]] = -1;
        }
    }
    T.n_chunks = chunk;
    T.chunk_col.assign((size_t)chunk * 2, 0);
    for (int32_t c = 0; c < chunk; ++c) {
        int lo_c = 255, hi_c = 0;
        for (int i = 0; i < CH; ++i) {
            const uint8_t v = T.elem_col[(size_t)c * CH + i];
            if (v == 0xFF) continue;
            lo_c = std::min(lo_c, (int)v);
            hi_c = std::max(hi_c, (int)v);
        }
        if (lo_c > hi_c) lo_c = hi_c = 0;
        T.chunk_col[2 * c] = (uint8_t)lo_c;
        T.chunk_col[2 * c + 1] = (uint8_t)hi_c;
    }
    T.slot_of_elem.assign(ne, -1);
    for (size_t s = 0; s < T.elem_of_slot.size(); ++s)
        if (T.elem_of_slot[s] >= 0) T.slot_of_elem[T.elem_of_slot[s]] = (int64_t)s;

    // node -> (element, local index) incidence in new ids, ascending element order
    T.n2e_ptr.assign(nn + 1, 0);
    for (int64_t e = 0; e < ne; ++e)
        for (int k = 0; k < npe; ++k) ++T.n2e_ptr[T.new_of_old[conn[npe * e + k]] + 1];
    for (int64_t i = 0; i < nn; ++i) T.n2e_ptr[i + 1] += T.n2e_ptr[i];
    T.n2e.resize(T.n2e_ptr[nn]);
    if (T.n2e_ptr[nn] >= (1LL << 31)) return "too many element-node incidences";
    {
        std::vector<int32_t> fill(T.n2e_ptr.begin(), T.n2e_ptr.end() - 1);
        for (int64_t e = 0; e < ne; ++e)
            for (int k = 0; k < npe; ++k) T.n2e[fill[T.new_of_old[conn[npe * e + k]]]++] = (e << 3) | k;
    }
    return "";
}

// Slot gather lists: every list entry names a filled slot of the tile whose position k is the
// list's node, the lists of a tile cover each (slot, k) of the tile exactly once.
static std::string validate_gather(const Tiling &T)
{
    for (int t = 0; t < T.n_tiles; ++t) {
        const TileInfo &ti = T.tiles[t];
        if (ti.gp_begin < 0 || (size_t)ti.gp_begin + ti.n_local >= T.gptr.size()) return "gather list offsets";
        const int64_t n_slots = (int64_t)ti.n_chunks * T.CH;
        std::vector<uint8_t> seen((size_t)n_slots * T.npe, 0);
        for (int32_t l = 0; l < ti.n_local; ++l) {
            const int32_t q0 = T.gptr[ti.gp_begin + l], q1 = T.gptr[ti.gp_begin + l + 1];
            if (q0 > q1 || q0 < 0 || (size_t)q1 > T.gidx.size()) return "gather list range";
            for (int32_t q = q0; q < q1; ++q) {
                const int64_t v = T.gidx[q];
                if (v < 0 || v >= n_slots * T.npe) return "gather entry outside the tile";
                const int64_t s = (int64_t)ti.chunk_begin * T.CH + v / T.npe;
                if (T.elem_of_slot[s] < 0) return "gather entry on a padding slot";
                if (T.lconn[s * T.npe + v % T.npe] != l) return "gather entry of another node";
                if (seen[v]++) return "gather entry twice";
            }
        }
        for (int64_t v = 0; v < n_slots * T.npe; ++v)
            if (T.elem_of_slot[(int64_t)ti.chunk_begin * T.CH + v / T.npe] >= 0 && !seen[v]) return "slot not gathered";
    }
    return "";
}

std::string validate_tiling(const Tiling &T)
{
    if (T.single_class) {
        const std::string g = validate_gather(T);
        if (!g.empty()) return g;
    }
    const int64_t n_slots = T.sptr.empty() ? 0 : T.sptr.back();
    int32_t chunks = 0;
    for (int t = 0; t < T.n_tiles; ++t) {
        const TileInfo &ti = T.tiles[t];
        if (ti.chunk_begin != chunks || ti.n_chunks < 1) return "tile chunk range";
        chunks += ti.n_chunks;
        if (ti.node_begin < 0 || ti.n_interior < 0 || ti.n_interior > ti.n_owned || ti.n_owned > ti.n_local ||
            ti.node_begin + (int64_t)ti.n_owned > T.nn || ti.n_local > T.max_local)
            return "tile node range";
        for (int64_t s = (int64_t)ti.chunk_begin * T.CH; s < (int64_t)(ti.chunk_begin + ti.n_chunks) * T.CH; ++s)
            for (int k = 0; k < T.npe; ++k)
                if (T.lconn[s * T.npe + k] >= ti.n_local) return "local id out of range";
        if (ti.sh_begin < 0 || ti.sh_begin + (int64_t)ti.sh_count > (int64_t)T.sh.size()) return "halo range";
        if (ti.sh_count != ti.n_local - ti.n_interior) return "halo count";
        for (int q = 0; q < ti.sh_count; ++q) {
            const int4 h = T.sh[ti.sh_begin + q];
            const int cnt = h.w & 0xFFFF, rank = h.w >> 16;
            if (h.x != ti.n_interior + q || h.y < 0 || h.y >= T.nn || cnt < 2 || rank >= cnt ||
                h.z < 0 || h.z + (int64_t)cnt > n_slots)
                return "halo entry out of range";
            if (h.x < ti.n_owned && (h.y != ti.node_begin + h.x || rank != 0)) return "owned halo entry";
            if (h.x >= ti.n_owned && rank == 0) return "ghost entry marked as owner";
        }
        if (ti.bnd_begin < 0 || ti.bnd_begin + (int64_t)ti.bnd_count > (int64_t)T.bnd.size()) return "boundary range";
        for (int q = 0; q < ti.bnd_count; ++q) {
            const int2 b = T.bnd[ti.bnd_begin + q];
            if (b.x < 0 || b.x >= ti.n_owned || b.y != ti.node_begin + b.x) return "boundary entry out of range";
        }
    }
    if (chunks != T.n_chunks) return "chunk count";
    if ((int)T.nbr_ptr.size() != T.n_tiles + 1) return "neighbour lists";
    for (int32_t v : T.nbr)
        if (v < 0 || v >= T.n_tiles) return "neighbour id out of range";
    for (int t = 0; t < T.n_tiles; ++t) {
        const TileInfo &ti = T.tiles[t];
        if (ti.n_colors < 1 || ti.col_begin < 0 || ti.col_begin + ti.n_colors >= (int)T.colptr.size() ||
            T.colptr[ti.col_begin] != 0 || T.colptr[ti.col_begin + ti.n_colors] != ti.n_chunks)
            return "colour boundaries";
        for (int c = 0; c < ti.n_colors; ++c) {
            const int u0 = T.colptr[ti.col_begin + c], u1 = T.colptr[ti.col_begin + c + 1];
            if (u1 <= u0) return "empty colour class";
            for (int64_t sl = ((int64_t)ti.chunk_begin + u0) * T.CH; sl < ((int64_t)ti.chunk_begin + u1) * T.CH; ++sl)
                if (T.elem_col[sl] != c && T.elem_col[sl] != 0xFF) return "chunk with two colours";
        }
    }
    // a colour class is a set of elements without a common node: the step kernel adds their
    // loads into shared memory without atomics (single-class tiles write per-element slots
    // instead and need no such class; their gather lists were checked above)
    if (!T.single_class) {
        std::vector<int64_t> stamp(T.max_local > 0 ? T.max_local : 1, -1);
        int64_t cls = 0;
        for (int t = 0; t < T.n_tiles; ++t) {
            const TileInfo &ti = T.tiles[t];
            for (int c = 0; c < ti.n_colors; ++c, ++cls) {
                const int u0 = T.colptr[ti.col_begin + c], u1 = T.colptr[ti.col_begin + c + 1];
                for (int64_t sl = ((int64_t)ti.chunk_begin + u0) * T.CH; sl < ((int64_t)ti.chunk_begin + u1) * T.CH;
                     ++sl) {
                    if (T.elem_col[sl] == 0xFF) continue;
                    for (int k = 0; k < T.npe; ++k) {
                        const int l = T.lconn[sl * T.npe + k];
                        if (l >= (int)stamp.size()) return "local id out of range";
                        if (stamp[l] == cls) return "two elements of one colour class share a node";
                        stamp[l] = cls;
                    }
                }
            }
        }
    }
    if (T.elem_col.size() != (size_t)T.n_chunks * T.CH || T.chunk_col.size() != (size_t)T.n_chunks * 2)
        return "colour arrays";
    for (int64_t e = 0; e < T.ne; ++e)
        if (T.slot_of_elem[e] < 0 || T.elem_of_slot[T.slot_of_elem[e]] != e) return "element slot map";
    return "";
}

void build_face_csr(int64_t nn, const std::vector<int32_t> &new_of_old, const int32_t *faces,
                    int64_t n_faces, int nv, std::vector<int32_t> &ptr, std::vector<int32_t> &idx)
{
    ptr.assign(nn + 1, 0);
    for (int64_t f = 0; f < n_faces; ++f)
        for (int k = 0; k < nv; ++k) ++ptr[new_of_old[faces[nv * f + k]] + 1];
    for (int64_t i = 0; i < nn; ++i) ptr[i + 1] += ptr[i];
    idx.resize(ptr[nn]);
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t f = 0; f < n_faces; ++f)
        for (int k = 0; k < nv; ++k) idx[fill[new_of_old[faces[nv * f + k]]]++] = (int32_t)f;
}

}  // namespace fedfem
