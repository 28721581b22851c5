// Internal declarations of libfedfem.so (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fedfem.h"
#include "law.cuh"

namespace fedfem {

// Pair order of the 28 (hex) / 6 (tet) off-diagonal conductances c_ij = -K0_e[i][j], i < j,
// enumerated row by row: (0,1) (0,2) ... (0,n-1) (1,2) ...  The diagonal follows from the zero
// row sums of K0_e (a constant field carries no heat), so F_i = sum_j c_ij (T_i - T_j).
constexpr int n_pairs(int npe) { return npe * (npe - 1) / 2; }

// Device error word bits.
enum : int32_t {
    ERRBIT_DIVERGED = 1,
    ERRBIT_TIMEOUT = 2,
    ERRBIT_MESH = 4,
    ERRBIT_BOUNDS = 8,
};

// One element tile: a contiguous run of chunks of the element stream plus the nodes it
// touches.  Local node numbering inside a tile: [interior | owned-shared | ghosts];
// interior and owned-shared nodes are the contiguous global range node_begin + local.
struct TileInfo {
    int32_t chunk_begin, n_chunks;
    int32_t node_begin, n_interior, n_owned, n_local;
    int32_t sh_begin, sh_count;      // shared entries (owned-shared and ghosts)
    int32_t bnd_begin, bnd_count;    // owned boundary nodes (surface loads)
    int32_t col_begin, n_colors;     // colour classes: chunks colptr[col_begin + c] .. [.. + c + 1]
    int32_t scenario;                // index into the physics table (batched scenarios)
    int32_t gp_begin;                // slot gather: the tile's node list offsets start at gptr[gp_begin]
    int32_t pad1, pad2;
};

// Physical constants of one problem (one scenario of a batch).
struct PhysParams {
    double k_lin, c_lin, h, T_inf, eps_sigma, T_amb, T_zero, T_guard;
    double k_a, c_a;  // f_k = k_a + k_lin T, f_c = c_a + c_lin T (k_a = 1 - k_lin T_ref)
};

// Host-side result of the tiling pass.
struct Tiling {
    int npe = 0, CH = 0, n_tiles = 0, n_chunks = 0, max_local = 0, max_colors = 0;
    int64_t ne = 0, nn = 0;
    std::vector<int32_t> new_of_old, old_of_new;   // node renumbering
    std::vector<TileInfo> tiles;
    std::vector<int32_t> elem_of_slot;             // [n_chunks*CH], -1 for padding
    std::vector<int64_t> slot_of_elem;             // [ne]
    std::vector<uint16_t> lconn;                   // [n_chunks*CH][npe] tile-local node ids
    std::vector<uint8_t> elem_col;                 // [n_chunks*CH] colour, 0xFF for padding
    std::vector<uint8_t> chunk_col;                // [n_chunks][2] (first, last colour)
    std::vector<int4> sh;                          // {local, gid, first slot, count | rank << 16}
    std::vector<int32_t> sptr;                     // [n_shared+1] halo slot ranges
    std::vector<int2> bnd;                         // {local, gid} owned boundary nodes
    std::vector<int32_t> colptr;                   // per tile: first chunk of each colour class
    std::vector<int32_t> nbr_ptr, nbr;             // per tile: tiles sharing a node (CSR)
    // slot gather (single-class tiles): per tile and local node, the element slots that touch
    // the node, ascending: gidx[gptr[gp_begin + l] .. gptr[gp_begin + l + 1]) = slot * npe + k
    // (slot relative to the tile's first chunk)
    bool single_class = false;
    int max_chunks = 0;                            // most chunks of one tile
    std::vector<int32_t> gptr, gidx;
    // incidence (new node ids), ascending element / face order inside each list
    std::vector<int32_t> n2e_ptr;                  // [nn+1]
    std::vector<int64_t> n2e;                      // (e << 3) | k
};

// Build the tiling.  conn [ne][npe] original ids; is_bnd [nn] (original ids) marks nodes
// with surface loads.  Returns "" on success, else a message.
// single_class: one class per tile (no colouring; chunks in Morton order) and the slot gather
// lists of every tile, for the slot-gather accumulation.
std::string build_tiling(int npe, int64_t ne, int64_t nn, const int32_t *conn, const double *xyz,
                         const uint8_t *is_bnd, int n_tiles, int CH, Tiling &out, bool single_class = false);

// Tiling of a batch of independent meshes packed one after the other: elements
// [group_elem[g], group_elem[g+1]) form scenario g and get tiles_per_group[g] tiles of their
// own (tiles never span scenarios); tiles, chunks and node numbers follow the group order.
std::string build_tiling_groups(int npe, int64_t ne, int64_t nn, const int32_t *conn, const double *xyz,
                                const uint8_t *is_bnd, const std::vector<int64_t> &group_elem,
                                const std::vector<int> &tiles_per_group, int CH, Tiling &out,
                                bool single_class = false);

// Check every index the step kernel will use against its buffers ("" if all in range).
std::string validate_tiling(const Tiling &T);

// Node -> face incidence CSR in new node ids (faces in ascending order).
void build_face_csr(int64_t nn, const std::vector<int32_t> &new_of_old, const int32_t *faces,
                    int64_t n_faces, int nv, std::vector<int32_t> &ptr, std::vector<int32_t> &idx);

// A device allocation owned by a context.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Ctx;
struct Batch;

// Parameters of the persistent time-step kernel.
struct StepArgs {
    const uint8_t *chunks;      // element stream: [n_chunks][chunk_bytes]
    const TileInfo *tiles;
    const int4 *sh;
    const int32_t *sptr;
    const int2 *bnd;
    const void *bnd_area;       // per boundary entry (A^c, A^r) of its node, working precision
    const int32_t *colptr;      // tile-relative chunk offsets of the colour classes
    const int32_t *gptr, *gidx; // slot gather lists (SCATTER = slots)
    void *T[2];                 // Real [nn]
    float *comp[2];             // [nn] (FP32 + Kahan)
    const double *A;            // [nn] dt / C0 (-0.0 on Dirichlet nodes: the sign bit marks them), FP64 form
    const float2 *A2;           // [nn] the same as a float pair (hi, lo), FP32 form
    const void *Qext;           // Real [nn]
    const void *Ac;             // Real [nn]
    const void *Ar;             // Real [nn]
    void *part[2];              // Real [n_slots] halo partial sums, step parity
    unsigned int *tile_done;    // [n_tiles] progress_base + steps completed by each tile in this launch
    uint32_t progress_base;     // counter value at launch start (the counters only grow between resets)
    const int32_t *nbr_ptr;     // tile neighbours (CSR over tiles)
    const int32_t *nbr;
    int32_t *err;               // device error word
    // time-dependent loads (NULL: constant): external-load multiplier, convection ambient
    // temperature and offset of the prescribed temperatures per global step, the last entry
    // held beyond sched_len
    const double *sched_q, *sched_Tinf, *sched_Tdir;
    int64_t sched_len;
    // tabulated f_k, f_c (used by the kernels instantiated for tables instead of the linear
    // laws of PhysParams): working-precision copies for the FP32 and FP64 forms
    HingeLaw<float> tk32, tc32;
    HingeLaw<double> tk64, tc64;
    // physics: one table entry per scenario, selected by TileInfo::scenario
    const PhysParams *phys;
    // CTA c processes tiles [cta_tile[c], cta_tile[c + 1]) (NULL: tiles_per_cta consecutive tiles)
    const int32_t *cta_tile;
    // launch
    int64_t n0;                 // global step index at launch start
    int32_t nsteps;
    int32_t n_tiles, tiles_per_cta;
    int32_t chunk_bytes, stages, chunk, colour_offset;
    uint64_t stage_magic;       // ceil(2^64 / stages): k / stages = high 64 bits of k * stage_magic
    int32_t l2_stream_policy;   // 0: evict_normal, 1: evict_first for the element stream
    int32_t scatter;
    int32_t withhold;           // test hook: CTA withhold-1 skips its first barrier arrival
    long long stagger_ns;       // consumers of CTA b start the launch stagger_ns * b / grid late
    // energy audit (non-NULL energy_acc selects the audit instantiation): per-CTA running sums
    // [grid][2] (stored heat change, boundary input), lumped masses at f_c = 1, the time step
    double *energy_acc;
    const double *C0;
    double dt;
    long long timeout_ns;
    // optional per-step recording of the state (adjoint segments): rec + s*rec_stride
    void *rec;
    int64_t rec_stride;
};

// Launchers (step.cu).  Return cudaError_t of the launch.
cudaError_t launch_step(const StepArgs &a, int precision, int kahan, int npe, int table, int grid, int block,
                        size_t smem, int ts_cap, cudaStream_t st);
cudaError_t prepare_step(int precision, int kahan, int npe, int scatter, int table, size_t smem);
size_t step_smem_bytes(int precision, int npe, int chunk, int stages, int max_local, int slot_cap = 0);
// (A^c, A^r) of the node of every boundary entry, gathered once after the pre-computation
cudaError_t launch_bnd_areas(int precision, int64_t n, const int2 *bnd, const void *Ac, const void *Ar, void *out,
                             cudaStream_t st);
int step_ts_cap(int precision, int max_local);
int step_max_blocks_per_sm(int precision, int kahan, int npe, int block, size_t smem);
int chunk_bytes_for(int precision, int npe, int CH);
int chunk_colour_offset(int precision, int npe, int CH);
int chunk_header_offset(int precision, int npe, int CH);
constexpr int NODE_PAD = 16;    // node arrays carry this many trailing pad entries (aligned bulk copies)

}  // namespace fedfem
