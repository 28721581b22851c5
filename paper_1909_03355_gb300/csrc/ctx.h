// The context behind the opaque fedfem_ctx handle.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fedfem_internal.h"
#include "precompute.cuh"

struct fedfem_ctx {
    // problem (host copies, original numbering)
    int npe = 8;
    int64_t nn = 0, ne = 0;
    std::vector<double> xyz, kscale, source, nodal_Q, dir_T;
    bool params_on_device = false;  // kscale / source last set from device arrays (d_kscale, d_source)
    std::vector<int32_t> conn, elem_mat, dir_nodes, conv_faces, rad_faces;
    std::vector<fedfem_material> mats;
    int face_nv = 4;
    int64_t n_conv = 0, n_rad = 0;
    double h = 0, T_inf = 0, eps = 0, T_amb = 0, T_zero = -273.15;
    double k_lin = 0, c_lin = 0, T_ref = 0;  // f_k = 1 + k_lin (T - T_ref), f_c likewise
    double k_a() const { return 1.0 - k_lin * T_ref; }  // f_k = k_a + k_lin T
    double c_a() const { return 1.0 - c_lin * T_ref; }
    // tabulated factors (fedfem_set_property_table): replace the linear laws when n_tab > 0
    int n_tab = 0;
    std::vector<double> tab_T, tab_fk, tab_fc;
    fedfem::HingeLaw<double> hk{}, hc{};
    const fedfem::HingeLaw<double> *tk_ptr() const { return n_tab ? &hk : nullptr; }
    double fk(double T) const { return n_tab ? fedfem::hinge_value(hk, T) : 1.0 + k_lin * (T - T_ref); }
    double fc(double T) const { return n_tab ? fedfem::hinge_value(hc, T) : 1.0 + c_lin * (T - T_ref); }
    // extrema of f_k and f_c over [lo, hi]: at the ends or at table points inside
    void law_extrema(double lo, double hi, double *fk_max, double *fk_min, double *fc_min) const
    {
        double kx = std::max(fk(lo), fk(hi)), kn = std::min(fk(lo), fk(hi)), cn = std::min(fc(lo), fc(hi));
        for (int j = 0; j < n_tab; ++j)
            if (tab_T[j] > lo && tab_T[j] < hi) {
                kx = std::max(kx, tab_fk[j]);
                kn = std::min(kn, tab_fk[j]);
                cn = std::min(cn, tab_fc[j]);
            }
        *fk_max = kx;
        *fk_min = kn;
        *fc_min = cn;
    }
    // time-dependent loads: at step n the external loads are sched_q[n] Q_ext, the convection
    // ambient temperature is sched_Tinf[n] and the prescribed temperatures are dir_T +
    // sched_Tdir[n] (last entry beyond the end)
    std::vector<double> sched_q, sched_Tinf, sched_Tdir;
    double *d_sched_q = nullptr, *d_sched_Tinf = nullptr, *d_sched_Tdir = nullptr;
    int64_t sched_len = 0, sched_cap = 0;
    double Tdir_at(int64_t n) const
    {
        return sched_Tdir.empty() ? 0.0
                                  : sched_Tdir[(size_t)std::max<int64_t>(0, std::min<int64_t>(n, sched_len - 1))];
    }
    double qs_at(int64_t n) const
    {
        return sched_q.empty() ? 1.0 : sched_q[(size_t)std::max<int64_t>(0, std::min<int64_t>(n, sched_len - 1))];
    }
    double Tinf_at(int64_t n) const
    {
        return sched_Tinf.empty() ? T_inf
                                  : sched_Tinf[(size_t)std::max<int64_t>(0, std::min<int64_t>(n, sched_len - 1))];
    }
    fedfem_options opt;
    int precision = 32, kahan = 1;
    int scatter_mode = 0;  // accumulation the plan chose: FEDFEM_SCATTER_COLOR, _ATOMIC or _SLOTS

    std::vector<int64_t> group_elem;  // batched scenarios: element range of each packed mesh

    // launch plan
    fedfem::Tiling til;
    int grid = 0, block = 0, stages = 0, tpc = 0, chunk_bytes = 0, chunk = 0, ts_cap = 0;
    size_t smem = 0;
    int device = -1, num_sms = 0, max_smem = 0;
    cudaStream_t stream = nullptr;

    // device arrays (new node numbering unless noted)
    std::vector<void *> allocs;
    uint8_t *d_chunks = nullptr;
    fedfem::TileInfo *d_tiles = nullptr;
    int4 *d_sh = nullptr;
    int32_t *d_sptr = nullptr;
    int2 *d_bnd = nullptr;
    void *d_bnd_area = nullptr;  // (A^c, A^r) per boundary entry, working precision
    int32_t *d_colptr = nullptr;
    int32_t *d_gptr = nullptr, *d_gidx = nullptr;  // slot gather lists (single-class tiling)
    int32_t *d_nbr_ptr = nullptr, *d_nbr = nullptr;
    unsigned int *d_tile_done = nullptr;
    uint32_t progress_base = 0;  // tile progress counters at the next launch's start (below 2^31)
    long long stagger_ns = 0;    // start stagger of the last CTA of a launch (launches of >= 8 steps)
    double *d_energy_acc = nullptr;  // energy audit: per-CTA running sums [grid][2]
    int64_t energy_steps = 0;        // steps summed there since the last set_T / set_state
    fedfem::PhysParams *d_phys = nullptr;
    int32_t *d_cta_tile = nullptr;  // NULL: tiles_per_cta consecutive tiles per CTA
    void *d_T[2] = {nullptr, nullptr};
    float *d_comp[2] = {nullptr, nullptr};
    void *d_part[2] = {nullptr, nullptr};
    float2 *d_A2 = nullptr;
    double *d_A = nullptr, *d_C0 = nullptr, *d_Qext64 = nullptr, *d_Ac64 = nullptr, *d_Ar64 = nullptr;
    void *d_Qext = nullptr, *d_Ac = nullptr, *d_Ar = nullptr;
    uint8_t *d_isdir = nullptr;
    int32_t *d_dir_new = nullptr;
    double *d_dir_T = nullptr;
    int32_t *d_err = nullptr;
    unsigned long long *d_bad_elem = nullptr;
    // pre-computation inputs (original numbering for elements)
    double *d_xyz = nullptr, *d_matk0 = nullptr, *d_matrhoc = nullptr, *d_kscale = nullptr, *d_source = nullptr;
    double *d_nodalQ = nullptr;
    int32_t *d_conn = nullptr, *d_gconn = nullptr, *d_mat = nullptr, *d_old_of_new = nullptr;
    int64_t *d_slot_of_elem = nullptr, *d_n2e = nullptr;
    int32_t *d_n2e_ptr = nullptr;
    double *d_cond64 = nullptr, *d_W = nullptr;
    int32_t *d_conv_faces = nullptr, *d_rad_faces = nullptr;
    int32_t *d_fc_ptr = nullptr, *d_fc_idx = nullptr, *d_fr_ptr = nullptr, *d_fr_idx = nullptr;
    double *d_fc_share = nullptr, *d_fr_share = nullptr;
    // FP64 scratch
    double *d_v[4] = {nullptr, nullptr, nullptr, nullptr};
    double *d_Y = nullptr, *d_red = nullptr;

    // state
    bool precomputed = false, has_dt = false, has_T = false;
    double dt = 0, dt_crit = 0, T_lo = 0, T_hi = 0, lambda_cond = 0;
    int power_iters = 0, power_max_iter = 1000;  // Lanczos steps for dt_crit: taken, limit
    double *d_lz = nullptr;                      // [power_max_iter][4] alpha_j, -, beta_j^2, -
    double power_tol = 1e-10;
    int64_t step = 0;
    std::string err;

    // method variants run by plain launches (variant.cu): conductivity at the quadrature points
    // (kT_eval = 1) and consistent integration of the face loads (face_quadrature = 1)
    int kT_qp = 0, face_cons = 0;
    int nq = 0, nfq = 0;                 // quadrature points per element / per boundary face
    double *d_cond_qp64 = nullptr;       // [ne][8][28] pair conductances per 2x2x2 point (hexahedra)
    double *d_vq64 = nullptr;            // [nq * n_pairs][ne] pair conductances per point, FP64 (SoA)
    void *d_vq = nullptr;                // the same in the working precision
    void *d_Yv = nullptr;                // [ne][npe] element loads of a step, working precision
    int32_t *d_cf_new = nullptr, *d_rf_new = nullptr;  // boundary faces in the tiling's node ids
    double *d_Mf64 = nullptr, *d_Wf64 = nullptr;       // [n_conv][nv][nv] face mass, [n_rad][nfq] weights
    void *d_Mf = nullptr, *d_Wf = nullptr;             // the same in the working precision
    void *d_Yf = nullptr;                // [n_conv + n_rad][nv] face loads of a step, working precision
    double *d_Yf64 = nullptr;            // the same in FP64 (energy and load queries)
    bool variant() const { return kT_qp || face_cons; }

    // adjoint record (adjoint.cu)
    std::vector<void *> adj_allocs;
    bool recorded = false;
    int64_t rec_steps = 0, rec_step0 = 0;
    int32_t rec_sample_every = 0, rec_ckpt_every = 0, rec_n_sensors = 0;
    int32_t *d_sensors = nullptr;     // new ids
    void *d_ckpt = nullptr;           // [n_ckpt][state bytes]
    size_t ckpt_bytes = 0;
};

namespace fedfem {
fedfem_status fail(fedfem_ctx *c, fedfem_status s, const std::string &msg);
fedfem_status cuda_fail(fedfem_ctx *c, cudaError_t e, const char *where);
cudaError_t dalloc(fedfem_ctx *c, void **p, size_t bytes);
cudaError_t upload(fedfem_ctx *c, void **p, const void *src, size_t bytes);
fedfem_status fedfem_ctx_init_device(fedfem_ctx *c);
fedfem_status create_ctx(const fedfem_mesh *mesh, const fedfem_material *mats, int32_t n_mats, const fedfem_bcs *bcs,
                         const fedfem_options *opt_in, const std::vector<int64_t> *group_elem, fedfem_ctx **out,
                         std::string &err);
// Largest eigenvalue of the m x m symmetric tridiagonal matrix with diagonal a and squared
// off-diagonal b2 (Sturm bisection).
double tridiag_max_eigenvalue(const std::vector<double> &a, const std::vector<double> &b2, int m);
fedfem_status check_device(fedfem_ctx *c);
fedfem_status run_precompute_arrays(fedfem_ctx *c);
fedfem_status install_T(fedfem_ctx *c, const double *T0_dev_old);
fedfem_status state_f64_new(fedfem_ctx *c, int64_t step, double *dst);
StepArgs step_args(fedfem_ctx *c);
fedfem_status enqueue_steps(fedfem_ctx *c, int64_t n, void *rec, int64_t rec_stride);
// method variants (variant.cu): device arrays at set-up, their pre-computation, n steps by plain
// launches, and the FP64 internal loads / surface loads of a state (new node order)
fedfem_status variant_init(fedfem_ctx *c);
fedfem_status variant_precompute(fedfem_ctx *c);
fedfem_status variant_steps(fedfem_ctx *c, int64_t n);
fedfem_status variant_loads64(fedfem_ctx *c, const double *T_new, int64_t step, double *F_new, double *Qs_new);
}  // namespace fedfem
