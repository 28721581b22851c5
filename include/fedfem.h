/*
 * fedfem.h: C ABI of the GB300 (sm_103a) FED-FEM library, libfedfem.so.
 *
 * FED-FEM is the fast explicit dynamics finite element method for transient heat conduction
 * of Zhang & Chauhan, "Fast explicit dynamics finite element algorithm for transient heat
 * transfer" (arXiv:1909.03355).  The calls follow the paper's problem statement (Section 2,
 * Eq. 1-7) and its three-stage algorithm (Section 3.5, Fig. 1): pre-computation, initialisation
 * and time stepping.
 *
 * Conventions for every call:
 *  - All arrays passed in are caller-owned HOST arrays unless a name ends in `_dev`; the
 *    library copies what it needs during the call and keeps no pointer to them.
 *  - Device memory is allocated and owned by the library (released by *_destroy).
 *  - Node and element ids are 0-based int32; node coordinates are FP64 [n][3] row-major.
 *  - Every call returns a fedfem_status; no exception crosses the ABI.  After an error the
 *    context's message is available from fedfem_error_string().  A device-side failure
 *    (watchdog or wait timeout) leaves the context usable: restore a state and continue.
 *  - Work is enqueued on the stream given in fedfem_options.stream (a cudaStream_t, NULL for
 *    the legacy default stream).  Calls that return data to the host synchronise that stream.
 *  - Temperatures are in the unit of T_zero (deg C by default, T_zero = -273.15).
 *  - Sign convention (a reading of Eq. 2 and Eq. 13): F = K0 T is the positive-semidefinite
 *    conduction load and the update is T <- T + dt (Q - F) / C.
 */
#ifndef FEDFEM_H
#define FEDFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fedfem_ctx fedfem_ctx;
typedef struct fedfem_batch fedfem_batch;

typedef enum {
    FEDFEM_OK = 0,
    FEDFEM_ERR_ARG = 1,         /* invalid argument (NULL pointer, bad size, bad id)          */
    FEDFEM_ERR_MESH = 2,        /* element with det J <= 0 / V <= 0, or a node id out of range */
    FEDFEM_ERR_UNSTABLE = 3,    /* dt > dt_crit without force (Section 3.4, Eq. 29)           */
    FEDFEM_ERR_DIVERGED = 4,    /* watchdog: a temperature became non-finite or > T_guard     */
    FEDFEM_ERR_TIMEOUT = 5,     /* a device-side wait (tile progress, TMA) exceeded its limit */
    FEDFEM_ERR_CUDA = 6,        /* CUDA runtime error                                         */
    FEDFEM_ERR_OOM = 7,         /* device allocation failed                                   */
    FEDFEM_ERR_STATE = 8,       /* call out of order (create -> precompute -> set_dt -> step) */
    FEDFEM_ERR_UNSUPPORTED = 9  /* option combination not supported                           */
} fedfem_status;

/* Precision of the time-stepping hot path (the pre-computation is always FP64). */
enum { FEDFEM_FP32 = 32, FEDFEM_FP64 = 64 };
/* Accumulation of element loads into nodal loads. */
enum {
    FEDFEM_SCATTER_COLOR = 0,   /* deterministic (default): colour phases in shared memory +
                                   fixed-order halo sums; the plan takes the slot gather instead
                                   when the colour classes pad the tiles to >= 1.5x the chunks
                                   their elements need and a tile's element loads fit in 48 KB
                                   of shared memory (many small classes: small tet meshes) */
    FEDFEM_SCATTER_ATOMIC = 1,  /* shared-memory atomics (non-deterministic order), measured variant */
    FEDFEM_SCATTER_SLOTS = 2,   /* deterministic slot gather: one class per tile, element loads
                                   into per-element shared-memory slots, then every node sums its
                                   slots in ascending order (one barrier instead of one per colour) */
    FEDFEM_SCATTER_CLASSES = 3  /* deterministic colour phases, never the slot gather */
};

/* Mesh (Section 2: the domain divided into elements).  nodes_per_elem = 8: trilinear
 * hexahedra in VTK / C3D8 order (bottom face counter-clockwise, then top); 4: linear tets. */
typedef struct {
    int32_t nodes_per_elem;
    int32_t reserved;
    int64_t n_nodes;
    int64_t n_elems;
    const double *xyz;          /* [n_nodes][3]                                           */
    const int32_t *conn;        /* [n_elems][nodes_per_elem]                              */
    const int32_t *elem_mat;    /* [n_elems] material index, or NULL (all material 0)     */
    const double *elem_kscale;  /* [n_elems] conductivity scale theta_e > 0, or NULL (1)  */
} fedfem_mesh;

/* Material (Eq. 1): density rho, conductivity k_ij(T) = k0_ij (1 + k_lin (T - T_ref)) with k0
 * 3x3 symmetric positive definite (row-major), specific heat c(T) = c0 (1 + c_lin (T - T_ref)):
 * k0 and c0 are the values at the reference temperature T_ref, and the laws interpolate
 * linearly between two tabulated points as in Section 4.2.2 (T_ref = 0: k0 (1 + k_lin T)).
 * All materials of one context must share k_lin, c_lin and T_ref. */
typedef struct {
    double rho;
    double k0[9];
    double k_lin;
    double c0;
    double c_lin;
    double T_ref;
} fedfem_material;

/* Boundary conditions and loads (Eq. 3-7).  Faces are boundary faces listed by node ids
 * (4 per quad face of a hex mesh, 3 per triangle of a tet mesh); each face contributes
 * area / n_vertices to each of its nodes (nodal-quadrature lumping). */
typedef struct {
    int64_t n_dir;              /* Eq. 3: Gamma_E                                          */
    const int32_t *dir_nodes;   /* [n_dir]                                                 */
    const double *dir_T;        /* [n_dir] prescribed temperatures T_Gamma                 */
    int64_t n_conv_faces;       /* Eq. 4: Gamma_C, outward flux h (T - T_inf)              */
    const int32_t *conv_faces;  /* [n_conv_faces][face_nv]                                 */
    double h, T_inf;
    int64_t n_rad_faces;        /* Eq. 7: Gamma_R, outward flux sigma eps ((T-T_z)^4 - (T_amb-T_z)^4) */
    const int32_t *rad_faces;   /* [n_rad_faces][face_nv]                                  */
    double eps, T_amb, T_zero;  /* T_zero: absolute zero in the temperature unit (-273.15) */
    int32_t face_nv;            /* 4 (hex meshes) or 3 (tet meshes)                        */
    int32_t reserved;
    const double *nodal_Q;      /* Eq. 5 as concentrated nodal heat flows (W) [n_nodes], or NULL */
    const double *elem_source;  /* Eq. 1 volumetric source Q (W/m^3) [n_elems], or NULL   */
} fedfem_bcs;

/* Options.  Zero-initialised fields select defaults (see fedfem_default_options). */
typedef struct {
    int32_t precision;          /* FEDFEM_FP32 (default) or FEDFEM_FP64                   */
    int32_t kahan;              /* FP32 only: 1 (default) Kahan-compensated T accumulator  */
    int32_t scatter;            /* FEDFEM_SCATTER_COLOR (default), _ATOMIC, _SLOTS or _CLASSES */
    int32_t block;              /* consumer threads per CTA (multiple of 32, <= 480; one producer
                                   warp is added), 0 = auto: 256 for FP64, 480 for FP32
                                   hexahedral meshes whose element stream fits in 64 MB
                                   (with one CTA per SM), else 224                           */
    int32_t steps_per_launch;   /* explicit steps fused in one persistent launch, 0 = auto */
    int32_t ctas_per_sm;        /* resident CTAs per SM, 0 = auto (two for FP32 with at most
                                   224 consumer threads, else one)                           */
    int32_t tiles_per_cta;      /* element tiles per CTA, 0 = auto                          */
    int32_t stages;             /* depth of the element-chunk TMA ring (2..63), 0 = auto     */
    int32_t chunk;              /* elements per TMA chunk, 32 or 64 (one chunk per warp), 0 = auto
                                   (64 for FP32 tets, else 32)                               */
    int32_t l2_policy;          /* element stream L2 policy: 0 = auto, 1 = evict_normal, 2 = evict_first
                                   (node operands are then prefetched evict_last) */
    double barrier_timeout_s;   /* device-side wait limit (default 1.0 s)                   */
    double T_guard;             /* watchdog threshold on |T| (default 1e6)                  */
    void *stream;               /* cudaStream_t, NULL = legacy default stream               */
    int32_t device;             /* CUDA device ordinal, -1 = current device                 */
    int32_t verbose;            /* 1: print the tiling / launch plan to stderr              */
    int32_t debug_withhold_barrier; /* test hook: k > 0 makes CTA k-1 withhold the publication of
                                   its completed steps, so its neighbours' bounded waits run out
                                   and the call returns FEDFEM_ERR_TIMEOUT; 0 = off */
    int32_t quadrature;         /* conduction matrix of hexahedra: 0 or 8 = 2x2x2 Gauss points
                                   (default), 1 = one point at the element centre with weight 8
                                   (Eq. 17, reduced integration without hourglass control: the
                                   element matrix has rank 3).  Lumped masses, source loads and
                                   face areas keep their exact integration.  Ignored for tets;
                                   other values give FEDFEM_ERR_ARG */
    int32_t kT_eval;            /* where k(T) is evaluated: 0 = element mean of the nodal factors
                                   (Section 4.2.2, default); 1 = at the quadrature points (Eq. 20
                                   with D(T) inside the integral: the 2x2x2 points of a hexahedron,
                                   its centre with quadrature = 1, the centroid of a tet) */
    int32_t face_quadrature;    /* surface loads of Eq. 4 / 7: 0 = nodal lumping of the face areas
                                   (default); 1 = consistent integration over every boundary face
                                   (face mass matrices for convection; radiation by 3x3 Gauss points
                                   on quadrilaterals, Radon's 7-point degree-5 rule on triangles).
                                   With either variant the step runs as three plain launches per
                                   step (elements, faces, nodes; deterministic gathers) instead of
                                   the persistent kernel; fedfem_energy, the adjoint, batches and
                                   the domain decomposition then return FEDFEM_ERR_UNSUPPORTED */
    int32_t reserved2;
    double start_stagger_us;    /* staggered start of the persistent launch (launches of >= 8 steps):
                                   the consumers of CTA b begin stagger * b / grid us late (at most
                                   1000 us), which spreads the CTAs' element and node phases in time
                                   from the first step.  <= 0 = off (default) */
    int32_t energy_audit;       /* 1: the step kernel also accumulates, in FP64, the stored-heat
                                   change and the boundary input of every step (an instantiation
                                   of the kernel with the extra work; colour scatter, linear laws,
                                   FP32 + Kahan or FP64); read by fedfem_energy_totals.  0 = off */
    int32_t reserved3;
} fedfem_options;

/* Fill *opt with defaults (FP32 + Kahan, colour scatter, automatic launch plan). */
void fedfem_default_options(fedfem_options *opt);

/*
 * Create a context: validates the problem (ids in range, one conductivity/heat law), copies
 * it, builds the element tiling (space-filling-curve tiles, node renumbering, element
 * colouring) on the host and allocates the device arrays.  Fig. 1 (i) 1 ("load object mesh
 * and boundary conditions").  *out is NULL on failure.
 * Errors: ARG (NULL / sizes / ids / laws), OOM, CUDA, UNSUPPORTED.
 */
fedfem_status fedfem_create(const fedfem_mesh *mesh, const fedfem_material *mats, int32_t n_mats,
                            const fedfem_bcs *bcs, const fedfem_options *opt, fedfem_ctx **out);

/*
 * Pre-computation stage, Fig. 1 (i) 2-3, in FP64 on the device: element conduction matrices
 * K0_e (Eq. 12 with 2x2x2 Gauss points for hexahedra, Eq. 18 for tets; the paper's G of
 * Eq. 19/22 folded with D into 28 / 6 pair conductances), lumped thermal masses (Eq. 14/21),
 * constant nodal loads and surface area shares; then the critical time step of Section 3.4
 * (Eq. 29): dt_crit = 2 / lambda with lambda from FP64 power iteration on C0^-1/2 K0 C0^-1/2,
 * scaled by max f_k / min f_c over [T_lo, T_hi], plus the largest linearised surface rate
 * (h + 4 sigma eps max|T - T_z|^3) A_i / (C0_i min f_c).
 * dt_crit_out may be NULL.  Errors: MESH (det J <= 0; the message names the element), CUDA.
 */
fedfem_status fedfem_precompute(fedfem_ctx *ctx, double T_lo, double T_hi, double *dt_crit_out);

/* Set the time step (Eq. 8) and the coefficient A = dt / C0 of Eq. 14/21 (0 on Gamma_E).
 * Errors: ARG (dt <= 0), UNSTABLE (dt > dt_crit and force == 0), STATE (before precompute). */
fedfem_status fedfem_set_dt(fedfem_ctx *ctx, double dt, int32_t force);

/* Initialisation stage, Fig. 1 (ii): T0 [n_nodes] host FP64; T_Gamma is re-imposed on the
 * Dirichlet nodes and the step counter is reset to 0.  Errors: ARG, STATE. */
fedfem_status fedfem_set_T(fedfem_ctx *ctx, const double *T0);

/* Same as fedfem_set_T with a DEVICE array T0_dev [n_nodes] (FP64, original node order). */
fedfem_status fedfem_set_T_device(fedfem_ctx *ctx, const double *T0_dev);

/*
 * Time-stepping stage, Fig. 1 (iii), n_steps times: element loads F_e = theta_e f_k,e K0_e T_e
 * (Eq. 20 with the element-mean conductivity law of Section 4.2.2), accumulated to nodes in a
 * fixed order, surface loads (Eq. 4, 7), explicit update (Eq. 16) and Dirichlet nodes held
 * fixed (Fig. 1 (iii) 2.3).  Launches persistent kernels of up to steps_per_launch steps on
 * the context stream and synchronises once at the end to read the device status word.
 * Errors: STATE (no dt / no T), DIVERGED, TIMEOUT, CUDA.
 */
fedfem_status fedfem_step(fedfem_ctx *ctx, int64_t n_steps);

/*
 * n_steps explicit steps with the time step adapted per launch (Section 3.4 evaluated on the
 * run): before every launch of up to steps_per_launch steps the current field's range
 * [min T - margin, max T + margin] gives dt_crit (lambda_cond from fedfem_precompute, the
 * f_k / f_c extrema and the surface rate over that range) and dt = safety dt_crit.  Nonlinear
 * runs whose temperatures leave the range given to fedfem_precompute stay stable without a
 * guessed upper bound.  *t_elapsed (may be NULL) receives the simulated time.  The context's dt
 * is the last launch's.  0 < safety <= 1, margin >= 0 (deg C).
 * Errors: ARG, STATE (no precompute / no T), DIVERGED, TIMEOUT, CUDA.
 */
fedfem_status fedfem_step_adaptive(fedfem_ctx *ctx, int64_t n_steps, double safety, double margin,
                                   double *t_elapsed);

/* Enqueue n_steps on the stream without synchronising; the device status is checked by the
 * next synchronising call (fedfem_sync, fedfem_get_T, fedfem_step).  Errors: STATE, CUDA. */
fedfem_status fedfem_step_async(fedfem_ctx *ctx, int64_t n_steps);

/* Wait for the context stream and report the device status word.  Errors as fedfem_step. */
fedfem_status fedfem_sync(fedfem_ctx *ctx);

/* Copy the current temperatures to T_host [n_nodes] FP64 (original node order).  In FP32 +
 * Kahan mode the value is T_hi - compensation evaluated in FP64. */
fedfem_status fedfem_get_T(fedfem_ctx *ctx, double *T_host);

/* Same into a DEVICE array T_dev [n_nodes] FP64 (original node order), stream-ordered. */
fedfem_status fedfem_get_T_device(fedfem_ctx *ctx, double *T_dev);

/* Number of explicit steps taken since the last set_T / set_state. */
fedfem_status fedfem_get_step(fedfem_ctx *ctx, int64_t *step);

/*
 * Energy balance of the most recent step n-1 -> n, in FP64 (a consequence of Eq. 11: the
 * internal loads sum to zero over all nodes):
 *   stored_change = sum_free C0_i f_c(T_i^{n-1}) (T_i^n - T_i^{n-1}),
 *   boundary_in   = dt (sum_free Q_i(T^{n-1}) + sum_Dirichlet F_i(T^{n-1})).
 * Errors: STATE (no step taken yet).
 */
fedfem_status fedfem_energy(fedfem_ctx *ctx, double *stored_change, double *boundary_in);

/* Internal conduction loads F = sum_e theta_e f_k,e K0_e T_e (Eq. 11/20) for a given field,
 * evaluated in FP64 from the stored (working-precision) element operators.  T_host, F_host:
 * [n_nodes] FP64, original order. */
fedfem_status fedfem_internal_loads(fedfem_ctx *ctx, const double *T_host, double *F_host);

/*
 * Replace the per-element conductivity scales theta_e and / or volumetric sources s_e
 * (NULL keeps the current values) and redo the dependent pre-computation (element operators,
 * nodal loads).  The time step and dt_crit are left unchanged.  Arrays: [n_elems] FP64 host.
 */
fedfem_status fedfem_set_params(fedfem_ctx *ctx, const double *kscale, const double *source);
/* The same with DEVICE arrays [n_elems] (e.g. torch tensors), copied on the context's stream;
 * kscale is checked (smallest value > 0, largest finite) from a few partial minima and maxima
 * read back, not from the array.  Errors: ARG (kscale not > 0), STATE, CUDA. */
fedfem_status fedfem_set_params_device(fedfem_ctx *ctx, const double *kscale_dev, const double *source_dev);

/*
 * Time-dependent loads and prescribed temperatures (the paper's boundary data are constant;
 * Eq. 3-7 with time-varying data): at step n (the global step counter, 0 after fedfem_set_T)
 * the constant external loads Q_ext (sources and nodal heat flows) are multiplied by
 * q_scale[n], the convection ambient temperature is T_inf[n], and every Dirichlet node holds
 * its dir_T value plus T_dir[n]; beyond n_entries - 1 the last entries hold.  Step n is the
 * step from T^n to T^(n+1).  Any array may be NULL (that term stays constant); n_entries = 0
 * removes the schedule.  fedfem_set_T imposes the Dirichlet values of step 0; when a field is
 * already installed and the Dirichlet offsets change, this call sets them to those of the
 * current step.  During the steps a Dirichlet node moves by T_dir[n+1] - T_dir[n] each step, so
 * it follows T_dir up to the rounding of the working precision.  The adjoint and fedfem_energy
 * use the same per-step values.  Arrays: [n_entries] FP64 host, copied.  Synchronises the
 * context's stream.
 * Errors: ARG (n_entries < 0, all arrays NULL, non-finite entries), UNSUPPORTED (batches), CUDA.
 */
fedfem_status fedfem_set_schedule(fedfem_ctx *ctx, int64_t n_entries, const double *q_scale, const double *T_inf,
                                  const double *T_dir);

/*
 * Tabulated property factors (Section 4.2.2 interpolates k and c linearly between the
 * temperatures at which they are given): f_k = k / k0 and f_c = c / c0 at the n_points
 * increasing temperatures T, linear between neighbouring points and held at the end values
 * outside the table.  As in Section 4.2.2, k enters an element as the mean of its nodal
 * factors f_k(T_i); c enters each node's lumped capacity as f_c(T_i).  The table replaces the
 * materials' linear laws (k_lin, c_lin, T_ref) in the time steps, dt_crit (extrema of the
 * factors over [T_lo, T_hi]: at the ends or at table points inside), fedfem_step_adaptive,
 * fedfem_energy, fedfem_internal_loads and the adjoint.  n_points = 0 removes it.  Arrays:
 * [n_points] FP64 host, copied.  Must precede fedfem_precompute.
 * Errors: ARG (n_points not 0 or 2..8, NULL arrays, temperatures not finite and increasing,
 * factors not finite and > 0), STATE (after fedfem_precompute), UNSUPPORTED (batches).
 */
fedfem_status fedfem_set_property_table(fedfem_ctx *ctx, int32_t n_points, const double *T, const double *fk,
                                        const double *fc);

/* Checkpoint / resume: the state is (T, Kahan compensation, step counter).  state_bytes
 * returns the size of the opaque blob; get/set copy it to/from a host buffer. */
fedfem_status fedfem_state_bytes(fedfem_ctx *ctx, size_t *bytes);
fedfem_status fedfem_get_state(fedfem_ctx *ctx, void *buf);
fedfem_status fedfem_set_state(fedfem_ctx *ctx, const void *buf);

/*
 * Forward run for the adjoint (no counterpart in the paper): n_steps explicit steps from the
 * current state, writing T at the sensor nodes after every sample_every-th step into
 * trace [n_steps / sample_every][n_sensors] (FP64 host) and keeping device checkpoints of the
 * state every ckpt_every steps for fedfem_adjoint.  n_steps must be a multiple of both.
 * Errors: ARG, STATE, DIVERGED, TIMEOUT, CUDA, OOM.
 */
fedfem_status fedfem_forward_record(fedfem_ctx *ctx, int64_t n_steps, const int32_t *sensors,
                                    int32_t n_sensors, int32_t sample_every, int32_t ckpt_every,
                                    double *trace);
/* The same with the trace written to a DEVICE array (sensors stay a host array). */
fedfem_status fedfem_forward_record_device(fedfem_ctx *ctx, int64_t n_steps, const int32_t *sensors,
                                           int32_t n_sensors, int32_t sample_every, int32_t ckpt_every,
                                           double *trace_dev);

/*
 * Reverse-time discrete adjoint of the recorded forward run (derived from Eq. 16 and Eq. 20;
 * the paper has no adjoint).  dL_dtrace [n_samples][n_sensors] FP64 host; outputs
 * dL_dkscale, dL_dsource [n_elems] FP64 host (original element order).  Each checkpoint
 * segment is recomputed forward bit-identically before the backward sweep.  The state after
 * the call is the state at the end of the recorded run.
 * Errors: STATE (no recorded run), ARG, CUDA, OOM.
 */
fedfem_status fedfem_adjoint(fedfem_ctx *ctx, const double *dL_dtrace, double *dL_dkscale,
                             double *dL_dsource);
/* The same with DEVICE input and outputs.  On a GPU that can keep all the sweep's blocks
 * resident, each checkpoint segment's reverse steps run in one cooperative launch with grid
 * barriers (bounded waits, FEDFEM_ERR_TIMEOUT when one runs out) between the element and node
 * passes; otherwise the passes are separate launches (same results). */
fedfem_status fedfem_adjoint_device(fedfem_ctx *ctx, const double *dL_dtrace_dev, double *dL_dkscale_dev,
                                    double *dL_dsource_dev);

/*
 * Cumulative energy balance since the last fedfem_set_T / fedfem_set_T_device / fedfem_set_state
 * (contexts created with energy_audit = 1): the sums over all steps taken since then of the
 * stored-heat change sum_free C0_i f_c(T_i^n) (T_i^{n+1} - T_i^n) and of the boundary input
 * dt (sum_free Q_i^n + sum_Dirichlet F_i^n), both accumulated in FP64 by the step kernel from the
 * working-precision state (values with their Kahan compensation) and loads; n_steps = steps
 * summed.  Energy conservation of the scheme (the internal loads sum to zero) makes the two
 * equal up to rounding.  Synchronises the stream.  Errors: UNSUPPORTED (no audit), CUDA.
 */
fedfem_status fedfem_energy_totals(fedfem_ctx *ctx, double *stored_change, double *boundary_in, int64_t *n_steps);

/* Physical constants of the energy-balance terms (the context's values for fedfem_energy). */
typedef struct {
    double dt, c_lin, h, T_inf, eps, T_amb, T_zero, T_ref;
} fedfem_energy_params;

/*
 * Energy-balance sums of one step for callers that cannot allocate device memory (no
 * counterpart in the paper; the sums are those of fedfem_energy).  Meant for code that must not
 * call cudaMalloc / cudaFree: a callback running while another library owns the device memory
 * pool, a process under a hard device-memory budget, or a loop that must not synchronise the
 * device.  It allocates nothing: its only scratch (one pair of partial sums per 4096 nodes) is a
 * 64 KB array compiled into the library, which every GPU that loads the library keeps until the
 * process exits.
 *   n_nodes <= 16,777,216 (larger: FEDFEM_ERR_ARG);  all arrays are DEVICE arrays of n_nodes
 *   entries in one common node order: T_prev, T_next (FP64 states of two consecutive steps),
 *   F (internal loads at T_prev, e.g. from fedfem_internal_loads), C0 (lumped thermal mass at
 *   f_c = 1), Qext, Ac, Ar (constant nodal loads and convection / radiation area shares) and
 *   is_dirichlet (1 on Gamma_E);  out: DEVICE array of 2 doubles receiving
 *   (stored_change, boundary_in);  stream: cudaStream_t or NULL.  Asynchronous on `stream`.
 * The capacity factor is the linear law of params (c_lin, T_ref); a context with a property
 * table gets its sums from fedfem_energy.  With a load schedule, pass the data of the step the
 * sums describe: Qext already multiplied by that step's load factor and T_inf that step's
 * convection temperature.
 * All calls on a device share the scratch array: calls that overlap on the GPU race.  Each call
 * overwrites every partial it reads, so nothing needs clearing between calls.  The first call
 * on a device looks the array's address up (cudaGetSymbolAddress) with that device current:
 * make it before any stream capture.  That address is kept for the life of the process, so
 * the entry point must not be used on a device after cudaDeviceReset (a reset primary context
 * reloads the library's device code).  Launch errors are those of this call's own launches.
 * Errors: ARG (NULL pointer, n_nodes out of range), CUDA.
 */
fedfem_status fedfem_energy_terms_noalloc(int64_t n_nodes, const double *T_prev, const double *T_next,
                                          const double *F, const double *C0, const double *Qext,
                                          const double *Ac, const double *Ar, const uint8_t *is_dirichlet,
                                          const fedfem_energy_params *params, double *out, void *stream);

/* Launch plan and sizes chosen by create: a fixed-size record for logging and benchmarks. */
typedef struct {
    int64_t n_nodes, n_elems;
    int32_t n_tiles, grid, block, stages, chunk, scatter;  /* scatter: the accumulation in use
                                                            (FEDFEM_SCATTER_COLOR, _ATOMIC, _SLOTS) */
    int32_t steps_per_launch, max_tile_nodes, n_colors_max, smem_bytes;
    int64_t n_shared_nodes, n_halo_slots, elem_bytes;   /* element stream bytes per step */
    double dt, dt_crit;
} fedfem_info;
fedfem_status fedfem_get_info(fedfem_ctx *ctx, fedfem_info *info);

/*
 * Host-only check of the element tiling the step kernel would use (no device call, no GPU
 * needed): validates the mesh as fedfem_create does, cuts it into n_tiles tiles (Morton order,
 * equal element counts) of `chunk`-element chunks (32 or 64), colours every tile and checks
 * every index the kernel would read: tile node ranges, tile-local element ids, halo entries and
 * their partial-load slots, boundary entries, and colour classes whose elements share no node.
 * single_class = 1 builds the tiles of the slot-gather accumulation instead (one class per
 * tile, chunks in Morton order) with their gather lists, and checks that every element slot
 * position is gathered exactly once by the node it belongs to.
 * For checking a mesh before it goes to a GPU, and for host-side tests of the tiling.
 *   mesh: as for fedfem_create (elem_mat and elem_kscale are not used);
 *   boundary_nodes [n_boundary] (nodes with surface loads) or NULL;  stats: out, or NULL.
 * Errors: ARG (bad mesh, sizes or boundary ids), MESH (the tiling or its check failed); the
 * message is fedfem_create_error().
 */
typedef struct {
    int32_t n_tiles, n_chunks, max_tile_nodes, n_colors_max;
    int64_t n_shared_nodes, n_halo_slots;  /* shared nodes, and their (tile, node) partial slots */
    int64_t n_padding_slots;               /* element slots of the chunks left empty            */
} fedfem_tiling_stats;
fedfem_status fedfem_check_tiling(const fedfem_mesh *mesh, int64_t n_boundary, const int32_t *boundary_nodes,
                                  int32_t n_tiles, int32_t chunk, int32_t single_class, fedfem_tiling_stats *stats);

/* Message of the last error on this context ("" if none).  Valid until the next call. */
const char *fedfem_error_string(fedfem_ctx *ctx);
/* Message of the last fedfem_create failure on this thread. */
const char *fedfem_create_error(void);
/* Release the context and all its device memory.  NULL is ignored. */
void fedfem_destroy(fedfem_ctx *ctx);

/* ---------------------------------------------------------------------------------------
 * Batched scenarios (no counterpart in the paper): many independent problems, each with its
 * own mesh, material, boundary data, time step and step count, advanced together.  Every
 * scenario keeps its own dt = dt_scale * dt_crit (computed as in fedfem_precompute over
 * [T_lo, T_hi]).  The launch sequence for all scenarios is captured once in a CUDA graph.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    fedfem_mesh mesh;
    fedfem_material mat;
    fedfem_bcs bcs;
    const double *T0;           /* [n_nodes] */
    int64_t n_steps;
    double T_lo, T_hi;          /* range for the critical step                  */
    double dt_scale;            /* dt = dt_scale * dt_crit (e.g. 0.9)           */
} fedfem_scenario;

/* Pack, tile, pre-compute (including every scenario's dt_crit) and capture the run.  All
 * scenarios use one element type and one material each; the fedfem_scenario arrays are host
 * arrays copied during the call.  *out is set even on failure, so that
 * fedfem_batch_error_string can explain it; release it with fedfem_batch_destroy.
 * Errors: ARG, MESH, UNSUPPORTED, CUDA, OOM. */
fedfem_status fedfem_batch_create(const fedfem_scenario *sc, int32_t n_scenarios,
                                  const fedfem_options *opt, fedfem_batch **out);
/* Reset every scenario to its T0 and run all of them to their step counts (graph replay).
 * Errors: DIVERGED, TIMEOUT, CUDA. */
fedfem_status fedfem_batch_run(fedfem_batch *b);
/* Completion time of each scenario in ns since the start of the last run, read from the
 * device's global timer [n_scenarios]; total element-steps and the dt of each scenario. */
fedfem_status fedfem_batch_times(fedfem_batch *b, double *t_done_ns, double *elem_steps_total,
                                 double *dt);
fedfem_status fedfem_batch_get_T(fedfem_batch *b, int32_t s, double *T_host);
const char *fedfem_batch_error_string(fedfem_batch *b);
void fedfem_batch_destroy(fedfem_batch *b);

/* ---------------------------------------------------------------------------------------
 * Domain decomposition of one mesh (Section 3, Eq. 15-16: with the lumped capacitance every
 * nodal equation is independent once its element loads are known, which permits a parallel
 * implementation).  The elements are cut into n_sub slabs of equal element count along the
 * longest axis of the bounding box (by element centroid; a coordinate bisection that also
 * serves unstructured meshes).  A node is owned by the lowest-numbered slab among its
 * elements.  Sub-domain s holds the elements of slab s plus every element touching a node it
 * owns (one ghost layer), so each owned node receives all its element loads locally; the other
 * nodes of those elements are its ghosts.  Each sub-domain is a context of its own.  One step
 * = one step of every sub-domain (ghosts held fixed, like Dirichlet nodes), then the halo
 * exchange: each owner packs the new values of its nodes that neighbours hold as ghosts into
 * a send buffer, one message per sub-domain pair moves send buffer to receive buffer, and the
 * receivers unpack into their ghost slots.  In FP32 + Kahan a message entry carries the value
 * and its compensation (8 bytes), in FP64 the value (8 bytes).  All sub-domains run on the
 * device and stream of `opt`; the field equals the undecomposed run's up to the order of the
 * floating-point sums.  Not available with schedules or property tables.
 * ------------------------------------------------------------------------------------- */
typedef struct fedfem_dd fedfem_dd;
typedef struct {
    int32_t n_sub, axis;          /* sub-domains, slab axis (0 = x, 1 = y, 2 = z)            */
    int32_t n_messages, reserved; /* sub-domain pairs that exchange ghost values each step   */
    int64_t halo_entries;         /* ghost values sent per step (all messages)               */
    int64_t halo_bytes_per_step;  /* bytes of those values                                   */
    int64_t ghost_elements;       /* elements held by a sub-domain other than their slab's   */
    int64_t step;                 /* steps since fedfem_dd_set_T                             */
    double dt_crit;               /* as returned by fedfem_dd_precompute                     */
} fedfem_dd_info;
/* Partition the mesh and create one context per sub-domain (arguments as fedfem_create; the
 * sub-domains' launch plans follow opt).  On failure *out is NULL and
 * fedfem_dd_error_string(NULL) explains it.  Errors: ARG, MESH, CUDA, OOM. */
fedfem_status fedfem_dd_create(const fedfem_mesh *mesh, const fedfem_material *mats, int32_t n_mats,
                               const fedfem_bcs *bcs, const fedfem_options *opt, int32_t n_sub,
                               fedfem_dd **out);
/* Pre-computation of every sub-domain (fedfem_precompute).  *dt_crit_out = the smallest
 * critical step over the sub-domains.  Each sub-domain's operator on its owned nodes is a
 * principal sub-matrix of the whole mesh's, so this is at least the whole mesh's dt_crit (equal
 * up to how much the highest mode is cut by the ghost boundaries; on the structured cubes
 * tested, within 1e-3): choose dt with a safety factor.  Errors: as fedfem_precompute. */
fedfem_status fedfem_dd_precompute(fedfem_dd *dd, double T_lo, double T_hi, double *dt_crit_out);
/* Time step of all sub-domains; UNSTABLE if dt > dt_crit and force == 0. */
fedfem_status fedfem_dd_set_dt(fedfem_dd *dd, double dt, int32_t force);
/* Initial field [n_nodes] (host, the mesh's node order); Dirichlet values re-imposed, ghosts
 * filled from their owners. */
fedfem_status fedfem_dd_set_T(fedfem_dd *dd, const double *T0_host);
/* n_steps explicit steps (one launch per sub-domain and step, then the halo exchange);
 * synchronises and reports device-side errors as fedfem_step. */
fedfem_status fedfem_dd_step(fedfem_dd *dd, int64_t n_steps);
/* Current field [n_nodes] (host, FP64, the mesh's node order), each node from its owner. */
fedfem_status fedfem_dd_get_T(fedfem_dd *dd, double *T_host);
fedfem_status fedfem_dd_get_info(fedfem_dd *dd, fedfem_dd_info *info);
/* Host-only query of the partition (no device call): sub-domain s of n_sub for this mesh, its
 * elements (ascending global ids, core and ghost layer) and nodes (ascending global ids) and,
 * per node, the owning sub-domain of a ghost (-1 for an owned node).  Pass NULL arrays to get
 * the counts first.  Errors: ARG, MESH (node id out of range). */
fedfem_status fedfem_dd_subdomain(const fedfem_mesh *mesh, int32_t n_sub, int32_t s, int64_t *n_elems,
                                  int32_t *elems, int64_t *n_nodes, int32_t *nodes, int32_t *ghost_owner);
/* ---------------------------------------------------------------------------------------
 * Measurement helpers (no counterpart in the paper): the denominators of the roofline
 * fractions of kernels that HBM does not bound.
 * ------------------------------------------------------------------------------------- */
/* Copy `bytes` (a multiple of 16) from src_dev to dst_dev (DEVICE buffers, 16-byte aligned)
 * `reps` times with the library's own vector copy kernel (blocks_per_sm x SMs blocks of 512
 * threads), after one untimed pass; *ms_out = the device time of the reps passes (CUDA events
 * on `stream`).  Bandwidth = 2 bytes reps / time: an L2 figure when both buffers fit in L2, an
 * HBM figure when they are much larger.  Synchronises the stream.  Errors: ARG, CUDA. */
fedfem_status fedfem_probe_copy(void *dst_dev, const void *src_dev, int64_t bytes, int32_t reps,
                                int32_t blocks_per_sm, void *stream, double *ms_out);
/* FP64 fused multiply-add rate: blocks_per_sm x SMs blocks of 256 threads, each running eight
 * independent chains of `iters` FMAs; *flops_out = 2 x FMAs issued, *ms_out = their device time.
 * Synchronises the stream.  Errors: ARG, OOM (8-byte sink), CUDA. */
fedfem_status fedfem_probe_fp64(int64_t iters, int32_t blocks_per_sm, void *stream, double *ms_out,
                                double *flops_out);

/* Message of the last error on dd; with NULL, of the last fedfem_dd_create on this thread. */
const char *fedfem_dd_error_string(fedfem_dd *dd);
/* Release all sub-domains.  NULL is ignored. */
void fedfem_dd_destroy(fedfem_dd *dd);

#ifdef __cplusplus
}
#endif
#endif /* FEDFEM_H */
