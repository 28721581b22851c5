// Launchers of the FP64 pre-computation and diagnostic kernels (precompute.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "law.cuh"

namespace fedfem {

struct ElemArgs {
    int64_t ne;
    const double *xyz;          // [nn][3] original order
    const int32_t *conn;        // [ne][npe] original ids
    const int32_t *mat;         // [ne] or NULL
    const double *mat_k0;       // [n_mats][9]
    const double *kscale;       // [ne] or NULL
    const int64_t *slot_of_elem;
    int CH, VW, precision, chunk_bytes;
    uint8_t *chunks;            // element stream (conductances written here)
    double *cond64;             // [ne][n_pairs] FP64 copy
    double *W;                  // [ne][npe] int_e N_i dV
    int quad;                   // hexahedron conduction matrix: 8 = 2x2x2 Gauss, 1 = centre point
    double *cond_qp;            // [ne][8][28] pair conductances of each 2x2x2 point, or NULL
    int32_t *err;
    unsigned long long *bad_elem;
};

struct NodeArgs {
    int64_t nn;
    int npe;
    const int32_t *n2e_ptr;
    const int64_t *n2e;
    const double *W;
    const int32_t *mat;
    const double *mat_rhoc;     // [n_mats] rho * c0
    const double *source;       // [ne] or NULL
    const double *nodal_Q;      // [nn] original order or NULL
    const int32_t *old_of_new;
    const int32_t *fc_ptr, *fc_idx, *fr_ptr, *fr_idx;
    const double *fc_share, *fr_share;
    double *C0, *Qext64, *Ac64, *Ar64;
    float *Qext32, *Ac32, *Ar32;  // NULL in FP64 mode
};

struct EnergyPhys {
    double dt, c_lin, h, T_inf, eps_sigma, T_amb, T_zero;
    double c_a;  // f_c = c_a + c_lin T
    double qs;   // multiplier of the external loads (time-dependent loads)
    int tab;     // 1: f_c from the table tc instead of the linear law
    HingeLaw<double> tc;
};

void launch_elem(int npe, const ElemArgs &a, cudaStream_t st);
void launch_face_share(int64_t nf, int nv, const int32_t *faces, const double *xyz, double *share, cudaStream_t st);
void launch_node_sums(const NodeArgs &a, cudaStream_t st);
void launch_set_A(int64_t nn, double dt, const double *C0, const uint8_t *isdir, double *A, float2 *A2,
                  cudaStream_t st);
// F = sum_e f_k,e K0_e x_e (fixed-order gather); f_k,e from the nodal Tk: k_a + k_lin mean T,
// or with tk the mean of the tabulated nodal factors (Tk == NULL: f_k,e = 1)
void launch_apply(int npe, int64_t ne, int64_t nn, const int32_t *gconn, const double *cond64, const int32_t *n2e_ptr,
                  const int64_t *n2e, const double *x, const double *Tk, double k_a, double k_lin,
                  const HingeLaw<double> *tk, double *Y, double *F, cudaStream_t st);
int reduce_blocks(int64_t nn);
void launch_power_init(int64_t nn, const uint8_t *isdir, double *x, cudaStream_t st);
void launch_scale_free(int64_t nn, const double *x, const double *C0, const uint8_t *isdir, double *u, cudaStream_t st);
void launch_power_dots(int64_t nn, const double *x, const double *F, const double *C0, const uint8_t *isdir, double *z,
                       double *partial, double *sums, cudaStream_t st);
// Lanczos for the largest eigenvalue of C0^-1/2 K0 C0^-1/2 (free nodes): start vector
// v0 = x / |x| (norm2 receives |x|^2), then one step per call; coef receives alpha_j at [0] and
// beta_j^2 at [2], and v_{j+1} is written over vprev.
void launch_lanczos_start(int64_t nn, const uint8_t *isdir, double *x, double *v0, double *partial, double *norm2,
                          cudaStream_t st);
void launch_lanczos_step(int npe, int64_t ne, int64_t nn, const int32_t *gconn, const double *cond64,
                         const int32_t *n2e_ptr, const int64_t *n2e, const double *C0, const uint8_t *isdir,
                         double *vprev, const double *vcur, double *u, double *F, double *Y, const double *beta2_prev,
                         double *coef, double *partial, cudaStream_t st);
// per-block (min, max) of x[0..nn) into partial[2 b], partial[2 b + 1]; returns the block count
int launch_minmax(int64_t nn, const double *x, double *partial, cudaStream_t st);
void launch_normalize(int64_t nn, const double *z, const double *sums, double *x, cudaStream_t st);
int launch_surface_rate(int64_t nn, const double *Ac, const double *Ar, const double *C0, const uint8_t *isdir, double h,
                        double rad_coef, double fc_min, double *partial, cudaStream_t st);
void launch_state_to_f64(int precision, int64_t nn, const void *T, const float *comp, double *out, cudaStream_t st);
void launch_set_state(int precision, int64_t nn, const double *T0_old, const int32_t *old_of_new, void *T, float *comp,
                      cudaStream_t st);
// prescribed values dir_T + offset into an old-order FP64 field
void launch_impose_dirichlet(int64_t nd, const int32_t *dir_new, const double *dir_T, double offset, double *T0_old,
                             const int32_t *old_of_new, cudaStream_t st);
// prescribed values dir_T + offset into the working state (new order; comp may be NULL)
void launch_impose_dirichlet_state(int precision, int64_t nd, const int32_t *dir_new, const double *dir_T,
                                   double offset, void *T, float *comp, cudaStream_t st);
void launch_permute_new_to_old(int64_t nn, const double *x_new, const int32_t *old_of_new, double *x_old, cudaStream_t st);
void launch_permute_old_to_new(int64_t nn, const double *x_old, const int32_t *old_of_new, double *x_new, cudaStream_t st);
void launch_energy(int64_t nn, const double *T0, const double *T1, const double *F, const double *C0, const double *Qext,
                   const double *Ac, const double *Ar, const uint8_t *isdir, const EnergyPhys &ph, double *partial,
                   double *sums, cudaStream_t st);

}  // namespace fedfem
