/*
 * FED-FEM oracle: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 CPU implementation of the fast explicit dynamics finite
 * element method (FED-FEM) for transient heat conduction (Zhang & Chauhan, arXiv:1909.03355).
 * Only the test suite, the smoke check and the CPU-baseline leg of bench.py may load it.  It
 * shares no code with the CUDA library: it follows the paper's equations in their textbook
 * form (full 8x8 / 4x4 element matrices, element loop and scatter, literal Eq. 7 radiation).
 * Everything runs on one thread except orc_run_mt, the same time stepping over all host cores
 * with a result bitwise equal to the single-threaded orc_run.
 *
 * Readings of the paper used here (where it is silent, garbled or at odds with itself):
 *  - Sign (Eq. 2, 11-13): the element load F_e = theta_e f_k,e K0_e T_e is the positive
 *    semidefinite conduction load and the update is T += dt (Q - F) / C.  The paper's K of
 *    Eq. 2 is therefore -K0.
 *  - Convection (Eq. 4): heat leaves when T > T_a, nodal load -A^c_i h (T_i - T_a).
 *  - Hexahedra integrate Eq. 12 with 2x2x2 Gauss points by default (the one-point rule of
 *    Eq. 17 has hourglass modes); the one-point conduction matrix of Eq. 17 is available as an
 *    option (orc_hex_matrix_centre), with masses, loads and areas integrated as by default.
 *    Tetrahedra use Eq. 18 exactly.
 *  - Temperature-dependent conductivity is evaluated at the element nodes and averaged over
 *    the element (Section 4.2.2): f_k,e = mean_i f_k(T_i); c(T) is evaluated per node (Eq. 16).
 *  - Lumped (diagonal) thermal mass by row sums, M_i = sum_e rho_e int_e N_i dV (Section 3.1).
 *  - Surface loads use nodal-quadrature lumping: every face gives A_f / n_f to each node.
 *  - Critical step (Section 3.4, Eq. 29): dt_crit = 2 / lambda_max of the linearised system,
 *    lambda from FP64 power iteration on C0^-1/2 K0 C0^-1/2, scaled by max f_k / min f_c over
 *    [T_lo, T_hi], plus the largest linearised surface rate.
 *
 * Parity pins live in tests/test_oracle_*.py (closed forms, patch tests, the slab recurrence,
 * energy balance, dense brute force, finite differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_SIGMA 5.67e-8 /* Stefan-Boltzmann constant as printed with Eq. 7 */

/* ------------------------------------------------------------------------------------------ */
/* small dense helpers                                                                          */
/* ------------------------------------------------------------------------------------------ */

static double det3(const double J[3][3])
{
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
         - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
         + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

static void inv3(const double J[3][3], double d, double Ji[3][3])
{
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / d;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / d;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / d;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / d;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / d;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / d;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / d;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / d;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / d;
}

/* ------------------------------------------------------------------------------------------ */
/* element matrices (pre-computation stage, Fig. 1 (i) 2)                                       */
/* ------------------------------------------------------------------------------------------ */

/* natural coordinates of the 8 hex nodes, VTK / C3D8 order */
static const double HEX_NAT[8][3] = {
    {-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
    {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

/*
 * The integrand of Eq. 12 for the trilinear hexahedron at Gauss point q of the 2x2x2 rule
 * (points +-1/sqrt(3), unit weights): Kq_ij = det J (grad N_i)^T k (grad N_j) (row-major 8x8)
 * and the shape function values N [8] at the point; *detJ = det J.  Returns -1 when
 * det J <= 0 (inverted or degenerate element).
 */
static int orc_hex_point(const double *x, const double *k, int q, double *Kq, double *N, double *detJ)
{
    const double g = 1.0 / sqrt(3.0);
    const double xi = HEX_NAT[q][0] * g, eta = HEX_NAT[q][1] * g, zeta = HEX_NAT[q][2] * g;
    double dN[8][3];
    for (int i = 0; i < 8; ++i) {
        const double a = 1.0 + xi * HEX_NAT[i][0];
        const double b = 1.0 + eta * HEX_NAT[i][1];
        const double c = 1.0 + zeta * HEX_NAT[i][2];
        N[i] = a * b * c / 8.0;
        dN[i][0] = HEX_NAT[i][0] * b * c / 8.0;
        dN[i][1] = a * HEX_NAT[i][1] * c / 8.0;
        dN[i][2] = a * b * HEX_NAT[i][2] / 8.0;
    }
    double J[3][3] = {{0}};
    for (int i = 0; i < 8; ++i)
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) J[r][s] += x[3 * i + r] * dN[i][s];
    const double d = det3(J);
    if (!(d > 0.0)) return -1;
    double Ji[3][3];
    inv3(J, d, Ji);
    double B[8][3]; /* grad_x N_i = J^-T grad_xi N_i */
    for (int i = 0; i < 8; ++i)
        for (int r = 0; r < 3; ++r) {
            B[i][r] = 0.0;
            for (int s = 0; s < 3; ++s) B[i][r] += Ji[s][r] * dN[i][s];
        }
    for (int i = 0; i < 8; ++i) {
        double kB[3];
        for (int r = 0; r < 3; ++r) {
            kB[r] = 0.0;
            for (int s = 0; s < 3; ++s) kB[r] += k[3 * r + s] * B[i][s];
        }
        for (int j = 0; j < 8; ++j) Kq[8 * j + i] = d * (B[j][0] * kB[0] + B[j][1] * kB[1] + B[j][2] * kB[2]);
    }
    *detJ = d;
    return 0;
}

/*
 * Eq. 12 for the trilinear hexahedron: K_ij = int_Ve (grad N_i)^T k (grad N_j) dV, evaluated by
 * 2x2x2 Gauss quadrature (points +-1/sqrt(3), unit weights), together with w_i = int_Ve N_i dV
 * and the element volume.  x: [8][3] node coordinates; k: 3x3 conductivity (row-major).
 * Returns 0, or -1 when det J <= 0 at a Gauss point (inverted or degenerate element).
 */
int orc_hex_matrices(const double *x, const double *k, double *K, double *w, double *vol)
{
    memset(K, 0, 64 * sizeof(double));
    memset(w, 0, 8 * sizeof(double));
    *vol = 0.0;
    for (int q = 0; q < 8; ++q) {
        double Kq[64], N[8], d;
        if (orc_hex_point(x, k, q, Kq, N, &d)) return -1;
        for (int i = 0; i < 64; ++i) K[i] += Kq[i];
        for (int i = 0; i < 8; ++i) w[i] += d * N[i];
        *vol += d;
    }
    return 0;
}

/*
 * The 2x2x2 Gauss-point matrices of Eq. 12 for conductivity evaluated at the points (Eq. 20
 * with D(T) inside the integral): Kq [8][8][8] (point, row, column) and the shape function
 * values Nq [8][8] (point, node).  Returns -1 when det J <= 0 at a point.
 */
int orc_hex_matrices_qp(const double *x, const double *k, double *Kq, double *Nq)
{
    for (int q = 0; q < 8; ++q) {
        double d;
        if (orc_hex_point(x, k, q, Kq + 64 * q, Nq + 8 * q, &d)) return -1;
    }
    return 0;
}

/*
 * One-point conduction matrix of the reduced-integration hexahedron (Eq. 17): the
 * gradients B of the trilinear shape functions at the element centre (xi = eta = zeta = 0),
 * K = 8 det J(0) B^T k B.  Returns -1 if det J(0) <= 0.
 */
int orc_hex_matrix_centre(const double *x, const double *k, double *K)
{
    double dN[8][3];
    for (int i = 0; i < 8; ++i)
        for (int s = 0; s < 3; ++s) dN[i][s] = HEX_NAT[i][s] / 8.0;
    double J[3][3] = {{0}};
    for (int i = 0; i < 8; ++i)
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) J[r][s] += x[3 * i + r] * dN[i][s];
    const double d = det3(J);
    if (!(d > 0.0)) return -1;
    double Ji[3][3];
    inv3(J, d, Ji);
    double B[8][3];
    for (int i = 0; i < 8; ++i)
        for (int r = 0; r < 3; ++r) {
            B[i][r] = 0.0;
            for (int s = 0; s < 3; ++s) B[i][r] += Ji[s][r] * dN[i][s];
        }
    for (int i = 0; i < 8; ++i) {
        double kB[3];
        for (int r = 0; r < 3; ++r) {
            kB[r] = 0.0;
            for (int s = 0; s < 3; ++s) kB[r] += k[3 * r + s] * B[i][s];
        }
        for (int j = 0; j < 8; ++j) K[8 * j + i] = 8.0 * d * (B[j][0] * kB[0] + B[j][1] * kB[1] + B[j][2] * kB[2]);
    }
    return 0;
}

/* Solve the 4x4 system P X = I by Gaussian elimination with partial pivoting. */
static int inv4(const double P[4][4], double X[4][4])
{
    double A[4][8];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 8; ++c) A[r][c] = c < 4 ? P[r][c] : (c - 4 == r ? 1.0 : 0.0);
    for (int c = 0; c < 4; ++c) {
        int p = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
        if (A[p][c] == 0.0) return -1;
        if (p != c)
            for (int j = 0; j < 8; ++j) {
                double t = A[c][j];
                A[c][j] = A[p][j];
                A[p][j] = t;
            }
        for (int r = 0; r < 4; ++r) {
            if (r == c) continue;
            const double f = A[r][c] / A[c][c];
            for (int j = 0; j < 8; ++j) A[r][j] -= f * A[c][j];
        }
    }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) X[r][c] = A[r][4 + c] / A[r][r];
    return 0;
}

/*
 * Eq. 18 for the linear tetrahedron: K = V B^T k B with B the (constant) gradients of the
 * barycentric shape functions, taken from the inverse of P = [1 x y z] (rows = nodes);
 * w_i = V / 4.  Returns -1 for V <= 0.
 */
int orc_tet_matrices(const double *x, const double *k, double *K, double *w, double *vol)
{
    double P[4][4], C[4][4];
    for (int i = 0; i < 4; ++i) {
        P[i][0] = 1.0;
        for (int r = 0; r < 3; ++r) P[i][1 + r] = x[3 * i + r];
    }
    const double J[3][3] = {
        {x[3] - x[0], x[6] - x[0], x[9] - x[0]},
        {x[4] - x[1], x[7] - x[1], x[10] - x[1]},
        {x[5] - x[2], x[8] - x[2], x[11] - x[2]}};
    const double V = det3(J) / 6.0;
    if (!(V > 0.0)) return -1;
    if (inv4(P, C)) return -1;
    /* N_i(x) = C[0][i] + C[1][i] x + C[2][i] y + C[3][i] z  => grad N_i = C[1..3][i] */
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int t = 0; t < 3; ++t) s += C[1 + r][i] * k[3 * r + t] * C[1 + t][j];
            K[4 * i + j] = V * s;
        }
        w[i] = V / 4.0;
    }
    *vol = V;
    return 0;
}

/* Area of a boundary face: half the cross product for a triangle; for a quadrilateral the
 * area of its bilinear patch, int |x_xi x x_eta| over [-1,1]^2 by 2x2 Gauss points. */
double orc_face_area(const double *x, int nv)
{
    if (nv == 3) {
        double a[3], b[3], c[3];
        for (int r = 0; r < 3; ++r) {
            a[r] = x[3 + r] - x[r];
            b[r] = x[6 + r] - x[r];
        }
        c[0] = a[1] * b[2] - a[2] * b[1];
        c[1] = a[2] * b[0] - a[0] * b[2];
        c[2] = a[0] * b[1] - a[1] * b[0];
        return 0.5 * sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    }
    static const double S[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
    const double g = 1.0 / sqrt(3.0);
    double A = 0.0;
    for (int q = 0; q < 4; ++q) {
        const double s = S[q][0] * g, t = S[q][1] * g;
        double xs[3] = {0, 0, 0}, xt[3] = {0, 0, 0};
        for (int i = 0; i < 4; ++i)
            for (int r = 0; r < 3; ++r) {
                xs[r] += x[3 * i + r] * S[i][0] * (1.0 + t * S[i][1]) / 4.0;
                xt[r] += x[3 * i + r] * (1.0 + s * S[i][0]) * S[i][1] / 4.0;
            }
        const double c0 = xs[1] * xt[2] - xs[2] * xt[1];
        const double c1 = xs[2] * xt[0] - xs[0] * xt[2];
        const double c2 = xs[0] * xt[1] - xs[1] * xt[0];
        A += sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    }
    return A;
}

/* ------------------------------------------------------------------------------------------ */
/* the model after pre-computation                                                              */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int64_t nn, ne;
    int32_t npe, pad;
    const int32_t *conn;  /* [ne][npe] */
    const double *K;      /* [ne][npe][npe]  K0_e (unit conductivity scale, f_k = 1) */
    const double *theta;  /* [ne] conductivity scale theta_e */
    const double *W;      /* [ne][npe] int_e N_i dV */
    const double *C0;     /* [nn] sum_e rho_e c0_e int_e N_i dV (lumped thermal mass at f_c = 1) */
    const double *Qext;   /* [nn] constant nodal heat flow (sources, concentrated fluxes) */
    const double *Ac;     /* [nn] convection area share */
    const double *Ar;     /* [nn] radiation area share */
    const int32_t *isdir; /* [nn] 1 on Gamma_E */
    double k_lin, c_lin;  /* f_k(T) = 1 + k_lin (T - T_ref), f_c(T) = 1 + c_lin (T - T_ref) */
    double h, T_inf, eps, T_amb, T_zero;
    double T_ref;         /* temperature at which k0 and c0 are given */
    /* time-dependent loads (optional): at step n the external loads are q_sched[n] Qext and
     * the convection ambient temperature is Tinf_sched[n] (the last entry beyond the end);
     * n counts from sched_step0 at the first step of a run */
    const double *q_sched;
    const double *Tinf_sched;
    int64_t n_sched, sched_step0;
    /* time-dependent Dirichlet values (optional): with Tdir_sched set, the value of Dirichlet
     * node i at step n is Tdir[i] + Tdir_sched[n] (same length and end rule as the load
     * schedule); Tdir [nn] holds the prescribed values of Gamma_E (read on Dirichlet nodes) */
    const double *Tdir;
    const double *Tdir_sched;
    /* tabulated property factors (optional, n_tab >= 2; they replace the linear laws above):
     * f_k and f_c given at the increasing temperatures tab_T, interpolated linearly between
     * neighbouring points and held at the end values outside [tab_T[0], tab_T[n_tab - 1]] */
    int64_t n_tab;
    const double *tab_T, *tab_fk, *tab_fc;
    /* conductivity evaluated at quadrature points (Eq. 20 with D(T) inside the integral; nq > 0
     * replaces the element mean of the nodal factors): F_e = theta_e sum_q f_k(T_q) Kq_{e,q} T_e
     * with T_q = sum_i Nq[q][i] T_i */
    int64_t nq;
    const double *Kq; /* [ne][nq][npe][npe] */
    const double *Nq; /* [nq][npe] */
    /* consistent integration of the surface loads of Eq. 4 and Eq. 7 over the boundary faces
     * (nfq > 0 replaces the nodal lumping of the areas Ac, Ar):
     *   Q_i -= h sum_j Mf_ij (T_j - T_inf) over convection faces,
     *   Q_i -= eps sigma sum_p Wf_p Nf_pi ((T_p - T_z)^4 - (T_amb - T_z)^4) over radiation faces */
    int64_t n_cf, n_rf;
    int32_t nvf, nfq;
    const int32_t *cfaces, *rfaces; /* [n][nvf] */
    const double *Mf;               /* [n_cf][nvf][nvf] int_f N_i N_j dA */
    const double *Wf;               /* [n_rf][nfq] quadrature weight x area Jacobian */
    const double *Nf;               /* [nfq][nvf] shape function values at the face points */
} orc_model;

/* Value of a tabulated factor v at T: linear between the two table points around T. */
static double orc_table(const orc_model *m, const double *v, double T)
{
    const double *t = m->tab_T;
    const int64_t n = m->n_tab;
    if (T <= t[0]) return v[0];
    if (T >= t[n - 1]) return v[n - 1];
    int64_t j = 0;
    while (T > t[j + 1]) ++j; /* t[j] < T <= t[j + 1] */
    return v[j] + (v[j + 1] - v[j]) * (T - t[j]) / (t[j + 1] - t[j]);
}

/* Slope of a tabulated factor at T (0 where the end values are held). */
static double orc_table_slope(const orc_model *m, const double *v, double T)
{
    const double *t = m->tab_T;
    const int64_t n = m->n_tab;
    if (T <= t[0] || T >= t[n - 1]) return 0.0;
    int64_t j = 0;
    while (T > t[j + 1]) ++j;
    return (v[j + 1] - v[j]) / (t[j + 1] - t[j]);
}

/* Conductivity and capacity factors at a nodal temperature (Section 4.2.2) and their slopes. */
static double orc_fk(const orc_model *m, double T)
{
    return m->n_tab >= 2 ? orc_table(m, m->tab_fk, T) : 1.0 + m->k_lin * (T - m->T_ref);
}

static double orc_fc(const orc_model *m, double T)
{
    return m->n_tab >= 2 ? orc_table(m, m->tab_fc, T) : 1.0 + m->c_lin * (T - m->T_ref);
}

static double orc_dfk(const orc_model *m, double T)
{
    return m->n_tab >= 2 ? orc_table_slope(m, m->tab_fk, T) : m->k_lin;
}

static double orc_dfc(const orc_model *m, double T)
{
    return m->n_tab >= 2 ? orc_table_slope(m, m->tab_fc, T) : m->c_lin;
}

/* Largest f_k and smallest f_c over [T_lo, T_hi]: a piecewise-linear factor takes its extrema
 * at the interval ends or at table points inside it. */
static void orc_factor_extrema(const orc_model *m, double T_lo, double T_hi, double *fk_max, double *fc_min)
{
    double kmax = fmax(orc_fk(m, T_lo), orc_fk(m, T_hi));
    double cmin = fmin(orc_fc(m, T_lo), orc_fc(m, T_hi));
    for (int64_t j = 0; m->n_tab >= 2 && j < m->n_tab; ++j)
        if (m->tab_T[j] > T_lo && m->tab_T[j] < T_hi) {
            kmax = fmax(kmax, m->tab_fk[j]);
            cmin = fmin(cmin, m->tab_fc[j]);
        }
    *fk_max = kmax;
    *fc_min = cmin;
}

/*
 * Pre-computation (Fig. 1 (i)): element matrices K0_e and shape-function integrals, lumped
 * thermal mass, constant external loads and boundary area shares.
 *   mat_k0 [n_mats][9], mat_rho, mat_c0 [n_mats]; elem_mat [ne] or NULL (material 0);
 *   source [ne] W/m^3 or NULL; nodal_Q [nn] W or NULL;
 *   conv/rad faces [n][nvf] node ids; dir_nodes [nd].
 * Outputs (caller-allocated): K [ne*npe*npe], W [ne*npe], C0, Qext, Ac, Ar [nn], isdir [nn].
 * Returns 0, or 1 + e for the first element e with det J <= 0.
 */
int64_t orc_precompute(int64_t nn, int64_t ne, int32_t npe, const double *xyz, const int32_t *conn,
                       const int32_t *elem_mat, const double *mat_k0, const double *mat_rho,
                       const double *mat_c0, const double *source, const double *nodal_Q,
                       int64_t n_conv, int32_t nv_conv, const int32_t *conv_faces,
                       int64_t n_rad, int32_t nv_rad, const int32_t *rad_faces,
                       int64_t n_dir, const int32_t *dir_nodes,
                       double *K, double *W, double *C0, double *Qext, double *Ac, double *Ar,
                       int32_t *isdir)
{
    memset(C0, 0, nn * sizeof(double));
    memset(Qext, 0, nn * sizeof(double));
    memset(Ac, 0, nn * sizeof(double));
    memset(Ar, 0, nn * sizeof(double));
    memset(isdir, 0, nn * sizeof(int32_t));
    double xe[8 * 3];
    for (int64_t e = 0; e < ne; ++e) {
        const int m = elem_mat ? elem_mat[e] : 0;
        for (int i = 0; i < npe; ++i)
            for (int r = 0; r < 3; ++r) xe[3 * i + r] = xyz[3 * (int64_t)conn[npe * e + i] + r];
        double vol;
        const int rc = npe == 8 ? orc_hex_matrices(xe, mat_k0 + 9 * m, K + 64 * e, W + 8 * e, &vol)
                                : orc_tet_matrices(xe, mat_k0 + 9 * m, K + 16 * e, W + 4 * e, &vol);
        if (rc) return 1 + e;
        for (int i = 0; i < npe; ++i) {
            const int64_t n = conn[npe * e + i];
            C0[n] += mat_rho[m] * mat_c0[m] * W[npe * e + i];
            if (source) Qext[n] += source[e] * W[npe * e + i];
        }
    }
    if (nodal_Q)
        for (int64_t i = 0; i < nn; ++i) Qext[i] += nodal_Q[i];
    double xf[4 * 3];
    for (int64_t f = 0; f < n_conv; ++f) {
        for (int i = 0; i < nv_conv; ++i)
            for (int r = 0; r < 3; ++r) xf[3 * i + r] = xyz[3 * (int64_t)conv_faces[nv_conv * f + i] + r];
        const double a = orc_face_area(xf, nv_conv) / nv_conv;
        for (int i = 0; i < nv_conv; ++i) Ac[conv_faces[nv_conv * f + i]] += a;
    }
    for (int64_t f = 0; f < n_rad; ++f) {
        for (int i = 0; i < nv_rad; ++i)
            for (int r = 0; r < 3; ++r) xf[3 * i + r] = xyz[3 * (int64_t)rad_faces[nv_rad * f + i] + r];
        const double a = orc_face_area(xf, nv_rad) / nv_rad;
        for (int i = 0; i < nv_rad; ++i) Ar[rad_faces[nv_rad * f + i]] += a;
    }
    for (int64_t d = 0; d < n_dir; ++d) isdir[dir_nodes[d]] = 1;
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* time stepping (Fig. 1 (iii))                                                                 */
/* ------------------------------------------------------------------------------------------ */

/* Eq. 11 / 20: F = sum_e F_e, F_e = theta_e f_k,e K0_e T_e with f_k,e the element mean of the
 * nodal f_k(T_i) (Section 4.2.2).  F [nn] is overwritten. */
/* Load vector of element e (Eq. 20): Fe[i] = theta_e f_k,e (K0_e T_e)_i with the element mean
 * f_k,e of the nodal factors (Section 4.2.2), or with nq > 0 the sum over the quadrature points
 * theta_e sum_q f_k(T_q) (Kq T_e)_i. */
static void orc_element_loads(const orc_model *m, int64_t e, const double *T, double *Fe)
{
    const int npe = m->npe;
    const int32_t *c = m->conn + npe * e;
    if (m->nq > 0) {
        double acc[8] = {0};
        for (int64_t q = 0; q < m->nq; ++q) {
            const double *Kq = m->Kq + ((int64_t)m->nq * e + q) * npe * npe;
            double Tq = 0.0;
            for (int i = 0; i < npe; ++i) Tq += m->Nq[npe * q + i] * T[c[i]];
            const double f = orc_fk(m, Tq);
            for (int i = 0; i < npe; ++i) {
                double kt = 0.0;
                for (int j = 0; j < npe; ++j) kt += Kq[npe * i + j] * T[c[j]];
                acc[i] += f * kt;
            }
        }
        for (int i = 0; i < npe; ++i) Fe[i] = m->theta[e] * acc[i];
        return;
    }
    const double *Ke = m->K + (int64_t)npe * npe * e;
    double fk = 0.0;
    for (int i = 0; i < npe; ++i) fk += orc_fk(m, T[c[i]]);
    fk /= npe;
    const double s = m->theta[e] * fk;
    for (int i = 0; i < npe; ++i) {
        double acc = 0.0;
        for (int j = 0; j < npe; ++j) acc += Ke[npe * i + j] * T[c[j]];
        Fe[i] = s * acc;
    }
}

void orc_internal_loads(const orc_model *m, const double *T, double *F)
{
    const int npe = m->npe;
    memset(F, 0, m->nn * sizeof(double));
    double Fe[8];
    for (int64_t e = 0; e < m->ne; ++e) {
        orc_element_loads(m, e, T, Fe);
        for (int i = 0; i < npe; ++i) F[m->conn[npe * e + i]] += Fe[i];
    }
}

/* Consistent surface loads (Eq. 4 and Eq. 7 integrated with the face shape functions) of the
 * field T at step n into Qs [nn] (overwritten): convection faces by their face mass matrices,
 * radiation faces by the face quadrature rule with the quartic of the interpolated temperature. */
static double orc_T_inf(const orc_model *m, int64_t n);
void orc_surface_loads(const orc_model *m, const double *T, int64_t n, double *Qs)
{
    const int nv = m->nvf;
    memset(Qs, 0, m->nn * sizeof(double));
    const double Tinf = orc_T_inf(m, n);
    for (int64_t f = 0; f < m->n_cf; ++f) {
        const int32_t *v = m->cfaces + (int64_t)nv * f;
        const double *M = m->Mf + (int64_t)nv * nv * f;
        for (int i = 0; i < nv; ++i) {
            double acc = 0.0;
            for (int j = 0; j < nv; ++j) acc += M[nv * i + j] * (T[v[j]] - Tinf);
            Qs[v[i]] -= m->h * acc;
        }
    }
    const double b = m->T_amb - m->T_zero;
    for (int64_t f = 0; f < m->n_rf; ++f) {
        const int32_t *v = m->rfaces + (int64_t)nv * f;
        const double *W = m->Wf + (int64_t)m->nfq * f;
        for (int p = 0; p < m->nfq; ++p) {
            double Tp = 0.0;
            for (int j = 0; j < nv; ++j) Tp += m->Nf[nv * p + j] * T[v[j]];
            const double a = Tp - m->T_zero;
            const double flux = ORC_SIGMA * m->eps * (a * a * a * a - b * b * b * b);
            for (int i = 0; i < nv; ++i) Qs[v[i]] -= W[p] * m->Nf[nv * p + i] * flux;
        }
    }
}

/* Load multiplier and convection ambient temperature at step n. */
static double orc_q_scale(const orc_model *m, int64_t n)
{
    if (!m->q_sched || m->n_sched <= 0) return 1.0;
    return m->q_sched[n < m->n_sched ? n : m->n_sched - 1];
}

static double orc_T_inf(const orc_model *m, int64_t n)
{
    if (!m->Tinf_sched || m->n_sched <= 0) return m->T_inf;
    return m->Tinf_sched[n < m->n_sched ? n : m->n_sched - 1];
}

/* Offset of the prescribed temperatures at step n (0 without a Dirichlet schedule). */
static double orc_T_dir_offset(const orc_model *m, int64_t n)
{
    if (!m->Tdir_sched || m->n_sched <= 0) return 0.0;
    return m->Tdir_sched[n < m->n_sched ? n : m->n_sched - 1];
}

/* Dirichlet values of step n written into T (Gamma_E of Eq. 3 with a time-dependent value). */
static void orc_impose_dirichlet(const orc_model *m, double *T, int64_t n)
{
    if (!m->Tdir_sched || !m->Tdir) return;
    const double d = orc_T_dir_offset(m, n);
    for (int64_t i = 0; i < m->nn; ++i)
        if (m->isdir[i]) T[i] = m->Tdir[i] + d;
}

/* Net external nodal heat flow Q_i at step n (Eq. 4, 5, 7 lumped to nodes). */
static double orc_nodal_Q_n(const orc_model *m, int64_t i, double Ti, int64_t n)
{
    const double a = Ti - m->T_zero, b = m->T_amb - m->T_zero;
    return orc_q_scale(m, n) * m->Qext[i] - m->Ac[i] * m->h * (Ti - orc_T_inf(m, n))
         - m->Ar[i] * ORC_SIGMA * m->eps * (a * a * a * a - b * b * b * b);
}

/* Net external nodal heat flow Q_i at the first step of a run. */
double orc_nodal_Q(const orc_model *m, int64_t i, double Ti)
{
    return orc_nodal_Q_n(m, i, Ti, m->sched_step0);
}

/* dQ_i/dT_i */
static double orc_nodal_dQ(const orc_model *m, int64_t i, double Ti)
{
    const double a = Ti - m->T_zero;
    return -m->Ac[i] * m->h - m->Ar[i] * ORC_SIGMA * m->eps * 4.0 * a * a * a;
}

/*
 * n explicit steps (Eq. 15 / 16) from T (in/out, Dirichlet values already imposed; with a
 * Dirichlet schedule they are set to those of step sched_step0 first and to those of step
 * n + 1 after step n).
 * energy (optional, [n][2]): per step S = sum_free C_i(T_i)(T_i' - T_i) and
 * B = dt (sum_free Q_i + sum_Dirichlet F_i).
 * trace (optional): T at the sensor nodes after every `sample_every`-th step, [n/sample_every][ns].
 */
void orc_run(const orc_model *m, double dt, int64_t nsteps, double *T, double *energy,
             const int32_t *sensors, int32_t ns, int32_t sample_every, double *trace)
{
    double *F = (double *)malloc(m->nn * sizeof(double));
    double *Qs = m->nfq > 0 ? (double *)malloc(m->nn * sizeof(double)) : NULL;
    orc_impose_dirichlet(m, T, m->sched_step0);
    for (int64_t n = 0; n < nsteps; ++n) {
        orc_internal_loads(m, T, F);
        if (Qs) orc_surface_loads(m, T, m->sched_step0 + n, Qs);
        double S = 0.0, B = 0.0;
        for (int64_t i = 0; i < m->nn; ++i) {
            if (m->isdir[i]) {
                B += dt * F[i];
                continue;
            }
            const double Q = Qs ? orc_q_scale(m, m->sched_step0 + n) * m->Qext[i] + Qs[i]
                                : orc_nodal_Q_n(m, i, T[i], m->sched_step0 + n);
            const double Ci = m->C0[i] * orc_fc(m, T[i]);
            const double Tn = T[i] + dt / Ci * (Q - F[i]);
            S += Ci * (Tn - T[i]);
            B += dt * Q;
            T[i] = Tn;
        }
        orc_impose_dirichlet(m, T, m->sched_step0 + n + 1);
        if (energy) {
            energy[2 * n] = S;
            energy[2 * n + 1] = B;
        }
        if (trace && sample_every > 0 && (n + 1) % sample_every == 0) {
            const int64_t k = (n + 1) / sample_every - 1;
            for (int s = 0; s < ns; ++s) trace[k * ns + s] = T[sensors[s]];
        }
    }
    free(F);
    free(Qs);
}

/*
 * Critical time step (Section 3.4, Eq. 29).  lambda_cond = largest eigenvalue of
 * C0^-1/2 K0 C0^-1/2 on the free nodes (K0 = sum_e theta_e K0_e) by FP64 power iteration
 * (stops when the Rayleigh quotient changes by < tol relative, or after max_iter);
 *   lambda = lambda_cond * max f_k / min f_c + max_i (A^c_i h + A^r_i 4 sigma eps max|T - T_z|^3)
 *            / (C0_i min f_c),  extrema over [T_lo, T_hi];   dt_crit = 2 / lambda.
 * out[0] = dt_crit, out[1] = lambda_cond, out[2] = iterations used.
 */
/*
 * dt_crit = 2 / (lambda_cond max f_k / min f_c + max_i (A^c_i h + A^r_i 4 sigma eps max|T - T_z|^3)
 * / (C0_i min f_c)) with the extrema over [T_lo, T_hi] (Section 3.4).
 */
double orc_dt_from_lambda(const orc_model *m, double lam, double T_lo, double T_hi)
{
    double fk_max, fc_min;
    orc_factor_extrema(m, T_lo, T_hi, &fk_max, &fc_min);
    const double rl = fabs(T_lo - m->T_zero), rh = fabs(T_hi - m->T_zero);
    const double r3 = fmax(rl * rl * rl, rh * rh * rh);
    double surf = 0.0;
    for (int64_t i = 0; i < m->nn; ++i) {
        if (m->isdir[i]) continue;
        const double s = (m->Ac[i] * m->h + m->Ar[i] * 4.0 * ORC_SIGMA * m->eps * r3) / (m->C0[i] * fc_min);
        if (s > surf) surf = s;
    }
    return 2.0 / (lam * fk_max / fc_min + surf);
}

typedef void (*orc_loads_fn)(const orc_model *m, const double *T, double *F, void *aux);

static void orc_loads_serial(const orc_model *m, const double *T, double *F, void *aux)
{
    (void)aux;
    orc_internal_loads(m, T, F);
}

static void orc_dt_crit_with(const orc_model *m, double T_lo, double T_hi, double tol, int64_t max_iter,
                             double *out, orc_loads_fn loads, void *aux);

void orc_dt_crit(const orc_model *m, double T_lo, double T_hi, double tol, int64_t max_iter, double *out)
{
    orc_dt_crit_with(m, T_lo, T_hi, tol, max_iter, out, orc_loads_serial, NULL);
}

static void orc_dt_crit_with(const orc_model *m, double T_lo, double T_hi, double tol, int64_t max_iter,
                             double *out, orc_loads_fn loads, void *aux)
{
    const int64_t nn = m->nn;
    double *x = (double *)malloc(nn * sizeof(double));
    double *y = (double *)malloc(nn * sizeof(double));
    double *F = (double *)malloc(nn * sizeof(double));
    orc_model lin = *m;
    lin.k_lin = 0.0;
    lin.n_tab = 0;
    lin.nq = 0; /* K0 itself (the sum of the point matrices) */
    double nrm = 0.0;
    for (int64_t i = 0; i < nn; ++i) {
        x[i] = m->isdir[i] ? 0.0 : 1.0 + 0.5 * sin(0.7 * (double)i + 0.3);
        nrm += x[i] * x[i];
    }
    nrm = sqrt(nrm);
    for (int64_t i = 0; i < nn; ++i) x[i] /= nrm;
    double lam = 0.0;
    int64_t it;
    for (it = 0; it < max_iter; ++it) {
        for (int64_t i = 0; i < nn; ++i) y[i] = m->isdir[i] ? 0.0 : x[i] / sqrt(m->C0[i]);
        loads(&lin, y, F, aux);
        double rq = 0.0, yy = 0.0;
        for (int64_t i = 0; i < nn; ++i) {
            y[i] = m->isdir[i] ? 0.0 : F[i] / sqrt(m->C0[i]);
            rq += x[i] * y[i];
            yy += y[i] * y[i];
        }
        yy = sqrt(yy);
        for (int64_t i = 0; i < nn; ++i) x[i] = y[i] / yy;
        const double done = fabs(rq - lam) <= tol * fabs(rq);
        lam = rq;
        if (done) break;
    }
    out[0] = orc_dt_from_lambda(m, lam, T_lo, T_hi);
    out[1] = lam;
    out[2] = (double)it;
    free(x);
    free(y);
    free(F);
}

/*
 * Discrete adjoint of n explicit steps (derived by hand from Eq. 16 and Eq. 20 for the loss
 * L(trace) with trace sampled after every `sample_every`-th step).  All states T^0..T^n are
 * kept (no checkpointing).  With a_i = dt / (C0_i f_c(T_i)) on free nodes (0 on Dirichlet),
 * mu_i = a_i lambda_i^{n+1}:
 *   lambda_j^n = dL/dT_j^n + lambda_j^{n+1} (1 + a_j'(T_j) R_j) + mu_j dQ_j/dT_j
 *              - sum_{e∋j} theta_e [ f_k,e (K0_e mu_e)_j + (mu_e . K0_e T_e) f_k'(T_j) / npe ],
 *   R_j = Q_j - F_j,  a_j' = -a_j f_c'(T_j) / f_c(T_j),
 *   dL/dtheta_e = -sum_n f_k,e mu_e . K0_e T_e^n,
 *   dL/ds_e = sum_n q_scale(n) sum_{i in e} mu_i w_ie (q_scale = 1 without a load schedule).
 * T0 [nn]: initial state (Dirichlet imposed); dLdtrace [n/sample_every][ns];
 * outputs g_theta [ne], g_source [ne] (overwritten); trace_out optional forward trace.
 */
void orc_adjoint(const orc_model *m, double dt, int64_t nsteps, const double *T0,
                 const int32_t *sensors, int32_t ns, int32_t sample_every, const double *dLdtrace,
                 double *g_theta, double *g_source)
{
    const int64_t nn = m->nn, ne = m->ne;
    const int npe = m->npe;
    double *states = (double *)malloc((size_t)(nsteps + 1) * nn * sizeof(double));
    memcpy(states, T0, nn * sizeof(double));
    orc_impose_dirichlet(m, states, m->sched_step0);
    for (int64_t n = 0; n < nsteps; ++n) {
        memcpy(states + (n + 1) * nn, states + n * nn, nn * sizeof(double));
        orc_model mn = *m;
        mn.sched_step0 = m->sched_step0 + n;
        orc_run(&mn, dt, 1, states + (n + 1) * nn, NULL, NULL, 0, 0, NULL);
    }
    double *lam = (double *)calloc(nn, sizeof(double));
    double *lnew = (double *)malloc(nn * sizeof(double));
    double *mu = (double *)malloc(nn * sizeof(double));
    double *F = (double *)malloc(nn * sizeof(double));
    double *musum = (double *)calloc(nn, sizeof(double));
    memset(g_theta, 0, ne * sizeof(double));
    for (int64_t n = nsteps; n >= 1; --n) {
        if (sample_every > 0 && n % sample_every == 0) {
            const int64_t k = n / sample_every - 1;
            for (int s = 0; s < ns; ++s) lam[sensors[s]] += dLdtrace[k * ns + s];
        }
        /* lam holds lambda^n; propagate through the step T^{n-1} -> T^n */
        const double *T = states + (n - 1) * nn;
        orc_internal_loads(m, T, F);
        for (int64_t i = 0; i < nn; ++i) {
            if (m->isdir[i]) {
                mu[i] = 0.0;
                lnew[i] = lam[i];
                continue;
            }
            const double fc = orc_fc(m, T[i]);
            const double a = dt / (m->C0[i] * fc);
            const int64_t step = m->sched_step0 + n - 1;
            const double R = orc_nodal_Q_n(m, i, T[i], step) - F[i];
            const double da = -a * orc_dfc(m, T[i]) / fc;
            mu[i] = a * lam[i];
            lnew[i] = lam[i] * (1.0 + da * R) + mu[i] * orc_nodal_dQ(m, i, T[i]);
            musum[i] += orc_q_scale(m, step) * mu[i];  /* d Q_i / d s_e = q_scale w_ie */
        }
        for (int64_t e = 0; e < ne; ++e) {
            const int32_t *c = m->conn + npe * e;
            const double *Ke = m->K + (int64_t)npe * npe * e;
            double fk = 0.0;
            for (int i = 0; i < npe; ++i) fk += orc_fk(m, T[c[i]]);
            fk /= npe;
            double muKT = 0.0;
            for (int i = 0; i < npe; ++i) {
                double kt = 0.0;
                for (int j = 0; j < npe; ++j) kt += Ke[npe * i + j] * T[c[j]];
                muKT += mu[c[i]] * kt;
            }
            for (int j = 0; j < npe; ++j) {
                double kmu = 0.0;
                for (int i = 0; i < npe; ++i) kmu += Ke[npe * i + j] * mu[c[i]];
                lnew[c[j]] -= m->theta[e] * (fk * kmu + muKT * orc_dfk(m, T[c[j]]) / npe);
            }
            g_theta[e] -= fk * muKT;
        }
        double *t = lam;
        lam = lnew;
        lnew = t;
    }
    for (int64_t e = 0; e < ne; ++e) {
        double s = 0.0;
        for (int i = 0; i < npe; ++i) s += musum[m->conn[npe * e + i]] * m->W[npe * e + i];
        g_source[e] = s;
    }
    free(states);
    free(lam);
    free(lnew);
    free(mu);
    free(F);
    free(musum);
}

/* ------------------------------------------------------------------------------------------ */
/* the same time stepping over all host cores (OpenMP)                                          */
/* ------------------------------------------------------------------------------------------ */

/*
 * Incidence of the mesh: for every node the (element, local index) pairs that touch it, in
 * increasing element order (ptr [nn + 1], ent [ne * npe] = e * npe + i).
 */
static void orc_node_incidence(const orc_model *m, int64_t *ptr, int64_t *ent)
{
    const int npe = m->npe;
    memset(ptr, 0, (m->nn + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < m->ne; ++e)
        for (int i = 0; i < npe; ++i) ++ptr[m->conn[npe * e + i] + 1];
    for (int64_t n = 0; n < m->nn; ++n) ptr[n + 1] += ptr[n];
    int64_t *fill = (int64_t *)malloc(m->nn * sizeof(int64_t));
    memcpy(fill, ptr, m->nn * sizeof(int64_t));
    for (int64_t e = 0; e < m->ne; ++e)
        for (int i = 0; i < npe; ++i) ent[fill[m->conn[npe * e + i]]++] = e * npe + i;
    free(fill);
}

/*
 * orc_run over nthreads host threads.  The element loop of Eq. 11 / 20 is split in two passes:
 * every element forms its load vector F_e = theta_e f_k,e K0_e T_e (elements in parallel),
 * then every node adds the loads of its elements in increasing element order (nodes in
 * parallel).  Each node therefore receives the same terms in the same order as in the serial
 * element loop with scatter, so the result is bitwise that of orc_run.  The nodal update is
 * independent per node (Eq. 16); the energy sums are added in node order afterwards.
 * Same arguments as orc_run; nthreads <= 0 uses the OpenMP default.
 */
void orc_run_mt(const orc_model *m, double dt, int64_t nsteps, double *T, double *energy,
                const int32_t *sensors, int32_t ns, int32_t sample_every, double *trace, int32_t nthreads)
{
    const int64_t nn = m->nn, ne = m->ne;
    const int npe = m->npe;
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    const int nt = 1;
    (void)nthreads;
#endif
    int64_t *ptr = (int64_t *)malloc((nn + 1) * sizeof(int64_t));
    int64_t *ent = (int64_t *)malloc((size_t)ne * npe * sizeof(int64_t));
    double *Fe = (double *)malloc((size_t)ne * npe * sizeof(double));
    double *Tn = (double *)malloc(nn * sizeof(double));
    double *Sn = energy ? (double *)malloc(nn * sizeof(double)) : NULL;
    double *Bn = energy ? (double *)malloc(nn * sizeof(double)) : NULL;
    double *Qs = m->nfq > 0 ? (double *)malloc(nn * sizeof(double)) : NULL;
    orc_node_incidence(m, ptr, ent);
    orc_impose_dirichlet(m, T, m->sched_step0);
    for (int64_t n = 0; n < nsteps; ++n) {
        const int64_t step = m->sched_step0 + n;
        if (Qs) orc_surface_loads(m, T, step, Qs);
#pragma omp parallel num_threads(nt)
        {
#pragma omp for schedule(static)
            for (int64_t e = 0; e < ne; ++e) orc_element_loads(m, e, T, Fe + npe * e);
#pragma omp for schedule(static)
            for (int64_t i = 0; i < nn; ++i) {
                double F = 0.0;
                for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) F += Fe[ent[q]];
                if (m->isdir[i]) {
                    Tn[i] = T[i];
                    if (energy) {
                        Sn[i] = 0.0;
                        Bn[i] = dt * F;
                    }
                    continue;
                }
                const double Q = Qs ? orc_q_scale(m, step) * m->Qext[i] + Qs[i] : orc_nodal_Q_n(m, i, T[i], step);
                const double Ci = m->C0[i] * orc_fc(m, T[i]);
                const double t = T[i] + dt / Ci * (Q - F);
                if (energy) {
                    Sn[i] = Ci * (t - T[i]);
                    Bn[i] = dt * Q;
                }
                Tn[i] = t;
            }
        }
        memcpy(T, Tn, nn * sizeof(double));
        orc_impose_dirichlet(m, T, step + 1);
        if (energy) {
            double S = 0.0, B = 0.0;
            for (int64_t i = 0; i < nn; ++i) {
                S += Sn[i];
                B += Bn[i];
            }
            energy[2 * n] = S;
            energy[2 * n + 1] = B;
        }
        if (trace && sample_every > 0 && (n + 1) % sample_every == 0) {
            const int64_t k = (n + 1) / sample_every - 1;
            for (int s = 0; s < ns; ++s) trace[k * ns + s] = T[sensors[s]];
        }
    }
    free(ptr);
    free(ent);
    free(Fe);
    free(Tn);
    free(Sn);
    free(Bn);
    free(Qs);
}

/* Eq. 11 / 20 over nthreads threads: element pass, then node gather in element order (bitwise
 * orc_internal_loads).  aux: the incidence and scratch of orc_loads_mt_ctx. */
typedef struct {
    int64_t *ptr, *ent;
    double *Fe;
    int nt;
} orc_loads_mt_ctx;

static void orc_loads_mt(const orc_model *m, const double *T, double *F, void *aux)
{
    const orc_loads_mt_ctx *x = (const orc_loads_mt_ctx *)aux;
    const int npe = m->npe;
    const int64_t ne = m->ne, nn = m->nn;
#pragma omp parallel num_threads(x->nt)
    {
#pragma omp for schedule(static)
        for (int64_t e = 0; e < ne; ++e) orc_element_loads(m, e, T, x->Fe + npe * e);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < nn; ++i) {
            double f = 0.0;
            for (int64_t q = x->ptr[i]; q < x->ptr[i + 1]; ++q) f += x->Fe[x->ent[q]];
            F[i] = f;
        }
    }
}

/* orc_dt_crit with the internal loads over nthreads threads (bitwise the same result). */
void orc_dt_crit_mt(const orc_model *m, double T_lo, double T_hi, double tol, int64_t max_iter, double *out,
                    int32_t nthreads)
{
    orc_loads_mt_ctx x;
#ifdef _OPENMP
    x.nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    x.nt = 1;
    (void)nthreads;
#endif
    x.ptr = (int64_t *)malloc((m->nn + 1) * sizeof(int64_t));
    x.ent = (int64_t *)malloc((size_t)m->ne * m->npe * sizeof(int64_t));
    x.Fe = (double *)malloc((size_t)m->ne * m->npe * sizeof(double));
    orc_node_incidence(m, x.ptr, x.ent);
    orc_dt_crit_with(m, T_lo, T_hi, tol, max_iter, out, orc_loads_mt, &x);
    free(x.ptr);
    free(x.ent);
    free(x.Fe);
}

/* ------------------------------------------------------------------------------------------ */
/* method variants: conductivity at quadrature points, consistent face integration            */
/* ------------------------------------------------------------------------------------------ */

/*
 * Quadrature rule of a boundary face: quadrilaterals (bilinear, corners (-1,-1), (1,-1), (1,1),
 * (-1,1)) by 3x3 Gauss-Legendre points (0, +-sqrt(3/5); weights 8/9, 5/9), exact for degree 5 in
 * each coordinate; triangles by Radon's 7-point rule of degree 5 (centroid, and two orbits of
 * three points with barycentric coordinates (a, a, 1 - 2a), a = (6 -+ sqrt 15) / 21), weights
 * normalised to sum 1.  Nf [nfq][nv] shape values, wref [nfq] reference weights.  Returns nfq.
 */
int orc_face_rule(int nv, double *Nf, double *wref)
{
    if (nv == 4) {
        const double g = sqrt(0.6);
        const double pt[3] = {-g, 0.0, g}, wt[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
        static const double S[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
        int p = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b, ++p) {
                for (int i = 0; i < 4; ++i) Nf[4 * p + i] = (1.0 + pt[a] * S[i][0]) * (1.0 + pt[b] * S[i][1]) / 4.0;
                wref[p] = wt[a] * wt[b];
            }
        return 9;
    }
    const double r = sqrt(15.0);
    const double a1 = (6.0 - r) / 21.0, a2 = (6.0 + r) / 21.0;
    const double w0 = 9.0 / 40.0, w1 = (155.0 - r) / 1200.0, w2 = (155.0 + r) / 1200.0;
    double L[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                      {a1, a1, 1 - 2 * a1}, {a1, 1 - 2 * a1, a1}, {1 - 2 * a1, a1, a1},
                      {a2, a2, 1 - 2 * a2}, {a2, 1 - 2 * a2, a2}, {1 - 2 * a2, a2, a2}};
    const double W[7] = {w0, w1, w1, w1, w2, w2, w2};
    for (int p = 0; p < 7; ++p) {
        for (int i = 0; i < 3; ++i) Nf[3 * p + i] = L[p][i];
        wref[p] = W[p];
    }
    return 7;
}

/*
 * Consistent face data of nf faces (node ids [nf][nv] into xyz): the face mass matrices
 * Mf [nf][nv][nv] = int_f N_i N_j dA and the quadrature weights times the area Jacobian
 * Wf [nf][nfq] of the rule of orc_face_rule (quadrilateral: |x_s x x_t| at the point, reference
 * area 4; triangle: the area, weights summing to 1).
 */
void orc_face_consistent(int64_t nf, int32_t nv, const int32_t *faces, const double *xyz, double *Mf, double *Wf)
{
    double Nf[9 * 4], wref[9];
    const int nfq = orc_face_rule(nv, Nf, wref);
    static const double S[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
    for (int64_t f = 0; f < nf; ++f) {
        double x[4][3];
        for (int i = 0; i < nv; ++i)
            for (int r = 0; r < 3; ++r) x[i][r] = xyz[3 * (int64_t)faces[nv * f + i] + r];
        double *W = Wf + (int64_t)nfq * f;
        if (nv == 3) {
            double a[3], b[3];
            for (int r = 0; r < 3; ++r) {
                a[r] = x[1][r] - x[0][r];
                b[r] = x[2][r] - x[0][r];
            }
            const double c0 = a[1] * b[2] - a[2] * b[1], c1 = a[2] * b[0] - a[0] * b[2], c2 = a[0] * b[1] - a[1] * b[0];
            const double A = 0.5 * sqrt(c0 * c0 + c1 * c1 + c2 * c2);
            for (int p = 0; p < nfq; ++p) W[p] = A * wref[p];
        } else {
            const double g = sqrt(0.6);
            const double pt[3] = {-g, 0.0, g};
            int p = 0;
            for (int ia = 0; ia < 3; ++ia)
                for (int ib = 0; ib < 3; ++ib, ++p) {
                    const double s = pt[ia], t = pt[ib];
                    double xs[3] = {0, 0, 0}, xt[3] = {0, 0, 0};
                    for (int i = 0; i < 4; ++i)
                        for (int r = 0; r < 3; ++r) {
                            xs[r] += x[i][r] * S[i][0] * (1.0 + t * S[i][1]) / 4.0;
                            xt[r] += x[i][r] * (1.0 + s * S[i][0]) * S[i][1] / 4.0;
                        }
                    const double c0 = xs[1] * xt[2] - xs[2] * xt[1];
                    const double c1 = xs[2] * xt[0] - xs[0] * xt[2];
                    const double c2 = xs[0] * xt[1] - xs[1] * xt[0];
                    W[p] = wref[p] * sqrt(c0 * c0 + c1 * c1 + c2 * c2);
                }
        }
        double *M = Mf + (int64_t)nv * nv * f;
        for (int i = 0; i < nv; ++i)
            for (int j = 0; j < nv; ++j) {
                double acc = 0.0;
                for (int p = 0; p < nfq; ++p) acc += W[p] * Nf[nv * p + i] * Nf[nv * p + j];
                M[nv * i + j] = acc;
            }
    }
}

/*
 * Quadrature-point matrices of every element for conductivity evaluated at the points:
 * hexahedra with the 2x2x2 rule (nq = 8, orc_hex_matrices_qp), or with one_point = 1 the single
 * centre point of Eq. 17 (nq = 1, N_i = 1/8); tetrahedra one point at the centroid (nq = 1,
 * N_i = 1/4, the exact matrix of Eq. 18: the gradients are constant).  Kq [ne][nq][npe][npe],
 * Nq [nq][npe].  Returns 0, or 1 + e for the first element e with det J <= 0.
 */
int64_t orc_precompute_qp(int64_t ne, int32_t npe, const double *xyz, const int32_t *conn, const int32_t *elem_mat,
                          const double *mat_k0, int32_t one_point, double *Kq, double *Nq)
{
    double xe[8 * 3];
    const int nq = (npe == 8 && !one_point) ? 8 : 1;
    for (int64_t e = 0; e < ne; ++e) {
        const int m = elem_mat ? elem_mat[e] : 0;
        for (int i = 0; i < npe; ++i)
            for (int r = 0; r < 3; ++r) xe[3 * i + r] = xyz[3 * (int64_t)conn[npe * e + i] + r];
        double *K = Kq + (int64_t)nq * npe * npe * e;
        if (npe == 8 && nq == 8) {
            double N[64];
            if (orc_hex_matrices_qp(xe, mat_k0 + 9 * m, K, N)) return 1 + e;
            if (e == 0) memcpy(Nq, N, sizeof(N));
        } else if (npe == 8) {
            if (orc_hex_matrix_centre(xe, mat_k0 + 9 * m, K)) return 1 + e;
            for (int i = 0; i < 8; ++i) Nq[i] = 1.0 / 8.0;
        } else {
            double w[4], v;
            if (orc_tet_matrices(xe, mat_k0 + 9 * m, K, w, &v)) return 1 + e;
            for (int i = 0; i < 4; ++i) Nq[i] = 0.25;
        }
    }
    return 0;
}
