"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: exact closed forms, textbook
identities, the paper's patch test (Section 4.1, Fig. 2), an exact 1-D reduction, library
eigen-solvers, and finite differences of its own forward loop for the adjoint.
"""
import numpy as np
import pytest
import scipy.linalg
from scipy.special import erfc

import fedfem_inputs as fi
from oracle import oracle as O
from tests import brute

RNG = np.random.default_rng(1234)


def _rand_spd(rng):
    A = rng.standard_normal((3, 3))
    return A @ A.T + 0.5 * np.eye(3)


# ------------------------------------------------------------------------- element matrices --

@pytest.mark.parametrize("seed", range(5))
def test_brick_matches_tensor_product_closed_form(seed):
    """Eq. 12 on a rectangular brick with a full anisotropic k vs exact 1-D integral products."""
    rng = np.random.default_rng(seed)
    dims = rng.uniform(0.2, 2.0, size=3)
    k = _rand_spd(rng)
    x0 = rng.uniform(-1, 1, size=3)
    x = x0 + brute.VTK_CORNERS * dims
    K, w, vol = O.hex_matrices(x, k)
    Kc = brute.brick_K(dims, k)
    assert np.max(np.abs(K - Kc)) <= 1e-14 * np.max(np.abs(Kc)) * 10
    assert np.allclose(w, np.prod(dims) / 8, rtol=1e-14)
    assert vol == pytest.approx(np.prod(dims), rel=1e-14)


@pytest.mark.parametrize("seed", range(5))
def test_tet_matches_face_vector_formula(seed):
    """Eq. 18 (V B^T k B via the inverse of [1 x y z]) vs K_ij = S_i.k S_j / 9V."""
    rng = np.random.default_rng(100 + seed)
    x = rng.uniform(0, 1, size=(4, 3))
    if np.dot(np.cross(x[1] - x[0], x[2] - x[0]), x[3] - x[0]) < 0:
        x[[1, 2]] = x[[2, 1]]
    k = _rand_spd(rng)
    K, w, vol = O.tet_matrices(x, k)
    Kf, V = brute.tet_K_facevec(x, k)
    assert np.max(np.abs(K - Kf)) <= 1e-13 * np.max(np.abs(Kf))
    assert vol == pytest.approx(V, rel=1e-14)
    assert np.allclose(w, V / 4, rtol=1e-14)


def _parallelepiped(rng):
    """Corner nodes (VTK order) x0 + (s_x a + s_y b + s_z c) / 2 of a random parallelepiped
    with edge vectors a, b, c (positively oriented), and the matrix [a b c]."""
    E = rng.uniform(-0.3, 0.3, size=(3, 3)) + np.diag(rng.uniform(0.5, 2.0, size=3))
    if np.linalg.det(E) < 0:
        E[:, 0] *= -1
    s = 2.0 * brute.VTK_CORNERS - 1.0
    return rng.uniform(-1, 1, size=3) + 0.5 * s @ E.T, E, s


@pytest.mark.parametrize("seed", range(5))
def test_hex_centre_rule_closed_form_on_parallelepipeds(seed):
    """Eq. 17 on a parallelepiped: the shape-function gradients at the centre are
    grad N_i = [a b c]^-T s_i / 4 and 8 det J = V = det [a b c], so K = V G^T k G."""
    rng = np.random.default_rng(300 + seed)
    x, E, s = _parallelepiped(rng)
    k = _rand_spd(rng)
    G = np.linalg.solve(E.T, s.T) / 4.0          # [3, 8] gradients
    Kc = np.linalg.det(E) * G.T @ k @ G
    K = O.hex_matrix_centre(x, k)
    assert np.max(np.abs(K - Kc)) <= 1e-13 * np.max(np.abs(Kc))


@pytest.mark.parametrize("seed", range(3))
def test_hex_centre_rule_matches_gauss_on_linear_fields(seed):
    """On a parallelepiped the gradient of a linear field is constant and the centre value of
    grad N_i equals its element mean, so the one-point and 2x2x2 loads agree for linear T."""
    rng = np.random.default_rng(400 + seed)
    x, _, _ = _parallelepiped(rng)
    k = _rand_spd(rng)
    T = x @ rng.standard_normal(3) + rng.standard_normal()
    K1 = O.hex_matrix_centre(x, k)
    K8, _, _ = O.hex_matrices(x, k)
    assert np.max(np.abs(K1 @ T - K8 @ T)) <= 1e-12 * np.max(np.abs(K8 @ T))
    # ... but not for a general field (the one-point matrix has rank 3: hourglass modes)
    assert np.linalg.matrix_rank(K1) == 3 and np.linalg.matrix_rank(K8) == 7


def test_hex_centre_rule_invariants(patch_nodes):
    """Distorted hexahedron of the patch: K 1 = 0, symmetry, rank 3."""
    k = _rand_spd(np.random.default_rng(9))
    p = fi.patch_problem(patch_nodes, "hex")
    for e in range(p.n_elems):
        K = O.hex_matrix_centre(p.xyz[p.conn[e]], k)
        assert np.max(np.abs(K.sum(axis=1))) <= 1e-13 * np.max(np.abs(K))
        assert np.max(np.abs(K - K.T)) <= 1e-14 * np.max(np.abs(K))
        assert np.linalg.matrix_rank(K, tol=1e-10 * np.max(np.abs(K))) == 3


def test_distorted_elements_invariants(patch_nodes):
    """K 1 = 0 (a constant field carries no heat), symmetry, sum_i w_i = volume."""
    k = _rand_spd(np.random.default_rng(7))
    for kind in ("hex", "tet"):
        p = fi.patch_problem(patch_nodes, kind)
        for c in p.conn:
            x = p.xyz[c]
            K, w, vol = (O.hex_matrices if kind == "hex" else O.tet_matrices)(x, k)
            scale = np.max(np.abs(K))
            assert np.max(np.abs(K.sum(axis=1))) <= 1e-13 * scale
            assert np.max(np.abs(K - K.T)) <= 1e-14 * scale
            assert w.sum() == pytest.approx(vol, rel=1e-13)
        # the patch fills the unit cube exactly
        tot = sum((O.hex_matrices if kind == "hex" else O.tet_matrices)(p.xyz[c], k)[2] for c in p.conn)
        assert tot == pytest.approx(1.0, rel=1e-12)


def test_hex_shape_integrals_on_distorted_elements(patch_nodes):
    """w_i = int_Ve N_i dV (lumped masses and source loads, Section 3.1) on non-parallelepiped
    hexahedra: the oracle's 2x2x2 values against an independent 3x3x3 Gauss-Legendre
    integration on every element of the distorted patch and of a jittered cube, and against
    exact rational integration (sympy) on the patch's inner element.  A centre-point det J or a
    permuted node order in N_i fails this; sum_i w_i = V alone would not."""
    k = np.eye(3)
    xyz, conn = fi.cube_mesh(4, "hex", jitter=0.3, seed=11)
    elems = [fi.patch_problem(patch_nodes, "hex")]
    cases = [(e.xyz, e.conn) for e in elems] + [(xyz, conn)]
    worst = 0.0
    for X, Cn in cases:
        for c in Cn:
            _, w, vol = O.hex_matrices(X[c], k)
            w3, v3 = brute.hex_shape_integrals_gauss3(X[c])
            worst = max(worst, np.max(np.abs(w - w3)) / np.max(np.abs(w3)))
            assert vol == pytest.approx(v3, rel=1e-14)
            # distorted: the shares are not all equal
            assert np.ptp(w3) > 1e-3 * np.max(w3) or X is xyz
    assert worst <= 1e-14
    # the lumped thermal mass and source loads of the jittered cube assemble those w_i
    p = fi.Problem("j", xyz, conn, [fi.Material(2.0, k, 0.0, 3.0, 0.0)], T0=np.zeros(len(xyz)),
                   elem_source=np.linspace(1.0, 2.0, len(conn)))
    m = O.OracleModel(p)
    M = np.zeros(len(xyz))
    Q = np.zeros(len(xyz))
    for e, c in enumerate(conn):
        w3, _ = brute.hex_shape_integrals_gauss3(xyz[c])
        np.add.at(M, c, 6.0 * w3)
        np.add.at(Q, c, p.elem_source[e] * w3)
    assert np.max(np.abs(m.C0 - M)) <= 1e-14 * np.max(M)
    assert np.max(np.abs(m.Qext - Q)) <= 1e-14 * np.max(Q)
    pytest.importorskip("sympy")
    pe = fi.patch_problem(patch_nodes, "hex")
    x = pe.xyz[pe.conn[0]]
    we, ve = brute.hex_shape_integrals_exact(x)
    _, w, vol = O.hex_matrices(x, k)
    assert np.max(np.abs(w - we)) <= 1e-14 * np.max(we)
    assert vol == pytest.approx(ve, rel=1e-14)


def test_face_areas():
    """Quad area by bilinear-patch quadrature and triangle area vs closed forms."""
    sq = np.array([[0, 0, 0], [2, 0, 0], [2, 3, 0], [0, 3, 0]], float)
    assert O.face_area(sq) == pytest.approx(6.0, rel=1e-15)
    par = np.array([[0, 0, 0], [2, 0, 0], [3, 1, 1], [1, 1, 1]], float)   # parallelogram
    assert O.face_area(par) == pytest.approx(np.linalg.norm(np.cross(par[1] - par[0], par[3] - par[0])), rel=1e-14)
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 2, 0]], float)
    assert O.face_area(tri) == pytest.approx(1.0, rel=1e-15)


# ---------------------------------------------------------------------- assembly / scatter --

def _tiny_problems(patch_nodes):
    out = []
    for n in (2, 3):
        xyz, conn = fi.cube_mesh(n, "hex")
        out.append(("hex", n, xyz, conn))
    xyz, conn = fi.cube_mesh(3, "tet")
    out.append(("tet", 3, xyz, conn))
    return out


@pytest.mark.parametrize("which", range(3))
def test_element_loop_matches_dense_assembly(which, patch_nodes):
    """Eq. 11 / 20: the element loop with scatter equals a dense assembled K(T) T, including
    the per-element scale theta_e and the element-mean f_k of Section 4.2.2."""
    kind, n, xyz, conn = _tiny_problems(patch_nodes)[which]
    rng = np.random.default_rng(50 + which)
    k = _rand_spd(rng)
    h = 1.0 / n
    if kind == "hex":
        Ke = np.array([brute.brick_K((h, h, h), k)] * len(conn))
    else:
        Ke = np.array([brute.tet_K_facevec(xyz[c], k)[0] for c in conn])
    theta = rng.uniform(0.5, 2.0, size=len(conn))
    k_lin = 0.003
    p = fi.Problem("t", xyz, conn, [fi.Material(1.0, k, k_lin, 1.0, 0.0)], elem_kscale=theta,
                   T0=np.zeros(len(xyz)))
    m = O.OracleModel(p)
    T = rng.uniform(0, 300, size=len(xyz))
    fk = np.array([np.mean(1 + k_lin * T[c]) for c in conn])
    Kd = brute.dense_assemble(conn, Ke, len(xyz), theta * fk)
    ref = Kd @ T
    got = m.internal_loads(T)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    # constant field: no internal load
    Fc = m.internal_loads(np.full(len(xyz), 37.0))
    assert np.max(np.abs(Fc)) <= 1e-13 * 37.0 * np.max(np.abs(Kd))
    # internal loads sum to zero (conservation, Eq. 11)
    assert abs(got.sum()) <= 1e-13 * np.abs(got).sum()
    # a property table: the element factor is the mean of the nodal factors from numpy's
    # interpolation (end values held), not the factor of the mean temperature
    tT, tk = np.array([20.0, 90.0, 150.0, 260.0]), np.array([1.0, 2.2, 0.7, 1.5])
    m.set_table(tT, tk, np.ones(4))
    fk_tab = np.array([np.mean(np.interp(T[c], tT, tk)) for c in conn])
    ref_tab = brute.dense_assemble(conn, Ke, len(xyz), theta * fk_tab) @ T
    got_tab = m.internal_loads(T)
    assert np.max(np.abs(got_tab - ref_tab)) <= 1e-13 * np.max(np.abs(ref_tab))
    fk_mean = np.array([np.interp(np.mean(T[c]), tT, tk) for c in conn])
    assert np.max(np.abs(fk_mean - fk_tab)) > 1e-3  # the two readings differ on this field


# -------------------------------------------------------------------------- patch tests -----

@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_patch_test_steady_state(kind, patch_nodes):
    """Section 4.1: T = 200x + 100y + 200z on the cube corners; interior nodes must follow the
    same linear field at steady state (direct solve and explicit run to steady state)."""
    k = np.array([[3.0, 0.5, 0.2], [0.5, 2.0, 0.3], [0.2, 0.3, 1.0]])   # anisotropic too
    for kk in (np.eye(3), k):
        p = fi.patch_problem(patch_nodes, kind, k0=kk)
        m = O.OracleModel(p)
        lin = p.xyz @ np.array([200.0, 100.0, 200.0])
        free = p.free_mask()
        Kd = brute.dense_assemble(p.conn, m.K, p.n_nodes)
        Tf = np.linalg.solve(Kd[np.ix_(free, free)], -Kd[np.ix_(free, ~free)] @ lin[~free])
        assert np.max(np.abs(Tf - lin[free])) <= 1e-12 * np.max(np.abs(lin))
        dt = 0.9 * m.dt_crit()[0]
        T = m.run(p.initial_T(), dt, 20000)
        assert np.max(np.abs(T - lin)) <= 1e-10 * np.max(np.abs(lin))


# ----------------------------------------------------------- fully discrete closed form (C1) --

@pytest.mark.parametrize("nsteps", [1, 10, 50, 100, 1000])
def test_plain_cube_discrete_closed_form(nsteps):
    """Plain cube (10^3 bricks, T0 = 100, T = 0 on the boundary): the oracle equals the exact
    sine-mode solution of the lumped-mass forward-Euler system at every step count."""
    p = fi.plain_cube(10)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    ref, lam_max = brute.c1_closed_form(10, dt, nsteps)
    T = m.run(p.initial_T(), dt, nsteps)
    assert np.max(np.abs(T - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_plain_cube_critical_step_closed_form():
    """Section 3.4: lambda_max of the plain cube is the largest sine-mode eigenvalue."""
    p = fi.plain_cube(10)
    m = O.OracleModel(p)
    dtc, lam, _ = m.dt_crit(tol=1e-14)
    _, lam_max = brute.c1_closed_form(10, 1e-3, 0)
    assert lam == pytest.approx(lam_max, rel=1e-9)
    assert dtc == pytest.approx(2.0 / lam_max, rel=1e-9)
    assert 0.9 * dtc == pytest.approx(4.6836e-3, rel=1e-4)


def test_plain_cube_vs_continuum_series():
    """Reported error vs the continuum separable series (O(h^2) + O(dt)); a loose bound."""
    p = fi.plain_cube(10)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    T = m.run(p.initial_T(), dt, 10)
    t = 10 * dt
    x = p.xyz
    ser = np.zeros(len(x))
    for l in range(1, 60, 2):
        for mm in range(1, 60, 2):
            for q in range(1, 60, 2):
                ser += (6400.0 / (np.pi ** 3 * l * mm * q)) * np.sin(l * np.pi * x[:, 0]) \
                    * np.sin(mm * np.pi * x[:, 1]) * np.sin(q * np.pi * x[:, 2]) \
                    * np.exp(-np.pi ** 2 * (l * l + mm * mm + q * q) * t)
    centre = np.argmin(np.sum((x - 0.5) ** 2, axis=1))
    assert abs(T[centre] - ser[centre]) / ser[centre] < 0.1


@pytest.mark.parametrize("n", [2, 3])
def test_critical_step_vs_dense_eigensolver(n):
    """Power iteration vs scipy's generalized symmetric eigen-solver on tiny meshes."""
    for kind in ("hex", "tet"):
        p = fi.nonlinear_cube(n, kind)
        p.dir_nodes = np.array([0, 1], np.int32)
        p.dir_T = np.array([20.0, 20.0])
        m = O.OracleModel(p)
        free = p.free_mask()
        Kd = brute.dense_assemble(p.conn, m.K, p.n_nodes)
        lam = scipy.linalg.eigh(Kd[np.ix_(free, free)], np.diag(m.C0[free]), eigvals_only=True).max()
        _, lam_o, _ = m.dt_crit(tol=1e-15, max_iter=500000)
        assert lam_o == pytest.approx(lam, rel=1e-8)


def test_reference_temperature_law_is_a_rescaled_law():
    """k0 (1 + k_lin (T - T_ref)) = k0 (1 - k_lin T_ref) (1 + k_lin / (1 - k_lin T_ref) T), and
    the same for c: a law with a reference temperature gives the same run as the rescaled law
    with T_ref = 0 (pinned elsewhere), including the critical step."""
    p = fi.nonlinear_cube(4, "hex", jitter=0.2)
    m0 = p.mats[0]
    ref = fi.nonlinear_cube(4, "hex", jitter=0.2)
    Tr = 60.0
    p.mats[0] = fi.Material(m0.rho, m0.k0, 0.004, m0.c0, 0.002, T_ref=Tr)
    sk, sc = 1.0 - 0.004 * Tr, 1.0 - 0.002 * Tr
    ref.mats[0] = fi.Material(m0.rho, np.asarray(m0.k0) * sk, 0.004 / sk, m0.c0 * sc, 0.002 / sc)
    a, b = O.OracleModel(p), O.OracleModel(ref)
    assert a.dt_crit()[0] == pytest.approx(b.dt_crit()[0], rel=1e-9)
    dt = 0.9 * b.dt_crit()[0]
    Ta, Tb = a.run(p.initial_T(), dt, 200), b.run(ref.initial_T(), dt, 200)
    assert np.max(np.abs(Ta - Tb)) <= 1e-11 * np.max(np.abs(Tb))
    T = fi.random_state(p, 5)
    assert np.max(np.abs(a.internal_loads(T) - b.internal_loads(T))) <= 1e-11 * np.max(np.abs(b.internal_loads(T)))


def test_two_point_law_of_section_4_2_2():
    """The tabulated laws of Section 4.2.2 (k = 200 / 2000, c = 2000 / 8000 at 37 / 337 deg C,
    6 W/(m K) and 20 J/(kg K) per degree) as (lin, T_ref) laws."""
    k_lin, Tr = fi.two_point_law(37.0, 200.0, 337.0, 2000.0)
    c_lin, _ = fi.two_point_law(37.0, 2000.0, 337.0, 8000.0)
    assert Tr == 37.0
    assert 200.0 * (1 + k_lin * (337.0 - Tr)) == pytest.approx(2000.0, rel=1e-14)
    assert 200.0 * k_lin == pytest.approx(6.0, rel=1e-14)
    assert 2000.0 * c_lin == pytest.approx(20.0, rel=1e-14)


def test_two_point_table_is_the_linear_law():
    """A two-point table through a linear law, spanning every temperature of the run, is that
    law (run and dt_crit); extra collinear points change nothing."""
    p = fi.nonlinear_cube(5, "hex")
    m_lin = O.OracleModel(p)
    kl, cl = p.mats[0].k_lin, p.mats[0].c_lin
    dt = 0.9 * m_lin.dt_crit()[0]
    T_lin = m_lin.run(p.initial_T(), dt, 200)
    lo, hi = p.T_lo - 50.0, max(p.T_hi, T_lin.max()) + 50.0
    for pts in (np.array([lo, hi]), np.array([lo, 0.7 * lo + 0.3 * hi, 0.5 * (lo + hi), hi])):
        q = fi.nonlinear_cube(5, "hex")
        q.table_T, q.table_fk, q.table_fc = pts, 1.0 + kl * pts, 1.0 + cl * pts
        m = O.OracleModel(q)
        assert np.max(np.abs(m.run(q.initial_T(), dt, 200) - T_lin)) <= 1e-12 * np.abs(T_lin).max()
        assert m.dt_crit()[0] == pytest.approx(m_lin.dt_crit()[0], rel=1e-12)


@pytest.mark.parametrize("ny", [1, 2])
def test_slab_table_law_reduces_to_1d_recurrence(ny):
    """Tabulated k(T), c(T) (linear between points, end values held; Section 4.2.2 with more
    points): the bar reduces exactly to the 1-D recurrence whose element factor is the mean of
    the two nodal values from numpy's interpolation; the hot end lies past the last point."""
    nx, k, rho, c0 = 20, 2.0, 3.0, 1.5
    tT = np.array([10.0, 30.0, 55.0, 80.0])
    tk = np.array([1.0, 2.5, 1.8, 3.0])
    tc = np.array([1.0, 0.7, 1.6, 1.2])
    p = fi.slab(nx, ny, ny, Lx=1.0, k=(k, 7.0, 9.0), rho=rho, c0=c0, T0=0.0, T_s=100.0,
                conv_end=(4.0, 10.0))
    p.table_T, p.table_fk, p.table_fc = tT, tk, tc
    m = O.OracleModel(p)
    h = 1.0 / nx
    dt = 0.2 * rho * c0 * 0.7 * h * h / (k * 3.0 * 3.0)
    T = m.run(p.initial_T(), dt, 400)
    ref = brute.ftcs_slab(nx, h, dt, 400, 0.0, 100.0, k, rho, c0, conv=(4.0, 10.0),
                          fk_fn=lambda t: np.interp(t, tT, tk), fc_fn=lambda t: np.interp(t, tT, tc))
    ix = np.rint(p.xyz[:, 0] / h).astype(int)
    assert np.max(np.abs(T - ref[ix])) <= 1e-13 * 100.0
    assert ref.min() < tT[0] and ref.max() > tT[-1] and np.sum((ref > tT[1]) & (ref < tT[2])) > 0


def test_single_brick_table_capacity():
    """A uniform brick cooling by convection from above the table to below it: every node
    follows the scalar recurrence with c(T) from numpy's interpolation (end values held)."""
    a, b, c = 0.3, 0.5, 0.7
    rho, c0, hc, Tinf = 800.0, 900.0, 40.0, 15.0
    tT = np.array([50.0, 150.0, 300.0])
    tc = np.array([0.8, 1.5, 1.1])
    p = fi.single_brick(a, b, c, rho, c0, 0.0, T0=400.0, conv=(hc, Tinf))
    p.table_T, p.table_fk, p.table_fc = tT, np.array([1.0, 3.0, 2.0]), tc
    m = O.OracleModel(p)
    A = (a * b + b * c + c * a) / 4.0
    Cn = rho * c0 * a * b * c / 8.0
    dt, n = 20.0, 400
    T = m.run(p.initial_T(), dt, n)
    s = 400.0
    for _ in range(n):
        s = s + dt / (Cn * np.interp(s, tT, tc)) * (-A * hc * (s - Tinf))
    assert s < tT[0]
    assert np.max(np.abs(T - s)) <= 1e-12 * 400.0


def test_table_critical_step_extrema():
    """dt_crit with a table: 2 min f_c / (lambda max f_k) with the extrema of the interpolated
    factors taken by brute force on a fine grid over [T_lo, T_hi] (no surface terms)."""
    p = fi.nonlinear_cube(3, "hex")
    p.h, p.eps = 0.0, 0.0
    p.conv_faces, p.rad_faces = None, None
    tT = np.array([-100.0, 137.0, 512.0, 2000.0])
    p.table_T, p.table_fk, p.table_fc = tT, np.array([1.0, 4.0, 2.0, 3.5]), np.array([2.0, 2.5, 0.6, 0.9])
    m = O.OracleModel(p)
    lam = 7.0
    for lo, hi in ((0.0, 1000.0), (200.0, 400.0), (-500.0, 3000.0)):
        g = np.linspace(lo, hi, 1_000_001)
        fk, fc = np.interp(g, tT, p.table_fk), np.interp(g, tT, p.table_fc)
        assert m.dt_from_lambda(lam, lo, hi) == pytest.approx(2.0 * fc.min() / (lam * fk.max()), rel=1e-6)


def test_adaptive_step_is_the_fixed_step_without_temperature_laws():
    """Without k(T), c(T) and radiation dt_crit does not depend on the temperature range, so
    the per-launch adaptive step is the fixed step: same field (bitwise) and time n dt."""
    p = fi.nonlinear_cube(4, "hex")
    m0 = p.mats[0]
    p.mats[0] = fi.Material(m0.rho, m0.k0, 0.0, m0.c0, 0.0)
    p.rad_faces = None
    m = O.OracleModel(p)
    lam = m.dt_crit()[1]
    dt = 0.8 * m.dt_from_lambda(lam, -100.0, 5000.0)
    T1, t = m.run_adaptive(p.initial_T(), 130, 40, 0.8, 7.0, lam)
    assert np.array_equal(T1, m.run(p.initial_T(), dt, 130))
    assert t == pytest.approx(130 * dt, rel=1e-15)


def test_adaptive_step_follows_the_heating_range():
    """Heating nonlinear cube: the critical step shrinks as the range grows (f_k and the
    radiation rate grow with T), so the adaptive steps do not increase, and the run stays finite
    far above the range a fixed step would have been chosen for."""
    p = fi.nonlinear_cube(6, "hex")
    m = O.OracleModel(p)
    lam = m.dt_crit()[1]
    assert m.dt_from_lambda(lam, 20.0, 400.0) < m.dt_from_lambda(lam, 20.0, 40.0)
    T, dts, done = p.initial_T(), [], 0
    while done < 400:
        dts.append(0.9 * m.dt_from_lambda(lam, T.min(), T.max()))
        T = m.run(T, dts[-1], 50, step0=done)
        done += 50
    assert np.all(np.isfinite(T)) and T.max() > 300.0
    assert np.all(np.diff(dts) <= 1e-12 * dts[0])


# ------------------------------------------------------------------------------ slab ------

@pytest.mark.parametrize("ny", [1, 2])
@pytest.mark.parametrize("nonlinear", [False, True])
def test_slab_reduces_to_1d_recurrence(ny, nonlinear):
    """A bar of bricks with T held at x = 0 and fields constant over cross-sections reduces
    exactly to the 1-D forward-Euler recurrence (consistent brick row sums = lumped mass);
    the nonlinear variant pins the element-mean k(T) and nodal c(T)."""
    nx, k, rho, c0 = 20, 2.0, 3.0, 1.5
    kl, cl = (0.01, 0.004) if nonlinear else (0.0, 0.0)
    src = 50.0
    p = fi.slab(nx, ny, ny, Lx=1.0, k=(k, 7.0, 9.0), rho=rho, c0=c0, k_lin=kl, c_lin=cl,
                T0=0.0, T_s=100.0, conv_end=(4.0, 10.0))
    p.elem_source = np.full(p.n_elems, src)
    m = O.OracleModel(p)
    h = 1.0 / nx
    dt = 0.2 * rho * c0 * h * h / (k * 3.0)
    T = m.run(p.initial_T(), dt, 300)
    ref = brute.ftcs_slab(nx, h, dt, 300, 0.0, 100.0, k, rho, c0, kl, cl, conv=(4.0, 10.0),
                          source=src)
    ix = np.rint(p.xyz[:, 0] / h).astype(int)
    assert np.max(np.abs(T - ref[ix])) <= 1e-13 * 100.0


@pytest.mark.parametrize("nonlinear", [False, True])
def test_slab_time_dependent_dirichlet(nonlinear):
    """A prescribed temperature that changes every step (T_s + d[n], the last entry held):
    the bar still reduces exactly to the 1-D recurrence with the same end values; a run split
    in two with step0 continues the schedule, and d = 0 is the constant-value run."""
    nx, k, rho, c0 = 16, 2.0, 3.0, 1.5
    kl, cl = (0.01, 0.004) if nonlinear else (0.0, 0.0)
    p = fi.slab(nx, 2, 2, Lx=1.0, k=(k, 7.0, 9.0), rho=rho, c0=c0, k_lin=kl, c_lin=cl,
                T0=20.0, T_s=20.0, conv_end=(4.0, 10.0))
    n = 120
    d = 60.0 * np.sin(0.05 * np.arange(n)) + 0.5 * np.arange(n)
    h = 1.0 / nx
    dt = 0.2 * rho * c0 * h * h / (k * 3.0)
    ix = np.rint(p.xyz[:, 0] / h).astype(int)
    m = O.OracleModel(p)
    T_const = m.run(p.initial_T(), dt, 200)
    m.set_schedule(T_dir=np.zeros(n))
    assert np.array_equal(m.run(p.initial_T(), dt, 200), T_const)
    m.set_schedule(T_dir=d)
    T = m.run(p.initial_T(), dt, 200)
    ref = brute.ftcs_slab(nx, h, dt, 200, 20.0, 20.0, k, rho, c0, kl, cl, conv=(4.0, 10.0),
                          Ts_offset=d)
    assert np.max(np.abs(T - ref[ix])) <= 1e-13 * 100.0
    assert np.all(T[p.dir_nodes] == 20.0 + d[-1])
    T1 = m.run(p.initial_T(), dt, 75)
    T2 = m.run(T1, dt, 125, step0=75)
    assert np.max(np.abs(T2 - T)) <= 1e-13 * 100.0


def test_slab_erfc_convergence():
    """Semi-infinite-slab closed form T0 + (Ts - T0) erfc(x / 2 sqrt(alpha t)): the error
    shrinks as the mesh is refined (O(h^2) with dt ~ h^2)."""
    errs = []
    for nx in (20, 40, 80):
        h = 1.0 / nx
        p = fi.slab(nx, 1, 1, Lx=1.0, k=(1.0, 1.0, 1.0), rho=1.0, c0=1.0, T0=0.0, T_s=1.0)
        m = O.OracleModel(p)
        dt = 0.25 * h * h
        t_end = 0.01
        ns = int(round(t_end / dt))
        T = m.run(p.initial_T(), dt, ns)
        x = p.xyz[:, 0]
        exact = erfc(x / (2.0 * np.sqrt(ns * dt)))
        sel = x <= 0.5
        errs.append(np.max(np.abs(T[sel] - exact[sel])))
    assert errs[1] < 0.5 * errs[0] and errs[2] < 0.5 * errs[1]


# ----------------------------------------------------------------------- surface loads ----

def test_single_brick_surface_ode():
    """One brick with convection and radiation on all faces: every node has the same
    area / mass ratio, a uniform field stays uniform and each node follows the scalar
    forward-Euler ODE  C(T) dT = -A [h (T - T_inf) + sigma eps (T_K^4 - T_aK^4)] dt  (Kelvin)."""
    a, b, c = 0.3, 0.5, 0.7
    rho, c0, cl = 800.0, 900.0, 0.002
    hc, Tinf, eps, Ta = 40.0, 15.0, 0.7, -50.0
    p = fi.single_brick(a, b, c, rho, c0, cl, T0=400.0, conv=(hc, Tinf), rad=(eps, Ta))
    m = O.OracleModel(p)
    A = (a * b + b * c + c * a) / 4.0
    Cn = rho * c0 * a * b * c / 8.0
    assert np.allclose(m.Ac, A, rtol=1e-14) and np.allclose(m.Ar, A, rtol=1e-14)
    assert np.allclose(m.C0, Cn, rtol=1e-14)
    dt = 0.5
    T = m.run(p.initial_T(), dt, 200)
    s = 400.0
    for _ in range(200):
        tk, tak = s + 273.15, Ta + 273.15
        q = -A * (hc * (s - Tinf) + 5.67e-8 * eps * (tk ** 4 - tak ** 4))
        s = s + dt / (Cn * (1 + cl * s)) * q
    assert np.max(np.abs(T - s)) <= 1e-12 * abs(s)


def test_single_brick_nodal_loads():
    """Concentrated nodal heat flows (Eq. 5 applied as nodal loads): uniform heating
    dT = dt q / C_i when every node receives the same q."""
    p = fi.single_brick(0.2, 0.3, 0.4, rho=10.0, c0=3.0, T0=5.0)
    p.nodal_Q = np.full(8, 0.7)
    m = O.OracleModel(p)
    Cn = 10.0 * 3.0 * 0.024 / 8
    T = m.run(p.initial_T(), 0.01, 7)
    assert np.allclose(T, 5.0 + 7 * 0.01 * 0.7 / Cn, rtol=1e-14)


def test_single_brick_time_dependent_loads():
    """Load schedule on the single brick: a nodal heat flow scaled by q(n) and a convection
    ambient temperature T_inf(n) at step n (the last entry held beyond the end) follow the
    scalar forward-Euler recurrence with the same per-step values; a run split in two with
    step0 continues the schedule."""
    a, b, c = 0.3, 0.5, 0.7
    rho, c0, cl = 800.0, 900.0, 0.002
    hc = 40.0
    p = fi.single_brick(a, b, c, rho, c0, cl, T0=100.0, conv=(hc, 15.0))
    p.nodal_Q = np.full(8, 3.0)
    n = 150
    steps = np.arange(n)
    p.q_schedule = 1.0 + 0.5 * np.sin(0.1 * steps)
    p.Tinf_schedule = 15.0 + 30.0 * (steps / n)
    m = O.OracleModel(p)
    A = (a * b + b * c + c * a) / 4.0
    Cn = rho * c0 * a * b * c / 8.0
    dt = 0.5
    T = m.run(p.initial_T(), dt, n + 40)
    s = 100.0
    for k in range(n + 40):
        j = min(k, n - 1)
        q = p.q_schedule[j] * 3.0 - A * hc * (s - p.Tinf_schedule[j])
        s = s + dt / (Cn * (1 + cl * s)) * q
    assert np.max(np.abs(T - s)) <= 1e-12 * abs(s)
    T1 = m.run(p.initial_T(), dt, 70)
    T2 = m.run(T1, dt, n + 40 - 70, step0=70)
    assert np.max(np.abs(T2 - T)) <= 1e-13 * abs(s)


@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_surface_area_shares_sum_to_face_areas(kind):
    """Nodal-quadrature lumping keeps the total area: sum A^c = 1 (top), sum A^r = 4 (sides)."""
    p = fi.nonlinear_cube(4, kind)
    m = O.OracleModel(p)
    assert m.Ac.sum() == pytest.approx(1.0, rel=1e-13)
    assert m.Ar.sum() == pytest.approx(4.0, rel=1e-13)
    assert m.C0.sum() == pytest.approx(2700.0 * 500.0, rel=1e-13)
    assert m.Qext.sum() == pytest.approx(1e5 / 8, rel=1e-13)


def test_critical_step_surface_term():
    """With negligible conduction, dt_crit reduces to the scalar forward-Euler limit of the
    linearised surface ODE, 2 C min(f_c) / (A (h + 4 sigma eps max|T - T_z|^3))."""
    p = fi.single_brick(0.5, 0.5, 0.5, rho=100.0, c0=10.0, c_lin=0.001, conv=(30.0, 20.0),
                        rad=(0.5, 20.0))
    p.mats[0].k0 = 1e-14 * np.eye(3)
    p.T_lo, p.T_hi = 20.0, 500.0
    m = O.OracleModel(p)
    A = 3 * 0.25 / 4
    Cn = 100.0 * 10.0 * 0.125 / 8
    rate = A * (30.0 + 4 * 5.67e-8 * 0.5 * (500 + 273.15) ** 3) / (Cn * 1.02)
    assert m.dt_crit()[0] == pytest.approx(2.0 / rate, rel=1e-9)


def test_stefan_law_spot_value():
    """Eq. 7 lumped on a node with unit radiating area: sigma eps ((T-Tz)^4 - (Ta-Tz)^4)."""
    p = fi.single_brick(1, 1, 1, T0=0.0, rad=(0.66, -50.0))
    m = O.OracleModel(p)
    # isolate the radiation term at node 0 (Qext = 0, no convection)
    q = m.nodal_Q(np.full(8, 37.0))[0]
    expect = -m.Ar[0] * 5.67e-8 * 0.66 * (310.15 ** 4 - 223.15 ** 4)
    assert q == pytest.approx(expect, rel=1e-13)


# -------------------------------------------------------------------------- energy ---------

@pytest.mark.parametrize("kind,moving", [("hex", False), ("tet", False), ("hex", True)])
def test_energy_balance(kind, moving):
    """Internal loads sum to zero, so the stored heat changes only by the boundary and source
    flows: S^n = B^n every step (FP64), also when the prescribed temperatures move."""
    p = fi.nonlinear_cube(5, kind)
    p.dir_nodes = np.arange(0, 6, dtype=np.int32)
    p.dir_T = np.full(6, 60.0)
    if moving:
        p.Tdir_schedule = 40.0 * np.sin(0.2 * np.arange(60))
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    T, E = m.run(p.initial_T(), dt, 60, energy=True)
    scale = np.abs(E).max()
    assert np.max(np.abs(E[:, 0] - E[:, 1])) <= 1e-12 * scale
    # heat input of the source is positive early on
    assert E[0, 1] > 0


# ------------------------------------------------------------------------- adjoint ---------

def _adjoint_setup():
    p = fi.nonlinear_cube(3, "hex", steps=30)
    rng = np.random.default_rng(9)
    p.elem_kscale = rng.uniform(0.5, 2.0, size=p.n_elems)
    p.elem_source = rng.uniform(0, 2e5, size=p.n_elems)
    sensors = np.array([5, 13, 21, 40, 62], np.int32)
    return p, sensors


@pytest.mark.parametrize("scheduled", [False, True, "table"])
def test_adjoint_matches_central_differences(scheduled):
    """Reverse-time adjoint vs central finite differences of the forward loop (FP64); also
    with a schedule (q(n) scales the sources, T_inf(n) moves, the bottom face is held at a
    temperature that moves every step)."""
    p, sensors = _adjoint_setup()
    if scheduled:
        k = np.arange(30)
        p.q_schedule = 1.0 + 0.8 * np.cos(0.3 * k)
        p.Tinf_schedule = 20.0 + 2.0 * k
        bottom = np.flatnonzero(np.abs(p.xyz[:, 2]) < 1e-9).astype(np.int32)
        p.dir_nodes, p.dir_T = bottom, np.full(len(bottom), 20.0)
        p.Tdir_schedule = 25.0 * np.sin(0.4 * k)
    if scheduled == "table":  # tabulated k(T), c(T): the adjoint carries the segment slopes
        p.q_schedule = p.Tinf_schedule = p.Tdir_schedule = None
        p.table_T = np.array([0.0, 150.0, 300.0, 450.0, 1000.0])
        p.table_fk = np.array([0.8, 1.0, 1.6, 1.3, 2.0])
        p.table_fc = np.array([1.1, 1.0, 0.8, 1.4, 1.2])
    m0 = O.OracleModel(p)
    dt = 0.9 * m0.dt_crit()[0]
    nsteps, se = 30, 5
    rng = np.random.default_rng(11)
    wts = rng.standard_normal((nsteps // se, len(sensors)))

    def loss(theta, src):
        m = O.OracleModel(p, theta=theta, source=src)
        _, tr = m.run(p.initial_T(), dt, nsteps, sensors=sensors, sample_every=se)
        return float(np.sum(wts * tr))

    gt, gs = m0.adjoint(dt, nsteps, p.initial_T(), sensors, se, wts)
    th, src = p.elem_kscale.copy(), p.elem_source.copy()
    for e in (0, 4, 13, 26):
        d = 1e-4 * th[e]
        tp, tm = th.copy(), th.copy()
        tp[e] += d
        tm[e] -= d
        fd = (loss(tp, src) - loss(tm, src)) / (2 * d)
        assert gt[e] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(gt).max())
        d = 1e-4 * max(src[e], 1.0)
        sp, sm = src.copy(), src.copy()
        sp[e] += d
        sm[e] -= d
        fd = (loss(th, sp) - loss(th, sm)) / (2 * d)
        assert gs[e] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(gs).max())


def test_adjoint_dot_product_linear():
    """For a linear problem (constant k, c, no radiation) the map source -> trace is affine:
    <J v, w> = <v, J^T w> for the Jacobian J of the trace wrt the element sources."""
    p = fi.nonlinear_cube(3, "hex")
    p.mats[0].k_lin = 0.0
    p.mats[0].c_lin = 0.0
    p.rad_faces = None
    sensors = np.array([5, 13, 21, 40, 62], np.int32)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    rng = np.random.default_rng(3)
    w = rng.standard_normal((4, len(sensors)))
    v = rng.standard_normal(p.n_elems)
    src = p.elem_source
    _, tr0 = O.OracleModel(p, source=src).run(p.initial_T(), dt, 20, sensors=sensors, sample_every=5)
    _, tr1 = O.OracleModel(p, source=src + v).run(p.initial_T(), dt, 20, sensors=sensors, sample_every=5)
    Jv = tr1 - tr0
    _, gs = m.adjoint(dt, 20, p.initial_T(), sensors, 5, w)
    assert np.sum(Jv * w) == pytest.approx(np.dot(v, gs), rel=1e-10)


# ------------------------------------------------------------ multi-threaded time stepping --

@pytest.mark.parametrize("case", ["hex_jitter", "tet", "moving_boundary_table", "sensors_schedule"])
def test_threaded_run_is_bitwise_the_serial_run(case):
    """The time stepping over several host threads (element pass, then a node gather in element
    order) gives bitwise the serial element loop's result: states, per-step energy terms and
    sensor traces, with Dirichlet nodes, schedules and property tables."""
    sensors, every = None, 0
    if case == "hex_jitter":
        p = fi.nonlinear_cube(9, "hex", jitter=0.2)
    elif case == "tet":
        p = fi.nonlinear_cube(6, "tet")
    elif case == "moving_boundary_table":
        p = fi.nonlinear_cube(7, "hex", jitter=0.1)
        bot = np.nonzero(p.xyz[:, 2] < 1e-12)[0].astype(np.int32)
        p.dir_nodes, p.dir_T = bot, 100.0 + 50.0 * p.xyz[bot, 0]
        p.Tdir_schedule = 80.0 * np.sin(0.04 * np.arange(120))
        p.table_T = np.array([0.0, 100.0, 250.0, 450.0])
        p.table_fk = np.array([1.0, 1.6, 1.2, 2.5])
        p.table_fc = np.array([1.0, 0.8, 1.4, 1.1])
    else:
        p = fi.large_cube(8)
        p.q_schedule = 1.0 + 0.5 * np.sin(0.1 * np.arange(90))
        p.Tinf_schedule = 20.0 + np.arange(90) * 0.3
        sensors, every = np.array([5, 77, 300, 601], np.int32), 7
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit(T_hi=900.0)[0]
    for threads in (2, 3, 0):
        a = m.run(p.initial_T(), dt, 150, energy=True, sensors=sensors, sample_every=every, step0=4)
        b = m.run(p.initial_T(), dt, 150, energy=True, sensors=sensors, sample_every=every, step0=4,
                  threads=threads)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_threaded_power_iteration_is_bitwise_the_serial_one():
    """The critical-step power iteration with the internal loads over several threads gives the
    serial result bitwise (dt_crit, lambda and the iteration count)."""
    for p in (fi.nonlinear_cube(7, "hex", jitter=0.2), fi.nonlinear_cube(5, "tet"), fi.plain_cube(6)):
        m = O.OracleModel(p)
        a = m.dt_crit(tol=1e-9, max_iter=3000)
        for threads in (3, 0):
            assert m.dt_crit(tol=1e-9, max_iter=3000, threads=threads) == a


# ------------------------------------------- method variants: quadrature-point k(T), faces --

def test_quadrature_point_conductivity_on_bricks_is_the_exact_integral():
    """Eq. 20 with D(T) inside the integral: on a rectangular brick with a linear law the 2x2x2
    Gauss-point loads equal the exact integral of grad N_i . k0 f_k(T(x)) grad T (independent
    3x3x3 integration), and differ from the element-mean reading of Section 4.2.2."""
    rng = np.random.default_rng(31)
    for _ in range(3):
        dims = rng.uniform(0.3, 1.5, 3)
        x = brute.VTK_CORNERS * dims + rng.uniform(-1, 1, 3)
        k = _rand_spd(rng)
        T = rng.uniform(10, 300, 8)
        a = 0.004
        Kq, Nq = O.hex_matrices_qp(x, k)
        F = sum((1 + a * (Nq[q] @ T)) * (Kq[q] @ T) for q in range(8))
        Fe = brute.hex_load_exact_qp(x, k, T, lambda t: 1 + a * t)
        assert np.max(np.abs(F - Fe)) <= 1e-13 * np.max(np.abs(Fe))
        K, _, _ = O.hex_matrices(x, k)
        assert np.max(np.abs(np.mean(1 + a * T) * (K @ T) - Fe)) > 1e-3 * np.max(np.abs(Fe))
        assert np.max(np.abs(Kq.sum(axis=0) - K)) <= 1e-14 * np.max(np.abs(K))


def test_quadrature_point_conductivity_assembly(patch_nodes):
    """The oracle's internal loads with kT_eval = 1 on the distorted patch and a jittered cube
    against a dense assembly of independently integrated element loads (the same 2x2x2 rule,
    numpy shape functions), with a property table; a constant field carries no load; for linear
    tetrahedra the single centroid point gives the element mean of a linear law."""
    k = _rand_spd(np.random.default_rng(5))
    tT, tk = np.array([20.0, 90.0, 150.0, 260.0]), np.array([1.0, 2.2, 0.7, 1.5])
    fk = lambda t: np.interp(t, tT, tk)
    for p in (fi.patch_problem(patch_nodes, "hex", k0=k), fi.nonlinear_cube(3, "hex", jitter=0.25)):
        p.kT_eval = 1
        p.table_T, p.table_fk, p.table_fc = tT, tk, np.ones(4)
        theta = np.random.default_rng(8).uniform(0.5, 2.0, p.n_elems)
        p.elem_kscale = theta
        m = O.OracleModel(p)
        T = np.random.default_rng(9).uniform(0, 300, p.n_nodes)
        ref = np.zeros(p.n_nodes)
        for e, c in enumerate(p.conn):
            k0 = np.asarray(p.mats[0].k0, float)
            ref[c] += theta[e] * brute.hex_load_exact_qp(p.xyz[c], k0, T[c], fk, order=2)
        got = m.internal_loads(T)
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
        assert np.max(np.abs(m.internal_loads(np.full(p.n_nodes, 42.0)))) <= 1e-12 * 42.0 * np.max(np.abs(m.K))
    q = fi.nonlinear_cube(4, "tet", jitter=0.2)
    a = O.OracleModel(q).run(q.initial_T(), 50.0, 60)
    q.kT_eval = 1
    b = O.OracleModel(q).run(q.initial_T(), 50.0, 60)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


def test_quadrature_point_conductivity_bar_reduces_to_1d():
    """A bar of bricks with a field constant over each cross-section: with the conductivity at
    the 2x2x2 points, the element factor of the 1-D recurrence is the mean of f_k at the two
    Gauss abscissae along the bar (T_L + (T_R - T_L)(1 -+ 1/sqrt 3)/2), here a property table."""
    nx, T0, Ts = 12, 20.0, 400.0
    tT, tk, tc = np.array([0.0, 100.0, 250.0, 450.0]), np.array([1.0, 1.6, 1.2, 2.5]), np.array([1.0, 0.8, 1.4, 1.1])
    p = fi.slab(nx, 1, 1, Lx=1.0, k=(3.0, 3.0, 3.0), rho=2.0, c0=5.0, T0=T0, T_s=Ts)
    p.table_T, p.table_fk, p.table_fc = tT, tk, tc
    p.kT_eval = 1
    m = O.OracleModel(p)
    h = 1.0 / nx
    dt = 0.2 * 2.0 * 5.0 * h * h / (3.0 * 2.5)
    got = m.run(p.initial_T(), dt, 300)
    g = 1.0 / np.sqrt(3.0)
    T = np.full(nx + 1, T0)
    T[0] = Ts
    for _ in range(300):
        TL, TR = T[:-1], T[1:]
        f = 0.5 * (np.interp(TL + (TR - TL) * (1 - g) / 2, tT, tk) + np.interp(TL + (TR - TL) * (1 + g) / 2, tT, tk))
        c = 5.0 * np.interp(T, tT, tc)
        Tn = T.copy()
        Tn[1:-1] = T[1:-1] + dt * 3.0 / (2.0 * c[1:-1] * h * h) * (f[1:] * (T[2:] - T[1:-1]) + f[:-1] * (T[:-2] - T[1:-1]))
        Tn[-1] = T[-1] + 2.0 * dt * 3.0 / (2.0 * c[-1] * h * h) * f[-1] * (T[-2] - T[-1])
        T = Tn
    x = np.round(p.xyz[:, 0] / h).astype(int)
    assert np.max(np.abs(got - T[x])) <= 1e-12 * Ts


def test_consistent_face_matrices_closed_forms():
    """Face mass matrices of the consistent surface integration: a rectangle a x b,
    (ab/36)[4 2 1 2; 2 4 2 1; 1 2 4 2; 2 1 2 4], a triangle of area A, (A/12)[2 1 1; 1 2 1;
    1 1 2]; the radiation weights sum to the area; on a rectangle with a bilinear field the
    quadrature of N_i ((T - T_z)^4 - (T_a - T_z)^4) equals a 10x10 Gauss-Legendre integral."""
    a, b = 0.7, 1.9
    rect = np.array([[0, 0, 0], [a, 0, 0], [a, b, 0], [0, b, 0]], float)
    Mf, Wf = O.face_consistent(np.array([[0, 1, 2, 3]]), rect)
    ref = a * b / 36.0 * np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]])
    assert np.max(np.abs(Mf[0] - ref)) <= 1e-15 * 4
    assert Wf[0].sum() == pytest.approx(a * b, rel=1e-14)
    tri = np.array([[0.1, 0.2, 0.3], [1.4, 0.1, 0.5], [0.4, 1.3, 0.9]])
    Mt, Wt = O.face_consistent(np.array([[0, 1, 2]]), tri)
    A = 0.5 * np.linalg.norm(np.cross(tri[1] - tri[0], tri[2] - tri[0]))
    assert np.max(np.abs(Mt[0] - A / 12.0 * (np.ones((3, 3)) + np.eye(3)))) <= 1e-15 * A
    assert Wt[0].sum() == pytest.approx(A, rel=1e-14)
    # radiation quadrature vs brute force on the rectangle
    Tn = np.array([300.0, 520.0, 610.0, 410.0])
    Tz, Ta = -273.15, 20.0
    Nf, _ = O.face_rule(4)
    Tp = Nf @ Tn
    got = (Wf[0][:, None] * Nf * ((Tp - Tz) ** 4 - (Ta - Tz) ** 4)[:, None]).sum(axis=0)
    g, gw = np.polynomial.legendre.leggauss(10)
    S = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], float)
    want = np.zeros(4)
    for s, ws in zip(g, gw):
        for t, wt in zip(g, gw):
            N = (1 + s * S[:, 0]) * (1 + t * S[:, 1]) / 4
            T = N @ Tn
            want += ws * wt * (a * b / 4) * N * ((T - Tz) ** 4 - (Ta - Tz) ** 4)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("consistent", [False, True])
def test_face_integration_bar_with_lateral_convection(consistent):
    """A bar with convection on its four lateral faces and T held at x = 0: lumped (nodal
    quadrature) and consistent face integration against their exact 1-D recurrences."""
    nx, w, T0, Ts, hc, Tinf = 10, 0.1, 20.0, 300.0, 40.0, 5.0
    p = fi.slab(nx, 1, 1, Lx=1.0, k=(2.0, 2.0, 2.0), rho=3.0, c0=4.0, T0=T0, T_s=Ts)
    h = 1.0 / nx
    # cross-section w x w instead of h x h
    p.xyz = p.xyz * np.array([1.0, w / h, w / h])
    bf = fi.boundary_faces(p.conn)
    p.conv_faces = np.concatenate([fi.faces_on_side(p.xyz, bf, sd) for sd in ("y0", "y1", "z0", "z1")])
    p.h, p.T_inf = hc, Tinf
    p.face_quadrature = 1 if consistent else 0
    m = O.OracleModel(p)
    dt = 0.5 * m.dt_crit(T_lo=0.0, T_hi=Ts)[0]
    got = m.run(p.initial_T(), dt, 400)
    ref = brute.bar_lateral_convection(nx, h, w, dt, 400, T0, Ts, 2.0, 3.0, 4.0, hc, Tinf, consistent)
    x = np.round(p.xyz[:, 0] / h).astype(int)
    assert np.max(np.abs(got - ref[x])) <= 1e-12 * Ts
    other = brute.bar_lateral_convection(nx, h, w, dt, 400, T0, Ts, 2.0, 3.0, 4.0, hc, Tinf, not consistent)
    assert np.max(np.abs(got - other[x])) > 1e-6 * Ts


def test_consistent_faces_keep_the_energy_balance():
    """With consistent face integration (convection and radiation) the per-step energy terms
    still balance: stored heat change = dt (sum of free-node loads + Dirichlet reactions)."""
    p = fi.nonlinear_cube(5, "hex", jitter=0.2)
    p.face_quadrature = 1
    p.kT_eval = 1
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    _, E = m.run(p.initial_T(), dt, 200, energy=True)
    assert np.max(np.abs(E[:, 0] - E[:, 1])) <= 1e-12 * np.max(np.abs(E))
