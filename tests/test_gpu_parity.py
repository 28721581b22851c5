"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (rel-L-infinity, max|T - T_oracle| / max|T_oracle|): 1e-10 for the FP64 form and
2e-4 for FP32 + Kahan after the stated step counts.  Sizes span several tiles with ragged
tails (element counts not multiples of the chunk size).
"""
import numpy as np
import pytest

import fedfem_inputs as fi
from oracle import oracle as O
from tests import brute

pytestmark = pytest.mark.gpu

TOL = {64: 1e-10, 32: 2e-4}


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1909_03355_gb300 import capi
    capi.load()


def FedFem(*a, **k):
    from paper_1909_03355_gb300.fedfem import FedFem as F
    return F(*a, **k)


def run_gpu(p, dt, nsteps, precision, **plan):
    f = FedFem(p, precision=precision, **plan)
    f.precompute()
    f.set_dt(dt, force=True)
    f.set_T(p.initial_T())
    f.step(nsteps)
    T = f.get_T()
    f.close()
    return T


# ------------------------------------------------------------------------- plain cube (C1) --

def test_plain_cube_fp64_vs_oracle_and_closed_form():
    p = fi.plain_cube(10)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    f = FedFem(p, precision=64)
    dtc = f.precompute()
    assert dtc == pytest.approx(m.dt_crit()[0], rel=1e-8)
    f.set_dt(dt)
    f.set_T(p.initial_T())
    Tref, done = p.initial_T(), 0
    for n in (1, 10, 50, 100, 1000):
        f.step(n - done)
        Tref = m.run(Tref, dt, n - done)
        done = n
        T = f.get_T()
        assert rel(T, Tref) <= 1e-10, n
        cf, _ = brute.c1_closed_form(10, dt, n)
        assert rel(T, cf) <= 1e-10, n
    f.close()


def test_plain_cube_fp32():
    p = fi.plain_cube(10)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    for n in (1, 10, 50):
        assert rel(run_gpu(p, dt, n, 32), m.run(p.initial_T(), dt, n)) <= 2e-4


# ------------------------------------------------------------------ nonlinear cubes (C2) ---

@pytest.mark.parametrize("kind", ["hex", "tet"])
@pytest.mark.parametrize("precision", [64, 32])
def test_nonlinear_cube(kind, precision):
    """k(T) anisotropic, c(T), convection top, radiation sides, central source."""
    p = fi.nonlinear_cube(11, kind, jitter=0.2)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    ref = m.run(p.initial_T(), dt, 400)
    assert rel(run_gpu(p, dt, 400, precision), ref) <= TOL[precision]


@pytest.mark.parametrize("precision", [64, 32])
def test_nonlinear_hex_full_step_count(precision):
    """Nonlinear hex cube physics at 16^3 for the full 5000 steps."""
    p = fi.nonlinear_cube(16, "hex")
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    ref = m.run(p.initial_T(), dt, 5000)
    assert rel(run_gpu(p, dt, 5000, precision), ref) <= TOL[precision]


@pytest.mark.parametrize("precision", [64, 32])
def test_large_cube_physics_full_step_count(precision):
    """Orthotropic k(T), conv + rad on all faces at 12^3 for the full 20000 steps (Kahan)."""
    p = fi.large_cube(12, jitter=0.2)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    ref = m.run(p.initial_T(), dt, 20000)
    assert rel(run_gpu(p, dt, 20000, precision), ref) <= TOL[precision]


def test_fp32_without_kahan_is_reported():
    """Plain FP32 accumulation (no Kahan) for comparison; must still be sane."""
    p = fi.large_cube(10)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    ref = m.run(p.initial_T(), dt, 5000)
    e_k = rel(run_gpu(p, dt, 5000, 32), ref)
    e_p = rel(run_gpu(p, dt, 5000, 32, kahan=False), ref)
    print(f"fp32 rel error after 5000 steps: kahan {e_k:.3e}, plain {e_p:.3e}")
    assert e_k <= 2e-4 and e_p < 1e-2


# --------------------------------------------------------------------- pre-computation -----

@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_internal_loads_and_dt_crit(kind):
    p = fi.nonlinear_cube(6, kind, jitter=0.25)
    p.elem_kscale = np.random.default_rng(1).uniform(0.5, 2, p.n_elems)
    m = O.OracleModel(p)
    f = FedFem(p, precision=64)
    dtc = f.precompute()
    T = fi.random_state(p, 3)
    assert rel(f.internal_loads(T), m.internal_loads(T)) <= 1e-12
    dto = m.dt_crit()[0]
    assert dtc == pytest.approx(dto, rel=1e-6)
    f.close()


@pytest.mark.parametrize("kind", ["hex", "tet"])
@pytest.mark.parametrize("n", [2, 3, 6])
def test_dt_crit_vs_dense_eigensolver(kind, n):
    """The GPU critical step (FP64 Lanczos) against scipy's dense generalized symmetric
    eigensolver: without surface terms dt_crit = 2 / (lambda_max(K0, C0 on the free nodes)
    max f_k / min f_c) (Section 3.4).  n = 2 has fewer free nodes than one convergence check
    takes, so the Krylov space is exhausted."""
    import scipy.linalg
    p = fi.nonlinear_cube(n, kind, jitter=0.2 if n > 2 else 0.0)
    p.conv_faces = None
    p.rad_faces = None
    p.dir_nodes = np.array([0, 1], np.int32)
    p.dir_T = np.array([20.0, 20.0])
    m = O.OracleModel(p)
    free = p.free_mask()
    Kd = brute.dense_assemble(p.conn, m.K, p.n_nodes)
    lam = scipy.linalg.eigh(Kd[np.ix_(free, free)], np.diag(m.C0[free]), eigvals_only=True).max()
    mat = p.mats[0]
    fk = max(1 + mat.k_lin * p.T_lo, 1 + mat.k_lin * p.T_hi)
    fc = min(1 + mat.c_lin * p.T_lo, 1 + mat.c_lin * p.T_hi)
    f = FedFem(p, precision=64)
    dtc = f.precompute()
    f.close()
    assert dtc == pytest.approx(2.0 / (lam * fk / fc), rel=1e-9)


@pytest.mark.parametrize("precision", [64, 32])
def test_hex_centre_rule_vs_oracle(precision):
    """The one-point conduction matrices of Eq. 17 (option quadrature = 1) on the jittered
    nonlinear hex cube: GPU against the oracle after 300 steps, and the critical step."""
    p = fi.nonlinear_cube(10, "hex", jitter=0.2)
    p8 = fi.nonlinear_cube(10, "hex", jitter=0.2)
    p.quadrature = 1
    m = O.OracleModel(p)
    dto = m.dt_crit()[0]
    dt = 0.9 * min(dto, O.OracleModel(p8).dt_crit()[0])
    T_ref = m.run(p.initial_T(), dt, 300)
    # the 2x2x2 operator gives a clearly different field on this distorted mesh
    assert rel(O.OracleModel(p8).run(p8.initial_T(), dt, 300), T_ref) > 1e-4
    f = FedFem(p, precision=precision)
    assert f.precompute() == pytest.approx(dto, rel=1e-6)
    f.close()
    T = run_gpu(p, dt, 300, precision)
    assert rel(T, T_ref) <= TOL[precision]


@pytest.mark.parametrize("precision", [64, 32])
def test_paper_cube_temperature_dependent_laws(precision):
    """The paper's cube with the two-point laws of Section 4.2.2 (k and c given at 37 deg C,
    T_ref = 37) at its own dt = 0.005 s: GPU against the oracle after 400 steps."""
    p = fi.paper_cube("tet", 8, td=True)
    m = O.OracleModel(p)
    f = FedFem(p, precision=precision)
    dtc = f.precompute()
    f.close()
    assert dtc == pytest.approx(m.dt_crit()[0], rel=1e-6)
    assert 0.005 < dtc
    T_ref = m.run(p.initial_T(), 0.005, 400)
    assert T_ref.max() > 37.2  # the loads have heated it
    assert rel(run_gpu(p, 0.005, 400, precision), T_ref) <= TOL[precision]


@pytest.mark.parametrize("precision", [64, 32])
def test_paper_cube_full_run(precision):
    """The paper-shaped 0.1 m cube (41,154 tets) at the paper's dt = 0.005 s for all 2000 steps
    of Section 4.3: GPU against the oracle."""
    p = fi.paper_cube("tet", 19)
    m = O.OracleModel(p)
    T_ref = m.run(p.initial_T(), 0.005, 2000)
    assert rel(run_gpu(p, 0.005, 2000, precision), T_ref) <= TOL[precision]


def _scheduled_cube():
    p = fi.nonlinear_cube(9, "hex", jitter=0.2)
    n = 250
    k = np.arange(n)
    p.q_schedule = 1.0 + 0.7 * np.sin(0.05 * k) + k / n
    p.Tinf_schedule = 20.0 + 200.0 * (k / n) ** 2
    return p


def _dirichlet_cube(kind):
    """Nonlinear cube with its bottom face held at 100 + 50 x plus an offset that moves every
    step (a ramp with a sine on it, 250 entries, the last one held)."""
    p = fi.nonlinear_cube(9, kind, jitter=0.2 if kind == "hex" else 0.0)
    bottom = np.flatnonzero(np.abs(p.xyz[:, 2]) < 1e-9).astype(np.int32)
    p.dir_nodes = bottom
    p.dir_T = 100.0 + 50.0 * p.xyz[bottom, 0]
    k = np.arange(250)
    p.Tdir_schedule = 80.0 * np.sin(0.04 * k) + 0.4 * k
    p.T_hi = max(p.T_hi, 400.0)
    return p


@pytest.mark.parametrize("kind", ["hex", "tet"])
@pytest.mark.parametrize("precision", [64, 32])
def test_time_dependent_dirichlet(kind, precision):
    """Prescribed temperatures that move every step (dir_T + d[n]): GPU against the oracle over
    300 steps in launches of 37 steps with the run split across two calls; the energy terms of
    the last step; a new offset schedule set at step 300 moves the Dirichlet values to those of
    that step and the run continues with it."""
    p = _dirichlet_cube(kind)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    T_ref, E = m.run(p.initial_T(), dt, 300, energy=True)
    f = FedFem(p, precision=precision, steps_per_launch=37)
    f.precompute()
    f.set_dt(dt, force=True)
    f.set_T(p.initial_T())
    f.step(123)
    f.step(177)
    T = f.get_T()
    scale = np.max(np.abs(T_ref))
    assert rel(T, T_ref) <= TOL[precision]
    assert np.max(np.abs(T[p.dir_nodes] - (p.dir_T + p.Tdir_schedule[-1]))) <= TOL[precision] * scale
    if precision == 64:
        S, B = f.energy()
        assert S == pytest.approx(E[-1, 0], rel=1e-8) and B == pytest.approx(E[-1, 1], rel=1e-8)
    d2 = 30.0 * np.cos(0.03 * np.arange(400))
    f.set_schedule(T_dir=d2)
    m.set_schedule(T_dir=d2)
    f.step(100)
    T2 = m.run(T_ref, dt, 100, step0=300)
    assert rel(f.get_T(), T2) <= TOL[precision]
    f.close()


def _table_cube(kind, npts=5):
    """Nonlinear cube with tabulated k(T), c(T): five (or eight) points across the 20-820 degree
    range of the run, the hottest nodes past the last point (held end values)."""
    p = fi.nonlinear_cube(9, kind, jitter=0.2 if kind == "hex" else 0.0)
    if npts == 5:
        p.table_T = np.array([0.0, 100.0, 250.0, 450.0, 650.0])
        p.table_fk = np.array([1.0, 1.6, 1.2, 2.5, 2.0])
        p.table_fc = np.array([1.0, 0.8, 1.4, 1.1, 1.6])
    else:
        p.table_T = np.array([0.0, 50.0, 120.0, 200.0, 300.0, 400.0, 480.0, 560.0])
        p.table_fk = np.array([1.0, 1.4, 1.1, 1.9, 1.5, 2.6, 2.1, 2.3])
        p.table_fc = np.array([1.0, 0.7, 1.2, 1.5, 1.0, 1.3, 1.8, 1.4])
    return p


@pytest.mark.parametrize("kind,npts", [("hex", 5), ("tet", 5), ("hex", 8), ("tet", 8)])
@pytest.mark.parametrize("precision", [64, 32])
def test_property_table(kind, npts, precision):
    """Tabulated factors (linear between points, end values held, nodal k averaged per element):
    dt_crit and internal loads at a random state against the oracle, then 300 steps in launches
    of 37 with the run split across two calls, and the energy terms of the last step.  Five
    points run in the step kernel that evaluates three hinges, eight points in the one that
    evaluates all six."""
    p = _table_cube(kind, npts)
    m = O.OracleModel(p)
    f = FedFem(p, precision=precision, steps_per_launch=37)
    dtc = f.precompute()
    assert dtc == pytest.approx(m.dt_crit()[0], rel=1e-6)
    Tr = fi.random_state(p, 3, lo=-50.0, hi=900.0)
    assert rel(f.internal_loads(Tr), m.internal_loads(Tr)) <= 1e-12
    dt = 0.9 * m.dt_crit()[0]
    T_ref, E = m.run(p.initial_T(), dt, 300, energy=True)
    assert np.sum(T_ref > p.table_T[-1]) > 0 and np.sum(T_ref < p.table_T[1]) > 0
    f.set_dt(dt, force=True)
    f.set_T(p.initial_T())
    f.step(123)
    f.step(177)
    assert rel(f.get_T(), T_ref) <= TOL[precision]
    if precision == 64:
        S, B = f.energy()
        assert S == pytest.approx(E[-1, 0], rel=1e-8) and B == pytest.approx(E[-1, 1], rel=1e-8)
    f.close()


def test_property_table_errors():
    from paper_1909_03355_gb300.fedfem import FedFemError
    p = _table_cube("hex")
    f = FedFem(fi.nonlinear_cube(3, "hex"), precision=64)
    for T, fk, fc in (([1.0], [1.0], [1.0]), ([0.0, 0.0], [1.0, 1.0], [1.0, 1.0]),
                      ([0.0, 1.0], [1.0, -1.0], [1.0, 1.0]), ([0.0, 1.0], [1.0, 1.0], [0.0, 1.0]),
                      (np.arange(9.0), np.ones(9), np.ones(9))):
        with pytest.raises(FedFemError):
            f.set_table(T, fk, fc)
    f.set_table(p.table_T, p.table_fk, p.table_fc)
    f.set_table(None)  # removing the table restores the linear laws
    m = O.OracleModel(fi.nonlinear_cube(3, "hex"))
    assert f.precompute() == pytest.approx(m.dt_crit()[0], rel=1e-6)
    with pytest.raises(FedFemError):
        f.set_table(p.table_T, p.table_fk, p.table_fc)
    f.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_time_dependent_loads(precision):
    """Load multiplier and convection ambient temperature per step (last entries held beyond
    the schedule): GPU against the oracle over 300 steps, with launches of 37 steps and the run
    split across two calls, so the schedule is indexed by the global step everywhere."""
    p = _scheduled_cube()
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    T_ref = m.run(p.initial_T(), dt, 300)
    assert rel(T_ref, O.OracleModel(fi.nonlinear_cube(9, "hex", jitter=0.2)).run(p.initial_T(), dt, 300)) > 1e-3
    f = FedFem(p, precision=precision, steps_per_launch=37)
    f.precompute()
    f.set_dt(dt, force=True)
    f.set_T(p.initial_T())
    f.step(123)
    f.step(177)
    assert rel(f.get_T(), T_ref) <= TOL[precision]
    # energy terms of the last step use the loads of that step
    _, E = m.run(p.initial_T(), dt, 300, energy=True)
    S, B = f.energy()
    if precision == 64:
        assert S == pytest.approx(E[-1, 0], rel=1e-8) and B == pytest.approx(E[-1, 1], rel=1e-8)
    f.set_schedule(None, None)  # removing the schedule restores constant loads
    f.set_T(p.initial_T())
    f.step(50)
    T_c = O.OracleModel(fi.nonlinear_cube(9, "hex", jitter=0.2)).run(p.initial_T(), dt, 50)
    assert rel(f.get_T(), T_c) <= TOL[precision]
    f.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_adaptive_time_step(precision):
    """dt re-evaluated before every launch from the current range: a heating cube precomputed for
    [20, 40] deg C runs far beyond that range; GPU against the oracle's adaptive run (the two
    lambda_cond estimates agree to ~1e-10, hence the FP64 bound of 1e-8)."""
    p = fi.nonlinear_cube(8, "hex")
    p.T_lo, p.T_hi = 20.0, 40.0
    m = O.OracleModel(p)
    T_ref, t_ref = m.run_adaptive(p.initial_T(), 600, 50, 0.9, 0.0)
    assert T_ref.max() > 500.0
    f = FedFem(p, precision=precision, steps_per_launch=50)
    f.precompute()
    f.set_T(p.initial_T())
    t = f.step_adaptive(600, 0.9, 0.0)
    tol = 1e-8 if precision == 64 else 2e-4
    assert t == pytest.approx(t_ref, rel=tol)
    assert rel(f.get_T(), T_ref) <= tol
    f.close()


def _single_element(kind):
    if kind == "hex":
        return fi.single_brick(0.3, 0.5, 0.7, rho=800.0, c0=900.0, c_lin=0.002, T0=400.0, conv=(40.0, 15.0),
                               rad=(0.7, -50.0), steps=200)
    xyz = np.array([[0, 0, 0], [0.4, 0, 0], [0, 0.5, 0], [0.1, 0.1, 0.6]], float)
    conn = np.array([[0, 1, 2, 3]], np.int32)
    bf = fi.boundary_faces(conn)
    return fi.Problem(name="tet1", xyz=xyz, conn=conn,
                      mats=[fi.Material(800.0, np.diag([1.0, 2.0, 3.0]), 0.001, 900.0, 0.002)],
                      conv_faces=bf, h=40.0, T_inf=15.0, rad_faces=bf, eps=0.7, T_amb=-50.0,
                      nodal_Q=np.array([5.0, 0.0, 0.0, 1.0]), T0=np.array([400.0, 350.0, 300.0, 250.0]),
                      steps=200, T_lo=-50.0, T_hi=400.0)


@pytest.mark.parametrize("kind", ["hex", "tet"])
@pytest.mark.parametrize("precision", [64, 32])
def test_single_element(kind, precision):
    """Degenerate mesh: one element (one tile, one mostly padded chunk, no shared nodes) with
    convection and radiation on every face: GPU against the oracle; zero steps leave the state
    and the step counter unchanged."""
    p = _single_element(kind)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    f = FedFem(p, precision=precision)
    f.precompute()
    f.set_dt(dt, force=True)
    f.set_T(p.initial_T())
    f.step(0)
    assert f.step_count == 0 and np.array_equal(f.get_T(), p.initial_T())
    f.step(p.steps)
    assert rel(f.get_T(), m.run(p.initial_T(), dt, p.steps)) <= TOL[precision]
    f.close()


def test_inverted_element_reported():
    p = fi.plain_cube(3)
    p.conn = p.conn.copy()
    p.conn[5] = p.conn[5][[4, 5, 6, 7, 0, 1, 2, 3]]
    from paper_1909_03355_gb300.capi import FedFemError
    f = FedFem(p, precision=64)
    with pytest.raises(FedFemError) as ei:
        f.precompute()
    assert ei.value.name == "ERR_MESH" and "element 5" in str(ei.value)
    f.close()


def test_call_order_and_stability_checks():
    from paper_1909_03355_gb300.capi import FedFemError
    p = fi.plain_cube(4)
    f = FedFem(p, precision=64)
    with pytest.raises(FedFemError) as ei:
        f.set_dt(1e-3)
    assert ei.value.name == "ERR_STATE"
    dtc = f.precompute()
    with pytest.raises(FedFemError) as ei:
        f.set_dt(1.5 * dtc)
    assert ei.value.name == "ERR_UNSTABLE"
    f.set_dt(0.5 * dtc)
    with pytest.raises(FedFemError) as ei:
        f.step(1)
    assert ei.value.name == "ERR_STATE"
    f.close()


# -------------------------------------------------------------------------- patch tests ----

@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_patch_test_steady_state_gpu(kind, patch_nodes):
    """Section 4.1: interior nodes follow T = 200x + 100y + 200z at steady state."""
    p = fi.patch_problem(patch_nodes, kind, k0=np.array([[3.0, 0.5, 0.2], [0.5, 2.0, 0.3], [0.2, 0.3, 1.0]]))
    lin = p.xyz @ np.array([200.0, 100.0, 200.0])
    f = FedFem(p, precision=64)
    dtc = f.precompute()
    f.set_dt(0.9 * dtc)
    f.set_T(p.initial_T())
    f.step(20000)
    assert np.max(np.abs(f.get_T() - lin)) <= 1e-9 * np.max(np.abs(lin))
    f.close()


def test_slab_gpu_matches_1d_recurrence():
    nx, k, rho, c0 = 40, 2.0, 3.0, 1.5
    p = fi.slab(nx, 2, 2, k=(k, 1.0, 1.0), rho=rho, c0=c0, k_lin=0.01, c_lin=0.004, T0=0.0, T_s=100.0,
                conv_end=(4.0, 10.0))
    h = 1.0 / nx
    dt = 0.2 * rho * c0 * h * h / (k * 3.0)
    T = run_gpu(p, dt, 500, 64)
    ref = brute.ftcs_slab(nx, h, dt, 500, 0.0, 100.0, k, rho, c0, 0.01, 0.004, conv=(4.0, 10.0))
    ix = np.rint(p.xyz[:, 0] / h).astype(int)
    assert np.max(np.abs(T - ref[ix])) <= 1e-11 * 100


# ---------------------------------------------------------------- energy, determinism ------

@pytest.mark.parametrize("precision,tol", [(64, 1e-10), (32, 1e-4)])
def test_energy_balance_gpu(precision, tol):
    p = fi.nonlinear_cube(9, "hex")
    p.dir_nodes = np.arange(0, 10, dtype=np.int32)
    p.dir_T = np.full(10, 80.0)
    f = FedFem(p, precision=precision)
    dt = 0.9 * f.precompute()
    f.set_dt(dt)
    f.set_T(p.initial_T())
    f.step(37)
    S, B = f.energy()
    assert abs(S - B) <= tol * abs(B)
    f.close()


def test_determinism_bitwise():
    p = fi.nonlinear_cube(12, "hex", jitter=0.1)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    a = run_gpu(p, dt, 300, 32)
    b = run_gpu(p, dt, 300, 32)
    assert np.array_equal(a, b)


def test_checkpoint_resume_bitwise():
    p = fi.nonlinear_cube(10, "tet")
    f = FedFem(p, precision=32)
    dt = 0.9 * f.precompute()
    f.set_dt(dt)
    f.set_T(p.initial_T())
    f.step(103)
    st = f.get_state()
    f.step(97)
    a = f.get_T()
    f.set_state(st)
    assert f.step_count == 103
    f.step(97)
    assert np.array_equal(a, f.get_T())
    # blobs that do not belong to this context are refused on the host, the state untouched
    from paper_1909_03355_gb300.capi import FedFemError
    for field, value in ((0, -5), (1, p.n_nodes + 1)):
        bad = st.copy()
        bad[8 * field:8 * field + 8] = np.frombuffer(np.int64(value).tobytes(), np.uint8)
        with pytest.raises(FedFemError):
            f.set_state(bad)
    assert f.step_count == 200 and np.array_equal(a, f.get_T())
    f.close()


def test_atomic_scatter_variant_close():
    p = fi.nonlinear_cube(10, "hex")
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    ref = m.run(p.initial_T(), dt, 300)
    from paper_1909_03355_gb300.capi import SCATTER_ATOMIC
    assert rel(run_gpu(p, dt, 300, 32, scatter=SCATTER_ATOMIC), ref) <= 2e-4
    assert rel(run_gpu(p, dt, 300, 64, scatter=SCATTER_ATOMIC), ref) <= 1e-10


@pytest.mark.parametrize("plan", [dict(block=256, chunk=64, stages=4, tiles_per_cta=1, steps_per_launch=1),
                                  dict(block=480, chunk=32, stages=40, tiles_per_cta=4, steps_per_launch=7),
                                  dict(block=256, chunk=64, stages=12, tiles_per_cta=3, steps_per_launch=33),
                                  dict(block=480, chunk=64, stages=2, tiles_per_cta=3, steps_per_launch=200),
                                  dict(block=192, chunk=32, stages=8, steps_per_launch=50)])
def test_launch_plans_agree(plan):
    """Different tilings / chunk sizes / launch splits agree with the oracle (FP64 plans whose
    element stages do not fit in shared memory are rejected at create and skipped here)."""
    from paper_1909_03355_gb300.capi import FedFemError
    p = fi.large_cube(14, jitter=0.15)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    ref = m.run(p.initial_T(), dt, 150)
    assert rel(run_gpu(p, dt, 150, 32, **plan), ref) <= 2e-4
    try:
        T64 = run_gpu(p, dt, 150, 64, **plan)
    except FedFemError as e:
        assert e.name == "ERR_UNSUPPORTED"  # the FP64 stages of this plan exceed shared memory
        return
    assert rel(T64, ref) <= 1e-10


# ------------------------------------------------------------------ failure detection -------

def test_watchdog_reports_divergence_and_context_recovers():
    from paper_1909_03355_gb300.capi import FedFemError
    p = fi.nonlinear_cube(8, "hex")
    f = FedFem(p, precision=32, T_guard=1e4)
    dtc = f.precompute()
    f.set_dt(0.9 * dtc)
    f.set_T(p.initial_T())
    st = f.get_state()
    f.set_dt(40 * dtc, force=True)
    with pytest.raises(FedFemError) as ei:
        f.step(400)
    assert ei.value.name == "ERR_DIVERGED"
    f.set_dt(0.9 * dtc)
    f.set_state(st)
    f.step(10)
    assert np.all(np.isfinite(f.get_T()))
    f.close()


def test_barrier_timeout_is_reported_not_hung():
    """A CTA withholds the publication of its completed steps; its neighbours' bounded waits run
    out, the call returns ERR_TIMEOUT and the context stays usable."""
    from paper_1909_03355_gb300.capi import FedFemError
    p = fi.nonlinear_cube(12, "hex")
    f = FedFem(p, precision=32, barrier_timeout_s=0.05, debug_withhold_barrier=1)
    dtc = f.precompute()
    assert f.info()["grid"] >= 2
    f.set_dt(0.9 * dtc)
    f.set_T(p.initial_T())
    with pytest.raises(FedFemError) as ei:
        f.step(5)
    assert ei.value.name == "ERR_TIMEOUT"
    f.close()
    g = FedFem(p, precision=32)
    g.precompute()
    g.set_dt(0.9 * dtc)
    g.set_T(p.initial_T())
    g.step(5)
    assert np.all(np.isfinite(g.get_T()))
    g.close()


# ------------------------------------------------------------------ full-size workload ------

@pytest.mark.parametrize("precision", [32, 64])
def test_full_size_large_cube_parity(precision):
    """The 128^3 workload in the launch configuration bench.py times: 10 steps from T0, the
    whole field against the oracle."""
    p = fi.large_cube(128)
    f = FedFem(p, precision=precision)
    dt = 0.9 * f.precompute()
    f.set_dt(dt)
    f.set_T(p.initial_T())
    f.step(10)
    T = f.get_T()
    f.close()
    m = O.OracleModel(p)
    ref = m.run(p.initial_T(), dt, 10)
    assert rel(T, ref) <= TOL[precision]
    # heat has started to flow: the field is not the initial one
    assert np.max(np.abs(ref - 20.0)) > 0


def test_full_config_fp32_vs_fp64_20000_steps():
    """The precision policy on the large-run configuration itself: 128^3, 20,000 steps, FP32 with
    the Kahan-compensated accumulator against the FP64 form (pinned to the oracle at 1e-10
    above), rel-L-infinity <= 2e-4."""
    p = fi.large_cube(128)
    out = {}
    for prec in (64, 32):
        f = FedFem(p, precision=prec)
        dtc = f.precompute()
        if prec == 64:
            dt = 0.9 * dtc
        f.set_dt(dt)
        f.set_T(p.initial_T())
        f.step(20000)
        out[prec] = f.get_T()
        f.close()
    assert np.all(np.isfinite(out[64])) and np.max(out[64]) > 100.0  # the cube has heated up
    assert rel(out[32], out[64]) <= TOL[32]
