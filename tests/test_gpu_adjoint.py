"""GPU reverse-time adjoint (fedfem_forward_record / fedfem_adjoint) against the FP64 oracle's
hand-derived adjoint and against central finite differences of the GPU forward run."""
import numpy as np
import pytest

import fedfem_inputs as fi
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def FedFem(*a, **k):
    from paper_1909_03355_gb300.fedfem import FedFem as F
    return F(*a, **k)


def small_setup(kind="hex", n=4):
    p = fi.nonlinear_cube(n, kind)
    rng = np.random.default_rng(21)
    p.elem_kscale = np.exp(0.3 * rng.standard_normal(p.n_elems))
    p.elem_source = rng.uniform(0, 2e5, p.n_elems)
    bnd = np.zeros(p.n_nodes, bool)
    bnd[np.unique(fi.boundary_faces(p.conn))] = True
    sensors = np.sort(rng.choice(np.nonzero(~bnd)[0] if (~bnd).sum() >= 6 else np.arange(p.n_nodes), 6,
                                 replace=False)).astype(np.int32)
    return p, sensors


@pytest.mark.parametrize("kind,T_ref,scheduled", [("hex", 0.0, False), ("tet", 0.0, False), ("hex", 60.0, False),
                                                   ("hex", 0.0, True), ("hex", 0.0, "table"), ("tet", 0.0, "table")])
def test_adjoint_matches_oracle_adjoint_fp64(kind, T_ref, scheduled):
    p, sensors = small_setup(kind)
    if scheduled == "table":  # tabulated k(T), c(T): the sweep carries the segment slopes
        scheduled = False
        p.table_T = np.array([0.0, 60.0, 150.0, 300.0, 600.0])
        p.table_fk = np.array([0.8, 1.0, 1.6, 1.3, 2.0])
        p.table_fc = np.array([1.1, 1.0, 0.8, 1.4, 1.2])
    if T_ref:  # laws given at a reference temperature (Section 4.2.2 form)
        m0 = p.mats[0]
        p.mats[0] = fi.Material(m0.rho, m0.k0, m0.k_lin, m0.c0, m0.c_lin, T_ref=T_ref)
    if scheduled:  # time-dependent loads (the source gradient carries q(n)) and Dirichlet values
        k = np.arange(45)
        p.q_schedule = 1.0 + 0.6 * np.cos(0.2 * k)
        p.Tinf_schedule = 20.0 + 3.0 * k
        bottom = np.flatnonzero(np.abs(p.xyz[:, 2]) < 1e-9).astype(np.int32)
        p.dir_nodes, p.dir_T = bottom, np.full(len(bottom), 20.0)
        p.Tdir_schedule = 15.0 * np.sin(0.3 * k)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    nsteps, se, ck = 60, 10, 20
    w = np.random.default_rng(3).standard_normal((nsteps // se, len(sensors)))
    gt_o, gs_o = m.adjoint(dt, nsteps, p.initial_T(), sensors, se, w)
    f = FedFem(p, precision=64)
    f.precompute()
    f.set_dt(dt, force=True)
    f.set_T(p.initial_T())
    tr = f.forward_record(nsteps, sensors, se, ck)
    _, tr_o = m.run(p.initial_T(), dt, nsteps, sensors=sensors, sample_every=se)
    assert np.max(np.abs(tr - tr_o)) <= 1e-10 * np.max(np.abs(tr_o))
    gt, gs = f.adjoint(w)
    assert np.max(np.abs(gt - gt_o)) <= 1e-9 * np.max(np.abs(gt_o))
    assert np.max(np.abs(gs - gs_o)) <= 1e-9 * np.max(np.abs(gs_o))
    # the context is left at the end state of the recorded run
    assert f.step_count == nsteps
    assert np.max(np.abs(f.get_T() - m.run(p.initial_T(), dt, nsteps))) <= 1e-9 * 1000
    f.close()


def test_adjoint_fp32_forward_close_to_oracle():
    p, sensors = small_setup("hex", 5)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    w = np.random.default_rng(4).standard_normal((8, len(sensors)))
    gt_o, gs_o = m.adjoint(dt, 80, p.initial_T(), sensors, 10, w)
    f = FedFem(p, precision=32)
    f.precompute()
    f.set_dt(dt, force=True)
    f.set_T(p.initial_T())
    f.forward_record(80, sensors, 10, 40)
    gt, gs = f.adjoint(w)
    assert np.max(np.abs(gt - gt_o)) <= 1e-3 * np.max(np.abs(gt_o))
    assert np.max(np.abs(gs - gs_o)) <= 1e-3 * np.max(np.abs(gs_o))
    f.close()


def test_adjoint_vs_central_differences_fp64():
    """Gradient of a sensor-misfit loss against central differences (delta = 1e-4 relative) of
    the GPU forward run on 20 random elements; bound 1e-5 relative."""
    p, sensors = small_setup("hex", 5)
    f = FedFem(p, precision=64)
    dt = 0.9 * f.precompute()
    f.set_dt(dt)
    nsteps, se, ck = 100, 10, 50
    th0, s0 = p.elem_kscale.copy(), p.elem_source.copy()
    target = np.random.default_rng(8).uniform(20, 40, (nsteps // se, len(sensors)))

    def loss(th, src):
        f.set_params(th, src)
        f.set_T(p.initial_T())
        tr = f.forward_record(nsteps, sensors, se, ck)
        return float(np.sum((tr - target) ** 2)), tr

    L0, tr = loss(th0, s0)
    gt, gs = f.adjoint(2.0 * (tr - target))
    rng = np.random.default_rng(9)
    for e in rng.choice(p.n_elems, 20, replace=False):
        d = 1e-4 * th0[e]
        tp, tm = th0.copy(), th0.copy()
        tp[e] += d
        tm[e] -= d
        fd = (loss(tp, s0)[0] - loss(tm, s0)[0]) / (2 * d)
        assert gt[e] == pytest.approx(fd, rel=1e-5, abs=1e-7 * np.max(np.abs(gt)))
        d = 1e-4 * max(s0[e], 1.0)
        sp, sm = s0.copy(), s0.copy()
        sp[e] += d
        sm[e] -= d
        fd = (loss(th0, sp)[0] - loss(th0, sm)[0]) / (2 * d)
        assert gs[e] == pytest.approx(fd, rel=1e-5, abs=1e-7 * np.max(np.abs(gs)))
    f.close()


def test_autograd_function_inverse_problem_small():
    import torch

    from paper_1909_03355_gb300.autograd import trace
    setup = fi.inverse_problem(n=6, steps=200, n_sensors=40, sample_every=10, ckpt_every=50)
    p = setup.problem
    f = FedFem(p, precision=64)
    dt = 0.9 * f.precompute()
    f.set_dt(dt)
    dev = torch.device("cuda")
    # ground truth trace
    src = torch.tensor(p.elem_source, device=dev, dtype=torch.float64)
    truth = trace(torch.tensor(setup.theta_true, device=dev), src, f, p.initial_T(), 200, setup.sensors, 10, 50).detach()
    th = torch.ones(p.n_elems, device=dev, dtype=torch.float64, requires_grad=True)
    s = src.clone().requires_grad_(True)
    loss = ((trace(th, s, f, p.initial_T(), 200, setup.sensors, 10, 50) - truth) ** 2).sum()
    loss.backward()
    m = O.OracleModel(p, theta=np.ones(p.n_elems))
    _, tr = m.run(p.initial_T(), dt, 200, sensors=setup.sensors, sample_every=10)
    gt_o, gs_o = m.adjoint(dt, 200, p.initial_T(), setup.sensors, 10, 2 * (tr - truth.cpu().numpy()))
    assert np.max(np.abs(th.grad.cpu().numpy() - gt_o)) <= 1e-8 * np.max(np.abs(gt_o))
    assert np.max(np.abs(s.grad.cpu().numpy() - gs_o)) <= 1e-8 * np.max(np.abs(gs_o))
    f.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_inverse_problem_full_size(precision):
    """The 32^3 inverse problem (2000 steps, 512 sensors every 10 steps, checkpoints every 100):
    GPU adjoint against the FP64 oracle adjoint."""
    setup = fi.inverse_problem()
    p = setup.problem
    m_true = O.OracleModel(p, theta=setup.theta_true)
    f = FedFem(p, precision=precision)
    dt = 0.9 * f.precompute()
    f.set_dt(dt)
    _, truth = m_true.run(p.initial_T(), dt, 2000, sensors=setup.sensors, sample_every=10)
    f.set_params(np.ones(p.n_elems), p.elem_source)
    f.set_T(p.initial_T())
    tr = f.forward_record(2000, setup.sensors, 10, 100)
    g = 2.0 * (tr - truth)
    gt, gs = f.adjoint(g)
    m = O.OracleModel(p, theta=np.ones(p.n_elems))
    gt_o, gs_o = m.adjoint(dt, 2000, p.initial_T(), setup.sensors, 10, g)
    tol = 1e-8 if precision == 64 else 2e-3
    assert np.max(np.abs(gt - gt_o)) <= tol * np.max(np.abs(gt_o))
    assert np.max(np.abs(gs - gs_o)) <= tol * np.max(np.abs(gs_o))
    f.close()


def test_device_entry_points_match_host_ones():
    """set_params / forward_record / adjoint with CUDA tensors give bitwise the host entry
    points' results; a non-positive conductivity scale on the device is refused."""
    import torch

    from paper_1909_03355_gb300.capi import FedFemError
    p, sensors = small_setup("hex", 5)
    f = FedFem(p, precision=64)
    dt = 0.9 * f.precompute()
    f.set_dt(dt)
    rng = np.random.default_rng(12)
    th = np.exp(0.2 * rng.standard_normal(p.n_elems))
    src = rng.uniform(0, 1e5, p.n_elems)
    w = rng.standard_normal((6, len(sensors)))
    f.set_params(th, src)
    f.set_T(p.initial_T())
    tr_h = f.forward_record(60, sensors, 10, 20)
    gk_h, gs_h = f.adjoint(w)
    dev = torch.device("cuda")
    f.set_params(np.ones(p.n_elems), np.zeros(p.n_elems))
    f.set_params_device(torch.tensor(th, device=dev), torch.tensor(src, device=dev))
    f.set_T_device(torch.tensor(p.initial_T(), device=dev))
    tr_d = torch.empty((6, len(sensors)), dtype=torch.float64, device=dev)
    f.forward_record_device(60, sensors, 10, 20, tr_d)
    gk_d = torch.empty(p.n_elems, dtype=torch.float64, device=dev)
    gs_d = torch.empty_like(gk_d)
    f.adjoint_device(torch.tensor(w, device=dev), gk_d, gs_d)
    assert np.array_equal(tr_d.cpu().numpy(), tr_h)
    assert np.array_equal(gk_d.cpu().numpy(), gk_h)
    assert np.array_equal(gs_d.cpu().numpy(), gs_h)
    bad = torch.tensor(th, device=dev)
    bad[7] = -1.0
    with pytest.raises(FedFemError) as ei:
        f.set_params_device(bad, None)
    assert ei.value.name == "ERR_ARG"
    f.close()
