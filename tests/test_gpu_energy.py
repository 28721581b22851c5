"""Cumulative energy balance of long runs (the energy-audit instantiation of the step kernel):
the stored-heat change and the boundary input summed in FP64 over every step since set_T,
against the oracle's per-step terms, and balanced over the full 20,000-step 128^3 run."""
import numpy as np
import pytest

import fedfem_inputs as fi
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1909_03355_gb300 import capi
    capi.load()


def FedFem(*a, **k):
    from paper_1909_03355_gb300.fedfem import FedFem as F
    return F(*a, **k)


def _problem(kind):
    p = fi.nonlinear_cube(10 if kind == "hex" else 7, kind, jitter=0.2)
    bot = np.nonzero(p.xyz[:, 2] < 1e-12)[0].astype(np.int32)
    p.dir_nodes, p.dir_T = bot, np.full(len(bot), 60.0)
    return p


@pytest.mark.parametrize("kind", ["hex", "tet"])
@pytest.mark.parametrize("precision", [64, 32])
def test_audit_totals_match_oracle_and_balance(kind, precision):
    p = _problem(kind)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit()[0]
    T, E = m.run(p.initial_T(), dt, 300, energy=True)
    S_o, B_o = E[:, 0].sum(), E[:, 1].sum()
    f = FedFem(p, precision=precision, energy_audit=True)
    f.precompute()
    f.set_dt(dt, force=True)
    f.set_T(p.initial_T())
    for k in (1, 7, 92, 200):  # split over launches of different lengths
        f.step(k)
    S, B, n = f.energy_totals()
    Tg = f.get_T()
    f.close()
    assert n == 300
    tol = 1e-10 if precision == 64 else 2e-4
    assert S == pytest.approx(S_o, rel=tol) and B == pytest.approx(B_o, rel=tol)
    assert abs(S - B) <= (1e-12 if precision == 64 else 1e-7) * abs(B)
    # the audit does not change the trajectory: same field as without it (the audit runs with
    # colour phases, so the comparison run takes them too)
    g = FedFem(p, precision=precision, scatter=3)
    g.precompute()
    g.set_dt(dt, force=True)
    g.set_T(p.initial_T())
    for k in (1, 7, 92, 200):
        g.step(k)
    assert np.array_equal(g.get_T(), Tg)
    g.close()


def test_audit_restarts_at_set_T_and_refusals():
    from paper_1909_03355_gb300.capi import FedFemError
    p = _problem("hex")
    f = FedFem(p, precision=64, energy_audit=True)
    dt = 0.9 * f.precompute()
    f.set_dt(dt)
    f.set_T(p.initial_T())
    f.step(50)
    a = f.energy_totals()
    f.set_T(p.initial_T())
    assert f.energy_totals()[2] == 0
    f.step(50)
    assert f.energy_totals() == a
    f.close()
    g = FedFem(p, precision=64)
    g.precompute()
    with pytest.raises(FedFemError) as ei:
        g.energy_totals()
    assert ei.value.name == "ERR_UNSUPPORTED"
    g.close()
    with pytest.raises(FedFemError) as ei:
        FedFem(p, precision=32, kahan=False, energy_audit=True)
    assert ei.value.name == "ERR_UNSUPPORTED"


@pytest.mark.parametrize("precision", [32, 64])
def test_cumulative_balance_full_large_run(precision):
    """The 128^3 workload for its 20,000 steps: cumulative stored heat = cumulative boundary
    and source input, within 1e-8 (FP32 + Kahan) and 1e-12 (FP64) relative."""
    p = fi.large_cube(128)
    f = FedFem(p, precision=precision, energy_audit=True)
    dt = 0.9 * f.precompute()
    f.set_dt(dt)
    f.set_T(p.initial_T())
    f.step(20000)
    S, B, n = f.energy_totals()
    f.close()
    print(f"fp{precision}: stored {S:.9e} J, input {B:.9e} J, rel residual {abs(S - B) / abs(B):.3e}")
    assert n == 20000 and B > 0
    assert abs(S - B) <= (1e-8 if precision == 32 else 1e-12) * abs(B)
