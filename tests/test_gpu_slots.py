"""The slot-gather accumulation (one class per tile, per-element load slots in shared memory,
every node summing its slots in ascending order) against the FP64 oracle and the colour-phase
accumulation, its run-to-run determinism, and the plan's choice between the two."""
import numpy as np
import pytest

import fedfem_inputs as fi
from oracle import oracle as O

pytestmark = pytest.mark.gpu

TOL = {64: 1e-10, 32: 2e-4}
SLOTS, CLASSES, COLOR = 2, 3, 0


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


def run(p, dt, n, precision, **plan):
    f = FedFem(p, precision=precision, **plan)
    f.precompute()
    f.set_dt(dt, force=True)
    f.set_T(p.initial_T())
    f.step(n)
    T, info = f.get_T(), f.info()
    f.close()
    return T, info


def _problem(kind):
    if kind == "hex":
        return fi.nonlinear_cube(12, "hex", jitter=0.2)
    if kind == "tet":
        return fi.nonlinear_cube(8, "tet", jitter=0.15)
    if kind == "table":
        p = fi.nonlinear_cube(10, "hex", jitter=0.2)
        p.table_T = np.array([0.0, 100.0, 250.0, 450.0, 650.0])
        p.table_fk = np.array([1.0, 1.6, 1.2, 2.5, 2.0])
        p.table_fc = np.array([1.0, 0.8, 1.4, 1.1, 1.6])
        return p
    return fi.paper_cube("tet", 9)


@pytest.mark.parametrize("kind", ["hex", "tet", "table", "paper"])
@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("plan", [{}, {"tiles_per_cta": 3}, {"chunk": 64}], ids=["1tile", "3tiles", "chunk64"])
def test_slot_gather_matches_oracle(kind, precision, plan):
    p = _problem(kind)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit(T_hi=900.0)[0] if kind != "paper" else 0.005
    ref = m.run(p.initial_T(), dt, 300)
    T, info = run(p, dt, 300, precision, scatter=SLOTS, **plan)
    assert info["scatter"] == SLOTS and info["n_colors_max"] == 1
    assert rel(T, ref) <= TOL[precision]
    Tc, ic = run(p, dt, 300, precision, scatter=CLASSES, **plan)
    assert ic["scatter"] == COLOR
    assert rel(T, Tc) <= (1e-12 if precision == 64 else 2e-4)


def test_slot_gather_is_bitwise_reproducible():
    p = _problem("tet")
    dt = 0.9 * O.OracleModel(p).dt_crit()[0]
    a, _ = run(p, dt, 200, 32, scatter=SLOTS)
    b, _ = run(p, dt, 200, 32, scatter=SLOTS)
    assert np.array_equal(a, b)


def test_plan_chooses_slots_for_padded_tiles_only():
    """Slots where the colour classes are many and small (the paper-shaped tet cube), colour
    phases where they fill their chunks (structured hexahedra, the 64^3 tet cube)."""
    small = fi.paper_cube("tet", 19)
    f = FedFem(small, precision=32)
    assert f.info()["scatter"] == SLOTS
    f.close()
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for q in (fi.nonlinear_cube(64, "hex"), fi.nonlinear_cube(64, "tet")):
        g = FedFem(q, precision=32)
        assert g.info()["scatter"] == COLOR
        # an L2-resident hexahedral mesh runs one CTA of 15 consumer warps per SM, tets two of 7
        assert (g.info()["block"], g.info()["grid"]) == ((480, sms) if q.npe == 8 else (224, 2 * sms))
        g.close()
    big = fi.large_cube(128)
    g = FedFem(big, precision=32)
    assert g.info()["scatter"] == COLOR and g.info()["n_colors_max"] >= 8
    assert (g.info()["block"], g.info()["grid"]) == (224, 2 * sms)
    g.close()
    h = FedFem(fi.paper_cube("tet", 19), precision=32, scatter=CLASSES)
    assert h.info()["scatter"] == COLOR
    h.close()
