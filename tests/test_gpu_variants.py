"""GPU parity of the method variants against the FP64 oracle: the conductivity evaluated at the
quadrature points (Eq. 20 with D(T) inside the integral) and the consistent integration of the
convection and radiation loads over the boundary faces (Eq. 4, 7).  Both run on the plain
three-launch path (elements, faces, nodes)."""
import numpy as np
import pytest

import fedfem_inputs as fi
from oracle import oracle as O

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


def _problem(kind, kT, faces, table=False, quadrature=8):
    p = fi.nonlinear_cube(9 if kind == "hex" else 6, kind, jitter=0.2)
    p.kT_eval, p.face_quadrature, p.quadrature = kT, faces, quadrature
    if table:
        p.table_T = np.array([0.0, 100.0, 250.0, 450.0, 650.0])
        p.table_fk = np.array([1.0, 1.6, 1.2, 2.5, 2.0])
        p.table_fc = np.array([1.0, 0.8, 1.4, 1.1, 1.6])
    return p


CASES = [("hex", 1, 0, False, 8), ("hex", 1, 0, True, 8), ("hex", 0, 1, False, 8), ("hex", 1, 1, True, 8),
         ("tet", 1, 1, True, 8), ("tet", 0, 1, False, 8), ("hex", 1, 0, True, 1)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-kT{c[1]}-faces{c[2]}-tab{int(c[3])}-q{c[4]}")
@pytest.mark.parametrize("precision", [64, 32])
def test_variant_run_matches_oracle(case, precision):
    kind, kT, faces, table, quad = case
    p = _problem(kind, kT, faces, table, quad)
    m = O.OracleModel(p)
    dt = 0.9 * m.dt_crit(T_hi=900.0)[0]
    steps = 600
    ref = m.run(p.initial_T(), dt, steps)
    f = FedFem(p, precision=precision)
    f.precompute()
    f.set_dt(dt, force=True)
    f.set_T(p.initial_T())
    f.step(steps)
    T = f.get_T()
    f.close()
    assert rel(T, ref) <= TOL[precision]
    # the variant changed the result (it is not the default path under another name)
    q = _problem(kind, 0, 0, table, quad)
    base = O.OracleModel(q).run(q.initial_T(), dt, steps)
    assert rel(base, ref) > 1e-6


def test_variant_internal_loads_and_energy():
    """FP64 internal loads with the conductivity at the quadrature points against the oracle's,
    and the energy balance of a step with consistent faces (stored heat = boundary input)."""
    p = _problem("hex", 1, 1, True)
    m = O.OracleModel(p)
    T = fi.random_state(p, 4)
    f = FedFem(p, precision=64)
    dt = 0.9 * f.precompute()
    assert rel(f.internal_loads(T), m.internal_loads(T)) <= 1e-12
    f.set_dt(dt)
    f.set_T(p.initial_T())
    f.step(50)
    S, B = f.energy()
    f.close()
    assert abs(S - B) <= 1e-10 * abs(B)
    _, E = m.run(p.initial_T(), dt, 50, energy=True)
    assert S == pytest.approx(E[-1, 0], rel=1e-9)


def test_variant_refusals():
    """Paths that cover the default forms only refuse the variants cleanly."""
    from paper_1909_03355_gb300.batch import FedFemBatch
    from paper_1909_03355_gb300.capi import FedFemError
    from paper_1909_03355_gb300.dd import FedFemDD
    p = _problem("hex", 1, 0)
    f = FedFem(p, precision=32)
    f.precompute()
    f.set_dt(0.9 * f.info()["dt_crit"])
    f.set_T(p.initial_T())
    with pytest.raises(FedFemError) as ei:
        f.forward_record(20, np.array([3, 5], np.int32), 10, 10)
    assert ei.value.name == "ERR_UNSUPPORTED"
    f.close()
    with pytest.raises(FedFemError) as ei:
        FedFemDD(p, 2)
    assert ei.value.name == "ERR_UNSUPPORTED"
    with pytest.raises(FedFemError) as ei:
        FedFemBatch([_problem("hex", 0, 0), _problem("hex", 0, 0)], kT_eval=1)
    assert ei.value.name == "ERR_UNSUPPORTED"
