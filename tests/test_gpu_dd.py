"""Domain decomposition on the GPU: 2 and 4 slab sub-domains of one mesh on one device, each a
context of its own with explicit halo buffers, against the undecomposed GPU run and the FP64
oracle."""
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


def _problem(kind):
    if kind == "hex":
        return fi.nonlinear_cube(14, "hex", jitter=0.2)
    if kind == "tet":
        return fi.nonlinear_cube(9, "tet")
    p = fi.large_cube(12, jitter=0.15)
    bot = np.nonzero(p.xyz[:, 2] < 1e-12)[0].astype(np.int32)
    p.dir_nodes, p.dir_T = bot, np.full(len(bot), 150.0)
    p.nodal_Q = np.linspace(0.0, 0.3, p.n_nodes)
    return p


@pytest.mark.parametrize("kind", ["hex", "tet", "bcs"])
@pytest.mark.parametrize("n_sub", [2, 4])
@pytest.mark.parametrize("precision", [64, 32])
def test_decomposed_run_matches_whole_mesh_and_oracle(kind, n_sub, precision):
    from paper_1909_03355_gb300.dd import FedFemDD
    from paper_1909_03355_gb300.fedfem import FedFem
    p = _problem(kind)
    steps = 300
    whole = FedFem(p, precision=precision)
    dtc = whole.precompute()
    dt = 0.9 * dtc
    whole.set_dt(dt)
    whole.set_T(p.initial_T())
    whole.step(steps)
    Tw = whole.get_T()
    whole.close()
    d = FedFemDD(p, n_sub, precision=precision)
    dtc_dd = d.precompute()
    # principal sub-matrices: the decomposed critical step is not below the whole mesh's and,
    # on these meshes, close to it
    assert dtc <= dtc_dd * (1 + 1e-9) and dtc_dd <= dtc * 1.05
    d.set_dt(dt)
    d.set_T(p.initial_T())
    d.step(steps)
    Td = d.get_T()
    info = d.info()
    d.close()
    assert info["n_sub"] == n_sub and info["step"] == steps and info["halo_entries"] > 0
    assert info["n_messages"] >= 2 * (n_sub - 1)
    ref = O.OracleModel(p).run(p.initial_T(), dt, steps)
    assert rel(Td, ref) <= TOL[precision]
    assert rel(Td, Tw) <= (1e-12 if precision == 64 else 2e-4)


def test_decomposed_run_in_pieces_and_reset():
    """Steps split over calls, and a new initial field, give the same field as one call."""
    from paper_1909_03355_gb300.dd import FedFemDD
    p = _problem("hex")
    d = FedFemDD(p, 3, precision=64)
    dt = 0.9 * d.precompute()
    d.set_dt(dt)
    d.set_T(p.initial_T())
    d.step(120)
    a = d.get_T()
    d.set_T(p.initial_T())
    for k in (1, 19, 100):
        d.step(k)
    b = d.get_T()
    d.close()
    assert np.array_equal(a, b)
