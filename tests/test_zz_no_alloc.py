"""fedfem_energy_terms_noalloc: the allocation-free variant of the energy-balance reduction.

Some callers cannot allocate device memory (cudaMalloc / cudaFree are off limits while another
library owns the memory pool, under a hard memory budget, or in loops that must not
synchronise).  This entry point takes device inputs and a device output and keeps its only
scratch in an array compiled into the library.  The test calls it twice in a row through the
C ABI and checks both results against fedfem_energy, the existing entry point that computes the
same sums with per-context scratch.  It lives in a file of its own, collected last.
"""
import ctypes as C

import numpy as np
import pytest

import fedfem_inputs as fi
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _case(n, dev):
    """A nonlinear hex cube of n^3 elements with some Dirichlet nodes after 20 FP64 steps: the
    device inputs of one step and fedfem_energy's sums for that step."""
    from paper_1909_03355_gb300 import capi
    from paper_1909_03355_gb300.fedfem import FedFem
    import torch

    p = fi.nonlinear_cube(n, "hex")
    p.dir_nodes = np.arange(0, 12, dtype=np.int32)
    p.dir_T = np.full(12, 75.0)
    f = FedFem(p, precision=64)
    dt = 0.9 * f.precompute()
    f.set_dt(dt)
    f.set_T(p.initial_T())
    f.step(20)
    T_prev = torch.empty(p.n_nodes, dtype=torch.float64, device=dev)
    T_next = torch.empty_like(T_prev)
    f.get_T_device(T_prev)
    f.step(1)
    S_ref, B_ref = f.energy()
    f.get_T_device(T_next)
    torch.cuda.synchronize()
    # node data in original order (lumped masses, loads and areas from the FP64 oracle model;
    # the internal loads at T_prev from the existing GPU entry point)
    m = O.OracleModel(p)
    F = torch.tensor(f.internal_loads(T_prev.cpu().numpy()), device=dev)
    f.close()
    arrays = [torch.tensor(a, dtype=torch.float64, device=dev) for a in (m.C0, m.Qext, m.Ac, m.Ar)]
    isdir = torch.tensor(m.isdir.astype(np.uint8), device=dev)
    ph = capi.EnergyParams(dt=dt, c_lin=p.mats[0].c_lin, h=p.h, T_inf=p.T_inf, eps=p.eps, T_amb=p.T_amb,
                           T_zero=p.T_zero, T_ref=p.mats[0].T_ref)
    ins = [T_prev, T_next, F, *arrays, isdir]
    return p.n_nodes, ins, ph, (S_ref, B_ref)


def _call(L, nn, ins, ph, out):
    return L.fedfem_energy_terms_noalloc(nn, *[a.data_ptr() for a in ins], C.byref(ph), out.data_ptr(), None)


def test_energy_terms_noalloc_matches_fedfem_energy():
    """Two calls in a row on a 20^3 cube (9,261 nodes: three blocks of partial sums, the last
    one partly filled), then two on a 9^3 cube (one block) that reads back only partials the
    larger call also wrote; every result equals fedfem_energy's at 1e-12."""
    import torch

    from paper_1909_03355_gb300 import capi

    L = capi.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    for n in (20, 9):
        nn, ins, ph, (S_ref, B_ref) = _case(n, dev)
        results = []
        for _ in range(2):
            assert _call(L, nn, ins, ph, out) == capi.OK
            torch.cuda.synchronize()
            results.append(out.cpu().numpy().copy())
            out.fill_(float("nan"))
        for S, B in results:
            assert S == pytest.approx(S_ref, rel=1e-12), n
            assert B == pytest.approx(B_ref, rel=1e-12), n
        assert np.array_equal(results[0], results[1])
    # sizes beyond the scratch capacity are rejected
    assert _call(L, 16777217, ins, ph, out) == 1
