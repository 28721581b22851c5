"""Batched scenarios on the GPU against per-scenario oracle runs."""
import numpy as np
import pytest

import fedfem_inputs as fi
from oracle import oracle as O

pytestmark = pytest.mark.gpu

TOL = {64: 1e-10, 32: 2e-4}


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision", [32, 64])
def test_batch_matches_oracle_per_scenario(precision):
    from paper_1909_03355_gb300.batch import FedFemBatch
    sc = fi.batched_scenarios(S=12, seed=7, n_lo=3, n_hi=10, steps_lo=20, steps_hi=150)
    sc[3].dir_nodes = np.array([0, 1, 2], np.int32)      # a Dirichlet set in one scenario
    sc[3].dir_T = np.array([50.0, 60.0, 70.0])
    b = FedFemBatch(sc, dt_scale=0.9, precision=precision)
    b.run()
    t, es, dt = b.times()
    assert es == pytest.approx(sum(p.n_elems * p.steps for p in sc))
    for s, p in enumerate(sc):
        m = O.OracleModel(p)
        # per-scenario Lanczos on the GPU, power iteration to 1e-12 in the oracle
        assert dt[s] == pytest.approx(0.9 * m.dt_crit()[0], rel=1e-8)
        ref = m.run(p.initial_T(), dt[s], p.steps)
        assert rel(b.get_T(s), ref) <= TOL[precision], s
    # scenarios with fewer steps finish no later
    order = np.argsort([p.steps for p in sc], kind="stable")
    assert np.all(np.diff(t[order]) >= 0)
    b.close()


def test_batch_replay_is_bitwise_reproducible():
    from paper_1909_03355_gb300.batch import FedFemBatch
    sc = fi.batched_scenarios(S=20, seed=11, n_lo=4, n_hi=14, steps_lo=30, steps_hi=120)
    b = FedFemBatch(sc)
    b.run()
    first = [b.get_T(s) for s in range(len(sc))]
    b.run()
    for s in range(len(sc)):
        assert np.array_equal(first[s], b.get_T(s))
    b.close()


def test_batch_launch_plans_and_autotuner():
    from paper_1909_03355_gb300.batch import FedFemBatch
    from paper_1909_03355_gb300.tune import autotune
    sc = fi.batched_scenarios(S=10, seed=13, n_lo=4, n_hi=12, steps_lo=20, steps_hi=90)
    refs = []
    for s, p in enumerate(sc):
        refs.append(O.OracleModel(p))
    plans = [dict(steps_per_launch=7), dict(steps_per_launch=50, block=256, chunk=64, stages=4, ctas_per_sm=1)]
    best, res = autotune(lambda **pl: FedFemBatch(sc, **pl), plans, lambda b: b.run(), reps=1)
    assert best in plans and all(r[1] < float("inf") for r in res)
    for plan in plans:
        b = FedFemBatch(sc, **plan)
        b.run()
        _, _, dt = b.times()
        for s, p in enumerate(sc):
            assert rel(b.get_T(s), refs[s].run(p.initial_T(), dt[s], p.steps)) <= 2e-4
        b.close()


def test_batch_rejects_bad_input():
    from paper_1909_03355_gb300.batch import FedFemBatch
    from paper_1909_03355_gb300.capi import FedFemError
    sc = fi.batched_scenarios(S=2, seed=1, n_lo=3, n_hi=4, steps_lo=5, steps_hi=9)
    sc[1].steps = 0
    with pytest.raises(FedFemError) as ei:
        FedFemBatch(sc)
    assert ei.value.name == "ERR_ARG" and "n_steps" in str(ei.value)
