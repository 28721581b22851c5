"""Autotuner of the launch plan (threads per CTA, chunk size, ring depth, steps per launch).

autotune(make, candidates, run, reps) builds one object per candidate plan with make(**plan),
times run(obj) with CUDA events (after one untimed call) and returns (best plan, timings).  Used
for batched scenarios on a reduced batch before the full batch is built, and for single
problems."""
from __future__ import annotations

import time


def autotune(make, candidates, run, reps=2, sync=None):
    import torch
    results = []
    for plan in candidates:
        try:
            obj = make(**plan)
        except Exception as e:  # a plan that does not fit is skipped
            results.append((plan, float("inf"), str(e)))
            continue
        try:
            run(obj)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                t0 = time.perf_counter()
                run(obj)
                torch.cuda.synchronize()
                best = min(best, time.perf_counter() - t0)
            results.append((plan, best, ""))
        finally:
            close = getattr(obj, "close", None)
            if close:
                close()
    ok = [r for r in results if r[1] != float("inf")]
    if not ok:
        raise RuntimeError("no candidate plan could be built: " + "; ".join(r[2] for r in results))
    return min(ok, key=lambda r: r[1])[0], results


BATCH_CANDIDATES = [
    dict(steps_per_launch=100),
    dict(steps_per_launch=500),
    dict(steps_per_launch=200, block=224, chunk=32, stages=9),
    dict(steps_per_launch=200, block=480, chunk=32, stages=16, ctas_per_sm=1),
    dict(steps_per_launch=200, block=224, chunk=64, stages=5),
]
