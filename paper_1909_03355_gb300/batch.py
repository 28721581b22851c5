"""Python front end of the batched-scenario API (fedfem_batch_*): many independent problems,
each with its own mesh, material, boundary data, time step and step count, advanced together
by the CUDA step kernel under one captured CUDA graph."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi
from .capi import FedFemError
from .fedfem import _f64, _ptr, make_options, problem_structs, _stream_handle


class FedFemBatch:
    def __init__(self, problems, dt_scale=0.9, precision=32, kahan=True, stream=None, **plan):
        # per-step schedules and property tables belong to single-problem contexts
        for p in problems:
            for f in ("q_schedule", "Tinf_schedule", "Tdir_schedule", "table_T"):
                if getattr(p, f, None) is not None:
                    raise ValueError(f"{f} is not available for batched scenarios")
            for f in ("kT_eval", "face_quadrature"):
                if getattr(p, f, 0):
                    raise ValueError(f"{f} is not available for batched scenarios")
        self.L = capi.load()
        keep = []
        S = len(problems)
        sc = (capi.Scenario * S)()
        for i, p in enumerate(problems):
            mesh, mats, bcs = problem_structs(p, keep)
            if len(p.mats) != 1:
                raise ValueError("one material per scenario")
            T0 = _f64(p.initial_T())
            keep += [mats, T0]
            sc[i].mesh, sc[i].mat, sc[i].bcs = mesh, mats[0], bcs
            sc[i].T0 = _ptr(T0)
            sc[i].n_steps = int(p.steps)
            sc[i].T_lo, sc[i].T_hi = float(p.T_lo), float(p.T_hi)
            sc[i].dt_scale = float(dt_scale)
        self.opt = make_options(precision=precision, kahan=kahan, stream=_stream_handle(stream), **plan)
        h = C.c_void_p()
        st = self.L.fedfem_batch_create(sc, S, C.byref(self.opt), C.byref(h))
        if st != capi.OK:
            msg = self.L.fedfem_batch_error_string(h).decode() if h.value else ""
            if h.value:
                self.L.fedfem_batch_destroy(h)
            raise FedFemError(st, msg)
        self.h = h
        self.S = S
        self.n_nodes = [p.n_nodes for p in problems]

    def _ck(self, st):
        if st != capi.OK:
            raise FedFemError(st, self.L.fedfem_batch_error_string(self.h).decode())

    def run(self):
        self._ck(self.L.fedfem_batch_run(self.h))

    def times(self):
        """(completion time of each scenario in ns since the run started, total element-steps,
        dt of each scenario)."""
        t = np.empty(self.S)
        dt = np.empty(self.S)
        es = C.c_double()
        self._ck(self.L.fedfem_batch_times(self.h, _ptr(t), C.byref(es), _ptr(dt)))
        return t, es.value, dt

    def get_T(self, s):
        out = np.empty(self.n_nodes[s])
        self._ck(self.L.fedfem_batch_get_T(self.h, int(s), _ptr(out)))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.L.fedfem_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
