"""Python front end of the domain-decomposition API (fedfem_dd_*): one mesh cut into slab
sub-domains with a ghost layer, stepped together with a halo exchange after every step."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi
from .capi import FedFemError
from .fedfem import _f64, _i32, _ptr, _stream_handle, make_options, problem_structs


def subdomain(problem, n_sub, s):
    """Host-only partition query: (elements, nodes, ghost owner per node; -1 = owned) of
    sub-domain s of n_sub, global ids, ascending."""
    L = capi.load()
    keep = []
    mesh, _, _ = problem_structs(problem, keep)
    ne, nn = C.c_int64(), C.c_int64()
    rc = L.fedfem_dd_subdomain(C.byref(mesh), int(n_sub), int(s), C.byref(ne), None, C.byref(nn), None, None)
    if rc != capi.OK:
        raise FedFemError(rc, "fedfem_dd_subdomain")
    el = np.empty(ne.value, np.int32)
    nd = np.empty(nn.value, np.int32)
    go = np.empty(nn.value, np.int32)
    rc = L.fedfem_dd_subdomain(C.byref(mesh), int(n_sub), int(s), C.byref(ne), _ptr(el), C.byref(nn), _ptr(nd),
                               _ptr(go))
    if rc != capi.OK:
        raise FedFemError(rc, "fedfem_dd_subdomain")
    return el, nd, go


class FedFemDD:
    """One mesh as n_sub sub-domains (fedfem_dd)."""

    def __init__(self, problem, n_sub, precision=32, kahan=True, stream=None, **plan):
        for f in ("q_schedule", "Tinf_schedule", "Tdir_schedule", "table_T"):
            if getattr(problem, f, None) is not None:
                raise ValueError(f"{f} is not available for a decomposed mesh")
        self.L = capi.load()
        self.p = problem
        keep = []
        mesh, mats, bcs = problem_structs(problem, keep)
        plan.setdefault("quadrature", getattr(problem, "quadrature", 8))
        plan.setdefault("kT_eval", getattr(problem, "kT_eval", 0))
        plan.setdefault("face_quadrature", getattr(problem, "face_quadrature", 0))
        self.opt = make_options(precision=precision, kahan=kahan, stream=_stream_handle(stream), **plan)
        h = C.c_void_p()
        rc = self.L.fedfem_dd_create(C.byref(mesh), mats, len(problem.mats), C.byref(bcs), C.byref(self.opt),
                                     int(n_sub), C.byref(h))
        if rc != capi.OK:
            raise FedFemError(rc, self.L.fedfem_dd_error_string(None).decode())
        self.h = h
        self.n_nodes = problem.n_nodes

    def _ck(self, rc):
        if rc != capi.OK:
            raise FedFemError(rc, self.L.fedfem_dd_error_string(self.h).decode())

    def precompute(self, T_lo=None, T_hi=None):
        T_lo = self.p.T_lo if T_lo is None else T_lo
        T_hi = self.p.T_hi if T_hi is None else T_hi
        d = C.c_double()
        self._ck(self.L.fedfem_dd_precompute(self.h, float(T_lo), float(T_hi), C.byref(d)))
        return d.value

    def set_dt(self, dt, force=False):
        self._ck(self.L.fedfem_dd_set_dt(self.h, float(dt), 1 if force else 0))

    def set_T(self, T0):
        T0 = _f64(T0)
        self._ck(self.L.fedfem_dd_set_T(self.h, _ptr(T0)))

    def step(self, n):
        self._ck(self.L.fedfem_dd_step(self.h, int(n)))

    def get_T(self):
        out = np.empty(self.n_nodes)
        self._ck(self.L.fedfem_dd_get_T(self.h, _ptr(out)))
        return out

    def info(self):
        i = capi.DDInfo()
        self._ck(self.L.fedfem_dd_get_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in capi.DDInfo._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.L.fedfem_dd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
