"""Python front end of libfedfem.so: one FedFem object per problem (a fedfem_ctx).

The object keeps the numpy inputs alive while the C call copies them, converts results and
raises FedFemError on any non-OK status.  Device memory, streams and the torch.autograd
wrapper use PyTorch; the arithmetic of the method runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi
from .capi import FedFemError


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data


def problem_structs(p, keep):
    """(Mesh, [Material], Bcs) C structs for a fedfem_inputs.Problem-like object; arrays that
    must stay alive during the call are appended to `keep`."""
    xyz, conn = _f64(p.xyz), _i32(p.conn)
    mat = _i32(p.elem_mat)
    ks = _f64(p.elem_kscale)
    keep += [xyz, conn, mat, ks]
    mesh = capi.Mesh(nodes_per_elem=conn.shape[1], reserved=0, n_nodes=xyz.shape[0], n_elems=conn.shape[0],
                     xyz=_ptr(xyz), conn=_ptr(conn), elem_mat=_ptr(mat), elem_kscale=_ptr(ks))
    mats = (capi.Material * len(p.mats))()
    for i, m in enumerate(p.mats):
        mats[i].rho = m.rho
        for r, v in enumerate(np.asarray(m.k0, float).reshape(9)):
            mats[i].k0[r] = v
        mats[i].k_lin, mats[i].c0, mats[i].c_lin = m.k_lin, m.c0, m.c_lin
        mats[i].T_ref = getattr(m, "T_ref", 0.0)
    dn = _i32(p.dir_nodes) if p.dir_nodes is not None and len(p.dir_nodes) else None
    dT = _f64(p.dir_T) if dn is not None else None
    cf = _i32(p.conv_faces) if p.conv_faces is not None and len(p.conv_faces) else None
    rf = _i32(p.rad_faces) if p.rad_faces is not None and len(p.rad_faces) else None
    nq = _f64(p.nodal_Q)
    src = _f64(p.elem_source)
    keep += [dn, dT, cf, rf, nq, src]
    nv = cf.shape[1] if cf is not None else (rf.shape[1] if rf is not None else (4 if conn.shape[1] == 8 else 3))
    bcs = capi.Bcs(n_dir=0 if dn is None else len(dn), dir_nodes=_ptr(dn), dir_T=_ptr(dT),
                   n_conv_faces=0 if cf is None else cf.shape[0], conv_faces=_ptr(cf), h=p.h, T_inf=p.T_inf,
                   n_rad_faces=0 if rf is None else rf.shape[0], rad_faces=_ptr(rf), eps=p.eps, T_amb=p.T_amb,
                   T_zero=p.T_zero, face_nv=nv, reserved=0, nodal_Q=_ptr(nq), elem_source=_ptr(src))
    return mesh, mats, bcs


def make_options(precision=32, kahan=True, scatter=0, block=0, steps_per_launch=0, ctas_per_sm=0,
                 tiles_per_cta=0, stages=0, chunk=0, l2_policy=0, barrier_timeout_s=1.0, T_guard=1e6, stream=None, device=-1,
                 verbose=False, debug_withhold_barrier=0, quadrature=0, kT_eval=0, face_quadrature=0,
                 start_stagger_us=0.0, energy_audit=False):
    L = capi.load()
    o = capi.Options()
    L.fedfem_default_options(C.byref(o))
    o.precision = precision
    o.kahan = 1 if kahan else 0
    o.scatter = scatter
    o.block = block
    o.steps_per_launch = steps_per_launch
    o.ctas_per_sm = ctas_per_sm
    o.tiles_per_cta = tiles_per_cta
    o.stages = stages
    o.chunk = chunk
    o.l2_policy = l2_policy
    o.barrier_timeout_s = barrier_timeout_s
    o.T_guard = T_guard
    o.stream = stream
    o.device = device
    o.verbose = 1 if verbose else 0
    o.debug_withhold_barrier = debug_withhold_barrier
    o.quadrature = quadrature
    o.kT_eval = kT_eval
    o.face_quadrature = face_quadrature
    o.start_stagger_us = start_stagger_us
    o.energy_audit = 1 if energy_audit else 0
    return o


def check_tiling(problem, n_tiles, chunk=32, single_class=False):
    """Host-only check of the tiling the step kernel would use for `problem` (no GPU needed):
    returns its statistics, or raises FedFemError with the reason.  The nodes of the problem's
    convection and radiation faces are the boundary nodes, as in fedfem_create."""
    L = capi.load()
    keep = []
    mesh, _, bcs = problem_structs(problem, keep)
    faces = [f for f in (problem.conv_faces, problem.rad_faces) if f is not None and len(f)]
    bnd = _i32(np.unique(np.concatenate([np.asarray(f).ravel() for f in faces]))) if faces else None
    st = capi.TilingStats()
    rc = L.fedfem_check_tiling(C.byref(mesh), 0 if bnd is None else len(bnd), _ptr(bnd), int(n_tiles), int(chunk),
                               1 if single_class else 0, C.byref(st))
    if rc != capi.OK:
        raise FedFemError(rc, L.fedfem_create_error().decode())
    return {f: getattr(st, f) for f, _ in capi.TilingStats._fields_}


def _stream_handle(stream):
    """cudaStream_t of a torch.cuda.Stream (or an int handle, or None for the legacy default)."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class FedFem:
    """One FED-FEM problem on the GPU (fedfem_ctx)."""

    def __init__(self, problem, precision=32, kahan=True, stream=None, **plan):
        self.L = capi.load()
        self.p = problem
        keep = []
        mesh, mats, bcs = problem_structs(problem, keep)
        plan.setdefault("quadrature", getattr(problem, "quadrature", 8))
        plan.setdefault("kT_eval", getattr(problem, "kT_eval", 0))
        plan.setdefault("face_quadrature", getattr(problem, "face_quadrature", 0))
        self.opt = make_options(precision=precision, kahan=kahan, stream=_stream_handle(stream), **plan)
        h = C.c_void_p()
        st = self.L.fedfem_create(C.byref(mesh), mats, len(problem.mats), C.byref(bcs), C.byref(self.opt),
                                  C.byref(h))
        if st != capi.OK:
            raise FedFemError(st, self.L.fedfem_create_error().decode())
        self.h = h
        self.n_nodes = problem.n_nodes
        self.n_elems = problem.n_elems
        self.precision = precision
        sched = [getattr(problem, f, None) for f in ("q_schedule", "Tinf_schedule", "Tdir_schedule")]
        if any(s is not None for s in sched):
            self.set_schedule(*sched)
        if getattr(problem, "table_T", None) is not None:
            self.set_table(problem.table_T, problem.table_fk, problem.table_fc)

    def set_table(self, T=None, fk=None, fc=None):
        """Tabulated factors of k0 and c0 at the increasing temperatures T (2 to 8 points,
        linear between points, end values held outside; nodal values averaged per element for
        k as in Section 4.2.2); they replace the materials' linear laws.  Call before
        precompute(); T=None removes the table."""
        if T is None:
            self._ck(self.L.fedfem_set_property_table(self.h, 0, None, None, None))
            return
        arrs = [_f64(a) for a in (T, fk, fc)]
        if len({len(a) for a in arrs}) != 1:
            raise ValueError("T, fk and fc must have the same length")
        self._table = tuple(arrs)
        self._ck(self.L.fedfem_set_property_table(self.h, len(arrs[0]), *[_ptr(a) for a in arrs]))

    def set_schedule(self, q_scale=None, T_inf=None, T_dir=None):
        """Time-dependent loads and prescribed temperatures: at step n the external loads are
        q_scale[n] Q_ext, the convection ambient temperature is T_inf[n] and every Dirichlet
        node holds its prescribed value plus T_dir[n] (the last entries hold beyond the end)."""
        arrs = [_f64(a) for a in (q_scale, T_inf, T_dir)]
        lens = {len(a) for a in arrs if a is not None}
        if len(lens) > 1:
            raise ValueError("q_scale, T_inf and T_dir must have the same length")
        self._sched = tuple(arrs)
        self._ck(self.L.fedfem_set_schedule(self.h, lens.pop() if lens else 0, *[_ptr(a) for a in arrs]))

    # -- errors
    def _ck(self, st):
        if st != capi.OK:
            raise FedFemError(st, self.L.fedfem_error_string(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.fedfem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- Fig. 1 (i)-(iii)
    def precompute(self, T_lo=None, T_hi=None):
        T_lo = self.p.T_lo if T_lo is None else T_lo
        T_hi = self.p.T_hi if T_hi is None else T_hi
        d = C.c_double()
        self._ck(self.L.fedfem_precompute(self.h, float(T_lo), float(T_hi), C.byref(d)))
        return d.value

    def set_dt(self, dt, force=False):
        self._ck(self.L.fedfem_set_dt(self.h, float(dt), 1 if force else 0))

    def set_T(self, T0):
        a = _f64(T0)
        assert a.shape == (self.n_nodes,)
        self._ck(self.L.fedfem_set_T(self.h, _ptr(a)))

    def set_T_device(self, t):
        """t: torch float64 CUDA tensor [n_nodes] (original node order)."""
        assert t.dtype.itemsize == 8 and t.is_contiguous() and t.numel() == self.n_nodes
        self._ck(self.L.fedfem_set_T_device(self.h, C.c_void_p(t.data_ptr())))

    def step(self, n):
        self._ck(self.L.fedfem_step(self.h, int(n)))

    def step_adaptive(self, n, safety=0.9, margin=0.0):
        """n steps with dt = safety dt_crit over the current temperature range (+- margin),
        re-evaluated before every launch; returns the simulated time."""
        t = C.c_double()
        self._ck(self.L.fedfem_step_adaptive(self.h, int(n), float(safety), float(margin), C.byref(t)))
        return t.value

    def step_async(self, n):
        self._ck(self.L.fedfem_step_async(self.h, int(n)))

    def sync(self):
        self._ck(self.L.fedfem_sync(self.h))

    def get_T(self, out=None):
        """Current field (original node order) into a new array, or into `out` (float64,
        contiguous, n_nodes; e.g. a view of pinned host memory)."""
        if out is None:
            out = np.empty(self.n_nodes)
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.shape == (self.n_nodes,)
        self._ck(self.L.fedfem_get_T(self.h, _ptr(out)))
        return out

    def get_T_device(self, t):
        assert t.dtype.itemsize == 8 and t.is_contiguous() and t.numel() == self.n_nodes
        self._ck(self.L.fedfem_get_T_device(self.h, C.c_void_p(t.data_ptr())))

    @property
    def step_count(self):
        v = C.c_int64()
        self._ck(self.L.fedfem_get_step(self.h, C.byref(v)))
        return v.value

    def energy(self):
        s, b = C.c_double(), C.c_double()
        self._ck(self.L.fedfem_energy(self.h, C.byref(s), C.byref(b)))
        return s.value, b.value

    def energy_totals(self):
        """(stored heat change, boundary input, steps) summed since the last set_T (contexts
        created with energy_audit=True)."""
        s, b, n = C.c_double(), C.c_double(), C.c_int64()
        self._ck(self.L.fedfem_energy_totals(self.h, C.byref(s), C.byref(b), C.byref(n)))
        return s.value, b.value, n.value

    def internal_loads(self, T):
        a = _f64(T)
        out = np.empty(self.n_nodes)
        self._ck(self.L.fedfem_internal_loads(self.h, _ptr(a), _ptr(out)))
        return out

    def set_params(self, kscale=None, source=None):
        k, s = _f64(kscale), _f64(source)
        self._ck(self.L.fedfem_set_params(self.h, _ptr(k), _ptr(s)))

    def set_params_device(self, kscale=None, source=None):
        """Per-element conductivity scales / sources from contiguous FP64 CUDA tensors."""
        for t in (kscale, source):
            assert t is None or (t.is_cuda and t.dtype.itemsize == 8 and t.is_contiguous() and t.numel() == self.n_elems)
        self._ck(self.L.fedfem_set_params_device(self.h, None if kscale is None else kscale.data_ptr(),
                                                 None if source is None else source.data_ptr()))

    def get_state(self):
        n = C.c_size_t()
        self._ck(self.L.fedfem_state_bytes(self.h, C.byref(n)))
        buf = np.empty(n.value, np.uint8)
        self._ck(self.L.fedfem_get_state(self.h, _ptr(buf)))
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, np.uint8)
        self._ck(self.L.fedfem_set_state(self.h, _ptr(buf)))

    def forward_record(self, n_steps, sensors, sample_every, ckpt_every):
        s = _i32(sensors)
        trace = np.empty((n_steps // sample_every, len(s)))
        self._ck(self.L.fedfem_forward_record(self.h, int(n_steps), _ptr(s), len(s), int(sample_every),
                                              int(ckpt_every), _ptr(trace)))
        return trace

    def forward_record_device(self, n_steps, sensors, sample_every, ckpt_every, trace):
        """forward_record with the trace written into a contiguous FP64 CUDA tensor
        [n_steps / sample_every, n_sensors]."""
        s = _i32(sensors)
        assert trace.is_cuda and trace.is_contiguous() and trace.numel() == (n_steps // sample_every) * len(s)
        self._ck(self.L.fedfem_forward_record_device(self.h, int(n_steps), _ptr(s), len(s), int(sample_every),
                                                     int(ckpt_every), trace.data_ptr()))
        return trace

    def adjoint_device(self, dL_dtrace, dL_dkscale, dL_dsource):
        """adjoint with contiguous FP64 CUDA tensors in and out."""
        for t in (dL_dtrace, dL_dkscale, dL_dsource):
            assert t.is_cuda and t.is_contiguous() and t.dtype.itemsize == 8
        self._ck(self.L.fedfem_adjoint_device(self.h, dL_dtrace.data_ptr(), dL_dkscale.data_ptr(),
                                              dL_dsource.data_ptr()))

    def adjoint(self, dL_dtrace):
        g = _f64(dL_dtrace)
        gk = np.empty(self.n_elems)
        gs = np.empty(self.n_elems)
        self._ck(self.L.fedfem_adjoint(self.h, _ptr(g), _ptr(gk), _ptr(gs)))
        return gk, gs

    def info(self):
        i = capi.Info()
        self._ck(self.L.fedfem_get_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in capi.Info._fields_}
