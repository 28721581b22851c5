"""FED-FEM oracle (Python side): TEST INFRASTRUCTURE ONLY.

Builds and loads ``fedfem_oracle.c`` (plain FP64 C; single-threaded, except the time stepping
``run(..., threads=n)`` over n host threads, bitwise equal to the single-threaded run) and wraps
it with numpy.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this module.  It shares no code with the CUDA library ``paper_1909_03355_gb300``; the
only common input is the problem statement built by ``fedfem_inputs``.

Function map (paper passages):
  OracleModel(...)            pre-computation stage, Fig. 1 (i): Eq. 12/17-19/22, lumped mass
                              (Section 3.1), surface area shares (Eq. 4/7 lumped to nodes)
  OracleModel.internal_loads  Eq. 11/20 with the element-mean k(T) of Section 4.2.2
  OracleModel.run             time-stepping stage, Fig. 1 (iii): Eq. 15/16, Dirichlet re-imposed
                              (threads > 1: element pass and node gather in element order)
  OracleModel.set_schedule    time-dependent loads, convection temperature and Dirichlet values
  OracleModel.set_table       tabulated k(T), c(T) factors, linear between points (Section 4.2.2)
  OracleModel.dt_crit         Section 3.4, Eq. 29
  OracleModel.adjoint         reverse-time discrete adjoint of Eq. 16/20 (derived, no paper
                              counterpart)
  kT_eval = 1 (problem field)  conductivity at the quadrature points: Eq. 20 with D(T) inside
                              the integral (orc_precompute_qp, orc_element_loads)
  face_quadrature = 1         consistent integration of Eq. 4 / 7 over the boundary faces
                              (orc_face_rule, orc_face_consistent, orc_surface_loads)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fedfem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SIGMA = 5.67e-8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Model(C.Structure):
    _fields_ = [("nn", C.c_int64), ("ne", C.c_int64), ("npe", C.c_int32), ("pad", C.c_int32),
                ("conn", C.c_void_p), ("K", C.c_void_p), ("theta", C.c_void_p), ("W", C.c_void_p),
                ("C0", C.c_void_p), ("Qext", C.c_void_p), ("Ac", C.c_void_p), ("Ar", C.c_void_p),
                ("isdir", C.c_void_p), ("k_lin", C.c_double), ("c_lin", C.c_double),
                ("h", C.c_double), ("T_inf", C.c_double), ("eps", C.c_double),
                ("T_amb", C.c_double), ("T_zero", C.c_double), ("T_ref", C.c_double),
                ("q_sched", C.c_void_p), ("Tinf_sched", C.c_void_p), ("n_sched", C.c_int64),
                ("sched_step0", C.c_int64), ("Tdir", C.c_void_p), ("Tdir_sched", C.c_void_p),
                ("n_tab", C.c_int64), ("tab_T", C.c_void_p), ("tab_fk", C.c_void_p), ("tab_fc", C.c_void_p),
                ("nq", C.c_int64), ("Kq", C.c_void_p), ("Nq", C.c_void_p),
                ("n_cf", C.c_int64), ("n_rf", C.c_int64), ("nvf", C.c_int32), ("nfq", C.c_int32),
                ("cfaces", C.c_void_p), ("rfaces", C.c_void_p), ("Mf", C.c_void_p), ("Wf", C.c_void_p),
                ("Nf", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.orc_hex_matrices.argtypes = [P, P, P, P, P]
            L.orc_hex_matrix_centre.argtypes = [P, P, P]
            L.orc_tet_matrices.argtypes = [P, P, P, P, P]
            L.orc_face_area.argtypes = [P, C.c_int]
            L.orc_face_area.restype = C.c_double
            L.orc_precompute.argtypes = [C.c_int64, C.c_int64, C.c_int32, P, P, P, P, P, P, P, P,
                                         C.c_int64, C.c_int32, P, C.c_int64, C.c_int32, P,
                                         C.c_int64, P, P, P, P, P, P, P, P]
            L.orc_precompute.restype = C.c_int64
            L.orc_internal_loads.argtypes = [P, P, P]
            L.orc_nodal_Q.argtypes = [P, C.c_int64, C.c_double]
            L.orc_nodal_Q.restype = C.c_double
            L.orc_run.argtypes = [P, C.c_double, C.c_int64, P, P, P, C.c_int32, C.c_int32, P]
            L.orc_run_mt.argtypes = [P, C.c_double, C.c_int64, P, P, P, C.c_int32, C.c_int32, P, C.c_int32]
            L.orc_dt_crit.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_int64, P]
            L.orc_dt_crit_mt.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_int64, P, C.c_int32]
            L.orc_dt_from_lambda.argtypes = [P, C.c_double, C.c_double, C.c_double]
            L.orc_dt_from_lambda.restype = C.c_double
            L.orc_adjoint.argtypes = [P, C.c_double, C.c_int64, P, P, C.c_int32, C.c_int32, P, P, P]
            L.orc_hex_matrices_qp.argtypes = [P, P, P, P]
            L.orc_face_rule.argtypes = [C.c_int, P, P]
            L.orc_face_consistent.argtypes = [C.c_int64, C.c_int32, P, P, P, P]
            L.orc_precompute_qp.argtypes = [C.c_int64, C.c_int32, P, P, P, P, C.c_int32, P, P]
            L.orc_precompute_qp.restype = C.c_int64
            L.orc_surface_loads.argtypes = [P, P, C.c_int64, P]
            _lib = L
    return _lib


def host_threads() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def hex_matrices(x, k):
    """(K [8,8], w [8], volume) of one hexahedron by 2x2x2 Gauss quadrature (Eq. 12)."""
    x, k = _f64(x), _f64(k)
    K, w, v = np.zeros((8, 8)), np.zeros(8), np.zeros(1)
    if lib().orc_hex_matrices(_p(x), _p(k), _p(K), _p(w), _p(v)):
        raise ValueError("det J <= 0")
    return K, w, float(v[0])


def hex_matrix_centre(x, k):
    """K [8,8] of one hexahedron by the one-point centre rule of Eq. 17 (weight 8)."""
    x, k = _f64(x), _f64(k)
    K = np.zeros((8, 8))
    if lib().orc_hex_matrix_centre(_p(x), _p(k), _p(K)):
        raise ValueError("det J <= 0")
    return K


def tet_matrices(x, k):
    """(K [4,4], w [4], volume) of one linear tetrahedron (Eq. 18)."""
    x, k = _f64(x), _f64(k)
    K, w, v = np.zeros((4, 4)), np.zeros(4), np.zeros(1)
    if lib().orc_tet_matrices(_p(x), _p(k), _p(K), _p(w), _p(v)):
        raise ValueError("V <= 0")
    return K, w, float(v[0])


def face_area(x):
    x = _f64(x)
    return lib().orc_face_area(_p(x), int(x.shape[0]))


def hex_matrices_qp(x, k):
    """(Kq [8,8,8], Nq [8,8]): the 2x2x2 Gauss-point matrices det J B^T k B and shape values."""
    x, k = _f64(x), _f64(k)
    Kq, Nq = np.zeros((8, 8, 8)), np.zeros((8, 8))
    if lib().orc_hex_matrices_qp(_p(x), _p(k), _p(Kq), _p(Nq)):
        raise ValueError("det J <= 0")
    return Kq, Nq


def face_rule(nv):
    """(Nf [nfq, nv], reference weights [nfq]) of the consistent face quadrature."""
    Nf, w = np.zeros(9 * 4), np.zeros(9)
    nfq = lib().orc_face_rule(int(nv), _p(Nf), _p(w))
    return Nf[:nfq * nv].reshape(nfq, nv).copy(), w[:nfq].copy()


def face_consistent(faces, xyz):
    """(Mf [n, nv, nv] face mass matrices, Wf [n, nfq] weights x area Jacobian)."""
    faces, xyz = _i32(faces), _f64(xyz)
    n, nv = faces.shape
    nfq = face_rule(nv)[0].shape[0]
    Mf, Wf = np.zeros((n, nv, nv)), np.zeros((n, nfq))
    lib().orc_face_consistent(n, nv, _p(faces), _p(xyz), _p(Mf), _p(Wf))
    return Mf, Wf


class OracleModel:
    """Pre-computed FP64 model of one problem (Fig. 1 (i))."""

    def __init__(self, p, theta=None, source=None):
        L = lib()
        self.p = p
        nn, ne, npe = p.n_nodes, p.n_elems, p.npe
        self.xyz = _f64(p.xyz)
        self.conn = _i32(p.conn)
        mats = p.mats
        self.mat_k0 = np.ascontiguousarray(np.stack([np.asarray(m.k0, float).reshape(9) for m in mats]))
        self.mat_rho = np.array([m.rho for m in mats], float)
        self.mat_c0 = np.array([m.c0 for m in mats], float)
        k_lin = {m.k_lin for m in mats}
        c_lin = {m.c_lin for m in mats}
        t_ref = {getattr(m, "T_ref", 0.0) for m in mats}
        if len(k_lin) != 1 or len(c_lin) != 1 or len(t_ref) != 1:
            raise ValueError("all materials must share k_lin, c_lin and T_ref")
        self.elem_mat = _i32(p.elem_mat)
        th = theta if theta is not None else p.elem_kscale
        self.theta = _f64(th) if th is not None else np.ones(ne)
        src = source if source is not None else p.elem_source
        self.source = _f64(src)
        self.nodal_Q_in = _f64(p.nodal_Q)
        conv = _i32(p.conv_faces) if p.conv_faces is not None and len(p.conv_faces) else None
        rad = _i32(p.rad_faces) if p.rad_faces is not None and len(p.rad_faces) else None
        dn = _i32(p.dir_nodes) if p.dir_nodes is not None and len(p.dir_nodes) else None
        self.K = np.zeros((ne, npe, npe))
        self.W = np.zeros((ne, npe))
        self.C0 = np.zeros(nn)
        self.Qext = np.zeros(nn)
        self.Ac = np.zeros(nn)
        self.Ar = np.zeros(nn)
        self.isdir = np.zeros(nn, np.int32)
        rc = L.orc_precompute(nn, ne, npe, _p(self.xyz), _p(self.conn), _p(self.elem_mat),
                              _p(self.mat_k0), _p(self.mat_rho), _p(self.mat_c0), _p(self.source),
                              _p(self.nodal_Q_in),
                              0 if conv is None else conv.shape[0], 0 if conv is None else conv.shape[1], _p(conv),
                              0 if rad is None else rad.shape[0], 0 if rad is None else rad.shape[1], _p(rad),
                              0 if dn is None else dn.shape[0], _p(dn),
                              _p(self.K), _p(self.W), _p(self.C0), _p(self.Qext), _p(self.Ac),
                              _p(self.Ar), _p(self.isdir))
        if rc:
            raise ValueError(f"element {rc - 1} has det J <= 0")
        if npe == 8 and getattr(p, "quadrature", 8) == 1:
            # one-point conduction matrices (Eq. 17); masses, loads and areas stay as computed
            for e in range(ne):
                m = 0 if p.elem_mat is None else int(p.elem_mat[e])
                if L.orc_hex_matrix_centre(_p(self.xyz[self.conn[e]]), _p(self.mat_k0[m]), _p(self.K[e])):
                    raise ValueError(f"element {e} has det J(0) <= 0")
        self._keep = (conv, rad, dn)
        self.Tdir = np.zeros(nn)
        if dn is not None:
            self.Tdir[dn] = _f64(p.dir_T)
        self.m = _Model(nn=nn, ne=ne, npe=npe, pad=0, conn=_p(self.conn), K=_p(self.K),
                        theta=_p(self.theta), W=_p(self.W), C0=_p(self.C0), Qext=_p(self.Qext),
                        Ac=_p(self.Ac), Ar=_p(self.Ar), isdir=_p(self.isdir),
                        k_lin=float(mats[0].k_lin), c_lin=float(mats[0].c_lin),
                        h=float(p.h), T_inf=float(p.T_inf), eps=float(p.eps), T_amb=float(p.T_amb),
                        T_zero=float(p.T_zero), T_ref=float(getattr(mats[0], "T_ref", 0.0)),
                        Tdir=_p(self.Tdir))
        self.mref = C.byref(self.m)
        self.variants = (int(getattr(p, "kT_eval", 0)), int(getattr(p, "face_quadrature", 0)))
        if self.variants[0] == 1:
            # conductivity at the quadrature points (Eq. 20 with D(T) inside the integral)
            one = 1 if (npe == 8 and getattr(p, "quadrature", 8) == 1) else 0
            nq = 8 if (npe == 8 and not one) else 1
            self.Kq = np.zeros((ne, nq, npe, npe))
            self.Nq = np.zeros((nq, npe))
            rc = L.orc_precompute_qp(ne, npe, _p(self.xyz), _p(self.conn), _p(self.elem_mat), _p(self.mat_k0), one,
                                     _p(self.Kq), _p(self.Nq))
            if rc:
                raise ValueError(f"element {rc - 1} has det J <= 0")
            self.m.nq, self.m.Kq, self.m.Nq = nq, _p(self.Kq), _p(self.Nq)
        if self.variants[1] == 1:
            # consistent integration of the surface loads over the boundary faces
            nv = conv.shape[1] if conv is not None else (rad.shape[1] if rad is not None else (4 if npe == 8 else 3))
            self.Nf, _ = face_rule(nv)
            self.Nf = np.ascontiguousarray(self.Nf)
            z = np.zeros((0, nv), np.int32)
            self.cf = conv if conv is not None else z
            self.rf = rad if rad is not None else z
            self.Mf, _ = face_consistent(self.cf, self.xyz)
            _, self.Wf = face_consistent(self.rf, self.xyz)
            self.m.n_cf, self.m.n_rf, self.m.nvf, self.m.nfq = len(self.cf), len(self.rf), nv, self.Nf.shape[0]
            self.m.cfaces, self.m.rfaces = _p(self.cf), _p(self.rf)
            self.m.Mf, self.m.Wf, self.m.Nf = _p(self.Mf), _p(self.Wf), _p(self.Nf)
        if getattr(p, "table_T", None) is not None:
            self.set_table(p.table_T, p.table_fk, p.table_fc)
        self._sched = (None, None, None)
        sched = [getattr(p, f, None) for f in ("q_schedule", "Tinf_schedule", "Tdir_schedule")]
        if any(s is not None for s in sched):
            self.set_schedule(*sched)

    def set_schedule(self, q_scale=None, T_inf=None, T_dir=None):
        """Time-dependent loads and Dirichlet values: at step n the external loads are
        q_scale[n] Qext, the convection ambient temperature is T_inf[n] and every prescribed
        temperature is its value in the problem plus T_dir[n] (the last entry beyond the end)."""
        q = _f64(q_scale)
        t = _f64(T_inf)
        d = _f64(T_dir)
        lens = {len(a) for a in (q, t, d) if a is not None}
        if len(lens) > 1:
            raise ValueError("q_scale, T_inf and T_dir must have the same length")
        self._sched = (q, t, d)
        self.m.q_sched = None if q is None else q.ctypes.data
        self.m.Tinf_sched = None if t is None else t.ctypes.data
        self.m.Tdir_sched = None if d is None else d.ctypes.data
        self.m.n_sched = lens.pop() if lens else 0

    def set_table(self, T, fk, fc):
        """Tabulated factors of k0 and c0 at the temperatures T (increasing; linear between
        points, end values held outside); None removes the table."""
        if T is None:
            self._tab = None
            self.m.n_tab, self.m.tab_T, self.m.tab_fk, self.m.tab_fc = 0, None, None, None
            return
        self._tab = tuple(_f64(a) for a in (T, fk, fc))
        n = len(self._tab[0])
        if n < 2 or any(len(a) != n for a in self._tab) or np.any(np.diff(self._tab[0]) <= 0):
            raise ValueError("a table needs >= 2 increasing temperatures and one factor of each kind per point")
        self.m.n_tab = n
        self.m.tab_T, self.m.tab_fk, self.m.tab_fc = (a.ctypes.data for a in self._tab)

    # lumped thermal mass at f_c = 1 (Section 3.1, Eq. 14 / 21)
    @property
    def mass(self):
        return self.C0

    def internal_loads(self, T):
        T = _f64(T)
        F = np.zeros(self.p.n_nodes)
        lib().orc_internal_loads(self.mref, _p(T), _p(F))
        return F

    def nodal_Q(self, T):
        T = _f64(T)
        L = lib()
        if self.variants[1] == 1:
            Qs = np.zeros(len(T))
            L.orc_surface_loads(self.mref, _p(T), int(self.m.sched_step0), _p(Qs))
            q = 1.0 if self._sched[0] is None else self._sched[0][min(int(self.m.sched_step0), len(self._sched[0]) - 1)]
            return q * self.Qext + Qs
        return np.array([L.orc_nodal_Q(self.mref, i, float(T[i])) for i in range(len(T))])

    def run(self, T, dt, nsteps, energy=False, sensors=None, sample_every=0, step0=0, threads=1):
        """n explicit steps from T (copied), the first being step `step0` of the load schedule;
        returns T (and per-step energy [n,2], trace).  threads > 1 (or 0: all host cores) runs
        the same steps over that many threads, with a bitwise equal result."""
        self.m.sched_step0 = int(step0)
        T = np.array(T, dtype=np.float64, copy=True)
        E = np.zeros((nsteps, 2)) if energy else None
        sens = _i32(sensors)
        trace = None
        if sens is not None and sample_every > 0:
            trace = np.zeros((nsteps // sample_every, len(sens)))
        if threads == 1:
            lib().orc_run(self.mref, float(dt), int(nsteps), _p(T), _p(E), _p(sens),
                          0 if sens is None else len(sens), int(sample_every), _p(trace))
        else:
            lib().orc_run_mt(self.mref, float(dt), int(nsteps), _p(T), _p(E), _p(sens),
                             0 if sens is None else len(sens), int(sample_every), _p(trace),
                             int(threads if threads > 0 else host_threads()))
        out = [T]
        if energy:
            out.append(E)
        if trace is not None:
            out.append(trace)
        return out[0] if len(out) == 1 else tuple(out)

    def dt_crit(self, T_lo=None, T_hi=None, tol=1e-12, max_iter=200000, threads=1):
        """(dt_crit, lambda_cond, iterations) of Section 3.4 (threads != 1: the same power
        iteration with the internal loads over several threads, bitwise the same result)."""
        T_lo = self.p.T_lo if T_lo is None else T_lo
        T_hi = self.p.T_hi if T_hi is None else T_hi
        out = np.zeros(3)
        if threads == 1:
            lib().orc_dt_crit(self.mref, float(T_lo), float(T_hi), float(tol), int(max_iter), _p(out))
        else:
            lib().orc_dt_crit_mt(self.mref, float(T_lo), float(T_hi), float(tol), int(max_iter), _p(out),
                                 int(threads if threads > 0 else host_threads()))
        return float(out[0]), float(out[1]), int(out[2])

    def dt_from_lambda(self, lam, T_lo, T_hi):
        """dt_crit of Section 3.4 for a given lambda_cond and temperature range."""
        return lib().orc_dt_from_lambda(self.mref, float(lam), float(T_lo), float(T_hi))

    def run_adaptive(self, T, nsteps, steps_per_launch, safety, margin, lam=None):
        """Steps in launches of `steps_per_launch`; before each launch dt = safety dt_crit over
        [min T - margin, max T + margin] of the current field.  Returns (T, simulated time)."""
        lam = self.dt_crit()[1] if lam is None else lam
        T = np.array(T, dtype=np.float64, copy=True)
        t, done = 0.0, 0
        while done < nsteps:
            k = min(steps_per_launch, nsteps - done)
            dt = safety * self.dt_from_lambda(lam, T.min() - margin, T.max() + margin)
            T = self.run(T, dt, k, step0=done)
            t += k * dt
            done += k
        return T, t

    def adjoint(self, dt, nsteps, T0, sensors, sample_every, dLdtrace):
        """(dL/dtheta [E], dL/dsource [E]) for a loss of the sensor trace."""
        if self.variants != (0, 0):
            raise ValueError("the adjoint covers the element-mean conductivity and lumped surface loads only")
        self.m.sched_step0 = 0
        T0 = _f64(T0)
        sens = _i32(sensors)
        g = _f64(dLdtrace)
        gt = np.zeros(self.p.n_elems)
        gs = np.zeros(self.p.n_elems)
        lib().orc_adjoint(self.mref, float(dt), int(nsteps), _p(T0), _p(sens), len(sens),
                          int(sample_every), _p(g), _p(gt), _p(gs))
        return gt, gs
