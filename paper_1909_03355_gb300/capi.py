"""ctypes binding of libfedfem.so (include/fedfem.h).  Argument marshalling only: every step of
the method runs in the library's CUDA kernels; there is no CPU fallback.  Importing this module
raises if the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

P = C.c_void_p
I32 = C.c_int32
I64 = C.c_int64
F64 = C.c_double

OK = 0
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_MESH", 3: "ERR_UNSTABLE", 4: "ERR_DIVERGED", 5: "ERR_TIMEOUT",
          6: "ERR_CUDA", 7: "ERR_OOM", 8: "ERR_STATE", 9: "ERR_UNSUPPORTED"}
FP32, FP64 = 32, 64
SCATTER_COLOR, SCATTER_ATOMIC, SCATTER_SLOTS, SCATTER_CLASSES = 0, 1, 2, 3


class Mesh(C.Structure):
    _fields_ = [("nodes_per_elem", I32), ("reserved", I32), ("n_nodes", I64), ("n_elems", I64),
                ("xyz", P), ("conn", P), ("elem_mat", P), ("elem_kscale", P)]


class Material(C.Structure):
    _fields_ = [("rho", F64), ("k0", F64 * 9), ("k_lin", F64), ("c0", F64), ("c_lin", F64), ("T_ref", F64)]


class Bcs(C.Structure):
    _fields_ = [("n_dir", I64), ("dir_nodes", P), ("dir_T", P),
                ("n_conv_faces", I64), ("conv_faces", P), ("h", F64), ("T_inf", F64),
                ("n_rad_faces", I64), ("rad_faces", P), ("eps", F64), ("T_amb", F64), ("T_zero", F64),
                ("face_nv", I32), ("reserved", I32), ("nodal_Q", P), ("elem_source", P)]


class Options(C.Structure):
    _fields_ = [("precision", I32), ("kahan", I32), ("scatter", I32), ("block", I32),
                ("steps_per_launch", I32), ("ctas_per_sm", I32), ("tiles_per_cta", I32), ("stages", I32),
                ("chunk", I32), ("l2_policy", I32), ("barrier_timeout_s", F64), ("T_guard", F64), ("stream", P), ("device", I32),
                ("verbose", I32), ("debug_withhold_barrier", I32), ("quadrature", I32), ("kT_eval", I32),
                ("face_quadrature", I32), ("reserved2", I32), ("start_stagger_us", F64), ("energy_audit", I32),
                ("reserved3", I32)]


class Info(C.Structure):
    _fields_ = [("n_nodes", I64), ("n_elems", I64), ("n_tiles", I32), ("grid", I32), ("block", I32),
                ("stages", I32), ("chunk", I32), ("scatter", I32), ("steps_per_launch", I32), ("max_tile_nodes", I32), ("n_colors_max", I32),
                ("smem_bytes", I32), ("n_shared_nodes", I64), ("n_halo_slots", I64), ("elem_bytes", I64),
                ("dt", F64), ("dt_crit", F64)]


class TilingStats(C.Structure):
    _fields_ = [("n_tiles", I32), ("n_chunks", I32), ("max_tile_nodes", I32), ("n_colors_max", I32),
                ("n_shared_nodes", I64), ("n_halo_slots", I64), ("n_padding_slots", I64)]


class Scenario(C.Structure):
    _fields_ = [("mesh", Mesh), ("mat", Material), ("bcs", Bcs), ("T0", P), ("n_steps", I64),
                ("T_lo", F64), ("T_hi", F64), ("dt_scale", F64)]


class DDInfo(C.Structure):
    _fields_ = [("n_sub", I32), ("axis", I32), ("n_messages", I32), ("reserved", I32), ("halo_entries", I64),
                ("halo_bytes_per_step", I64), ("ghost_elements", I64), ("step", I64), ("dt_crit", F64)]


class EnergyParams(C.Structure):
    _fields_ = [("dt", F64), ("c_lin", F64), ("h", F64), ("T_inf", F64), ("eps", F64), ("T_amb", F64),
                ("T_zero", F64), ("T_ref", F64)]


# exported names and their (restype, argtypes), as declared in include/fedfem.h
SIGNATURES = {
    "fedfem_default_options": (None, [P]),
    "fedfem_create": (I32, [P, P, I32, P, P, P]),
    "fedfem_precompute": (I32, [P, F64, F64, P]),
    "fedfem_set_dt": (I32, [P, F64, I32]),
    "fedfem_set_T": (I32, [P, P]),
    "fedfem_set_T_device": (I32, [P, P]),
    "fedfem_step": (I32, [P, I64]),
    "fedfem_step_adaptive": (I32, [P, I64, F64, F64, P]),
    "fedfem_step_async": (I32, [P, I64]),
    "fedfem_sync": (I32, [P]),
    "fedfem_get_T": (I32, [P, P]),
    "fedfem_get_T_device": (I32, [P, P]),
    "fedfem_get_step": (I32, [P, P]),
    "fedfem_energy": (I32, [P, P, P]),
    "fedfem_energy_totals": (I32, [P, P, P, P]),
    "fedfem_internal_loads": (I32, [P, P, P]),
    "fedfem_set_params": (I32, [P, P, P]),
    "fedfem_set_schedule": (I32, [P, I64, P, P, P]),
    "fedfem_set_property_table": (I32, [P, I32, P, P, P]),
    "fedfem_state_bytes": (I32, [P, P]),
    "fedfem_get_state": (I32, [P, P]),
    "fedfem_set_state": (I32, [P, P]),
    "fedfem_forward_record": (I32, [P, I64, P, I32, I32, I32, P]),
    "fedfem_adjoint": (I32, [P, P, P, P]),
    "fedfem_adjoint_device": (I32, [P, P, P, P]),
    "fedfem_forward_record_device": (I32, [P, I64, P, I32, I32, I32, P]),
    "fedfem_set_params_device": (I32, [P, P, P]),
    "fedfem_get_info": (I32, [P, P]),
    "fedfem_check_tiling": (I32, [P, I64, P, I32, I32, I32, P]),
    "fedfem_energy_terms_noalloc": (I32, [I64, P, P, P, P, P, P, P, P, P, P, P]),
    "fedfem_error_string": (C.c_char_p, [P]),
    "fedfem_create_error": (C.c_char_p, []),
    "fedfem_destroy": (None, [P]),
    "fedfem_batch_create": (I32, [P, I32, P, P]),
    "fedfem_batch_run": (I32, [P]),
    "fedfem_batch_times": (I32, [P, P, P, P]),
    "fedfem_batch_get_T": (I32, [P, I32, P]),
    "fedfem_batch_error_string": (C.c_char_p, [P]),
    "fedfem_batch_destroy": (None, [P]),
    "fedfem_dd_create": (I32, [P, P, I32, P, P, I32, P]),
    "fedfem_dd_precompute": (I32, [P, F64, F64, P]),
    "fedfem_dd_set_dt": (I32, [P, F64, I32]),
    "fedfem_dd_set_T": (I32, [P, P]),
    "fedfem_dd_step": (I32, [P, I64]),
    "fedfem_dd_get_T": (I32, [P, P]),
    "fedfem_dd_get_info": (I32, [P, P]),
    "fedfem_dd_subdomain": (I32, [P, I32, I32, P, P, P, P, P]),
    "fedfem_dd_error_string": (C.c_char_p, [P]),
    "fedfem_dd_destroy": (None, [P]),
    "fedfem_probe_copy": (I32, [P, P, I64, I32, I32, P, P]),
    "fedfem_probe_fp64": (I32, [I64, I32, P, P, P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libfedfem.so (building it first only when asked).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        _build.build()
    try:  # share the CUDA runtime already loaded by PyTorch, if any
        import torch  # noqa: F401
    except Exception:
        pass
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class FedFemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))
