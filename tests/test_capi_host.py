"""CPU-only checks of the C ABI boundary: the library builds, loads without a GPU and exports
exactly the entry points declared in include/fedfem.h; the Python binding mirrors the C structs."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fedfem.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(fedfem_[A-Za-z_0-9]+)\s*\(", src))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1909_03355_gb300 import build
    return build.build()


def test_library_exports_every_declared_function(lib_path):
    decl = declared_functions()
    assert len(decl) >= 25
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(fedfem_[A-Za-z_0-9]+)$", out, flags=re.M))
    assert decl - exported == set(), f"declared but not exported: {sorted(decl - exported)}"
    assert exported - decl == set(), f"exported but not declared: {sorted(exported - decl)}"


def test_binding_signatures_cover_header(lib_path):
    from paper_1909_03355_gb300 import capi
    assert set(capi.SIGNATURES) == declared_functions()
    L = capi.load()
    for name in capi.SIGNATURES:
        assert getattr(L, name) is not None


def test_struct_layouts_match_header(lib_path):
    """Compile a tiny C program against the header and compare sizeof / offsetof with ctypes."""
    from paper_1909_03355_gb300 import capi
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "fedfem.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(fedfem_mesh), sizeof(fedfem_material), sizeof(fedfem_bcs),
         sizeof(fedfem_options), sizeof(fedfem_info), sizeof(fedfem_scenario));
  printf("%zu %zu %zu %zu\n", offsetof(fedfem_bcs, face_nv), offsetof(fedfem_bcs, elem_source),
         offsetof(fedfem_options, stream), offsetof(fedfem_options, debug_withhold_barrier));
  printf("%zu %zu\n", offsetof(fedfem_info, dt), offsetof(fedfem_scenario, dt_scale));
  printf("%zu %zu %zu %zu\n", sizeof(fedfem_energy_params), sizeof(fedfem_tiling_stats),
         offsetof(fedfem_tiling_stats, n_shared_nodes), offsetof(fedfem_options, quadrature));
  printf("%zu %zu %zu\n", sizeof(fedfem_dd_info), offsetof(fedfem_dd_info, halo_entries),
         offsetof(fedfem_dd_info, dt_crit));
  return 0;
}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "s.c")
        exe = os.path.join(d, "s")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out]
    want = [C.sizeof(capi.Mesh), C.sizeof(capi.Material), C.sizeof(capi.Bcs), C.sizeof(capi.Options),
            C.sizeof(capi.Info), C.sizeof(capi.Scenario),
            capi.Bcs.face_nv.offset, capi.Bcs.elem_source.offset, capi.Options.stream.offset,
            capi.Options.debug_withhold_barrier.offset, capi.Info.dt.offset, capi.Scenario.dt_scale.offset,
            C.sizeof(capi.EnergyParams), C.sizeof(capi.TilingStats), capi.TilingStats.n_shared_nodes.offset,
            capi.Options.quadrature.offset,
            C.sizeof(capi.DDInfo), capi.DDInfo.halo_entries.offset, capi.DDInfo.dt_crit.offset]
    assert got == want


def test_create_rejects_bad_input_without_gpu(lib_path):
    """Argument validation runs on the host before any device call."""
    import numpy as np

    import fedfem_inputs as fi
    from paper_1909_03355_gb300 import capi
    from paper_1909_03355_gb300.fedfem import FedFem
    p = fi.plain_cube(2)
    p.conn = p.conn.copy()
    p.conn[0, 0] = p.n_nodes + 5
    with pytest.raises(capi.FedFemError) as ei:
        FedFem(p)
    assert ei.value.name == "ERR_ARG" and "out of range" in str(ei.value)
    p = fi.nonlinear_cube(2)
    p.mats.append(fi.Material(1.0, np.eye(3), k_lin=0.5, c0=1.0))
    with pytest.raises(capi.FedFemError) as ei:
        FedFem(p)
    assert "share k_lin" in str(ei.value)
    with pytest.raises(capi.FedFemError) as ei:
        FedFem(fi.plain_cube(2), quadrature=4)
    assert ei.value.name == "ERR_ARG" and "quadrature" in str(ei.value)
    # empty inputs
    p = fi.plain_cube(2)
    p.conn = p.conn[:0]
    with pytest.raises(capi.FedFemError) as ei:
        FedFem(p)
    assert ei.value.name == "ERR_ARG" and "empty" in str(ei.value)
    p = fi.plain_cube(2)
    p.mats = []
    with pytest.raises(capi.FedFemError) as ei:
        FedFem(p)
    assert ei.value.name == "ERR_ARG"


def test_batch_rejects_schedules_and_tables_without_gpu():
    """Batched scenarios carry constant loads and the linear laws: a problem with a schedule or a
    property table is refused before any library call."""
    import numpy as np

    import fedfem_inputs as fi
    from paper_1909_03355_gb300.batch import FedFemBatch
    for field, value in (("q_schedule", np.ones(3)), ("Tinf_schedule", np.ones(3)),
                         ("Tdir_schedule", np.zeros(3)), ("table_T", np.array([0.0, 1.0]))):
        p = fi.nonlinear_cube(2, "hex")
        setattr(p, field, value)
        with pytest.raises(ValueError, match=field):
            FedFemBatch([fi.nonlinear_cube(2, "hex"), p])


def test_decomposition_rejects_bad_input_without_gpu(lib_path):
    """The domain decomposition validates its arguments on the host, and refuses schedules and
    property tables in the binding."""
    import numpy as np

    import fedfem_inputs as fi
    from paper_1909_03355_gb300 import capi, dd
    p = fi.plain_cube(2)
    for n_sub in (0, 9, 65):
        with pytest.raises(capi.FedFemError) as ei:
            dd.FedFemDD(p, n_sub)
        assert ei.value.name == "ERR_ARG"
    with pytest.raises(capi.FedFemError):
        dd.subdomain(p, 2, 2)
    q = fi.plain_cube(2)
    q.conn = q.conn.copy()
    q.conn[0, 0] = -1
    with pytest.raises(capi.FedFemError) as ei:
        dd.FedFemDD(q, 2)
    assert ei.value.name == "ERR_MESH"
    r = fi.nonlinear_cube(2, "hex")
    r.q_schedule = np.ones(3)
    with pytest.raises(ValueError, match="q_schedule"):
        dd.FedFemDD(r, 2)
