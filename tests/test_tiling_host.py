"""CPU-only checks of the tiling the step kernel runs on (fedfem_check_tiling: no device call).

The library builds the tiling on the host and checks every index the kernel will read before
any launch; these tests drive that code on structured, jittered, renumbered and tetrahedral
meshes, at tile counts from one to one element per tile, and through its error paths.
"""
import numpy as np
import pytest

import fedfem_inputs as fi


@pytest.fixture(scope="module")
def check():
    from paper_1909_03355_gb300 import build
    build.build()
    from paper_1909_03355_gb300.fedfem import check_tiling
    return check_tiling


def _renumbered(p, seed):
    """The same mesh with its node ids and element order permuted."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(p.n_nodes)          # new id of old node i
    inv = np.argsort(perm)
    p.xyz = p.xyz[inv]
    p.conn = perm[p.conn][rng.permutation(p.n_elems)].astype(np.int32)
    for f in ("conv_faces", "rad_faces"):
        if getattr(p, f) is not None:
            setattr(p, f, perm[getattr(p, f)].astype(np.int32))
    return p


@pytest.mark.parametrize("n_tiles", [1, 8, 37])
def test_structured_hex_cube(check, n_tiles):
    p = fi.nonlinear_cube(16, "hex")
    s = check(p, n_tiles)
    assert s["n_tiles"] == n_tiles
    assert s["n_colors_max"] == 8            # the parity colouring of a structured brick grid
    assert s["n_chunks"] * 32 == p.n_elems + s["n_padding_slots"]
    if n_tiles == 1:
        assert s["n_shared_nodes"] == 0 and s["n_halo_slots"] == 0
    else:
        assert s["n_shared_nodes"] > 0 and s["n_halo_slots"] >= 2 * s["n_shared_nodes"]


def test_jittered_renumbered_hex_keeps_eight_colours(check):
    """Node jitter and arbitrary node / element numbering change nothing: the tiles follow the
    element centroids, and the parity colouring of the quantised centroids stays proper."""
    a = check(fi.nonlinear_cube(12, "hex", jitter=0.25), 16)
    b = check(_renumbered(fi.nonlinear_cube(12, "hex", jitter=0.25), 7), 16)
    assert a["n_colors_max"] == b["n_colors_max"] == 8
    assert a["n_shared_nodes"] == b["n_shared_nodes"] and a["n_halo_slots"] == b["n_halo_slots"]


@pytest.mark.parametrize("chunk", [32, 64])
def test_tet_meshes(check, chunk):
    p = fi.nonlinear_cube(10, "tet")
    s = check(p, 12, chunk)
    assert s["n_chunks"] * chunk == p.n_elems + s["n_padding_slots"]
    assert 8 <= s["n_colors_max"] <= 64
    q = fi.paper_cube("tet", 19)
    assert check(q, 304)["n_tiles"] == 304


def test_tet_colouring_close_to_the_clique_bound(check):
    """The Kuhn-type 6-tet cube puts 24 tets on an interior node, so no colouring of a tile
    needs fewer than 24 classes; the tiling's saturation-degree candidate keeps the 64^3 cube's
    tiles within 28 (plain greedy orders needed 30), and the paper-shaped cube's within 24."""
    s = check(fi.nonlinear_cube(64, "tet"), 304, 64)
    assert 24 <= s["n_colors_max"] <= 28
    q = check(fi.paper_cube("tet", 19), 183, 64)
    assert q["n_colors_max"] <= 24


def test_one_element_per_tile(check):
    p = fi.nonlinear_cube(3, "hex")
    s = check(p, p.n_elems)
    assert s["n_tiles"] == p.n_elems and s["n_colors_max"] == 1
    assert s["n_padding_slots"] == p.n_elems * 31


def test_errors(check):
    from paper_1909_03355_gb300.capi import FedFemError
    p = fi.nonlinear_cube(4, "hex")
    with pytest.raises(FedFemError, match="chunk"):
        check(p, 4, chunk=48)
    with pytest.raises(FedFemError, match="n_tiles"):
        check(p, 0)
    bad = fi.nonlinear_cube(4, "hex")
    bad.conn = bad.conn.copy()
    bad.conn[5, 3] = bad.n_nodes
    with pytest.raises(FedFemError, match="out of range"):
        check(bad, 4)
    big = fi.nonlinear_cube(41, "hex")       # 74,088 nodes: more than a tile can number
    with pytest.raises(FedFemError, match="65535"):
        check(big, 1)
    assert check(big, 2)["n_tiles"] == 2


def test_mixed_element_orientation_still_colours_properly(check):
    """Hexahedra whose local node order is rotated about their z axis (same geometry, other
    face pairs): the lattice propagation over faces no longer agrees with itself, and the
    tiling falls back to the centroid pattern or greedy colourings, still checked proper."""
    p = fi.nonlinear_cube(10, "hex", jitter=0.2)
    c = p.conn.copy()
    c[::3] = c[::3][:, [1, 2, 3, 0, 5, 6, 7, 4]]
    p.conn = c
    s = check(p, 8)
    assert s["n_tiles"] == 8 and 8 <= s["n_colors_max"] <= 64


@pytest.mark.parametrize("case", ["hex", "hex_jitter", "tet", "paper_cube", "renumbered"])
@pytest.mark.parametrize("chunk", [32, 64])
def test_single_class_tiling_and_gather_lists(case, chunk, check):
    """The slot-gather tiling: one class per tile (padding only in a tile's last chunk), and
    gather lists that name every filled slot position exactly once, by its own node (checked
    by the library's validation, which rejects the tiling otherwise)."""
    if case == "hex":
        p = fi.nonlinear_cube(9, "hex")
    elif case == "hex_jitter":
        p = fi.nonlinear_cube(9, "hex", jitter=0.25)
    elif case == "tet":
        p = fi.nonlinear_cube(6, "tet")
    elif case == "paper_cube":
        p = fi.paper_cube("tet", 7)
    else:
        p = fi.nonlinear_cube(7, "hex")
        perm = np.random.default_rng(4).permutation(p.n_nodes)
        inv = np.empty_like(perm)
        inv[perm] = np.arange(p.n_nodes)
        p.xyz = p.xyz[perm]
        p.conn = inv[p.conn].astype(np.int32)
        p.conv_faces = inv[p.conv_faces].astype(np.int32) if p.conv_faces is not None else None
        p.rad_faces = inv[p.rad_faces].astype(np.int32) if p.rad_faces is not None else None
    for n_tiles in (1, 5, 23):
        st = check(p, n_tiles, chunk, single_class=True)
        assert st["n_colors_max"] == 1
        # one class per tile: at most one partly filled chunk per tile
        assert st["n_padding_slots"] < st["n_tiles"] * chunk
