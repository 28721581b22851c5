"""Seeded synthetic inputs for FED-FEM transient heat-conduction problems.

This module is the only code shared between the FP64 CPU oracle (``oracle/``) and the CUDA
path (``paper_1909_03355_gb300``).  It builds the *problem statement* of Section 2 of the
paper (Eq. 1-7): a mesh of 8-node hexahedra (VTK / C3D8 node order) or 4-node tetrahedra,
material laws, initial temperature and the boundary sets Gamma_E (Dirichlet), Gamma_C
(convection), Gamma_R (radiation), plus volumetric and nodal heat sources.  It holds none of
the method's arithmetic: no shape functions, no quadrature, no element matrices, no lumping,
no time step.  Random numbers come from ``numpy.random.default_rng(seed)`` (PCG64).

The paper's own meshes (a 0.1 m cube of 40021 tets, plates, fin cooler, radiator) are not
published, so structured unit-cube meshes stand in for them; the workload recipes below
(cube sizes, laws, boundary sets, sources, step counts) define the synthetic benchmark
problems.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

# VTK hexahedron faces, each listed in cyclic order (used only to extract boundary quads).
_HEX_FACES = ((0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7))
_TET_FACES = ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1))
SIDES = ("x0", "x1", "y0", "y1", "z0", "z1")


@dataclasses.dataclass
class Material:
    """Thermal material: density rho, conductivity k(T) = k0 * (1 + k_lin*(T - T_ref)) with k0
    a 3x3 SPD tensor (Eq. 1, isotropic / orthotropic / anisotropic), and specific heat
    c(T) = c0 * (1 + c_lin*(T - T_ref)); k0 and c0 are the values at T_ref."""
    rho: float
    k0: np.ndarray
    k_lin: float = 0.0
    c0: float = 1.0
    c_lin: float = 0.0
    T_ref: float = 0.0


@dataclasses.dataclass
class Problem:
    """One transient heat-transfer problem (Eq. 1-7 of the paper), all arrays FP64 / int32."""
    name: str
    xyz: np.ndarray                      # [N,3] node coordinates (m)
    conn: np.ndarray                     # [E,npe] int32, hex in VTK order, tets positively oriented
    mats: List[Material]
    elem_mat: Optional[np.ndarray] = None       # [E] int32 material id, or None (all 0)
    elem_kscale: Optional[np.ndarray] = None    # [E] per-element conductivity scale theta_e
    elem_source: Optional[np.ndarray] = None    # [E] volumetric source (W/m^3)
    nodal_Q: Optional[np.ndarray] = None        # [N] concentrated nodal heat flow (W)
    dir_nodes: Optional[np.ndarray] = None      # [nd] int32 Dirichlet node ids
    dir_T: Optional[np.ndarray] = None          # [nd] prescribed temperatures
    conv_faces: Optional[np.ndarray] = None     # [nc, 4|3] int32 faces with convection
    h: float = 0.0
    T_inf: float = 0.0
    rad_faces: Optional[np.ndarray] = None      # [nr, 4|3] int32 faces with radiation
    eps: float = 0.0
    T_amb: float = 0.0
    T_zero: float = -273.15                     # absolute zero in the temperature unit (deg C)
    T0: Optional[np.ndarray] = None             # [N] initial temperature
    steps: int = 1
    T_lo: float = 0.0                           # temperature range used for the critical step
    T_hi: float = 0.0
    quadrature: int = 8                         # hexahedron conduction matrix: 8 = 2x2x2 Gauss,
                                                # 1 = one centre point (Eq. 17)
    kT_eval: int = 0                            # conductivity law: 0 = element mean of the nodal
                                                # factors (Section 4.2.2), 1 = at the quadrature points
    face_quadrature: int = 0                    # surface loads: 0 = nodal lumping of the face areas,
                                                # 1 = consistent integration over each face
    q_schedule: Optional[np.ndarray] = None     # [n] multiplier of the external loads at step n
    Tinf_schedule: Optional[np.ndarray] = None  # [n] convection ambient temperature at step n
    Tdir_schedule: Optional[np.ndarray] = None  # [n] offset added to every dir_T at step n
    # tabulated property factors (replace the materials' linear laws): f_k, f_c of k0, c0 at the
    # increasing temperatures table_T, linear between points, end values held outside
    table_T: Optional[np.ndarray] = None
    table_fk: Optional[np.ndarray] = None
    table_fc: Optional[np.ndarray] = None

    @property
    def npe(self) -> int:
        return int(self.conn.shape[1])

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.conn.shape[0])

    def free_mask(self) -> np.ndarray:
        m = np.ones(self.n_nodes, dtype=bool)
        if self.dir_nodes is not None:
            m[self.dir_nodes] = False
        return m

    def initial_T(self) -> np.ndarray:
        """T0 with the Dirichlet values imposed (initialisation stage, Fig. 1 (ii))."""
        T = np.array(self.T0, dtype=np.float64, copy=True)
        if self.dir_nodes is not None and len(self.dir_nodes):
            T[self.dir_nodes] = self.dir_T
        return T


# ----------------------------------------------------------------------------------------------
# Meshes
# ----------------------------------------------------------------------------------------------

def grid_nodes(nx: int, ny: int, nz: int, L=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Nodes of a structured nx*ny*nz brick grid; node id = i + (nx+1)*(j + (ny+1)*k)."""
    x = origin[0] + np.linspace(0.0, L[0], nx + 1)
    y = origin[1] + np.linspace(0.0, L[1], ny + 1)
    z = origin[2] + np.linspace(0.0, L[2], nz + 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def _nid(i, j, k, nx, ny):
    return i + (nx + 1) * (j + (ny + 1) * k)


def grid_hex_conn(nx: int, ny: int, nz: int) -> np.ndarray:
    """8-node bricks in VTK order: bottom face counter-clockwise, then the top face."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    c = [_nid(i, j, k, nx, ny), _nid(i + 1, j, k, nx, ny), _nid(i + 1, j + 1, k, nx, ny),
         _nid(i, j + 1, k, nx, ny), _nid(i, j, k + 1, nx, ny), _nid(i + 1, j, k + 1, nx, ny),
         _nid(i + 1, j + 1, k + 1, nx, ny), _nid(i, j + 1, k + 1, nx, ny)]
    return np.stack(c, axis=1).astype(np.int32)


def grid_tet_conn(nx: int, ny: int, nz: int) -> np.ndarray:
    """Kuhn split of every brick into 6 tets along its (0,0,0)->(1,1,1) diagonal: for each
    permutation (a,b,c) of the axes the tet v0, v0+e_a, v0+e_a+e_b, v0+e_a+e_b+e_c.  The split
    is conforming because every cell uses the same orientation."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    tets = []
    perms = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
    for p in perms:
        off = np.zeros(3, dtype=np.int64)
        verts = [_nid(i, j, k, nx, ny)]
        for ax in p:
            off[ax] += 1
            verts.append(_nid(i + off[0], j + off[1], k + off[2], nx, ny))
        tets.append(np.stack(verts, axis=1))
    # interleave so that the 6 tets of a cell are consecutive
    t = np.stack(tets, axis=1).reshape(-1, 4)
    return t.astype(np.int32)


def orient_tets(xyz: np.ndarray, conn: np.ndarray) -> np.ndarray:
    """Swap two vertices of every tet whose signed volume is negative (mesh generation)."""
    p = xyz[conn]
    d = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])
    conn = conn.copy()
    neg = d < 0
    conn[neg, 1], conn[neg, 2] = conn[neg, 2].copy(), conn[neg, 1].copy()
    return conn


def boundary_faces(conn: np.ndarray) -> np.ndarray:
    """Faces that belong to exactly one element, each in the element's cyclic order."""
    npe = conn.shape[1]
    local = _HEX_FACES if npe == 8 else _TET_FACES
    faces = np.concatenate([conn[:, list(f)] for f in local], axis=0)
    key = np.sort(faces, axis=1)
    order = np.lexsort(key.T[::-1])
    ks = key[order]
    same_prev = np.r_[False, np.all(ks[1:] == ks[:-1], axis=1)]
    same_next = np.r_[np.all(ks[1:] == ks[:-1], axis=1), False]
    single = ~(same_prev | same_next)
    return faces[order[single]].astype(np.int32)


def faces_on_side(xyz: np.ndarray, faces: np.ndarray, side: str, tol: float = 1e-9) -> np.ndarray:
    """Boundary faces whose nodes all lie on one side of the bounding box."""
    ax = "xyz".index(side[0])
    lo = xyz[:, ax].min()
    hi = xyz[:, ax].max()
    v = lo if side[1] == "0" else hi
    on = np.all(np.abs(xyz[faces, ax] - v) <= tol * max(1.0, abs(hi - lo)), axis=1)
    return faces[on]


def boundary_node_ids(faces: np.ndarray) -> np.ndarray:
    return np.unique(faces.ravel()).astype(np.int32)


def jitter_interior(xyz: np.ndarray, h: float, amount: float, rng) -> np.ndarray:
    """Move strictly interior nodes by U[-amount*h, amount*h] per axis (structure-free meshes)."""
    lo, hi = xyz.min(axis=0), xyz.max(axis=0)
    tol = 1e-9
    interior = np.all((xyz > lo + tol) & (xyz < hi - tol), axis=1)
    out = xyz.copy()
    out[interior] += rng.uniform(-amount * h, amount * h, size=(int(interior.sum()), 3))
    return out


def cube_mesh(n: int, kind: str = "hex", L: float = 1.0, jitter: float = 0.0, seed: int = 0):
    """Unit (or L-sized) cube meshed with n^3 bricks, or their 6-tet Kuhn split."""
    xyz = grid_nodes(n, n, n, (L, L, L))
    if jitter > 0:
        xyz = jitter_interior(xyz, L / n, jitter, np.random.default_rng(seed + 1000))
    if kind == "hex":
        conn = grid_hex_conn(n, n, n)
    elif kind == "tet":
        conn = orient_tets(xyz, grid_tet_conn(n, n, n))
    else:
        raise ValueError(kind)
    return xyz, conn


def random_spd(rng, lo: float = 0.5, hi: float = 5.0) -> np.ndarray:
    """k0 = Q diag(lambda) Q^T with Q from the QR of a 3x3 normal matrix (sign-fixed) and
    eigenvalues uniform in [lo, hi]."""
    A = rng.standard_normal((3, 3))
    Q, R = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(R))[None, :]
    lam = rng.uniform(lo, hi, size=3)
    k = (Q * lam[None, :]) @ Q.T
    return 0.5 * (k + k.T)


def centroids(xyz: np.ndarray, conn: np.ndarray) -> np.ndarray:
    return xyz[conn].mean(axis=1)


def box_source(xyz, conn, lo, hi, value) -> np.ndarray:
    """Volumetric source `value` (W/m^3) on elements whose centroid lies in the box [lo, hi]."""
    c = centroids(xyz, conn)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    m = np.all((c >= lo - 1e-12) & (c <= hi + 1e-12), axis=1)
    s = np.zeros(conn.shape[0])
    s[m] = value
    return s


# ----------------------------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------------------------

def plain_cube(n: int = 10, steps: int = 1000) -> Problem:
    """Plain linear FED-FEM workload: unit cube of n^3 bricks, isotropic k = 1, rho = c = 1,
    T0 = 100 everywhere, T = 0 held on all six faces."""
    xyz, conn = cube_mesh(n, "hex")
    bf = boundary_faces(conn)
    dn = boundary_node_ids(bf)
    return Problem(name=f"plain_cube_{n}", xyz=xyz, conn=conn,
                   mats=[Material(rho=1.0, k0=np.eye(3), c0=1.0)],
                   dir_nodes=dn, dir_T=np.zeros(len(dn)),
                   T0=np.full(xyz.shape[0], 100.0), steps=steps, T_lo=0.0, T_hi=100.0)


def nonlinear_cube(n: int = 64, kind: str = "hex", seed: int = 2, steps: int = 5000,
                   jitter: float = 0.0) -> Problem:
    """Nonlinear anisotropic cube: k(T) = k0 (1 + 0.002 T) with k0 random SPD (eigenvalues in
    [0.5, 5]), c(T) = 500 (1 + 0.001 T), rho = 2700, convection h = 25, T_inf = 20 on z = 1,
    radiation eps = 0.8 (ambient 20) on the four side faces, 1e5 W/m^3 in the central 1/8,
    T0 = 20."""
    rng = np.random.default_rng(seed)
    k0 = random_spd(rng)
    xyz, conn = cube_mesh(n, kind, jitter=jitter, seed=seed)
    bf = boundary_faces(conn)
    conv = faces_on_side(xyz, bf, "z1")
    rad = np.concatenate([faces_on_side(xyz, bf, s) for s in ("x0", "x1", "y0", "y1")])
    src = box_source(xyz, conn, (0.25,) * 3, (0.75,) * 3, 1e5)
    return Problem(name=f"nonlinear_{kind}_{n}", xyz=xyz, conn=conn,
                   mats=[Material(rho=2700.0, k0=k0, k_lin=0.002, c0=500.0, c_lin=0.001)],
                   elem_source=src, conv_faces=conv, h=25.0, T_inf=20.0,
                   rad_faces=rad, eps=0.8, T_amb=20.0,
                   T0=np.full(xyz.shape[0], 20.0), steps=steps, T_lo=20.0, T_hi=1000.0)


def large_cube(n: int = 128, seed: int = 3, steps: int = 20000, jitter: float = 0.0,
               kind: str = "hex") -> Problem:
    """Large explicit run: n^3 bricks, orthotropic k = diag(1, 5, 20) (1 + 0.002 T),
    c(T) = 500 (1 + 0.001 T), rho = 2700, convection (h = 25, T_inf = 20) and radiation
    (eps = 0.8, ambient 20) on all six faces, 1e5 W/m^3 in the central 1/8, T0 = 20."""
    xyz, conn = cube_mesh(n, kind, jitter=jitter, seed=seed)
    bf = boundary_faces(conn)
    src = box_source(xyz, conn, (0.25,) * 3, (0.75,) * 3, 1e5)
    return Problem(name=f"large_{kind}_{n}", xyz=xyz, conn=conn,
                   mats=[Material(rho=2700.0, k0=np.diag([1.0, 5.0, 20.0]), k_lin=0.002,
                                  c0=500.0, c_lin=0.001)],
                   elem_source=src, conv_faces=bf, h=25.0, T_inf=20.0,
                   rad_faces=bf, eps=0.8, T_amb=20.0,
                   T0=np.full(xyz.shape[0], 20.0), steps=steps, T_lo=20.0, T_hi=1000.0)


def batched_scenarios(S: int = 256, seed: int = 4, n_lo: int = 8, n_hi: int = 48,
                      steps_lo: int = 500, steps_hi: int = 5000) -> List[Problem]:
    """S independent cubes: n ~ U{n_lo..n_hi} bricks per edge, random SPD k0, h ~ U[5, 100],
    eps ~ U[0.1, 0.9], a 1e5 W/m^3 source sub-cube of side 1/2 whose corner ~ U[0, 1/2]^3 is
    snapped to the grid, steps ~ U{steps_lo..steps_hi}; convection on top, radiation on the
    four sides, bottom adiabatic, laws as the nonlinear cube."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(S):
        n = int(rng.integers(n_lo, n_hi + 1))
        k0 = random_spd(rng)
        h = float(rng.uniform(5.0, 100.0))
        eps = float(rng.uniform(0.1, 0.9))
        corner = np.floor(rng.uniform(0.0, 0.5, size=3) * n) / n
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        xyz, conn = cube_mesh(n, "hex")
        bf = boundary_faces(conn)
        conv = faces_on_side(xyz, bf, "z1")
        rad = np.concatenate([faces_on_side(xyz, bf, sd) for sd in ("x0", "x1", "y0", "y1")])
        src = box_source(xyz, conn, corner, corner + 0.5, 1e5)
        out.append(Problem(name=f"scenario_{s}_n{n}", xyz=xyz, conn=conn,
                           mats=[Material(rho=2700.0, k0=k0, k_lin=0.002, c0=500.0, c_lin=0.001)],
                           elem_source=src, conv_faces=conv, h=h, T_inf=20.0,
                           rad_faces=rad, eps=eps, T_amb=20.0,
                           T0=np.full(xyz.shape[0], 20.0), steps=steps, T_lo=20.0, T_hi=1000.0))
    return out


@dataclasses.dataclass
class InverseSetup:
    problem: Problem
    theta_true: np.ndarray      # [E] ground-truth conductivity scales
    sensors: np.ndarray         # [n_sensors] int32 interior node ids
    sample_every: int
    ckpt_every: int


def inverse_problem(n: int = 32, seed: int = 5, steps: int = 2000, n_sensors: int = 512,
                    sample_every: int = 10, ckpt_every: int = 100) -> InverseSetup:
    """Differentiable inverse problem: n^3 bricks with the nonlinear-cube laws, convection on
    top only (other faces adiabatic, no Dirichlet set), 1e5 W/m^3 in the central 1/8, T0 = 20.
    Ground truth: per-element conductivity scale lognormal(0, 0.3); guess theta = 1.  Sensors:
    distinct random interior nodes; samples every `sample_every` steps."""
    rng = np.random.default_rng(seed)
    k0 = random_spd(rng)
    xyz, conn = cube_mesh(n, "hex")
    bf = boundary_faces(conn)
    conv = faces_on_side(xyz, bf, "z1")
    src = box_source(xyz, conn, (0.25,) * 3, (0.75,) * 3, 1e5)
    theta_true = np.exp(0.3 * rng.standard_normal(conn.shape[0]))
    bnd = np.zeros(xyz.shape[0], dtype=bool)
    bnd[boundary_node_ids(bf)] = True
    interior = np.nonzero(~bnd)[0]
    sensors = np.sort(rng.choice(interior, size=min(n_sensors, len(interior)), replace=False))
    p = Problem(name=f"inverse_{n}", xyz=xyz, conn=conn,
                mats=[Material(rho=2700.0, k0=k0, k_lin=0.002, c0=500.0, c_lin=0.001)],
                elem_source=src, elem_kscale=np.ones(conn.shape[0]),
                conv_faces=conv, h=25.0, T_inf=20.0,
                T0=np.full(xyz.shape[0], 20.0), steps=steps, T_lo=20.0, T_hi=1000.0)
    return InverseSetup(p, theta_true, sensors.astype(np.int32), sample_every, ckpt_every)


def slab(nx: int, ny: int = 1, nz: int = 1, Lx: float = 1.0, k=(1.0, 1.0, 1.0), rho: float = 1.0,
         c0: float = 1.0, k_lin: float = 0.0, c_lin: float = 0.0, T0: float = 0.0,
         T_s: float = 1.0, steps: int = 100, conv_end: Optional[tuple] = None) -> Problem:
    """Bar of nx*ny*nz bricks of edge h = Lx/nx (cross-section ny*h by nz*h): T = T_s held at
    x = 0, adiabatic elsewhere (optionally convection (h, T_inf) on the x = Lx end face);
    orthotropic k = diag(k)."""
    h = Lx / nx
    xyz = grid_nodes(nx, ny, nz, (Lx, ny * h, nz * h))
    conn = grid_hex_conn(nx, ny, nz)
    dn = np.nonzero(np.abs(xyz[:, 0]) < 1e-12)[0].astype(np.int32)
    p = Problem(name=f"slab_{nx}x{ny}x{nz}", xyz=xyz, conn=conn,
                mats=[Material(rho=rho, k0=np.diag(np.asarray(k, float)), k_lin=k_lin,
                               c0=c0, c_lin=c_lin)],
                dir_nodes=dn, dir_T=np.full(len(dn), T_s), T0=np.full(xyz.shape[0], T0),
                steps=steps, T_lo=min(T0, T_s), T_hi=max(T0, T_s))
    if conv_end is not None:
        bf = boundary_faces(conn)
        p.conv_faces = faces_on_side(xyz, bf, "x1")
        p.h, p.T_inf = float(conv_end[0]), float(conv_end[1])
    return p


def single_brick(a: float = 1.0, b: float = 1.0, c: float = 1.0, rho: float = 1.0,
                 c0: float = 1.0, c_lin: float = 0.0, T0: float = 100.0, conv=None, rad=None,
                 steps: int = 10) -> Problem:
    """One a*b*c brick with convection (h, T_inf) and / or radiation (eps, T_amb) on all six
    faces; used for single-node lumped-ODE checks of the surface loads."""
    xyz = grid_nodes(1, 1, 1, (a, b, c))
    conn = grid_hex_conn(1, 1, 1)
    bf = boundary_faces(conn)
    p = Problem(name="brick", xyz=xyz, conn=conn,
                mats=[Material(rho=rho, k0=np.eye(3), c0=c0, c_lin=c_lin)],
                T0=np.full(8, T0), steps=steps, T_lo=-50.0, T_hi=max(T0, 100.0))
    if conv is not None:
        p.conv_faces, p.h, p.T_inf = bf, float(conv[0]), float(conv[1])
    if rad is not None:
        p.rad_faces, p.eps, p.T_amb = bf, float(rad[0]), float(rad[1])
    return p


def patch_hex_mesh(coords: np.ndarray):
    """The 7-element hexahedral patch of Fig. 2(a): an inner distorted hex (nodes 9-16) plus
    one hex per face of the unit cube (nodes 1-8), returned with 0-based ids.  `coords` is the
    16x3 node table of Fig. 2(c).  Corner / inner correspondences: 9-1, 10-2, 11-4, 12-3,
    13-5, 14-6, 15-8, 16-7 (1-based)."""
    # inner hex in VTK order (1-based ids from the table)
    inner = [9, 10, 11, 12, 13, 14, 15, 16]
    outer = [1, 2, 4, 3, 5, 6, 8, 7]          # cube corner matching each inner vertex
    conn = [inner]
    for f in _HEX_FACES:
        conn.append([outer[i] for i in f] + [inner[i] for i in f])
    conn = np.asarray(conn, dtype=np.int64) - 1
    xyz = np.asarray(coords, dtype=np.float64)
    # orient each hex so that the signed volume of its corner tetrahedron at node 0 is
    # positive (mesh generation: swap bottom/top quads when inverted)
    for e in range(conn.shape[0]):
        p = xyz[conn[e]]
        vol = np.dot(np.cross(p[1] - p[0], p[3] - p[0]), p[4] - p[0])
        if vol < 0:
            conn[e] = np.r_[conn[e][4:], conn[e][:4]]
    return xyz, conn.astype(np.int32)


def patch_tet_mesh(coords: np.ndarray):
    """A conforming tetrahedralisation of the 16 patch-test points of Fig. 2(c) (Delaunay;
    the paper's own tet connectivity is printed only as a figure)."""
    from scipy.spatial import Delaunay
    xyz = np.asarray(coords, dtype=np.float64)
    tri = Delaunay(xyz)
    conn = orient_tets(xyz, tri.simplices.astype(np.int32))
    return xyz, conn


def patch_problem(coords: np.ndarray, kind: str = "hex", field=(200.0, 100.0, 200.0),
                  k0=None, steps: int = 1) -> Problem:
    """Patch test of Section 4.1: T = 200x + 100y + 200z prescribed on the 8 cube corners,
    interior nodes free, starting from T = 0 inside."""
    xyz, conn = patch_hex_mesh(coords) if kind == "hex" else patch_tet_mesh(coords)
    lin = xyz @ np.asarray(field, float)
    corner = np.nonzero(np.all((np.abs(xyz) < 1e-12) | (np.abs(xyz - 1) < 1e-12), axis=1))[0]
    T0 = np.zeros(xyz.shape[0])
    return Problem(name=f"patch_{kind}", xyz=xyz, conn=conn,
                   mats=[Material(rho=1.0, k0=np.eye(3) if k0 is None else np.asarray(k0), c0=1.0)],
                   dir_nodes=corner.astype(np.int32), dir_T=lin[corner], T0=T0, steps=steps,
                   T_lo=0.0, T_hi=float(lin.max()))


def two_point_law(T1: float, v1: float, T2: float, v2: float):
    """(lin, T_ref) of the law v(T) = v1 (1 + lin (T - T_ref)) through (T1, v1) and (T2, v2):
    linear interpolation between two tabulated points (Section 4.2.2)."""
    return (v2 / v1 - 1.0) / (T2 - T1), T1


def paper_cube(kind: str = "tet", n: int = 19, L: float = 0.1, k="iso", steps: int = 2000,
               td: bool = False) -> Problem:
    """Stand-in for the paper's 0.1 m cube (Section 4.2.1): n^3 cells (x6 tets), k = 200
    (iso), 300/400/200 (ortho) or the anisotropic tensor of Section 4.2.1, rho = 1000,
    c = 2000, T0 = 37, T = 37 held on the back face (y = L), 0.2 W on every node of the front,
    top and two side faces, bottom adiabatic.  td: the temperature-dependent laws the paper
    tabulates in Section 4.2.2 (k = 200 at 37 and 2000 at 337, c = 2000 at 37 and 8000 at 337,
    linear in between), with k scaled for the ortho / aniso tensors."""
    xyz, conn = cube_mesh(n, kind, L=L)
    if k == "iso":
        k0 = 200.0 * np.eye(3)
    elif k == "ortho":
        k0 = np.diag([300.0, 400.0, 200.0])
    else:
        k0 = np.array([[200.0, 50.0, 50.0], [50.0, 300.0, 50.0], [50.0, 50.0, 400.0]])
    bf = boundary_faces(conn)
    back = boundary_node_ids(faces_on_side(xyz, bf, "y1"))
    loaded = np.unique(np.concatenate([boundary_node_ids(faces_on_side(xyz, bf, s))
                                       for s in ("y0", "z1", "x0", "x1")]))
    nq = np.zeros(xyz.shape[0])
    nq[loaded] = 0.2
    nq[back] = 0.0
    k_lin, T_ref = two_point_law(37.0, 200.0, 337.0, 2000.0) if td else (0.0, 0.0)
    c_lin, _ = two_point_law(37.0, 2000.0, 337.0, 8000.0) if td else (0.0, 0.0)
    return Problem(name=f"paper_cube_{kind}_{n}{'_td' if td else ''}", xyz=xyz, conn=conn,
                   mats=[Material(rho=1000.0, k0=k0, k_lin=k_lin, c0=2000.0, c_lin=c_lin, T_ref=T_ref)],
                   nodal_Q=nq,
                   dir_nodes=back, dir_T=np.full(len(back), 37.0),
                   T0=np.full(xyz.shape[0], 37.0), steps=steps, T_lo=37.0, T_hi=100.0)


def random_state(p: Problem, seed: int, lo: float = 20.0, hi: float = 400.0) -> np.ndarray:
    """A seeded random temperature field (Dirichlet values imposed) for one-step checks."""
    rng = np.random.default_rng(seed)
    T = rng.uniform(lo, hi, size=p.n_nodes)
    if p.dir_nodes is not None and len(p.dir_nodes):
        T[p.dir_nodes] = p.dir_T
    return T


def save_npz(p: Problem, path: str) -> None:
    d = {k: v for k, v in dataclasses.asdict(p).items() if k != "mats" and v is not None}
    for i, m in enumerate(p.mats):
        d[f"mat{i}_rho"], d[f"mat{i}_k0"] = m.rho, m.k0
        d[f"mat{i}_k_lin"], d[f"mat{i}_c0"], d[f"mat{i}_c_lin"] = m.k_lin, m.c0, m.c_lin
        d[f"mat{i}_T_ref"] = m.T_ref
    d["n_mats"] = len(p.mats)
    np.savez(path, **d)


def load_npz(path: str) -> Problem:
    z = np.load(path, allow_pickle=False)
    mats = [Material(float(z[f"mat{i}_rho"]), z[f"mat{i}_k0"], float(z[f"mat{i}_k_lin"]),
                     float(z[f"mat{i}_c0"]), float(z[f"mat{i}_c_lin"]),
                     float(z[f"mat{i}_T_ref"]) if f"mat{i}_T_ref" in z.files else 0.0)
            for i in range(int(z["n_mats"]))]
    kw = {}
    for f in dataclasses.fields(Problem):
        if f.name == "mats":
            continue
        if f.name in z.files:
            v = z[f.name]
            kw[f.name] = v.item() if v.ndim == 0 and f.name not in ("xyz",) else v
    kw["name"] = str(kw["name"])
    return Problem(mats=mats, **kw)
