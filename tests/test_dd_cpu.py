"""Domain decomposition on the CPU: the library's partition (host-only query) and the halo
exchange among gloo ranks.

Each rank takes one sub-domain of the library's plan (its slab's elements plus the ghost layer),
runs the FP64 oracle on it with the ghost nodes held fixed during a step, and after every step
receives the new ghost values from their owners and sends its own nodes that other ranks hold
as ghosts (point-to-point, ordered by global node id).  Every owned node then sees all of its
elements in ascending element order, as in the undecomposed oracle run, so the assembled field
must equal that run bitwise.
"""
import socket

import numpy as np
import pytest

import fedfem_inputs as fi


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(kind):
    if kind == "hex":
        return fi.nonlinear_cube(8, "hex", jitter=0.2)
    if kind == "tet":
        return fi.nonlinear_cube(5, "tet")
    p = fi.large_cube(7, jitter=0.15)            # conv + rad on all faces, plus a Dirichlet set
    bot = np.nonzero(p.xyz[:, 2] < 1e-12)[0].astype(np.int32)
    p.dir_nodes, p.dir_T = bot, np.full(len(bot), 150.0)
    p.nodal_Q = np.linspace(0.0, 0.3, p.n_nodes)
    return p


def sub_problem(p, el, nd, go):
    """The sub-domain's problem in local node ids (= positions in nd): its elements, the
    boundary faces whose nodes all belong to it, and the Dirichlet set extended by the ghosts
    (value placeholder 0; the exchange writes the real one)."""
    loc = -np.ones(p.n_nodes, np.int64)
    loc[nd] = np.arange(len(nd))

    def faces(f):
        if f is None or not len(f):
            return f
        keep = np.all(loc[f] >= 0, axis=1)
        return loc[f[keep]].astype(np.int32)

    isdir = np.zeros(p.n_nodes, bool)
    dT = np.zeros(p.n_nodes)
    if p.dir_nodes is not None and len(p.dir_nodes):
        isdir[p.dir_nodes] = True
        dT[p.dir_nodes] = p.dir_T
    held = isdir[nd] | (go >= 0)
    q = fi.Problem(name=p.name + "_sub", xyz=p.xyz[nd], conn=loc[p.conn[el]].astype(np.int32), mats=p.mats,
                   elem_kscale=None if p.elem_kscale is None else p.elem_kscale[el],
                   elem_source=None if p.elem_source is None else p.elem_source[el],
                   nodal_Q=None if p.nodal_Q is None else p.nodal_Q[nd],
                   dir_nodes=np.nonzero(held)[0].astype(np.int32), dir_T=np.where(isdir[nd], dT[nd], 0.0)[held],
                   conv_faces=faces(p.conv_faces), h=p.h, T_inf=p.T_inf, rad_faces=faces(p.rad_faces), eps=p.eps,
                   T_amb=p.T_amb, T_zero=p.T_zero, T0=p.initial_T()[nd], T_lo=p.T_lo, T_hi=p.T_hi)
    return q


@pytest.mark.parametrize("kind", ["hex", "tet", "bcs"])
@pytest.mark.parametrize("n_sub", [2, 3, 4])
def test_partition_properties(kind, n_sub):
    """Every node has one owner; a sub-domain holds every element that touches a node it owns;
    each ghost is owned by the sub-domain its owner field names; core slabs differ in size by
    at most one element."""
    from paper_1909_03355_gb300 import dd
    p = _problem(kind)
    owner = -np.ones(p.n_nodes, int)
    core = np.zeros(p.n_elems, int)
    subs = [dd.subdomain(p, n_sub, s) for s in range(n_sub)]
    for s, (el, nd, go) in enumerate(subs):
        assert np.all(np.diff(el) > 0) and np.all(np.diff(nd) > 0)
        own = nd[go < 0]
        assert np.all(owner[own] == -1)
        owner[own] = s
        # elements touching an owned node are all present
        touching = np.nonzero(np.isin(p.conn, own).any(axis=1))[0]
        assert np.all(np.isin(touching, el))
        # the nodes are exactly those of the elements
        assert np.array_equal(np.unique(p.conn[el]), nd)
        core[el] += 1
    assert np.all(owner >= 0)
    for s, (el, nd, go) in enumerate(subs):
        g = go >= 0
        assert np.all(owner[nd[g]] == go[g]) and np.all(go[g] != s)
    assert np.all(core >= 1)


def _worker(rank, world, port, kind, q):
    import torch
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_1909_03355_gb300 import dd
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        p = _problem(kind)
        dt = 0.9 * O.OracleModel(p).dt_crit()[0]
        subs = [dd.subdomain(p, world, s) for s in range(world)]
        el, nd, go = subs[rank]
        sp = sub_problem(p, el, nd, go)
        m = O.OracleModel(sp)
        # plan of this rank's messages: ghosts it receives from each owner, and its owned nodes
        # each other rank holds as ghosts (global ids ascending on both sides)
        recv = {o: np.nonzero(go == o)[0] for o in range(world) if o != rank and np.any(go == o)}
        send = {}
        for d in range(world):
            if d == rank:
                continue
            _, ndd, god = subs[d]
            g = ndd[god == rank]
            if len(g):
                send[d] = np.searchsorted(nd, g)
                assert np.array_equal(nd[send[d]], g)

        def exchange(T):
            reqs = [dist.isend(torch.from_numpy(np.ascontiguousarray(T[idx])), dst=d) for d, idx in send.items()]
            for o, idx in recv.items():
                buf = torch.empty(len(idx), dtype=torch.float64)
                dist.recv(buf, src=o)
                T[idx] = buf.numpy()
            for r in reqs:
                r.wait()

        T = p.initial_T()[nd].copy()
        if p.dir_nodes is not None and len(p.dir_nodes):
            isd = np.isin(nd, p.dir_nodes)
            T[isd] = sp.dir_T[np.searchsorted(sp.dir_nodes, np.nonzero(isd)[0])]
        exchange(T)
        for _ in range(40):
            T = m.run(T, dt, 1)
            exchange(T)
        q.put((rank, nd[go < 0], T[go < 0], dt, sum(len(v) for v in recv.values())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["hex", "tet", "bcs"])
def test_two_ranks_exchange_equals_undecomposed_oracle(kind):
    import torch.multiprocessing as mp

    from oracle import oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, kind, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    try:
        res = [q.get(timeout=240) for _ in range(2)]
    finally:
        for pr in procs:
            pr.join(timeout=60)
    assert [pr.exitcode for pr in procs] == [0, 0]
    p = _problem(kind)
    dt = res[0][3]
    ref = O.OracleModel(p).run(p.initial_T(), dt, 40)
    T = np.full(p.n_nodes, np.nan)
    for _, own, vals, _, n_recv in res:
        T[own] = vals
        assert n_recv > 0
    assert np.array_equal(T, ref)
