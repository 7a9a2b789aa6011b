"""Partitioned runs on CPU ranks (gloo): the element decomposition the library's partition
groups use, run with the oracle's DG operator as each rank's local operator.

Each rank takes its own elements and one-element halo from the library's host partitioner
(``pcexp_partition`` / ``pcexp_partition_halo``), builds the submesh of those elements (halo
faces with no partner in it become symmetry planes: their rows are discarded) and runs the
partitioned algorithm of the library's group steps:

* every operator pass (R(u), J v) first replaces the halo rows of its input by the owners' rows
  (exchange), and its output keeps only the own rows (zero halo rows);
* the Arnoldi process is classical Gram-Schmidt with one re-orthogonalisation (two passes), each
  pass summing its j + 2 inner products over the ranks (one allreduce per pass), on vectors with
  zero halo rows;
* phi_1 of the Hessenberg matrix (every rank holds the same) is the oracle's.

The assembled results equal the oracle's on the whole mesh (one rank) to round-off: the
residual and J v exactly up to the order of the face-point sums, the Hessenberg matrix and one
PCEXP step (Eq. s9, s10) within 1e-12 relative.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import workloads as W  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(name):
    if name == "vortex2d":
        mesh = W.periodic_square(8, 10.0, 0.15, 3)
        return mesh, 1, W.Freestream(0.5, 45.0), 0.05, 8
    if name == "bump2d":
        mesh = W.bump_channel(12, 4, 0.1, 2)
        return mesh, 2, W.Freestream(0.5, 0.0), 0.02, 8
    if name == "cube3d":
        mesh = W.periodic_cube_kuhn(3, 2.0, 0.1, 4)
        return mesh, 1, W.Freestream(0.5, 30.0), 0.05, 6
    raise ValueError(name)


def _state(dg, seed):
    u = np.zeros((dg.E, dg.nv, dg.N))
    u[:, :, 0] = dg.freestream_state()[None, :] * np.sqrt(dg.area)[:, None]
    return u + 0.05 * W.random_coeffs(seed, u.shape) * np.abs(u[:, :, :1])


def submesh(mesh, own, halo):
    """Mesh of the elements own + halo in increasing global index (so that every face keeps the
    whole mesh's L element, whose face points it uses), written here from the mesh alone.
    Returns (submesh, global index of each local element)."""
    D = mesh.dim
    el = np.sort(np.concatenate([own, halo]))
    is_own = np.isin(el, own)
    ev = mesh.elems[el]
    verts = np.unique(np.concatenate([ev.ravel(), mesh.vert_master[ev.ravel()]]))
    elems = np.searchsorted(verts, ev).astype(np.int32)
    master = np.searchsorted(verts, mesh.vert_master[verts]).astype(np.int32)
    # faces match on master vertices; tags are looked up by an element's own face vertices
    count, own_key = {}, {}
    for le, e in enumerate(el):
        for f in range(D + 1):
            vs = [int(mesh.elems[e, (f + 1 + k) % (D + 1)]) for k in range(D)]
            key = tuple(sorted(int(mesh.vert_master[v]) for v in vs))
            count.setdefault(key, []).append((le, tuple(sorted(vs))))
            own_key[tuple(sorted(vs))] = key
    bf, bt, tagged = [], [], set()
    for vs, t in zip(mesh.bfaces, mesh.btags):
        key = tuple(sorted(int(v) for v in vs))
        if key in own_key:
            tagged.add(own_key[key])
            bf.append(np.searchsorted(verts, vs))
            bt.append(int(t))
    for key, users in sorted(count.items()):
        if len(users) == 1 and key not in tagged:
            le, vs = users[0]
            assert not is_own[le], "an own element's face has no partner and no tag"
            bf.append(np.searchsorted(verts, np.array(vs)))
            bt.append(3)  # symmetry plane
    return W.Mesh(D, mesh.coords[verts], elems, master, np.array(bf, np.int32).reshape(-1, D),
                  np.array(bt, np.int32)), el


def _rank(rank, world, port, name, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = _partitioned(rank, world, name)
    finally:
        dist.destroy_process_group()


def _partitioned(rank, world, name):
    from oracle.dg import DGOracle
    from oracle.krylov import phi_e1
    from paper_1801_06300_gb300 import capi

    mesh, p, free, dt, m = _case(name)
    part = capi.partition(mesh, world)
    own, halo = capi.partition_halo(mesh, part, rank)
    sub, el = submesh(mesh, own, halo)
    dg = DGOracle(sub, p, free)
    gdg = DGOracle(mesh, p, free)  # only for the global shapes and the seeded inputs
    E, shape = mesh.n_elem, (gdg.nv, gdg.N)
    mine = np.isin(el, own)

    def allsum(a):
        t = torch.from_numpy(np.ascontiguousarray(a, np.float64).copy())
        dist.all_reduce(t)
        return t.numpy()

    def local(gv):
        return gv[el].copy()

    def assemble(x):
        g = np.zeros((E,) + shape)
        g[el[mine]] = x[mine]
        return allsum(g)

    def exchange(x):
        x = x.copy()
        x[~mine] = assemble(x)[el[~mine]]
        return x

    def own_rows(x):
        x = x.copy()
        x[~mine] = 0.0
        return x

    def R(u):
        return own_rows(dg.residual(exchange(u)))

    def J(u, v):
        return own_rows(dg.jvp(exchange(u), exchange(v)))

    def dot(a, b):
        return float(allsum(np.array([np.sum(a * b)]))[0])

    def arnoldi(mv, b):
        # classical Gram-Schmidt, two passes, one sum over the ranks per pass
        beta = np.sqrt(dot(b, b))
        V = [b / beta]
        H = np.zeros((m + 1, m))
        for j in range(m):
            w = mv(V[j])
            s = allsum(np.array([np.sum(V[i] * w) for i in range(j + 1)] + [np.sum(w * w)]))
            w0 = np.sqrt(s[j + 1])
            h = s[: j + 1]
            w = w - sum(h[i] * V[i] for i in range(j + 1))
            h2 = allsum(np.array([np.sum(V[i] * w) for i in range(j + 1)]))
            w = w - sum(h2[i] * V[i] for i in range(j + 1))
            H[: j + 1, j] = h + h2
            hn = np.sqrt(dot(w, w))
            H[j + 1, j] = hn
            assert hn > 1e-12 * w0  # no breakdown in these cases
            V.append(w / hn)
        return V, H, beta

    def phi1(mv, b):
        V, H, beta = arnoldi(mv, b)
        y, _ = phi_e1(H[:m, :m], dt)
        return beta * sum(y[i] * V[i] for i in range(m)), H, beta

    u = own_rows(local(_state(gdg, 11)))
    v = own_rows(local(W.random_coeffs(12, (E,) + shape)))
    res = dict(R=assemble(R(u)), Jv=assemble(J(u, v)), own=own, halo=halo)
    _, H, beta = arnoldi(lambda x: J(u, x), own_rows(local(W.random_coeffs(13, (E,) + shape))))
    res.update(H=H, beta=beta)
    # one PCEXP step
    Rn = R(u)
    x1, _, _ = phi1(lambda x: J(u, x), Rn)
    us = u + dt * x1
    d = R(us) - Rn - J(u, us - u)
    x2, _, _ = phi1(lambda x: J(u, x), d)
    res["step"] = assemble(us + 0.5 * dt * x2)
    return res


def _run(world, name):
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, name, out), nprocs=world, join=True)
        return dict(out)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("world,name", [(2, "vortex2d"), (3, "bump2d"), (2, "cube3d")])
def test_partitioned_ranks_equal_one_rank(world, name):
    from oracle import krylov, pcexp
    from oracle.dg import DGOracle

    res = _run(world, name)
    assert sorted(res) == list(range(world))
    mesh, p, free, dt, m = _case(name)
    # own elements of the ranks tile the mesh; halos are other ranks' elements
    own = np.concatenate([res[r]["own"] for r in range(world)])
    assert np.array_equal(np.sort(own), np.arange(mesh.n_elem))
    for r in range(world):
        assert len(res[r]["halo"]) > 0 and not np.isin(res[r]["halo"], res[r]["own"]).any()
    dg = DGOracle(mesh, p, free)
    u = _state(dg, 11)
    v = W.random_coeffs(12, u.shape)
    b = W.random_coeffs(13, u.shape)
    R = dg.residual(u)
    Jv = dg.jvp(u, v)
    for r in range(world):
        assert _rel(res[r]["R"], R) <= 1e-13
        assert _rel(res[r]["Jv"], Jv) <= 1e-13
    _, Hb, k, beta, _ = krylov.arnoldi(lambda x: dg.jvp(u, x.reshape(u.shape)).reshape(-1), b.reshape(-1), m)
    assert k == m
    for r in range(world):
        assert np.abs(res[r]["H"] - Hb).max() <= 1e-12 * np.abs(Hb).max()
        assert abs(res[r]["beta"] - beta) <= 1e-14 * beta
        # every rank holds the same Hessenberg matrix
        assert np.array_equal(res[r]["H"], res[0]["H"])
    flat = lambda x: dg.residual(x.reshape(u.shape)).reshape(-1)  # noqa: E731
    jv = lambda a, x: dg.jvp(a.reshape(u.shape), x.reshape(u.shape)).reshape(-1)  # noqa: E731
    un1, _ = pcexp.pcexp_step(u.reshape(-1), flat, jv, dt, m)
    assert _rel(un1 - u.reshape(-1), un1) > 1e-6  # the step moves the state
    for r in range(world):
        assert _rel(res[r]["step"], un1) <= 1e-12


def _adjacency(mesh):
    """Face neighbours by brute force over master-vertex sets."""
    D = mesh.dim
    faces = {}
    for e in range(mesh.n_elem):
        for f in range(D + 1):
            key = tuple(sorted(int(mesh.vert_master[mesh.elems[e, (f + 1 + k) % (D + 1)]]) for k in range(D)))
            faces.setdefault(key, []).append(e)
    nbr = [set() for _ in range(mesh.n_elem)]
    for lst in faces.values():
        if len(lst) == 2:
            nbr[lst[0]].add(lst[1])
            nbr[lst[1]].add(lst[0])
    return nbr


@pytest.mark.parametrize("n_parts", [1, 2, 3, 5, 8])
def test_library_partition_and_halo(n_parts):
    from paper_1801_06300_gb300 import capi

    mesh = W.periodic_cube_kuhn(3, 1.0, 0.1, 7) if n_parts % 2 else W.bump_channel(16, 6, 0.1, 3)
    part = capi.partition(mesh, n_parts)
    sizes = np.bincount(part, minlength=n_parts)
    assert len(sizes) == n_parts and sizes.min() >= mesh.n_elem // n_parts - 2 and sizes.max() - sizes.min() <= 3
    nbr = _adjacency(mesh)
    for k in range(n_parts):
        own, halo = capi.partition_halo(mesh, part, k)
        assert np.array_equal(own, np.flatnonzero(part == k))
        expect = sorted({n for e in own for n in nbr[e] if part[n] != k})
        assert list(halo) == expect


def test_bisection_splits_along_the_longest_axis():
    from paper_1801_06300_gb300 import capi

    mesh = W.bump_channel(24, 4, 0.0, 0)  # long in x
    part = capi.partition(mesh, 2)
    cx = mesh.coords[mesh.elems].mean(axis=1)[:, 0]
    assert cx[part == 0].max() <= cx[part == 1].min()
    assert abs(int((part == 0).sum()) - int((part == 1).sum())) <= 1


def test_partition_rejects_bad_requests():
    from paper_1801_06300_gb300 import capi

    mesh = W.periodic_square(2, 1.0)
    with pytest.raises(capi.PcexpError):
        capi.partition(mesh, 0)
    with pytest.raises(capi.PcexpError):
        capi.partition(mesh, 17)
    with pytest.raises(capi.PcexpError):
        capi.partition(mesh, mesh.n_elem + 1)
