"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds only input generation: mesh vertices and connectivity,
boundary tags, periodic vertex identification, flow-case parameters and
seeded random arrays.  It contains none of the DG or PCEXP arithmetic
(no quadrature, basis, flux, Krylov or time-stepping code), so both sides
of every parity test can draw their inputs from it without sharing method
code.

Random numbers come from splitmix64, written from its published definition
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): state += 0x9E3779B97F4A7C15, then two xor-shift-multiply
rounds and a final xor-shift.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Boundary tags of the mesh interface (same numbers as the C header).
BC_SLIP_WALL = 1
BC_FARFIELD = 2

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """The first ``n`` outputs of splitmix64 started from state ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed % (1 << 64)) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int) -> np.ndarray:
    """``n`` doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm(seed: int, n: int) -> np.ndarray:
    """``n`` doubles in [-1, 1)."""
    return 2.0 * uniform(seed, n) - 1.0


@dataclasses.dataclass
class Mesh:
    """A conforming simplex mesh in the form the C interface takes.

    coords      [n_vert][dim] float64
    elems       [n_elem][dim+1] int32, positively oriented
    vert_master [n_vert] int32: vertices with equal master are one periodic vertex
    bfaces      [n_bface][dim] int32 vertex ids of tagged boundary faces
    btags       [n_bface] int32 (BC_SLIP_WALL or BC_FARFIELD)
    """

    dim: int
    coords: np.ndarray
    elems: np.ndarray
    vert_master: np.ndarray
    bfaces: np.ndarray
    btags: np.ndarray
    name: str = ""
    volume: float = 0.0

    @property
    def n_elem(self) -> int:
        return int(self.elems.shape[0])

    @property
    def n_vert(self) -> int:
        return int(self.coords.shape[0])


def _split_quads(nx: int, ny: int, vid) -> np.ndarray:
    """Each quad (i, j) split along its (0,0)-(1,1) diagonal into two CCW triangles."""
    tris = np.empty((nx * ny * 2, 3), dtype=np.int32)
    t = 0
    for j in range(ny):
        for i in range(nx):
            v00, v10, v11, v01 = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            tris[t] = (v00, v10, v11)
            tris[t + 1] = (v00, v11, v01)
            t += 2
    return tris


def periodic_square(n: int, length: float, jitter: float = 0.0, seed: int = 0) -> Mesh:
    """n x n quads on the periodic square [0, length]^2, each split into 2 triangles.

    Every vertex is moved by a uniform offset in [-jitter, jitter) x h per
    coordinate; periodic images share one offset, so the mesh stays periodic.
    """
    h = length / n
    nv = n + 1
    ii, jj = np.meshgrid(np.arange(nv), np.arange(nv), indexing="xy")
    ii = ii.ravel()
    jj = jj.ravel()
    master = ((jj % n) * n + (ii % n)).astype(np.int32)
    off = np.zeros((n * n, 2))
    if jitter > 0.0:
        r = uniform_pm(seed, 2 * n * n).reshape(n * n, 2)
        off = jitter * h * r
    coords = np.stack([ii * h + off[master, 0], jj * h + off[master, 1]], axis=1)
    elems = _split_quads(n, n, lambda i, j: j * nv + i)
    return Mesh(dim=2, coords=coords, elems=elems, vert_master=master,
                bfaces=np.zeros((0, 2), np.int32), btags=np.zeros(0, np.int32),
                name=f"periodic{n}x{n}", volume=length * length)


def bump_height(x, h: float = 0.1):
    """Lower wall of the bump channel: h sin^2(pi x) on [0, 1], zero elsewhere."""
    x = np.asarray(x, dtype=np.float64)
    return np.where((x >= 0.0) & (x <= 1.0), h * np.sin(np.pi * x) ** 2, 0.0)


def bump_channel(nx: int, ny: int, jitter: float = 0.0, seed: int = 0,
                 bump_h: float = 0.1) -> Mesh:
    """Channel x in [-1, 2], y in [y_b(x), 1] with a sin^2 bump on the lower wall.

    Vertical grid lines, linear blend in y, each quad split into 2 triangles.
    Interior vertices move by up to +-jitter of the local spacing in x and y;
    wall vertices move only along x and stay on the wall; inlet/outlet vertices
    move only along y; corners stay fixed.  Lower and upper walls are slip
    walls, inlet and outlet are far-field boundaries.
    """
    dx = 3.0 / nx
    nvx, nvy = nx + 1, ny + 1
    r = uniform_pm(seed, 2 * nvx * nvy).reshape(nvy, nvx, 2) if jitter > 0 else np.zeros((nvy, nvx, 2))
    coords = np.zeros((nvx * nvy, 2))
    for j in range(nvy):
        for i in range(nvx):
            x = -1.0 + dx * i
            eta = j / ny
            jx = r[j, i, 0] * jitter
            jy = r[j, i, 1] * jitter
            corner = (i in (0, nx)) and (j in (0, ny))
            if corner:
                pass
            elif j == 0 or j == ny:
                x = x + jx * dx
            elif i == 0 or i == nx:
                eta = (j + jy) / ny
            else:
                x = x + jx * dx
                eta = (j + jy) / ny
            yb = float(bump_height(x, bump_h))
            coords[j * nvx + i] = (x, yb + (1.0 - yb) * eta)
    vid = lambda i, j: j * nvx + i  # noqa: E731
    elems = _split_quads(nx, ny, vid)
    bf, bt = [], []
    for i in range(nx):
        bf.append((vid(i, 0), vid(i + 1, 0)))
        bt.append(BC_SLIP_WALL)
        bf.append((vid(i + 1, ny), vid(i, ny)))
        bt.append(BC_SLIP_WALL)
    for j in range(ny):
        bf.append((vid(0, j + 1), vid(0, j)))
        bt.append(BC_FARFIELD)
        bf.append((vid(nx, j), vid(nx, j + 1)))
        bt.append(BC_FARFIELD)
    # channel area: 3 minus the bump area (h/2 for sin^2 over a unit length)
    return Mesh(dim=2, coords=coords, elems=elems,
                vert_master=np.arange(nvx * nvy, dtype=np.int32),
                bfaces=np.asarray(bf, np.int32), btags=np.asarray(bt, np.int32),
                name=f"bump{nx}x{ny}", volume=3.0 - 0.5 * bump_h)


def stretched_periodic_square(n: int, length: float, power: int = 3) -> Mesh:
    """The paper's stiff vortex mesh (Sec. 5.1): node j = 1..n+1 of each direction at
    x_j = (1 - xi_j^p) x_L / 2 + (1 + xi_j^p) x_R / 2, xi_j = 2 (j - 1) / n - 1 (x_L = 0,
    x_R = length, p = 3), clustered about the centre; n x n quads, each split into 2
    triangles, periodic in both directions (node n+1 is node 1's periodic image)."""
    j = np.arange(1, n + 2)
    xi = 2.0 * (j - 1) / n - 1.0
    xs = 0.5 * (1.0 - xi ** power) * 0.0 + 0.5 * (1.0 + xi ** power) * length
    nv = n + 1
    ii, jj = np.meshgrid(np.arange(nv), np.arange(nv), indexing="xy")
    ii = ii.ravel()
    jj = jj.ravel()
    master = ((jj % n) * n + (ii % n)).astype(np.int32)
    coords = np.stack([xs[ii], xs[jj]], axis=1)
    elems = _split_quads(n, n, lambda i, k: k * nv + i)
    return Mesh(dim=2, coords=coords, elems=elems, vert_master=master,
                bfaces=np.zeros((0, 2), np.int32), btags=np.zeros(0, np.int32),
                name=f"stretched{n}x{n}", volume=length * length)


def periodic_cube_kuhn(n: int, length: float, jitter: float = 0.0, seed: int = 0,
                       periodic: bool = True) -> Mesh:
    """n^3 cubes on the cube [0, length]^3, each split into 6 Kuhn tetrahedra.

    The six tetrahedra of a cube share its main diagonal, so neighbouring cubes
    meet conformingly.  Vertex jitter works as in ``periodic_square`` (periodic
    images share one offset).  With ``periodic=False`` the outer faces are far-field
    boundary faces and boundary vertices are not moved.  Tetrahedra are ordered by
    cube (x fastest) and, within a cube, by the path order of the unit steps.
    """
    h = length / n
    nv = n + 1
    idx = np.arange(nv)
    kk, jj, ii = np.meshgrid(idx, idx, idx, indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    if periodic:
        master = (((kk % n) * n + (jj % n)) * n + (ii % n)).astype(np.int32)
        off = np.zeros((n ** 3, 3))
        if jitter > 0.0:
            off = jitter * h * uniform_pm(seed, 3 * n ** 3).reshape(n ** 3, 3)
        off = off[master]
    else:
        master = np.arange(nv ** 3, dtype=np.int32)
        off = np.zeros((nv ** 3, 3))
        if jitter > 0.0:
            off = jitter * h * uniform_pm(seed, 3 * nv ** 3).reshape(nv ** 3, 3)
            inner = (ii > 0) & (ii < n) & (jj > 0) & (jj < n) & (kk > 0) & (kk < n)
            off[~inner] = 0.0
    coords = np.stack([ii * h + off[:, 0], jj * h + off[:, 1], kk * h + off[:, 2]], axis=1)
    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = np.stack([ck.ravel(), cj.ravel(), ci.ravel()], axis=1)  # (i, j, k), x fastest
    base = base[np.lexsort((base[:, 0], base[:, 1], base[:, 2]))]
    vid = lambda p: (p[:, 2] * nv + p[:, 1]) * nv + p[:, 0]  # noqa: E731
    # Kuhn simplices: paths from (0,0,0) to (1,1,1) adding one unit vector at a time
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    unit = np.eye(3, dtype=np.int64)
    tets = np.empty((n ** 3, 6, 4), np.int32)
    for t, perm in enumerate(perms):
        p0 = base
        p1 = p0 + unit[perm[0]]
        p2 = p1 + unit[perm[1]]
        p3 = p2 + unit[perm[2]]
        tets[:, t] = np.stack([vid(p0), vid(p1), vid(p2), vid(p3)], axis=1)
    tets = tets.reshape(-1, 4)
    # orient positively
    X = coords[tets]
    vol = np.einsum("ed,ed->e", np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), X[:, 3] - X[:, 0])
    neg = vol < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    bfaces = np.zeros((0, 3), np.int32)
    btags = np.zeros(0, np.int32)
    if not periodic:
        # faces of tetrahedra that lie on the outer boundary
        fl = []
        for f in range(4):
            fv = tets[:, [(f + 1) % 4, (f + 2) % 4, (f + 3) % 4]]
            P = np.stack([ii[fv], jj[fv], kk[fv]], axis=-1)  # [E, 3, 3] lattice indices
            on = np.zeros(len(tets), bool)
            for d in range(3):
                for side in (0, n):
                    on |= np.all(P[:, :, d] == side, axis=1)
            fl.append(fv[on])
        bfaces = np.concatenate(fl).astype(np.int32)
        btags = np.full(len(bfaces), BC_FARFIELD, np.int32)
    return Mesh(dim=3, coords=coords, elems=tets, vert_master=master, bfaces=bfaces, btags=btags,
                name=f"kuhn{n}^3", volume=length ** 3)


# --------------------------------------------------------------------------
# Flow cases (parameters only; each side evaluates and projects them itself)
# --------------------------------------------------------------------------

GAMMA = 1.4


@dataclasses.dataclass
class Freestream:
    """Nondimensional free stream: rho = p = 1, speed Ma * sqrt(gamma p / rho)."""

    mach: float = 0.5
    alpha_deg: float = 0.0
    gamma: float = GAMMA
    rho: float = 1.0
    p: float = 1.0


@dataclasses.dataclass
class Vortex:
    """Isentropic vortex of strength ``eps`` centred at ``center``, carried by the free stream;
    ``radius`` is the core radius (the length unit of its profile)."""

    eps: float = 5.0
    center: tuple = (5.0, 5.0)
    radius: float = 1.0


@dataclasses.dataclass
class Case:
    name: str
    mesh: Mesh
    p: int
    m: int
    free: Freestream
    vortex: Vortex | None = None
    cfl: float = 1.0
    steps: int = 1
    blobs: np.ndarray | None = None  # [n][4]: (x, y, amplitude_rho, amplitude_p)
    blob_radius: float = 0.1


def blob_params(seed: int, n: int = 4, amplitude: float = 1e-2,
                box=((-0.5, 1.5), (0.2, 0.8))) -> np.ndarray:
    """Seeded centres and signed amplitudes of Gaussian (rho, p) perturbations."""
    r = uniform(seed, 4 * n).reshape(n, 4)
    out = np.empty((n, 4))
    out[:, 0] = box[0][0] + (box[0][1] - box[0][0]) * r[:, 0]
    out[:, 1] = box[1][0] + (box[1][1] - box[1][0]) * r[:, 1]
    out[:, 2] = amplitude * (2 * r[:, 2] - 1)
    out[:, 3] = amplitude * (2 * r[:, 3] - 1)
    return out


def case_vortex2d_small(n: int = 16) -> Case:
    """Isentropic vortex, periodic [0,10]^2, n x n split quads, P1, m = 10, CFL 5, 20 steps."""
    return Case("vortex2d_p1", periodic_square(n, 10.0), p=1, m=10,
                free=Freestream(mach=0.5, alpha_deg=45.0), vortex=Vortex(5.0, (5.0, 5.0)),
                cfl=5.0, steps=20)


def case_bump2d(nx: int = 192, ny: int = 64, p: int = 2, seed: int = 1) -> Case:
    """Subsonic bump channel, Ma 0.5, +-15% jitter, P2, m = 30, local time steps."""
    return Case(f"bump2d_p{p}", bump_channel(nx, ny, 0.15, seed), p=p, m=30,
                free=Freestream(mach=0.5, alpha_deg=0.0), cfl=100.0, steps=1)


def case_vortex2d_large(n: int = 256, p: int = 3, seed: int = 3) -> Case:
    """Isentropic vortex, periodic [0,20]^2, jittered n x n split quads, P3, m = 30, CFL 20."""
    return Case(f"vortex2d_p{p}_n{n}", periodic_square(n, 20.0, 0.15, seed), p=p, m=30,
                free=Freestream(mach=0.5, alpha_deg=45.0), vortex=Vortex(5.0, (10.0, 10.0)),
                cfl=20.0, steps=200)


def case_bump_adjoint(nx: int = 96, ny: int = 32, seed: int = 4) -> Case:
    """Bump channel 96 x 32, P2, freestream plus 4 seeded Gaussian blobs, 50 PCEXP steps."""
    return Case("bump2d_adjoint", bump_channel(nx, ny, 0.15, 1), p=2, m=30,
                free=Freestream(mach=0.5, alpha_deg=0.0), cfl=5.0, steps=50,
                blobs=blob_params(seed))


def case_vortex3d(n: int = 48, p: int = 2, seed: int = 5) -> Case:
    """3D isentropic vortex (axis along z) on periodic [0,10]^3: n^3 cubes as Kuhn tetrahedra
    (6 n^3 elements, 663,552 at n = 48) with +-10% jitter, P2, m = 30, CFL 10, 50 steps."""
    return Case(f"vortex3d_p{p}_n{n}", periodic_cube_kuhn(n, 10.0, 0.10, seed), p=p, m=30,
                free=Freestream(mach=0.5, alpha_deg=45.0), vortex=Vortex(5.0, (5.0, 5.0)),
                cfl=10.0, steps=50)


def case_vortex_stretched(n: int = 24, p: int = 1) -> Case:
    """The paper's stiff vortex case (Sec. 5.1): periodic [0, 0.1]^2 on the stretched n x n
    mesh (minimum spacing 2.9e-5, maximum 0.0115 at n = 24), Ma 0.5 along x, vortex with
    beta = 0.2 and core radius R = 0.05 at (0.05, 0.05), PCEXP at CFL 1000, m = 30, one
    period T = 0.1 / U_inf.  With rho_inf = p_inf = 1 the paper's vortex is the isentropic
    vortex of core radius R and strength eps = 2 pi beta U_inf exp(-1/2)."""
    free = Freestream(mach=0.5, alpha_deg=0.0)
    u_inf = vortex_speed(free)
    eps = 2.0 * math.pi * 0.2 * u_inf * math.exp(-0.5)
    return Case(f"vortex_stretched_p{p}_n{n}", stretched_periodic_square(n, 0.1), p=p, m=30, free=free,
                vortex=Vortex(eps, (0.05, 0.05), 0.05), cfl=1000.0, steps=0)


def random_coeffs(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    """Seeded random array in [-scale, scale)."""
    n = int(np.prod(shape))
    return scale * uniform_pm(seed, n).reshape(shape)


def vortex_speed(free: Freestream) -> float:
    return free.mach * math.sqrt(free.gamma * free.p / free.rho)
