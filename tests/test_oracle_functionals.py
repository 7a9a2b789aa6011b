"""Pins of the oracle's output functionals and diagnostics against closed forms.

* ``wall_force``: for a state at rest whose pressure is linear in the coordinates (exactly
  representable at p >= 1), the pressure force on straight wall facets is the trapezoid sum
  p_bar (dy, -dx) over the facets' own vertex coordinates (2D, outward normal of the fluid
  pointing into the wall), and on the flat z-walls of a cube a L^3 for p = p0 + a z (3D).
  A flipped normal, a dropped face weight or a missing factor 2 on triangular faces fails.
* ``entropy_error`` (Eq. entropy_error, Sec. 5.1): 0 in the free stream; sqrt(c^2 - 1) for a
  constant entropy ratio s/s0 = c; sqrt(sum_e c_e^2 |E| / |Omega| - 1) for piecewise-constant
  ratios (element areas by the shoelace formula); and the closed-form integral of
  (1 + a x)^2 for a ratio linear in x.
* ``density_residual_norm`` (Eq. cfl, second line): sqrt(sum of squared density
  coefficients) / |Omega| on hand-built residual vectors.
* The unsteady scheme reproduces the exact translation of the isentropic vortex: the L2 error
  after a fixed time falls like h^(p+1) = h^2 at p = 1 (PCEXP at fixed CFL is second order in
  time, so both errors scale as h^2).
"""
import numpy as np
import pytest

import workloads as W
from oracle import pcexp
from oracle.cases import vortex_state
from oracle.dg import DGOracle


def rest_state_linear_pressure(dg, p0, grad):
    """Coefficients of rho = 1, zero velocity, p = p0 + grad . x (E = p / (gamma - 1))."""
    def fn(x):
        p = p0 + np.einsum("...d,d->...", x, np.asarray(grad, float))
        U = np.zeros(x.shape[:-1] + (dg.nv,))
        U[..., 0] = 1.0
        U[..., -1] = p / (dg.gamma - 1.0)
        return U
    return dg.project(fn)


def bump_facets(mesh):
    """Lower and upper wall facets of ``workloads.bump_channel`` as vertex coordinate pairs
    ordered by increasing x."""
    X = mesh.coords
    low, up = [], []
    for (a, b), t in zip(mesh.bfaces, mesh.btags):
        if t != W.BC_SLIP_WALL:
            continue
        A, B = X[a], X[b]
        if A[0] > B[0]:
            A, B = B, A
        (up if A[1] > 0.5 else low).append((A, B))
    return low, up


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("grad", [(0.3, 0.0), (0.0, -0.4), (0.2, 0.5)])
def test_wall_force_linear_pressure_trapezoid_2d(p, grad):
    mesh = W.bump_channel(12, 4, 0.15, 3)
    dg = DGOracle(mesh, p, W.Freestream(0.5, 0.0))
    p0 = 1.7
    u = rest_state_linear_pressure(dg, p0, grad)
    pf = lambda P: p0 + grad[0] * P[0] + grad[1] * P[1]  # noqa: E731
    low, up = bump_facets(mesh)
    Fx = Fy = 0.0
    for A, B in low:  # fluid above: outward normal (dy, -dx) / |AB|
        pb = 0.5 * (pf(A) + pf(B))
        Fx += pb * (B[1] - A[1])
        Fy += -pb * (B[0] - A[0])
    for A, B in up:  # fluid below: outward normal (-dy, dx) / |AB| = (0, 1) on y = 1
        pb = 0.5 * (pf(A) + pf(B))
        Fx += -pb * (B[1] - A[1])
        Fy += pb * (B[0] - A[0])
    assert len(low) == 12 and len(up) == 12
    assert dg.wall_force(u, (1.0, 0.0)) == pytest.approx(Fx, rel=1e-12, abs=1e-13)
    assert dg.wall_force(u, (0.0, 1.0)) == pytest.approx(Fy, rel=1e-12, abs=1e-13)


def test_wall_force_uniform_pressure_closed_channel_2d():
    """Uniform p on the walls of the channel: F_x = p (y_end - y_start) = 0 on either wall and
    F_y = p (3 - 3) = 0 (both walls span x in [-1, 2]); only the upper wall: F_y = 3 p."""
    mesh = W.bump_channel(16, 4, 0.15, 5)
    dg = DGOracle(mesh, 2, W.Freestream(0.5, 0.0))
    u = rest_state_linear_pressure(dg, 2.5, (0.0, 0.0))
    assert abs(dg.wall_force(u, (1.0, 0.0))) < 1e-13
    assert abs(dg.wall_force(u, (0.0, 1.0))) < 1e-12
    # the upper wall alone: a copy of the mesh whose lower wall is far field
    low_tag = np.array([W.BC_FARFIELD if (t == W.BC_SLIP_WALL and mesh.coords[a, 1] < 0.5) else t
                        for (a, _), t in zip(mesh.bfaces, mesh.btags)], np.int32)
    import dataclasses
    dg2 = DGOracle(dataclasses.replace(mesh, btags=low_tag), 2, W.Freestream(0.5, 0.0))
    u2 = rest_state_linear_pressure(dg2, 2.5, (0.0, 0.0))
    assert dg2.wall_force(u2, (0.0, 1.0)) == pytest.approx(3.0 * 2.5, rel=1e-13)


def cube_with_z_walls(n, L):
    """Non-periodic Kuhn cube whose faces on z = 0 and z = L are slip walls (the rest far field)."""
    mesh = W.periodic_cube_kuhn(n, L, 0.0, 0, periodic=False)
    z = mesh.coords[mesh.bfaces][:, :, 2]
    on_z = np.all(np.isclose(z, 0.0), axis=1) | np.all(np.isclose(z, L), axis=1)
    tags = np.where(on_z, W.BC_SLIP_WALL, W.BC_FARFIELD).astype(np.int32)
    import dataclasses
    return dataclasses.replace(mesh, btags=tags)


@pytest.mark.parametrize("p", [1, 2])
def test_wall_force_linear_pressure_cube_3d(p):
    """p = p0 + a z on the walls z = 0 (normal -z) and z = L (normal +z): F_z = a L^3 and
    F_x = F_y = 0; the triangular face rule's weights sum to 1/2, so a missing factor 2
    halves F_z."""
    L, a = 2.0, 0.35
    dg = DGOracle(cube_with_z_walls(2, L), p, W.Freestream(0.5, 0.0))
    u = rest_state_linear_pressure(dg, 1.3, (0.0, 0.0, a))
    assert dg.wall_force(u, (0.0, 0.0, 1.0)) == pytest.approx(a * L ** 3, rel=1e-12)
    assert abs(dg.wall_force(u, (1.0, 0.0, 0.0))) < 1e-12
    assert abs(dg.wall_force(u, (0.0, 1.0, 0.0))) < 1e-12


# ------------------------------------------------------------------ entropy error
def state_with_entropy_ratio(dg, ratio):
    """rho = rho_inf, zero velocity, p = ratio(x) p_inf: s / s0 = ratio (s = p / rho^gamma)."""
    f = dg.free

    def fn(x):
        U = np.zeros(x.shape[:-1] + (dg.nv,))
        U[..., 0] = f.rho
        U[..., -1] = ratio(x) * f.p / (dg.gamma - 1.0)
        return U
    return dg.project(fn)


def test_entropy_error_zero_in_free_stream():
    dg = DGOracle(W.periodic_square(5, 10.0, 0.15, 7), 2, W.Freestream(0.5, 30.0))
    u = np.zeros((dg.E, dg.nv, dg.N))
    u[:, :, 0] = dg.freestream_state()[None, :] * np.sqrt(dg.area)[:, None]
    # sqrt of a rounding-level difference of two sums equal to |Omega|
    assert dg.entropy_error(u, 100.0) < 1e-7


@pytest.mark.parametrize("c", [1.5, 0.8])
def test_entropy_error_constant_ratio(c):
    """s / s0 = c everywhere: E = sqrt(c^2 - 1) when c > 1; the radicand c^2 - 1 < 0 is clipped to 0."""
    dg = DGOracle(W.periodic_square(4, 10.0, 0.1, 2), 1, W.Freestream(0.5, 0.0))
    u = state_with_entropy_ratio(dg, lambda x: np.full(x.shape[:-1], c))
    expect = np.sqrt(max(c * c - 1.0, 0.0))
    assert dg.entropy_error(u, 100.0) == pytest.approx(expect, rel=1e-12, abs=1e-7)


def test_entropy_error_piecewise_constant_ratio():
    mesh = W.periodic_square(6, 10.0, 0.15, 4)
    dg = DGOracle(mesh, 0, W.Freestream(0.5, 0.0))
    X = mesh.coords[mesh.elems]  # [E, 3, 2]
    area = 0.5 * ((X[:, 1, 0] - X[:, 0, 0]) * (X[:, 2, 1] - X[:, 0, 1])
                  - (X[:, 2, 0] - X[:, 0, 0]) * (X[:, 1, 1] - X[:, 0, 1]))
    cen = X.mean(axis=1)
    c = np.where(cen[:, 0] < 5.0, 1.2, 1.6)
    u = np.zeros((dg.E, dg.nv, dg.N))
    u[:, 0, 0] = 1.0 * np.sqrt(area)              # rho = 1 (P0 basis: 1 / sqrt|E|)
    u[:, -1, 0] = c * 1.0 / 0.4 * np.sqrt(area)   # p = c p_inf, E = p / (gamma - 1)
    expect = np.sqrt(np.sum(c * c * area) / 100.0 - 1.0)
    assert dg.entropy_error(u, 100.0) == pytest.approx(expect, rel=1e-12)


def test_entropy_error_linear_ratio_closed_form():
    """s / s0 = 1 + a x on the square [0, L]^2 (exact at p = 1; the volume rule is exact to
    degree 3): int (1 + a x)^2 = L ((1 + a L)^3 - 1) / (3 a).  No jitter, so that the elements
    tile [0, L]^2 exactly (jittered periodic images leave it)."""
    L, a = 10.0, 0.04
    dg = DGOracle(W.periodic_square(4, L, 0.0, 0), 1, W.Freestream(0.5, 0.0))
    u = state_with_entropy_ratio(dg, lambda x: 1.0 + a * x[..., 0])
    integral = L * ((1.0 + a * L) ** 3 - 1.0) / (3.0 * a)
    expect = np.sqrt(integral / (L * L) - 1.0)
    assert dg.entropy_error(u, L * L) == pytest.approx(expect, rel=1e-12)


# --------------------------------------------------------- density residual norm
def test_density_residual_norm_hand_built():
    dg = DGOracle(W.periodic_square(3, 1.0, 0.0, 0), 2, W.Freestream(0.5, 0.0))
    R = np.zeros((dg.E, dg.nv, dg.N))
    R[4, 0, 2] = 3.0
    R[7, 0, 0] = -4.0
    R[1, 1:, :] = 100.0  # momentum and energy residuals do not enter
    assert dg.density_residual_norm(R.reshape(-1), 2.0) == pytest.approx(5.0 / 2.0, rel=1e-15)
    R[:, 0, :] = 0.0
    R[0, 0, 5] = 1e-3
    assert dg.density_residual_norm(R, 0.5) == pytest.approx(2e-3, rel=1e-15)


# ---------------------------------------------------- exact translation of the vortex
def test_vortex_translation_error_rate_p1():
    """PCEXP at CFL 2 (m = 10) to t ~ 1 on the periodic square [0, 10]^2: the L2 error against
    the exactly translated vortex falls like h^2 at p = 1."""
    case = W.case_vortex2d_small()
    free, vortex = case.free, case.vortex
    t_end = 1.0
    errs = []
    for n in (8, 16, 32):
        dg = DGOracle(W.periodic_square(n, 10.0), 1, free)
        u = dg.project(lambda x: vortex_state(x, free, vortex, period=10.0)).reshape(-1)
        dt0 = float(np.min(dg.local_dt(u, 2.0)))
        steps = int(np.ceil(t_end / dt0))
        dt = t_end / steps
        for _ in range(steps):
            u, _ = pcexp.pcexp_step(u, dg.residual, dg.jvp, dt, 10)
        err = dg.l2_error(u, lambda x: vortex_state(x, free, vortex, t=t_end, period=10.0))
        errs.append(err)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < errs[0]
    assert rates[-1] > 1.7, (errs, rates)
