"""Pins of the oracle's element time-step rule (Eq. x3d) and of its steady march (Eq. cfl,
Sec. 5.2) against closed forms:
* h = 2 d |E| / |dE| is the diameter of the inscribed circle (sphere) of a simplex, which for
  a right isosceles triangle with legs a is a (2 - sqrt 2) and for a Kuhn tetrahedron of a
  cube with edge a is a (sqrt 2 - 1); in the free stream |v| + c = (1 + Ma) c.
* On a linear system R(u) = -a (u - u_inf) every PCEXP and EXP1 step with m at least the
  number of distinct local steps is exact, so one unit pseudo-step of du/dtau = D R(u)
  multiplies the residual of element e by exp(-a dt_e): the march's residual history,
  stopping index and final state follow in closed form.
"""
import numpy as np
import pytest

import workloads as W
from oracle import pcexp
from oracle.dg import DGOracle


def freestream_coeffs(dg):
    u = np.zeros((dg.E, dg.nv, dg.N))
    u[:, :, 0] = dg.freestream_state()[None, :] * np.sqrt(dg.area)[:, None]
    return u.reshape(-1)


def sound_speed(free):
    return np.sqrt(free.gamma * free.p / free.rho)


@pytest.mark.parametrize("p", [0, 1, 2])
def test_local_dt_inscribed_circle_of_right_triangles(p):
    n, L, cfl = 6, 3.0, 2.5
    free = W.Freestream(0.5, 30.0)
    dg = DGOracle(W.periodic_square(n, L, 0.0, 0), p, free)
    a = L / n
    expect = cfl * a * (2.0 - np.sqrt(2.0)) / ((2 * p + 1) * (1.0 + free.mach) * sound_speed(free))
    dte = dg.local_dt(freestream_coeffs(dg), cfl)
    assert dte.shape == (dg.E,)
    np.testing.assert_allclose(dte, expect, rtol=1e-13, atol=0)


@pytest.mark.parametrize("p", [0, 1])
def test_local_dt_inscribed_sphere_of_kuhn_tetrahedra(p):
    n, L, cfl = 3, 3.0, 1.5
    free = W.Freestream(0.5, 20.0)
    dg = DGOracle(W.periodic_cube_kuhn(n, L, 0.0, 0), p, free)
    a = L / n
    expect = cfl * a * (np.sqrt(2.0) - 1.0) / ((2 * p + 1) * (1.0 + free.mach) * sound_speed(free))
    dte = dg.local_dt(freestream_coeffs(dg), cfl)
    assert dte.shape == (dg.E,)
    np.testing.assert_allclose(dte, expect, rtol=1e-13, atol=0)


class LinearRelaxation:
    """Stand-in for the DG operator with the members the steady march uses: E elements of
    nv x N unknowns, R(u) = -a (u - u_inf), J v = -a v, local steps dt_e = CFL c_e."""

    def __init__(self, c=(0.05, 0.11, 0.23), nv=4, N=3, p=1, a=0.7, seed=3):
        self.c = np.asarray(c, dtype=np.float64)
        self.E, self.nv, self.N, self.p, self.a = len(c), nv, N, p, a
        self.uinf = W.random_coeffs(seed, (self.E * nv * N,))

    def residual(self, u):
        return -self.a * (u - self.uinf)

    def jvp(self, u, v):
        return -self.a * v

    def local_dt(self, u, cfl):
        return cfl * self.c

    def density_residual_norm(self, R, volume):
        return np.sqrt(np.sum(np.asarray(R).reshape(self.E, self.nv, self.N)[:, 0, :] ** 2)) / volume


@pytest.mark.parametrize("scheme", ["exp1", "pcexp"])
def test_steady_march_on_linear_relaxation_follows_exact_decay(scheme):
    op = LinearRelaxation()
    u0 = op.uinf + 2.0 * W.random_coeffs(4, op.uinf.shape)
    volume, cfl_max, decades = 1.0, 50.0, 10.0
    u, hist = pcexp.steady_march(op, u0, cfl_max, decades, 400, m=8, volume=volume, scheme=scheme)
    # closed form: the residual of element e shrinks by exp(-a CFL_n c_e) in iteration n
    g = (-op.a * (u0 - op.uinf)).reshape(op.E, op.nv, op.N)
    shrink = np.ones(op.E)
    expect = []
    for n in range(1, 401):
        r = np.sqrt(np.sum((g[:, 0, :] * shrink[:, None]) ** 2)) / volume
        expect.append(r)
        if r <= expect[0] * 10.0 ** (-decades):
            break
        cfl = min(cfl_max, max(r ** -3, 1.0 + (n - 1) / (2 * op.p + 1)))
        shrink *= np.exp(-op.a * cfl * op.c)
    expect = np.asarray(expect)
    assert len(hist) == len(expect) and len(expect) < 400
    np.testing.assert_allclose(hist, expect, rtol=1e-9, atol=1e-14 * expect[0])
    uo = op.uinf + ((u0 - op.uinf).reshape(op.E, -1) * shrink[:, None]).reshape(-1)
    np.testing.assert_allclose(u, uo, rtol=0, atol=1e-12 * np.abs(u0 - op.uinf).max())
