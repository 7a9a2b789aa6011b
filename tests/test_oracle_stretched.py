"""Pins of the stiff vortex case of Sec. 5.1 (stretched 24 x 24 mesh, CFL 1000).

* The mesh generator reproduces the spacings the paper prints for its stretched mesh:
  minimum about 3e-5 and maximum 0.0115 (x_j = (1 - xi^3) x_L / 2 + (1 + xi^3) x_R / 2 over
  the n + 1 nodes of a direction).
* The isentropic vortex with core radius R = 0.05 and eps = 2 pi beta U_inf exp(-1/2) is the
  paper's vortex: u = U_inf - beta U_inf (y - y_c)/R exp(-r^2/2), v = beta U_inf (x - x_c)/R
  exp(-r^2/2), T = T_inf - (beta U_inf)^2 / (2 C_p) exp(-r^2) (the squared amplitude of the
  temperature dip is our reading of the garbled line), isentropic density, at sample points.
* Two oracle PCEXP steps at CFL 1000 stay finite, and the global dt is the closed form
  CFL h / ((2p+1)(|v| + c)) of the smallest cell: the central right triangles have
  h = a (2 - sqrt 2) with a the smallest spacing, and |v| + c at their centroids is within
  a few percent of U_inf + c_inf.
"""
import math

import numpy as np

import workloads as W
from oracle import pcexp
from oracle.cases import vortex_state
from oracle.dg import DGOracle


def test_stretched_mesh_spacings_match_the_paper():
    mesh = W.stretched_periodic_square(24, 0.1)
    xs = np.unique(np.round(mesh.coords[:, 0], 15))
    d = np.diff(xs)
    assert len(xs) == 25
    assert 2.5e-5 <= d.min() <= 3.5e-5
    assert abs(d.max() - 0.0115) <= 5e-5
    assert mesh.n_elem == 2 * 24 * 24


def test_radius_vortex_is_the_paper_vortex():
    case = W.case_vortex_stretched()
    free, vx = case.free, case.vortex
    g = free.gamma
    U = W.vortex_speed(free)
    beta, R, xc, yc = 0.2, 0.05, 0.05, 0.05
    rng = np.random.default_rng(4)
    x = rng.uniform(0.0, 0.1, size=(40, 2))
    got = vortex_state(x, free, vx, period=0.1)
    dx, dy = x[:, 0] - xc, x[:, 1] - yc
    r2 = (dx * dx + dy * dy) / R ** 2
    u = U - beta * U * dy / R * np.exp(-r2 / 2)
    v = beta * U * dx / R * np.exp(-r2 / 2)
    Tinf = free.p / free.rho
    cp = g / (g - 1.0)  # gas constant 1 in these units (T = p / rho)
    T = Tinf - (beta * U) ** 2 / (2 * cp) * np.exp(-r2)
    rho = free.rho * (T / Tinf) ** (1.0 / (g - 1.0))
    p = rho * T
    E = p / (g - 1) + 0.5 * rho * (u * u + v * v)
    want = np.stack([rho, rho * u, rho * v, E], axis=1)
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13)


def test_cfl1000_steps_and_time_step():
    case = W.case_vortex_stretched(24, 1)
    dg = DGOracle(case.mesh, 1, case.free)
    u = dg.project(lambda x: vortex_state(x, case.free, case.vortex, period=0.1)).reshape(-1)
    a = np.diff(np.unique(np.round(case.mesh.coords[:, 0], 15))).min()
    c = math.sqrt(case.free.gamma * case.free.p / case.free.rho)
    dt0 = float(np.min(dg.local_dt(u, case.cfl)))
    guess = case.cfl * a * (2 - math.sqrt(2)) / (3 * (W.vortex_speed(case.free) + c))
    assert abs(dt0 / guess - 1.0) < 0.05
    for _ in range(2):
        dt = float(np.min(dg.local_dt(u, case.cfl)))
        u, info = pcexp.pcexp_step(u, dg.residual, dg.jvp, dt, case.m)
        assert np.all(np.isfinite(u)) and info["k1"] == case.m
