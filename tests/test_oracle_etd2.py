"""Pins of the oracle's ETD2 step (Eq. s7, with phi_2 of Eq. Phi2):

* scalar closed form: one unknown, m = 1 (the Krylov projection is exact), against
  phi_1(z) = expm1(z)/z and phi_2(z) = (expm1(z) - z)/z^2 evaluated directly, over
  steps of different sizes (the dt / dt_{n-1} factor of the divided difference);
* the first step has no N_{n-1} and equals the EXP1 stage (ETD1, Eq. s8) exactly;
* affine systems R(u) = A u + c have constant N, so ETD2 reproduces the exact flow
  u(t) = exp(t A) u_0 + t phi_1(t A) c over several steps;
* ETD2 on the DG vortex converges at second order in dt (Sec. 2.1: k = 2 of Eq. s5).
"""
import math

import numpy as np
import scipy.linalg

import workloads as W
from oracle import pcexp
from oracle.dg import DGOracle


def phi1(z):
    return math.expm1(z) / z


def phi2(z):
    return (math.expm1(z) - z) / (z * z)


def test_etd2_scalar_closed_form_variable_steps():
    R = lambda x: -x ** 2 + 0.3 * x  # noqa: E731
    Jf = lambda x: -2.0 * x + 0.3  # noqa: E731
    jvp = lambda x0, v: Jf(x0[0]) * v  # noqa: E731
    u = np.array([0.9])
    prev = None
    hist = []
    for dt in (0.25, 0.4, 0.3):
        un, _, prev_new = pcexp.etd2_step(u, R, jvp, dt, 1, prev)
        x = float(u[0])
        J = Jf(x)
        expect = x + dt * phi1(dt * J) * R(x)
        if prev is not None:
            xp, Rp, dtp = float(prev[0][0]), float(prev[1][0]), prev[2]
            d = R(x) - Rp - J * (x - xp)
            expect += dt * (dt / dtp) * phi2(dt * J) * d
        assert abs(un[0] - expect) <= 1e-14 * abs(expect)
        hist.append(un[0])
        u, prev = un, prev_new
    assert len(hist) == 3


def test_etd2_first_step_is_exp1():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((12, 12)) - 2.5 * np.eye(12)
    R = lambda x: A @ x - 0.1 * x ** 3  # noqa: E731
    jvp = lambda x0, v: A @ v - 0.3 * x0 ** 2 * v  # noqa: E731
    u = rng.standard_normal(12)
    a, _, _ = pcexp.etd2_step(u, R, jvp, 0.2, 12)
    b, _ = pcexp.pcexp_step(u, R, jvp, 0.2, 12, scheme="exp1")
    assert np.array_equal(a, b)


def test_etd2_exact_for_affine_systems():
    rng = np.random.default_rng(7)
    n = 10
    A = rng.standard_normal((n, n)) - 3.0 * np.eye(n)
    c = rng.standard_normal(n)
    u0 = rng.standard_normal(n)
    R = lambda x: A @ x + c  # noqa: E731
    jvp = lambda x0, v: A @ v  # noqa: E731
    u, prev, t = u0.copy(), None, 0.0
    for dt in (0.3, 0.3, 0.45):
        u, _, prev = pcexp.etd2_step(u, R, jvp, dt, n, prev)
        t += dt
    # u(t) = exp(tA) u0 + A^{-1} (exp(tA) - I) c
    E = scipy.linalg.expm(t * A)
    ref = E @ u0 + np.linalg.solve(A, (E - np.eye(n)) @ c)
    assert np.allclose(u, ref, atol=1e-11 * np.abs(ref).max())


def test_etd2_temporal_order_two():
    from oracle.cases import vortex_state
    case = W.case_vortex2d_small()
    dg = DGOracle(W.periodic_square(6, 10.0), 1, case.free)
    u0 = dg.project(lambda x: vortex_state(x, case.free, case.vortex, period=10.0)).reshape(-1)
    T = 0.8

    def run(n):
        u, _ = pcexp.etd2_run(dg, u0, 0.0, n, 8, dts=[T / n] * n)
        return u

    ref = run(64)
    e = [np.linalg.norm(run(n) - ref) for n in (2, 4)]
    assert 3.2 < e[0] / e[1] < 4.8, e
