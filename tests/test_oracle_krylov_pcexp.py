"""Pins of the oracle's Arnoldi, phi functions, PCEXP/EXP1 steps and Sec. 3 stability results."""
import os

import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle import krylov, pcexp, stability
from oracle.dg import DGOracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ phi
@pytest.mark.parametrize("z", [-50.0, -3.0, -1e-9, 0.0, 1e-7, 0.7, 4.0])
def test_phi_scalar_closed_form(z):
    """phi_1(z) = (e^z - 1)/z (Eq. Phi1 for 1x1), phi_2(z) = (e^z - 1 - z)/z^2 (Eq. Phi2)."""
    p1, p2 = krylov.phi_e1(np.array([[z]]), 1.0)
    if abs(z) < 1e-5:
        e1 = 1 + z / 2 + z * z / 6
        e2 = 0.5 + z / 6 + z * z / 24
    else:
        e1 = np.expm1(z) / z
        e2 = (np.expm1(z) - z) / z ** 2
    assert abs(p1[0] - e1) <= 1e-15 * max(1, abs(e1))
    assert abs(p2[0] - e2) <= 1e-15 * max(1, abs(e2))


def test_phi_diagonalisable():
    rng = np.random.default_rng(1)
    S = rng.standard_normal((6, 6))
    lam = np.array([-3.0, -1.0, -0.2, 0.0, 0.5, -10.0])
    H = S @ np.diag(lam) @ np.linalg.inv(S)
    ph = np.array([np.expm1(l) / l if l != 0 else 1.0 for l in lam])
    ref = S @ (ph * np.linalg.solve(S, np.eye(6)[:, 0]))
    got, _ = krylov.phi_e1(H, 1.0)
    assert np.allclose(got, ref, atol=1e-12, rtol=1e-12)


@pytest.mark.parametrize("scale", [0.1, 3.0, 100.0])
def test_phi_matches_library_expm(scale):
    rng = np.random.default_rng(2)
    H = rng.standard_normal((12, 12)) * scale
    H -= 2 * scale * np.eye(12)
    A = np.zeros((14, 14))
    A[:12, :12] = H
    A[0, 12] = 1
    A[12, 13] = 1
    X = scipy.linalg.expm(A)
    p1, p2 = krylov.phi_e1(H, 1.0)
    assert np.allclose(p1, X[:12, 12], rtol=1e-11, atol=1e-14 * np.abs(X[:12, 12]).max())
    assert np.allclose(p2, X[:12, 13], rtol=1e-11, atol=1e-14 * np.abs(X[:12, 13]).max())


# ------------------------------------------------------------------ Arnoldi
def test_arnoldi_relation_and_orthonormality():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((200, 200)) / 10
    b = rng.standard_normal(200)
    V, Hb, k, beta, brk = krylov.arnoldi(lambda v: A @ v, b, 25)
    assert k == 25 and not brk
    assert np.abs(V.T @ V - np.eye(26)).max() < 1e-13
    assert np.abs(A @ V[:, :25] - V @ Hb).max() < 1e-12
    assert np.allclose(np.triu(Hb, -1), Hb)  # upper Hessenberg
    assert abs(beta - np.linalg.norm(b)) < 1e-12


def test_arnoldi_happy_breakdown_at_invariant_subspace():
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((50, 50)))
    D = np.diag(np.r_[np.arange(1, 6) * -1.0, np.zeros(45)])
    A = Q @ D @ Q.T
    b = Q[:, :5] @ rng.standard_normal(5)  # lies in a 5-dim invariant subspace
    V, Hb, k, beta, brk = krylov.arnoldi(lambda v: A @ v, b, 20)
    assert brk and k == 5


def test_krylov_full_dimension_equals_dense_phi_on_dg_jacobian():
    """m = K: the Krylov phi_1 equals phi_1 of the dense DG Jacobian (Eq. final, exact)."""
    dg = DGOracle(W.periodic_square(3, 1.0, 0.1, 1), 0, W.Freestream(0.5, 30.0))
    u = np.zeros((dg.E, dg.nv, dg.N))
    u[:, :, 0] = dg.freestream_state() * np.sqrt(dg.area)[:, None]
    u = u * (1 + 0.05 * W.random_coeffs(2, u.shape))
    J = dg.dense_jacobian(u)
    b = W.random_coeffs(3, (dg.K,))
    dt = 0.05
    x, info = krylov.krylov_phi1(lambda v: J @ v, b, dt, dg.K, eta=1e-12)
    A = np.zeros((dg.K + 1, dg.K + 1))
    A[:dg.K, :dg.K] = dt * J
    A[:dg.K, dg.K] = b
    ref = scipy.linalg.expm(A)[:dg.K, dg.K]
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


# ------------------------------------------------------------------ PCEXP
def test_pcexp_exact_for_linear_systems():
    """N = 0 (R linear, J exact): PCEXP gives exp(dt A) u (Eq. growthfactor)."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((20, 20)) - 3 * np.eye(20)
    u = rng.standard_normal(20)
    un, info = pcexp.pcexp_step(u, lambda x: A @ x, lambda x0, v: A @ v, 0.7, 20)
    ref = scipy.linalg.expm(0.7 * A) @ u
    assert np.allclose(un, ref, atol=1e-11 * np.abs(ref).max())


def test_pcexp_with_zero_jacobian_is_heun():
    """J -> 0: PCEXP is the second-order Runge-Kutta (Heun) step (Eq. rk2)."""
    R = lambda x: -x ** 3 + np.sin(x)  # noqa: E731
    u = np.linspace(-1, 1, 9)
    dt = 0.3
    un, _ = pcexp.pcexp_step(u, R, lambda x0, v: 0.0 * v, dt, 5)
    k1 = R(u)
    k2 = R(u + dt * k1)
    assert np.allclose(un, u + 0.5 * dt * (k1 + k2), atol=1e-14)


@pytest.mark.parametrize("a,b", [(-0.3, -1.0), (-2.0, -5.0), (0.5, -0.2), (-1.0, 0.3), (-7.0, -20.0)])
def test_pcexp_scalar_growth_factor(a, b):
    """PCEXP on u' = J u + lambda u with the scheme's J = J: u_{n+1}/u_n = r(a, b) of Eq. grow."""
    dt = 0.5
    lam, J = a / dt, b / dt
    u = np.array([1.0])
    un, _ = pcexp.pcexp_step(u, lambda x: (J + lam) * x, lambda x0, v: J * v, dt, 1)
    assert abs(un[0] - stability.r_pcexp(a, b)) < 1e-13 * max(1, abs(un[0]))
    ue, _ = pcexp.pcexp_step(u, lambda x: (J + lam) * x, lambda x0, v: J * v, dt, 1, scheme="exp1")
    assert abs(ue[0] - stability.r_exp1(a, b)) < 1e-13 * max(1, abs(ue[0]))


def test_growth_series_y_poly():
    for a in [-0.5, 0.2, 1.0]:
        for b in [1e-2, 2e-2]:
            err = abs(stability.r_pcexp(a, b) - stability.r_pcexp_series(a, b))
            assert err < 2 * b ** 3 * (1 + abs(a)) ** 3


def test_local_truncation_errors():
    """PCEXP: e^{a+b} - r = O(dt^3) with coefficient lambda (lambda - J)(lambda + J)/6
    (derived from Eq. grow; differs from the printed Eq. trun1); EXP1: Eq. trun2."""
    lam, J = 0.7, -1.3
    for dt in [1e-2, 5e-3]:
        a, b = dt * lam, dt * J
        lte = np.exp(a + b) - stability.r_pcexp(a, b)
        assert abs(lte / dt ** 3 - lam * (lam - J) * (lam + J) / 6) < 0.05
        lte1 = np.exp(a + b) - stability.r_exp1(a, b)
        assert abs(lte1 / dt ** 2 - 0.5 * lam * (J + lam)) < 0.05


def test_table_timesize_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "timesize.txt")) if l.strip() and not l.startswith("#")]
    for m, val, tol in rows:
        got = stability.max_stable_real(int(m))
        assert abs(got - float(val)) <= float(tol), (m, got, val)


def test_tvdrk3_strip():
    off = stability.tvdrk3_strip_offset()
    assert abs(off - (-2.512745)) < 1e-6
    assert abs(abs(stability.r_tvdrk3(off, 0.0)) - 1) < 1e-12


def test_pcexp_and_exp1_stability_regions_negative_b():
    """Eq. pcexp_bd and exp1_bd agree with brute-force |r| <= 1 for b < 0."""
    bs = np.linspace(-10, -0.05, 120)
    as_ = np.linspace(-10, 10, 121)
    A, B = np.meshgrid(as_, bs)
    stable = np.abs(stability.r_pcexp(A, B)) <= 1 + 1e-12
    pred = (A <= -B) & (A >= stability.pcexp_boundary_lower(B))
    margin = (np.abs(A + B) < 0.1) | (np.abs(A - stability.pcexp_boundary_lower(B)) < 0.1)
    assert np.all((stable == pred) | margin)
    stable1 = np.abs(stability.r_exp1(A, B)) <= 1 + 1e-12
    pred1 = (A <= -B) & (A >= stability.exp1_boundary_lower(B))
    margin1 = (np.abs(A + B) < 0.1) | (np.abs(A - stability.exp1_boundary_lower(B)) < 0.1)
    assert np.all((stable1 == pred1) | margin1)


def test_temporal_order_two():
    """PCEXP on the DG vortex converges at second order in dt (Sec. 5.1)."""
    from oracle.cases import vortex_state
    case = W.case_vortex2d_small()
    dg = DGOracle(W.periodic_square(6, 10.0), 1, case.free)
    u0 = dg.project(lambda x: vortex_state(x, case.free, case.vortex, period=10.0)).reshape(-1)
    T = 0.8

    def run(n):
        u = u0.copy()
        for _ in range(n):
            u, _ = pcexp.pcexp_step(u, dg.residual, dg.jvp, T / n, 8)
        return u

    ref = run(64)
    e = [np.linalg.norm(run(n) - ref) for n in (2, 4)]
    assert 3.2 < e[0] / e[1] < 4.8
