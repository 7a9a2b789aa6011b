"""Pins of the Krylov error estimate and the adaptive dimension (reading of the paper's
Krylov tolerance 1e-5, Sec. 5; estimate of Saad 1992, cited in Sec. 2.2).

* The estimate dt h_{k+1,k} |e_k^T phi_2(dt H_k) e_1| / ||phi_1(dt H_k) e_1|| tracks the true
  relative error of the Krylov phi_1 product, computed against phi_1(dt J) b from a dense
  exponential (scipy.linalg.expm of the augmented matrix [[dt J, b], [0, 0]]): within a
  factor of 3 wherever the error is between 1e-13 and 1e-2, on a symmetric negative
  definite matrix and on the dense DG Jacobian of a small channel.
* With a tolerance the process stops at the first checkpoint k (multiple of 5) whose
  estimate is within it (every earlier checkpoint's estimate exceeds it), the true error
  there is within 5x the tolerance, and a tolerance that is never met gives k = m.
* The steady march's CFL cap follows cfl_cap_update: halving-type cuts when the estimate
  exceeds the tolerance, growth by at most 2x otherwise.
"""
import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle import krylov, pcexp
from oracle.dg import DGOracle


def phi1_dense(J, b, dt):
    n = len(b)
    A = np.zeros((n + 1, n + 1))
    A[:n, :n] = dt * J
    A[:n, n] = b
    return scipy.linalg.expm(A)[:n, n]


def spd_case(n=80, seed=2):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = -np.logspace(-1, 2, n)
    return Q @ np.diag(lam) @ Q.T, rng.standard_normal(n)


def dg_case():
    dg = DGOracle(W.bump_channel(6, 3, 0.1, 2), 1, W.Freestream(0.5, 0.0))
    u = np.zeros((dg.E, dg.nv, dg.N))
    u[:, :, 0] = dg.freestream_state()[None, :] * np.sqrt(dg.area)[:, None]
    u = u.reshape(-1) + 0.02 * W.random_coeffs(5, (dg.K,)) * np.repeat(np.sqrt(dg.area), dg.nv * dg.N)
    J = dg.dense_jacobian(u)
    return J, W.random_coeffs(6, (dg.K,))


@pytest.mark.parametrize("case,dt", [("spd", 0.05), ("spd", 0.2), ("dg", 0.02), ("dg", 0.005)])
def test_error_estimate_tracks_true_error(case, dt):
    J, b = spd_case() if case == "spd" else dg_case()
    exact = phi1_dense(J, b, dt)
    checked = 0
    for m in range(2, 31, 2):
        x, info = krylov.krylov_phi1(lambda v: J @ v, b, dt, m)
        true = np.linalg.norm(x - exact) / np.linalg.norm(exact)
        est = info["err"]
        if 1e-13 < true < 1e-2:
            assert true / 3.0 <= est <= 3.0 * true, (m, true, est)
            checked += 1
    assert checked >= 3


@pytest.mark.parametrize("tol", [1e-5, 1e-8])
def test_adaptive_dimension_stops_at_first_checkpoint_within_tolerance(tol):
    J, b = spd_case()
    dt = 0.1
    x, info = krylov.krylov_phi1(lambda v: J @ v, b, dt, 30, tol=tol)
    k = info["k"]
    assert k % 5 == 0 and k < 30
    assert info["err"] <= tol
    for kk in range(5, k, 5):
        _, i2 = krylov.krylov_phi1(lambda v: J @ v, b, dt, kk)
        assert i2["err"] > tol, kk
    exact = phi1_dense(J, b, dt)
    assert np.linalg.norm(x - exact) / np.linalg.norm(exact) <= 5 * tol


def test_adaptive_dimension_falls_back_to_m():
    J, b = spd_case()
    x, info = krylov.krylov_phi1(lambda v: J @ v, b, 5.0, 12, tol=1e-14)
    assert info["k"] == 12 and info["err"] > 1e-14
    y, _ = krylov.krylov_phi1(lambda v: J @ v, b, 5.0, 12)
    assert np.array_equal(x, y)


def test_cfl_cap_update():
    assert pcexp.cfl_cap_update(100.0, 0.0, 1e-5) == 200.0
    assert pcexp.cfl_cap_update(100.0, 1e-9, 1e-5) == 200.0           # far within: 2x
    assert pcexp.cfl_cap_update(100.0, 1e-3, 1e-5) == 25.0            # far outside: 1/4
    assert pcexp.cfl_cap_update(100.0, 4e-5, 1e-5) == pytest.approx(40.0)  # 0.8 (1/4)^(1/2)
