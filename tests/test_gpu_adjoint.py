"""Adjoint operators of the CUDA path against the oracle: J^T w (transpose of the exact
Jacobian of Eq. jac1/jac2) and the second-order term (d(J(u) v)/du)^T w that the adjoint of
a PCEXP step needs because J_n = J(u_n)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_1801_06300_gb300 import build
    build()
    from paper_1801_06300_gb300 import capi as c
    c.load()
    return c


def state(dg, seed, amp=0.05):
    u = np.zeros((dg.E, dg.nv, dg.N))
    u[:, :, 0] = dg.freestream_state()[None, :] * np.sqrt(dg.area)[:, None]
    return (u + amp * W.random_coeffs(seed, u.shape) * np.abs(u[:, :, :1])).reshape(-1)


CASES = {
    "periodic_p2": lambda: (W.periodic_square(6, 10.0, 0.15, 3), 2, W.Freestream(0.5, 30.0)),
    "bump_p1": lambda: (W.bump_channel(8, 4, 0.15, 1), 1, W.Freestream(0.5, 0.0)),
    "bump_p3": lambda: (W.bump_channel(6, 3, 0.15, 2), 3, W.Freestream(0.5, 0.0)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_vjp_dot_product_and_dense_transpose(capi, case):
    from oracle.dg import DGOracle
    mesh, p, free = CASES[case]()
    dg = DGOracle(mesh, p, free)
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=2)
    u = state(dg, 1)
    v = W.random_coeffs(2, (dg.K,))
    w = W.random_coeffs(3, (dg.K,))
    Jv = ctx.jvp(u, v)
    JTw = ctx.vjp(u, w)
    lhs, rhs = w @ Jv, JTw @ v
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(w) @ np.abs(Jv))
    if dg.K <= 600:
        J = dg.dense_jacobian(u)
        ref = J.T @ w
        assert np.linalg.norm(JTw - ref) <= 1e-12 * np.linalg.norm(ref)
    ctx.close()


@pytest.mark.parametrize("case", list(CASES))
def test_jvp_state_adjoint_against_oracle_differences(capi, case):
    """delta . (d(w^T J(u) v)/du) equals the central difference of w^T J(u) v (oracle dual numbers)."""
    from oracle.dg import DGOracle
    mesh, p, free = CASES[case]()
    dg = DGOracle(mesh, p, free)
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=2)
    u = state(dg, 4)
    v = W.random_coeffs(5, (dg.K,))
    w = W.random_coeffs(6, (dg.K,))
    g = ctx.jvp_state_adjoint(u, v, w)
    for seed in (7, 8):
        delta = W.random_coeffs(seed, (dg.K,)) * np.abs(u) * 1e-2
        h = 1e-3
        fd = (w @ dg.jvp(u + h * delta, v) - w @ dg.jvp(u - h * delta, v)) / (2 * h)
        assert abs(g @ delta - fd) <= 1e-6 * max(abs(fd), 1e-30) + 1e-12 * np.abs(g) @ np.abs(delta)
    ctx.close()
