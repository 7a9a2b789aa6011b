"""The rotating frame of reference (Sec. 4.1, Eq. euler) and the symmetry-plane condition on
the GPU against the oracle (whose rotating frame is pinned in test_oracle_rotating).

R and J v at <= 1e-12 (FP64) and 2e-5 (FP32-mixed), the transpose by the dot-product
identity, the time-step rule with the velocity relative to the frame, and PCEXP steps at
<= 1e-10, on a walled 2D box (rotation about z) and a walled Kuhn cube (a general omega).
The library's source term is the coefficient-wise -omega x m of the orthonormal basis; the
oracle integrates psi_i S(U_h) by quadrature (two independent forms of Eq. euler3's term).
"""
import dataclasses

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def capi():
    from paper_1801_06300_gb300 import build
    build()
    from paper_1801_06300_gb300 import capi as c
    c.load()
    return c


def walled(kind):
    if kind == "box2d":
        mesh = W.bump_channel(10, 5, 0.15, 4, bump_h=0.0)
        om = (0.0, 0.0, 0.7)
    else:
        mesh = W.periodic_cube_kuhn(3, 2.0, 0.1, 2, periodic=False)
        om = (0.3, -0.2, 0.5)
    return dataclasses.replace(mesh, btags=np.full(len(mesh.btags), W.BC_SLIP_WALL, np.int32)), om


def state(dg, seed, amp=0.05):
    u = np.zeros((dg.E, dg.nv, dg.N))
    U = [1.05, 0.3, -0.2] + ([0.15] if dg.dim == 3 else []) + [2.7]
    u[:, :, 0] = np.asarray(U)[None, :] * np.sqrt(dg.area)[:, None]
    return (u + amp * W.random_coeffs(seed, u.shape) * np.abs(u[:, :, :1])).reshape(-1)


@pytest.mark.parametrize("kind,p", [("box2d", 1), ("box2d", 3), ("cube3d", 1), ("cube3d", 2)])
def test_rotating_operators_match_oracle(capi, kind, p):
    from oracle.dg import DGOracle
    mesh, om = walled(kind)
    free = W.Freestream(0.5, 0.0)
    dg = DGOracle(mesh, p, free, omega=om)
    u = state(dg, 10 + p)
    v = W.random_coeffs(20 + p, (dg.K,))
    w = W.random_coeffs(30 + p, (dg.K,))
    Ro, Jo = dg.residual(u), dg.jvp(u, v)
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=4, omega=om)
    assert rel(ctx.residual(u), Ro) <= 1e-12
    assert rel(ctx.jvp(u, v), Jo) <= 1e-12
    JTw = ctx.vjp(u, w)
    assert abs(JTw @ v - w @ Jo) <= 1e-12 * (np.abs(w) @ np.abs(Jo))
    ctx.set_state(u)
    assert rel(ctx.compute_dt(4.0, local=True), dg.local_dt(u, 4.0)) <= 1e-13
    ctx.close()
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP32_MIXED, m_max=4, omega=om)
    assert rel(ctx.residual(u), Ro) <= 2e-5
    assert rel(ctx.jvp(u, v), Jo) <= 2e-5
    ctx.close()


@pytest.mark.parametrize("kind", ["box2d", "cube3d"])
def test_rotating_pcexp_steps_match_oracle(capi, kind):
    from oracle import pcexp
    from oracle.dg import DGOracle
    mesh, om = walled(kind)
    free = W.Freestream(0.5, 0.0)
    p = 1
    # the uniform absolute velocity moves at up to Mach 1.2 relative to the walls of the
    # rotating box (|omega x x| reaches 1.5): its wall shocks give negative pressures within
    # three steps of 0.005 (CFL 0.4) at P1 without a limiter, on both sides alike; 0.002 stays
    # physical
    dt = 0.002 if kind == "box2d" else 0.01
    dg = DGOracle(mesh, p, free, omega=om)
    u = state(dg, 5, 0.02)
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=10, omega=om)
    ctx.set_state(u)
    for n in range(3):
        u, info = pcexp.pcexp_step(u, dg.residual, dg.jvp, dt, 10)
        g = ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, dt, 10)
        assert g["k"] == (info["k1"], info["k2"])
        assert rel(ctx.get_state(), u) <= 1e-10, n
    # the FP32-mixed Krylov path (face blocks + the tile element kernel with the frame terms)
    ctx32 = capi.Context(mesh, p, free, capi.PCEXP_FP32_MIXED, m_max=10, omega=om)
    u0 = state(dg, 5, 0.02)
    ctx32.set_state(u0)
    uo = u0.copy()
    for n in range(3):
        uo, _ = pcexp.pcexp_step(uo, dg.residual, dg.jvp, dt, 10)
        ctx32.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, dt, 10)
    assert rel(ctx32.get_state(), uo) <= 2e-5
    ctx.close()
    ctx32.close()


def test_symmetry_plane_matches_slip_wall(capi):
    from oracle.dg import DGOracle
    mesh = W.bump_channel(12, 4, 0.15, 2)
    sym = np.where(mesh.btags == W.BC_SLIP_WALL, capi.PCEXP_BC_SYMMETRY, mesh.btags).astype(np.int32)
    mesh_s = dataclasses.replace(mesh, btags=sym)
    free = W.Freestream(0.5, 0.0)
    dg = DGOracle(mesh_s, 2, free)
    u = state(dg, 3)
    v = W.random_coeffs(4, (dg.K,))
    cw = capi.Context(mesh, 2, free, capi.PCEXP_FP64, m_max=4)
    cs = capi.Context(mesh_s, 2, free, capi.PCEXP_FP64, m_max=4)
    assert rel(cs.residual(u), dg.residual(u)) <= 1e-12
    assert rel(cs.jvp(u, v), dg.jvp(u, v)) <= 1e-12
    assert np.array_equal(cs.residual(u), cw.residual(u))
    assert cw.functional(capi.PCEXP_FUNC_WALL_FY, u)[0] != 0.0
    assert cs.functional(capi.PCEXP_FUNC_WALL_FY, u)[0] == 0.0
    cw.close()
    cs.close()


def test_rotating_frame_rejections(capi):
    free = W.Freestream(0.5, 0.0)
    for mesh, om in ((W.periodic_square(4, 1.0), (0, 0, 1.0)), (W.bump_channel(4, 2, 0.1, 1), (0, 0, 1.0)),
                     (walled("box2d")[0], (0.2, 0.0, 1.0))):
        with pytest.raises(capi.PcexpError) as ei:
            capi.Context(mesh, 1, free, capi.PCEXP_FP64, m_max=2, omega=om)
        assert ei.value.code == capi.PCEXP_ERR_INVALID_ARG
    mesh, om = walled("box2d")
    ctx = capi.Context(mesh, 1, free, capi.PCEXP_FP64, m_max=2, omega=om)
    u = ctx.get_state()
    with pytest.raises(capi.PcexpError) as ei:
        ctx.step_backward(u, 0.01, 2, u)
    assert ei.value.code == capi.PCEXP_ERR_UNSUPPORTED
    ctx.close()
