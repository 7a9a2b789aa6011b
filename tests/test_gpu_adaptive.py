"""Adaptive Krylov dimension and the Krylov-error cap of the steady march on the GPU,
against the oracle (krylov_tol > 0; reading of the paper's Krylov tolerance, Sec. 5).

* PCEXP steps with tolerance 1e-5 on the periodic vortex: the dimension of each stage, its
  error estimate and the state match the oracle (<= 1e-10), and the dimensions are below m.
* The steady march with a tolerance: iteration count, residual norms and final state match
  the oracle's march with the same CFL cap controller.
"""
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


@pytest.mark.parametrize("tol", [1e-5, 1e-7])
def test_adaptive_steps_match_oracle(capi, tol):
    from oracle import pcexp
    from oracle.cases import vortex_state
    from oracle.dg import DGOracle
    case = W.case_vortex2d_small(12)
    dg = DGOracle(case.mesh, case.p, case.free)
    u = dg.project(lambda x: vortex_state(x, case.free, case.vortex, period=10.0)).reshape(-1)
    m = 30
    ctx = capi.Context(case.mesh, case.p, case.free, capi.PCEXP_FP64, m_max=m, krylov_tol=tol)
    ctx.set_state(u)
    ks = []
    for n in range(6):
        dt = float(np.min(dg.local_dt(u, case.cfl)))
        u, info = pcexp.pcexp_step(u, dg.residual, dg.jvp, dt, m, tol=tol)
        g = ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, case.cfl, m)
        assert g["k"] == (info["k1"], info["k2"]), n
        assert abs(g["err"][0] - info["err1"]) <= 1e-6 * info["err1"]
        assert abs(g["err"][1] - info["err2"]) <= 1e-6 * max(info["err2"], 1e-300)
        assert rel(ctx.get_state(), u) <= 1e-10, n
        ks += list(g["k"])
    assert max(ks) < m  # the tolerance was met before m in every stage
    ctx.close()


def test_adaptive_fixed_m_reports_estimate(capi):
    from oracle import pcexp
    from oracle.cases import vortex_state
    from oracle.dg import DGOracle
    case = W.case_vortex2d_small(8)
    dg = DGOracle(case.mesh, case.p, case.free)
    u = dg.project(lambda x: vortex_state(x, case.free, case.vortex, period=10.0)).reshape(-1)
    ctx = capi.Context(case.mesh, case.p, case.free, capi.PCEXP_FP64, m_max=10)
    ctx.set_state(u)
    dt = float(np.min(dg.local_dt(u, case.cfl)))
    uo, info = pcexp.pcexp_step(u, dg.residual, dg.jvp, dt, 10)
    g = ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, case.cfl, 10)
    assert g["k"] == (10, 10)
    assert abs(g["err"][0] - info["err1"]) <= 1e-6 * info["err1"]
    assert abs(g["err"][1] - info["err2"]) <= 1e-6 * info["err2"]
    ctx.close()


@pytest.mark.parametrize("scheme", ["exp1", "pcexp"])
def test_steady_march_with_krylov_cap_matches_oracle(capi, scheme):
    from oracle import pcexp
    from oracle.dg import DGOracle
    mesh, free = W.bump_channel(24, 8, 0.15, 1), W.Freestream(0.5, 0.0)
    dg = DGOracle(mesh, 1, free)
    u0 = np.zeros((dg.E, dg.nv, dg.N))
    u0[:, :, 0] = dg.freestream_state()[None, :] * np.sqrt(dg.area)[:, None]
    u0 = u0.reshape(-1)
    vol = float(dg.area.sum())
    tol, cflmax, iters = 1e-5, 1000.0, 12
    uo, hist = pcexp.steady_march(dg, u0, cflmax, 12.0, iters, 20, vol, scheme=scheme, tol=tol)
    ctx = capi.Context(mesh, 1, free, capi.PCEXP_FP64, m_max=20, krylov_tol=tol)
    ctx.set_state(u0)
    sc = capi.PCEXP_SCHEME_PCEXP if scheme == "pcexp" else capi.PCEXP_SCHEME_EXP1
    info = ctx.march_steady(sc, cflmax, 12.0, iters, 20)
    assert info["iterations"] == iters and not info["converged"]
    assert abs(info["res_first"] - hist[0]) <= 1e-12 * hist[0]
    last = dg.density_residual_norm(dg.residual(uo), vol)
    assert abs(info["res_last"] - last) <= 1e-8 * last
    assert rel(ctx.get_state(), uo) <= 1e-9
    ctx.close()
