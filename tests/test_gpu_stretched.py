"""The stiff vortex of Sec. 5.1 on the GPU: the stretched 24 x 24 periodic mesh (smallest
spacing 2.9e-5, largest 0.0115), PCEXP at CFL 1000, m = 30.

* The first steps at CFL 1000 match the oracle step by step (equal Krylov dimensions).  At
  this stiffness the step map amplifies rounding: a 2e-16 relative perturbation of the
  oracle's own input moves its P2 step by 1e-10 to 5e-10 (about 1e-12 at P1).  The bound
  after step n is therefore (n + 1) max(1e-10, 10 x that self-sensitivity, measured here on
  the first step).
* One full period at CFL 1000 stays finite, and its L2 error against the exactly translated
  vortex is within 2x that of the same run at CFL 50 (nearly time-exact; measured 1.8x at
  P1, 1.3x at P2): the large steps add little to the spatial error, the paper's observation
  for PCEXP on this mesh.
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


def _prm(case):
    v = case.vortex
    return [v.eps, *v.center, 0.1, v.radius]


@pytest.mark.parametrize("p", [1, 2])
def test_cfl1000_steps_match_oracle(capi, p):
    from oracle import pcexp
    from oracle.cases import vortex_state
    from oracle.dg import DGOracle
    case = W.case_vortex_stretched(24, p)
    dg = DGOracle(case.mesh, p, case.free)
    u = dg.project(lambda x: vortex_state(x, case.free, case.vortex, period=0.1)).reshape(-1)
    ctx = capi.Context(case.mesh, p, case.free, capi.PCEXP_FP64, m_max=case.m)
    ctx.project_state(capi.PCEXP_PROJ_VORTEX, _prm(case))
    assert rel(ctx.get_state(), u) <= 1e-13
    # rounding sensitivity of the oracle's own first step
    dt0 = float(np.min(dg.local_dt(u, case.cfl)))
    a, _ = pcexp.pcexp_step(u, dg.residual, dg.jvp, dt0, case.m)
    sens = 0.0
    for seed in (1, 2):
        b, _ = pcexp.pcexp_step(u * (1.0 + 2e-16 * W.uniform_pm(seed, u.size)), dg.residual, dg.jvp, dt0, case.m)
        sens = max(sens, rel(b, a))
    tol = max(1e-10, 10.0 * sens)
    # the first dt comes from the same state on both sides; later steps take the oracle's dt
    # (dt is a minimum over the smallest central cells, whose local state differences exceed
    # the global relative L2 difference)
    assert abs(ctx.compute_dt(case.cfl) - dt0) <= 1e-13 * dt0
    for n in range(3):
        dt = float(np.min(dg.local_dt(u, case.cfl)))
        u, info = pcexp.pcexp_step(u, dg.residual, dg.jvp, dt, case.m)
        g = ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, dt, case.m)
        assert g["k"] == (info["k1"], info["k2"])
        # every step injects a rounding perturbation of this size: the bound grows with n
        assert rel(ctx.get_state(), u) <= (n + 1) * tol, (n, tol)
    ctx.close()


def _period(capi, case, cfl, T):
    ctx = capi.Context(case.mesh, case.p, case.free, capi.PCEXP_FP64, m_max=case.m)
    ctx.project_state(capi.PCEXP_PROJ_VORTEX, _prm(case))
    t, n = 0.0, 0
    while t < T * (1 - 1e-12):
        dt = min(ctx.compute_dt(cfl), T - t)
        ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, dt, case.m, info=False)
        t += dt
        n += 1
    u = ctx.get_state()
    ctx.close()
    return u, n


@pytest.mark.parametrize("p", [1, 2])
def test_one_period_at_cfl1000_close_to_time_exact(capi, p):
    from oracle.cases import vortex_state
    from oracle.dg import DGOracle
    case = W.case_vortex_stretched(24, p)
    T = 0.1 / W.vortex_speed(case.free)
    dg = DGOracle(case.mesh, p, case.free)
    exact = lambda x: vortex_state(x, case.free, case.vortex, t=T, period=0.1)  # noqa: E731
    u_big, n_big = _period(capi, case, 1000.0, T)
    u_ref, n_ref = _period(capi, case, 50.0, T)
    assert np.all(np.isfinite(u_big))
    e_big, e_ref = dg.l2_error(u_big, exact), dg.l2_error(u_ref, exact)
    assert n_ref > 10 * n_big
    assert e_big <= 2.0 * e_ref, (n_big, e_big, n_ref, e_ref)
