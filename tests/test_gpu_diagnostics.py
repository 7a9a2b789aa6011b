"""CUDA path vs the FP64 oracle for the diagnostics of the master state and for the
far-field ghost state's supersonic branches, through the C interface.

* pcexp_output(kind=1): the entropy error of Eq. entropy_error (Sec. 5.1), evaluated in FP64
  on the FP64 master state in either precision form; relative error <= 1e-10 against
  ``DGOracle.entropy_error`` (itself pinned to closed forms in test_oracle_functionals).
* Far field (reading: characteristic ghost state with supersonic branches): at Ma 1.5 the
  inlet is supersonic inflow (normal Mach <= -1, ghost state all free stream) and the outlet
  supersonic outflow (normal Mach >= 1, ghost state all interior); at Ma 0.97 perturbations
  put outlet points on both sides of Mach 1.  R and J v at <= 1e-12 (FP64) and 2e-5
  (FP32-mixed), J^T by the dot-product identity against the oracle's J v.
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


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_entropy_error_matches_oracle(capi, dim, p, precision):
    from oracle.cases import vortex_state
    from oracle.dg import DGOracle
    if dim == 2:
        mesh, free, L = W.periodic_square(8, 10.0, 0.15, 21), W.Freestream(0.5, 45.0), 10.0
    else:
        mesh, free, L = W.periodic_cube_kuhn(4, 10.0, 0.10, 5), W.Freestream(0.5, 45.0), 10.0
    vortex = W.Vortex(5.0, (5.0, 5.0))
    dg = DGOracle(mesh, p, free)
    u = dg.project(lambda x: vortex_state(x, free, vortex, period=L))
    u[:, -1, :] *= 1.1  # raise the energy: s / s0 about 1.1 (the vortex alone is isentropic)
    u = u.reshape(-1)
    prec = capi.PCEXP_FP64 if precision == "fp64" else capi.PCEXP_FP32_MIXED
    ctx = capi.Context(mesh, p, free, prec, m_max=2)
    ctx.set_state(u)
    got = ctx.output(1)
    want = dg.entropy_error(u, float(np.sum(dg.area)))
    assert want > 0.1
    assert abs(got - want) <= 1e-10 * want
    ctx.close()


def test_entropy_error_zero_in_free_stream(capi):
    mesh, free = W.bump_channel(16, 6, 0.15, 1), W.Freestream(0.5, 0.0)
    ctx = capi.Context(mesh, 2, free, capi.PCEXP_FP64, m_max=2)  # starts from the free stream
    assert ctx.output(1) < 1e-7
    ctx.close()


def _perturbed(dg, seed, amp):
    u = np.zeros((dg.E, dg.nv, dg.N))
    u[:, :, 0] = dg.freestream_state()[None, :] * np.sqrt(dg.area)[:, None]
    r = W.random_coeffs(seed, u.shape)
    return (u + amp * r * np.abs(u[:, :, :1])).reshape(-1)


def _normal_mach_range(dg, u):
    """Interior normal Mach numbers at the far-field face points (outward normals)."""
    from oracle import euler
    e, f, tag = dg.fb.T
    ff = tag == W.BC_FARFIELD
    U = np.einsum("fqi,fvi->fqv", dg.fb_psi[ff], np.asarray(u).reshape(dg.E, dg.nv, dg.N)[e[ff]])
    rho, vel, p, _ = euler.primitives(U, dg.gamma)
    vel = np.stack(vel, axis=-1) if isinstance(vel, (list, tuple)) else vel
    qn = np.einsum("fqd,fd->fq", vel, dg.fb_n[ff])
    c = np.sqrt(dg.gamma * p / rho)
    return (qn / c).min(), (qn / c).max()


@pytest.mark.parametrize("mach,amp", [(1.5, 0.05), (0.97, 0.08)])
@pytest.mark.parametrize("p", [1, 2])
def test_supersonic_farfield_branches(capi, mach, amp, p):
    from oracle.dg import DGOracle
    mesh, free = W.bump_channel(16, 6, 0.15, 1), W.Freestream(mach, 0.0)
    dg = DGOracle(mesh, p, free)
    u = _perturbed(dg, 300 + p, amp)
    lo, hi = _normal_mach_range(dg, u)
    if mach > 1:
        assert lo <= -1.0 and hi >= 1.0  # supersonic inflow and outflow points exist
    else:
        assert hi > 1.0 and np.sort([lo, hi])[0] < 0  # outlet points on both sides of Mach 1
    v = W.random_coeffs(400 + p, (dg.K,))
    w = W.random_coeffs(500 + p, (dg.K,))
    Ro, Jo = dg.residual(u), dg.jvp(u, v)
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=2)
    assert rel(ctx.residual(u), Ro) <= 1e-12
    assert rel(ctx.jvp(u, v), Jo) <= 1e-12
    JTw = ctx.vjp(u, w)
    assert abs(np.dot(JTw, v) - np.dot(w, Jo)) <= 1e-11 * np.linalg.norm(w) * np.linalg.norm(Jo)
    ctx.close()
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP32_MIXED, m_max=2)
    assert rel(ctx.residual(u), Ro) <= 2e-5
    assert rel(ctx.jvp(u, v), Jo) <= 2e-5
    ctx.close()
