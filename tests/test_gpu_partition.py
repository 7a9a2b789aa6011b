"""Partitioned runs on the GPU (pcexp_group_*): 2 and 3 partitions of one mesh, all on device 0,
against one context on the whole mesh.

* R(u), J(u) v, and the adjoint passes J(u)^T w and (d(J(u) v)/du)^T w: each partition
  receives only its own rows; the halo rows come from the exchange kernel reading the owners'
  buffers.  A face keeps the whole mesh's L element and an element sums its faces in the same
  order, so R and J v equal the single context's bit for bit, the adjoint passes to 1e-14
  (their face terms are gathered per element in the submesh's face order).
* Arnoldi: the Gram-Schmidt sums are split over the partitions (partition order), so H matches
  to round-off (1e-13 relative) and every partition holds the same H (checked by the call).
* Steps (PCEXP at the global CFL dt, ETD2, EXP1): the same Krylov dimensions, dt to the last
  bit or two, and states within 1e-11 (FP64) after three steps; FP32-mixed within 1e-6 of the single FP32 context
  (the FP32 basis vectors round differently once the projections differ in their last bits).
"""
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


CASES = {
    "vortex2d": lambda: (W.periodic_square(16, 10.0, 0.15, 3), 1, W.Freestream(0.5, 45.0)),
    "bump2d": lambda: (W.bump_channel(24, 8, 0.1, 2), 2, W.Freestream(0.5, 0.0)),
    "cube3d": lambda: (W.periodic_cube_kuhn(4, 2.0, 0.1, 4), 2, W.Freestream(0.5, 30.0)),
}


def _state(ctx, seed):
    u = ctx.get_state().reshape(ctx.E, ctx.nv, ctx.nb)
    u = u + 0.03 * W.random_coeffs(seed, u.shape) * np.abs(u[:, :, :1])
    return u.reshape(-1)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name,n", [("vortex2d", 2), ("bump2d", 3), ("cube3d", 2), ("cube3d", 3)])
def test_group_operator_and_arnoldi(capi, name, n):
    mesh, p, free = CASES[name]()
    part = capi.partition(mesh, n)
    one = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=12)
    grp = capi.Group(mesh, part, p, free, capi.PCEXP_FP64, m_max=12)
    for k in range(n):
        own, halo = grp.sizes(k)
        assert own == int((part == k).sum()) and halo > 0
    u = _state(one, 1)
    v = W.random_coeffs(2, u.size)
    R1, Rg = one.residual(u), grp.residual(u)
    assert np.abs(Rg - R1).max() <= 1e-15 * np.abs(R1).max()
    J1, Jg = one.jvp(u, v), grp.jvp(u, v)
    assert np.abs(Jg - J1).max() <= 1e-15 * np.abs(J1).max()
    w = W.random_coeffs(3, u.size)
    A1, Ag = one.vjp(u, w), grp.vjp(u, w)
    assert np.abs(Ag - A1).max() <= 1e-14 * np.abs(A1).max()
    S1, Sg = one.jvp_state_adjoint(u, v, w), grp.jvp_state_adjoint(u, v, w)
    assert np.abs(Sg - S1).max() <= 1e-14 * np.abs(S1).max()
    m = 10
    H1 = one.arnoldi(u, v, m, want_V=False)
    Hg, kg, bg = grp.arnoldi(u, v, m)
    assert kg == H1[2] == m
    assert abs(bg - H1[3]) <= 1e-14 * H1[3]
    assert np.abs(Hg - H1[1]).max() <= 1e-13 * np.abs(H1[1]).max()
    one.close()
    grp.close()


@pytest.mark.parametrize("name,n,scheme", [("vortex2d", 2, "PCEXP"), ("bump2d", 3, "PCEXP"), ("cube3d", 3, "PCEXP"),
                                           ("vortex2d", 3, "ETD2"), ("bump2d", 2, "EXP1")])
def test_group_steps_match_one_context(capi, name, n, scheme):
    mesh, p, free = CASES[name]()
    sc = getattr(capi, f"PCEXP_SCHEME_{scheme}")
    part = capi.partition(mesh, n)
    one = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=12)
    grp = capi.Group(mesh, part, p, free, capi.PCEXP_FP64, m_max=12)
    u = _state(one, 3)
    one.set_state(u)
    grp.set_state(u)
    assert np.array_equal(grp.get_state(), one.get_state())
    for _ in range(3):
        a = one.step(sc, capi.PCEXP_DT_GLOBAL_CFL, 2.0, 12)
        b = grp.step(sc, capi.PCEXP_DT_GLOBAL_CFL, 2.0, 12)
        # dt: equal at the first step; later steps start from states that differ by the
        # rounding of the split Gram-Schmidt sums, so dt may differ in its last bits
        assert a["k"] == b["k"] and abs(a["dt"] - b["dt"]) <= 4e-16 * a["dt"]
        assert abs(a["res_norm"] - b["res_norm"]) <= 1e-12 * a["res_norm"]
        assert abs(a["beta"][0] - b["beta"][0]) <= 1e-13 * a["beta"][0]
    s1, sg = one.get_state(), grp.get_state()
    assert rel(s1, u) > 1e-5  # the steps move the state
    assert rel(sg, s1) <= 1e-11
    one.close()
    grp.close()


@pytest.mark.parametrize("name", ["cube3d", "bump2d"])
def test_group_fp32_mixed_step(capi, name):
    mesh, p, free = CASES[name]()
    part = capi.partition(mesh, 2)
    one = capi.Context(mesh, p, free, capi.PCEXP_FP32_MIXED, m_max=12)
    grp = capi.Group(mesh, part, p, free, capi.PCEXP_FP32_MIXED, m_max=12)
    u = _state(one, 4)
    one.set_state(u)
    grp.set_state(u)
    for _ in range(2):
        a = one.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, 2.0, 12)
        b = grp.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, 2.0, 12)
        assert a["k"] == b["k"] and abs(a["dt"] - b["dt"]) <= 1e-7 * a["dt"]
    s1, sg = one.get_state(), grp.get_state()
    assert rel(s1, u) > 1e-5
    assert rel(sg, s1) <= 1e-6
    one.close()
    grp.close()


def test_group_projection_and_rejected_modes(capi):
    mesh = W.periodic_square(12, 10.0, 0.1, 5)
    free = W.Freestream(0.5, 45.0)
    part = capi.partition(mesh, 2)
    one = capi.Context(mesh, 2, free, capi.PCEXP_FP64, m_max=8)
    grp = capi.Group(mesh, part, 2, free, capi.PCEXP_FP64, m_max=8)
    prm = [5.0, 5.0, 5.0, 0.0]
    one.project_state(capi.PCEXP_PROJ_VORTEX, prm)
    grp.project_state(capi.PCEXP_PROJ_VORTEX, prm)
    assert np.array_equal(grp.get_state(), one.get_state())
    with pytest.raises(capi.PcexpError) as e:
        grp.step(capi.PCEXP_SCHEME_ETD2, capi.PCEXP_DT_LOCAL_CFL, 10.0, 8)
    assert e.value.code == capi.PCEXP_ERR_INVALID_ARG
    # a failed call leaves the group usable
    grp.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, 0.01, 8)
    one.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, 0.01, 8)
    assert rel(grp.get_state(), one.get_state()) <= 1e-12
    one.close()
    grp.close()


@pytest.mark.parametrize("n,tol", [(2, 0.0), (3, 1e-5)])
def test_group_local_steps_and_steady_march(capi, n, tol):
    """Local time steps (each partition scales its own rows by its own elements' steps) and the
    steady march (norms summed over the partitions before the stop test and the CFL ramp; with
    a Krylov tolerance, the error cap from the shared estimate) against one context.  The march
    amplifies the rounding of the split Gram-Schmidt sums (7e-8 in the residual norm after 40
    iterations; with a Krylov tolerance a checkpoint decision can flip), so the comparison is
    tight over the first iterations: the same iterations and norms, states within 1e-10 after 5;
    without a tolerance the norms stay within 1e-6 over 40."""
    mesh, p, free = CASES["bump2d"]()
    part = capi.partition(mesh, n)
    one = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=12, krylov_tol=tol)
    grp = capi.Group(mesh, part, p, free, capi.PCEXP_FP64, m_max=12, krylov_tol=tol)
    u = _state(one, 5)
    one.set_state(u)
    grp.set_state(u)
    a = one.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_LOCAL_CFL, 10.0, 12)
    b = grp.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_LOCAL_CFL, 10.0, 12)
    assert a["k"] == b["k"] and b["dt"] == 1.0
    s1 = one.get_state()
    assert rel(s1, u) > 1e-6 and rel(grp.get_state(), s1) <= 1e-12
    one.project_state(capi.PCEXP_PROJ_FREESTREAM, [])
    grp.project_state(capi.PCEXP_PROJ_FREESTREAM, [])
    m1 = one.march_steady(capi.PCEXP_SCHEME_PCEXP, 10.0, 10.0, 5, 12)
    mg = grp.march_steady(capi.PCEXP_SCHEME_PCEXP, 10.0, 10.0, 5, 12)
    assert mg["iterations"] == m1["iterations"] == 5
    assert abs(mg["res_first"] - m1["res_first"]) <= 1e-13 * m1["res_first"]
    assert abs(mg["res_last"] - m1["res_last"]) <= 1e-10 * m1["res_last"]
    assert m1["res_last"] != m1["res_first"]
    assert rel(grp.get_state(), one.get_state()) <= 1e-10
    if tol == 0.0:
        m1 = one.march_steady(capi.PCEXP_SCHEME_PCEXP, 10.0, 10.0, 35, 12)
        mg = grp.march_steady(capi.PCEXP_SCHEME_PCEXP, 10.0, 10.0, 35, 12)
        assert mg["iterations"] == m1["iterations"] == 35
        assert abs(mg["res_last"] - m1["res_last"]) <= 1e-6 * m1["res_last"]
    one.close()
    grp.close()


@pytest.mark.parametrize("name,n", [("bump2d", 2), ("bump2d", 3), ("cube3d", 2)])
def test_group_step_backward_matches_one_context(capi, name, n):
    """The reverse step partitioned (the forward step recomputed partitioned, every reduction of
    the reverse Gram-Schmidt summed over the partitions before its finishing step, the adjoint
    operator passes with exchanged inputs, theta_bar summed over the partitions' own elements)
    against one context: ubar_n within 1e-11 and the free-stream parameter adjoint within
    1e-11 relative (far-field faces in the channel; none in the periodic cube)."""
    mesh, p, free = CASES[name]()
    part = capi.partition(mesh, n)
    one = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=8)
    grp = capi.Group(mesh, part, p, free, capi.PCEXP_FP64, m_max=8)
    u = _state(one, 7)
    ub = W.random_coeffs(8, u.size)
    dt = 0.002
    a, ta = one.step_backward(u, dt, 8, ub, with_theta=True)
    b, tb = grp.step_backward(u, dt, 8, ub)
    assert rel(b, a) <= 1e-11
    if name == "bump2d":
        assert np.all(np.abs(ta) > 0)
        assert np.abs(tb - ta).max() <= 1e-11 * np.abs(ta).max()
    else:
        assert np.abs(tb).max() <= 1e-14 and np.abs(ta).max() <= 1e-14
    one.close()
    grp.close()


def test_group_of_one_partition_is_the_single_context(capi):
    """A group of one partition (no halo, no exchange partner) reproduces the single context
    exactly: the same mesh order, the same kernels, sums over one partition."""
    mesh, p, free = CASES["vortex2d"]()
    part = np.zeros(mesh.n_elem, np.int32)
    one = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=8)
    grp = capi.Group(mesh, part, p, free, capi.PCEXP_FP64, m_max=8)
    assert grp.sizes(0) == (mesh.n_elem, 0)
    u = _state(one, 9)
    one.set_state(u)
    grp.set_state(u)
    assert np.array_equal(grp.residual(u), one.residual(u))
    for _ in range(2):
        a = one.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, 2.0, 8)
        b = grp.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, 2.0, 8)
        assert a["k"] == b["k"] and a["dt"] == b["dt"]
    assert rel(grp.get_state(), one.get_state()) <= 1e-14
    one.close()
    grp.close()
