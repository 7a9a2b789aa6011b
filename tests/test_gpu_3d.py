"""The CUDA path on tetrahedra (the 3D vortex case) against the FP64 oracle, element by
element, through the C interface: operators, projection, time steps, PCEXP steps,
adjoints and the vortex-error functional."""
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


def oracle_dg(mesh, p, free):
    from oracle.dg import DGOracle
    return DGOracle(mesh, p, free)


def perturbed_state(dg, seed, amp=0.05):
    u = np.zeros((dg.E, dg.nv, dg.N))
    u[:, :, 0] = dg.freestream_state()[None, :] * np.sqrt(dg.area)[:, None]
    r = W.random_coeffs(seed, u.shape)
    return (u + amp * r * np.abs(u[:, :, :1])).reshape(-1)


def walled_cube(n, seed):
    """Non-periodic jittered Kuhn cube: slip walls on z = 0 and z = L, far field elsewhere."""
    mesh = W.periodic_cube_kuhn(n, 1.0, 0.15, seed, periodic=False)
    z = mesh.coords[mesh.bfaces][:, :, 2]
    wall = np.all(np.abs(z) < 1e-12, axis=1) | np.all(np.abs(z - 1.0) < 1e-12, axis=1)
    mesh.btags = np.where(wall, W.BC_SLIP_WALL, W.BC_FARFIELD).astype(np.int32)
    return mesh


MESHES = {
    "periodic": lambda: (W.periodic_cube_kuhn(3, 10.0, 0.1, 21), W.Freestream(0.5, 30.0)),
    "walls": lambda: (walled_cube(3, 4), W.Freestream(0.5, 20.0)),
}


@pytest.mark.parametrize("kind", ["periodic", "walls"])
@pytest.mark.parametrize("p", [0, 1, 2])
def test_residual_and_jvp_fp64_3d(capi, kind, p):
    mesh, free = MESHES[kind]()
    dg = oracle_dg(mesh, p, free)
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=4)
    assert ctx.nv == 5 and ctx.K == dg.K
    u = perturbed_state(dg, 100 + p)
    v = W.random_coeffs(200 + p, (dg.K,))
    assert rel(ctx.residual(u), dg.residual(u)) <= 1e-12
    assert rel(ctx.jvp(u, v), dg.jvp(u, v)) <= 1e-12
    ctx.close()


def test_residual_and_jvp_fp32_mixed_3d(capi):
    mesh, free = MESHES["walls"]()
    dg = oracle_dg(mesh, 2, free)
    ctx = capi.Context(mesh, 2, free, capi.PCEXP_FP32_MIXED, m_max=4)
    u = perturbed_state(dg, 7)
    v = W.random_coeffs(8, (dg.K,))
    assert rel(ctx.residual(u), dg.residual(u)) <= 2e-5
    assert rel(ctx.jvp(u, v), dg.jvp(u, v)) <= 2e-5
    ctx.close()


@pytest.mark.parametrize("kind", ["periodic", "walls", "ragged48"])
@pytest.mark.parametrize("p", [0, 1, 2])
def test_fp32_krylov_jvp_matches_oracle_3d(capi, kind, p):
    """The J v inside the FP32-mixed Krylov process on tetrahedra (volume flux tangents
    recomputed per element, 32 elements per block) against the oracle's J v: 162 elements
    (five full blocks and a ragged one) or 48 (one full, one half).  With m = 1 the
    Arnoldi relation gives J v_0 = h_00 v_0 + h_10 v_1."""
    mesh, free = (walled_cube(2, 9), W.Freestream(0.5, 20.0)) if kind == "ragged48" else MESHES[kind]()
    dg = oracle_dg(mesh, p, free)
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP32_MIXED, m_max=2)
    u = perturbed_state(dg, 400 + p)
    b = W.random_coeffs(401 + p, (dg.K,))
    V, H, k, beta = ctx.arnoldi(u, b, 1)
    assert k == 1
    Jv = H[0, 0] * V[0] + H[1, 0] * V[1]
    assert rel(Jv, dg.jvp(u, V[0])) <= 2e-5
    ctx.close()


def test_order_above_two_is_unsupported_in_3d(capi):
    mesh, free = MESHES["periodic"]()
    with pytest.raises(capi.PcexpError) as ei:
        capi.Context(mesh, 3, free, capi.PCEXP_FP64, m_max=4)
    assert ei.value.code == capi.PCEXP_ERR_UNSUPPORTED


def test_vortex_projection_and_dt_3d(capi):
    from oracle.cases import vortex_state
    case = W.case_vortex3d(n=3)
    dg = oracle_dg(case.mesh, case.p, case.free)
    ctx = capi.Context(case.mesh, case.p, case.free, capi.PCEXP_FP64, m_max=4)
    ctx.project_state(capi.PCEXP_PROJ_VORTEX, [case.vortex.eps, *case.vortex.center, 10.0])
    uo = dg.project(lambda x: vortex_state(x, case.free, case.vortex, period=10.0)).reshape(-1)
    assert rel(ctx.get_state(), uo) <= 1e-13
    dte = ctx.compute_dt(3.0, local=True)
    assert rel(dte, dg.local_dt(uo, 3.0)) <= 1e-13
    ctx.close()


@pytest.mark.parametrize("p", [1, 2])
def test_pcexp_steps_vortex_3d_per_step(capi, p):
    """5 PCEXP steps at CFL 10, m = 12 on a jittered periodic 4^3 Kuhn mesh (384 tets)."""
    from oracle import pcexp
    from oracle.cases import vortex_state
    case = W.case_vortex3d(n=4, p=p)
    dg = oracle_dg(case.mesh, p, case.free)
    u0 = dg.project(lambda x: vortex_state(x, case.free, case.vortex, period=10.0)).reshape(-1)
    ctx = capi.Context(case.mesh, p, case.free, capi.PCEXP_FP64, m_max=12)
    ctx.set_state(u0)
    u = u0.copy()
    for n in range(5):
        dt = float(np.min(dg.local_dt(u, case.cfl)))
        u, info = pcexp.pcexp_step(u, dg.residual, dg.jvp, dt, 12)
        g = ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, case.cfl, 12)
        assert abs(g["dt"] - dt) <= 1e-13 * dt
        assert g["k"] == (info["k1"], info["k2"])
        assert rel(ctx.get_state(), u) <= 1e-10, n
    ctx.close()


def test_vjp_3d_dot_product_and_dense_transpose(capi):
    mesh, free = MESHES["walls"]()
    for p in (0, 1, 2):
        dg = oracle_dg(mesh, p, free)
        ctx = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=2)
        u = perturbed_state(dg, 1)
        v = W.random_coeffs(2, (dg.K,))
        w = W.random_coeffs(3, (dg.K,))
        Jv = ctx.jvp(u, v)
        JTw = ctx.vjp(u, w)
        assert abs(w @ Jv - JTw @ v) <= 1e-13 * (np.abs(w) @ np.abs(Jv))
        if p == 0:
            ref = dg.dense_jacobian(u).T @ w
            assert np.linalg.norm(JTw - ref) <= 1e-12 * np.linalg.norm(ref)
        ctx.close()


@pytest.mark.parametrize("kind,p", [("walls", 1), ("walls", 2), ("periodic", 2)])
def test_jvp_state_adjoint_3d_against_oracle_differences(capi, kind, p):
    mesh, free = MESHES[kind]()
    dg = oracle_dg(mesh, p, free)
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=2)
    u = perturbed_state(dg, 4)
    v = W.random_coeffs(5, (dg.K,))
    w = W.random_coeffs(6, (dg.K,))
    g = ctx.jvp_state_adjoint(u, v, w)
    for seed in (7, 8):
        delta = W.random_coeffs(seed, (dg.K,)) * np.abs(u) * 1e-2
        h = 1e-3
        fd = (w @ dg.jvp(u + h * delta, v) - w @ dg.jvp(u - h * delta, v)) / (2 * h)
        assert abs(g @ delta - fd) <= 1e-6 * abs(fd) + 1e-12 * np.abs(g) @ np.abs(delta)
    ctx.close()


@pytest.mark.parametrize("p", [1, 2])
def test_step_backward_3d_directional_against_oracle(capi, p):
    from oracle import pcexp
    case = W.case_vortex3d(n=3, p=p)
    dg = oracle_dg(case.mesh, p, case.free)
    u = perturbed_state(dg, 11, 0.05)
    dt, m = 0.3, 8
    ctx = capi.Context(case.mesh, p, case.free, capi.PCEXP_FP64, m_max=m)
    gT = W.random_coeffs(12, (dg.K,))
    ub = ctx.step_backward(u, dt, m, gT)

    def J(x):
        return gT @ pcexp.pcexp_step(x, dg.residual, dg.jvp, dt, m)[0]

    for seed in (13, 14):
        delta = W.random_coeffs(seed, (dg.K,)) * np.abs(u)
        h = 1e-5
        fd = (J(u + h * delta) - J(u - h * delta)) / (2 * h)
        assert abs(ub @ delta - fd) <= 1e-4 * abs(fd), (seed, ub @ delta, fd)
    ctx.close()


def test_vortex_error_functional_matches_oracle(capi):
    """||U_h - U_exact|| at t = 0.4 and its gradient (directional) against the oracle."""
    from oracle.adscalar import Dual
    from oracle.cases import vortex_state
    case = W.case_vortex3d(n=3, p=2)
    dg = oracle_dg(case.mesh, 2, case.free)
    u = dg.project(lambda x: vortex_state(x, case.free, case.vortex, period=10.0)).reshape(-1)
    u = u + 1e-3 * W.random_coeffs(9, u.shape) * np.abs(u)
    t = 0.4
    prm = [case.vortex.eps, *case.vortex.center, 10.0, t]
    ex = lambda x: vortex_state(x, case.free, case.vortex, t=t, period=10.0)  # noqa: E731
    ctx = capi.Context(case.mesh, 2, case.free, capi.PCEXP_FP64, m_max=2)
    grad = np.zeros(dg.K)
    val, _ = ctx.functional(capi.PCEXP_FUNC_VORTEX_L2, u, grad, params=prm)
    assert abs(val - dg.l2_error(u, ex)) <= 1e-12 * val
    for seed in (3, 4):
        d = W.random_coeffs(seed, (dg.K,))
        ref = dg.l2_error(Dual(u, d), ex).der
        assert abs(grad @ d - ref) <= 1e-11 * abs(ref)
    ctx.close()


def test_vortex3d_strength_gradient_small(capi):
    """dJ/deps of the vortex error after 5 steps on a 4^3 Kuhn mesh (P2, m = 10) by the
    adjoint rollout, against central differences of whole GPU rollouts."""
    torch = pytest.importorskip("torch")
    from paper_1801_06300_gb300.autograd import adjoint_rollout
    case = W.case_vortex3d(n=4, p=2)
    m, steps = 10, 5
    ctx = capi.Context(case.mesh, 2, case.free, capi.PCEXP_FP64, m_max=m)
    eps0, (xc, yc) = case.vortex.eps, case.vortex.center

    def init(eps):
        ctx.project_state(capi.PCEXP_PROJ_VORTEX, [eps, xc, yc, 10.0])
        return ctx.get_state(torch.empty(ctx.K, dtype=torch.float64, device="cuda"))

    u0 = init(eps0)
    ctx.set_state(u0)
    dt = ctx.compute_dt(case.cfl)
    T = steps * dt
    fparams = lambda eps: [eps, xc, yc, 10.0, T]  # noqa: E731
    res = adjoint_rollout(ctx, u0, dt, m, steps, kind=capi.PCEXP_FUNC_VORTEX_L2,
                          functional_params=fparams(eps0), initial=(capi.PCEXP_PROJ_VORTEX, [eps0, xc, yc, 10.0]))

    def J(x, eps):
        u = x
        for _ in range(steps):
            ctx.set_state(u)
            ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, dt, m, info=False)
            u = ctx.get_state(torch.empty_like(u))
        return ctx.functional(capi.PCEXP_FUNC_VORTEX_L2, u, None, params=fparams(eps))[0]

    delta = torch.tensor(W.random_coeffs(41, (ctx.K,)), device="cuda") * u0.abs()
    hu = 1e-6
    fdu = (J(u0 + hu * delta, eps0) - J(u0 - hu * delta, eps0)) / (2 * hu)
    gu = float(torch.dot(res.grad_u0, delta))
    # PCEXP uses the exact Jacobian, whose Roe part holds sign(q_n): wherever a face-point
    # wave speed crosses zero, J_n (and so the step) jumps.  The difference width is kept
    # below the distance to the nearest crossing (h = 1e-4 already straddles one here).
    h = 1e-6
    fd = (J(init(eps0 + h), eps0 + h) - J(init(eps0 - h), eps0 - h)) / (2 * h)
    print(f"small 3D: J = {res.value:.6e}; u0 direction {gu:.6e} vs {fdu:.6e}; "
          f"eps {res.grad_params['eps']:.6e} vs {fd:.6e}")
    assert abs(gu - fdu) <= 1e-4 * abs(fdu)
    assert abs(res.grad_params["eps"] - fd) <= 1e-4 * abs(fd)
    ctx.close()
