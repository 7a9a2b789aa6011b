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


@pytest.mark.parametrize("k,scale", [(1, 0.7), (6, 2.0), (20, 8.0)])
def test_phi_adjoint_against_oracle_differences(capi, k, scale):
    """Hbar = (dy/dH)^T ybar for y = phi_1(dt H) e_1: GPU Frechet-derivative form against
    central differences of the oracle's Taylor/long-double phi."""
    from oracle.krylov import phi_e1
    rng = np.random.default_rng(k)
    H = np.triu(rng.standard_normal((k, k)), -1) * scale / np.sqrt(k) - 0.5 * scale * np.eye(k)
    ybar = rng.standard_normal(k)
    dt = 0.6
    mesh, p, free = CASES["periodic_p2"]()
    ctx = capi.Context(mesh, 0, free, capi.PCEXP_FP64, m_max=4)
    Hb = ctx.phi_adjoint(H, dt, ybar)
    h = 1e-6 * scale
    fd = np.zeros_like(H)
    for i in range(k):
        for j in range(k):
            E = np.zeros_like(H)
            E[i, j] = h
            fd[i, j] = ybar @ (phi_e1(H + E, dt)[0] - phi_e1(H - E, dt)[0]) / (2 * h)
    assert np.linalg.norm(Hb - fd) <= 1e-7 * np.linalg.norm(fd)
    ctx.close()


STEP_CASES = {
    "vortex_p1": lambda: (W.periodic_square(4, 10.0, 0.1, 5), 1, W.Freestream(0.5, 45.0), 0.4, 8),
    "bump_p2": lambda: (W.bump_channel(6, 3, 0.15, 1), 2, W.Freestream(0.5, 0.0), 0.02, 10),
}


def step_fixture(name):
    from oracle.dg import DGOracle
    mesh, p, free, dt, m = STEP_CASES[name]()
    dg = DGOracle(mesh, p, free)
    u = state(dg, 11, 0.05)
    return dg, mesh, p, free, dt, m, u


@pytest.mark.parametrize("name", list(STEP_CASES))
def test_step_backward_directional_against_oracle(capi, name):
    """delta . ubar_n equals the central difference of g . PCEXP(u_n) (oracle step, Eq. s9/s10)."""
    from oracle import pcexp
    dg, mesh, p, free, dt, m, u = step_fixture(name)
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=m)
    g = W.random_coeffs(12, (dg.K,))
    ub = ctx.step_backward(u, dt, m, g)

    def J(x):
        return g @ pcexp.pcexp_step(x, dg.residual, dg.jvp, dt, m)[0]

    for seed in (13, 14, 15):
        delta = W.random_coeffs(seed, (dg.K,)) * np.abs(u)
        h = 1e-5
        fd = (J(u + h * delta) - J(u - h * delta)) / (2 * h)
        got = ub @ delta
        assert abs(got - fd) <= 1e-4 * abs(fd), (seed, got, fd)
    ctx.close()


def test_step_backward_full_gradient_dense(capi):
    """Whole gradient on a tiny mesh against the oracle's finite-difference step Jacobian."""
    from oracle import pcexp
    from oracle.dg import DGOracle
    mesh, p, free = W.periodic_square(3, 3.0, 0.1, 2), 0, W.Freestream(0.4, 20.0)
    dg = DGOracle(mesh, p, free)
    u = state(dg, 21, 0.1)
    dt, m = 0.05, 6
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=m)
    g = W.random_coeffs(22, (dg.K,))
    ub = ctx.step_backward(u, dt, m, g)
    ref = np.zeros(dg.K)
    for i in range(dg.K):
        h = 1e-6 * max(abs(u[i]), 1.0)
        e = np.zeros(dg.K)
        e[i] = h
        ref[i] = g @ (pcexp.pcexp_step(u + e, dg.residual, dg.jvp, dt, m)[0]
                      - pcexp.pcexp_step(u - e, dg.residual, dg.jvp, dt, m)[0]) / (2 * h)
    assert np.linalg.norm(ub - ref) <= 1e-4 * np.linalg.norm(ref)
    ctx.close()


@pytest.mark.parametrize("name", list(STEP_CASES))
def test_step_backward_against_gpu_forward_differences(capi, name):
    """Self-consistency: the reverse step against central differences of the GPU's own step."""
    dg, mesh, p, free, dt, m, u = step_fixture(name)
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP64, m_max=m)
    g = W.random_coeffs(31, (dg.K,))
    ub = ctx.step_backward(u, dt, m, g)

    def J(x):
        ctx.set_state(x)
        ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, dt, m, info=False)
        return g @ ctx.get_state()

    delta = W.random_coeffs(32, (dg.K,)) * np.abs(u)
    h = 1e-5
    fd = (J(u + h * delta) - J(u - h * delta)) / (2 * h)
    assert abs(ub @ delta - fd) <= 1e-5 * abs(fd)
    ctx.close()


def test_wall_force_functional_matches_oracle(capi):
    from oracle.dg import DGOracle
    torch = pytest.importorskip("torch")
    mesh, free = W.bump_channel(12, 4, 0.15, 1), W.Freestream(0.5, 0.0)
    dg = DGOracle(mesh, 2, free)
    ctx = capi.Context(mesh, 2, free, capi.PCEXP_FP64, m_max=2)
    u = state(dg, 41, 0.05)
    for kind, dirn in ((capi.PCEXP_FUNC_WALL_FX, (1.0, 0.0)), (capi.PCEXP_FUNC_WALL_FY, (0.0, 1.0))):
        g = np.empty(dg.K)
        val, _ = ctx.functional(kind, u, g)
        ref = dg.wall_force(u, dirn)
        assert abs(val - ref) <= 1e-13 * abs(ref)
        from oracle import adscalar as ad
        delta = W.random_coeffs(42, (dg.K,))
        dref = dg.wall_force(ad.Dual(u, delta), dirn).der
        assert abs(g @ delta - dref) <= 1e-12 * max(abs(dref), 1.0)
    ctx.close()


def test_autograd_rollout_gradient(capi):
    """torch.autograd through 4 PCEXP steps (checkpointed): gradient of the wall force with
    respect to the initial state against a central difference of the oracle rollout."""
    torch = pytest.importorskip("torch")
    from oracle import pcexp
    from oracle.dg import DGOracle
    from paper_1801_06300_gb300.autograd import PCEXPStep, WallForce, adjoint_rollout
    mesh, free = W.bump_channel(8, 4, 0.15, 1), W.Freestream(0.5, 0.0)
    dg = DGOracle(mesh, 1, free)
    dt, m, steps = 0.02, 10, 4
    ctx = capi.Context(mesh, 1, free, capi.PCEXP_FP64, m_max=m)
    u0 = state(dg, 51, 0.02)
    x = torch.tensor(u0, device="cuda", requires_grad=True)
    theta = torch.tensor([free.mach, free.alpha_deg], dtype=torch.float64, device="cuda")
    u = x
    for _ in range(steps):
        u = PCEXPStep.apply(u, theta, ctx, free, dt, m)
    J = WallForce.apply(u, ctx, capi.PCEXP_FUNC_WALL_FX)
    J.backward()
    g = x.grad.cpu().numpy()

    def J_oracle(v):
        for _ in range(steps):
            v, _ = pcexp.pcexp_step(v, dg.residual, dg.jvp, dt, m)
        return dg.wall_force(v)

    assert abs(J.item() - J_oracle(u0)) <= 1e-10 * abs(J_oracle(u0))
    for seed in (52, 53):
        delta = W.random_coeffs(seed, (dg.K,)) * np.abs(u0)
        h = 1e-5
        fd = (J_oracle(u0 + h * delta) - J_oracle(u0 - h * delta)) / (2 * h)
        assert abs(g @ delta - fd) <= 1e-4 * abs(fd)
    # the explicit reverse loop gives the same gradient
    res = adjoint_rollout(ctx, torch.tensor(u0, device="cuda"), dt, m, steps)
    assert np.allclose(res.grad_u0.cpu().numpy(), g, rtol=1e-12, atol=1e-14 * np.abs(g).max())
    ctx.close()


def test_freestream_parameter_gradients(capi):
    """dJ/dMach and dJ/dalpha from the adjoint rollout (library reverse steps with their
    theta adjoint, the projection adjoint of the initial state) against central differences
    of the whole GPU rollout, and the same gradient through torch.autograd."""
    torch = pytest.importorskip("torch")
    import dataclasses
    from paper_1801_06300_gb300.autograd import PCEXPStep, ProjectedState, WallForce, adjoint_rollout
    mesh, free = W.bump_channel(8, 4, 0.15, 1), W.Freestream(0.5, 2.0)
    dt, m, steps = 0.02, 10, 3
    ctx = capi.Context(mesh, 1, free, capi.PCEXP_FP64, m_max=m)

    def u_init(fr):
        ctx.set_physics(fr)
        ctx.project_state(capi.PCEXP_PROJ_FREESTREAM)
        return ctx.get_state(torch.empty(ctx.K, dtype=torch.float64, device="cuda"))

    u0 = u_init(free)
    res = adjoint_rollout(ctx, u0, dt, m, steps, initial=(capi.PCEXP_PROJ_FREESTREAM, []))

    def J_of(fr):
        u = u_init(fr)
        for _ in range(steps):
            ctx.set_state(u)
            ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, dt, m, info=False)
            u = ctx.get_state(torch.empty_like(u))
        return ctx.functional(capi.PCEXP_FUNC_WALL_FX, u)[0]

    for name, h in (("mach", 1e-4), ("alpha_deg", 1e-2)):
        th = getattr(free, name)
        fd = (J_of(dataclasses.replace(free, **{name: th + h})) - J_of(dataclasses.replace(free, **{name: th - h}))) / (2 * h)
        assert abs(res.grad_params[name] - fd) <= 1e-4 * abs(fd) + 1e-12, (name, res.grad_params[name], fd)
    # torch.autograd: theta as a leaf through the projection, the steps and the functional
    theta = torch.tensor([free.mach, free.alpha_deg], dtype=torch.float64, device="cuda", requires_grad=True)
    u = ProjectedState.apply(theta, ctx, free, capi.PCEXP_PROJ_FREESTREAM, [])
    for _ in range(steps):
        u = PCEXPStep.apply(u, theta, ctx, free, dt, m)
    WallForce.apply(u, ctx, capi.PCEXP_FUNC_WALL_FX).backward()
    g = theta.grad.cpu().numpy()
    assert abs(g[0] - res.grad_params["mach"]) <= 1e-10 * abs(g[0])
    assert abs(g[1] - res.grad_params["alpha_deg"]) <= 1e-10 * abs(g[1])
    ctx.close()


def test_rollout_gradients_match_oracle_complex_step(capi):
    """The whole gradient of J(u_N) (wall force after 3 PCEXP steps on a 8 x 4 bump, P1,
    m = 10, from the projected free stream plus a fixed perturbation) against the oracle's
    complex step through the same rollout: a state direction of u_0, the Mach number and the
    flow angle (the far-field ghost state in every R and J v, and the initial state)."""
    torch = pytest.importorskip("torch")
    import dataclasses
    from oracle import pcexp
    from oracle.cases import freestream_state
    from oracle.dg import DGOracle
    from paper_1801_06300_gb300.autograd import adjoint_rollout
    mesh, free = W.bump_channel(8, 4, 0.15, 1), W.Freestream(0.5, 2.0)
    dt, m, steps = 0.02, 10, 3
    pert = 0.03 * W.random_coeffs(5, (mesh.n_elem * 4 * 3,))

    def J_oracle(fr, du=None):
        dg = DGOracle(mesh, 1, fr)
        u = dg.project(lambda x: freestream_state(x, fr)).reshape(-1) + pert
        if du is not None:
            u = u + du
        for _ in range(steps):
            u, _ = pcexp.pcexp_step(u, dg.residual, dg.jvp, dt, m)
        return dg.wall_force(u, (1.0, 0.0))

    ctx = capi.Context(mesh, 1, free, capi.PCEXP_FP64, m_max=m)
    ctx.project_state(capi.PCEXP_PROJ_FREESTREAM)
    u0 = ctx.get_state(torch.empty(ctx.K, dtype=torch.float64, device="cuda")) + torch.tensor(pert, device="cuda")
    res = adjoint_rollout(ctx, u0, dt, m, steps, initial=(capi.PCEXP_PROJ_FREESTREAM, []))
    assert abs(res.value - float(np.real(J_oracle(free)))) <= 1e-10 * abs(res.value)
    h = 1e-30
    delta = W.random_coeffs(6, (ctx.K,))
    cs_u = np.imag(J_oracle(free, 1j * h * delta)) / h
    assert abs(float(torch.dot(res.grad_u0, torch.tensor(delta, device="cuda"))) - cs_u) <= 1e-8 * abs(cs_u)
    for name in ("mach", "alpha_deg"):
        th = getattr(free, name)
        cs = np.imag(J_oracle(dataclasses.replace(free, **{name: th + 1j * h}))) / h
        assert abs(res.grad_params[name] - cs) <= 1e-8 * abs(cs), (name, res.grad_params[name], cs)
    ctx.close()
