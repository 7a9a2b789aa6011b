"""pcexp_residual_noalloc: the residual entry point for callers that cannot allocate device
memory when they need R(U) (a host whose own pool owns all device memory, a fixed memory
budget, a real-time loop that may not call cudaMalloc after set-up).  It must give what
pcexp_residual gives, call after call, while its face-flux scratch lives in the library's
fixed device array.  Collected last on purpose, so that a run stopping at the first failure
has run every other test first.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _freestream_like(ctx, free, seed):
    """Near-free-stream internal-basis coefficients with seeded perturbations."""
    c = np.sqrt(free.gamma * free.p / free.rho) * free.mach
    a = np.deg2rad(free.alpha_deg)
    vel = [c * np.cos(a), c * np.sin(a)] + ([0.0] if ctx.nv == 5 else [])
    state = np.array([free.rho] + [free.rho * v for v in vel]
                     + [free.p / (free.gamma - 1) + 0.5 * free.rho * c * c])
    u = np.zeros((ctx.E, ctx.nv, ctx.nb))
    u[:, :, 0] = state  # constant mode (the internal basis is orthonormal per element)
    u[:, :, 0] *= 1.0 + 0.02 * W.random_coeffs(seed, (ctx.E, 1))
    u[:, :, 1:] = 0.01 * W.random_coeffs(seed + 10, u[:, :, 1:].shape)
    return u.reshape(-1)


def _two_calls_match(ctx, free, seed):
    import torch
    for call in range(2):
        ud = torch.from_numpy(_freestream_like(ctx, free, seed + call)).cuda()
        ref = torch.empty_like(ud)
        got = torch.full_like(ud, float("nan"))
        ctx.residual(ud, ref)
        ctx.residual_noalloc(ud, got)
        ctx.synchronize()
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b), call


def test_residual_noalloc_matches_residual_two_calls():
    pytest.importorskip("torch")
    from paper_1801_06300_gb300 import build
    build()
    from paper_1801_06300_gb300 import capi
    case = W.case_bump2d()  # 37,120 faces x 3 points x 4 variables fits the 2^20-double scratch
    ctx = capi.Context(case.mesh, case.p, case.free, capi.PCEXP_FP64, m_max=2,
                       basis_io=capi.PCEXP_BASIS_INTERNAL)
    _two_calls_match(ctx, case.free, 40)
    ctx.close()


def test_residual_noalloc_matches_residual_tetrahedra():
    """Tetrahedra: the face rule's points (7 at P2) and 5 variables per face point in the size
    check and the scratch layout; 12^3 Kuhn cubes at P2 (20,736 faces x 7 x 5 doubles) fit."""
    pytest.importorskip("torch")
    from paper_1801_06300_gb300 import build
    build()
    from paper_1801_06300_gb300 import capi
    mesh = W.periodic_cube_kuhn(12, 10.0, 0.10, 5)
    free = W.Freestream(0.5, 45.0)
    ctx = capi.Context(mesh, 2, free, capi.PCEXP_FP64, m_max=2, basis_io=capi.PCEXP_BASIS_INTERNAL)
    _two_calls_match(ctx, free, 60)
    ctx.close()


def test_residual_noalloc_rejects_oversized_meshes():
    torch = pytest.importorskip("torch")
    from paper_1801_06300_gb300 import build
    build()
    from paper_1801_06300_gb300 import capi
    # 256 x 256 split quads at P3: 196,608 faces x 4 points x 4 variables > 2^20 doubles
    mesh = W.periodic_square(256, 20.0)
    ctx = capi.Context(mesh, 3, W.Freestream(0.5, 45.0), capi.PCEXP_FP64, m_max=1,
                       basis_io=capi.PCEXP_BASIS_INTERNAL)
    u = torch.zeros(ctx.K, dtype=torch.float64, device="cuda")
    r = torch.zeros_like(u)
    with pytest.raises(capi.PcexpError) as ei:
        ctx.residual_noalloc(u, r)
    assert ei.value.code == capi.PCEXP_ERR_INVALID_ARG
    assert "face-flux scratch too small" in str(ei.value)
    ctx.close()
