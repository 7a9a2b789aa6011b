"""pcexp_residual_noalloc: the residual entry point for callers that cannot allocate
device memory at call time (inside stream capture, under a fixed memory budget or a
custom allocator).  It must give what pcexp_residual gives, call after call, while its
face-flux scratch lives in the library's fixed device array.  Collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_residual_noalloc_matches_residual_two_calls():
    torch = pytest.importorskip("torch")
    from paper_1801_06300_gb300 import build
    build()
    from paper_1801_06300_gb300 import capi
    case = W.case_bump2d()  # 37,120 faces x 3 points x 4 variables fits the 2^20-double scratch
    ctx = capi.Context(case.mesh, case.p, case.free, capi.PCEXP_FP64, m_max=2,
                       basis_io=capi.PCEXP_BASIS_INTERNAL)
    sq = np.zeros((ctx.E, ctx.nv, ctx.nb))
    free = case.free
    c = np.sqrt(free.gamma * free.p / free.rho) * free.mach
    state = np.array([free.rho, free.rho * c, 0.0, free.p / (free.gamma - 1) + 0.5 * free.rho * c * c])
    for call in range(2):
        u = np.zeros_like(sq)
        u[:, :, 0] = state  # constant mode (internal basis is orthonormal per element)
        u[:, :, 0] *= 1.0 + 0.02 * W.random_coeffs(40 + call, (ctx.E, 1))
        u[:, :, 1:] = 0.01 * W.random_coeffs(50 + call, u[:, :, 1:].shape)
        ud = torch.from_numpy(u.reshape(-1)).cuda()
        ref = torch.empty_like(ud)
        got = torch.full_like(ud, float("nan"))
        ctx.residual(ud, ref)
        ctx.residual_noalloc(ud, got)
        ctx.synchronize()
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b), call
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
    ctx.close()
