"""Re-orthogonalisation of the Arnoldi process (Sec. 2.2, Eq. vm-vm2) through the C interface.

PCEXP_REORTH_ALWAYS runs the second classical Gram-Schmidt pass on every column (CGS2);
PCEXP_REORTH_SELECTIVE, the FP32-mixed form's default, runs it only where the first pass
cancelled, ||w_1|| < ||w|| / sqrt(2) (Daniel, Gragg, Kaufman & Stewart 1976).  On the DG
Euler operator ||w_1|| / ||w|| sits near 0.72 (the operator is close to skew-symmetric, so
w = J v_j has about half its energy on v_{j-1} and v_j), and most columns keep the first pass.

* the step info reports which columns ran the second pass: all of them for FP64 contexts and
  for ALWAYS, fewer for SELECTIVE;
* SELECTIVE: the Arnoldi relation J V_k = V_{k+1} H~_k and the orthonormality of V hold to
  FP32 rounding, the first columns of H match the oracle's Arnoldi (MGS with a full second
  pass), and PCEXP steps match both the two-pass FP32-mixed context and the FP64 oracle within
  the form's stated error;
* partitioned runs take the decision from the partition-summed norms, so every partition
  takes it alike, and a two-partition group matches one context.
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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def all_cols(k):
    return (1 << k) - 1


def bits(x):
    return bin(x).count("1")


MESHES = {
    "vortex2d_p2": lambda: (W.periodic_square(12, 10.0, 0.15, 3), 2, W.Freestream(0.5, 45.0)),
    "cube3d_p2": lambda: (W.periodic_cube_kuhn(4, 10.0, 0.1, 21), 2, W.Freestream(0.5, 30.0)),
}


def vortex_start(dg, free):
    from oracle.cases import vortex_state
    vx = W.Vortex(5.0, (5.0, 5.0))
    return dg.project(lambda x: vortex_state(x, free, vx, period=10.0)).reshape(-1)


def test_fp64_and_always_run_the_second_pass_on_every_column(capi):
    mesh, p, free = MESHES["cube3d_p2"]()
    for prec, reorth in ((capi.PCEXP_FP64, capi.PCEXP_REORTH_AUTO), (capi.PCEXP_FP64, capi.PCEXP_REORTH_ALWAYS),
                         (capi.PCEXP_FP32_MIXED, capi.PCEXP_REORTH_ALWAYS)):
        ctx = capi.Context(mesh, p, free, prec, m_max=12, reorth=reorth)
        ctx.project_state(capi.PCEXP_PROJ_VORTEX, [5.0, 5.0, 5.0, 10.0])
        info = ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, 10.0, 12)
        assert info["k"] == (12, 12)
        assert info["reorth_cols"] == (all_cols(12), all_cols(12)), (prec, reorth)
        ctx.close()


@pytest.mark.parametrize("name", list(MESHES))
def test_selective_arnoldi_relation_orthonormality_and_oracle(capi, name):
    from oracle.dg import DGOracle
    from oracle.krylov import arnoldi
    mesh, p, free = MESHES[name]()
    dg = DGOracle(mesh, p, free)
    u = vortex_start(dg, free)
    b = dg.residual(u)
    m = 24
    ctx = capi.Context(mesh, p, free, capi.PCEXP_FP32_MIXED, m_max=m, reorth=capi.PCEXP_REORTH_SELECTIVE)
    V, H, k, beta = ctx.arnoldi(u, b, m)
    assert k == m and np.all(np.isfinite(H))
    assert abs(beta - np.linalg.norm(b)) <= 1e-6 * beta
    # orthonormal to FP32 rounding
    assert np.abs(V @ V.T - np.eye(m + 1)).max() <= 1e-5
    # J V_m = V_{m+1} H~_m, column by column, with the library's FP32 J v
    for j in range(m):
        jv = ctx.jvp(u, V[j])
        assert rel(H[: j + 2, j] @ V[: j + 2], jv) <= 2e-5, j
    # the first columns against the oracle's Arnoldi (later columns of any FP32 Krylov basis
    # drift from the FP64 one by amplified rounding)
    Vo, Ho, ko, _, _ = arnoldi(lambda x: dg.jvp(u, x), b, m)
    assert ko == m
    assert rel(H[:6, :5], Ho[:6, :5]) <= 1e-4
    ctx.close()


def test_selective_steps_match_two_pass_and_oracle(capi):
    """Four PCEXP steps at CFL 10, m = 20 on the jittered periodic 4^3 Kuhn mesh at P2."""
    from oracle import pcexp
    from oracle.dg import DGOracle
    mesh, p, free = MESHES["cube3d_p2"]()
    dg = DGOracle(mesh, p, free)
    u0 = vortex_start(dg, free)
    m = 20
    sel = capi.Context(mesh, p, free, capi.PCEXP_FP32_MIXED, m_max=m)  # AUTO: selective
    two = capi.Context(mesh, p, free, capi.PCEXP_FP32_MIXED, m_max=m, reorth=capi.PCEXP_REORTH_ALWAYS)
    sel.set_state(u0)
    two.set_state(u0)
    u = u0.copy()
    passes = cols = 0
    for n in range(4):
        dt = float(np.min(dg.local_dt(u, 10.0)))
        u, info = pcexp.pcexp_step(u, dg.residual, dg.jvp, dt, m)
        a = sel.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, dt, m)
        b = two.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, dt, m)
        assert a["k"] == b["k"] == (info["k1"], info["k2"])
        assert b["reorth_cols"] == (all_cols(m), all_cols(m))
        passes += bits(a["reorth_cols"][0]) + bits(a["reorth_cols"][1])
        cols += 2 * m
    print(f"selective: second pass on {passes} of {cols} columns")
    assert passes < cols // 2  # most columns keep the first pass
    s, t = sel.get_state(), two.get_state()
    assert rel(s, u0) > 1e-5  # the steps move the state
    assert rel(s, t) <= 2e-6
    es, et = rel(s, u), rel(t, u)
    print(f"FP32-mixed state error vs FP64 oracle after 4 steps: selective {es:.2e}, two passes {et:.2e}")
    assert es <= 1e-5 and es <= 2.0 * et + 1e-7
    sel.close()
    two.close()


def test_group_selective_matches_one_context(capi):
    mesh, p, free = MESHES["cube3d_p2"]()
    part = capi.partition(mesh, 2)
    one = capi.Context(mesh, p, free, capi.PCEXP_FP32_MIXED, m_max=16)
    grp = capi.Group(mesh, part, p, free, capi.PCEXP_FP32_MIXED, m_max=16)
    one.project_state(capi.PCEXP_PROJ_VORTEX, [5.0, 5.0, 5.0, 10.0])
    u = one.get_state()
    grp.set_state(u)
    for _ in range(2):
        a = one.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, 10.0, 16)
        b = grp.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GLOBAL_CFL, 10.0, 16)
        assert a["k"] == b["k"] == (16, 16)
        assert bits(b["reorth_cols"][0]) < 16 and bits(a["reorth_cols"][0]) < 16
    s1, sg = one.get_state(), grp.get_state()
    assert rel(s1, u) > 1e-5
    assert rel(sg, s1) <= 1e-6
    one.close()
    grp.close()
