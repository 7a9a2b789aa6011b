"""Faults injected from the host, checked at the C interface.

* Non-conforming meshes (a face shared by three elements, an untagged boundary face, an
  inverted element, a vertex index out of range) and invalid options are rejected by
  pcexp_create before any device work: PCEXP_ERR_MESH / PCEXP_ERR_INVALID_ARG with a
  pcexp_last_error text.  These run without a GPU (host set-up only).
* A non-finite state (a NaN written into one coefficient from the host) makes the next step
  return PCEXP_ERR_NONFINITE: the Krylov norm is flagged on the device and read back at the
  step's synchronising call; the context stays usable.  NaN arithmetic is not a GPU fault.
"""
import dataclasses
import shutil
import os

import numpy as np
import pytest

import workloads as W


def _lib_or_skip():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit to build the library")
    from paper_1801_06300_gb300 import build
    build()
    from paper_1801_06300_gb300 import capi
    return capi


def _create_error(capi, mesh, p=1, **kw):
    with pytest.raises(capi.PcexpError) as ei:
        capi.Context(mesh, p, W.Freestream(0.5, 0.0), stream=0, **kw)
    return ei.value


def _two_triangles_plus_one():
    """Three triangles on the edge (0, 1): a face shared by more than two elements."""
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 1.0], [0.5, -1.0], [0.5, 2.0]])
    elems = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]], np.int32)
    bf = np.array([[1, 2], [2, 0], [0, 3], [3, 1], [1, 4], [4, 0]], np.int32)
    return W.Mesh(2, coords, elems, np.arange(5, dtype=np.int32), bf,
                  np.full(len(bf), W.BC_FARFIELD, np.int32))


def test_face_shared_by_three_elements_is_a_mesh_error():
    capi = _lib_or_skip()
    e = _create_error(capi, _two_triangles_plus_one())
    assert e.code == capi.PCEXP_ERR_MESH
    assert "more than two" in str(e)


def test_untagged_boundary_face_is_a_mesh_error():
    """A periodic square without its periodic identification leaves untagged boundary edges."""
    capi = _lib_or_skip()
    mesh = W.periodic_square(4, 1.0)
    mesh = dataclasses.replace(mesh, vert_master=np.arange(mesh.n_vert, dtype=np.int32))
    e = _create_error(capi, mesh)
    assert e.code == capi.PCEXP_ERR_MESH
    assert "no tag" in str(e)


def test_inverted_element_is_a_mesh_error():
    capi = _lib_or_skip()
    mesh = W.periodic_square(3, 1.0)
    elems = mesh.elems.copy()
    elems[4, 1], elems[4, 2] = elems[4, 2], elems[4, 1]  # clockwise
    e = _create_error(capi, dataclasses.replace(mesh, elems=elems))
    assert e.code == capi.PCEXP_ERR_MESH
    assert "inverted" in str(e)


def test_vertex_out_of_range_is_a_mesh_error():
    capi = _lib_or_skip()
    mesh = W.periodic_square(3, 1.0)
    elems = mesh.elems.copy()
    elems[0, 0] = mesh.n_vert + 7
    e = _create_error(capi, dataclasses.replace(mesh, elems=elems))
    assert e.code == capi.PCEXP_ERR_MESH


@pytest.mark.parametrize("kw", [dict(m_max=0), dict(m_max=33), dict(precision=7), dict(basis_io=5),
                                dict(reorth=3), dict(reorth=-1)])
def test_invalid_options_are_rejected(kw):
    capi = _lib_or_skip()
    e = _create_error(capi, W.periodic_square(3, 1.0), **kw)
    assert e.code == capi.PCEXP_ERR_INVALID_ARG


def test_selective_reorthogonalisation_is_not_offered_in_fp64():
    """The FP64 form keeps both Gram-Schmidt passes (its reverse step replays them)."""
    capi = _lib_or_skip()
    e = _create_error(capi, W.periodic_square(3, 1.0), precision=capi.PCEXP_FP64,
                      reorth=capi.PCEXP_REORTH_SELECTIVE)
    assert e.code == capi.PCEXP_ERR_UNSUPPORTED
    assert "FP32-mixed" in str(e)


def test_order_beyond_support_is_rejected():
    capi = _lib_or_skip()
    e = _create_error(capi, W.periodic_square(3, 1.0), p=4)
    assert e.code == capi.PCEXP_ERR_INVALID_ARG
    e = _create_error(capi, W.periodic_cube_kuhn(2, 1.0), p=3)
    assert e.code == capi.PCEXP_ERR_UNSUPPORTED


# ------------------------------------------------------------------ on the GPU
@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nan_state_gives_nonfinite_and_context_recovers(precision):
    pytest.importorskip("torch")
    capi = _lib_or_skip()
    case = W.case_vortex2d_small(8)
    prec = capi.PCEXP_FP64 if precision == "fp64" else capi.PCEXP_FP32_MIXED
    ctx = capi.Context(case.mesh, case.p, case.free, prec, m_max=case.m)
    ctx.project_state(capi.PCEXP_PROJ_VORTEX, [case.vortex.eps, *case.vortex.center, 10.0])
    good = ctx.get_state()
    bad = good.copy()
    bad[5 * ctx.nv * ctx.nb + 2] = np.nan
    ctx.set_state(bad)
    with pytest.raises(capi.PcexpError) as ei:
        ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, 0.05, case.m)
    assert ei.value.code == capi.PCEXP_ERR_NONFINITE
    # the Arnoldi entry point flags a non-finite start vector the same way
    with pytest.raises(capi.PcexpError) as ei:
        ctx.arnoldi(good, bad, 4, want_V=False)
    assert ei.value.code == capi.PCEXP_ERR_NONFINITE
    # the context stays usable: a finite state steps normally
    ctx.set_state(good)
    info = ctx.step(capi.PCEXP_SCHEME_PCEXP, capi.PCEXP_DT_GIVEN, 0.05, case.m)
    assert info["k"][0] > 0 and np.all(np.isfinite(ctx.get_state()))
    ctx.close()


@pytest.mark.gpu
def test_nan_state_stops_the_steady_march():
    pytest.importorskip("torch")
    capi = _lib_or_skip()
    case = W.case_bump2d(12, 4, 1, 1)
    ctx = capi.Context(case.mesh, case.p, case.free, capi.PCEXP_FP64, m_max=10)
    u = ctx.get_state()
    u[3] = np.inf
    ctx.set_state(u)
    with pytest.raises(capi.PcexpError) as ei:
        ctx.march_steady(capi.PCEXP_SCHEME_EXP1, 10.0, 5.0, 20, 10)
    assert ei.value.code == capi.PCEXP_ERR_NONFINITE
    ctx.close()
