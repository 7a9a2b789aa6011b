"""Pins of the rotating frame of reference (Sec. 4.1, Eq. euler; Appendix Eq. dfdu, dsdu) and
of the symmetry-plane boundary condition in the oracle.

* Closed form: a uniform state U (absolute velocity v) has R_e = int_E psi_i S(U) on every
  element without a boundary face: the volume and face integrals of F_abs cancel, and those
  of -U v_r^T cancel as well because v_r = omega x x is divergence-free and linear (the rules
  integrate every term exactly); only the source remains, S = -omega x (rho v).  On the
  orthonormal basis that is the constant mode: R_e[1+k][0] = -(omega x m)_k sqrt|E|.
* The volume block of the exact Jacobian equals the quadrature of Eq. dfdu (with the frame
  term B_2 = (omega x x) . grad psi, written out here from the Appendix) plus
  psi_i psi_j dS/dU; dS/dU is the negative of the printed Eq. dsdu (reading: Eq. euler's
  S = -rho omega x v is followed; Eq. dsdu carries the opposite sign).
* Complex-step and dual-number J v agree with rotation.
* A symmetry plane gives the slip wall's residual and is not part of the wall force.
"""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import adscalar as ad
from oracle.dg import BC_SYMMETRY, DGOracle

OMEGA = (0.3, -0.2, 0.5)
G = 1.4


def walled_cube(n=2, L=2.0, jitter=0.0, seed=0):
    mesh = W.periodic_cube_kuhn(n, L, jitter, seed, periodic=False)
    return dataclasses.replace(mesh, btags=np.full(len(mesh.btags), W.BC_SLIP_WALL, np.int32))


def walled_box_2d(nx=6, ny=3):
    mesh = W.bump_channel(nx, ny, 0.15, 4, bump_h=0.0)
    return dataclasses.replace(mesh, btags=np.full(len(mesh.btags), W.BC_SLIP_WALL, np.int32))


def uniform(dg, U):
    u = np.zeros((dg.E, dg.nv, dg.N))
    u[:, :, 0] = np.asarray(U)[None, :] * np.sqrt(dg.area)[:, None]
    return u


def interior_elements(dg):
    touch = np.zeros(dg.E, bool)
    touch[dg.fb[:, 0]] = True
    return ~touch


@pytest.mark.parametrize("dim,p", [(3, 1), (3, 2), (2, 1), (2, 3)])
def test_uniform_state_interior_residual_is_the_source(dim, p):
    if dim == 3:
        mesh, om = walled_cube(3, 2.0, 0.1, 2), OMEGA
        U = np.array([1.1, 0.3, -0.2, 0.15, 2.9])
    else:
        mesh, om = walled_box_2d(8, 4), (0.0, 0.0, 0.7)
        U = np.array([1.1, 0.3, -0.2, 2.9])
    dg = DGOracle(mesh, p, W.Freestream(0.5, 0.0), omega=om)
    R = dg.residual(uniform(dg, U))
    inner = interior_elements(dg)
    assert inner.sum() > 0
    m = np.zeros(3)
    m[:dim] = U[1:1 + dim]
    src = -np.cross(om, m)[:dim]
    expect = np.zeros((dg.E, dg.nv, dg.N))
    expect[:, 1:1 + dim, 0] = src[None, :] * np.sqrt(dg.area)[:, None]
    assert np.abs(R[inner] - expect[inner]).max() <= 1e-12 * np.abs(U).max()
    # the frame terms matter: without rotation the same elements have R = 0
    R0 = DGOracle(mesh, p, W.Freestream(0.5, 0.0)).residual(uniform(dg, U))
    assert np.abs(R0[inner]).max() <= 1e-12


def appendix_jacobian_3d(U, gpsi, x, om):
    """Eq. dfdu (3D, rows and columns rho, m_x, m_y, m_z, rho E) at a point x with grad psi =
    gpsi, written out from the Appendix: a0 = (gamma-1)|v|^2/2, a1 = gamma E - a0 (E the total
    specific energy), a2 = gamma - 1, a3 = gamma - 2, B1 = v . grad psi,
    B2 = (omega x x) . grad psi."""
    rho = U[0]
    u, v, w = U[1] / rho, U[2] / rho, U[3] / rho
    E = U[4] / rho
    px, py, pz = gpsi
    a0 = 0.5 * (G - 1) * (u * u + v * v + w * w)
    a1 = G * E - a0
    a2, a3 = G - 1, G - 2
    B1 = u * px + v * py + w * pz
    B2 = np.cross(om, x) @ gpsi
    return np.array([
        [-B2, px, py, pz, 0.0],
        [a0 * px - B1 * u, B1 - B2 - a3 * u * px, u * py - a2 * v * px, u * pz - a2 * w * px, a2 * px],
        [a0 * py - B1 * v, v * px - a2 * u * py, B1 - B2 - a3 * v * py, v * pz - a2 * w * py, a2 * py],
        [a0 * pz - B1 * w, w * px - a2 * u * pz, w * py - a2 * v * pz, B1 - B2 - a3 * w * pz, a2 * pz],
        [(a0 - a1) * B1, a1 * px - a2 * B1 * u, a1 * py - a2 * v * B1, a1 * pz - a2 * B1 * w, G * B1 - B2],
    ])


def appendix_source_jacobian(om):
    """Eq. dsdu as printed."""
    wx, wy, wz = om
    return np.array([
        [0, 0, 0, 0, 0],
        [0, 0, -wz, wy, 0],
        [0, wz, 0, -wx, 0],
        [0, -wy, wx, 0, 0],
        [0, 0, 0, 0, 0],
    ], dtype=float)


def test_volume_jacobian_matches_appendix_with_rotation():
    mesh = walled_cube(2, 2.0, 0.1, 3)
    dg = DGOracle(mesh, 2, W.Freestream(0.5, 0.0), omega=OMEGA)
    rng = np.random.default_rng(5)
    u = uniform(dg, [1.05, 0.2, -0.1, 0.3, 2.7])
    u = u + 0.03 * rng.standard_normal(u.shape) * np.abs(u[:, :, :1])
    e = 7
    N, nv = dg.N, dg.nv
    Uq = np.einsum("qi,vi->qv", dg.psi_q[e], u[e])
    dS = -appendix_source_jacobian(OMEGA)  # reading: Eq. euler's sign
    Jref = np.zeros((nv * N, nv * N))
    for q in range(Uq.shape[0]):
        for i in range(N):
            A = appendix_jacobian_3d(Uq[q], dg.gpsi_wq[e, q, i], dg.xq[e, q], np.asarray(OMEGA))
            for j in range(N):
                blk = dg.psi_q[e, q, j] * A + dg.wq[e, q] * dg.psi_q[e, q, i] * dg.psi_q[e, q, j] * dS
                for a in range(nv):
                    for b in range(nv):
                        Jref[a * N + i, b * N + j] += blk[a, b]
    Jblk = np.zeros((nv * N, nv * N))
    for k in range(nv * N):
        v = np.zeros_like(u)
        v[e].reshape(-1)[k] = 1.0
        Jblk[:, k] = dg.jvp(u, v, faces=False)[e].reshape(-1)
    assert np.abs(Jblk - Jref).max() <= 1e-12 * np.abs(Jref).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_rotating_jvp_dual_matches_complex_step(dim):
    if dim == 3:
        mesh, om, U = walled_cube(2, 2.0, 0.1, 1), OMEGA, [1.0, 0.2, -0.1, 0.3, 2.7]
    else:
        mesh, om, U = walled_box_2d(6, 3), (0.0, 0.0, 0.9), [1.0, 0.2, -0.1, 2.7]
    dg = DGOracle(mesh, 2, W.Freestream(0.5, 0.0), omega=om)
    u = uniform(dg, U)
    u = u + 0.05 * W.random_coeffs(8, u.shape) * np.abs(u[:, :, :1])
    v = W.random_coeffs(9, u.shape)
    j1 = dg.jvp(u, v)
    j2 = dg.jvp_complex_step(u, v)
    assert np.abs(j1 - j2).max() <= 1e-12 * np.abs(j1).max()


def test_symmetry_plane_is_a_slip_wall_and_not_a_wall():
    mesh = W.bump_channel(8, 4, 0.15, 2)
    sym = np.where(mesh.btags == W.BC_SLIP_WALL, BC_SYMMETRY, mesh.btags).astype(np.int32)
    free = W.Freestream(0.5, 0.0)
    dw = DGOracle(mesh, 2, free)
    ds = DGOracle(dataclasses.replace(mesh, btags=sym), 2, free)
    u = uniform(dw, dw.freestream_state())
    u = u + 0.05 * W.random_coeffs(3, u.shape) * np.abs(u[:, :, :1])
    assert np.array_equal(dw.residual(u), ds.residual(u))
    assert dw.wall_force(u, (0.0, 1.0)) != 0.0
    assert ds.wall_force(u, (0.0, 1.0)) == 0.0


def test_rotating_frame_rejects_periodic_and_farfield():
    with pytest.raises(ValueError):
        DGOracle(W.periodic_square(4, 1.0), 1, W.Freestream(0.5, 0.0), omega=(0, 0, 1.0))
    with pytest.raises(ValueError):
        DGOracle(W.bump_channel(4, 2, 0.1, 1), 1, W.Freestream(0.5, 0.0), omega=(0, 0, 1.0))
    with pytest.raises(ValueError):
        DGOracle(walled_box_2d(4, 2), 1, W.Freestream(0.5, 0.0), omega=(0.1, 0, 1.0))
