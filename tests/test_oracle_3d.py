"""Pins of the oracle on tetrahedra (the 3D vortex case): flux, basis, quadrature
on faces, residual invariants and J v, each against what the paper or the mathematics
fixes rather than against the oracle itself."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import euler
from oracle.cases import freestream_state, vortex_state
from oracle.dg import DGOracle, build_faces, face_vertices

G = 1.4


def cons(rho, vel, p):
    vel = np.asarray(vel, float)
    return np.array([rho, *(rho * vel), p / (G - 1) + 0.5 * rho * vel @ vel])


def appendix_jacobian_3d(U, n):
    """Eq. dfdu (the 5 x 5 matrix of the Appendix) with omega = 0 (so B2 = 0) and grad psi
    replaced by the unit normal n: a0 = (gamma-1)|v|^2/2, a1 = gamma E - a0 with E the
    total specific energy, a2 = gamma-1, a3 = gamma-2, B1 = v . n.  Written out here from
    the Appendix, independently of the oracle's flux code."""
    rho = U[0]
    u, v, w = U[1] / rho, U[2] / rho, U[3] / rho
    E = U[4] / rho
    nx, ny, nz = n
    a0 = 0.5 * (G - 1) * (u * u + v * v + w * w)
    a1 = G * E - a0
    a2, a3 = G - 1, G - 2
    B1 = u * nx + v * ny + w * nz
    return np.array([
        [0.0, nx, ny, nz, 0.0],
        [a0 * nx - B1 * u, B1 - a3 * u * nx, u * ny - a2 * v * nx, u * nz - a2 * w * nx, a2 * nx],
        [a0 * ny - B1 * v, v * nx - a2 * u * ny, B1 - a3 * v * ny, v * nz - a2 * w * ny, a2 * ny],
        [a0 * nz - B1 * w, w * nx - a2 * u * nz, w * ny - a2 * v * nz, B1 - a3 * w * nz, a2 * nz],
        [(a0 - a1) * B1, a1 * nx - a2 * B1 * u, a1 * ny - a2 * v * B1, a1 * nz - a2 * B1 * w, G * B1],
    ])


def roe_state(UL, UR):
    d = len(UL) - 2

    def prim(U):
        rho = U[0]
        vel = U[1:1 + d] / rho
        p = (G - 1) * (U[d + 1] - 0.5 * rho * vel @ vel)
        return rho, vel, p, (U[d + 1] + p) / rho
    rL, vL, pL, HL = prim(UL)
    rR, vR, pR, HR = prim(UR)
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    vel = (sL * vL + sR * vR) / (sL + sR)
    H = (sL * HL + sR * HR) / (sL + sR)
    rho = sL * sR
    p = rho * (H - 0.5 * vel @ vel) * (G - 1) / G
    return cons(rho, vel, p)


def unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


CASES = [
    (cons(1.0, [0.3, -0.2, 0.25], 1.0), cons(0.8, [0.1, 0.4, -0.1], 0.7), unit([0.6, 0.8, 0.3])),
    (cons(1.2, [-0.5, 0.2, 0.0], 1.3), cons(1.0, [0.2, 0.1, 0.3], 0.9), unit([0.0, 0.0, 1.0])),
    (cons(0.5, [1.5, 0.0, -0.4], 0.4), cons(0.6, [1.2, 0.3, 0.2], 0.5), unit([-0.28, 0.96, -0.5])),
]


@pytest.mark.parametrize("UL,UR,n", CASES)
def test_roe_property_3d_with_appendix_jacobian(UL, UR, n):
    """Roe's property F_n(U_R) - F_n(U_L) = A(U^) (U_R - U_L) with A from Eq. dfdu at the
    Roe-average state, and F~(U, U) = F_n(U)."""
    fL = np.array(euler.flux_normal(UL, n, G))
    fR = np.array(euler.flux_normal(UR, n, G))
    A = appendix_jacobian_3d(roe_state(UL, UR), n)
    assert np.allclose(fR - fL, A @ (UR - UL), rtol=1e-12, atol=1e-13)
    assert np.allclose(euler.roe_flux(UL, UL, n, G), fL, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("UL,UR,n", CASES)
def test_roe_dissipation_3d_is_abs_A(UL, UR, n):
    """The dissipation of the 3D Roe flux is |A(U^)| (U_R - U_L), |A| from the eigen-
    decomposition of the Appendix matrix."""
    A = appendix_jacobian_3d(roe_state(UL, UR), n)
    lam, R = np.linalg.eig(A)
    absA = (R @ np.diag(np.abs(lam)) @ np.linalg.inv(R)).real
    dis = np.array(euler.roe_dissipation(UL, UR, n, G))
    assert np.allclose(dis, absA @ (UR - UL), rtol=1e-10, atol=1e-12)


def test_roe_3d_in_plane_reduces_to_2d():
    """For states with w = 0 and a normal in the x-y plane, the 3D Roe flux is the 2D one
    with a zero z-momentum flux inserted."""
    UL2, UR2 = cons(1.1, [0.3, -0.2], 1.0), cons(0.9, [0.1, 0.4], 0.8)
    n2 = unit([0.6, -0.8])
    UL3 = np.insert(UL2, 3, 0.0)
    UR3 = np.insert(UR2, 3, 0.0)
    f2 = euler.roe_flux(UL2, UR2, n2, G)
    f3 = euler.roe_flux(UL3, UR3, np.append(n2, 0.0), G)
    assert np.allclose(np.insert(f2, 3, 0.0), f3, rtol=1e-14, atol=1e-15)


def test_face_rule_integrates_face_polynomials():
    """The collapsed triangle rule on the faces of a jittered tetrahedron mesh integrates
    polynomials of degree 2p+1 exactly: the surface integral of x^a y^b z^c over a face
    against the closed form from the face's own barycentric expansion (Dirichlet
    integrals: int over the reference triangle of l0^i l1^j l2^k = 2 |f| i! j! k!/(i+j+k+2)!)."""
    mesh = W.periodic_cube_kuhn(2, 1.0, 0.1, 3, periodic=False)
    p = 2
    dg = DGOracle(mesh, p, W.Freestream())
    rng = np.random.default_rng(0)
    for _ in range(5):
        i = int(rng.integers(len(dg.fb)))
        e, f, _ = dg.fb[i]
        V = dg.verts[e, face_vertices(3, f)]
        x = dg.fb_x[i]
        area = dg.fb_w[i].sum()
        # integrand (x . a)^(2p+1) for a random direction a: expand over barycentrics
        a = rng.normal(size=3)
        got = np.sum(dg.fb_w[i] * (x @ a) ** (2 * p + 1))
        c = V @ a  # linear function at the 3 corners
        deg = 2 * p + 1
        exact = 0.0
        for i0 in range(deg + 1):
            for i1 in range(deg + 1 - i0):
                i2 = deg - i0 - i1
                mult = math.factorial(deg) / (math.factorial(i0) * math.factorial(i1) * math.factorial(i2))
                exact += mult * c[0] ** i0 * c[1] ** i1 * c[2] ** i2 * \
                    2 * area * math.factorial(i0) * math.factorial(i1) * math.factorial(i2) / math.factorial(deg + 2)
        assert abs(got - exact) <= 1e-13 * max(1.0, abs(exact))


@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_paper_basis_orthonormal_on_tetrahedra(p):
    dg = DGOracle(W.periodic_cube_kuhn(3, 4.0, 0.1, 11), p, W.Freestream())
    M = np.einsum("eq,eqi,eqj->eij", dg.wq, dg.psi_q, dg.psi_q)
    assert np.abs(M - np.eye(dg.N)).max() < 1e-12
    assert np.all(np.abs(np.triu(dg.basis.C, 1)) == 0.0)
    assert np.all(np.diagonal(dg.basis.C, axis1=1, axis2=2) > 0)
    assert np.allclose(dg.psi_q[:, :, 0], 1.0 / np.sqrt(dg.area)[:, None], rtol=1e-13)
    assert dg.N == (p + 1) * (p + 2) * (p + 3) // 6


def test_element_measures_fill_the_cube():
    """The tetrahedra of the Kuhn split tile the cube: sum |E| = L^3, every face matched."""
    mesh = W.periodic_cube_kuhn(3, 2.0, 0.1, 4)
    dg = DGOracle(mesh, 0, W.Freestream())
    assert abs(dg.area.sum() - 8.0) < 1e-12
    interior, boundary = build_faces(mesh)
    assert len(interior) == 2 * mesh.n_elem and len(boundary) == 0


@pytest.mark.parametrize("p", [1, 2])
def test_projection_reproduces_polynomials_3d(p):
    dg = DGOracle(W.periodic_cube_kuhn(3, 2.0, 0.1, 3), p, W.Freestream())

    def poly(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        f = 0.3 + 0.2 * X ** p - 0.7 * Z * Y ** (p - 1) + 0.1 * Y
        return np.stack([f, 2 * f, -f, f + Z, f + 1], axis=-1)

    u = dg.project(poly)
    xs = dg.xq + 0.01
    assert np.allclose(dg.state_at(u, xs), poly(xs), atol=1e-12)
    # the L2-error functional of a projected polynomial is zero to round-off
    assert dg.l2_error(u, poly) < 1e-12


@pytest.mark.parametrize("p", [1, 2])
def test_traces_agree_on_shared_faces(p):
    """A global polynomial of degree p projected onto the mesh has equal traces from both
    sides of every interior face: both sides evaluate the same physical face points (the
    L element's face rule mapped through the R element's vertex permutation)."""
    mesh = W.periodic_cube_kuhn(3, 1.0, 0.15, 9, periodic=False)
    dg = DGOracle(mesh, p, W.Freestream())

    def poly(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        f = 0.5 + X ** p - 0.3 * Y * Z ** (p - 1) + 0.2 * Z
        return np.stack([f, -f, 2 * f, f * 0.5, f + 2], axis=-1)

    u = dg.project(poly)
    eL, fL, eR, fR = dg.fi.T
    UL = np.einsum("fqi,fvi->fqv", dg.fi_psiL, u[eL])
    UR = np.einsum("fqi,fvi->fqv", dg.fi_psiR, u[eR])
    assert np.abs(UL - UR).max() < 1e-12


@pytest.mark.parametrize("p", [0, 1, 2])
def test_freestream_preserved_kuhn_periodic(p):
    dg = DGOracle(W.periodic_cube_kuhn(3, 10.0, 0.1, 2), p, W.Freestream(0.5, 30.0))
    u = dg.project(lambda x: freestream_state(x, dg.free))
    assert np.abs(dg.residual(u)).max() < 1e-13


@pytest.mark.parametrize("p", [1, 2])
def test_freestream_preserved_kuhn_farfield(p):
    dg = DGOracle(W.periodic_cube_kuhn(3, 1.0, 0.15, 6, periodic=False), p, W.Freestream(0.5, 30.0))
    u = dg.project(lambda x: freestream_state(x, dg.free))
    assert np.abs(dg.residual(u)).max() < 1e-13


def test_conservation_periodic_3d():
    """sum_e int_E R dx = 0 on a periodic tetrahedron mesh (face fluxes cancel in pairs)."""
    dg = DGOracle(W.periodic_cube_kuhn(3, 3.0, 0.1, 4), 2, W.Freestream(0.5, 10.0))
    u = dg.project(lambda x: freestream_state(x, dg.free))
    u = u + 0.05 * W.random_coeffs(17, u.shape) * np.abs(u[:, :, :1])
    R = dg.residual(u)
    total = np.einsum("ev,e->v", R[:, :, 0], np.sqrt(dg.area))
    assert np.abs(total).max() < 1e-13


def test_p0_is_finite_volume_roe_3d():
    """At p = 0 the scheme is the first-order finite-volume Roe scheme on tetrahedra
    (brute-force loop over faces with normals from cross products)."""
    mesh = W.periodic_cube_kuhn(3, 1.0, 0.1, 8)
    dg = DGOracle(mesh, 0, W.Freestream(0.4, 20.0))
    u = dg.project(lambda x: freestream_state(x, dg.free))
    u = u + 0.3 * W.random_coeffs(5, u.shape) * np.abs(u[:, :, :1])
    U = u[:, :, 0] / np.sqrt(dg.area)[:, None]
    interior, _ = build_faces(mesh)
    Rref = np.zeros_like(U)
    X = mesh.coords
    for eL, fL, eR, fR in interior:
        a, b, c = (X[mesh.elems[eL, k]] for k in face_vertices(3, fL))
        nn = np.cross(b - a, c - a)
        opp = X[mesh.elems[eL, fL]]
        if nn @ (a - opp) < 0:
            nn = -nn
        area = 0.5 * np.linalg.norm(nn)
        F = euler.roe_flux(U[eL][None], U[eR][None], (nn / (2 * area))[None], 1.4)[0]
        Rref[eL] -= area * F
        Rref[eR] += area * F
    R = dg.residual(u)[:, :, 0] * np.sqrt(dg.area)[:, None]
    assert np.allclose(R, Rref, atol=1e-13)


def test_jvp_dual_matches_complex_step_3d():
    dg = DGOracle(W.periodic_cube_kuhn(3, 10.0, 0.1, 1), 2, W.Freestream(0.5, 45.0))
    u = dg.project(lambda x: vortex_state(x, dg.free, W.Vortex(5.0, (5.0, 5.0)), period=10.0)).reshape(-1)
    v = W.random_coeffs(3, (dg.K,))
    a = dg.jvp(u, v)
    b = dg.jvp_complex_step(u, v)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def test_vortex_3d_is_the_planar_vortex():
    """The 3D vortex is the 2D field in x-y, uniform in z, with zero z-velocity."""
    free, vx = W.Freestream(0.5, 45.0), W.Vortex(5.0, (5.0, 5.0))
    rng = np.random.default_rng(1)
    x3 = rng.uniform(0, 10, size=(50, 3))
    U3 = vortex_state(x3, free, vx, t=0.7, period=10.0)
    U2 = vortex_state(x3[:, :2], free, vx, t=0.7, period=10.0)
    assert np.array_equal(U3[:, 3], np.zeros(50))
    assert np.allclose(U3[:, [0, 1, 2, 4]], U2, rtol=1e-15, atol=1e-15)


def test_l2_error_gradient_by_differences():
    """The oracle's vortex-error functional: its dual-number derivative along a direction
    matches a central difference."""
    from oracle.adscalar import Dual
    dg = DGOracle(W.periodic_cube_kuhn(3, 10.0, 0.1, 1), 1, W.Freestream(0.5, 45.0))
    vx = W.Vortex(5.0, (5.0, 5.0))
    ex = lambda x: vortex_state(x, dg.free, vx, t=0.3, period=10.0)  # noqa: E731
    u = dg.project(lambda x: vortex_state(x, dg.free, vx, period=10.0)).reshape(-1)
    v = W.random_coeffs(8, (dg.K,))
    d = dg.l2_error(Dual(u, v), ex).der
    h = 1e-6
    fd = (dg.l2_error(u + h * v, ex) - dg.l2_error(u - h * v, ex)) / (2 * h)
    assert abs(d - fd) <= 1e-7 * abs(fd)
