"""Pins of the oracle's Euler/Roe flux and ghost states (Sec. 4.1, 4.4, Appendix Eq. dfdu)."""
import numpy as np
import pytest

from oracle import euler

G = 1.4


def cons(rho, vel, p):
    vel = np.asarray(vel, float)
    return np.array([rho, *(rho * vel), p / (G - 1) + 0.5 * rho * vel @ vel])


def appendix_jacobian(U, n):
    """Eq. dfdu with omega = 0 and grad psi replaced by the unit normal n (2D rows/cols).

    Written here from the Appendix, independently of the oracle: a0 = (gamma-1)|v|^2/2,
    a1 = gamma E - a0 (E the total specific energy), a2 = gamma-1, a3 = gamma-2, B1 = v.n.
    """
    rho = U[0]
    u, v = U[1] / rho, U[2] / rho
    E = U[3] / rho
    nx, ny = n
    a0 = 0.5 * (G - 1) * (u * u + v * v)
    a1 = G * E - a0
    a2, a3 = G - 1, G - 2
    B1 = u * nx + v * ny
    return np.array([
        [0.0, nx, ny, 0.0],
        [a0 * nx - B1 * u, B1 - a3 * u * nx, u * ny - a2 * v * nx, a2 * nx],
        [a0 * ny - B1 * v, v * nx - a2 * u * ny, B1 - a3 * v * ny, a2 * ny],
        [(a0 - a1) * B1, a1 * nx - a2 * B1 * u, a1 * ny - a2 * v * B1, G * B1],
    ])


def roe_state(UL, UR):
    def prim(U):
        rho = U[0]
        vel = U[1:3] / rho
        p = (G - 1) * (U[3] - 0.5 * rho * vel @ vel)
        return rho, vel, p, (U[3] + p) / rho
    rL, vL, pL, HL = prim(UL)
    rR, vR, pR, HR = prim(UR)
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    vel = (sL * vL + sR * vR) / (sL + sR)
    H = (sL * HL + sR * HR) / (sL + sR)
    rho = sL * sR
    p = rho * (H - 0.5 * vel @ vel) * (G - 1) / G
    return cons(rho, vel, p)


CASES = [
    (cons(1.0, [0.3, -0.2], 1.0), cons(0.8, [0.1, 0.4], 0.7), np.array([0.6, 0.8])),
    (cons(1.2, [-0.5, 0.2], 1.3), cons(1.0, [0.2, 0.1], 0.9), np.array([1.0, 0.0])),
    (cons(0.5, [1.5, 0.0], 0.4), cons(0.6, [1.2, 0.3], 0.5), np.array([-0.28, 0.96])),
]


@pytest.mark.parametrize("UL,UR,n", CASES)
def test_roe_consistency(UL, UR, n):
    f = euler.roe_flux(UL[None], UL[None], n[None], G)[0]
    fn = np.array(euler.flux_normal(UL[None], n[None], G))[:, 0]
    assert f.shape == fn.shape == (4,)
    assert np.allclose(f, fn, atol=1e-15, rtol=0)


@pytest.mark.parametrize("UL,UR,n", CASES)
def test_roe_property_with_appendix_jacobian(UL, UR, n):
    """F_n(U_R) - F_n(U_L) = A(U_roe) (U_R - U_L): Roe's defining property, A from Eq. dfdu."""
    A = appendix_jacobian(roe_state(UL, UR), n)
    fL = np.array(euler.flux_normal(UL[None], n[None], G))[:, 0]
    fR = np.array(euler.flux_normal(UR[None], n[None], G))[:, 0]
    assert np.allclose(fR - fL, A @ (UR - UL), atol=1e-13)


@pytest.mark.parametrize("UL,UR,n", CASES)
def test_roe_dissipation_is_abs_A(UL, UR, n):
    """The wave sum equals |A| (U_R - U_L) with |A| = R |Lambda| R^-1 from an eigensolver."""
    A = appendix_jacobian(roe_state(UL, UR), n)
    lam, Rv = np.linalg.eig(A)
    absA = np.real(Rv @ np.diag(np.abs(lam)) @ np.linalg.inv(Rv))
    d = np.array(euler.roe_dissipation(UL[None], UR[None], n[None], G))[:, 0]
    assert np.allclose(d, absA @ (UR - UL), atol=1e-12)


def test_roe_supersonic_is_upwind():
    UL = cons(1.0, [3.0, 0.1], 1.0)
    UR = cons(0.9, [2.8, -0.2], 0.95)
    n = np.array([1.0, 0.0])
    f = euler.roe_flux(UL[None], UR[None], n[None], G)[0]
    fL = np.array(euler.flux_normal(UL[None], n[None], G))[:, 0]
    assert np.allclose(f, fL, atol=1e-13)


def test_slip_wall_blocks_mass_and_energy():
    UL = cons(1.1, [0.4, -0.3], 0.9)
    for ang in [0.1, 1.0, 2.5, 4.0]:
        n = np.array([np.cos(ang), np.sin(ang)])
        Ug = euler.ghost_slip_wall(UL[None], n[None], G)
        f = euler.roe_flux(UL[None], Ug, n[None], G)[0]
        assert abs(f[0]) < 1e-14 and abs(f[3]) < 1e-14
        # momentum flux is normal to the wall
        t = np.array([-n[1], n[0]])
        assert abs(f[1:3] @ t) < 1e-14


def test_farfield_ghost_special_cases():
    rho_inf, p_inf = 1.0, 1.0
    vel_inf = [0.5 * np.sqrt(1.4), 0.0]
    Uinf = cons(rho_inf, vel_inf, p_inf)
    for n in [np.array([1.0, 0.0]), np.array([-1.0, 0.0]), np.array([0.6, -0.8])]:
        Ug = euler.ghost_farfield(Uinf[None], n[None], G, rho_inf, vel_inf, p_inf)[0]
        assert np.allclose(Ug, Uinf, atol=1e-14)
    # supersonic outflow takes the interior state; supersonic inflow the free stream
    Uout = cons(0.9, [2.5, 0.1], 0.8)
    Ug = euler.ghost_farfield(Uout[None], np.array([[1.0, 0.0]]), G, rho_inf, vel_inf, p_inf)[0]
    assert np.allclose(Ug, Uout, atol=1e-13)
    vel_sup = [3.0, 0.0]
    Ug = euler.ghost_farfield(Uout[None], np.array([[-1.0, 0.0]]), G, rho_inf, vel_sup, p_inf)[0]
    assert np.allclose(Ug, cons(rho_inf, vel_sup, p_inf), atol=1e-13)
