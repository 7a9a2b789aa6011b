"""Euler fluxes, Roe's Riemann flux and ghost states for the oracle.

Sec. 4.1 (Eq. euler): U = (rho, rho v, rho E) with the absolute velocity v,
p = (gamma - 1) rho e, E = e + |v|^2 / 2, H = E + p / rho.  In a frame rotating with
angular velocity omega the flux is F = F_abs - U v_r^T with v_r = omega x x (reading:
the mass row rho (v - v_r), the momentum rows rho v (v - v_r)^T + p I and the energy
row rho H v - rho E v_r, the form whose Jacobian is the Appendix's Eq. dfdu -- the
printed energy row rho H (v - v_r) would give gamma (B_1 - B_2) on its diagonal where
Eq. dfdu has gamma B_1 - B_2).  The source S = (0, -rho omega x v, 0) enters the DG
residual in ``dg``.  omega = 0 gives the fixed-frame equations.

Riemann flux (Sec. 4.2, after Eq. euler3): Roe's approximate solver with
square-root-density averages and no entropy fix (the paper names none):
    F~ = 1/2 (F_n(U_L) + F_n(U_R)) - 1/2 sum_k |lambda_k| alpha_k r_k.
Boundary faces use the same Roe flux against a ghost state (Sec. 4.4):
  * slip wall: normal velocity mirrored, density and pressure kept;
  * far field: one-dimensional characteristic (Riemann-invariant) state.

States at points are arrays [..., nv] of any scalar type in ``adscalar``;
normals are real arrays [..., dim].
"""
import numpy as np

from . import adscalar as ad


def primitives(U, gamma):
    """(rho, [v_k], p, E) of conservative states U[..., nv]."""
    nv = U.shape[-1]
    dim = nv - 2
    rho = U[..., 0]
    vel = [U[..., 1 + k] / rho for k in range(dim)]
    E = U[..., dim + 1]
    ke = 0.5 * sum(vk * vk for vk in vel)
    p = (gamma - 1.0) * (E - rho * ke)
    return rho, vel, p, E


def flux_dir(U, k, gamma, vr=None):
    """Flux component along Cartesian axis k -> list of nv arrays; with the frame velocity
    component vr_k (array, rotating frame) the relative part -U vr_k is included."""
    rho, vel, p, E = primitives(U, gamma)
    dim = len(vel)
    vk = vel[k]
    out = [rho * vk]
    for j in range(dim):
        f = rho * vel[j] * vk
        if j == k:
            f = f + p
        out.append(f)
    out.append((E + p) * vk)
    if vr is not None:
        out = [out[j] - U[..., j] * vr for j in range(len(out))]
    return out


def flux_normal(U, n, gamma):
    """F(U) . n -> list of nv arrays (n real, [..., dim])."""
    rho, vel, p, E = primitives(U, gamma)
    dim = len(vel)
    qn = sum(vel[k] * n[..., k] for k in range(dim))
    out = [rho * qn]
    for j in range(dim):
        out.append(rho * vel[j] * qn + p * n[..., j])
    out.append((E + p) * qn)
    return out


def roe_dissipation(UL, UR, n, gamma, vrn=None):
    """|A_roe| (U_R - U_L) written as the sum over waves |lambda_k| alpha_k r_k.  In a
    rotating frame the normal flux Jacobian is A_n - (v_r . n) I: same waves, eigenvalues
    shifted by -vrn."""
    rL, vL, pL, EL = primitives(UL, gamma)
    rR, vR, pR, ER = primitives(UR, gamma)
    dim = len(vL)
    HL = (EL + pL) / rL
    HR = (ER + pR) / rR
    sL = ad.sqrt(rL)
    sR = ad.sqrt(rR)
    den = sL + sR
    rho_h = sL * sR
    vel_h = [(sL * vL[k] + sR * vR[k]) / den for k in range(dim)]
    H_h = (sL * HL + sR * HR) / den
    q2 = sum(v * v for v in vel_h)
    c2 = (gamma - 1.0) * (H_h - 0.5 * q2)
    c = ad.sqrt(c2)
    qn = sum(vel_h[k] * n[..., k] for k in range(dim))
    dp = pR - pL
    drho = rR - rL
    dvel = [vR[k] - vL[k] for k in range(dim)]
    dqn = sum(dvel[k] * n[..., k] for k in range(dim))
    qs = qn if vrn is None else qn - vrn  # the waves' speeds relative to the frame
    l1 = ad.absval(qs - c)
    l2 = ad.absval(qs)
    l4 = ad.absval(qs + c)
    a1 = (dp - rho_h * c * dqn) / (2.0 * c2)
    a4 = (dp + rho_h * c * dqn) / (2.0 * c2)
    a2 = drho - dp / c2
    d = [l1 * a1 + l2 * a2 + l4 * a4]
    for k in range(dim):
        d.append(l1 * a1 * (vel_h[k] - c * n[..., k])
                 + l2 * (a2 * vel_h[k] + rho_h * (dvel[k] - dqn * n[..., k]))
                 + l4 * a4 * (vel_h[k] + c * n[..., k]))
    vdv = sum(vel_h[k] * dvel[k] for k in range(dim))
    d.append(l1 * a1 * (H_h - c * qn)
             + l2 * (a2 * 0.5 * q2 + rho_h * (vdv - qn * dqn))
             + l4 * a4 * (H_h + c * qn))
    return d


def roe_flux(UL, UR, n, gamma, vrn=None):
    """Roe's Riemann flux F~(U_L, U_R) . n -> stacked [..., nv]; vrn = v_r . n at the face
    points in a rotating frame (F . n = F_abs . n - vrn U)."""
    fL = flux_normal(UL, n, gamma)
    fR = flux_normal(UR, n, gamma)
    if vrn is not None:
        fL = [fL[v] - vrn * UL[..., v] for v in range(len(fL))]
        fR = [fR[v] - vrn * UR[..., v] for v in range(len(fR))]
    dis = roe_dissipation(UL, UR, n, gamma, vrn)
    return ad.stack([0.5 * (fL[v] + fR[v]) - 0.5 * dis[v] for v in range(len(fL))])


def conservative(rho, vel, p, gamma):
    """Stacked conservative state from primitives."""
    ke = 0.5 * sum(v * v for v in vel)
    return ad.stack([rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + rho * ke])


def ghost_slip_wall(UL, n, gamma, vrn=None):
    """Mirror state: v_g = v - 2 ((v - v_r) . n) n (the velocity relative to the wall, which
    moves with the frame, is mirrored), same density and pressure.  Also the symmetry plane."""
    rho, vel, p, E = primitives(UL, gamma)
    dim = len(vel)
    qn = sum(vel[k] * n[..., k] for k in range(dim))
    if vrn is not None:
        qn = qn - vrn
    velg = [vel[k] - 2.0 * qn * n[..., k] for k in range(dim)]
    return conservative(rho, velg, p, gamma)


def ghost_farfield(UL, n, gamma, rho_inf, vel_inf, p_inf):
    """Characteristic far-field state from the Riemann invariants R+- = q_n +- 2c/(gamma-1).

    R+ comes from the interior unless the interior normal Mach number is
    <= -1 (supersonic inflow); R- comes from the free stream unless it is
    >= 1 (supersonic outflow).  Entropy p/rho^gamma and the tangential
    velocity come from the interior when the boundary normal velocity is
    outward (>= 0), else from the free stream.
    """
    rho, vel, p, E = primitives(UL, gamma)
    dim = len(vel)
    g1 = gamma - 1.0
    c = ad.sqrt(gamma * p / rho)
    qn = sum(vel[k] * n[..., k] for k in range(dim))
    c_inf = np.sqrt(gamma * p_inf / rho_inf)
    qn_inf = sum(vel_inf[k] * n[..., k] for k in range(dim))
    mn = ad.real(qn) / ad.real(c)
    rp = ad.where(mn > -1.0, qn + 2.0 * c / g1, qn_inf + 2.0 * c_inf / g1)
    rm = ad.where(mn < 1.0, qn_inf - 2.0 * c_inf / g1 + 0.0 * qn, qn - 2.0 * c / g1)
    qb = 0.5 * (rp + rm)
    cb = 0.25 * g1 * (rp - rm)
    out = ad.real(qb) >= 0.0
    s_in = p / ad.power(rho, gamma)
    s_inf = p_inf / rho_inf ** gamma
    sb = ad.where(out, s_in, s_inf + 0.0 * s_in)
    vt = [ad.where(out, vel[k] - qn * n[..., k], vel_inf[k] - qn_inf * n[..., k] + 0.0 * qn) for k in range(dim)]
    velb = [vt[k] + qb * n[..., k] for k in range(dim)]
    rhob = ad.power(cb * cb / (gamma * sb), 1.0 / g1)
    pb = rhob * cb * cb / gamma
    return conservative(rhob, velb, pb, gamma)
