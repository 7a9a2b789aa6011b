"""PCEXP and EXP1 steps, time-step rules and the steady march (Sec. 2, 5).

PCEXP (Eq. s9, s10), with J_n the Jacobian at u_n and N(u) = R(u) - J_n u:
    u_*     = u_n + dt phi_1(dt J_n) R_n
    u_{n+1} = u_* + dt/2 phi_1(dt J_n) (N_* - N_n),
    N_* - N_n = R(u_*) - R_n - J_n (u_* - u_n)   (one explicit J v; reading).
EXP1 is the first stage alone.  Both phi_1 products use ``krylov.krylov_phi1``.

Steady runs (Sec. 5.2): the CFL number follows Eq. cfl; reading of local time
stepping: the scheme is applied to du/dtau = D R(u), D = diag(dt_e) per
element, with a unit pseudo-step.
"""
import numpy as np

from . import krylov


def pcexp_step(u, R, jvp, dt: float, m: int, eta: float = 1e-12, scheme: str = "pcexp"):
    """One PCEXP (or EXP1) step of du/dt = R(u).

    R(u) -> residual vector; jvp(u_n, v) -> J(u_n) v.  Returns (u_{n+1}, info).
    """
    u = np.asarray(u, dtype=np.float64)
    Rn = R(u)
    x1, i1 = krylov.krylov_phi1(lambda v: jvp(u, v), Rn, dt, m, eta)
    u_star = u + dt * x1
    info = dict(k1=i1["k"], beta1=i1["beta"], k2=0, beta2=0.0)
    if scheme == "exp1":
        return u_star, info
    d = R(u_star) - Rn - jvp(u, u_star - u)
    x2, i2 = krylov.krylov_phi1(lambda v: jvp(u, v), d, dt, m, eta)
    info.update(k2=i2["k"], beta2=i2["beta"])
    return u_star + 0.5 * dt * x2, info


def scaled_system(R, jvp, scale):
    """R and J v of du/dtau = D R(u) for a per-unknown scale vector D."""
    return (lambda u: scale * R(u)), (lambda u, v: scale * jvp(u, v))


def cfl_ramp(n: int, p: int, res_norm: float, cfl_max: float) -> float:
    """CFL(n) = min{CFL_max, max[||R(rho_n)||^-3, 1 + (n-1)/(2p+1)]} (Eq. cfl)."""
    a = res_norm ** -3 if res_norm > 0 else np.inf
    return float(min(cfl_max, max(a, 1.0 + (n - 1) / (2 * p + 1))))


def unsteady_run(dg, u0, cfl: float, steps: int, m: int, eta: float = 1e-12, scheme="pcexp",
                 callback=None):
    """Global dt = min_e dt_e (Eq. x3d) recomputed from u_n each step."""
    u = np.asarray(u0, np.float64).reshape(-1).copy()
    t = 0.0
    for n in range(steps):
        dt = float(np.min(dg.local_dt(u, cfl)))
        u, info = pcexp_step(u, dg.residual, dg.jvp, dt, m, eta, scheme)
        t += dt
        if callback is not None:
            callback(n, u, dt, info)
    return u, t


def steady_step(dg, u, cfl: float, m: int, eta: float = 1e-12, scheme="pcexp"):
    """One local-time-step iteration on du/dtau = D R(u), unit pseudo-step."""
    dte = dg.local_dt(u, cfl)
    scale = np.repeat(dte, dg.nv * dg.N)
    Rs, Js = scaled_system(dg.residual, dg.jvp, scale)
    return pcexp_step(u, Rs, Js, 1.0, m, eta, scheme)


def steady_march(dg, u0, cfl_max: float, decades: float, max_iter: int, m: int,
                 volume: float, eta: float = 1e-12, scheme="exp1"):
    """March to a residual drop ||R(rho_n)|| / ||R(rho_1)|| <= 10^-decades with Eq. cfl."""
    u = np.asarray(u0, np.float64).reshape(-1).copy()
    hist = []
    r1 = None
    for n in range(1, max_iter + 1):
        rn = dg.density_residual_norm(dg.residual(u), volume)
        if r1 is None:
            r1 = rn
        hist.append(rn)
        if rn <= r1 * 10.0 ** (-decades):
            break
        cfl = cfl_ramp(n, dg.p, rn, cfl_max)
        u, _ = steady_step(dg, u, cfl, m, eta, scheme)
    return u, np.asarray(hist)
