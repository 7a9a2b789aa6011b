"""PCEXP and EXP1 steps, time-step rules and the steady march (Sec. 2, 5).

PCEXP (Eq. s9, s10), with J_n the Jacobian at u_n and N(u) = R(u) - J_n u:
    u_*     = u_n + dt phi_1(dt J_n) R_n
    u_{n+1} = u_* + dt/2 phi_1(dt J_n) (N_* - N_n),
    N_* - N_n = R(u_*) - R_n - J_n (u_* - u_n)   (one explicit J v; reading).
EXP1 is the first stage alone.  Both phi_1 products use ``krylov.krylov_phi1``.
ETD2 (Eq. s7) adds dt phi_2(dt J_n) (N_n - N_{n-1}) to the ETD1 step (``etd2_step``).

Steady runs (Sec. 5.2): the CFL number follows Eq. cfl; reading of local time
stepping: the scheme is applied to du/dtau = D R(u), D = diag(dt_e) per
element, with a unit pseudo-step.
"""
import numpy as np

from . import krylov


def pcexp_step(u, R, jvp, dt: float, m: int, eta: float = 1e-12, scheme: str = "pcexp", tol: float = 0.0):
    """One PCEXP (or EXP1) step of du/dt = R(u).

    R(u) -> residual vector; jvp(u_n, v) -> J(u_n) v.  tol > 0: adaptive Krylov dimension
    (``krylov.krylov_phi1``).  Returns (u_{n+1}, info); info err1, err2 are the Krylov
    error estimates of the two stages.
    """
    u = np.asarray(u, dtype=np.result_type(u, np.float64))  # complex for a complex step
    Rn = R(u)
    x1, i1 = krylov.krylov_phi1(lambda v: jvp(u, v), Rn, dt, m, eta, tol)
    u_star = u + dt * x1
    info = dict(k1=i1["k"], beta1=i1["beta"], k2=0, beta2=0.0, err1=i1["err"], err2=0.0)
    if scheme == "exp1":
        return u_star, info
    d = R(u_star) - Rn - jvp(u, u_star - u)
    x2, i2 = krylov.krylov_phi1(lambda v: jvp(u, v), d, dt, m, eta, tol)
    info.update(k2=i2["k"], beta2=i2["beta"], err2=i2["err"])
    return u_star + 0.5 * dt * x2, info


def etd2_step(u, R, jvp, dt: float, m: int, prev=None, eta: float = 1e-12):
    """One ETD2 step (Eq. s7, Sec. 2.1) of du/dt = R(u):

        u_{n+1} = u_n + dt phi_1(dt J_n) R_n + dt (dt / dt_{n-1}) phi_2(dt J_n) (N_n - N_{n-1}),

    with N(u) = R(u) - J_n u for the Jacobian J_n at u_n, so N_n - N_{n-1} =
    R_n - R_{n-1} - J_n (u_n - u_{n-1}) (one explicit J v).  Readings: the divided
    difference of N uses the previous step size (the factor dt / dt_{n-1}, 1 for uniform
    steps); the first step, which has no N_{n-1}, is ETD1 (Eq. s8, the EXP1 stage).

    prev = (u_{n-1}, R(u_{n-1}), dt_{n-1}) or None.  Returns (u_{n+1}, info, (u_n, R_n, dt))."""
    u = np.asarray(u, dtype=np.float64)
    Rn = R(u)
    x1, i1 = krylov.krylov_phi1(lambda v: jvp(u, v), Rn, dt, m, eta)
    un1 = u + dt * x1
    info = dict(k1=i1["k"], beta1=i1["beta"], k2=0, beta2=0.0)
    if prev is not None:
        up, Rp, dtp = prev
        d = Rn - Rp - jvp(u, u - up)
        x2, i2 = krylov.krylov_phi2(lambda v: jvp(u, v), d, dt, m, eta)
        un1 = un1 + dt * (dt / dtp) * x2
        info.update(k2=i2["k"], beta2=i2["beta"])
    return un1, info, (u, Rn, dt)


def etd2_run(dg, u0, cfl: float, steps: int, m: int, eta: float = 1e-12, dts=None):
    """ETD2 steps with the global dt = min_e dt_e (Eq. x3d) from u_n (or the given dts)."""
    u = np.asarray(u0, np.float64).reshape(-1).copy()
    prev = None
    out = []
    for n in range(steps):
        dt = float(np.min(dg.local_dt(u, cfl))) if dts is None else float(dts[n])
        u, info, prev = etd2_step(u, dg.residual, dg.jvp, dt, m, prev, eta)
        out.append((u.copy(), dt, info))
    return u, out


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


def steady_step(dg, u, cfl: float, m: int, eta: float = 1e-12, scheme="pcexp", tol: float = 0.0):
    """One local-time-step iteration on du/dtau = D R(u), unit pseudo-step."""
    dte = dg.local_dt(u, cfl)
    scale = np.repeat(dte, dg.nv * dg.N)
    Rs, Js = scaled_system(dg.residual, dg.jvp, scale)
    return pcexp_step(u, Rs, Js, 1.0, m, eta, scheme, tol)


def cfl_cap_update(cfl_used: float, err: float, tol: float) -> float:
    """Next cap on the steady march's CFL from the Krylov error estimate of the last
    iteration (reading, not in the paper: the paper's ramp alone raises the CFL into the
    range where the m = 30 Krylov phi_1 is inaccurate).  A multiplicative controller:
    cap = CFL_used * clamp(0.8 (tol / err)^(1/2), 1/4, 2)."""
    f = 2.0 if err <= 0.0 else min(2.0, max(0.25, 0.8 * (tol / err) ** 0.5))
    return cfl_used * f


def steady_march(dg, u0, cfl_max: float, decades: float, max_iter: int, m: int,
                 volume: float, eta: float = 1e-12, scheme="exp1", tol: float = 0.0):
    """March to a residual drop ||R(rho_n)|| / ||R(rho_1)|| <= 10^-decades with Eq. cfl.

    tol > 0: adaptive Krylov dimension in every stage, and the CFL of Eq. cfl is further
    capped by ``cfl_cap_update`` from the first stage's error estimate."""
    u = np.asarray(u0, np.float64).reshape(-1).copy()
    hist = []
    r1 = None
    cap = cfl_max
    for n in range(1, max_iter + 1):
        rn = dg.density_residual_norm(dg.residual(u), volume)
        if r1 is None:
            r1 = rn
        hist.append(rn)
        if rn <= r1 * 10.0 ** (-decades):
            break
        cfl = cfl_ramp(n, dg.p, rn, min(cfl_max, cap))
        u, info = steady_step(dg, u, cfl, m, eta, scheme, tol)
        if tol > 0:
            cap = min(cfl_max, cfl_cap_update(cfl, info["err1"], tol))
    return u, np.asarray(hist)
