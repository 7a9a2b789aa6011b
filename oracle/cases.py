"""Pointwise initial states of the synthetic flow cases, for the oracle.

Isentropic vortex (reading of the configs: the standard nondimensional
vortex, not the paper's beta = 0.2, R = 0.05 form of Sec. 5.1):
  T_inf = p_inf / rho_inf, mean velocity Ma c_inf (cos alpha, sin alpha),
  dv = eps / (2 pi) exp((1 - r^2) / 2) (-(y - y_c), x - x_c),
  T = T_inf - (gamma - 1) eps^2 / (8 gamma pi^2) exp(1 - r^2),
  rho = rho_inf (T / T_inf)^(1 / (gamma - 1)), p = rho T  (isentropic).
On a periodic domain the distance uses the nearest periodic image.  A core radius R
measures (x - x_c, y - y_c) in units of R (the paper's vortex of Sec. 5.1, with the
temperature perturbation read as -(beta U_inf)^2 / (2 C_p) exp(-r^2), is this vortex with
R = 0.05 and eps = 2 pi beta U_inf exp(-1/2)).  The
exact solution is this field translated with the mean velocity.  In 3D the same
field lies in the x-y plane, uniform in z, with zero z-velocity (the vortex axis
is along z); states then have 5 components (rho, rho u, rho v, rho w, rho E).
"""
import numpy as np


def freestream_velocity(free, dim: int = 2):
    """Free-stream velocity: Ma c_inf (cos alpha, sin alpha) in the x-y plane (w = 0 in 3D)."""
    c = np.sqrt(free.gamma * free.p / free.rho)
    a = free.alpha_deg * (np.pi / 180.0)  # the deg2rad constant; also takes a complex step
    vel = (free.mach * c * np.cos(a), free.mach * c * np.sin(a))
    return vel if dim == 2 else vel + (0.0,)


def _conservative(rho, vel, p, gamma):
    E = p / (gamma - 1) + 0.5 * rho * sum(v * v for v in vel)
    return np.stack([rho] + [rho * v for v in vel] + [E], axis=-1)


def vortex_state(x, free, vortex, t: float = 0.0, period=None):
    """Conservative state [..., dim+2] of the translated isentropic vortex at points x [..., dim]."""
    g = free.gamma
    u0, v0 = freestream_velocity(free)[:2]
    dx = x[..., 0] - (vortex.center[0] + u0 * t)
    dy = x[..., 1] - (vortex.center[1] + v0 * t)
    if period is not None:
        dx = dx - period * np.round(dx / period)
        dy = dy - period * np.round(dy / period)
    rad = getattr(vortex, "radius", 1.0)  # core radius: distances in its units
    dx, dy = dx / rad, dy / rad
    r2 = dx * dx + dy * dy
    eps = vortex.eps
    f = eps / (2 * np.pi) * np.exp(0.5 * (1.0 - r2))
    u = u0 - f * dy
    v = v0 + f * dx
    Tinf = free.p / free.rho
    T = Tinf - (g - 1) * eps ** 2 / (8 * g * np.pi ** 2) * np.exp(1.0 - r2)
    rho = free.rho * (T / Tinf) ** (1.0 / (g - 1))
    p = rho * T
    vel = [u, v] if x.shape[-1] == 2 else [u, v, np.zeros_like(u)]
    return _conservative(rho, vel, p, g)


def freestream_state(x, free):
    vel = freestream_velocity(free, x.shape[-1])
    one = np.ones(x.shape[:-1])
    return _conservative(free.rho * one, [v * one for v in vel], free.p * one, free.gamma)


def blob_state(x, free, blobs, radius):
    """Free stream with Gaussian perturbations of density and pressure (velocity unchanged)."""
    g = free.gamma
    u0, v0 = freestream_velocity(free)
    rho = np.full(x.shape[:-1], free.rho)
    p = np.full(x.shape[:-1], free.p)
    for bx, by, arho, ap in blobs:
        w = np.exp(-((x[..., 0] - bx) ** 2 + (x[..., 1] - by) ** 2) / radius ** 2)
        rho = rho + arho * w
        p = p + ap * w
    E = p / (g - 1) + 0.5 * rho * (u0 * u0 + v0 * v0)
    return np.stack([rho, rho * u0, rho * v0, E], axis=-1)
