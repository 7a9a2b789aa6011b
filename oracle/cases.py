"""Pointwise initial states of the synthetic flow cases, for the oracle.

Isentropic vortex (reading of the configs: the standard nondimensional
vortex, not the paper's beta = 0.2, R = 0.05 form of Sec. 5.1):
  T_inf = p_inf / rho_inf, mean velocity Ma c_inf (cos alpha, sin alpha),
  dv = eps / (2 pi) exp((1 - r^2) / 2) (-(y - y_c), x - x_c),
  T = T_inf - (gamma - 1) eps^2 / (8 gamma pi^2) exp(1 - r^2),
  rho = rho_inf (T / T_inf)^(1 / (gamma - 1)), p = rho T  (isentropic).
On a periodic domain the distance uses the nearest periodic image.  The
exact solution is this field translated with the mean velocity.
"""
import numpy as np


def freestream_velocity(free):
    c = np.sqrt(free.gamma * free.p / free.rho)
    a = np.deg2rad(free.alpha_deg)
    return free.mach * c * np.cos(a), free.mach * c * np.sin(a)


def vortex_state(x, free, vortex, t: float = 0.0, period=None):
    """Conservative state [..., 4] of the translated isentropic vortex at points x [..., 2]."""
    g = free.gamma
    u0, v0 = freestream_velocity(free)
    dx = x[..., 0] - (vortex.center[0] + u0 * t)
    dy = x[..., 1] - (vortex.center[1] + v0 * t)
    if period is not None:
        dx = dx - period * np.round(dx / period)
        dy = dy - period * np.round(dy / period)
    r2 = dx * dx + dy * dy
    eps = vortex.eps
    f = eps / (2 * np.pi) * np.exp(0.5 * (1.0 - r2))
    u = u0 - f * dy
    v = v0 + f * dx
    Tinf = free.p / free.rho
    T = Tinf - (g - 1) * eps ** 2 / (8 * g * np.pi ** 2) * np.exp(1.0 - r2)
    rho = free.rho * (T / Tinf) ** (1.0 / (g - 1))
    p = rho * T
    E = p / (g - 1) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E], axis=-1)


def freestream_state(x, free):
    u0, v0 = freestream_velocity(free)
    E = free.p / (free.gamma - 1) + 0.5 * free.rho * (u0 * u0 + v0 * v0)
    out = np.empty(x.shape[:-1] + (4,))
    out[...] = [free.rho, free.rho * u0, free.rho * v0, E]
    return out


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
