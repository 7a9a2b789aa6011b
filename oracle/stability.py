"""Scalar linear-stability results of Sec. 3 for the oracle.

Model problem u' = J u + lambda u (Eq. model), a = dt lambda, b = dt J.
  * G_m: degree-m Taylor polynomial of exp(dt zeta) (Eq. G_m); Table 1 lists
    the largest stable |dt zeta| for real zeta < 0.
  * PCEXP growth factor r(a, b) (Eq. grow) and its b-series (Eq. y_poly).
  * EXP1 growth factor (Eq. exp1_grow) and TVDRK3 growth factor (Eq. rkgrow).
"""
import math

import numpy as np


def G_m(z, m: int):
    """1 + z + z^2/2! + ... + z^m/m! (Eq. G_m)."""
    z = np.asarray(z, dtype=np.complex128 if np.iscomplexobj(z) else np.float64)
    out = np.ones_like(z)
    term = np.ones_like(z)
    for k in range(1, m + 1):
        term = term * z / k
        out = out + term
    return out


def max_stable_real(m: int, tol: float = 1e-12) -> float:
    """Largest x with |G_m(-y)| <= 1 for all y in [0, x] (scan, then bisection)."""
    step = 1e-3
    x = step
    while abs(G_m(-x, m)) <= 1.0:
        x += step
    lo, hi = x - step, x
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if abs(G_m(-mid, m)) <= 1.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def r_pcexp(a, b):
    """PCEXP growth factor of Eq. grow."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return (a * (a - b) + np.exp(2 * b) * (a + b) * a + 2 * np.exp(b) * (b * b - a * a)) / (2 * b * b)


def r_pcexp_series(a, b):
    """Leading terms of Eq. y_poly (error O(b^3))."""
    c0 = 1 + a + a * a / 2
    return c0 + c0 * b + (0.5 + 2 * a / 3 + 7 * a * a / 24) * b * b


def r_exp1(a, b):
    """EXP1 growth factor of Eq. exp1_grow."""
    return (a * (np.exp(b) - 1) + b * np.exp(b)) / b


def r_tvdrk3(a, b):
    """TVDRK3 growth factor of Eq. rkgrow."""
    z = a + b
    return 1 + z + z * z / 2 + z ** 3 / 6


def pcexp_boundary_lower(b):
    """Lower bound a >= 2b / (1 - e^b) of Eq. pcexp_bd."""
    return 2 * b / (1 - np.exp(b))


def exp1_boundary_lower(b):
    """Lower bound a >= -b coth(b/2) of Eq. exp1_bd."""
    return -b / np.tanh(b / 2)


def tvdrk3_strip_offset() -> float:
    """-1 - (4 + sqrt 17)^(1/3) + (4 + sqrt 17)^(-1/3) (TVDRK3 bound, Sec. 3.1)."""
    c = (4 + math.sqrt(17)) ** (1.0 / 3.0)
    return -1 - c + 1 / c
