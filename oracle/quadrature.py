"""Quadrature rules for the oracle (the paper leaves them unspecified, Sec. 4.2).

Reading: Gauss rules generated by the Golub-Welsch eigenvalue method.
  * edges: Gauss-Legendre with p+1 points on [0, 1];
  * triangles: collapsed (Duffy) rule, Gauss-Legendre x Gauss-Jacobi(1, 0)
    with p+1 points per direction, exact for total degree 2p+1.  On the
    physical triangle (v0, v1, v2) the point (xi, eta) maps to
    v0 + xi (v1 - v0) + eta (v2 - v0), with xi = a (1 - b), eta = b.
  * tetrahedra: collapsed rule Gauss-Legendre x GJ(1,0) x GJ(2,0).
"""
import math

import numpy as np


def gauss_jacobi(n: int, alpha: float = 0.0, beta: float = 0.0):
    """Nodes/weights on [-1, 1] for the weight (1-x)^alpha (1+x)^beta (Golub-Welsch).

    The symmetric tridiagonal Jacobi matrix of the monic Jacobi recurrence is
    diagonalised; nodes are its eigenvalues and weights mu0 times the squared
    first components of the normalised eigenvectors.
    """
    a, b = float(alpha), float(beta)
    k = np.arange(n, dtype=np.float64)
    s = 2 * k + a + b
    diag = np.empty(n)
    with np.errstate(divide="ignore", invalid="ignore"):
        diag[:] = (b * b - a * a) / (s * (s + 2))
    diag[0] = (b - a) / (a + b + 2)  # the k = 0 term without the 0/0 at alpha + beta = 0
    kk = np.arange(1, n, dtype=np.float64)
    ss = 2 * kk + a + b
    off = np.sqrt(4 * kk * (kk + a) * (kk + b) * (kk + a + b) / (ss * ss * (ss + 1) * (ss - 1)))
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    x, V = np.linalg.eigh(T)
    mu0 = 2.0 ** (a + b + 1) * math.gamma(a + 1) * math.gamma(b + 1) / math.gamma(a + b + 2)
    w = mu0 * V[0, :] ** 2
    return x, w


def gauss_legendre01(n: int):
    """Gauss-Legendre nodes/weights on [0, 1] (weights sum to 1)."""
    x, w = gauss_jacobi(n, 0.0, 0.0)
    return 0.5 * (x + 1.0), 0.5 * w


def triangle_rule(n: int):
    """Collapsed rule on the reference triangle {xi, eta >= 0, xi + eta <= 1}.

    Returns points [n*n, 2] and weights [n*n] (summing to the area 1/2).
    """
    a, wa = gauss_legendre01(n)
    xb, wb = gauss_jacobi(n, 1.0, 0.0)  # weight (1 - x) on [-1, 1]
    b = 0.5 * (xb + 1.0)
    wb = wb / 4.0  # (1 - x) dx = 4 (1 - b) db
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            pts.append((a[i] * (1.0 - b[j]), b[j]))
            wts.append(wa[i] * wb[j])
    return np.asarray(pts), np.asarray(wts)


def tetra_rule(n: int):
    """Collapsed rule on the reference tetrahedron (volume 1/6)."""
    a, wa = gauss_legendre01(n)
    xb, wb = gauss_jacobi(n, 1.0, 0.0)
    xc, wc = gauss_jacobi(n, 2.0, 0.0)
    b, c = 0.5 * (xb + 1.0), 0.5 * (xc + 1.0)
    wb, wc = wb / 4.0, wc / 8.0
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                pts.append((a[i] * (1 - b[j]) * (1 - c[k]), b[j] * (1 - c[k]), c[k]))
                wts.append(wa[i] * wb[j] * wc[k])
    return np.asarray(pts), np.asarray(wts)
