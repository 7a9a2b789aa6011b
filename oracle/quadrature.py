"""Quadrature rules for the oracle (the paper leaves them unspecified, Sec. 4.2).

Reading: Gauss rules generated by the Golub-Welsch eigenvalue method.
  * edges: Gauss-Legendre with p+1 points on [0, 1];
  * triangles: collapsed (Duffy) rule, Gauss-Legendre x Gauss-Jacobi(1, 0)
    with p+1 points per direction, exact for total degree 2p+1.  On the
    physical triangle (v0, v1, v2) the point (xi, eta) maps to
    v0 + xi (v1 - v0) + eta (v2 - v0), with xi = a (1 - b), eta = b.
  * tetrahedra: collapsed rule Gauss-Legendre x GJ(1,0) x GJ(2,0).
  * tetrahedra at p = 2: fully symmetric rules of the same degree (5) with fewer
    points, 14 in the volume and 7 on each face, from Newton's method on their
    moment equations (volume_rule, face_rule).
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


# ------------------------------------------------------- fully symmetric rules at p = 2
# Tetrahedra at p = 2 use fully symmetric rules of the same exactness as the collapsed ones
# (total degree 2p + 1 = 5) with fewer points: 14 in the volume instead of 27, and 7 on each
# triangular face instead of 9.  A symmetric rule is a union of orbits of barycentric points
# under the vertex permutations, each orbit with one weight; exactness for every polynomial
# of degree <= 5 reduces to exactness for the symmetric ones, one equation per invariant.
# The orbit parameters are found here by Newton's method on those moment equations.


def simplex_monomial_integral(alpha) -> float:
    """Integral over the reference simplex (volume 1/d!) of prod_i lam_i^alpha_i over all
    d + 1 barycentric coordinates: prod(alpha_i!) / (sum(alpha) + d)!."""
    d = len(alpha) - 1
    num = 1
    for a in alpha:
        num *= math.factorial(a)
    return num / math.factorial(sum(alpha) + d)


def _orbit(base):
    """Distinct permutations of a barycentric tuple (an orbit of the simplex's symmetries)."""
    import itertools
    return sorted(set(itertools.permutations(base)))


def _sym_points(orbits):
    """orbits: list of (barycentric base tuple, weight) -> barycentrics [n, d+1], weights [n]."""
    pts, wts = [], []
    for base, w in orbits:
        for q in _orbit(base):
            pts.append(q)
            wts.append(w)
    return pts, wts


def _newton_moments(orbits_of, x0, tests):
    """Newton's method for the orbit parameters x: sum_q w_q prod lam_q^alpha = exact for every
    alpha in tests.  The residual is a polynomial in x, so its Jacobian is taken by the complex
    step (exact to rounding).  The moment equations are moderately ill-conditioned, so the
    double-precision iterate is refined with residuals evaluated in long double."""
    def residual(x, dt):
        pts, wts = _sym_points(orbits_of([dt(v) for v in x]))
        r = []
        for al in tests:
            num = 1
            for a in al:
                num *= math.factorial(a)
            s = dt(0)
            for q, w in zip(pts, wts):
                t = w
                for lam, a in zip(q, al):
                    t = t * lam ** a
                s = s + t
            r.append(s - dt(num) / dt(math.factorial(sum(al) + len(al) - 1)))
        return np.array(r)

    def jacobian(x):
        h = 1e-30
        J = np.empty((len(tests), len(x)))
        for k in range(len(x)):
            xc = np.asarray(x, dtype=np.complex128)
            xc[k] += 1j * h
            J[:, k] = residual(xc, np.complex128).imag / h
        return J

    x = np.asarray(x0, dtype=np.float64)
    for _ in range(60):
        dx = np.linalg.solve(jacobian(x), -residual(x, np.float64))
        x = x + dx
        if np.max(np.abs(dx)) < 1e-15:
            break
    J = jacobian(x)
    xl = np.asarray(x, dtype=np.longdouble)
    for _ in range(4):  # refinement: long-double residual, double-precision correction
        r = residual(xl, np.longdouble)
        xl = xl - np.linalg.solve(J, r.astype(np.float64)).astype(np.longdouble)
    if np.max(np.abs(residual(xl, np.longdouble).astype(np.float64))) > 1e-17:
        raise RuntimeError("symmetric rule: Newton's method did not converge")
    return xl


def triangle_rule_sym7():
    """7-point fully symmetric rule on the reference triangle, exact for degree 5: the centroid
    and two orbits (a, a, 1 - 2a).  Returns points [7, 2] (xi, eta) = (lam1, lam2) and weights
    summing to the area 1/2."""
    tests = [(0, 0, 0), (2, 0, 0), (3, 0, 0), (4, 0, 0), (5, 0, 0)]

    def orbits_of(x):
        w0, a1, w1, a2, w2 = x
        third = type(w0)(1) / type(w0)(3)
        return [((third, third, third), w0), ((a1, a1, 1 - 2 * a1), w1), ((a2, a2, 1 - 2 * a2), w2)]

    x = _newton_moments(orbits_of, [0.1, 0.1, 0.06, 0.45, 0.07], tests)
    pts, wts = _sym_points(orbits_of(x))
    pts = np.array([[q[1], q[2]] for q in pts], dtype=np.longdouble).astype(np.float64)
    return pts, np.array(wts, dtype=np.longdouble).astype(np.float64)


def tetra_rule_sym14():
    """14-point fully symmetric rule on the reference tetrahedron, exact for degree 5: two
    orbits (a, a, a, 1 - 3a) of 4 points and one orbit (b, b, 1/2 - b, 1/2 - b) of 6.  Returns
    points [14, 3] (xi, eta, zeta) = (lam1, lam2, lam3) and weights summing to the volume 1/6."""
    tests = [(0, 0, 0, 0), (2, 0, 0, 0), (3, 0, 0, 0), (4, 0, 0, 0), (2, 2, 0, 0), (3, 2, 0, 0)]

    def orbits_of(x):
        a1, w1, a2, w2, b, w3 = x
        return [((a1, a1, a1, 1 - 3 * a1), w1), ((a2, a2, a2, 1 - 3 * a2), w2),
                ((b, b, 0.5 - b, 0.5 - b), w3)]

    x = _newton_moments(orbits_of, [0.1, 0.01, 0.3, 0.02, 0.05, 0.007], tests)
    pts, wts = _sym_points(orbits_of(x))
    pts = np.array([[q[1], q[2], q[3]] for q in pts], dtype=np.longdouble).astype(np.float64)
    return pts, np.array(wts, dtype=np.longdouble).astype(np.float64)


def volume_rule(dim: int, p: int):
    """The element rule of the discretisation: collapsed with p + 1 points per direction,
    except tetrahedra at p = 2 (the 14-point symmetric rule)."""
    if dim == 3 and p == 2:
        return tetra_rule_sym14()
    return triangle_rule(p + 1) if dim == 2 else tetra_rule(p + 1)


def face_rule(dim: int, p: int):
    """The face rule: Gauss-Legendre with p + 1 points on [0, 1] (weights summing to 1) for
    edges; for triangular faces the collapsed rule (weights summing to 1/2), except at p = 2
    (the 7-point symmetric rule).  Returns the face points as barycentrics over the face's
    vertices [nfq, dim] and the weights."""
    if dim == 2:
        s, ws = gauss_legendre01(p + 1)
        return np.stack([1.0 - s, s], axis=1), ws
    st, ws = triangle_rule_sym7() if p == 2 else triangle_rule(p + 1)
    return np.stack([1.0 - st[:, 0] - st[:, 1], st[:, 0], st[:, 1]], axis=1), ws
