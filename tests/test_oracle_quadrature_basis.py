"""Pins of the oracle's quadrature and paper basis (Sec. 4.2-4.3, Eq. basis, Algorithm 1)."""
import math

import numpy as np
import pytest
import scipy.special

import workloads as W
from oracle import quadrature as Q
from oracle.basis import PaperBasis, monomial_exponents
from oracle.dg import DGOracle


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_gauss_legendre_matches_library(n):
    x, w = Q.gauss_legendre01(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(np.sort(x), np.sort(0.5 * (xr + 1)), atol=1e-15, rtol=0)
    assert np.allclose(w[np.argsort(x)], 0.5 * wr[np.argsort(xr)], atol=1e-15, rtol=0)


@pytest.mark.parametrize("n,a", [(2, 1.0), (4, 1.0), (3, 2.0), (5, 2.0)])
def test_gauss_jacobi_matches_library(n, a):
    x, w = Q.gauss_jacobi(n, a, 0.0)
    xr, wr = scipy.special.roots_jacobi(n, a, 0.0)
    i, j = np.argsort(x), np.argsort(xr)
    assert np.allclose(x[i], xr[j], atol=1e-14, rtol=0)
    assert np.allclose(w[i], wr[j], atol=1e-14, rtol=0)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_triangle_rule_exact_to_degree_2n_minus_1(n):
    pts, wts = Q.triangle_rule(n)
    for i in range(2 * n):
        for j in range(2 * n - i):
            exact = math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
            got = np.sum(wts * pts[:, 0] ** i * pts[:, 1] ** j)
            assert abs(got - exact) < 1e-15, (i, j)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_tetra_rule_exact(n):
    pts, wts = Q.tetra_rule(n)
    for i in range(2 * n):
        for j in range(2 * n - i):
            for k in range(2 * n - i - j):
                exact = math.factorial(i) * math.factorial(j) * math.factorial(k) / math.factorial(i + j + k + 3)
                got = np.sum(wts * pts[:, 0] ** i * pts[:, 1] ** j * pts[:, 2] ** k)
                assert abs(got - exact) < 1e-15


def test_monomial_order_reading():
    assert monomial_exponents(3, 2) == [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2),
                                        (3, 0), (2, 1), (1, 2), (0, 3)]
    assert len(monomial_exponents(2, 3)) == 10  # N = (p+1)(p+2)(p+3)/6


@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_paper_basis_orthonormal_and_triangular(p):
    mesh = W.periodic_square(6, 10.0, 0.15, 11)
    dg = DGOracle(mesh, p, W.Freestream())
    M = np.einsum("eq,eqi,eqj->eij", dg.wq, dg.psi_q, dg.psi_q)
    assert np.abs(M - np.eye(dg.N)).max() < 1e-13
    C = dg.basis.C
    assert np.all(np.abs(np.triu(C, 1)) == 0.0)
    assert np.all(np.diagonal(C, axis1=1, axis2=2) > 0)  # s_i > 0
    # psi_1 is the normalised constant
    assert np.allclose(dg.psi_q[:, :, 0], 1.0 / np.sqrt(dg.area)[:, None], rtol=1e-13)


def test_paper_basis_p1_closed_form():
    """For p = 1, psi_2 is X minus its element mean, normalised (MGS against the constant)."""
    mesh = W.periodic_square(3, 1.0, 0.2, 5)
    dg = DGOracle(mesh, 1, W.Freestream())
    X = (dg.xq[..., 0] - dg.basis.xc[:, None, 0]) / dg.basis.L[:, None, 0]
    Xm = np.sum(dg.wq * X, axis=1) / np.sum(dg.wq, axis=1)
    f = X - Xm[:, None]
    f /= np.sqrt(np.sum(dg.wq * f * f, axis=1))[:, None]
    assert np.allclose(dg.psi_q[:, :, 1], f, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_projection_reproduces_polynomials(p):
    """L2 projection onto span(psi) reproduces any polynomial of degree p exactly."""
    mesh = W.periodic_square(4, 2.0, 0.1, 3)
    dg = DGOracle(mesh, p, W.Freestream())

    def poly(x):
        X, Y = x[..., 0], x[..., 1]
        f = 0.3 + 0.2 * X ** p - 0.7 * X * Y ** (p - 1) + 0.1 * Y
        return np.stack([f, 2 * f, -f, f + 1], axis=-1)

    u = dg.project(poly)
    xs = dg.xq + 0.01  # other points inside the element
    got = dg.state_at(u, xs)
    assert np.allclose(got, poly(xs), atol=1e-12)


# ---------------------------------------------------- the symmetric rules of tetrahedra at p = 2
def _bary(pts):
    return np.concatenate([1.0 - pts.sum(axis=1, keepdims=True), pts], axis=1)


def test_symmetric_triangle_rule_is_radons():
    """The 7-point rule is Radon's degree-5 rule, whose closed form is textbook: the centroid
    with weight 9/40 of the area and the orbits (a, a, 1 - 2a), a = (6 -+ sqrt 15)/21, with
    weights (155 -+ sqrt 15)/1200 of the area."""
    pts, wts = Q.triangle_rule_sym7()
    r = math.sqrt(15.0)
    want = [((1 / 3, 1 / 3, 1 / 3), 9 / 80)]
    for a, w in (((6 - r) / 21, (155 - r) / 2400), ((6 + r) / 21, (155 + r) / 2400)):
        for k in range(3):
            b = [a, a, a]
            b[k] = 1 - 2 * a
            want.append((tuple(b), w))
    lam = _bary(pts)
    assert len(lam) == 7
    for b, w in want:
        d = np.abs(lam - np.array(b)).max(axis=1)
        q = int(np.argmin(d))
        assert d[q] < 1e-15 and abs(wts[q] - w) < 1e-16, (b, w)


@pytest.mark.parametrize("rule,dim,n", [(Q.triangle_rule_sym7, 2, 7), (Q.tetra_rule_sym14, 3, 14)])
def test_symmetric_rules_exact_to_degree_5_only(rule, dim, n):
    """Every monomial of degree <= 5 integrates to its closed form i! j! (k!) / (i+j(+k)+dim)!;
    some monomial of degree 6 does not (the rules are of degree 5 exactly)."""
    pts, wts = rule()
    assert pts.shape == (n, dim)
    worst6 = 0.0
    for deg in range(7):
        for ex in np.ndindex(*([deg + 1] * dim)):
            if sum(ex) != deg:
                continue
            exact = math.prod(math.factorial(e) for e in ex) / math.factorial(deg + dim)
            got = np.sum(wts * np.prod(pts ** np.array(ex), axis=1))
            if deg <= 5:
                assert abs(got - exact) < 1e-16, ex  # a few ulps of the summation
            else:
                worst6 = max(worst6, abs(got - exact))
    assert worst6 > 1e-7


@pytest.mark.parametrize("rule", [Q.triangle_rule_sym7, Q.tetra_rule_sym14])
def test_symmetric_rules_positive_interior_and_invariant(rule):
    """Positive weights, points strictly inside, and the weighted point set maps to itself
    under every permutation of the simplex's vertices."""
    import itertools
    pts, wts = rule()
    lam = _bary(pts)
    assert np.all(wts > 0) and np.all(lam > 0) and np.all(lam < 1)
    key = sorted((tuple(np.round(b, 13)), round(w, 15)) for b, w in zip(lam, wts))
    for perm in itertools.permutations(range(lam.shape[1])):
        pk = sorted((tuple(np.round(b[list(perm)], 13)), round(w, 15)) for b, w in zip(lam, wts))
        assert pk == key


def test_rule_selection():
    """Tetrahedra at p = 2 take the symmetric rules; every other case the collapsed rules."""
    assert len(Q.volume_rule(3, 2)[1]) == 14 and len(Q.face_rule(3, 2)[1]) == 7
    assert len(Q.volume_rule(3, 1)[1]) == 8 and len(Q.face_rule(3, 1)[1]) == 4
    assert len(Q.volume_rule(2, 2)[1]) == 9 and len(Q.face_rule(2, 2)[1]) == 3
    lam, w = Q.face_rule(3, 2)
    assert lam.shape == (7, 3) and abs(w.sum() - 0.5) < 1e-16


def test_tetra_p2_basis_orthonormal_and_reproduces_quadratics():
    """On tetrahedra at p = 2 the paper basis is orthonormal under the 14-point rule and the
    projection reproduces a quadratic exactly (both need exactness to degree 4)."""
    mesh = W.periodic_cube_kuhn(3, 1.0, 0.1, 4)
    dg = DGOracle(mesh, 2, W.Freestream())
    M = np.einsum("eq,eqi,eqj->eij", dg.wq, dg.psi_q, dg.psi_q)
    assert np.abs(M - np.eye(dg.N)).max() < 1e-13

    def poly(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        f = 0.3 + 0.2 * X * X - 0.7 * X * Z + 0.1 * Y * Y + 0.05 * Z
        return np.stack([f, 2 * f, -f, 0.5 * f, f + 1], axis=-1)

    u = dg.project(poly)
    xs = dg.xq + 0.001
    assert np.allclose(dg.state_at(u, xs), poly(xs), atol=1e-12)
