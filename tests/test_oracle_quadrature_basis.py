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
