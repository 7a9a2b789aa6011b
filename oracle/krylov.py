"""Krylov projection and the small phi-function for the oracle (Sec. 2.2).

Arnoldi (Eq. vm, vm1, vm2): J V_m = V_{m+1} H~_m with v_1 = b / ||b||.  The
oracle orthogonalises with modified Gram-Schmidt followed by one full
re-orthogonalisation pass; any Gram-Schmidt variant spans the same Krylov
space and gives the same H~_m to rounding.  Reading of the paper's "Krylov
tolerance": the dimension m is fixed; a happy breakdown at step j
(h_{j+1,j} <= eta ||J v_j||) truncates V and H to j columns.

phi functions (Eq. Phi1, Phi2, final): phi_1(dt H) e_1 and phi_2(dt H) e_1
are read off the exponential of the augmented matrix
    [[dt H, e_1, 0], [0, 0, 1], [0, 0, 0]]
(the (0,1) block of exp is phi_1 e_1 and the (0,2) block phi_2 e_1), which
avoids H^{-1} (H may be singular).  The oracle takes that exponential by a
truncated Taylor series with scaling and squaring in extended precision
(numpy longdouble), not by the Pade/Chebyshev rational forms.
"""
import math

import numpy as np


def arnoldi(matvec, b, m: int, eta: float = 1e-12):
    """Arnoldi with MGS + one re-orthogonalisation pass.

    Returns (V [K, k+1], Hbar [k+1, k], k, beta, breakdown) where k <= m is the
    dimension reached.  beta = ||b||; beta == 0 returns k = 0.
    """
    b = np.asarray(b, dtype=np.float64)
    beta = float(np.sqrt(np.dot(b, b)))
    K = b.shape[0]
    if beta == 0.0:
        return np.zeros((K, 1)), np.zeros((1, 0)), 0, 0.0, True
    V = np.zeros((K, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = b / beta
    for j in range(m):
        w = np.asarray(matvec(V[:, j]), dtype=np.float64).copy()
        w0 = float(np.sqrt(np.dot(w, w)))
        for _ in range(2):
            for i in range(j + 1):
                h = float(np.dot(V[:, i], w))
                H[i, j] += h
                w -= h * V[:, i]
        hn = float(np.sqrt(np.dot(w, w)))
        H[j + 1, j] = hn
        if not np.isfinite(hn):
            raise FloatingPointError("non-finite Arnoldi norm")
        if hn <= eta * w0:
            k = j + 1
            return V[:, :k], H[: k + 1, :k], k, beta, True
        V[:, j + 1] = w / hn
    return V, H, m, beta, False


def expm_taylor(A: np.ndarray) -> np.ndarray:
    """exp(A) by Taylor series after scaling A / 2^s to 1-norm <= 1/2, then squaring.

    Runs in numpy longdouble (80-bit on x86-64, 128-bit on AArch64).
    """
    A = np.asarray(A, dtype=np.longdouble)
    n = A.shape[0]
    nrm = float(np.max(np.sum(np.abs(A), axis=0))) if n else 0.0
    s = 0
    if nrm > 0.5:
        s = int(math.ceil(math.log2(nrm / 0.5)))
    B = A / np.longdouble(2.0) ** s
    eps = np.finfo(np.longdouble).eps
    T = np.eye(n, dtype=np.longdouble)
    term = np.eye(n, dtype=np.longdouble)
    for k in range(1, 80):
        term = term @ B / np.longdouble(k)
        T = T + term
        if float(np.max(np.abs(term))) <= float(eps) * float(np.max(np.abs(T))):
            break
    for _ in range(s):
        T = T @ T
    return T


def phi_e1(H: np.ndarray, dt: float):
    """(phi_1(dt H) e_1, phi_2(dt H) e_1) for square H [k, k] via the augmented exponential."""
    k = H.shape[0]
    A = np.zeros((k + 2, k + 2), dtype=np.longdouble)
    A[:k, :k] = np.asarray(H, dtype=np.longdouble) * np.longdouble(dt)
    if k:
        A[0, k] = 1.0
    A[k, k + 1] = 1.0
    X = expm_taylor(A)
    return np.asarray(X[:k, k], dtype=np.float64), np.asarray(X[:k, k + 1], dtype=np.float64)


def krylov_phi1(matvec, b, dt: float, m: int, eta: float = 1e-12):
    """phi_1(dt J) b ~= ||b|| V_k phi_1(dt H_k) e_1 (Eq. final).

    Returns (x, info) with info = dict(k=..., beta=..., breakdown=...).
    """
    V, Hb, k, beta, brk = arnoldi(matvec, b, m, eta)
    if k == 0:
        return np.zeros_like(np.asarray(b, np.float64)), dict(k=0, beta=0.0, breakdown=True)
    y, _ = phi_e1(Hb[:k, :k], dt)
    return beta * (V[:, :k] @ y), dict(k=k, beta=beta, breakdown=brk, H=Hb)
