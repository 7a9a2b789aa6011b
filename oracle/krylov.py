"""Krylov projection and the small phi-function for the oracle (Sec. 2.2).

Arnoldi (Eq. vm, vm1, vm2): J V_m = V_{m+1} H~_m with v_1 = b / ||b||.  The
oracle orthogonalises with modified Gram-Schmidt followed by one full
re-orthogonalisation pass; any Gram-Schmidt variant spans the same Krylov
space and gives the same H~_m to rounding.  Reading of the paper's "Krylov
tolerance" (Sec. 5, 1e-5): by default the dimension m is fixed; with a tolerance the
process stops at the first checkpoint whose a-posteriori error estimate (Saad 1992) is
within it.  A happy breakdown at step j (h_{j+1,j} <= eta ||J v_j||) truncates V and H
to j columns.

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


def arnoldi(matvec, b, m: int, eta: float = 1e-12, stop=None, check: int = 5):
    """Arnoldi with MGS + one re-orthogonalisation pass.

    Returns (V [K, k+1], Hbar [k+1, k], k, beta, breakdown) where k <= m is the
    dimension reached.  beta = ||b||; beta == 0 returns k = 0.  stop(k, Hbar_k) (optional)
    is asked after every ``check``-th column k < m; True ends the process at dimension k.
    """
    # real (FP64) or complex (a complex step through the whole process: dot products without
    # conjugation, decisions on real parts)
    ty = np.result_type(b, np.float64)
    b = np.asarray(b, dtype=ty)
    beta = np.sqrt(np.dot(b, b))
    K = b.shape[0]
    if beta == 0.0:
        return np.zeros((K, 1), ty), np.zeros((1, 0), ty), 0, 0.0, True
    V = np.zeros((K, m + 1), ty)
    H = np.zeros((m + 1, m), ty)
    V[:, 0] = b / beta
    for j in range(m):
        w = np.asarray(matvec(V[:, j]), dtype=ty).copy()
        w0 = np.sqrt(np.dot(w, w))
        for _ in range(2):
            for i in range(j + 1):
                h = np.dot(V[:, i], w)
                H[i, j] += h
                w -= h * V[:, i]
        hn = np.sqrt(np.dot(w, w))
        H[j + 1, j] = hn
        if not np.isfinite(hn):
            raise FloatingPointError("non-finite Arnoldi norm")
        if np.real(hn) <= eta * np.real(w0):
            k = j + 1
            return V[:, :k], H[: k + 1, :k], k, beta, True
        V[:, j + 1] = w / hn
        k = j + 1
        if stop is not None and k < m and k % check == 0 and stop(k, H[: k + 1, :k]):
            return V[:, : k + 1], H[: k + 1, :k], k, beta, False
    return V, H, m, beta, False


def expm_taylor(A: np.ndarray) -> np.ndarray:
    """exp(A) by Taylor series after scaling A / 2^s to 1-norm <= 1/2, then squaring.

    Runs in numpy longdouble (80-bit on x86-64, 128-bit on AArch64), complex longdouble for
    complex input.
    """
    A = np.asarray(A, dtype=np.clongdouble if np.iscomplexobj(A) else np.longdouble)
    n = A.shape[0]
    nrm = float(np.max(np.sum(np.abs(A), axis=0))) if n else 0.0
    s = 0
    if nrm > 0.5:
        s = int(math.ceil(math.log2(nrm / 0.5)))
    B = A / np.longdouble(2.0) ** s
    eps = np.finfo(np.longdouble).eps
    T = np.eye(n, dtype=A.dtype)
    term = np.eye(n, dtype=A.dtype)
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
    cx = np.iscomplexobj(H)
    A = np.zeros((k + 2, k + 2), dtype=np.clongdouble if cx else np.longdouble)
    A[:k, :k] = np.asarray(H, dtype=A.dtype) * np.longdouble(dt)
    if k:
        A[0, k] = 1.0
    A[k, k + 1] = 1.0
    X = expm_taylor(A)
    out = np.complex128 if cx else np.float64
    return np.asarray(X[:k, k], dtype=out), np.asarray(X[:k, k + 1], dtype=out)


def error_estimate(Hb, dt: float):
    """Relative a-posteriori error of the Krylov phi_1 product of dimension k (Saad 1992,
    cited in Sec. 2.2; the leading term of the error expansion of Eq. final):

        ||phi_1(dt J) b - beta V_k phi_1(dt H_k) e_1|| / ||beta V_k phi_1(dt H_k) e_1||
          ~= dt h_{k+1,k} |e_k^T phi_2(dt H_k) e_1| / ||phi_1(dt H_k) e_1||,

    from Hbar [k+1, k] (row k holds h_{k+1,k}).  Both phi columns come from one augmented
    exponential (Eq. Phi1, Phi2)."""
    k = Hb.shape[1]
    y1, y2 = phi_e1(Hb[:k, :k], dt)
    return float(dt * abs(Hb[k, k - 1]) * abs(y2[k - 1]) / np.linalg.norm(y1))


def krylov_phi1(matvec, b, dt: float, m: int, eta: float = 1e-12, tol: float = 0.0, check: int = 5):
    """phi_1(dt J) b ~= ||b|| V_k phi_1(dt H_k) e_1 (Eq. final).

    tol > 0 reads the paper's Krylov tolerance (Sec. 5) as an adaptive dimension: the
    Arnoldi process stops at the first k (a multiple of ``check``, k < m) whose relative
    error estimate (``error_estimate``) is <= tol; otherwise k = m (or the breakdown
    dimension).  Returns (x, info) with info = dict(k, beta, breakdown, H, err) where err is
    the estimate at the dimension used.
    """
    stop = (lambda k, Hk: error_estimate(Hk, dt) <= tol) if tol > 0 else None
    V, Hb, k, beta, brk = arnoldi(matvec, b, m, eta, stop, check)
    if k == 0:
        return np.zeros_like(np.asarray(b, np.result_type(b, np.float64))), dict(k=0, beta=0.0, breakdown=True,
                                                                                  err=0.0)
    y, _ = phi_e1(Hb[:k, :k], dt)
    err = error_estimate(np.real(Hb[: k + 1, :k]), dt)
    return beta * (V[:, :k] @ y), dict(k=k, beta=beta, breakdown=brk, H=Hb, err=err)


def krylov_phi2(matvec, b, dt: float, m: int, eta: float = 1e-12):
    """phi_2(dt J) b ~= ||b|| V_k phi_2(dt H_k) e_1 (Eq. Phi2 through the projection of
    Eq. final; the second phi column of the same augmented exponential).

    Returns (x, info) as ``krylov_phi1``."""
    V, Hb, k, beta, brk = arnoldi(matvec, b, m, eta)
    if k == 0:
        return np.zeros_like(np.asarray(b, np.result_type(b, np.float64))), dict(k=0, beta=0.0, breakdown=True)
    _, y2 = phi_e1(Hb[:k, :k], dt)
    return beta * (V[:, :k] @ y2), dict(k=k, beta=beta, breakdown=brk, H=Hb)

