"""The paper's element basis (Sec. 4.3, Eq. basis2, basis and Algorithm 1).

Each element E gets its own orthonormal basis of P^p built in global
Cartesian coordinates:
  * scaled monomials chi about the centroid x_c with half-extents L
    (Eq. basis2), listed by total degree, then by descending x-power, then by
    descending y-power (reading of the garbled index range of Eq. basis2):
    1, X, Y, X^2, XY, Y^2, X^3, X^2 Y, X Y^2, Y^3 in 2D;
  * modified Gram-Schmidt in the element inner product <f, g>_E (Algorithm 1,
    read as standard MGS: psi_i <- chi_i, psi_i -= <psi_i, psi_j> psi_j for
    j < i, then psi_i /= ||psi_i||_E, so s_i > 0).

psi_i = sum_k C[i, k] chi_k with C lower triangular.

Points are passed as offsets r = x - v_0 from each element's first vertex.  The
edge vectors v_k - v_0 are exact in floating point, so X = (r - r_c) / L keeps
full relative precision on elements far from the origin; the same X formed from
absolute points x would carry an error of order eps |x| / L, which on a fine
mesh far from the origin dominates the residual of a uniform state (exactly zero).
"""
import numpy as np


def monomial_exponents(p: int, dim: int):
    """Exponent tuples of the scaled monomials in the order used for Eq. basis2."""
    out = []
    for deg in range(p + 1):
        if dim == 2:
            for px in range(deg, -1, -1):
                out.append((px, deg - px))
        else:
            for px in range(deg, -1, -1):
                for py in range(deg - px, -1, -1):
                    out.append((px, py, deg - px - py))
    return out


def n_basis(p: int, dim: int) -> int:
    return len(monomial_exponents(p, dim))


class PaperBasis:
    """Per-element orthonormal basis of Eq. basis built by Algorithm 1.

    verts: [E, dim+1, dim] element vertices.  rq, wq: volume quadrature points as
    offsets from verts[:, 0] [E, nq, dim] and weights [E, nq] (including the
    element Jacobian) used for the centroid and the inner products.  xc is the
    absolute centroid, rc its offset from verts[:, 0].
    """

    def __init__(self, verts: np.ndarray, p: int, rq: np.ndarray, wq: np.ndarray):
        self.p = p
        self.dim = verts.shape[2]
        self.exps = np.array(monomial_exponents(p, self.dim), dtype=np.int64)  # [N, dim]
        N = len(self.exps)
        vol = wq.sum(axis=1)
        self.origin = verts[:, 0, :].copy()
        self.rc = np.einsum("eq,eqd->ed", wq, rq) / vol[:, None]  # centroid offset
        self.xc = self.origin + self.rc
        self.L = 0.5 * (verts.max(axis=1) - verts.min(axis=1))
        chi = self.monomials(rq)  # [E, nq, N]
        E = verts.shape[0]
        C = np.zeros((E, N, N))
        psi = np.zeros_like(chi)
        for i in range(N):
            ci = np.zeros((E, N))
            ci[:, i] = 1.0
            vi = chi[:, :, i].copy()
            for j in range(i):
                w = np.einsum("eq,eq,eq->e", wq, vi, psi[:, :, j])
                vi -= w[:, None] * psi[:, :, j]
                ci -= w[:, None] * C[:, j, :]
            nrm = np.sqrt(np.einsum("eq,eq,eq->e", wq, vi, vi))
            psi[:, :, i] = vi / nrm[:, None]
            C[:, i, :] = ci / nrm[:, None]
        self.C = C

    def local(self, x: np.ndarray, rows=None) -> np.ndarray:
        """Offsets of absolute points x [E or len(rows), npts, dim] from each element's v_0."""
        o = self.origin if rows is None else self.origin[rows]
        return x - o[:, None, :]

    def _X(self, r, rows):
        rc = self.rc if rows is None else self.rc[rows]
        L = self.L if rows is None else self.L[rows]
        return (r - rc[:, None, :]) / L[:, None, :], L

    def monomials(self, r: np.ndarray, rows=None) -> np.ndarray:
        """chi_k at local points r [E, npts, dim] -> [E, npts, N]."""
        X, _ = self._X(r, rows)
        out = np.ones(r.shape[:2] + (len(self.exps),))
        for k, ex in enumerate(self.exps):
            for d in range(self.dim):
                if ex[d]:
                    out[:, :, k] *= X[:, :, d] ** ex[d]
        return out

    def monomial_grads(self, r: np.ndarray) -> np.ndarray:
        """d chi_k / d x_d at local points r [E, npts, dim] -> [E, npts, N, dim]."""
        X, _ = self._X(r, None)
        out = np.zeros(r.shape[:2] + (len(self.exps), self.dim))
        for k, ex in enumerate(self.exps):
            for d in range(self.dim):
                if ex[d] == 0:
                    continue
                g = ex[d] * X[:, :, d] ** (ex[d] - 1) / self.L[:, None, d]
                for d2 in range(self.dim):
                    if d2 != d and ex[d2]:
                        g = g * X[:, :, d2] ** ex[d2]
                out[:, :, k, d] = g
        return out

    def eval(self, r: np.ndarray) -> np.ndarray:
        """psi_i at local points r [E, npts, dim] -> [E, npts, N]."""
        return np.einsum("eik,eqk->eqi", self.C, self.monomials(r))

    def grad(self, r: np.ndarray) -> np.ndarray:
        """grad psi_i at local points r [E, npts, dim] -> [E, npts, N, dim]."""
        return np.einsum("eik,eqkd->eqid", self.C, self.monomial_grads(r))

    def eval_rows(self, rows: np.ndarray, r: np.ndarray) -> np.ndarray:
        """psi of elements ``rows`` at their local points r [len(rows), npts, dim]."""
        return np.einsum("eik,eqk->eqi", self.C[rows], self.monomials(r, rows))
