"""DG spatial operator R(u) of Eq. euler3 for the oracle (Sec. 4.2-4.4).

    R_i = - sum_faces int psi_i F~ . n dsigma + int_E F . grad psi_i dx

with the element-specific orthonormal basis of ``basis.PaperBasis`` (so the
mass matrix is the identity and du/dt = R(u), Eq. starteq), Roe's flux on
interior and periodic faces and Roe's flux against a ghost state on boundary
faces.  Quadrature per ``quadrature``; non-rotating frame (S = 0).

Unknowns are ordered u[e, v, i]: element e, conservative variable v, basis
function i, flattened to a vector of length K = E * nv * N.

J v is the derivative part of R evaluated on dual numbers (the paper's
exact Jacobian by automatic differentiation, Eq. jac1 / jac2).
"""
import numpy as np

from . import adscalar as ad
from . import euler
from .basis import PaperBasis, n_basis
from .quadrature import gauss_legendre01, triangle_rule

BC_SLIP_WALL = 1
BC_FARFIELD = 2


def build_faces(mesh):
    """Face list of a 2D mesh by matching edges on periodic master vertices.

    Local face f of triangle (v0, v1, v2) runs from vertex (f+1)%3 to (f+2)%3.
    Returns interior (incl. periodic) faces as arrays (eL, fL, eR, fR) and
    boundary faces as (e, f, tag).
    """
    elems = mesh.elems
    master = mesh.vert_master
    edges = {}
    for e in range(elems.shape[0]):
        for f in range(3):
            a = int(elems[e, (f + 1) % 3])
            b = int(elems[e, (f + 2) % 3])
            key = tuple(sorted((int(master[a]), int(master[b]))))
            edges.setdefault(key, []).append((e, f))
    btag = {}
    for (a, b), t in zip(mesh.bfaces, mesh.btags):
        btag[tuple(sorted((int(a), int(b))))] = int(t)
    interior, boundary = [], []
    for key, lst in edges.items():
        if len(lst) == 2:
            (eL, fL), (eR, fR) = lst
            interior.append((eL, fL, eR, fR))
        elif len(lst) == 1:
            e, f = lst[0]
            a = int(elems[e, (f + 1) % 3])
            b = int(elems[e, (f + 2) % 3])
            k2 = tuple(sorted((a, b)))
            if k2 not in btag:
                raise ValueError(f"unmatched boundary edge {a}-{b}")
            boundary.append((e, f, btag[k2]))
        else:
            raise ValueError("non-conforming mesh: edge shared by more than two elements")
    return np.array(interior, dtype=np.int64).reshape(-1, 4), np.array(boundary, dtype=np.int64).reshape(-1, 3)


class DGOracle:
    """R(u), J(u) v, time-step sizes and diagnostics on a 2D triangle mesh."""

    def __init__(self, mesh, p: int, free):
        if mesh.dim != 2:
            raise NotImplementedError("oracle residual is written for triangles")
        self.mesh = mesh
        self.p = p
        self.gamma = free.gamma
        self.free = free
        self.dim = 2
        self.nv = 4
        self.N = n_basis(p, 2)
        self.E = mesh.n_elem
        self.K = self.E * self.nv * self.N
        X = mesh.coords
        verts = X[mesh.elems]  # [E, 3, 2]
        self.verts = verts
        # volume quadrature on each physical triangle
        rp, rw = triangle_rule(p + 1)
        Aff = verts[:, 1:, :] - verts[:, 0:1, :]  # rows: v1 - v0, v2 - v0
        det = Aff[:, 0, 0] * Aff[:, 1, 1] - Aff[:, 0, 1] * Aff[:, 1, 0]
        if np.any(det <= 0):
            raise ValueError("elements must be positively oriented")
        self.area = 0.5 * det
        self.rq = np.einsum("qk,ekd->eqd", rp, Aff)  # offsets from v0 (exact edge vectors)
        self.xq = verts[:, 0:1, :] + self.rq
        self.wq = rw[None, :] * det[:, None]
        self.basis = PaperBasis(verts, p, self.rq, self.wq)
        self.psi_q = self.basis.eval(self.rq)  # [E, nq, N]
        self.gpsi_wq = self.basis.grad(self.rq) * self.wq[:, :, None, None]  # [E, nq, N, 2]
        # faces
        interior, boundary = build_faces(mesh)
        s, ws = gauss_legendre01(p + 1)
        self.s, self.ws = s, ws
        self._setup_interior(interior)
        self._setup_boundary(boundary)
        # perimeter for h = 2 d |E| / |dE| (Eq. x3d)
        perim = np.zeros(self.E)
        for f in range(3):
            a = verts[:, (f + 1) % 3]
            b = verts[:, (f + 2) % 3]
            perim += np.linalg.norm(b - a, axis=1)
        self.perimeter = perim
        # free-stream velocity
        c_inf = np.sqrt(self.gamma * free.p / free.rho)
        a = np.deg2rad(free.alpha_deg)
        self.vel_inf = [free.mach * c_inf * np.cos(a), free.mach * c_inf * np.sin(a)]

    # ------------------------------------------------------------------ faces
    def _edge(self, e, f):
        a = self.verts[e, (f + 1) % 3]
        b = self.verts[e, (f + 2) % 3]
        return a, b

    def _setup_interior(self, faces):
        self.fi = faces
        if len(faces) == 0:
            return
        eL, fL, eR, fR = faces.T
        aL, bL = self._edge(eL, fL)
        aR, bR = self._edge(eR, fR)
        # L traverses a -> b; R traverses its copy of the edge in the opposite sense,
        # so L's point a + s (b - a) is R's point bR + s (aR - bR).
        v0 = self.verts[:, 0, :]
        xL = (aL - v0[eL])[:, None, :] + self.s[None, :, None] * (bL - aL)[:, None, :]
        xR = (bR - v0[eR])[:, None, :] + self.s[None, :, None] * (aR - bR)[:, None, :]
        t = bL - aL
        ln = np.linalg.norm(t, axis=1)
        self.fi_n = np.stack([t[:, 1], -t[:, 0]], axis=1) / ln[:, None]
        self.fi_w = ln[:, None] * self.ws[None, :]
        self.fi_psiL = self.basis.eval_rows(eL, xL)  # [F, nfq, N]
        self.fi_psiR = self.basis.eval_rows(eR, xR)

    def _setup_boundary(self, faces):
        self.fb = faces
        if len(faces) == 0:
            return
        e, f, tag = faces.T
        a, b = self._edge(e, f)
        r = (a - self.verts[e, 0, :])[:, None, :] + self.s[None, :, None] * (b - a)[:, None, :]
        x = a[:, None, :] + self.s[None, :, None] * (b - a)[:, None, :]
        t = b - a
        ln = np.linalg.norm(t, axis=1)
        self.fb_n = np.stack([t[:, 1], -t[:, 0]], axis=1) / ln[:, None]
        self.fb_w = ln[:, None] * self.ws[None, :]
        self.fb_psi = self.basis.eval_rows(e, r)
        self.fb_x = x

    # --------------------------------------------------------------- operator
    def unflat(self, u):
        return u.reshape(self.E, self.nv, self.N) if not isinstance(u, ad.Dual) else ad.Dual(
            u.val.reshape(self.E, self.nv, self.N), u.der.reshape(self.E, self.nv, self.N))

    def residual(self, u, volume=True, faces=True):
        """R(u) of Eq. euler3 for u [E, nv, N] (or flat) of any oracle scalar type."""
        flat = (u.val.ndim if isinstance(u, ad.Dual) else np.ndim(u)) == 1
        u = self.unflat(u)
        g = self.gamma
        R = ad.zeros_like_var(u, (self.E, self.nv, self.N))
        if volume:
            Uq = ad.lin(lambda a: np.einsum("eqi,evi->eqv", self.psi_q, a), u)
            for k in range(self.dim):
                Fk = ad.stack(euler.flux_dir(Uq, k, g))  # [E, nq, nv]
                R = R + ad.lin(lambda a, k=k: np.einsum("eqi,eqv->evi", self.gpsi_wq[:, :, :, k], a), Fk)
        if faces and len(self.fi):
            eL, fL, eR, fR = self.fi.T
            UL = ad.lin(lambda a: np.einsum("fqi,fvi->fqv", self.fi_psiL, a[eL]), u)
            UR = ad.lin(lambda a: np.einsum("fqi,fvi->fqv", self.fi_psiR, a[eR]), u)
            n = np.broadcast_to(self.fi_n[:, None, :], UL.shape[:2] + (2,))
            Fn = euler.roe_flux(UL, UR, n, g)  # [F, nfq, nv]
            Fn = Fn * self.fi_w[:, :, None]
            cL = ad.lin(lambda a: np.einsum("fqi,fqv->fvi", self.fi_psiL, a), Fn)
            cR = ad.lin(lambda a: np.einsum("fqi,fqv->fvi", self.fi_psiR, a), Fn)
            R = ad.add_at(R, eL, -cL)
            R = ad.add_at(R, eR, cR)
        if faces and len(self.fb):
            e, f, tag = self.fb.T
            UL = ad.lin(lambda a: np.einsum("fqi,fvi->fqv", self.fb_psi, a[e]), u)
            n = np.broadcast_to(self.fb_n[:, None, :], UL.shape[:2] + (2,))
            wall = (tag == BC_SLIP_WALL)[:, None]
            Ug_w = euler.ghost_slip_wall(UL, n, g)
            Ug_f = euler.ghost_farfield(UL, n, g, self.free.rho, self.vel_inf, self.free.p)
            Ug = ad.where(wall[:, :, None], Ug_w, Ug_f)
            Fn = euler.roe_flux(UL, Ug, n, g) * self.fb_w[:, :, None]
            c = ad.lin(lambda a: np.einsum("fqi,fqv->fvi", self.fb_psi, a), Fn)
            R = ad.add_at(R, e, -c)
        if flat:
            return _flatten(R)
        return R

    def jvp(self, u, v, **kw):
        """J(u) v by forward-mode dual numbers through ``residual`` (Eq. jac1, jac2)."""
        ud = ad.Dual(np.asarray(u, np.float64).reshape(self.E, self.nv, self.N),
                     np.asarray(v, np.float64).reshape(self.E, self.nv, self.N))
        r = self.residual(ud, **kw)
        return r.der.reshape(np.shape(u))

    def jvp_complex_step(self, u, v, h=1e-30, **kw):
        """J(u) v by the complex step Im R(u + i h v) / h (independent pin of ``jvp``)."""
        uc = np.asarray(u, np.complex128).reshape(self.E, self.nv, self.N) + 1j * h * np.asarray(v).reshape(self.E, self.nv, self.N)
        r = self.residual(uc, **kw)
        return (r.imag / h).reshape(np.shape(u))

    def dense_jacobian(self, u):
        """Dense J(u) column by column (tiny meshes only)."""
        uf = np.asarray(u, np.float64).reshape(-1)
        J = np.zeros((self.K, self.K))
        for k in range(self.K):
            ek = np.zeros(self.K)
            ek[k] = 1.0
            J[:, k] = self.jvp(uf, ek)
        return J

    # ------------------------------------------------------------- functionals
    def wall_force(self, u, direction=(1.0, 0.0)):
        """Pressure force on the slip walls along ``direction``: sum over wall faces and Gauss
        points of |e| w_q p(U_L) (n . a) (the bump-force functional of the adjoint case)."""
        u = self.unflat(u)
        if not len(self.fb):
            return 0.0
        e, f, tag = self.fb.T
        UL = ad.lin(lambda a: np.einsum("fqi,fvi->fqv", self.fb_psi, a[e]), u)
        rho, vel, p, E = euler.primitives(UL, self.gamma)
        na = self.fb_n[:, 0] * direction[0] + self.fb_n[:, 1] * direction[1]
        wgt = self.fb_w * (na * (tag == BC_SLIP_WALL))[:, None]
        tot = p * wgt
        if isinstance(tot, ad.Dual):
            return ad.Dual(np.sum(tot.val), np.sum(tot.der))
        return np.sum(tot)

    # ------------------------------------------------------------ projections
    def project(self, fn):
        """L2 projection of a pointwise state function fn(x [E,nq,2]) -> [E,nq,nv]."""
        Uq = fn(self.xq)
        return np.einsum("eq,eqi,eqv->evi", self.wq, self.psi_q, Uq)

    def state_at(self, u, x, local=False):
        """U_h at points x [E, npts, 2] of each element (offsets from v0 when ``local``)."""
        u = np.asarray(u).reshape(self.E, self.nv, self.N)
        psi = self.basis.eval(x if local else self.basis.local(x))
        return np.einsum("eqi,evi->eqv", psi, u)

    def freestream_state(self):
        f = self.free
        vel = self.vel_inf
        E = f.p / (f.gamma - 1.0) + 0.5 * f.rho * (vel[0] ** 2 + vel[1] ** 2)
        return np.array([f.rho, f.rho * vel[0], f.rho * vel[1], E])

    # ------------------------------------------------------------- time steps
    def local_dt(self, u, cfl):
        """Delta t_e = CFL h / ((2p+1)(|v| + c)), h = 2 d |E| / |dE| (Eq. x3d), v at the centroid."""
        U = self.state_at(u, self.basis.rc[:, None, :], local=True)[:, 0, :]
        rho = U[:, 0]
        vel = U[:, 1:3] / rho[:, None]
        p = (self.gamma - 1.0) * (U[:, 3] - 0.5 * rho * np.sum(vel ** 2, axis=1))
        c = np.sqrt(self.gamma * p / rho)
        h = 2.0 * self.dim * self.area / self.perimeter
        return cfl * h / ((2 * self.p + 1) * (np.linalg.norm(vel, axis=1) + c))

    def density_residual_norm(self, R, volume):
        """||R(rho)||_2 of Eq. cfl: (1/|Omega|) sqrt(int R(rho)^2) (orthonormal basis)."""
        R = np.asarray(R).reshape(self.E, self.nv, self.N)
        return np.sqrt(np.sum(R[:, 0, :] ** 2)) / volume

    def entropy_error(self, u, volume):
        """E_L2(s) of Eq. entropy_error, s = p / rho^gamma, s0 of the free stream."""
        U = self.state_at(u, self.rq, local=True)
        rho = U[..., 0]
        vel = U[..., 1:3] / rho[..., None]
        p = (self.gamma - 1.0) * (U[..., 3] - 0.5 * rho * np.sum(vel ** 2, axis=-1))
        s = p / rho ** self.gamma
        s0 = self.free.p / self.free.rho ** self.gamma
        val = np.sum(self.wq * (s / s0) ** 2) / volume - 1.0
        return np.sqrt(max(val, 0.0))


def _flatten(R):
    if isinstance(R, ad.Dual):
        return ad.Dual(R.val.reshape(-1), R.der.reshape(-1))
    return R.reshape(-1)
