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
from .cases import freestream_velocity
from .quadrature import face_rule, volume_rule

BC_SLIP_WALL = 1
BC_FARFIELD = 2
BC_SYMMETRY = 3  # symmetry plane: the slip-wall ghost state (inviscid), not part of the wall force


def face_vertices(dim: int, f: int):
    """Local vertices of local face f: the face opposite vertex f, listed from vertex
    f+1 on (mod dim+1).  For a positively oriented triangle this runs counter-clockwise
    around the element, so the edge (a, b) has outward normal (b - a) rotated by -90
    degrees; in 3D the outward normal is fixed by the opposite vertex."""
    return [(f + k) % (dim + 1) for k in range(1, dim + 1)]


def build_faces(mesh):
    """Face list by matching element faces on periodic master vertices.

    Returns interior (incl. periodic) faces as arrays (eL, fL, eR, fR) with eL the
    element met first (the lower index), and boundary faces as (e, f, tag).
    """
    elems = mesh.elems
    master = mesh.vert_master
    dim = mesh.dim
    faces = {}
    for e in range(elems.shape[0]):
        for f in range(dim + 1):
            vs = [int(elems[e, k]) for k in face_vertices(dim, f)]
            key = tuple(sorted(int(master[v]) for v in vs))
            faces.setdefault(key, []).append((e, f))
    btag = {}
    for verts, t in zip(mesh.bfaces, mesh.btags):
        btag[tuple(sorted(int(v) for v in verts))] = int(t)
    interior, boundary = [], []
    for key, lst in faces.items():
        if len(lst) == 2:
            (eL, fL), (eR, fR) = lst
            interior.append((eL, fL, eR, fR))
        elif len(lst) == 1:
            e, f = lst[0]
            k2 = tuple(sorted(int(elems[e, k]) for k in face_vertices(dim, f)))
            if k2 not in btag:
                raise ValueError(f"unmatched boundary face {k2}")
            boundary.append((e, f, btag[k2]))
        else:
            raise ValueError("non-conforming mesh: face shared by more than two elements")
    return (np.array(interior, dtype=np.int64).reshape(-1, 4),
            np.array(boundary, dtype=np.int64).reshape(-1, 3))


class DGOracle:
    """R(u), J(u) v, time-step sizes and diagnostics on a triangle or tetrahedron mesh.

    omega (optional, 3 components; only omega_z in 2D): angular velocity of a rotating
    frame of reference (Eq. euler): frame velocity v_r = omega x x in the fluxes and the
    source -rho omega x v.  v_r depends on position, so a rotating frame needs a mesh
    without periodic faces, and far-field faces are not defined for it."""

    def __init__(self, mesh, p: int, free, omega=None):
        self.mesh = mesh
        self.p = p
        self.gamma = free.gamma
        self.free = free
        self.dim = dim = mesh.dim
        self.nv = dim + 2
        self.N = n_basis(p, dim)
        self.E = mesh.n_elem
        self.K = self.E * self.nv * self.N
        X = mesh.coords
        verts = X[mesh.elems]  # [E, dim+1, dim]
        self.verts = verts
        # volume quadrature on each physical simplex
        rp, rw = volume_rule(dim, p)
        Aff = verts[:, 1:, :] - verts[:, 0:1, :]  # rows: v_k - v_0 (exact in floating point)
        if dim == 2:
            det = Aff[:, 0, 0] * Aff[:, 1, 1] - Aff[:, 0, 1] * Aff[:, 1, 0]
        else:
            det = np.einsum("ed,ed->e", np.cross(Aff[:, 0], Aff[:, 1]), Aff[:, 2])
        if np.any(det <= 0):
            raise ValueError("elements must be positively oriented")
        self.area = det / (2.0 if dim == 2 else 6.0)  # element measure |E|
        self.rq = np.einsum("qk,ekd->eqd", rp, Aff)  # offsets from v0
        self.xq = verts[:, 0:1, :] + self.rq
        self.wq = rw[None, :] * det[:, None]
        self.basis = PaperBasis(verts, p, self.rq, self.wq)
        self.psi_q = self.basis.eval(self.rq)  # [E, nq, N]
        self.gpsi_wq = self.basis.grad(self.rq) * self.wq[:, :, None, None]  # [E, nq, N, dim]
        # face rule: Gauss-Legendre on [0, 1] (weights sum 1) or a triangle rule (weights
        # sum 1/2); a face point has barycentrics lam over the face vertices
        self.face_bary, ws = face_rule(dim, p)
        self.ws = ws
        interior, boundary = build_faces(mesh)
        self.perimeter = np.zeros(self.E)  # |dE|
        for f in range(dim + 1):
            _, meas = self._face_normal(np.arange(self.E), f)
            self.perimeter += meas
        self._setup_interior(interior)
        self._setup_boundary(boundary)
        self.vel_inf = list(freestream_velocity(free, dim))
        self.omega = None
        if omega is not None and np.any(np.asarray(omega) != 0.0):
            om = np.asarray(omega, dtype=np.float64)
            if dim == 2 and (om[0] != 0.0 or om[1] != 0.0):
                raise ValueError("in 2D the frame rotates about z: omega = (0, 0, omega_z)")
            if np.any(mesh.vert_master != np.arange(mesh.n_vert)):
                raise ValueError("a rotating frame needs a mesh without periodic faces")
            if len(self.fb) and np.any(self.fb[:, 2] == BC_FARFIELD):
                raise ValueError("far-field faces are not defined in a rotating frame")
            self.omega = om
            self.vr_q = self.frame_velocity(self.xq)      # [E, nq, dim]
            if len(self.fi):
                self.vrn_i = np.einsum("fqd,fd->fq", self.frame_velocity(self.fi_x), self.fi_n)
            if len(self.fb):
                self.vrn_b = np.einsum("fqd,fd->fq", self.frame_velocity(self.fb_x), self.fb_n)

    def frame_velocity(self, x):
        """v_r = omega x x at points x [..., dim] (the x-y components in 2D)."""
        om = self.omega
        X = np.zeros(x.shape[:-1] + (3,))
        X[..., : self.dim] = x
        vr = np.cross(np.broadcast_to(om, X.shape), X)
        return vr[..., : self.dim]

    # ------------------------------------------------------------------ faces
    def _face_normal(self, e, f):
        """Outward unit normal and measure of local face f of elements e."""
        f = np.broadcast_to(np.asarray(f), np.shape(e))
        fv = face_vertices(self.dim, f)  # arrays of local vertex indices, one per face
        V = self.verts[e]
        i = np.arange(len(e))
        a = V[i, fv[0]]
        if self.dim == 2:
            t = V[i, fv[1]] - a
            meas = np.linalg.norm(t, axis=1)
            n = np.stack([t[:, 1], -t[:, 0]], axis=1) / meas[:, None]
        else:
            c = np.cross(V[i, fv[1]] - a, V[i, fv[2]] - a)
            meas = 0.5 * np.linalg.norm(c, axis=1)
            sign = np.sign(np.einsum("ed,ed->e", c, a - V[i, f]))
            n = c * (sign / (2.0 * meas))[:, None]
        return n, meas

    def _face_points(self, e, corners):
        """Face points as offsets from v0 of elements e, given each element's own copies of
        the face vertices in the L element's order (corners [F, dim, dim]):
        x = c_0 + sum_k lam_k (c_k - c_0)."""
        r0 = corners[:, 0, :] - self.verts[e, 0, :]
        edges = corners[:, 1:, :] - corners[:, 0:1, :]
        return r0[:, None, :] + np.einsum("qk,fkd->fqd", self.face_bary[:, 1:], edges)

    def _setup_interior(self, faces):
        self.fi = faces
        if len(faces) == 0:
            return
        eL, fL, eR, fR = faces.T
        master = self.mesh.vert_master
        elems = self.mesh.elems
        F = len(faces)
        cornL = np.empty((F, self.dim, self.dim))
        cornR = np.empty((F, self.dim, self.dim))
        for i in range(F):
            lv = [int(elems[eL[i], k]) for k in face_vertices(self.dim, fL[i])]
            rloc = {int(master[elems[eR[i], k]]): k for k in face_vertices(self.dim, fR[i])}
            for j, v in enumerate(lv):
                cornL[i, j] = self.verts[eL[i], face_vertices(self.dim, fL[i])[j]]
                cornR[i, j] = self.verts[eR[i], rloc[int(master[v])]]
        n, meas = self._face_normal(eL, fL)
        self.fi_n = n
        self.fi_w = (meas * (2.0 if self.dim == 3 else 1.0))[:, None] * self.ws[None, :]
        rL = self._face_points(eL, cornL)
        self.fi_x = self.verts[eL, 0, :][:, None, :] + rL  # face points (the L element's copy)
        self.fi_psiL = self.basis.eval_rows(eL, rL)  # [F, nfq, N]
        self.fi_psiR = self.basis.eval_rows(eR, self._face_points(eR, cornR))

    def _setup_boundary(self, faces):
        self.fb = faces
        if len(faces) == 0:
            return
        e, f, tag = faces.T
        corn = np.stack([self.verts[e[i], face_vertices(self.dim, f[i])] for i in range(len(faces))])
        n, meas = self._face_normal(e, f)
        self.fb_n = n
        self.fb_w = (meas * (2.0 if self.dim == 3 else 1.0))[:, None] * self.ws[None, :]
        r = self._face_points(e, corn)
        self.fb_psi = self.basis.eval_rows(e, r)
        self.fb_x = self.verts[e, 0, :][:, None, :] + r

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
        rot = self.omega is not None
        if volume:
            Uq = ad.lin(lambda a: np.einsum("eqi,evi->eqv", self.psi_q, a), u)
            for k in range(self.dim):
                Fk = ad.stack(euler.flux_dir(Uq, k, g, self.vr_q[..., k] if rot else None))  # [E, nq, nv]
                R = R + ad.lin(lambda a, k=k: np.einsum("eqi,eqv->evi", self.gpsi_wq[:, :, :, k], a), Fk)
            if rot:
                # int_E psi_i S(U_h) dx, S = (0, -omega x (rho v), 0) (Eq. euler3)
                om = self.omega
                m = [Uq[..., 1 + k] for k in range(self.dim)] + ([0.0 * Uq[..., 0]] if self.dim == 2 else [])
                cross = [om[1] * m[2] - om[2] * m[1], om[2] * m[0] - om[0] * m[2], om[0] * m[1] - om[1] * m[0]]
                zero = 0.0 * Uq[..., 0]
                Sq = ad.stack([zero] + [-cross[k] for k in range(self.dim)] + [zero])
                R = R + ad.lin(lambda a: np.einsum("eq,eqi,eqv->evi", self.wq, self.psi_q, a), Sq)
        if faces and len(self.fi):
            eL, fL, eR, fR = self.fi.T
            UL = ad.lin(lambda a: np.einsum("fqi,fvi->fqv", self.fi_psiL, a[eL]), u)
            UR = ad.lin(lambda a: np.einsum("fqi,fvi->fqv", self.fi_psiR, a[eR]), u)
            n = np.broadcast_to(self.fi_n[:, None, :], UL.shape[:2] + (self.dim,))
            Fn = euler.roe_flux(UL, UR, n, g, self.vrn_i if rot else None)  # [F, nfq, nv]
            Fn = Fn * self.fi_w[:, :, None]
            cL = ad.lin(lambda a: np.einsum("fqi,fqv->fvi", self.fi_psiL, a), Fn)
            cR = ad.lin(lambda a: np.einsum("fqi,fqv->fvi", self.fi_psiR, a), Fn)
            R = ad.add_at(R, eL, -cL)
            R = ad.add_at(R, eR, cR)
        if faces and len(self.fb):
            e, f, tag = self.fb.T
            UL = ad.lin(lambda a: np.einsum("fqi,fvi->fqv", self.fb_psi, a[e]), u)
            n = np.broadcast_to(self.fb_n[:, None, :], UL.shape[:2] + (self.dim,))
            wall = ((tag == BC_SLIP_WALL) | (tag == BC_SYMMETRY))[:, None]
            Ug_w = euler.ghost_slip_wall(UL, n, g, self.vrn_b if rot else None)
            if rot:
                Ug = Ug_w  # only slip walls and symmetry planes in a rotating frame
            else:
                Ug_f = euler.ghost_farfield(UL, n, g, self.free.rho, self.vel_inf, self.free.p)
                Ug = ad.where(wall[:, :, None], Ug_w, Ug_f)
            Fn = euler.roe_flux(UL, Ug, n, g, self.vrn_b if rot else None) * self.fb_w[:, :, None]
            c = ad.lin(lambda a: np.einsum("fqi,fqv->fvi", self.fb_psi, a), Fn)
            R = ad.add_at(R, e, -c)
        if flat:
            return _flatten(R)
        return R

    def jvp(self, u, v, **kw):
        """J(u) v by forward-mode dual numbers through ``residual`` (Eq. jac1, jac2)."""
        ud = ad.Dual(np.asarray(u).reshape(self.E, self.nv, self.N),
                     np.asarray(v).reshape(self.E, self.nv, self.N))
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
        na = sum(self.fb_n[:, k] * direction[k] for k in range(self.dim))
        wgt = self.fb_w * (na * (tag == BC_SLIP_WALL))[:, None]
        tot = p * wgt
        if isinstance(tot, ad.Dual):
            return ad.Dual(np.sum(tot.val), np.sum(tot.der))
        return np.sum(tot)

    # ------------------------------------------------------------ projections
    def project(self, fn):
        """L2 projection of a pointwise state function fn(x [E,nq,dim]) -> [E,nq,nv]."""
        Uq = fn(self.xq)
        return np.einsum("eq,eqi,eqv->evi", self.wq, self.psi_q, Uq)

    def state_at(self, u, x, local=False):
        """U_h at points x [E, npts, dim] of each element (offsets from v0 when ``local``)."""
        u = np.asarray(u).reshape(self.E, self.nv, self.N)
        psi = self.basis.eval(x if local else self.basis.local(x))
        return np.einsum("eqi,evi->eqv", psi, u)

    def freestream_state(self):
        f = self.free
        vel = self.vel_inf
        E = f.p / (f.gamma - 1.0) + 0.5 * f.rho * sum(v * v for v in vel)
        return np.array([f.rho] + [f.rho * v for v in vel] + [E])

    # ------------------------------------------------------------- time steps
    def local_dt(self, u, cfl):
        """Delta t_e = CFL h / ((2p+1)(|v| + c)), h = 2 d |E| / |dE| (Eq. x3d), v at the centroid."""
        U = self.state_at(u, self.basis.rc[:, None, :], local=True)[:, 0, :]
        rho = U[:, 0]
        vel = U[:, 1:1 + self.dim] / rho[:, None]
        p = (self.gamma - 1.0) * (U[:, self.dim + 1] - 0.5 * rho * np.sum(vel ** 2, axis=1))
        c = np.sqrt(self.gamma * p / rho)
        h = 2.0 * self.dim * self.area / self.perimeter
        if self.omega is not None:
            # reading: in a rotating frame the waves travel with the velocity relative to it
            vel = vel - self.frame_velocity(self.verts.mean(axis=1))
        return cfl * h / ((2 * self.p + 1) * (np.linalg.norm(vel, axis=1) + c))

    def density_residual_norm(self, R, volume):
        """||R(rho)||_2 of Eq. cfl: (1/|Omega|) sqrt(int R(rho)^2) (orthonormal basis)."""
        R = np.asarray(R).reshape(self.E, self.nv, self.N)
        return np.sqrt(np.sum(R[:, 0, :] ** 2)) / volume

    def entropy_error(self, u, volume):
        """E_L2(s) of Eq. entropy_error, s = p / rho^gamma, s0 of the free stream."""
        U = self.state_at(u, self.rq, local=True)
        rho = U[..., 0]
        vel = U[..., 1:1 + self.dim] / rho[..., None]
        p = (self.gamma - 1.0) * (U[..., self.dim + 1] - 0.5 * rho * np.sum(vel ** 2, axis=-1))
        s = p / rho ** self.gamma
        s0 = self.free.p / self.free.rho ** self.gamma
        val = np.sum(self.wq * (s / s0) ** 2) / volume - 1.0
        return np.sqrt(max(val, 0.0))

    def l2_error(self, u, exact):
        """||U_h - U_exact||_L2 over the domain and all conservative variables: the square
        root of sum_e sum_q w_q sum_v (U_h - U_ex)_v^2 at the volume points, exact(x) being
        the pointwise exact state (the vortex-error functional of the 3D case)."""
        uu = self.unflat(u)
        Uq = ad.lin(lambda a: np.einsum("eqi,evi->eqv", self.psi_q, a), uu)
        D = Uq - exact(self.xq)
        tot = (D * D) * self.wq[:, :, None]
        if isinstance(tot, ad.Dual):
            v = np.sqrt(np.sum(tot.val))
            return ad.Dual(v, 0.5 * np.sum(tot.der) / v)
        return np.sqrt(np.sum(tot))


def _flatten(R):
    if isinstance(R, ad.Dual):
        return ad.Dual(R.val.reshape(-1), R.der.reshape(-1))
    return R.reshape(-1)
