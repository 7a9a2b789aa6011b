"""ctypes binding of include/pcexp.h: the same entry points, argument marshalling only.

Every step of the compute path runs in libpcexp.so.  Arrays may be numpy
float64 arrays (host, ``on_device=0``) or CUDA torch tensors (``on_device=1``);
torch is used only for device memory and the stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, up_to_date

PCEXP_OK = 0
PCEXP_ERR_INVALID_ARG = -1
PCEXP_ERR_MESH = -2
PCEXP_ERR_CUDA = -3
PCEXP_ERR_OOM = -4
PCEXP_ERR_NONFINITE = -5
PCEXP_ERR_TIMEOUT = -6
PCEXP_ERR_UNSUPPORTED = -7
PCEXP_BC_SLIP_WALL = 1
PCEXP_BC_FARFIELD = 2
PCEXP_BC_SYMMETRY = 3
PCEXP_FP64 = 0
PCEXP_FP32_MIXED = 1
PCEXP_BASIS_PAPER = 0
PCEXP_BASIS_INTERNAL = 1
PCEXP_REORTH_AUTO = 0
PCEXP_REORTH_ALWAYS = 1
PCEXP_REORTH_SELECTIVE = 2
PCEXP_SCHEME_PCEXP = 0
PCEXP_SCHEME_EXP1 = 1
PCEXP_SCHEME_ETD2 = 2
PCEXP_DT_GIVEN = 0
PCEXP_DT_GLOBAL_CFL = 1
PCEXP_DT_LOCAL_CFL = 2
PCEXP_PROJ_FREESTREAM = 0
PCEXP_PROJ_VORTEX = 1
PCEXP_PROJ_BLOBS = 2
PCEXP_MAX_KRYLOV = 32
PCEXP_FUNC_WALL_FX = 0
PCEXP_FUNC_WALL_FY = 1
PCEXP_FUNC_VORTEX_L2 = 2
PCEXP_FUNC_WALL_FZ = 3
KERNEL_CLASSES = ["residual_face", "residual_elem", "jvp_face", "jvp_elem", "cgs_norm", "cgs_proj",
                  "cgs_upd_proj", "cgs_upd_norm", "phi", "axpy", "dt", "other", "linearize", "cgs_upd1",
                  "cgs_proj2"]


class pcexp_mesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_vert", C.c_int64), ("coords", C.POINTER(C.c_double)),
                ("n_elem", C.c_int64), ("elem_vert", C.POINTER(C.c_int32)),
                ("vert_master", C.POINTER(C.c_int32)), ("n_bface", C.c_int64),
                ("bface_vert", C.POINTER(C.c_int32)), ("bface_tag", C.POINTER(C.c_int32))]


class pcexp_physics(C.Structure):
    _fields_ = [("gamma", C.c_double), ("mach", C.c_double), ("alpha_deg", C.c_double),
                ("rho_inf", C.c_double), ("p_inf", C.c_double), ("omega", C.c_double * 3)]


def _physics(free, omega):
    om = (C.c_double * 3)(*(omega if omega is not None else (0.0, 0.0, 0.0)))
    return pcexp_physics(free.gamma, free.mach, free.alpha_deg, free.rho, free.p, om)


class pcexp_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("m_max", C.c_int32), ("breakdown_eta", C.c_double),
                ("basis_io", C.c_int32), ("krylov_tol", C.c_double), ("reorth", C.c_int32)]


class pcexp_step_info(C.Structure):
    _fields_ = [("krylov_dim", C.c_int32 * 2), ("beta", C.c_double * 2), ("dt", C.c_double),
                ("res_norm", C.c_double), ("krylov_err", C.c_double * 2), ("reorth_cols", C.c_uint32 * 2)]


class pcexp_steady_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("res_first", C.c_double), ("res_last", C.c_double),
                ("converged", C.c_int32)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
SIGNATURES = {
    "pcexp_create": (C.c_int, [C.POINTER(_P), C.POINTER(pcexp_mesh), C.c_int, C.POINTER(pcexp_physics),
                               C.POINTER(pcexp_options), _P]),
    "pcexp_destroy": (C.c_int, [_P]),
    "pcexp_sizes": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                              C.POINTER(C.c_int64)]),
    "pcexp_set_state": (C.c_int, [_P, _P, C.c_int]),
    "pcexp_get_state": (C.c_int, [_P, _P, C.c_int]),
    "pcexp_project_state": (C.c_int, [_P, C.c_int, _D, C.c_int]),
    "pcexp_residual": (C.c_int, [_P, _P, _P, C.c_int]),
    "pcexp_jvp": (C.c_int, [_P, _P, _P, _P, C.c_int]),
    "pcexp_vjp": (C.c_int, [_P, _P, _P, _P, C.c_int]),
    "pcexp_jvp_state_adjoint": (C.c_int, [_P, _P, _P, _P, _P, C.c_int]),
    "pcexp_compute_dt": (C.c_int, [_P, C.c_double, C.c_int, _P, C.c_int]),
    "pcexp_arnoldi": (C.c_int, [_P, _P, _P, C.c_int, _P, _D, C.POINTER(C.c_int), _D, C.c_int]),
    "pcexp_phi": (C.c_int, [_P, _D, C.c_int, C.c_int, C.c_double, _D, _D]),
    "pcexp_step": (C.c_int, [_P, C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(pcexp_step_info)]),
    "pcexp_phi_adjoint": (C.c_int, [_P, _D, C.c_int, C.c_int, C.c_double, _D, _D]),
    "pcexp_step_backward": (C.c_int, [_P, _P, C.c_double, C.c_int, _P, _P, _D, C.c_int]),
    "pcexp_project_state_adjoint": (C.c_int, [_P, C.c_int, _D, C.c_int, _P, _D, C.c_int]),
    "pcexp_functional_param_grad": (C.c_int, [_P, C.c_int, _D, C.c_int, _P, _D, C.c_int]),
    "pcexp_march_steady": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                     C.POINTER(pcexp_steady_info)]),
    "pcexp_output": (C.c_int, [_P, C.c_int, _D]),
    "pcexp_functional": (C.c_int, [_P, C.c_int, _P, _D, _P, C.c_int]),
    "pcexp_functional_params": (C.c_int, [_P, C.c_int, _D, C.c_int, _P, _D, _P, C.c_int]),
    "pcexp_set_physics": (C.c_int, [_P, C.POINTER(pcexp_physics)]),
    "pcexp_synchronize": (C.c_int, [_P]),
    "pcexp_residual_noalloc": (C.c_int, [_P, _P, _P]),
    "pcexp_profile_enable": (C.c_int, [_P, C.c_int]),
    "pcexp_profile_read": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int64), _D]),
    "pcexp_fp64_fma_rate": (C.c_int, [_D]),
    "pcexp_fp32_fma_rate": (C.c_int, [_D]),
    "pcexp_partition": (C.c_int, [C.POINTER(pcexp_mesh), C.c_int, _P]),
    "pcexp_partition_halo": (C.c_int, [C.POINTER(pcexp_mesh), _P, C.c_int, C.c_int, C.POINTER(C.c_int64),
                                       C.POINTER(C.c_int64), _P]),
    "pcexp_group_create": (C.c_int, [C.POINTER(_P), C.POINTER(pcexp_mesh), _P, C.c_int, _P, C.c_int,
                                     C.POINTER(pcexp_physics), C.POINTER(pcexp_options)]),
    "pcexp_group_destroy": (C.c_int, [_P]),
    "pcexp_group_sizes": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "pcexp_group_set_state": (C.c_int, [_P, _P]),
    "pcexp_group_get_state": (C.c_int, [_P, _P]),
    "pcexp_group_project_state": (C.c_int, [_P, C.c_int, _D, C.c_int]),
    "pcexp_group_residual": (C.c_int, [_P, _P, _P]),
    "pcexp_group_jvp": (C.c_int, [_P, _P, _P, _P]),
    "pcexp_group_arnoldi": (C.c_int, [_P, _P, _P, C.c_int, _D, C.POINTER(C.c_int), _D]),
    "pcexp_group_vjp": (C.c_int, [_P, _P, _P, _P]),
    "pcexp_group_step_backward": (C.c_int, [_P, _P, C.c_double, C.c_int, _P, _P, _D]),
    "pcexp_group_jvp_state_adjoint": (C.c_int, [_P, _P, _P, _P, _P]),
    "pcexp_group_step": (C.c_int, [_P, C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(pcexp_step_info)]),
    "pcexp_group_march_steady": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                           C.POINTER(pcexp_steady_info)]),
    "pcexp_status_string": (C.c_char_p, [C.c_int]),
    "pcexp_last_error": (C.c_char_p, []),
}

_lib = None


def load(path: str | None = None):
    """Load libpcexp.so (built in-tree by ``build()``); raises if it is missing or stale."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_1801_06300_gb300.build() (no CPU fallback exists)")
    if not up_to_date():
        raise RuntimeError(f"{path} is older than its sources: rebuild with paper_1801_06300_gb300.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def fp64_fma_rate() -> float:
    """FP64 FMA rate of the current device in TFLOP/s (DFMA chains on every SM)."""
    lib = load()
    v = C.c_double()
    check(lib.pcexp_fp64_fma_rate(C.byref(v)), "pcexp_fp64_fma_rate")
    return v.value


def fp32_fma_rate() -> float:
    """FP32 FMA rate of the current device in TFLOP/s (FFMA chains on every SM)."""
    lib = load()
    v = C.c_double()
    check(lib.pcexp_fp32_fma_rate(C.byref(v)), "pcexp_fp32_fma_rate")
    return v.value


class PcexpError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        super().__init__(f"{where}: {lib.pcexp_status_string(code).decode()} ({code}): "
                         f"{lib.pcexp_last_error().decode()}")
        self.code = code


def check(code: int, where: str):
    if code != PCEXP_OK:
        raise PcexpError(code, where)


def _ptr(x):
    """(pointer, on_device) of a numpy float64 array or a CUDA torch tensor."""
    if isinstance(x, np.ndarray):
        assert x.dtype == np.float64 and x.flags.c_contiguous
        return x.ctypes.data_as(C.c_void_p), 0
    # torch tensor
    assert x.is_contiguous() and str(x.dtype) == "torch.float64"
    return C.c_void_p(x.data_ptr()), 1 if x.is_cuda else 0


def _mesh_struct(mesh):
    """(pcexp_mesh, arrays it points into): keep the arrays alive while the struct is used."""
    coords = np.ascontiguousarray(mesh.coords, np.float64)
    elems = np.ascontiguousarray(mesh.elems, np.int32)
    master = np.ascontiguousarray(mesh.vert_master, np.int32)
    bfv = np.ascontiguousarray(mesh.bfaces, np.int32).reshape(-1)
    btag = np.ascontiguousarray(mesh.btags, np.int32)
    ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))  # noqa: E731
    m = pcexp_mesh(mesh.dim, coords.shape[0], coords.ctypes.data_as(_D), elems.shape[0], ip(elems),
                   ip(master), btag.shape[0], ip(bfv) if bfv.size else None, ip(btag) if btag.size else None)
    return m, [coords, elems, master, bfv, btag]


def partition(mesh, n_parts: int) -> np.ndarray:
    """pcexp_partition: int32 partition index of every element (host only)."""
    lib = load()
    m, keep = _mesh_struct(mesh)
    part = np.empty(len(mesh.elems), np.int32)
    check(lib.pcexp_partition(C.byref(m), n_parts, part.ctypes.data_as(_P)), "pcexp_partition")
    return part


def partition_halo(mesh, part, k: int):
    """pcexp_partition_halo: (own elements, halo elements) of partition k (host only)."""
    lib = load()
    m, keep = _mesh_struct(mesh)
    part = np.ascontiguousarray(part, np.int32)
    el = np.empty(len(mesh.elems), np.int64)
    no, nt = C.c_int64(), C.c_int64()
    check(lib.pcexp_partition_halo(C.byref(m), part.ctypes.data_as(_P), int(part.max()) + 1, k, C.byref(no),
                                   C.byref(nt), el.ctypes.data_as(_P)), "pcexp_partition_halo")
    return el[:no.value].copy(), el[no.value:nt.value].copy()


class Group:
    """Owns one pcexp_group (a partitioned run, host arrays of the whole mesh)."""

    def __init__(self, mesh, part, p: int, free, precision: int = PCEXP_FP64, m_max: int = 30,
                 eta: float = 0.0, basis_io: int = PCEXP_BASIS_PAPER, devices=None, omega=None,
                 krylov_tol: float = 0.0, reorth: int = 0):
        lib = load()
        m, self._keep = _mesh_struct(mesh)
        part = np.ascontiguousarray(part, np.int32)
        self.n = int(part.max()) + 1
        dev = None if devices is None else np.ascontiguousarray(devices, np.int32)
        ph = _physics(free, omega)
        op = pcexp_options(precision, m_max, eta, basis_io, krylov_tol, reorth)
        self.g = C.c_void_p()
        check(lib.pcexp_group_create(C.byref(self.g), C.byref(m), part.ctypes.data_as(_P), self.n,
                                     dev.ctypes.data_as(_P) if dev is not None else None, p, C.byref(ph),
                                     C.byref(op)), "pcexp_group_create")
        self.lib = lib
        nv = mesh.dim + 2
        nb = {2: (p + 1) * (p + 2) // 2, 3: (p + 1) * (p + 2) * (p + 3) // 6}[mesh.dim]
        self.K = len(mesh.elems) * nv * nb

    def sizes(self, k: int):
        a, b = C.c_int64(), C.c_int64()
        check(self.lib.pcexp_group_sizes(self.g, k, C.byref(a), C.byref(b)), "pcexp_group_sizes")
        return a.value, b.value

    def close(self):
        if getattr(self, "g", None) is not None and self.g.value:
            self.lib.pcexp_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _host(self, x):
        x = np.ascontiguousarray(x, np.float64)
        assert x.size == self.K
        return x

    def set_state(self, U):
        U = self._host(U)
        check(self.lib.pcexp_group_set_state(self.g, U.ctypes.data_as(_P)), "pcexp_group_set_state")

    def get_state(self):
        out = np.empty(self.K)
        check(self.lib.pcexp_group_get_state(self.g, out.ctypes.data_as(_P)), "pcexp_group_get_state")
        return out

    def project_state(self, kind: int, params=()):
        prm = np.ascontiguousarray(params, np.float64)
        check(self.lib.pcexp_group_project_state(self.g, kind, prm.ctypes.data_as(_D) if prm.size else None,
                                                 prm.size), "pcexp_group_project_state")

    def residual(self, U):
        U, out = self._host(U), np.empty(self.K)
        check(self.lib.pcexp_group_residual(self.g, U.ctypes.data_as(_P), out.ctypes.data_as(_P)),
              "pcexp_group_residual")
        return out

    def jvp(self, U, v):
        U, v, out = self._host(U), self._host(v), np.empty(self.K)
        check(self.lib.pcexp_group_jvp(self.g, U.ctypes.data_as(_P), v.ctypes.data_as(_P), out.ctypes.data_as(_P)),
              "pcexp_group_jvp")
        return out

    def step_backward(self, U, dt: float, m: int, ubar_next):
        """(ubar_n, theta_bar = d/d(Mach, alpha in degrees)) of one PCEXP step at fixed dt."""
        U, ub, out = self._host(U), self._host(ubar_next), np.empty(self.K)
        th = np.zeros(2)
        check(self.lib.pcexp_group_step_backward(self.g, U.ctypes.data_as(_P), dt, m, ub.ctypes.data_as(_P),
                                                 out.ctypes.data_as(_P), th.ctypes.data_as(_D)),
              "pcexp_group_step_backward")
        return out, th

    def vjp(self, U, w):
        U, w, out = self._host(U), self._host(w), np.empty(self.K)
        check(self.lib.pcexp_group_vjp(self.g, U.ctypes.data_as(_P), w.ctypes.data_as(_P), out.ctypes.data_as(_P)),
              "pcexp_group_vjp")
        return out

    def jvp_state_adjoint(self, U, v, w):
        U, v, w, out = self._host(U), self._host(v), self._host(w), np.empty(self.K)
        check(self.lib.pcexp_group_jvp_state_adjoint(self.g, U.ctypes.data_as(_P), v.ctypes.data_as(_P),
                                                     w.ctypes.data_as(_P), out.ctypes.data_as(_P)),
              "pcexp_group_jvp_state_adjoint")
        return out

    def arnoldi(self, U, b, m: int):
        U, b = self._host(U), self._host(b)
        H = np.zeros((m + 1) * m)
        k, beta = C.c_int(), C.c_double()
        check(self.lib.pcexp_group_arnoldi(self.g, U.ctypes.data_as(_P), b.ctypes.data_as(_P), m,
                                           H.ctypes.data_as(_D), C.byref(k), C.byref(beta)), "pcexp_group_arnoldi")
        return H.reshape(m + 1, m), k.value, beta.value

    def march_steady(self, scheme: int, cfl_max: float, decades: float, max_iter: int, m: int):
        inf = pcexp_steady_info()
        check(self.lib.pcexp_group_march_steady(self.g, scheme, cfl_max, decades, max_iter, m, C.byref(inf)),
              "pcexp_group_march_steady")
        return dict(iterations=inf.iterations, res_first=inf.res_first, res_last=inf.res_last,
                    converged=bool(inf.converged))

    def step(self, scheme: int, dt_mode: int, dt_or_cfl: float, m: int):
        inf = pcexp_step_info()
        check(self.lib.pcexp_group_step(self.g, scheme, dt_mode, dt_or_cfl, m, C.byref(inf)), "pcexp_group_step")
        return dict(k=(inf.krylov_dim[0], inf.krylov_dim[1]), beta=(inf.beta[0], inf.beta[1]), dt=inf.dt,
                    res_norm=inf.res_norm, err=(inf.krylov_err[0], inf.krylov_err[1]),
                    reorth_cols=(int(inf.reorth_cols[0]), int(inf.reorth_cols[1])))


class Context:
    """Owns one pcexp_ctx; each method is one C call with its arguments marshalled."""

    def __init__(self, mesh, p: int, free, precision: int = PCEXP_FP64, m_max: int = 30,
                 eta: float = 0.0, basis_io: int = PCEXP_BASIS_PAPER, stream=None, krylov_tol: float = 0.0,
                 omega=None, reorth: int = 0):
        lib = load()
        m, self._keep = _mesh_struct(mesh)
        ph = _physics(free, omega)
        self.omega = omega
        op = pcexp_options(precision, m_max, eta, basis_io, krylov_tol, reorth)
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except ImportError:
                stream = 0
        self.ctx = C.c_void_p()
        check(lib.pcexp_create(C.byref(self.ctx), C.byref(m), p, C.byref(ph), C.byref(op), C.c_void_p(stream)),
              "pcexp_create")
        ne, nb, nv, K = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int64()
        check(lib.pcexp_sizes(self.ctx, C.byref(ne), C.byref(nb), C.byref(nv), C.byref(K)), "pcexp_sizes")
        self.E, self.nb, self.nv, self.K = ne.value, nb.value, nv.value, K.value
        self.lib = lib

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.pcexp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, U):
        p, dev = _ptr(U)
        check(self.lib.pcexp_set_state(self.ctx, p, dev), "pcexp_set_state")

    def get_state(self, out=None):
        out = np.empty(self.K) if out is None else out
        p, dev = _ptr(out)
        check(self.lib.pcexp_get_state(self.ctx, p, dev), "pcexp_get_state")
        return out

    def project_state(self, kind: int, params=()):
        prm = np.ascontiguousarray(params, np.float64)
        check(self.lib.pcexp_project_state(self.ctx, kind, prm.ctypes.data_as(_D) if prm.size else None,
                                           prm.size), "pcexp_project_state")

    def residual(self, U, out=None):
        out = (np.empty(self.K) if isinstance(U, np.ndarray) else U.new_empty(self.K)) if out is None else out
        pu, dev = _ptr(U)
        po, _ = _ptr(out)
        check(self.lib.pcexp_residual(self.ctx, pu, po, dev), "pcexp_residual")
        return out

    def jvp(self, U, v, out=None):
        out = (np.empty(self.K) if isinstance(U, np.ndarray) else U.new_empty(self.K)) if out is None else out
        pu, dev = _ptr(U)
        pv, _ = _ptr(v)
        po, _ = _ptr(out)
        check(self.lib.pcexp_jvp(self.ctx, pu, pv, po, dev), "pcexp_jvp")
        return out

    def vjp(self, U, w, out=None):
        out = (np.empty(self.K) if isinstance(U, np.ndarray) else U.new_empty(self.K)) if out is None else out
        pu, dev = _ptr(U)
        pw, _ = _ptr(w)
        po, _ = _ptr(out)
        check(self.lib.pcexp_vjp(self.ctx, pu, pw, po, dev), "pcexp_vjp")
        return out

    def jvp_state_adjoint(self, U, v, w, out=None):
        out = (np.empty(self.K) if isinstance(U, np.ndarray) else U.new_empty(self.K)) if out is None else out
        pu, dev = _ptr(U)
        pv, _ = _ptr(v)
        pw, _ = _ptr(w)
        po, _ = _ptr(out)
        check(self.lib.pcexp_jvp_state_adjoint(self.ctx, pu, pv, pw, po, dev), "pcexp_jvp_state_adjoint")
        return out

    def residual_noalloc(self, U, out):
        """R(U) in the internal basis on device tensors, with no device allocation (enqueue only)."""
        pu, dev = _ptr(U)
        po, dev2 = _ptr(out)
        assert dev and dev2, "pcexp_residual_noalloc takes device pointers"
        check(self.lib.pcexp_residual_noalloc(self.ctx, pu, po), "pcexp_residual_noalloc")
        return out

    def compute_dt(self, cfl: float, local: bool = False):
        out = np.empty(self.E if local else 1)
        check(self.lib.pcexp_compute_dt(self.ctx, cfl, int(local), out.ctypes.data_as(C.c_void_p), 0),
              "pcexp_compute_dt")
        return out if local else float(out[0])

    def arnoldi(self, U, b, m: int, want_V: bool = True):
        V = np.zeros((m + 1, self.K)) if want_V else None
        H = np.zeros((m + 1) * m)
        k, beta = C.c_int(), C.c_double()
        pu, dev = _ptr(U)
        pb, _ = _ptr(b)
        check(self.lib.pcexp_arnoldi(self.ctx, pu, pb, m, V.ctypes.data_as(C.c_void_p) if want_V else None,
                                     H.ctypes.data_as(_D), C.byref(k), C.byref(beta), dev), "pcexp_arnoldi")
        return V, H.reshape(m + 1, m), k.value, beta.value

    def phi(self, H, dt: float):
        H = np.ascontiguousarray(H, np.float64)
        k = H.shape[0]
        p1, p2 = np.zeros(k), np.zeros(k)
        check(self.lib.pcexp_phi(self.ctx, H.ctypes.data_as(_D), k, H.shape[1], dt, p1.ctypes.data_as(_D),
                                 p2.ctypes.data_as(_D)), "pcexp_phi")
        return p1, p2

    def phi_adjoint(self, H, dt: float, ybar):
        H = np.ascontiguousarray(H, np.float64)
        yb = np.ascontiguousarray(ybar, np.float64)
        k = H.shape[0]
        Hb = np.zeros_like(H)
        check(self.lib.pcexp_phi_adjoint(self.ctx, H.ctypes.data_as(_D), k, H.shape[1], dt, yb.ctypes.data_as(_D),
                                         Hb.ctypes.data_as(_D)), "pcexp_phi_adjoint")
        return Hb

    def step_backward(self, U, dt: float, m: int, ubar_next, out=None, with_theta: bool = False):
        """ubar_n = (du_{n+1}/du_n)^T ubar_next; with_theta also returns the adjoint of
        (Mach, alpha in degrees) of the step as a numpy array of 2."""
        out = (np.empty(self.K) if isinstance(U, np.ndarray) else U.new_empty(self.K)) if out is None else out
        pu, dev = _ptr(U)
        pg, _ = _ptr(ubar_next)
        po, _ = _ptr(out)
        th = np.zeros(2)
        check(self.lib.pcexp_step_backward(self.ctx, pu, dt, m, pg, po, th.ctypes.data_as(_D) if with_theta else None,
                                           dev), "pcexp_step_backward")
        return (out, th) if with_theta else out

    def project_state_adjoint(self, kind: int, params, ubar0):
        """(du_0/dtheta)^T ubar0 for theta = (Mach, alpha in degrees[, eps for the vortex])."""
        prm = np.ascontiguousarray(params, np.float64)
        pu, dev = _ptr(ubar0)
        th = np.zeros(3)
        check(self.lib.pcexp_project_state_adjoint(self.ctx, kind, prm.ctypes.data_as(_D) if prm.size else None,
                                                   prm.size, pu, th.ctypes.data_as(_D), dev),
              "pcexp_project_state_adjoint")
        return th if kind == PCEXP_PROJ_VORTEX else th[:2]

    def functional_param_grad(self, kind: int, U, params=None):
        """dJ/d(Mach, alpha in degrees, eps) of an output functional at a fixed state U."""
        prm = np.ascontiguousarray(params if params is not None else [], np.float64)
        pu, dev = _ptr(U)
        dj = np.zeros(3)
        check(self.lib.pcexp_functional_param_grad(self.ctx, kind, prm.ctypes.data_as(_D) if prm.size else None,
                                                   prm.size, pu, dj.ctypes.data_as(_D), dev),
              "pcexp_functional_param_grad")
        return dj

    def step(self, scheme: int, dt_mode: int, dt_or_cfl: float, m: int, info: bool = True):
        inf = pcexp_step_info()
        check(self.lib.pcexp_step(self.ctx, scheme, dt_mode, dt_or_cfl, m, C.byref(inf) if info else None),
              "pcexp_step")
        if not info:
            return None
        return dict(k=(inf.krylov_dim[0], inf.krylov_dim[1]), beta=(inf.beta[0], inf.beta[1]), dt=inf.dt,
                    res_norm=inf.res_norm, err=(inf.krylov_err[0], inf.krylov_err[1]),
                    reorth_cols=(int(inf.reorth_cols[0]), int(inf.reorth_cols[1])))

    def march_steady(self, scheme: int, cfl_max: float, decades: float, max_iter: int, m: int):
        inf = pcexp_steady_info()
        check(self.lib.pcexp_march_steady(self.ctx, scheme, cfl_max, decades, max_iter, m, C.byref(inf)),
              "pcexp_march_steady")
        return dict(iterations=inf.iterations, res_first=inf.res_first, res_last=inf.res_last,
                    converged=bool(inf.converged))

    def functional(self, kind: int, U, grad=None, params=None):
        """(value, gradient) of an output functional at U; gradient is None unless grad is given.
        params: the functional's parameters (PCEXP_FUNC_VORTEX_L2: eps, x_c, y_c, period, t)."""
        v = C.c_double()
        pu, dev = _ptr(U)
        pg = _ptr(grad)[0] if grad is not None else None
        if params is None:
            check(self.lib.pcexp_functional(self.ctx, kind, pu, C.byref(v), pg, dev), "pcexp_functional")
        else:
            prm = np.ascontiguousarray(params, np.float64)
            check(self.lib.pcexp_functional_params(self.ctx, kind, prm.ctypes.data_as(_D), len(prm), pu,
                                                   C.byref(v), pg, dev), "pcexp_functional_params")
        return v.value, grad

    def set_physics(self, free):
        ph = _physics(free, self.omega)
        check(self.lib.pcexp_set_physics(self.ctx, C.byref(ph)), "pcexp_set_physics")

    def output(self, kind: int = 0) -> float:
        v = C.c_double()
        check(self.lib.pcexp_output(self.ctx, kind, C.byref(v)), "pcexp_output")
        return v.value

    def synchronize(self):
        check(self.lib.pcexp_synchronize(self.ctx), "pcexp_synchronize")

    def profile_enable(self, on: bool = True):
        check(self.lib.pcexp_profile_enable(self.ctx, int(on)), "pcexp_profile_enable")

    def profile_read(self):
        """{class name: (launches, total ms)} since profiling was enabled."""
        out = {}
        for i, name in enumerate(KERNEL_CLASSES):
            n, ms = C.c_int64(), C.c_double()
            check(self.lib.pcexp_profile_read(self.ctx, i, C.byref(n), C.byref(ms)), "pcexp_profile_read")
            out[name] = (n.value, ms.value)
        return out
