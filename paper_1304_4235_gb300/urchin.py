"""Thin ctypes binding of liburchin (include/urchin.h).

Every function marshals arguments and calls the C ABI of the same name; all
computation happens in the library's CUDA kernels.  Device arrays are torch
CUDA tensors, host arrays numpy arrays.  A failing call raises UrchinError
with the library's status and message.  There is no CPU fallback: without the
compiled library (and a CUDA device for the compute calls) these functions
raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

URCHIN_OK = 0
URCHIN_ERR_ARG = -1
URCHIN_ERR_CUDA = -2
URCHIN_ERR_NOMEM = -3
URCHIN_ERR_NOT_CONVERGED = -4
URCHIN_ERR_NONFINITE = -5

KERNEL_M4, KERNEL_GT = 0, 1
F32, F64 = 0, 1
CASE_A, CASE_B, CASE_AUTO = 0, 1, 2
XSEC_VERNER, XSEC_HYDROGENIC, XSEC_POWERLAW, XSEC_HEII = 0, 1, 2, 3
METHOD_PLAIN, METHOD_NEWTON = 0, 1
SLAB_THRESHOLD, SLAB_SPECTRUM = 1, 2
SEG_RECOMPUTE, SEG_STORE, SEG_AUTO = 0, 1, 2
MAX_RAYS = 192
MAX_BINS = 4096

_vp = C.c_void_p


class urchin_particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos_x", _vp), ("pos_y", _vp), ("pos_z", _vp),
                ("h", _vp), ("mass_H", _vp)]


class urchin_box(C.Structure):
    _fields_ = [("periodic", C.c_int), ("L", C.c_double), ("unit_cm", C.c_double)]


class urchin_spectrum(C.Structure):
    _fields_ = [("F", C.c_int), ("s", _vp), ("w", _vp), ("s_he1", _vp), ("s_he2", _vp)]


class urchin_solve_params(C.Structure):
    _fields_ = [("R", C.c_int), ("dirs", _vp), ("l_ray", C.c_double),
                ("spectrum", urchin_spectrum), ("nH", _vp), ("T", _vp), ("y", C.c_double),
                ("tol", C.c_double), ("tau_skip", C.c_double), ("max_iter", C.c_int),
                ("method", C.c_int), ("segments", C.c_int), ("gmres_m", C.c_int),
                ("kernel", C.c_int), ("precision", C.c_int), ("case_rule", C.c_int),
                ("warm_start", C.c_int), ("profile", C.c_int), ("history_maxrel", _vp),
                ("history_unconverged", _vp), ("blocks", C.c_int), ("newton_switch", C.c_double),
                ("newton_eta", C.c_double), ("state", _vp), ("he1", _vp), ("he2", _vp), ("near_far", C.c_int)]


class urchin_solve_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("traversals", C.c_int), ("rays", C.c_int64),
                ("particle_updates", C.c_int64), ("n_active", C.c_int64), ("nnz", C.c_int64),
                ("max_rel_dx", C.c_double), ("wall_s", C.c_double), ("converged", C.c_int),
                ("segments_stored", C.c_int), ("hits", C.c_int64), ("trace_s", C.c_double),
                ("trace_launches", C.c_int), ("sphere_tests", C.c_int64), ("node_visits", C.c_int64),
                ("newton_fallbacks", C.c_int), ("newton_start", C.c_int), ("spmv_s", C.c_double),
                ("spmv_launches", C.c_int), ("spmv_bytes", C.c_int64), ("sweep_s", C.c_double),
                ("sweep_launches", C.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class UrchinError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"urchin status {status}: {message}")
        self.status = status


# exported entry points: name -> (restype, argtypes)
SIGNATURES = {
    "urchin_last_error": (C.c_char_p, []),
    "urchin_version": (C.c_char_p, []),
    "urchin_kernel_launches": (C.c_int64, []),
    "urchin_trim_memory": (C.c_int, [C.c_int, C.POINTER(C.c_uint64)]),
    "urchin_healpix_dirs": (C.c_int, [C.c_int, _vp]),
    "urchin_spectrum_weights": (C.c_int, [C.c_int, _vp, _vp, C.c_int, C.c_double, _vp, _vp]),
    "urchin_build_bvh": (C.c_int, [C.POINTER(urchin_particles), C.POINTER(urchin_box),
                                   C.POINTER(_vp), _vp]),
    "urchin_free_bvh": (None, [_vp]),
    "urchin_bvh_size": (C.c_int64, [_vp]),
    "urchin_trace_columns": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_double, _vp, C.c_int64,
                                       C.c_int, C.c_int, _vp, _vp]),
    "urchin_trace_columns_noalloc": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_double, _vp, C.c_int64,
                                               C.c_int, C.c_int, _vp, _vp]),
    "urchin_gamma": (C.c_int, [_vp, C.c_int, C.c_int64, C.c_int, C.POINTER(urchin_spectrum),
                               _vp, _vp, _vp]),
    "urchin_equilibrium": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int64, C.c_int, C.c_double,
                                     _vp, _vp]),
    "urchin_solve": (C.c_int, [_vp, C.POINTER(urchin_solve_params), _vp,
                               C.POINTER(urchin_solve_stats), _vp]),
    "urchin_tangent": (C.c_int, [_vp, C.POINTER(urchin_solve_params), _vp, _vp, _vp, _vp, _vp]),
    "urchin_trace_columns_vjp": (C.c_int, [_vp, _vp, C.c_int, C.c_double, _vp, C.c_int64, C.c_int, C.c_int,
                                           _vp, _vp, _vp]),
    "urchin_gamma_vjp": (C.c_int, [_vp, C.c_int, C.c_int64, C.c_int, C.POINTER(urchin_spectrum), _vp, _vp, _vp,
                                   _vp]),
    "urchin_equilibrium_vjp": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int64, C.c_int, C.c_double, _vp, _vp, _vp]),
    "urchin_solve_vjp": (C.c_int, [_vp, C.POINTER(urchin_solve_params), _vp, _vp, _vp,
                                   C.POINTER(urchin_solve_stats), _vp]),
    "urchin_gamma_he": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int64, C.c_int, C.POINTER(urchin_spectrum),
                                  _vp, _vp, _vp]),
    "urchin_cross_section_ratio": (C.c_int, [C.c_int, _vp, C.c_int, _vp]),
    "urchin_trace_columns_nearfar": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_double, _vp, C.c_int64,
                                               C.c_int, C.c_int, _vp, _vp, _vp]),
    "urchin_gamma_nearfar": (C.c_int, [_vp, _vp, C.c_int, C.c_int64, C.c_int, C.POINTER(urchin_spectrum),
                                       _vp, _vp, _vp, C.c_int, _vp, _vp, _vp]),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liburchin.so (compiling it with nvcc first if it is missing or
    stale).  Raises when the library cannot be built or loaded."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"liburchin.so not found at {path}")
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(status: int):
    if status != URCHIN_OK:
        msg = load().urchin_last_error().decode(errors="replace")
        raise UrchinError(status, msg)


def _dev(t, dtype=None):
    """Pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return _vp(t.data_ptr())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return _vp(s.cuda_stream)


def _host(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------------------
def urchin_version() -> str:
    return load().urchin_version().decode()


def urchin_kernel_launches() -> int:
    return int(load().urchin_kernel_launches())


def urchin_trim_memory(device: int = -1) -> int:
    """Return the library pool's unused device memory (all devices for -1);
    the bytes still reserved afterwards."""
    left = C.c_uint64(0)
    _check(load().urchin_trim_memory(int(device), C.byref(left)))
    return int(left.value)


def urchin_healpix_dirs(nside: int) -> np.ndarray:
    out = np.zeros((12 * nside * nside, 3))
    _check(load().urchin_healpix_dirs(int(nside), out.ctypes.data_as(_vp)))
    return out


def urchin_spectrum_weights(edges, J, gamma_thin: float, xsec: int = XSEC_VERNER):
    edges, J = _host(edges), _host(J)
    F = J.shape[0]
    if edges.shape[0] != F + 1:
        raise ValueError("edges must have F+1 entries")
    s = np.zeros(F)
    w = np.zeros(F)
    _check(load().urchin_spectrum_weights(F, edges.ctypes.data_as(_vp), J.ctypes.data_as(_vp),
                                          int(xsec), float(gamma_thin), s.ctypes.data_as(_vp),
                                          w.ctypes.data_as(_vp)))
    return s, w


def urchin_cross_section_ratio(edges, xsec: int) -> np.ndarray:
    """sigma(E_j) / sigma_th at the geometric bin centres (XSEC_HEII: He II)."""
    edges = _host(edges)
    F = edges.shape[0] - 1
    out = np.zeros(F)
    _check(load().urchin_cross_section_ratio(F, edges.ctypes.data_as(_vp), int(xsec), out.ctypes.data_as(_vp)))
    return out


class Bvh:
    """Owner of a urchin_bvh* (freed on close / garbage collection)."""

    def __init__(self, handle, n, keep):
        self._h = handle
        self.n = n
        self._keep = keep

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("BVH already freed")
        return self._h

    def close(self):
        if self._h is not None:
            load().urchin_free_bvh(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def urchin_build_bvh(pos_x, pos_y, pos_z, h, mass_H, periodic: bool, L: float, unit_cm: float,
                     stream=None) -> Bvh:
    """Device float32 positions and h, float64 mass_H (m/m_p)."""
    import torch
    n = int(pos_x.numel())
    p = urchin_particles(n, _dev(pos_x, torch.float32), _dev(pos_y, torch.float32),
                         _dev(pos_z, torch.float32), _dev(h, torch.float32),
                         _dev(mass_H, torch.float64))
    box = urchin_box(int(bool(periodic)), float(L), float(unit_cm))
    out = _vp()
    _check(load().urchin_build_bvh(C.byref(p), C.byref(box), C.byref(out), _stream(stream)))
    return Bvh(out, n, None)


def _trace_buffers(bvh: Bvh, x, origins, R: int, precision: int, outs):
    """Checks shared by the column entry points, made before any call into
    the library (the C side cannot check a raw pointer's size or device):
    x holds bvh.n values, origins is int32, every output is a contiguous
    [n_orig, R] tensor of the precision's dtype, and all of them sit on the
    current CUDA device (the one whose work arrays the call uses).  Returns
    (n_orig, dtype, outputs) with missing outputs allocated."""
    import torch
    if x.numel() != bvh.n:
        raise ValueError(f"x has {x.numel()} values, the BVH has {bvh.n} particles")
    if origins is not None and origins.dtype != torch.int32:
        raise TypeError(f"origins must be int32, got {origins.dtype}")
    n_orig = bvh.n if origins is None else int(origins.numel())
    dt = torch.float64 if precision == F64 else torch.float32
    res = []
    for o in outs:
        if o is not None:
            if tuple(o.shape) != (n_orig, R):
                raise ValueError(f"out has shape {tuple(o.shape)}, expected {(n_orig, R)}")
            if o.dtype != dt:
                raise TypeError(f"out has dtype {o.dtype}, expected {dt} for this precision")
            if not o.is_contiguous():
                raise ValueError("out must be contiguous")
        res.append(o)
    dev = torch.cuda.current_device()
    for t in [x, origins] + res:
        if t is not None and (not t.is_cuda or t.device.index != dev):
            raise ValueError(f"every array must be on the current CUDA device cuda:{dev}, got {t.device}")
    res = [torch.empty((n_orig, R), dtype=dt, device=x.device) if o is None else o for o in res]
    return n_orig, dt, res


def urchin_trace_columns(bvh: Bvh, x, dirs, l_ray: float, origins=None, kernel: int = KERNEL_M4,
                         precision: int = F32, out=None, stream=None):
    """Threshold optical depths tau[o, k] (float32 or float64 CUDA tensor)."""
    import torch
    dirs = _host(dirs).reshape(-1, 3)
    R = dirs.shape[0]
    n_orig, dt, (out,) = _trace_buffers(bvh, x, origins, R, precision, [out])
    _check(load().urchin_trace_columns(bvh.handle, _dev(x, torch.float64), dirs.ctypes.data_as(_vp), R,
                                       float(l_ray), _dev(origins, torch.int32), n_orig, int(kernel),
                                       int(precision), _dev(out, dt), _stream(stream)))
    return out


def urchin_trace_columns_noalloc(bvh: Bvh, x, dirs, l_ray: float, origins=None, kernel: int = KERNEL_M4,
                                 precision: int = F32, out=None, stream=None):
    """Same columns as urchin_trace_columns, but the library allocates no
    device memory: its work space is a fixed device array (see
    include/urchin.h for the size limit and the sharing rules).  Pass a
    preallocated `out` to keep the whole call free of allocation (with
    out=None this wrapper allocates it through torch)."""
    import torch
    dirs = _host(dirs).reshape(-1, 3)
    R = dirs.shape[0]
    n_orig, dt, (out,) = _trace_buffers(bvh, x, origins, R, precision, [out])
    _check(load().urchin_trace_columns_noalloc(bvh.handle, _dev(x, torch.float64), dirs.ctypes.data_as(_vp), R,
                                               float(l_ray), _dev(origins, torch.int32), n_orig, int(kernel),
                                               int(precision), _dev(out, dt), _stream(stream)))
    return out


def urchin_trace_columns_nearfar(bvh: Bvh, x, dirs, l_ray: float, origins=None, kernel: int = KERNEL_M4,
                                 precision: int = F32, stream=None):
    """(tau_far, tau_near) [n_orig, R] with the near/far split of Sec. 3.3.3."""
    import torch
    dirs = _host(dirs).reshape(-1, 3)
    R = dirs.shape[0]
    n_orig, dt, (tf, tn) = _trace_buffers(bvh, x, origins, R, precision, [None, None])
    _check(load().urchin_trace_columns_nearfar(bvh.handle, _dev(x, torch.float64), dirs.ctypes.data_as(_vp), R,
                                               float(l_ray), _dev(origins, torch.int32), n_orig, int(kernel),
                                               int(precision), _dev(tf, dt), _dev(tn, dt), _stream(stream)))
    return tf, tn


def urchin_gamma_nearfar(tau_far, tau_near, s, w, nH, T, caseB=None, slab: int = SLAB_THRESHOLD, stream=None):
    """(Gamma float64, tau_eff float32) per origin with the slab solution for
    the near particles; caseB: uint8 CUDA tensor or None (case A); slab:
    SLAB_THRESHOLD (analytic) or SLAB_SPECTRUM (numerical, binned spectrum)."""
    import torch
    precision = F64 if tau_far.dtype == torch.float64 else F32
    n_orig, R = tau_far.shape
    sp = urchin_spectrum(int(s.numel()), _dev(s, torch.float64), _dev(w, torch.float64))
    g = torch.empty(n_orig, dtype=torch.float64, device=tau_far.device)
    te = torch.empty(n_orig, dtype=torch.float32, device=tau_far.device)
    _check(load().urchin_gamma_nearfar(_dev(tau_far), _dev(tau_near, tau_far.dtype), int(precision), n_orig, R,
                                       C.byref(sp), _dev(nH, torch.float64), _dev(T, torch.float64),
                                       _dev(caseB, torch.uint8), int(slab), _dev(g), _dev(te), _stream(stream)))
    return g, te


def urchin_gamma_he(tau, tau_he1, tau_he2, s, w, s_he1, s_he2, stream=None):
    """(Gamma float64, tau_eff float32) behind H I, He I and He II columns."""
    import torch
    precision = F64 if tau.dtype == torch.float64 else F32
    n_orig, R = tau.shape
    sp = urchin_spectrum(int(s.numel()), _dev(s, torch.float64), _dev(w, torch.float64),
                         _dev(s_he1, torch.float64), _dev(s_he2, torch.float64))
    g = torch.empty(n_orig, dtype=torch.float64, device=tau.device)
    te = torch.empty(n_orig, dtype=torch.float32, device=tau.device)
    _check(load().urchin_gamma_he(_dev(tau), _dev(tau_he1, tau.dtype), _dev(tau_he2, tau.dtype), int(precision),
                                  n_orig, R, C.byref(sp), _dev(g), _dev(te), _stream(stream)))
    return g, te


def urchin_gamma(tau, s, w, precision: int = None, stream=None):
    """Gamma (float64) and tau_eff (float32) per row of tau [n_orig, R]."""
    import torch
    if precision is None:
        precision = F64 if tau.dtype == torch.float64 else F32
    n_orig, R = tau.shape
    sp = urchin_spectrum(int(s.numel()), _dev(s, torch.float64), _dev(w, torch.float64))
    g = torch.empty(n_orig, dtype=torch.float64, device=tau.device)
    te = torch.empty(n_orig, dtype=torch.float32, device=tau.device)
    _check(load().urchin_gamma(_dev(tau), int(precision), n_orig, R, C.byref(sp), _dev(g), _dev(te),
                               _stream(stream)))
    return g, te


def urchin_equilibrium(gamma, tau_eff, nH, T, case_rule: int = CASE_AUTO, y: float = 0.0, stream=None):
    import torch
    n = int(gamma.numel())
    x = torch.empty(n, dtype=torch.float64, device=gamma.device)
    _check(load().urchin_equilibrium(_dev(gamma, torch.float64), _dev(tau_eff, torch.float32),
                                     _dev(nH, torch.float64), _dev(T, torch.float64), n,
                                     int(case_rule), float(y), _dev(x), _stream(stream)))
    return x


def urchin_solve(bvh: Bvh, dirs, l_ray: float, s, w, nH, T, x=None, *, y: float = 0.0,
                 tol: float = 1e-3, tau_skip: float = 1e-4, max_iter: int = 100,
                 method: int = METHOD_PLAIN, segments: int = SEG_RECOMPUTE, gmres_m: int = 10,
                 kernel: int = KERNEL_M4, precision: int = F32, case_rule: int = CASE_AUTO,
                 warm_start: bool = False, profile: bool = False, raise_not_converged: bool = True,
                 history: bool = False, blocks: int = 1, newton_switch: float = 0.01, newton_eta: float = 0.0,
                 state=None, near_far: int = 0, s_he1=None, s_he2=None, he1=None, he2=None, stream=None):
    """Returns (x, stats dict).  x (float64 CUDA tensor, original order) is
    updated in place when given.  `state` (uint8 CUDA tensor [n]) receives
    each particle's final case / frozen flags for urchin_solve_vjp.  Helium:
    s_he1 / s_he2 (bin cross sections / sigma_th) with he1 / he2 (He I / He II
    atoms per H atom of each particle)."""
    import torch
    dirs = _host(dirs).reshape(-1, 3)
    if x is None:
        x = torch.zeros(bvh.n, dtype=torch.float64, device=nH.device)
    P = urchin_solve_params()
    P.R = dirs.shape[0]
    P.dirs = dirs.ctypes.data_as(_vp)
    P.l_ray = float(l_ray)
    P.spectrum = urchin_spectrum(int(s.numel()), _dev(s, torch.float64), _dev(w, torch.float64),
                                 _dev(s_he1, torch.float64), _dev(s_he2, torch.float64))
    P.he1 = _dev(he1, torch.float64)
    P.he2 = _dev(he2, torch.float64)
    P.nH = _dev(nH, torch.float64)
    P.T = _dev(T, torch.float64)
    P.y = float(y)
    P.tol = float(tol)
    P.tau_skip = float(tau_skip)
    P.max_iter = int(max_iter)
    P.method = int(method)
    P.segments = int(segments)
    P.gmres_m = int(gmres_m)
    P.kernel = int(kernel)
    P.precision = int(precision)
    P.case_rule = int(case_rule)
    P.warm_start = int(bool(warm_start))
    P.profile = int(bool(profile))
    P.blocks = int(blocks)
    P.newton_switch = float(newton_switch)
    P.newton_eta = float(newton_eta)
    P.state = _dev(state, torch.uint8)
    P.near_far = int(near_far)
    hist_max = hist_unc = None
    if history:
        hist_max = np.zeros(int(max_iter))
        hist_unc = np.zeros(int(max_iter), dtype=np.int64)
        P.history_maxrel = hist_max.ctypes.data_as(_vp)
        P.history_unconverged = hist_unc.ctypes.data_as(_vp)
    st = urchin_solve_stats()
    rc = load().urchin_solve(bvh.handle, C.byref(P), _dev(x, torch.float64), C.byref(st), _stream(stream))
    out = st.as_dict()
    if history:
        k = out["iterations"]
        out["history_maxrel"] = hist_max[:k].tolist()
        out["history_unconverged"] = hist_unc[:k].tolist()
    if rc == URCHIN_ERR_NOT_CONVERGED and not raise_not_converged:
        return x, out
    _check(rc)
    return x, out


def urchin_tangent(bvh: Bvh, dirs, l_ray: float, s, w, nH, T, x, v, *, y: float = 0.0,
                   kernel: int = KERNEL_M4, precision: int = F32, case_rule: int = CASE_AUTO, stream=None):
    """(E(x), d ln E / d ln x . v) of one sweep over all particles (float64
    CUDA tensors, original order)."""
    import torch
    dirs = _host(dirs).reshape(-1, 3)
    P = urchin_solve_params()
    P.R = dirs.shape[0]
    P.dirs = dirs.ctypes.data_as(_vp)
    P.l_ray = float(l_ray)
    P.spectrum = urchin_spectrum(int(s.numel()), _dev(s, torch.float64), _dev(w, torch.float64))
    P.nH = _dev(nH, torch.float64)
    P.T = _dev(T, torch.float64)
    P.y = float(y)
    P.tol = 1e-3
    P.max_iter = 1
    P.kernel = int(kernel)
    P.precision = int(precision)
    P.case_rule = int(case_rule)
    E = torch.empty(bvh.n, dtype=torch.float64, device=x.device)
    dl = torch.empty(bvh.n, dtype=torch.float64, device=x.device)
    _check(load().urchin_tangent(bvh.handle, C.byref(P), _dev(x, torch.float64), _dev(v, torch.float64),
                                 _dev(E), _dev(dl), _stream(stream)))
    return E, dl



# ---------------------------------------------------------------------------
# reverse mode
def urchin_trace_columns_vjp(bvh: Bvh, dirs, l_ray: float, tau_bar, origins=None, kernel: int = KERNEL_M4,
                             precision: int = None, x_bar=None, stream=None):
    """x_bar[j] (+)= sum_{o,k} tau_bar[o, k] d tau[o, k] / d x_j (float64 CUDA
    tensor [n], original order; accumulated into x_bar when given)."""
    import torch
    dirs = _host(dirs).reshape(-1, 3)
    R = dirs.shape[0]
    if precision is None:
        precision = F64 if tau_bar.dtype == torch.float64 else F32
    dt = torch.float64 if precision == F64 else torch.float32
    n_orig = bvh.n if origins is None else int(origins.numel())
    if tuple(tau_bar.shape) != (n_orig, R):
        raise ValueError(f"tau_bar must have shape ({n_orig}, {R})")
    if x_bar is None:
        x_bar = torch.zeros(bvh.n, dtype=torch.float64, device=tau_bar.device)
    elif x_bar.numel() != bvh.n:
        raise ValueError(f"x_bar has {x_bar.numel()} values, the BVH has {bvh.n} particles")
    _check(load().urchin_trace_columns_vjp(bvh.handle, dirs.ctypes.data_as(_vp), R, float(l_ray),
                                           _dev(origins, torch.int32), n_orig, int(kernel), int(precision),
                                           _dev(tau_bar, dt), _dev(x_bar, torch.float64), _stream(stream)))
    return x_bar


def urchin_gamma_vjp(tau, s, w, gamma_bar, want_tau: bool = True, want_w: bool = True, precision: int = None,
                     stream=None):
    """(tau_bar [n_orig, R] in tau's dtype or None, w_bar [F] float64 or None)."""
    import torch
    if precision is None:
        precision = F64 if tau.dtype == torch.float64 else F32
    n_orig, R = tau.shape
    sp = urchin_spectrum(int(s.numel()), _dev(s, torch.float64), _dev(w, torch.float64))
    tb = torch.empty_like(tau) if want_tau else None
    wb = torch.zeros(int(s.numel()), dtype=torch.float64, device=tau.device) if want_w else None
    _check(load().urchin_gamma_vjp(_dev(tau), int(precision), n_orig, R, C.byref(sp),
                                   _dev(gamma_bar, torch.float64), _dev(tb), _dev(wb), _stream(stream)))
    return tb, wb


def urchin_equilibrium_vjp(gamma, tau_eff, nH, T, x_bar, case_rule: int = CASE_AUTO, y: float = 0.0,
                           stream=None):
    import torch
    n = int(gamma.numel())
    gb = torch.empty(n, dtype=torch.float64, device=gamma.device)
    _check(load().urchin_equilibrium_vjp(_dev(gamma, torch.float64), _dev(tau_eff, torch.float32),
                                         _dev(nH, torch.float64), _dev(T, torch.float64), n, int(case_rule),
                                         float(y), _dev(x_bar, torch.float64), _dev(gb), _stream(stream)))
    return gb


def urchin_solve_vjp(bvh: Bvh, dirs, l_ray: float, s, w, nH, T, x_star, state, x_bar, *, y: float = 0.0,
                     tau_skip: float = 1e-4, tol: float = 1e-10, max_iter: int = 2000, gmres_m: int = 30,
                     segments: int = SEG_RECOMPUTE, kernel: int = KERNEL_M4, precision: int = F32,
                     case_rule: int = CASE_AUTO, warm_start: bool = False, raise_not_converged: bool = True,
                     profile: bool = False, stream=None):
    """dL/dw (float64 CUDA tensor [F]) at the converged x* of urchin_solve
    (whose `state` output must be passed), for x_bar = dL/dx*.  tol and
    max_iter bound the adjoint GMRES solve; profile times the column passes
    (trace_s, spmv_s).  Returns (w_bar, stats dict)."""
    import torch
    dirs = _host(dirs).reshape(-1, 3)
    P = urchin_solve_params()
    P.R = dirs.shape[0]
    P.dirs = dirs.ctypes.data_as(_vp)
    P.l_ray = float(l_ray)
    P.spectrum = urchin_spectrum(int(s.numel()), _dev(s, torch.float64), _dev(w, torch.float64))
    P.nH = _dev(nH, torch.float64)
    P.T = _dev(T, torch.float64)
    P.y = float(y)
    P.tol = float(tol)
    P.tau_skip = float(tau_skip)
    P.max_iter = int(max_iter)
    P.segments = int(segments)
    P.gmres_m = int(gmres_m)
    P.kernel = int(kernel)
    P.precision = int(precision)
    P.case_rule = int(case_rule)
    P.warm_start = int(bool(warm_start))
    P.profile = int(bool(profile))
    P.state = _dev(state, torch.uint8)
    wb = torch.zeros(int(s.numel()), dtype=torch.float64, device=x_star.device)
    st = urchin_solve_stats()
    rc = load().urchin_solve_vjp(bvh.handle, C.byref(P), _dev(x_star, torch.float64), _dev(x_bar, torch.float64),
                                 _dev(wb), C.byref(st), _stream(stream))
    if not (rc == URCHIN_ERR_NOT_CONVERGED and not raise_not_converged):
        _check(rc)
    return wb, st.as_dict()
