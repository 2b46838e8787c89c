"""FP64 CPU oracle for the Urchin reverse ray tracer — TEST INFRASTRUCTURE.

Plain, slow restatement of what the paper (Altay & Theuns, arXiv:1304.4235)
defines, written in C (``urchin_oracle.c``) and wrapped here with ctypes.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline/reference
leg of ``bench.py`` may import this package.  It shares no code with the CUDA
library and the CUDA library never imports it.

Functions (FP64 throughout; each follows the passage named in the C source):
  sigma_th, sigma(E, which), spectrum(...)        App. C1, Eq. gamma
  m4_shape(q), gt_shape(q), chord(kernel, b,u1,u2) Eq. spline, Eq. Gt, I(h,b,z1,z2)
  columns(...), columns_points(...)               Eq. nhi, Eq. colden (brute force)
  Grid(w, cell).columns(...)                      the same sums from a uniform-grid candidate search
  healpix(nside)                                  Sec. 3.2 (Gorski et al. 2005)
  gamma(...)                                      Eq. gamma_shld
  rates(T), xeq(...)                              App. C3, Eqs. xroots / xphys
  solve(...)                                      Sec. 4 iteration driver (Jacobi)
  column_matrix(...)                              Eq. colden as tau = M x
  gamma_partials(...), xeq_dgamma(...)            derivatives of Eq. gamma_shld, Eq. xroots
  columns_vjp(...), solve_vjp(...)                reverse-mode derivatives (dense)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "urchin_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liburchin_oracle.so")
_lock = threading.Lock()
_lib = None

KERNEL_M4 = 0
KERNEL_GT = 1
XSEC_VERNER = 0
XSEC_HYDROGENIC = 1
XSEC_POWERLAW = 2
CASE_A, CASE_B, CASE_AUTO = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, strict IEEE: no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i, i64, vp = C.c_double, C.c_int, C.c_int64, C.c_void_p
            sig = {
                "oracle_sigma_th": (d, []),
                "oracle_E_th": (d, []),
                "oracle_sigma_hydrogenic": (d, [d, d]),
                "oracle_sigma_powerlaw": (d, [d]),
                "oracle_sigma_verner": (d, [d]),
                "oracle_sigma": (d, [i, d]),
                "oracle_spectrum": (None, [i, vp, vp, i, d, vp, vp]),
                "oracle_m4_shape": (d, [d]),
                "oracle_gt_shape": (d, [d]),
                "oracle_chord_m4": (d, [d, d, d]),
                "oracle_chord_gt": (d, [d, d, d]),
                "oracle_chord": (d, [i, d, d, d]),
                "oracle_columns_points": (None, [i64, vp, vp, vp, vp, vp, vp, i, d, d,
                                                 vp, i64, vp, i, d, i, vp]),
                "oracle_columns": (None, [i64, vp, vp, vp, vp, vp, vp, i, d, d,
                                          vp, i64, vp, i, d, i, vp]),
                "oracle_healpix": (None, [i, vp]),
                "oracle_gamma": (None, [vp, i64, i, i, vp, vp, vp, vp]),
                "oracle_rates": (None, [d, vp, vp, vp]),
                "oracle_xeq": (d, [d, d, d, d, i]),
                "oracle_solve": (i, [i64, vp, vp, vp, vp, vp, vp, vp, d, i, d, d,
                                     vp, i, d, i, i, vp, vp, d, d, i, i, i, i, vp, vp, vp, vp,
                                     vp, vp, vp, vp, vp, d]),
                "oracle_grid_build": (vp, [i64, vp, vp, vp, vp, i, d, d]),
                "oracle_grid_free": (None, [vp]),
                "oracle_grid_entries": (i64, [vp]),
                "oracle_grid_columns": (None, [vp, vp, vp, vp, vp, vp, vp, d, vp, i64, vp, i, d, i, vp]),
                "oracle_gamma_he": (None, [vp, vp, vp, i64, i, i, vp, vp, vp, vp, vp, vp]),
                "oracle_columns_nearfar": (None, [i64, vp, vp, vp, vp, vp, vp, i, d, d,
                                                  vp, i64, vp, i, d, i, vp, vp]),
                "oracle_slab_lngamma": (d, [d, d, d, i, d]),
                "oracle_gamma_nearfar": (None, [vp, vp, i64, i, i, vp, vp, vp, vp, vp, i, vp, vp]),
                "oracle_slab_poly_lngamma": (d, [i, vp, vp, d, d, d, i, d]),
                "oracle_ns_slab": (d, [i, vp, vp, d, d, i, d, i64, vp]),
                "oracle_ns_slab2": (d, [i, vp, vp, d, d, i, d, i64, d, i, vp]),
                "oracle_xeq_dgamma": (d, [d, d, d, d, i]),
                "oracle_column_matrix": (None, [i64, vp, vp, vp, vp, vp, i, d, d,
                                                vp, i64, vp, i, d, i, vp]),
                "oracle_num_threads": (i, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


# -- cross sections and spectrum (App. C1) ----------------------------------
def sigma_th() -> float:
    return _load().oracle_sigma_th()


def E_th() -> float:
    return _load().oracle_E_th()


def sigma(E_eV, which: int = XSEC_VERNER):
    lib = _load()
    return np.array([lib.oracle_sigma(which, float(e)) for e in np.atleast_1d(E_eV)])


def sigma_hydrogenic(E_eV, Z=1.0):
    lib = _load()
    return np.array([lib.oracle_sigma_hydrogenic(float(e), float(Z)) for e in np.atleast_1d(E_eV)])


def spectrum(edges, J, gamma_thin: float, xsec: int = XSEC_VERNER):
    """s_j = sigma_j / sigma_th and w_j (sum w = gamma_thin)."""
    edges, J = _f64(edges), _f64(J)
    F = J.shape[0]
    s = np.zeros(F)
    w = np.zeros(F)
    _load().oracle_spectrum(F, _p(edges), _p(J), xsec, gamma_thin, _p(s), _p(w))
    return s, w


# -- kernels (Eq. spline, Eq. Gt) --------------------------------------------
def m4_shape(q: float) -> float:
    return _load().oracle_m4_shape(float(q))


def gt_shape(q: float) -> float:
    return _load().oracle_gt_shape(float(q))


def chord(kernel: int, b: float, u1: float, u2: float) -> float:
    """int_{u1}^{u2} shape(sqrt(b^2+u^2)) du, lengths in units of h."""
    return _load().oracle_chord(kernel, float(b), float(u1), float(u2))


# -- columns (Eq. colden) ----------------------------------------------------
def _particles(w):
    pos = np.asarray(w.pos, dtype=np.float64)
    return (np.ascontiguousarray(pos[:, 0]), np.ascontiguousarray(pos[:, 1]),
            np.ascontiguousarray(pos[:, 2]), _f64(w.h), _f64(w.mass_H))


def columns(w, x, dirs, origins=None, l_ray=None, kernel=KERNEL_M4):
    """Threshold optical depth tau[o, k] = sigma_th N_HI of ray k from particle
    origins[o] (all particles when None).  ``w`` is a workloads.Workload."""
    px, py, pz, h, m = _particles(w)
    x = _f64(x)
    dirs = _f64(dirs).reshape(-1, 3)
    R = dirs.shape[0]
    org = None if origins is None else np.ascontiguousarray(origins, dtype=np.int64)
    n_orig = w.n if org is None else org.shape[0]
    out = np.zeros((n_orig, R))
    _load().oracle_columns(w.n, _p(px), _p(py), _p(pz), _p(h), _p(m), _p(x),
                           int(w.periodic), float(w.box), float(w.unit_cm),
                           _p(org), n_orig, _p(dirs), R,
                           float(w.l_ray if l_ray is None else l_ray), kernel, _p(out))
    return out


class Grid:
    """Uniform-grid candidate search over a workload's particles (positions
    and h only): every particle listed in each cell its sphere's bounding box
    overlaps, rays walking the cells their segments cross.  columns() then
    gives the brute-force sums of Eq. colden up to the order of the sum."""

    def __init__(self, w, cell: float):
        self.w = w
        px, py, pz, h, _ = _particles(w)
        self._keep = (px, py, pz, h)
        self._g = _load().oracle_grid_build(w.n, _p(px), _p(py), _p(pz), _p(h), int(w.periodic), float(w.box),
                                            float(cell))
        if not self._g:
            raise ValueError("grid query: a periodic sphere spans the box at this cell size")

    @property
    def entries(self) -> int:
        return int(_load().oracle_grid_entries(self._g))

    def columns(self, x, dirs, origins=None, l_ray=None, kernel=KERNEL_M4):
        w = self.w
        px, py, pz, h, m = _particles(w)
        x = _f64(x)
        dirs = _f64(dirs).reshape(-1, 3)
        org = None if origins is None else np.ascontiguousarray(origins, dtype=np.int64)
        n_orig = w.n if org is None else org.shape[0]
        out = np.zeros((n_orig, dirs.shape[0]))
        _load().oracle_grid_columns(self._g, _p(px), _p(py), _p(pz), _p(h), _p(m), _p(x), float(w.unit_cm),
                                    _p(org), n_orig, _p(dirs), dirs.shape[0],
                                    float(w.l_ray if l_ray is None else l_ray), kernel, _p(out))
        return out

    def close(self):
        if self._g:
            _load().oracle_grid_free(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def columns_points(w, x, points, dirs, l_ray, kernel=KERNEL_M4):
    px, py, pz, h, m = _particles(w)
    x = _f64(x)
    pts = _f64(points).reshape(-1, 3)
    dirs = _f64(dirs).reshape(-1, 3)
    out = np.zeros((pts.shape[0], dirs.shape[0]))
    _load().oracle_columns_points(w.n, _p(px), _p(py), _p(pz), _p(h), _p(m), _p(x),
                                  int(w.periodic), float(w.box), float(w.unit_cm),
                                  _p(pts), pts.shape[0], _p(dirs), dirs.shape[0],
                                  float(l_ray), kernel, _p(out))
    return out


# -- rays (Sec. 3.2) ---------------------------------------------------------
def healpix(nside: int) -> np.ndarray:
    out = np.zeros((12 * nside * nside, 3))
    _load().oracle_healpix(nside, _p(out))
    return out


# -- Gamma (Eq. gamma_shld) --------------------------------------------------
def gamma(tau, s, w):
    tau = _f64(tau)
    n_orig, R = tau.shape
    s, w = _f64(s), _f64(w)
    g = np.zeros(n_orig)
    te = np.zeros(n_orig)
    _load().oracle_gamma(_p(tau), n_orig, R, s.shape[0], _p(s), _p(w), _p(g), _p(te))
    return g, te


# -- rates and equilibrium (App. C3) -----------------------------------------
def rates(T: float):
    a = (C.c_double * 3)()
    lib = _load()
    aA, aB, gc = C.c_double(), C.c_double(), C.c_double()
    lib.oracle_rates(float(T), C.byref(aA), C.byref(aB), C.byref(gc))
    del a
    return aA.value, aB.value, gc.value


def xeq(Gamma, nH, T, y=0.0, caseB=False):
    lib = _load()
    G, nH, T, cb = np.broadcast_arrays(np.atleast_1d(np.asarray(Gamma, dtype=np.float64)),
                                       np.asarray(nH, dtype=np.float64),
                                       np.asarray(T, dtype=np.float64),
                                       np.asarray(caseB, dtype=bool))
    return np.array([lib.oracle_xeq(float(g), float(n), float(t), float(y), int(c))
                     for g, n, t, c in zip(G, nH, T, cb)])


# -- driver (Sec. 4) ---------------------------------------------------------
def solve(w, s, wts, dirs, tol=1e-3, tau_skip=1e-4, max_iter=100, case_rule=CASE_AUTO,
          kernel=KERNEL_M4, y=0.0, x_start=None, sweeps=None, l_ray=None, blocks=1, near_far=0, he=None,
          grid_cell=0.0):
    """Iteration of Sec. 4: Jacobi (blocks=1) or the high-to-low density
    update order in `blocks` blocks.  ``sweeps`` = exact sweep count
    (step-matched mode) instead of the tolerance test.  Returns (x, frozen,
    stats) with stats = dict(sweeps, max_rel_dx, rays, converged, caseB), caseB
    the case of each particle's last update.  he = dict(tau1, tau2 [n, R],
    s1, s2 [F]) adds fixed He I / He II columns (gamma_he).  grid_cell > 0
    takes the columns from the uniform-grid query (Grid) instead of brute
    force (not with near_far)."""
    px, py, pz, h, m = _particles(w)
    nH, T = _f64(w.nH), _f64(w.T)
    dirs = _f64(dirs).reshape(-1, 3)
    s, wts = _f64(s), _f64(wts)
    x = np.zeros(w.n)
    frozen = np.zeros(w.n, dtype=np.int32)
    caseB = np.zeros(w.n, dtype=np.int32)
    st = np.zeros(3)
    xs = None if x_start is None else _f64(x_start)
    mi = -int(sweeps) if sweeps is not None else int(max_iter)
    h1 = h2 = hs1 = hs2 = None
    if he is not None:
        h1, h2 = _f64(he["tau1"]).reshape(-1), _f64(he["tau2"]).reshape(-1)
        hs1, hs2 = _f64(he["s1"]), _f64(he["s2"])
    rc = _load().oracle_solve(w.n, _p(px), _p(py), _p(pz), _p(h), _p(m), _p(nH), _p(T),
                              float(y), int(w.periodic), float(w.box), float(w.unit_cm),
                              _p(dirs), dirs.shape[0],
                              float(w.l_ray if l_ray is None else l_ray), kernel,
                              s.shape[0], _p(s), _p(wts), float(tol), float(tau_skip),
                              mi, case_rule, int(blocks), int(near_far), _p(h1), _p(h2), _p(hs1), _p(hs2),
                              _p(xs), _p(x), _p(frozen), _p(caseB), _p(st), float(grid_cell))
    if rc == 2:
        raise ValueError("near_far needs blocks <= 1, helium needs near_far = 0 and blocks <= 1")
    if rc == 3:
        raise ValueError("grid query: a periodic sphere spans the box at this cell size")
    return x, frozen.astype(bool), dict(sweeps=int(st[0]), max_rel_dx=float(st[1]),
                                        rays=float(st[2]), converged=(rc == 0),
                                        caseB=caseB.astype(bool))


# -- near/far split and the slab solution (Sec. 3.3.3, App. slab) -----------
def columns_nearfar(w, x, dirs, origins=None, l_ray=None, kernel=KERNEL_M4):
    """(tau_far, tau_near) [n_orig, R]: far particles weighted by x, near
    particles (whose smoothing sphere holds the origin) with x = 1."""
    px, py, pz, h, m = _particles(w)
    x = _f64(x)
    dirs = _f64(dirs).reshape(-1, 3)
    R = dirs.shape[0]
    org = None if origins is None else np.ascontiguousarray(origins, dtype=np.int64)
    n_orig = w.n if org is None else org.shape[0]
    tf = np.zeros((n_orig, R))
    tn = np.zeros((n_orig, R))
    _load().oracle_columns_nearfar(w.n, _p(px), _p(py), _p(pz), _p(h), _p(m), _p(x),
                                   int(w.periodic), float(w.box), float(w.unit_cm),
                                   _p(org), n_orig, _p(dirs), R,
                                   float(w.l_ray if l_ray is None else l_ray), kernel, _p(tf), _p(tn))
    return tf, tn


def slab_lngamma(Gamma0, nH, T, caseB, tau_near):
    """ln Gamma at the bottom of the uniform slab (monochromatic, y = 0)."""
    lib = _load()
    G, nH, T, cb, tn = np.broadcast_arrays(np.atleast_1d(np.asarray(Gamma0, dtype=np.float64)),
                                           np.asarray(nH, dtype=np.float64), np.asarray(T, dtype=np.float64),
                                           np.asarray(caseB, dtype=bool), np.asarray(tau_near, dtype=np.float64))
    return np.array([lib.oracle_slab_lngamma(float(g), float(a), float(t), int(c), float(u))
                     for g, a, t, c, u in zip(G, nH, T, cb, tn)])


def slab_poly_lngamma(s, w, tau_far, nH, T, caseB, tau_near):
    """ln Gamma at the bottom of the slab for the binned spectrum (s, w)
    attenuated by tau_far (the numerical slab solution)."""
    s, w = _f64(s), _f64(w)
    lib = _load()
    tf, nH, T, cb, tn = np.broadcast_arrays(np.atleast_1d(np.asarray(tau_far, dtype=np.float64)),
                                            np.asarray(nH, dtype=np.float64), np.asarray(T, dtype=np.float64),
                                            np.asarray(caseB, dtype=bool), np.asarray(tau_near, dtype=np.float64))
    return np.array([lib.oracle_slab_poly_lngamma(s.shape[0], _p(s), _p(w), float(a), float(b), float(c), int(e),
                                                  float(f)) for a, b, c, e, f in zip(tf, nH, T, cb, tn)])


def ns_slab(s, w, nH, T, caseB, tau_total, n_slices):
    """Test 1's slab solver: (x per slice from the lit surface, N_HI sigma_th
    through the slab) for plane-parallel radiation with rates w_b."""
    s, w = _f64(s), _f64(w)
    x = np.zeros(int(n_slices))
    t = _load().oracle_ns_slab(s.shape[0], _p(s), _p(w), float(nH), float(T), int(bool(caseB)), float(tau_total),
                               int(n_slices), _p(x))
    return x, t


def ns_slab2(s, w, nH, T, caseB, tau_total, n_slices, tol=1e-8, max_pass=100000):
    """Test 3's slab solver (lit from both sides, half the rate each)."""
    s, w = _f64(s), _f64(w)
    x = np.zeros(int(n_slices))
    t = _load().oracle_ns_slab2(s.shape[0], _p(s), _p(w), float(nH), float(T), int(bool(caseB)), float(tau_total),
                                int(n_slices), float(tol), int(max_pass), _p(x))
    return x, t


def gamma_nearfar(tau_far, tau_near, s, w, nH, T, caseB, poly=False):
    """(ln(Gamma/Gamma_thin), Gamma) per origin with the slab solution
    (analytic at the threshold, or polychromatic when poly)."""
    tf, tn = _f64(tau_far), _f64(tau_near)
    n_orig, R = tf.shape
    s, w = _f64(s), _f64(w)
    nH = _f64(np.broadcast_to(nH, (n_orig,)))
    T = _f64(np.broadcast_to(T, (n_orig,)))
    cb = np.ascontiguousarray(np.broadcast_to(caseB, (n_orig,)), dtype=np.int32)
    lr = np.zeros(n_orig)
    g = np.zeros(n_orig)
    _load().oracle_gamma_nearfar(_p(tf), _p(tn), n_orig, R, s.shape[0], _p(s), _p(w), _p(nH), _p(T),
                                 _p(cb), int(bool(poly)), _p(lr), _p(g))
    return lr, g


# -- derivatives (reverse mode, dense) ----------------------------------------
def column_matrix(w, dirs, origins=None, l_ray=None, kernel=KERNEL_M4):
    """M[o, k, j] with tau[o, k] = sum_j M[o, k, j] x_j (Eq. colden is linear
    in x).  Dense: n_orig * R * n doubles."""
    px, py, pz, h, m = _particles(w)
    dirs = _f64(dirs).reshape(-1, 3)
    R = dirs.shape[0]
    org = None if origins is None else np.ascontiguousarray(origins, dtype=np.int64)
    n_orig = w.n if org is None else org.shape[0]
    M = np.zeros((n_orig, R, w.n))
    _load().oracle_column_matrix(w.n, _p(px), _p(py), _p(pz), _p(h), _p(m),
                                 int(w.periodic), float(w.box), float(w.unit_cm),
                                 _p(org), n_orig, _p(dirs), R,
                                 float(w.l_ray if l_ray is None else l_ray), kernel, _p(M))
    return M


def columns_vjp(w, dirs, tau_bar, origins=None, l_ray=None, kernel=KERNEL_M4, chunk=256):
    """x_bar[j] = sum_{o,k} tau_bar[o, k] dtau[o, k]/dx_j = (M^T tau_bar)_j."""
    tau_bar = _f64(tau_bar)
    org = np.arange(w.n) if origins is None else np.asarray(origins, dtype=np.int64)
    out = np.zeros(w.n)
    for a in range(0, org.shape[0], chunk):
        M = column_matrix(w, dirs, org[a:a + chunk], l_ray, kernel)
        out += np.einsum("okj,ok->j", M, tau_bar[a:a + chunk])
    return out


def gamma_partials(tau, s, w):
    """Partial derivatives of Eq. gamma_shld, Gamma_o = (1/R) sum_k sum_b
    w_b exp(-s_b tau_ok):  dGamma_o/dtau_ok = -(1/R) sum_b w_b s_b
    exp(-s_b tau_ok)  [n_orig, R]  and  dGamma_o/dw_b = (1/R) sum_k
    exp(-s_b tau_ok)  [n_orig, F]."""
    tau, s, w = _f64(tau), _f64(s), _f64(w)
    R = tau.shape[1]
    e = np.exp(-tau[:, :, None] * s[None, None, :])          # [n_orig, R, F]
    dG_dtau = -(e * (w * s)[None, None, :]).sum(axis=2) / R
    dG_dw = e.sum(axis=1) / R
    return dG_dtau, dG_dw


def xeq_dgamma(Gamma, nH, T, y=0.0, caseB=False):
    """d x_- / d Gamma of the equilibrium root (App. C3)."""
    lib = _load()
    G, nH, T, cb = np.broadcast_arrays(np.atleast_1d(np.asarray(Gamma, dtype=np.float64)),
                                       np.asarray(nH, dtype=np.float64),
                                       np.asarray(T, dtype=np.float64),
                                       np.asarray(caseB, dtype=bool))
    return np.array([lib.oracle_xeq_dgamma(float(g), float(n), float(t), float(y), int(c))
                     for g, n, t, c in zip(G, nH, T, cb)])


def solve_vjp(w, s, wts, dirs, x_star, frozen, caseB, x_bar, case_rule=CASE_AUTO, y=0.0,
              kernel=KERNEL_M4, l_ray=None, warm_start=False, chunk=256):
    """Gradient of a loss L(x*) with respect to the spectrum weights w_b by
    the implicit function theorem at the fixed point of Sec. 4.

    Non-frozen particles a satisfy x_a = E_a(Gamma_a(x, w)) with their case
    held (caseB); frozen particles f hold x_thin,f = E_f(Gamma_thin), with
    Gamma_thin = sum_b w_b (constants when warm_start).  With
    J[a, j] = dE_a/dGamma_a * sum_k dGamma_a/dtau_ak * M[a, k, j],
        mu = (I - J[:, act])^{-T} x_bar[act],   Gamma_bar_a = mu_a dE_a/dGamma_a,
        dL/dw_b = sum_a Gamma_bar_a dGamma_a/dw_b
                  + sum_f (x_bar_f + (J^T mu)_f) dE_f/dGamma(Gamma_thin).
    Everything is evaluated at the given x_star.  Returns (w_bar[F], mu[n_act])."""
    s, wts, x_star, x_bar = _f64(s), _f64(wts), _f64(x_star), _f64(x_bar)
    frozen = np.asarray(frozen, dtype=bool)
    caseB = np.asarray(caseB, dtype=bool)
    act = np.flatnonzero(~frozen)
    fro = np.flatnonzero(frozen)
    na = act.shape[0]
    J = np.zeros((na, w.n))
    dGdw = np.zeros((na, s.shape[0]))
    dEdG = np.zeros(na)
    for a in range(0, na, chunk):
        ids = act[a:a + chunk]
        M = column_matrix(w, dirs, ids, l_ray, kernel)
        tau = np.einsum("okj,j->ok", M, x_star)
        G, _ = gamma(tau, s, wts)
        dG_dtau, dG_dw = gamma_partials(tau, s, wts)
        e1 = xeq_dgamma(G, w.nH[ids], w.T[ids], y, caseB[ids])
        J[a:a + len(ids)] = e1[:, None] * np.einsum("ok,okj->oj", dG_dtau, M)
        dGdw[a:a + len(ids)] = dG_dw
        dEdG[a:a + len(ids)] = e1
    mu = np.linalg.solve((np.eye(na) - J[:, act]).T, x_bar[act])
    w_bar = (mu * dEdG) @ dGdw
    if fro.shape[0] and not warm_start:
        gthin = float(wts.sum())
        xbar_f = x_bar[fro] + J[:, fro].T @ mu
        cb = np.full(fro.shape[0], case_rule == CASE_B)
        w_bar = w_bar + float(xbar_f @ xeq_dgamma(gthin, w.nH[fro], w.T[fro], y, cb))
    return w_bar, mu


# -- helium columns (not in the paper: hydrogen only) --------------------------
def gamma_he(tau, tau1, tau2, s, s1, s2, w):
    """(Gamma, tau_eff) behind H I, He I and He II columns (threshold units)."""
    tau, tau1, tau2 = _f64(tau), _f64(tau1), _f64(tau2)
    n_orig, R = tau.shape
    s, s1, s2, w = _f64(s), _f64(s1), _f64(s2), _f64(w)
    g = np.zeros(n_orig)
    te = np.zeros(n_orig)
    _load().oracle_gamma_he(_p(tau), _p(tau1), _p(tau2), n_orig, R, s.shape[0], _p(s), _p(s1), _p(s2), _p(w),
                            _p(g), _p(te))
    return g, te


def num_threads() -> int:
    return _load().oracle_num_threads()
