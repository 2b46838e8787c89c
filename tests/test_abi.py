"""The C-ABI library: builds, loads, exports every declared entry point, and
rejects bad arguments before touching a GPU.  CPU only (no compute calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_1304_4235_gb300 import urchin as U

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"URCHIN_API[^;(]*?\b(urchin_\w+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = U.load()
    names = declared_symbols()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    # the binding wraps each one
    assert set(names) == set(U.SIGNATURES)


def test_only_abi_symbols_exported():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", U.library_path()], capture_output=True,
                         text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported == set(declared_symbols())


def test_library_resolves_every_symbol_at_load():
    """Loaded with immediate binding, so that a function the library calls
    but does not define (one left with internal linkage in another
    translation unit, say) fails here rather than at its first call."""
    C.CDLL(U.library_path(), mode=os.RTLD_NOW | os.RTLD_LOCAL)
    import subprocess
    out = subprocess.run(["nm", "-D", "--undefined-only", U.library_path()], capture_output=True,
                         text=True).stdout
    assert not [l for l in out.splitlines() if "urchin" in l], out


def test_version():
    assert "sm_103a" in U.urchin_version()


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_healpix_matches_oracle(nside):
    assert np.allclose(U.urchin_healpix_dirs(nside), O.healpix(nside), atol=1e-14, rtol=0)


@pytest.mark.parametrize("xsec", [U.XSEC_VERNER, U.XSEC_HYDROGENIC, U.XSEC_POWERLAW])
@pytest.mark.parametrize("F", [1, 50, 100, 400])
def test_spectrum_weights_match_oracle(xsec, F):
    e, J = W.powerlaw_spectrum(F, 13.6, 54.4)
    s1, w1 = U.urchin_spectrum_weights(e, J, 1e-12, xsec)
    s2, w2 = O.spectrum(e, J, 1e-12, xsec)
    assert np.allclose(s1, s2, rtol=1e-13, atol=0)
    assert np.allclose(w1, w2, rtol=1e-13, atol=0)


def _err(fn, *args):
    rc = fn(*args)
    return rc, U.load().urchin_last_error().decode()


def test_heii_cross_section_is_hydrogenic_with_charge_two():
    """URCHIN_XSEC_HEII: the exact hydrogenic form with Z = 2 (threshold
    54.4 eV), against the oracle's hydrogenic cross section."""
    edges = np.exp(np.linspace(np.log(13.6), np.log(136.0), 201))
    got = U.urchin_cross_section_ratio(edges, U.XSEC_HEII)
    Ec = np.sqrt(edges[:-1] * edges[1:])
    ref = np.array([O.sigma_hydrogenic(E, 2.0) for E in Ec]).ravel() / O.sigma_th()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
    assert got[Ec < 54.4].max() == 0.0 and got[Ec > 55].min() > 0.0
    hi = U.urchin_cross_section_ratio(edges, U.XSEC_HYDROGENIC)
    ref1 = np.array([O.sigma_hydrogenic(E, 1.0) for E in Ec]).ravel() / O.sigma_th()
    np.testing.assert_allclose(hi, ref1, rtol=1e-12, atol=0)


def test_host_argument_errors():
    lib = U.load()
    rc, msg = _err(lib.urchin_healpix_dirs, 0, None)
    assert rc == U.URCHIN_ERR_ARG and "nside" in msg
    rc, _ = _err(lib.urchin_healpix_dirs, 5, (C.c_double * 900)())     # 300 rays > max
    assert rc == U.URCHIN_ERR_ARG
    rc, _ = _err(lib.urchin_healpix_dirs, 1, None)
    assert rc == U.URCHIN_ERR_ARG
    e = np.array([13.6, 20.0, 15.0])                                    # not increasing
    J = np.ones(2)
    s = np.zeros(2)
    rc, _ = _err(lib.urchin_spectrum_weights, 2, e.ctypes.data_as(C.c_void_p), J.ctypes.data_as(C.c_void_p),
                 0, 1e-12, s.ctypes.data_as(C.c_void_p), s.ctypes.data_as(C.c_void_p))
    assert rc == U.URCHIN_ERR_ARG
    e = np.array([10.0, 20.0])                                          # below threshold
    rc, _ = _err(lib.urchin_spectrum_weights, 1, e.ctypes.data_as(C.c_void_p), J.ctypes.data_as(C.c_void_p),
                 0, 1e-12, s.ctypes.data_as(C.c_void_p), s.ctypes.data_as(C.c_void_p))
    assert rc == U.URCHIN_ERR_ARG


def test_device_entry_points_reject_bad_arguments_without_gpu_work():
    lib = U.load()
    out = C.c_void_p()
    assert lib.urchin_build_bvh(None, None, C.byref(out), None) == U.URCHIN_ERR_ARG
    p = U.urchin_particles(0, None, None, None, None, None)
    box = U.urchin_box(0, 0.0, 1.0)
    assert lib.urchin_build_bvh(C.byref(p), C.byref(box), C.byref(out), None) == U.URCHIN_ERR_ARG
    p.n = 10
    assert lib.urchin_build_bvh(C.byref(p), C.byref(box), C.byref(out), None) == U.URCHIN_ERR_ARG
    assert out.value is None
    dirs = np.zeros(3)
    assert lib.urchin_trace_columns(None, None, dirs.ctypes.data_as(C.c_void_p), 1, 1.0, None, 0, 0, 0,
                                    None, None) == U.URCHIN_ERR_ARG
    sp = U.urchin_spectrum(0, None, None)
    assert lib.urchin_gamma(None, 0, 10, 12, C.byref(sp), None, None, None) == U.URCHIN_ERR_ARG
    sp = U.urchin_spectrum(10, C.c_void_p(16), C.c_void_p(16))
    assert lib.urchin_gamma(None, 0, 10, 0, C.byref(sp), None, None, None) == U.URCHIN_ERR_ARG
    assert lib.urchin_gamma(None, 7, 10, 12, C.byref(sp), None, None, None) == U.URCHIN_ERR_ARG
    assert lib.urchin_equilibrium(None, None, None, None, 5, 9, 0.0, None, None) == U.URCHIN_ERR_ARG
    assert lib.urchin_equilibrium(None, None, None, None, -1, 0, 0.0, None, None) == U.URCHIN_ERR_ARG
    # CASE_AUTO without tau_eff
    assert lib.urchin_equilibrium(C.c_void_p(16), None, C.c_void_p(16), C.c_void_p(16), 5, 2, 0.0,
                                  C.c_void_p(16), None) == U.URCHIN_ERR_ARG
    assert lib.urchin_solve(None, None, None, None, None) == U.URCHIN_ERR_ARG
    # reverse-mode entry points
    assert lib.urchin_trace_columns_vjp(None, dirs.ctypes.data_as(C.c_void_p), 1, 1.0, None, 5, 0, 0, None,
                                        None, None) == U.URCHIN_ERR_ARG
    assert lib.urchin_gamma_vjp(C.c_void_p(16), 0, 10, 12, C.byref(sp), C.c_void_p(16), None, None,
                                None) == U.URCHIN_ERR_ARG                  # no output requested
    assert lib.urchin_gamma_vjp(None, 5, 10, 12, C.byref(sp), None, None, None, None) == U.URCHIN_ERR_ARG
    assert lib.urchin_equilibrium_vjp(None, None, None, None, 5, 9, 0.0, None, None, None) == U.URCHIN_ERR_ARG
    assert lib.urchin_equilibrium_vjp(None, None, None, None, 0, 0, 0.0, None, None, None) == U.URCHIN_OK
    assert lib.urchin_gamma_vjp(None, 0, 0, 12, C.byref(sp), None, None, None, None) == U.URCHIN_OK
    assert lib.urchin_solve_vjp(None, None, None, None, None, None, None) == U.URCHIN_ERR_ARG
    # the memory pool: bad device; nothing to trim before any GPU work
    assert lib.urchin_trim_memory(-2, None) == U.URCHIN_ERR_ARG
    left = C.c_uint64(7)
    assert lib.urchin_trim_memory(-1, C.byref(left)) == U.URCHIN_OK and left.value == 0
    # zero-size requests are no-ops
    assert lib.urchin_equilibrium(None, None, None, None, 0, 0, 0.0, None, None) == U.URCHIN_OK
    assert lib.urchin_gamma(None, 0, 0, 12, C.byref(sp), None, None, None) == U.URCHIN_OK


def test_solve_params_validation():
    lib = U.load()
    P = U.urchin_solve_params()
    dirs = U.urchin_healpix_dirs(1)
    P.R = 12
    P.dirs = dirs.ctypes.data_as(C.c_void_p)
    P.l_ray = 1.0
    P.spectrum = U.urchin_spectrum(10, C.c_void_p(16), C.c_void_p(16))
    P.nH = C.c_void_p(16)
    P.T = C.c_void_p(16)
    P.tol = 0.0                                   # invalid
    P.max_iter = 10
    st = U.urchin_solve_stats()
    fake = C.c_void_p(16)
    assert lib.urchin_solve(fake, C.byref(P), fake, C.byref(st), None) == U.URCHIN_ERR_ARG
    P.tol = 1e-3
    bad = dirs.copy()
    bad[0] *= 2.0                                 # not a unit vector
    P.dirs = bad.ctypes.data_as(C.c_void_p)
    assert lib.urchin_solve(fake, C.byref(P), fake, C.byref(st), None) == U.URCHIN_ERR_ARG
    assert "unit" in lib.urchin_last_error().decode()
    P.dirs = dirs.ctypes.data_as(C.c_void_p)
    P.method = 3                                  # no such method
    assert lib.urchin_solve(fake, C.byref(P), fake, C.byref(st), None) == U.URCHIN_ERR_ARG
    assert "method" in lib.urchin_last_error().decode()
    P.method = U.METHOD_PLAIN
    P.gmres_m = 10
    xb = C.c_void_p(16)
    assert lib.urchin_solve_vjp(fake, C.byref(P), fake, xb, xb, C.byref(st), None) == U.URCHIN_ERR_ARG
    assert "state" in lib.urchin_last_error().decode()       # the forward state is required
    for method in (U.METHOD_NEWTON,):
        P.method = method
        for m in (0, 65):                         # Krylov dimension out of range
            P.gmres_m = m
            assert lib.urchin_solve(fake, C.byref(P), fake, C.byref(st), None) == U.URCHIN_ERR_ARG
            assert "gmres_m" in lib.urchin_last_error().decode()
