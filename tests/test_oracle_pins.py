"""Pins of the FP64 oracle to facts fixed outside it (paper, textbooks,
mathematics).  CPU only.  Each test names the passage or fact it checks;
together they are chosen so that a dropped term, wrong sign, wrong index or
transposed operand anywhere in the oracle fails at least one of them."""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import brentq

import oracle as O
import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


# --------------------------------------------------------------------------
# cross sections, App. C1
# --------------------------------------------------------------------------
def test_sigma_th_literature():
    g = GOLD["sigma_th_cm2"]
    assert abs(O.sigma_th() / g["value"] - 1) < g["rel_tol"]


def test_hydrogenic_threshold_and_Z_scaling():
    # Eq. sigma_ana tends to sigma_th at nu -> nu_th, and an ion of charge Z
    # has its threshold at Z^2 E_th with sigma reduced by Z^2.
    Eth = O.E_th()
    assert abs(O.sigma_hydrogenic([Eth * (1 + 1e-10)])[0] / O.sigma_th() - 1) < 1e-8
    assert O.sigma_hydrogenic([Eth * 0.999])[0] == 0.0
    for E in (15.0, 30.0, 54.0):
        s1 = O.sigma_hydrogenic([E], 1.0)[0]
        s2 = O.sigma_hydrogenic([4 * E], 2.0)[0]
        assert abs(s2 * 4 / s1 - 1) < 1e-12


def test_verner_fit_matches_exact_hydrogenic():
    # The Verner fit (with the exponent -P on (1+sqrt(x/x_a))) reproduces the
    # exact hydrogenic cross section over 1-4 Ryd to <1 per cent; the form
    # as printed (without -P) would be off by more than an order of magnitude.
    E = np.linspace(O.E_th() * 1.0001, 54.4, 40)
    r = O.sigma(E, O.XSEC_VERNER) / O.sigma_hydrogenic(E)
    assert np.all(np.abs(r - 1) < 0.01)
    g = GOLD["verner_HI"]
    x = O.E_th() / g["E0_eV"]
    printed = g["sigma0_Mb"] * 1e-18 * (x - 1) ** 2 * x ** (0.5 * g["P"] - 5.5) * (1 + math.sqrt(x / g["x_a"]))
    assert printed / O.sigma_th() > 10


def test_powerlaw_cross_section():
    Eth = O.E_th()
    assert abs(O.sigma([Eth * (1 + 1e-12)], O.XSEC_POWERLAW)[0] / O.sigma_th() - 1) < 1e-9
    assert abs(O.sigma([2 * Eth], O.XSEC_POWERLAW)[0] / O.sigma_th() - 0.125) < 1e-12


# --------------------------------------------------------------------------
# kernels, Sec. 4.1.1 and App. B
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [O.m4_shape, O.gt_shape])
def test_kernel_normalisation(shape):
    # 4 pi int_0^h r^2 W dr = 1 with W = 8/(pi h^3) shape(r/h)  (App. B)
    val = quad(lambda q: 4 * math.pi * q * q * 8 / math.pi * shape(q), 0, 1,
               points=[0.5], epsabs=1e-15, epsrel=1e-14)[0]
    assert abs(val - 1) < 1e-12


def test_kernel_difference_appendix_b():
    g = GOLD["kernel_difference"]
    q = np.linspace(0, 1, 2001)
    m4 = np.array([O.m4_shape(v) for v in q])
    gt = np.array([O.gt_shape(v) for v in q])
    assert np.max(np.abs(m4 - gt)) < g["max_diff_frac"] * m4.max()
    assert gt[-1] < g["gt_at_h_frac"] * m4.max()
    assert O.m4_shape(1.0001) == 0.0 and O.gt_shape(1.0001) == 0.0


def test_gt_central_value_matches_m4():
    # sigma(h) is fixed by G(0, sigma^2) = M4(0, h): (2 pi sigma^2)^(-3/2) = 8/(pi h^3)
    t = GOLD["gt_kernel"]["t"]
    assert abs(t - 2 * math.pi ** (1 / 6)) < 1e-15
    sig2 = 1.0 / (8 * math.pi ** (1 / 3))
    assert abs((2 * math.pi * sig2) ** -1.5 / (8 / math.pi) - 1) < 1e-14
    # so the untruncated Gaussian's centre equals the M4 centre; G_t is that
    # Gaussian renormalised for truncation at h, hence larger by 1/D > 1
    assert O.gt_shape(0.0) > 1.0 and O.gt_shape(0.0) < 1.05


@pytest.mark.parametrize("kernel,shape", [(O.KERNEL_M4, O.m4_shape), (O.KERNEL_GT, O.gt_shape)])
def test_chord_integral_vs_quadrature(kernel, shape):
    # closed-form line integral (Eq. I(h,b,z1,z2) for G_t, antiderivatives for
    # M4) against adaptive quadrature of the kernel along the line
    rng = np.random.default_rng(11)
    for _ in range(400):
        b = rng.random()
        c = math.sqrt(1 - b * b)
        u1, u2 = np.sort(rng.uniform(-1.2 * c, 1.2 * c, 2))
        val = O.chord(kernel, b, u1, u2)
        lo, hi = max(u1, -c), min(u2, c)
        if hi <= lo:
            assert val == 0.0
            continue
        s = math.sqrt(max(0.0, 0.25 - b * b))
        pts = [p for p in (-s, 0.0, s) if lo < p < hi]
        ref = quad(lambda u: shape(math.sqrt(b * b + u * u)), lo, hi, points=pts or None,
                   epsabs=1e-16, epsrel=1e-13, limit=400)[0]
        assert abs(val - ref) < 1e-13 + 1e-11 * abs(ref), (b, u1, u2, val, ref)


def test_full_chord_centre_column():
    # M4: int_{-h}^{h} W(|u|/h) du = 6/(pi h^2);  G_t: N sqrt(pi) erf(t)/A
    assert abs(8 / math.pi * O.chord(O.KERNEL_M4, 0.0, -1, 1) - 6 / math.pi) < 1e-14
    t = 2 * math.pi ** (1 / 6)
    D = math.erf(t) - 2 * t * math.exp(-t * t) / math.sqrt(math.pi)
    expect = (8 / math.pi / D) * math.sqrt(math.pi) * math.erf(t) / t
    assert abs(8 / math.pi * O.chord(O.KERNEL_GT, 0.0, -1, 1) - expect) < 1e-13


@pytest.mark.parametrize("kernel", [O.KERNEL_M4, O.KERNEL_GT])
def test_projected_kernel_integrates_to_mass(kernel):
    def K(b):
        c = math.sqrt(max(0.0, 1 - b * b))
        return 8 / math.pi * O.chord(kernel, b, -c, c)
    val = quad(lambda b: 2 * math.pi * b * K(b), 0, 1, points=[0.5], epsabs=1e-15, epsrel=1e-13)[0]
    assert abs(val - 1) < 1e-11


# --------------------------------------------------------------------------
# columns, Eq. nhi / Eq. colden
# --------------------------------------------------------------------------
def _tiny_isolated(n=14, seed=3):
    rng = np.random.default_rng(seed)
    w = W.halo(n=200, seed=seed)
    w = W.subset(w, np.arange(n))
    w.pos = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    w.h = rng.uniform(0.4, 0.9, n).astype(np.float32)
    w.mass_H = rng.uniform(0.5, 2.0, n) * 1e62
    w.l_ray = 1.5
    return w


@pytest.mark.parametrize("kernel,shape", [(O.KERNEL_M4, O.m4_shape), (O.KERNEL_GT, O.gt_shape)])
def test_columns_vs_density_line_integral(kernel, shape):
    # N_HI = int_0^L n_HI(r(l)) dl with n_HI from the scatter sum Eq. nhi,
    # integrated numerically, equals the per-particle chord sum Eq. colden.
    w = _tiny_isolated()
    rng = np.random.default_rng(5)
    x = rng.uniform(0.1, 1.0, w.n)
    dirs = O.healpix(1)
    tau = O.columns(w, x, dirs, origins=np.array([0, 3, 7]), kernel=kernel)
    p = w.pos.astype(np.float64)
    h = w.h.astype(np.float64)
    cm = w.unit_cm
    for oi, i in enumerate([0, 3, 7]):
        for k in range(12):
            def nHI(l):
                r = p[i] + l * dirs[k]
                q = np.linalg.norm(p - r, axis=1) / h
                return sum(w.mass_H[j] * x[j] * 8 / (math.pi * (h[j] * cm) ** 3) * shape(q[j])
                           for j in range(w.n) if q[j] < 1)
            # breakpoints where some q crosses 1/2 or 1 or is minimal
            bps = set()
            for j in range(w.n):
                d = p[j] - p[i]
                tc = d @ dirs[k]
                b2 = d @ d - tc * tc
                for rad in (0.5 * h[j], h[j]):
                    if b2 < rad * rad:
                        hc = math.sqrt(rad * rad - b2)
                        bps.update([tc - hc, tc + hc])
                bps.add(tc)
            pts = sorted(v for v in bps if 0 < v < w.l_ray)
            N = quad(nHI, 0, w.l_ray, points=pts or None, epsabs=0, epsrel=1e-11, limit=500)[0] * cm
            assert abs(O.sigma_th() * N / tau[oi, k] - 1) < 1e-9


def test_periodic_images_equal_explicit_replication():
    rng = np.random.default_rng(9)
    n, L = 30, 10.0
    base = _tiny_isolated(n=n)
    base.pos = rng.uniform(0, L, (n, 3)).astype(np.float32)
    base.h = rng.uniform(1.5, 3.5, n).astype(np.float32)
    base.periodic, base.box, base.l_ray = True, L, 6.0
    x = rng.uniform(0.2, 1.0, n)
    dirs = O.healpix(2)
    org = np.arange(0, n, 3)
    tau_p = O.columns(base, x, dirs, origins=org)
    # explicit 5x5x5 tiling, isolated
    shifts = np.array([(a, b, c) for a in range(-2, 3) for b in range(-2, 3) for c in range(-2, 3)]) * L
    rep = W.subset(base, np.tile(np.arange(n), len(shifts)))
    rep.pos = (base.pos.astype(np.float64)[None] + shifts[:, None]).reshape(-1, 3)  # exact images
    rep.periodic, rep.box = False, 0.0
    centre = int(np.where((shifts == 0).all(1))[0][0])
    tau_r = O.columns(rep, np.tile(x, len(shifts)), dirs, origins=centre * n + org)
    assert np.allclose(tau_p, tau_r, rtol=1e-13, atol=0)


def test_uniform_box_face_averaged_column():
    # Mass conservation: rays of length L across a periodic box, averaged over
    # the face, give N_H = sum_j m_j / L^2 (= n_H L for uniform gas).
    w = W.lattice_box(n_side=8, box_kpc=1.0, n_ngb=32, seed=7)
    G = 40
    g = (np.arange(G) + 0.5) / G
    Y, Z = np.meshgrid(g, g, indexing="ij")
    for axis, plane in ((0, 0.123), (1, 0.77)):
        pts = np.zeros((G * G, 3))
        pts[:, axis] = plane
        others = [a for a in range(3) if a != axis]
        pts[:, others[0]] = Y.ravel()
        pts[:, others[1]] = Z.ravel()
        d = np.zeros((1, 3))
        d[0, axis] = 1.0
        tau = O.columns_points(w, np.ones(w.n), pts, d, l_ray=1.0)
        N = tau / O.sigma_th()
        expect = w.mass_H.sum() / (w.box * w.unit_cm) ** 2
        assert abs(N.mean() / expect - 1) < 1e-5


def test_zero_length_and_zero_x_give_zero_column():
    w = _tiny_isolated()
    dirs = O.healpix(1)
    assert np.all(O.columns(w, np.ones(w.n), dirs, l_ray=0.0) == 0)
    assert np.all(O.columns(w, np.zeros(w.n), dirs) == 0)


def test_self_column_is_half_chord():
    # a lone particle: every ray sees half the central column, 3/(pi h^2) m x
    w = _tiny_isolated(n=1)
    tau = O.columns(w, np.array([0.5]), O.healpix(1))
    hcm = float(w.h[0]) * w.unit_cm
    expect = O.sigma_th() * w.mass_H[0] * 0.5 * 3 / (math.pi * hcm * hcm)
    assert np.allclose(tau, expect, rtol=1e-13)


# --------------------------------------------------------------------------
# HEALPix, Sec. 3.2 / App. A
# --------------------------------------------------------------------------
def test_healpix_nside1():
    d = O.healpix(1)
    assert d.shape == (12, 3)
    z = np.sort(np.unique(np.round(d[:, 2], 12)))[::-1]
    assert np.allclose(z, GOLD["healpix_nside1"]["rings_z"])
    for zz in z:
        ring = d[np.isclose(d[:, 2], zz)]
        assert len(ring) == 4
        phi = np.sort(np.mod(np.arctan2(ring[:, 1], ring[:, 0]), 2 * np.pi))
        assert np.allclose(np.diff(phi), np.pi / 2)
        off = np.pi / 4 if abs(zz) > 0.1 else 0.0
        assert np.isclose(np.mod(phi[0] - off + 1e-12, np.pi / 2), 1e-12, atol=1e-9)


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_healpix_properties(nside):
    d = O.healpix(nside)
    assert d.shape == (12 * nside * nside, 3)
    assert np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-14)
    assert np.allclose(d.sum(0), 0, atol=1e-12)
    # ring latitudes: caps z = +-(1 - i^2/(3 Ns^2)), belt z = 4/3 - 2i/(3 Ns)
    zs = sorted(set(np.round(d[:, 2], 10)))
    expect = set()
    for i in range(1, nside):
        expect.update([round(1 - i * i / (3 * nside * nside), 10), round(-(1 - i * i / (3 * nside * nside)), 10)])
    for i in range(nside, 3 * nside + 1):
        expect.add(round(4 / 3 - 2 * i / (3 * nside), 10))
    assert set(zs) == expect
    # equal-area: each ring holds 4i (cap) or 4 Ns (belt) pixels
    for zz in zs:
        cnt = int(np.sum(np.isclose(d[:, 2], zz, atol=1e-9)))
        if abs(zz) > 2 / 3 + 1e-9:
            i = round(math.sqrt(3 * nside * nside * (1 - abs(zz))))
            assert cnt == 4 * i
        else:
            assert cnt == 4 * nside
    # all directions distinct
    dots = d @ d.T - 2 * np.eye(len(d))
    assert dots.max() < 1 - 1e-6


# --------------------------------------------------------------------------
# spectrum and Gamma, Eq. gamma / Eq. gamma_shld
# --------------------------------------------------------------------------
def test_spectrum_normalisation_and_quadrature():
    F = 400
    edges, J = W.powerlaw_spectrum(F, 13.6, 54.4, 1.5)
    s, w = O.spectrum(edges, J, 1e-12)
    assert abs(w.sum() / 1e-12 - 1) < 1e-13
    assert np.all(s > 0) and np.all(w > 0)
    # sum_j w_j s_j / Gamma_thin -> int J sigma^2/E dE / (sigma_th int J sigma/E dE)
    f1 = lambda E: (E / 13.6) ** -1.5 * O.sigma([E])[0] / E
    num = quad(lambda E: f1(E) * O.sigma([E])[0] / O.sigma_th(), 13.6, 54.4, epsrel=1e-10)[0]
    den = quad(f1, 13.6, 54.4, epsrel=1e-10)[0]
    assert abs((w * s).sum() / w.sum() / (num / den) - 1) < 1e-4


def test_gamma_thin_reproduced():
    # x = 0 or l_ray = 0 gives Gamma = Gamma_thin exactly, tau_eff = 0
    edges, J = W.powerlaw_spectrum(50, 13.6, 54.4)
    s, wts = O.spectrum(edges, J, 1e-12)
    w = _tiny_isolated()
    for x, L in ((np.zeros(w.n), w.l_ray), (np.ones(w.n), 0.0)):
        tau = O.columns(w, x, O.healpix(1), l_ray=L)
        g, te = O.gamma(tau, s, wts)
        # equal up to the summation order of sum_j w_j (a few ulp)
        assert np.all(np.abs(g / wts.sum() - 1) < 1e-14)
        assert np.all(np.abs(te) < 1e-14)


def test_gamma_monochromatic_attenuation():
    # one bin with s = 1: Gamma / Gamma_thin = mean_k exp(-tau_k)
    rng = np.random.default_rng(2)
    tau = rng.uniform(0, 30, (7, 12))
    g, te = O.gamma(tau, np.array([1.0]), np.array([3e-12]))
    assert np.allclose(g / 3e-12, np.exp(-tau).mean(1), rtol=1e-14)
    assert np.allclose(te, -np.log(np.exp(-tau).mean(1)), rtol=1e-12)


# --------------------------------------------------------------------------
# rates and equilibrium, App. C3
# --------------------------------------------------------------------------
def test_recombination_rates_textbook():
    g = GOLD["recombination_1e4K"]
    aA, aB, gc = O.rates(1e4)
    assert abs(aA / g["alpha_A"] - 1) < g["rel_tol_A"]
    assert abs(aB / g["alpha_B"] - 1) < g["rel_tol_B"]
    assert aA > aB
    assert 1e-16 < gc < 1e-14          # collisional ionisation negligible at 1e4 K


def test_collisional_rate_vs_independent_fit():
    # Voronov (1997) fit for H I: A (U^K) e^-U / (X + U), A = 2.91e-8,
    # X = 0.232, K = 0.39, U = 13.6 eV / kT; independent of the Hui & Gnedin fit
    for T in (3e4, 1e5, 3e5, 1e6):
        U = 13.6 / (8.617333262e-5 * T)
        vor = 2.91e-8 * U ** 0.39 * math.exp(-U) / (0.232 + U)
        assert abs(O.rates(T)[2] / vor - 1) < 0.15


@pytest.mark.parametrize("T", [5e3, 1e4, 3e4, 1e5])
@pytest.mark.parametrize("caseB", [False, True])
def test_xeq_without_radiation(T, caseB):
    # Eq. xphys: Gamma = 0, y = 0 -> x = alpha / (alpha + gamma)
    aA, aB, gc = O.rates(T)
    a = aB if caseB else aA
    assert abs(O.xeq(0.0, 1e-2, T, 0.0, caseB)[0] / (a / (a + gc)) - 1) < 1e-14


def test_xeq_against_high_precision_root():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(4)
    for _ in range(200):
        G = 10 ** rng.uniform(-20, -10)
        nH = 10 ** rng.uniform(-6, 2)
        T = 10 ** rng.uniform(3.7, 6)
        y = rng.uniform(0, 0.1)
        cb = bool(rng.integers(2))
        aA, aB, gc = O.rates(T)
        a = mp.mpf(aB if cb else aA)
        g = mp.mpf(gc)
        R = (g + a) * nH
        Q = -(G + a * nH + R * (1 + y))
        P = a * nH * (1 + y)
        roots = sorted(mp.polyroots([R, Q, P], maxsteps=200, extraprec=200), key=lambda r: mp.re(r))
        ref = float(mp.re(roots[0]))
        got = O.xeq(G, nH, T, y, cb)[0]
        assert abs(got / ref - 1) < 1e-13
        assert 0 < got <= 1


def test_xeq_optically_thin_limit():
    # Sec. 5.4: in thin gas x = alpha n_H / Gamma
    aA = O.rates(1e4)[0]
    for G in (1e-8, 1e-6):
        x = O.xeq(G, 1e-4, 1e4)[0]
        assert abs(x * G / (aA * 1e-4) - 1) < 1e-4


# --------------------------------------------------------------------------
# iteration driver, Sec. 4
# --------------------------------------------------------------------------
def _spec(F=20):
    edges, J = W.powerlaw_spectrum(F, 13.6, 54.4)
    return O.spectrum(edges, J, 1e-12)


def _lone(mass):
    w = _tiny_isolated(n=1)
    w.mass_H = np.array([mass])
    w.h = np.array([2.0], dtype=np.float32)
    w.nH = np.array([0.05])
    w.l_ray = 5.0                          # longer than h: full half chord
    return w


@pytest.mark.parametrize("mass", [1e62, 3e62, 3e63])
@pytest.mark.parametrize("case_rule", [O.CASE_A, O.CASE_B])
def test_lone_particle_fixed_point(mass, case_rule):
    # One particle: every ray sees its own half chord, tau_k = c x; with a
    # fixed recombination case the equilibrium is the scalar root of
    # x = E(Gamma(x)), found here by a bracketing root finder on an
    # independently integrated column.
    w = _lone(mass)
    s, wts = _spec()
    hcm = 2.0 * w.unit_cm
    half = quad(lambda l: 8 / (math.pi * hcm ** 3) * O.m4_shape(l / hcm), 0, hcm,
                points=[0.5 * hcm], epsabs=0, epsrel=1e-13)[0]
    c = O.sigma_th() * w.mass_H[0] * half
    aA, aB, gc = O.rates(1e4)
    a = aB if case_rule == O.CASE_B else aA

    def E(x):
        G = float(np.sum(wts * np.exp(-s * c * x)))
        # x_- = (-Q - sqrt(Q^2 - 4PR)) / (2R), y = 0, in the form of the
        # smaller root that avoids cancellation: 2P / (-Q + sqrt(...))
        R = (a + gc) * 0.05
        Q = -(G + a * 0.05 + R)
        P = a * 0.05
        return 2 * P / (-Q + math.sqrt(max(Q * Q - 4 * P * R, 0.0)))
    xs = brentq(lambda x: x - E(x), 1e-12, 1.0, xtol=1e-15, rtol=1e-14)
    x, frozen, st = O.solve(w, s, wts, O.healpix(1), tol=1e-13, max_iter=500, case_rule=case_rule)
    assert st["converged"] and not frozen[0]
    assert abs(x[0] / xs - 1) < 1e-10


def test_lone_particle_case_switch_latch():
    # With the automatic switch (case B iff tau_eff >= 1) this particle has no
    # self-consistent state: its case-A equilibrium is thick (tau_eff > 1) and
    # its case-B equilibrium thin.  Applied afresh each sweep the rule makes
    # Jacobi alternate between the two forever; the driver latches case B
    # once tau_eff has reached 1, so the run settles on the case-B state.
    w = _lone(3e62)
    s, wts = _spec()
    xa, _, _ = O.solve(w, s, wts, O.healpix(1), tol=1e-13, max_iter=500, case_rule=O.CASE_A)
    xb, _, _ = O.solve(w, s, wts, O.healpix(1), tol=1e-13, max_iter=500, case_rule=O.CASE_B)
    g = lambda x: O.gamma(O.columns(w, x, O.healpix(1)), s, wts)[1][0]
    assert g(xa) > 1 and g(xb) < 1
    # the rule applied afresh every sweep alternates A and B
    x = O.xeq(wts.sum(), w.nH, w.T, 0.0, False)
    seen = []
    for _ in range(60):
        te = g(x)
        x = O.xeq(O.gamma(O.columns(w, x, O.healpix(1)), s, wts)[0], w.nH, w.T, 0.0, te >= 1)
        seen.append(te >= 1)
    assert any(seen[-10:]) and not all(seen[-10:])
    x3, _, st3 = O.solve(w, s, wts, O.healpix(1), tol=1e-12, max_iter=500)
    assert st3["converged"]
    assert abs(x3[0] / xb[0] - 1) < 1e-9


def test_driver_freezes_thin_particles():
    w = _tiny_isolated()
    w.mass_H = w.mass_H * 1e-12            # columns far below tau_skip
    s, wts = _spec()
    x, frozen, st = O.solve(w, s, wts, O.healpix(1))
    assert frozen.all() and st["sweeps"] == 1 and st["converged"]
    xt = O.xeq(wts.sum(), w.nH, w.T, 0.0, False)
    assert np.array_equal(x, xt)


def test_driver_sweep_semantics():
    # two sweeps of the driver equal the Jacobi composition of its primitives
    w = _tiny_isolated()
    w.mass_H = w.mass_H * 300
    s, wts = _spec()
    dirs = O.healpix(1)
    x2, frozen, st = O.solve(w, s, wts, dirs, sweeps=2)
    x0 = O.xeq(wts.sum(), w.nH, w.T, 0.0, False)
    tau = O.columns(w, x0, dirs)
    g, te = O.gamma(tau, s, wts)
    act = te >= 1e-4
    assert np.array_equal(act, ~frozen)
    x1 = x0.copy()
    x1[act] = O.xeq(g[act], w.nH[act], w.T[act], 0.0, te[act] >= 1)
    idx = np.where(act)[0]
    tau = O.columns(w, x1, dirs, origins=idx)
    g, te = O.gamma(tau, s, wts)
    xe = x1.copy()
    xe[idx] = O.xeq(g, w.nH[idx], w.T[idx], 0.0, te >= 1)
    assert np.allclose(x2, xe, rtol=1e-14, atol=0)
    assert st["rays"] == (w.n + act.sum()) * 12


def test_density_ordered_blocks_semantics():
    # two sweeps with the high-to-low density order in 3 blocks equal the
    # composition of the primitives in that order (Sec. 4 update order)
    w = _tiny_isolated(n=14)
    w.mass_H = w.mass_H * 300
    w.nH = np.linspace(1.0, 0.1, w.n)[::-1].copy()       # density rises with index
    s, wts = _spec()
    dirs = O.healpix(1)
    x2, frozen, st = O.solve(w, s, wts, dirs, sweeps=2, blocks=3)
    x0 = O.xeq(wts.sum(), w.nH, w.T, 0.0, False)
    g, te = O.gamma(O.columns(w, x0, dirs), s, wts)
    act = np.where(te >= 1e-4)[0]
    x1 = x0.copy()
    x1[act] = O.xeq(g[act], w.nH[act], w.T[act], 0.0, te[act] >= 1)
    latch = np.zeros(w.n, bool)
    latch[act] = te[act] >= 1
    order = sorted(act, key=lambda i: (-np.float32(w.nH[i]), i))
    m = len(order)
    xe = x1.copy()
    for b in range(3):
        blk = np.array(order[(b * m) // 3:((b + 1) * m) // 3])
        g, te = O.gamma(O.columns(w, xe, dirs, origins=blk), s, wts)
        cb = (te >= 1) | latch[blk]
        latch[blk] = cb
        xe[blk] = O.xeq(g, w.nH[blk], w.T[blk], 0.0, cb)
    assert np.allclose(x2, xe, rtol=1e-14, atol=0)


def test_density_order_reaches_jacobi_fixed_point():
    w = _tiny_isolated(n=14)
    w.mass_H = w.mass_H * 300
    s, wts = _spec()
    dirs = O.healpix(1)
    xj, _, sj = O.solve(w, s, wts, dirs, tol=1e-12, max_iter=2000, case_rule=O.CASE_A)
    xb, _, sb = O.solve(w, s, wts, dirs, tol=1e-12, max_iter=2000, case_rule=O.CASE_A, blocks=4)
    assert sj["converged"] and sb["converged"]
    assert np.allclose(xj, xb, rtol=1e-9)
    assert sb["sweeps"] <= sj["sweeps"]


# -- uniform-grid query (the timed CPU baseline) -------------------------------
@pytest.mark.parametrize("case", ["lattice", "halo", "small_box_long_rays"])
def test_grid_columns_equal_brute_force(case):
    """The grid query changes only how the candidate particles of a ray are
    found: its columns equal the brute-force sum over all particles (and
    all periodic images) of Eq. colden to rounding order, rel 1e-12, for
    periodic and isolated sets, both kernels, N_side 1 and 2, and rays
    longer than half a small periodic box (several images of a particle on
    one ray)."""
    if case == "lattice":
        w, cells = W.lattice_box(), (40.0, 130.0, 300.0)
    elif case == "halo":
        w, cells = W.halo(n=4096, seed=1405), (2.0, 8.0, 30.0)
    else:
        w, cells = W.lattice_box(n_side=6, box_kpc=100.0, seed=21), (8.0, 10.0)
        w.l_ray = 90.0
    rng = np.random.default_rng(3)
    x = np.exp(rng.uniform(np.log(1e-4), 0.0, w.n))
    org = W.random_origins(w.n, 200, 4)
    for nside, kernel in ((1, O.KERNEL_M4), (2, O.KERNEL_GT)):
        dirs = O.healpix(nside)
        ref = O.columns(w, x, dirs, origins=org, kernel=kernel)
        for cell in cells:
            got = O.Grid(w, cell).columns(x, dirs, origins=org, kernel=kernel)
            assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref)), (case, nside, cell)


def test_grid_refuses_a_sphere_spanning_the_box():
    w = W.lattice_box(n_side=6, box_kpc=100.0, seed=21)
    with pytest.raises(ValueError):
        O.Grid(w, 60.0)


def test_grid_solve_step_matched_equals_brute_force():
    """The Sec. 4 driver with grid columns takes the brute-force driver's
    steps (same freeze and case decisions, x to 1e-12)."""
    w = W.halo(n=3000, seed=1406)
    e, J = w.spectrum()
    s, wts = O.spectrum(e, J, w.gamma_thin)
    dirs = O.healpix(1)
    xb, fb, sb = O.solve(w, s, wts, dirs, sweeps=4)
    xg, fg, sg = O.solve(w, s, wts, dirs, sweeps=4, grid_cell=5.0)
    assert np.array_equal(fb, fg) and np.array_equal(sb["caseB"], sg["caseB"])
    assert np.all(np.abs(xg - xb) <= 1e-12 * xb)
