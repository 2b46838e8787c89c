"""Pins of the oracle's helium columns (not in the paper, which treats
hydrogen only: fixed He I / He II columns attenuate the same spectrum)."""
import numpy as np

import oracle as O
import workloads as W


def test_gamma_he_without_helium_is_the_hydrogen_rate():
    rng = np.random.default_rng(1)
    w = W.halo(n=10, seed=1, F=40)
    e, J = w.spectrum()
    s, wts = O.spectrum(e, J, w.gamma_thin)
    tau = np.exp(rng.uniform(np.log(1e-3), np.log(30.0), (7, 12)))
    z = np.zeros_like(tau)
    g, te = O.gamma_he(tau, z, z, s, 0.5 * s, 0.2 * s, wts)
    g0, te0 = O.gamma(tau, s, wts)
    np.testing.assert_allclose(g, g0, rtol=1e-14)


def test_gamma_he_single_bin_closed_form():
    s, s1, s2, w = np.array([0.7]), np.array([1.9]), np.array([0.4]), np.array([2e-12])
    tau = np.array([[0.3, 2.0]])
    t1 = np.array([[0.1, 0.5]])
    t2 = np.array([[1.0, 0.0]])
    g, te = O.gamma_he(tau, t1, t2, s, s1, s2, w)
    ref = 2e-12 * np.mean(np.exp(-(0.7 * tau + 1.9 * t1 + 0.4 * t2)))
    assert abs(g[0] / ref - 1) < 1e-14


def test_solve_with_zero_helium_is_the_hydrogen_solve():
    w = W.halo(n=300, seed=3, n0=0.3, F=20)
    e, J = w.spectrum()
    s, wts = O.spectrum(e, J, w.gamma_thin)
    dirs = O.healpix(1)
    zero = np.zeros((w.n, 12))
    he = dict(tau1=zero, tau2=zero, s1=0.3 * s, s2=0.1 * s)
    x1, f1, s1_ = O.solve(w, s, wts, dirs, sweeps=4, he=he)
    x0, f0, s0_ = O.solve(w, s, wts, dirs, sweeps=4)
    np.testing.assert_array_equal(x1, x0)


def test_helium_columns_shield_more():
    """Adding absorbing helium columns can only lower the rate."""
    rng = np.random.default_rng(2)
    w = W.halo(n=10, seed=1, F=40)
    e, J = w.spectrum()
    s, wts = O.spectrum(e, J, w.gamma_thin)
    tau = np.exp(rng.uniform(np.log(1e-3), np.log(30.0), (7, 12)))
    t1 = rng.uniform(0, 3, tau.shape)
    g, _ = O.gamma_he(tau, t1, np.zeros_like(tau), s, s, np.zeros_like(s), wts)
    g0, _ = O.gamma(tau, s, wts)
    assert np.all(g <= g0)
