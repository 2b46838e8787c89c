"""Pins of the oracle's derivatives (CPU only).  Each derivative is checked
against something other than itself: central finite differences of the
oracle's forward functions, the adjoint (dot-product) identity of the linear
column map, and a closed-form limit of the equilibrium root."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _spec(w):
    e, J = w.spectrum()
    return O.spectrum(e, J, w.gamma_thin)


def test_column_matrix_reproduces_columns():
    """tau = M x (Eq. colden is linear in x), periodic lattice and halo."""
    for w in (W.lattice_box(n_side=6, box_kpc=375.0, l_ray=250.0), W.halo(n=300, seed=3)):
        rng = np.random.default_rng(1)
        x = rng.uniform(1e-3, 1.0, w.n)
        org = np.arange(0, w.n, 7)
        dirs = O.healpix(1)
        M = O.column_matrix(w, dirs, org)
        tau = O.columns(w, x, dirs, origins=org)
        np.testing.assert_allclose(M @ x, tau, rtol=1e-12, atol=0)


def test_columns_vjp_adjoint_identity():
    """<tau_bar, tau(v)> = <columns_vjp(tau_bar), v> for random v, tau_bar."""
    w = W.halo(n=400, seed=5)
    dirs = O.healpix(1)
    rng = np.random.default_rng(2)
    org = rng.choice(w.n, 60, replace=False)
    tb = rng.standard_normal((org.shape[0], 12))
    v = rng.standard_normal(w.n)
    lhs = float((tb * O.columns(w, v, dirs, origins=org)).sum())
    xb = O.columns_vjp(w, dirs, tb, origins=org, chunk=17)
    assert abs(lhs - float(xb @ v)) <= 1e-11 * np.abs(tb).sum() * np.abs(O.columns(w, np.abs(v), dirs, origins=org)).max()


def test_gamma_partials_match_finite_differences():
    rng = np.random.default_rng(3)
    w = W.halo(n=10, seed=1)
    s, wts = _spec(w)
    tau = np.exp(rng.uniform(np.log(1e-3), np.log(30.0), (5, 12)))
    dG_dtau, dG_dw = O.gamma_partials(tau, s, wts)
    for o, k in ((0, 0), (2, 5), (4, 11)):
        d = 1e-6 * tau[o, k]
        tp, tm = tau.copy(), tau.copy()
        tp[o, k] += d
        tm[o, k] -= d
        fd = (O.gamma(tp, s, wts)[0][o] - O.gamma(tm, s, wts)[0][o]) / (2 * d)
        assert abs(dG_dtau[o, k] - fd) <= 1e-6 * abs(fd)
    for b in (0, 37, 99):
        d = 1e-6 * wts[b]
        wp, wm = wts.copy(), wts.copy()
        wp[b] += d
        wm[b] -= d
        fd = (O.gamma(tau, s, wp)[0] - O.gamma(tau, s, wm)[0]) / (2 * d)
        np.testing.assert_allclose(dG_dw[:, b], fd, rtol=1e-6)


@pytest.mark.parametrize("caseB", [False, True])
def test_xeq_dgamma_matches_finite_differences(caseB):
    # (at Gamma = 0 with collisional ionisation ~0 the root behaves like
    # 1 - sqrt(Gamma / alpha n_H): the derivative is finite but far outside
    # any finite-difference step's linear range, so Gamma = 0 is not sampled)
    for G in (1e-16, 1e-13, 1e-12, 1e-10):
        for nH in (1e-5, 1e-3, 1e-1, 10.0):
            for T in (5e3, 1e4, 3e4):
                d = 1e-5 * G
                a = O.xeq_dgamma(G, nH, T, 0.0, caseB)[0]
                fd = (O.xeq(G + d, nH, T, 0.0, caseB)[0] - O.xeq(G - d, nH, T, 0.0, caseB)[0]) / (2 * d)
                assert a < 0
                assert abs(a - fd) <= 2e-5 * abs(fd), (G, nH, T)


def test_xeq_dgamma_thin_limit():
    """x -> alpha n_H / Gamma when Gamma >> alpha n_H, so dx/dGamma ->
    -alpha n_H / Gamma^2 (relative corrections of order alpha n_H / Gamma)."""
    aA, aB, gc = O.rates(1e4)
    nH = 1e-6
    G = 1e6 * aA * nH
    a = O.xeq_dgamma(G, nH, 1e4, 0.0, False)[0]
    assert abs(a / (-aA * nH / G**2) - 1.0) < 1e-5


def _loss_weights(n, seed=11):
    return np.random.default_rng(seed).standard_normal(n)


@pytest.mark.parametrize("n0,tau_skip", [(0.1, 1e-2), (0.3, 1e-4)])
def test_solve_vjp_matches_finite_differences_of_the_solve(n0, tau_skip):
    """dL/dw_b of L = sum_i c_i ln x*_i by the implicit function theorem
    against central differences of the converged Jacobi iteration; the
    first case has frozen particles (whose x_thin depends on sum w), case A
    and case B particles."""
    w = W.halo(n=400, seed=7, n0=n0, F=20)
    s, wts = _spec(w)
    dirs = O.healpix(1)
    x, fr, st = O.solve(w, s, wts, dirs, tol=1e-14, max_iter=5000, tau_skip=tau_skip)
    assert st["converged"]
    c = _loss_weights(w.n)
    wbar, mu = O.solve_vjp(w, s, wts, dirs, x, fr, st["caseB"], c / x)
    for b in (0, 7, 19):
        d = 1e-4 * wts[b]
        wp, wm = wts.copy(), wts.copy()
        wp[b] += d
        wm[b] -= d
        xp, frp, sp = O.solve(w, s, wp, dirs, tol=1e-14, max_iter=5000, tau_skip=tau_skip)
        xm, frm, sm = O.solve(w, s, wm, dirs, tol=1e-14, max_iter=5000, tau_skip=tau_skip)
        assert (frp == fr).all() and (frm == fr).all()
        assert (sp["caseB"] == st["caseB"]).all() and (sm["caseB"] == st["caseB"]).all()
        fd = (c @ np.log(xp) - c @ np.log(xm)) / (2 * d)
        assert abs(wbar[b] - fd) <= 1e-5 * abs(fd) + 1e-7 * np.abs(wbar).max(), (b, wbar[b], fd)
    if n0 == 0.1:
        assert fr.sum() > 0 and st["caseB"].sum() > 0 and (~st["caseB"] & ~fr).sum() > 0
