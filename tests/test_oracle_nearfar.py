"""Pins of the oracle's near/far split and slab solution (Sec. 3.3.3 and
the appendix on a plane-parallel slab), CPU only."""
import numpy as np
import pytest

import oracle as O
import workloads as W

scipy_integrate = pytest.importorskip("scipy.integrate")


def _slab_by_ode(G0, nH, T, caseB, tau_near):
    """ln Gamma at depth tau_near by integrating the slab equations directly:
    with t = sigma_th nH z, dtau_HI/dt = x(t), x(t) the equilibrium neutral
    fraction at Gamma(t) = G0 exp(-tau_HI(t)) (monochromatic at threshold)."""
    def rhs(t, y):
        return [O.xeq(G0 * np.exp(-y[0]), nH, T, 0.0, caseB)[0]]
    sol = scipy_integrate.solve_ivp(rhs, (0.0, tau_near), [0.0], method="LSODA", rtol=1e-11, atol=1e-13)
    return np.log(G0) - sol.y[0, -1]


@pytest.mark.parametrize("caseB", [False, True])
@pytest.mark.parametrize("ratio", [1e-3, 1.0, 30.0])
@pytest.mark.parametrize("tau_near", [0.1, 3.0, 40.0])
def test_slab_solution_matches_direct_integration(caseB, ratio, tau_near):
    nH, T = 1e-3, 1e4
    aA, aB, gc = O.rates(T)
    G0 = ratio * (aB if caseB else aA) * nH
    got = O.slab_lngamma(G0, nH, T, caseB, tau_near)[0]
    ref = _slab_by_ode(G0, nH, T, caseB, tau_near)
    assert abs(got - ref) <= 1e-7 * max(1.0, abs(ref))


def test_slab_limits():
    nH, T = 1e-2, 1e4
    aA, aB, gc = O.rates(T)
    G0 = 5.0 * aA * nH
    assert O.slab_lngamma(G0, nH, T, False, 0.0)[0] == np.log(G0)
    assert O.slab_lngamma(0.0, nH, T, False, 5.0)[0] == -np.inf
    # deep in the slab the gas is at x_ce: Gamma falls as exp(-x_ce dtau)
    xce = aA / (aA + gc)
    l1 = O.slab_lngamma(G0, nH, T, False, 400.0)[0]
    l2 = O.slab_lngamma(G0, nH, T, False, 500.0)[0]
    assert abs((l2 - l1) / 100.0 + xce) < 1e-9
    # thicker slabs shield more
    vals = O.slab_lngamma(G0, nH, T, False, np.array([0.01, 0.1, 1.0, 10.0]))
    assert np.all(np.diff(vals) < 0)


def test_near_far_columns_partition_the_column():
    """With every x = 1 the far and near columns add up to the full column,
    and the origin itself is always near (periodic lattice and halo)."""
    for w in (W.lattice_box(n_side=6, box_kpc=375.0, l_ray=250.0), W.halo(n=300, seed=3)):
        dirs = O.healpix(1)
        org = np.arange(0, w.n, 5)
        one = np.ones(w.n)
        tf, tn = O.columns_nearfar(w, one, dirs, origins=org)
        tot = O.columns(w, one, dirs, origins=org)
        np.testing.assert_allclose(tf + tn, tot, rtol=1e-12, atol=0)
        assert (tn > 0).all()
        # far columns scale with x, near columns do not
        tf2, tn2 = O.columns_nearfar(w, 0.25 * one, dirs, origins=org)
        np.testing.assert_allclose(tf2, 0.25 * tf, rtol=1e-13, atol=0)
        np.testing.assert_allclose(tn2, tn, rtol=0, atol=0)


def test_near_set_is_the_scatter_neighbourhood():
    """A particle is near for origin i exactly when it contributes to the
    density at r_i in Eq. nhi: two particles, the second placed just inside
    and just outside the first's... own smoothing radius of the second."""
    base = W.halo(n=2, seed=1)
    for inside, expect_near in ((0.99, True), (1.01, False)):
        pos = np.array([[0.0, 0.0, 0.0], [inside * 2.0, 0.0, 0.0]], dtype=np.float32)
        w = W.subset(base, np.arange(2))
        w = w.__class__(**{**w.__dict__, "pos": pos, "h": np.array([1.0, 2.0], dtype=np.float32),
                           "l_ray": 10.0})
        d = np.array([[1.0, 0.0, 0.0]])
        tf, tn = O.columns_nearfar(w, np.ones(2), d, origins=[0])
        tot = O.columns(w, np.ones(2), d, origins=[0])
        self_only = O.columns(W.subset(w, np.arange(1)), np.ones(1), d, origins=[0])
        if expect_near:
            assert tf[0, 0] == 0.0 and abs(tn[0, 0] - tot[0, 0]) <= 1e-12 * tot[0, 0]
        else:
            assert abs(tn[0, 0] - self_only[0, 0]) <= 1e-12 * self_only[0, 0]
            assert abs(tf[0, 0] + tn[0, 0] - tot[0, 0]) <= 1e-12 * tot[0, 0]


def test_gamma_nearfar_without_near_column_is_the_plain_rate():
    rng = np.random.default_rng(4)
    w = W.halo(n=10, seed=1)
    e, J = w.spectrum()
    s, wts = O.spectrum(e, J, w.gamma_thin)
    tau = np.exp(rng.uniform(np.log(1e-3), np.log(20.0), (6, 12)))
    lr, g = O.gamma_nearfar(tau, np.zeros_like(tau), s, wts, 1e-3, 1e4, False)
    g0, te0 = O.gamma(tau, s, wts)
    np.testing.assert_allclose(g, g0, rtol=1e-12)
    np.testing.assert_allclose(-lr, te0, rtol=1e-11, atol=1e-14)


def test_gamma_nearfar_fully_shielded_is_zero():
    """Eq. gammashld: when the far column of every ray is so thick that no
    radiation reaches the slab (every bin's attenuation underflows), the
    particle's rate is the empty sum: Gamma = 0, and the equilibrium is the
    collisional x = alpha / (alpha + gamma_c).  The analytic slab, lit by the
    far-attenuated rate, reports ln(Gamma / Gamma_thin) = -inf; the
    polychromatic slab carries the attenuation in log form and reports its
    finite logarithm (far below the smallest double).  A ray that still lets
    radiation through keeps the rate finite."""
    w = W.halo(n=10, seed=1)
    e, J = w.spectrum()
    s, wts = O.spectrum(e, J, w.gamma_thin)
    tf = np.full((2, 12), 1e6)
    tf[1, 3] = 2.0
    tn = np.full((2, 12), 5.0)
    for poly in (False, True):
        lr, g = O.gamma_nearfar(tf, tn, s, wts, np.array([1.0, 1.0]), np.array([1e4, 1e4]),
                                np.array([True, True]), poly=poly)
        assert g[0] == 0.0 and (lr[0] < -745.0 if poly else lr[0] == -np.inf), (poly, lr[0])
        assert np.isfinite(lr[1]) and g[1] > 0.0, poly
        aA, aB, gc = O.rates(1e4)
        assert abs(O.xeq(g[0], 1.0, 1e4, 0.0, True)[0] - aB / (aB + gc)) <= 1e-15


def test_near_far_iteration_converges_faster_than_the_plain_scheme():
    """Sec. 3.3.3: with the near particles modelled as a slab, Gamma of a
    particle no longer depends on its own and its neighbours' x, which
    removes the slow growth of neutral regions of the plain scheme."""
    w = W.halo(n=400, seed=7, n0=0.3, F=20)
    e, J = w.spectrum()
    s, wts = O.spectrum(e, J, w.gamma_thin)
    dirs = O.healpix(1)
    xp, fp, sp = O.solve(w, s, wts, dirs, tol=1e-8, max_iter=3000)
    xn, fn, sn = O.solve(w, s, wts, dirs, tol=1e-8, max_iter=3000, near_far=True)
    assert sp["converged"] and sn["converged"]
    assert sn["sweeps"] < sp["sweeps"]


# -- the polychromatic slab (numerical slab solution) --------------------------
@pytest.mark.parametrize("caseB", [False, True])
@pytest.mark.parametrize("tau_far", [0.0, 2.0])
@pytest.mark.parametrize("tau_near", [0.05, 5.0, 60.0])
def test_poly_slab_reduces_to_the_analytic_slab_for_one_bin(caseB, tau_far, tau_near):
    """A single bin at the threshold (s = 1) is monochromatic radiation: the
    numerical slab integration must give the appendix's analytic solution."""
    nH, T = 3e-3, 1.2e4
    aA, aB, gc = O.rates(T)
    w = np.array([20.0 * (aB if caseB else aA) * nH])
    s = np.array([1.0])
    got = O.slab_poly_lngamma(s, w, tau_far, nH, T, caseB, tau_near)[0]
    ref = O.slab_lngamma(w[0] * np.exp(-tau_far), nH, T, caseB, tau_near)[0]
    assert abs(got - ref) <= 1e-8 * max(1.0, abs(ref))


def test_poly_slab_limits_and_hardening():
    w_ = W.halo(n=10, seed=1, F=50)
    e, J = w_.spectrum()
    s, wts = O.spectrum(e, J, w_.gamma_thin)
    nH, T = 1e-2, 1e4
    for tf in (0.0, 3.0):
        lgf = np.log((wts * np.exp(-s * tf)).sum())
        assert abs(O.slab_poly_lngamma(s, wts, tf, nH, T, False, 0.0)[0] - lgf) < 1e-14 * max(1, abs(lgf))
        # every bin at or above the threshold has s <= 1: the slab is at least
        # as transparent as one lit at the threshold with the same rate
        for tn in (0.1, 3.0, 30.0, 300.0):
            poly = O.slab_poly_lngamma(s, wts, tf, nH, T, False, tn)[0]
            mono = O.slab_lngamma(np.exp(lgf), nH, T, False, tn)[0]
            assert poly >= mono - 1e-10
        vals = O.slab_poly_lngamma(s, wts, tf, nH, T, False, np.array([0.01, 0.1, 1.0, 10.0, 100.0]))
        assert np.all(np.diff(vals) < 0)


def test_poly_near_far_iteration_converges():
    w = W.halo(n=400, seed=7, n0=0.3, F=20)
    e, J = w.spectrum()
    s, wts = O.spectrum(e, J, w.gamma_thin)
    dirs = O.healpix(1)
    x1, f1, s1 = O.solve(w, s, wts, dirs, tol=1e-8, max_iter=300, near_far=1)
    x2, f2, s2 = O.solve(w, s, wts, dirs, tol=1e-8, max_iter=300, near_far=2)
    assert s1["converged"] and s2["converged"]
    # the hardened spectrum penetrates the near slab further: less neutral gas
    assert np.median(x2 / x1) <= 1.0 + 1e-12


# -- Test 1's slab solver (NS) ---------------------------------------------------
def test_ns_slab_matches_the_slab_solutions():
    """The slice-by-slice slab solver converges (first order in the slice
    thickness) to the integrated slab equations, and for one threshold bin to
    the analytic solution."""
    w_ = W.halo(n=10, seed=1, F=50)
    e, J = w_.spectrum()
    s, wts = O.spectrum(e, J, 1e-12)
    sth = O.sigma_th()
    for nH in (1.1e-3, 1.3e-3):
        tot = sth * nH * 200.0 * 3.0856775814913673e21
        x, t = O.ns_slab(s, wts, nH, 1e4, False, tot, 200000)
        lg = O.slab_poly_lngamma(s, wts, 0.0, nH, 1e4, False, tot)[0]
        xb = O.xeq(np.exp(lg), nH, 1e4, 0.0, False)[0]
        assert abs(x[-1] / xb - 1) < 1e-3
        x2, t2 = O.ns_slab(s, wts, nH, 1e4, False, tot, 100000)
        assert abs(t2 / t - 1) < 1e-3
    aA, aB, gc = O.rates(1e4)
    one_s, one_w = np.array([1.0]), np.array([30.0 * aA * 1e-3])
    x, t = O.ns_slab(one_s, one_w, 1e-3, 1e4, False, 20.0, 400000)
    xa = O.xeq(np.exp(O.slab_lngamma(one_w[0], 1e-3, 1e4, False, 20.0)[0]), 1e-3, 1e4, 0.0, False)[0]
    assert abs(x[-1] / xa - 1) < 1e-3


def test_ns_slab_two_sided():
    """Test 3's solver: symmetric about the mid-plane, equal to the one-sided
    solver in the optically thin limit, and, when thick, holding less neutral
    gas than the slab lit from one side with the whole rate (which in turn
    holds less than with half of it)."""
    w_ = W.halo(n=10, seed=1, F=50)
    e, J = w_.spectrum()
    s, wts = O.spectrum(e, J, 1e-12)
    sth = O.sigma_th()
    L = 200.0 * 3.0856775814913673e21
    x, t = O.ns_slab2(s, wts, 1e-4, 1e4, False, sth * 1e-4 * L, 2000)
    x1, t1 = O.ns_slab(s, wts, 1e-4, 1e4, False, sth * 1e-4 * L, 2000)
    assert abs(t / t1 - 1) < 2e-3
    x, t = O.ns_slab2(s, wts, 1.3e-3, 1e4, False, sth * 1.3e-3 * L, 4000)
    np.testing.assert_allclose(x, x[::-1], rtol=1e-9)
    _, t_full = O.ns_slab(s, wts, 1.3e-3, 1e4, False, sth * 1.3e-3 * L, 4000)
    _, t_half = O.ns_slab(s, 0.5 * wts, 1.3e-3, 1e4, False, sth * 1.3e-3 * L, 4000)
    assert t < t_full < t_half


def test_each_ray_slab_takes_its_share_of_the_radiation():
    """Eq. gammashld: ray k carries 4 pi / N_ray of the radiation, so its
    slab is lit by (1/R) of the far-attenuated rate and the slabs' bottom
    rates add up: with R identical rays the rate is R G(Gamma_far / R)."""
    w_ = W.halo(n=10, seed=1, F=30)
    e, J = w_.spectrum()
    s, wts = O.spectrum(e, J, w_.gamma_thin)
    nH, T = 2e-3, 1e4
    for R in (1, 2, 12):
        tf = np.full((1, R), 0.7)
        tn = np.full((1, R), 4.0)
        lr, g = O.gamma_nearfar(tf, tn, s, wts, nH, T, False)
        gfar = (wts * np.exp(-s * 0.7)).sum()
        ref = R * np.exp(O.slab_lngamma(gfar / R, nH, T, False, 4.0)[0])
        assert abs(g[0] / ref - 1) < 1e-12
        lrp, gp = O.gamma_nearfar(tf, tn, s, wts, nH, T, False, poly=True)
        refp = R * np.exp(O.slab_poly_lngamma(s, wts / R, 0.7, nH, T, False, 4.0)[0])
        assert abs(gp[0] / refp - 1) < 1e-12
