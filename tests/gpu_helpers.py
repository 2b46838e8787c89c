"""Shared helpers for the GPU tests: move a workload to the device and run the
oracle on the same inputs."""
import numpy as np

import oracle as O
import workloads as W
from paper_1304_4235_gb300 import urchin as U


def device_particles(w, torch):
    dev = "cuda"
    pos = np.asarray(w.pos, dtype=np.float32)
    return dict(
        px=torch.from_numpy(np.ascontiguousarray(pos[:, 0])).to(dev),
        py=torch.from_numpy(np.ascontiguousarray(pos[:, 1])).to(dev),
        pz=torch.from_numpy(np.ascontiguousarray(pos[:, 2])).to(dev),
        h=torch.from_numpy(np.ascontiguousarray(w.h, dtype=np.float32)).to(dev),
        m=torch.from_numpy(np.ascontiguousarray(w.mass_H, dtype=np.float64)).to(dev),
        nH=torch.from_numpy(np.ascontiguousarray(w.nH, dtype=np.float64)).to(dev),
        T=torch.from_numpy(np.ascontiguousarray(w.T, dtype=np.float64)).to(dev),
    )


def build(w, torch):
    d = device_particles(w, torch)
    bvh = U.urchin_build_bvh(d["px"], d["py"], d["pz"], d["h"], d["m"], w.periodic, w.box, w.unit_cm)
    return bvh, d


def spectra(w, torch):
    """(s, w) from the library for the GPU and from the oracle for the oracle."""
    e, J = w.spectrum()
    s_g, w_g = U.urchin_spectrum_weights(e, J, w.gamma_thin)
    s_o, w_o = O.spectrum(e, J, w.gamma_thin)
    return (torch.from_numpy(s_g).cuda(), torch.from_numpy(w_g).cuda()), (s_o, w_o)


def rel_err(a, b, floor=0.0):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def small_halo(n=20000, seed=1405):
    return W.halo(n=n, seed=seed)


def lnrate_sensitivity(tau, s, w):
    """D_o = sum_k tau_ok |d ln Gamma_o / d tau_ok| of Eq. gamma_shld, in
    log-sum-exp form (no underflow at large tau): a relative error eps in
    every column of origin o moves ln Gamma_o by at most eps D_o."""
    from scipy.special import logsumexp
    tau = np.asarray(tau, dtype=np.float64)
    s, w = np.asarray(s, dtype=np.float64), np.asarray(w, dtype=np.float64)
    e = -tau[:, :, None] * s[None, None, :]                       # [n, R, F]
    n = tau.shape[0]
    with np.errstate(divide="ignore"):
        num = logsumexp((e + np.log(w * s)[None, None, :] + np.log(tau)[:, :, None]).reshape(n, -1), axis=1)
    den = logsumexp((e + np.log(w)[None, None, :]).reshape(n, -1), axis=1)
    return np.exp(num - den)


def helium_rate(w, so, he, columns, eps_col):
    """A rate for check_sweep with fixed helium columns: he = dict(t1, t2
    [n, R] (the oracle's He I / He II columns of every particle), s1, s2).
    The GPU traces the helium columns in FP32 too, so the sensitivity is that
    of ln Gamma to all three columns at once, by central differences of the
    oracle's rate under a common relative change (every partial derivative
    has the same sign, so this is the sum of their magnitudes)."""
    def rate(x_prev, org):
        tau = columns(x_prev, org)
        t1, t2 = he["t1"][org], he["t2"][org]
        G, te = O.gamma_he(tau, t1, t2, so[0], he["s1"], he["s2"], so[1])
        d = 1e-4
        gp, _ = O.gamma_he(tau * (1 + d), t1 * (1 + d), t2 * (1 + d), so[0], he["s1"], he["s2"], so[1])
        gm, _ = O.gamma_he(tau * (1 - d), t1 * (1 - d), t2 * (1 - d), so[0], he["s1"], he["s2"], so[1])
        with np.errstate(divide="ignore", invalid="ignore"):
            D = np.nan_to_num(np.abs(np.log(gm) - np.log(gp)) / (2 * d), nan=0.0)
        return G, te, D
    return rate


def check_sweep(w, so, x_prev, state_prev, x_next, org, nside, sweep0, tau_skip=1e-4, case_rule=2,
                eps_col=1e-6, eps_fold=2e-6, columns=None, rate=None):
    """One FP32 sweep of the GPU against the oracle's update of the GPU's own
    previous state, particle by particle, with a stated error model instead
    of a quantile: the FP32 columns carry a relative error <= eps_col (the
    column tests measure <= 3e-7) and the spectral fold <= eps_fold in ln
    Gamma, so |ln Gamma_gpu - ln Gamma| <= dl = eps_fold + eps_col D
    (lnrate_sensitivity) and |ln x_gpu - ln x| <= |d ln x / d ln Gamma| dl.
    Decisions that the error can flip are checked for validity: within dl of
    tau_eff = 1 (unlatched) either recombination case is accepted, within dl
    of tau_skip in sweep 0 either freezing or updating.  state_prev: uint8
    per particle (bit 0 case B latched, bit 1 frozen) or None for sweep 0.
    rate (optional) replaces the hydrogen-only fold: rate(x_prev, org) ->
    (Gamma, tau_eff, D) (helium_rate).  Asserts, and returns the largest
    error / bound (<= 1) over `org`."""
    dirs = O.healpix(nside)
    org = np.asarray(org)
    cols = columns if columns is not None else (lambda x, o: O.columns(w, x, dirs, origins=o))
    if rate is None:
        tau = cols(x_prev, org)
        G, te = O.gamma(tau, so[0], so[1])
        D = lnrate_sensitivity(tau, so[0], so[1])
    else:
        G, te, D = rate(x_prev, org)
    dl = eps_fold + eps_col * D
    worst = 0.0
    for a, i in enumerate(org):
        xn, xp = float(x_next[i]), float(x_prev[i])
        if not sweep0 and state_prev is not None and (state_prev[i] & 2):
            assert xn == xp, ("frozen particle changed", i)
            continue
        # frozen in sweep 0 (allowed within dl of tau_skip): x stays at x_thin, which
        # the device and the oracle compute with their own math libraries
        if sweep0 and te[a] < tau_skip + dl[a] and abs(xn - xp) <= 1e-12 * xp:
            continue
        assert not sweep0 or te[a] >= tau_skip - dl[a], ("particle should be frozen", i)
        latched = (not sweep0) and state_prev is not None and bool(state_prev[i] & 1)
        if case_rule == 2:
            cases = [True] if (latched or te[a] - dl[a] >= 1.0) else ([False] if te[a] + dl[a] < 1.0 else [False, True])
        else:
            cases = [case_rule == 1]
        best = np.inf
        for cb in cases:
            e = float(O.xeq(G[a], w.nH[i], w.T[i], 0.0, cb)[0])
            el = abs(G[a] * float(O.xeq_dgamma(G[a], w.nH[i], w.T[i], 0.0, cb)[0]) / e)
            bound = el * dl[a] + 1e-12
            best = min(best, abs(xn - e) / e / bound)
        worst = max(worst, best)
        assert best <= 1.0, ("sweep update outside the error model", int(i), best, float(te[a]), float(dl[a]))
    return worst
