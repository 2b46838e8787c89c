"""Reverse mode of the CUDA path against the oracle's derivatives (which are
pinned by finite differences of the forward oracle).  Tolerances:
  columns transpose   FP64 rel 1e-10 (atomic summation order), FP32 rel 1e-5
  gamma / equilibrium transposes on identical inputs, double arithmetic: rel 1e-10
  gradient of the converged x w.r.t. the spectrum weights (FP64 columns,
  adjoint GMRES to 1e-12): rel 1e-7 per component (floor 1e-3 of the
  largest component, where the sum over particles cancels); with FP32
  columns (adjoint to 1e-6) rel 5e-4 per component, same floor
Every check is per component: a transpose that sums terms of both signs is
measured against the sum of the terms' magnitudes (the natural bound of a
reordered sum), a product against itself.  In FP64 a grazing chord's
closed form cancels to ~1e-16 of the kernel's central value on both sides,
so components made of grazing chords only are held to a floor of 1e-6 of
the largest component.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import build, small_halo, spectra

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1304_4235_gb300 import urchin as U  # noqa: E402
from paper_1304_4235_gb300 import autograd as UA  # noqa: E402


def _rel(a, b, mag=None, floor=0.0):
    """Largest per-component error |a - b| relative to mag (the sum of the
    terms' magnitudes where b is a sum with cancelling terms), else to |b|,
    never below floor * max |b|."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    m = np.abs(b) if mag is None else np.asarray(mag, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(m, max(floor * np.abs(b).max(), 1e-300))))


@pytest.mark.parametrize("precision", [U.F64, U.F32])
def test_columns_vjp_matches_oracle(precision):
    w = W.halo(n=3000, seed=21)
    bvh, d = build(w, torch)
    dirs = U.urchin_healpix_dirs(1)
    org = W.random_origins(w.n, 300, 4)
    rng = np.random.default_rng(5)
    tb = rng.standard_normal((org.shape[0], 12))
    tb[::7] = 0.0                                   # rays skipped by the zero test
    dt = torch.float64 if precision == U.F64 else torch.float32
    xb = U.urchin_trace_columns_vjp(bvh, dirs, w.l_ray, torch.from_numpy(tb).to(dt).cuda(),
                                    origins=torch.from_numpy(org.astype(np.int32)).cuda(), precision=precision)
    tbu = tb.astype(np.float32).astype(np.float64) if precision == U.F32 else tb
    ref = O.columns_vjp(w, O.healpix(1), tbu, origins=org)
    mag = O.columns_vjp(w, O.healpix(1), np.abs(tbu), origins=org)
    assert _rel(xb.cpu().numpy(), ref, mag, floor=1e-6) < (1e-10 if precision == U.F64 else 1e-5)


def test_columns_vjp_all_origins_periodic_accumulates():
    """All origins (Morton traversal, original-order rows), periodic images,
    and accumulation into a given x_bar."""
    w = W.lattice_box(n_side=10, box_kpc=625.0, l_ray=312.5)
    bvh, d = build(w, torch)
    dirs = U.urchin_healpix_dirs(1)
    tb = np.random.default_rng(6).uniform(-1, 1, (w.n, 12))
    x0 = torch.ones(w.n, dtype=torch.float64, device="cuda")
    xb = U.urchin_trace_columns_vjp(bvh, dirs, w.l_ray, torch.from_numpy(tb).cuda(), precision=U.F64, x_bar=x0)
    ref = O.columns_vjp(w, O.healpix(1), tb) + 1.0
    mag = O.columns_vjp(w, O.healpix(1), np.abs(tb)) + 1.0
    assert _rel(xb.cpu().numpy(), ref, mag, floor=1e-6) < 1e-10


@pytest.mark.parametrize("precision", [U.F64, U.F32])
def test_gamma_vjp_matches_oracle(precision):
    w = small_halo()
    sg, so = spectra(w, torch)
    rng = np.random.default_rng(7)
    tau = np.exp(rng.uniform(np.log(1e-4), np.log(50.0), (500, 12)))
    dt = torch.float64 if precision == U.F64 else torch.float32
    tau_t = torch.from_numpy(tau).to(dt).cuda()
    tau_used = tau_t.double().cpu().numpy()
    gbar = rng.standard_normal(500)
    tb, wb = U.urchin_gamma_vjp(tau_t, sg[0], sg[1], torch.from_numpy(gbar).cuda())
    dG_dtau, dG_dw = O.gamma_partials(tau_used, so[0], so[1])
    assert _rel(tb.double().cpu().numpy(), gbar[:, None] * dG_dtau) < (1e-10 if precision == U.F64 else 2e-7)
    # w_bar: double sums in FP64; in FP32 the per-bin sum runs in float over
    # tiles of 128 rays (k_wbar_tiles_f32), within 2e-6 of the magnitude sum
    assert _rel(wb.cpu().numpy(), gbar @ dG_dw, np.abs(gbar) @ dG_dw) < (1e-10 if precision == U.F64 else 2e-6)


@pytest.mark.parametrize("case_rule", [U.CASE_A, U.CASE_B, U.CASE_AUTO])
def test_equilibrium_vjp_matches_oracle(case_rule):
    rng = np.random.default_rng(8)
    n = 2000
    G = np.exp(rng.uniform(np.log(1e-17), np.log(1e-11), n))
    nH = np.exp(rng.uniform(np.log(1e-5), np.log(10.0), n))
    T = rng.uniform(5e3, 3e4, n)
    te = rng.uniform(0, 2, n).astype(np.float32)
    xb = rng.standard_normal(n)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gb = U.urchin_equilibrium_vjp(c(G), c(te), c(nH), c(T), c(xb), case_rule)
    caseB = {U.CASE_A: np.zeros(n, bool), U.CASE_B: np.ones(n, bool), U.CASE_AUTO: te >= 1}[case_rule]
    ref = xb * O.xeq_dgamma(G, nH, T, 0.0, caseB)
    np.testing.assert_allclose(gb.cpu().numpy(), ref, rtol=1e-10, atol=0)


def _tiny(n0):
    w = W.halo(n=400, seed=7, n0=n0, F=20)
    bvh, d = build(w, torch)
    sg, so = spectra(w, torch)
    return w, bvh, d, sg, so


@pytest.mark.parametrize("segments", [U.SEG_RECOMPUTE, U.SEG_STORE])
@pytest.mark.parametrize("n0,tau_skip", [(0.1, 1e-2), (0.3, 1e-4)])
def test_solve_vjp_matches_oracle(n0, tau_skip, segments):
    """dL/dw of L = sum c_i ln x*_i on the GPU against the oracle's dense
    implicit-function gradient at the same x* and state (frozen particles,
    case A and case B present in the first case)."""
    w, bvh, d, sg, so = _tiny(n0)
    dirs = U.urchin_healpix_dirs(1)
    state = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    x, st = U.urchin_solve(bvh, dirs, w.l_ray, sg[0], sg[1], d["nH"], d["T"], tol=1e-13, max_iter=5000,
                           tau_skip=tau_skip, precision=U.F64, segments=segments, state=state)
    xs = x.cpu().numpy()
    stt = state.cpu().numpy()
    frozen, caseB = (stt & 2) > 0, (stt & 1) > 0
    xo, fo, so_ = O.solve(w, so[0], so[1], O.healpix(1), tol=1e-13, max_iter=5000, tau_skip=tau_skip)
    assert (frozen == fo).all() and (caseB == so_["caseB"]).all()
    c = np.random.default_rng(11).standard_normal(w.n)
    xbar = c / xs
    wb, vst = U.urchin_solve_vjp(bvh, dirs, w.l_ray, sg[0], sg[1], d["nH"], d["T"], x, state,
                                 torch.from_numpy(xbar).cuda(), tol=1e-12, max_iter=3000, gmres_m=40,
                                 tau_skip=tau_skip, precision=U.F64, segments=segments)
    assert vst["converged"] and vst["max_rel_dx"] <= 1e-12
    ref, mu = O.solve_vjp(w, so[0], so[1], O.healpix(1), xs, frozen, caseB, xbar)
    assert _rel(wb.cpu().numpy(), ref, floor=1e-3) < 1e-7


@pytest.mark.parametrize("segments", [U.SEG_RECOMPUTE, U.SEG_STORE])
def test_solve_vjp_f32_columns(segments):
    """The FP32 transposed products (scatter traversal, or atomics over the
    padded stored segments) on a 3000-particle halo against the oracle's gradient at the same x* and state.
    FP32 columns carry ~1e-6 relative rounding into E, the ray coefficients
    and the GMRES products, so the adjoint is solved to 1e-6 and compared to
    1e-4 of the largest component."""
    w = W.halo(n=3000, seed=9, n0=0.3, F=20)
    bvh, d = build(w, torch)
    sg, so = spectra(w, torch)
    dirs = U.urchin_healpix_dirs(1)
    state = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    x, st = U.urchin_solve(bvh, dirs, w.l_ray, sg[0], sg[1], d["nH"], d["T"], tol=1e-6, max_iter=5000,
                           tau_skip=1e-3, precision=U.F32, segments=segments, state=state)
    xs = x.cpu().numpy()
    stt = state.cpu().numpy()
    xbar = np.random.default_rng(15).standard_normal(w.n) / xs
    wb, vst = U.urchin_solve_vjp(bvh, dirs, w.l_ray, sg[0], sg[1], d["nH"], d["T"], x, state,
                                 torch.from_numpy(xbar).cuda(), tol=1e-6, max_iter=3000, gmres_m=40,
                                 tau_skip=1e-3, precision=U.F32, segments=segments)
    assert vst["converged"]
    ref, _ = O.solve_vjp(w, so[0], so[1], O.healpix(1), xs, (stt & 2) > 0, (stt & 1) > 0, xbar)
    assert _rel(wb.cpu().numpy(), ref, floor=1e-3) < 5e-4


def test_solve_vjp_warm_start_drops_the_frozen_term():
    w, bvh, d, sg, so = _tiny(0.1)
    dirs = U.urchin_healpix_dirs(1)
    state = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    x, st = U.urchin_solve(bvh, dirs, w.l_ray, sg[0], sg[1], d["nH"], d["T"], tol=1e-13, max_iter=5000,
                           tau_skip=1e-2, precision=U.F64, state=state)
    stt = state.cpu().numpy()
    xs = x.cpu().numpy()
    xbar = np.random.default_rng(12).standard_normal(w.n) / xs
    wb, _ = U.urchin_solve_vjp(bvh, dirs, w.l_ray, sg[0], sg[1], d["nH"], d["T"], x, state,
                               torch.from_numpy(xbar).cuda(), tol=1e-12, tau_skip=1e-2, precision=U.F64,
                               warm_start=True)
    ref, _ = O.solve_vjp(w, so[0], so[1], O.healpix(1), xs, (stt & 2) > 0, (stt & 1) > 0, xbar, warm_start=True)
    assert _rel(wb.cpu().numpy(), ref, floor=1e-3) < 1e-7


def test_autograd_column_misfit_gradient_matches_finite_differences():
    """The differentiation workload in miniature: loss = sum over rays of
    (log10 N_HI - log10 N_target)^2 at the converged x*(w), N_target from a
    run with the bin weights perturbed by a seeded +-20 %; d loss / d w by
    autograd (solve adjoint + column transpose) against central differences
    of the GPU forward solve, FP64 columns."""
    w, bvh, d, sg, so = _tiny(0.3)
    dirs = U.urchin_healpix_dirs(1)
    kw = dict(tol=1e-13, max_iter=5000, precision=U.F64)
    rng = np.random.default_rng(13)
    w_t = sg[1] * torch.from_numpy(rng.uniform(0.8, 1.2, sg[1].numel())).cuda()
    x_t, _ = U.urchin_solve(bvh, dirs, w.l_ray, sg[0], w_t, d["nH"], d["T"], **kw)
    target = torch.log10(U.urchin_trace_columns(bvh, x_t, dirs, w.l_ray, precision=U.F64))

    def loss_of(wv, grad):
        wv = wv.clone().requires_grad_(grad)
        x = UA.converged_x(wv, bvh, dirs, w.l_ray, sg[0], d["nH"], d["T"], solve_kw=kw,
                           vjp_kw=dict(tol=1e-12, max_iter=3000, gmres_m=40))
        tau = UA.columns(x, bvh, dirs, w.l_ray, precision=U.F64)
        L = ((torch.log10(tau) - target) ** 2).sum()
        if grad:
            L.backward()
            return L.item(), wv.grad.cpu().numpy()
        return L.item(), None

    L0, g = loss_of(sg[1], True)
    for b in (0, 9, 19):
        dw = 1e-4 * float(sg[1][b])
        wp, wm = sg[1].clone(), sg[1].clone()
        wp[b] += dw
        wm[b] -= dw
        fd = (loss_of(wp, False)[0] - loss_of(wm, False)[0]) / (2 * dw)
        assert abs(g[b] - fd) <= 1e-4 * abs(fd) + 1e-6 * np.abs(g).max(), (b, g[b], fd)


def test_c4_column_misfit_gradient_200_bins():
    """The column-misfit gradient of the differentiation workload (the halo's
    density law, 200 bins, loss = sum over all rays of (log10 N_HI -
    log10 N_target)^2 with the target from seeded +-20 % bin weights) on a
    4000-particle halo, FP64 stored segments: autograd against central
    differences of the forward solve at four seeded bins."""
    w = W.halo(n=4000, seed=41, F=200)
    bvh, d = build(w, torch)
    sg, so = spectra(w, torch)
    dirs = U.urchin_healpix_dirs(1)
    kw = dict(tol=1e-12, max_iter=20000, precision=U.F64, segments=U.SEG_STORE)
    rng = np.random.default_rng(42)
    w_t = sg[1] * torch.from_numpy(rng.uniform(0.8, 1.2, sg[1].numel())).cuda()
    x_t, st_t = U.urchin_solve(bvh, dirs, w.l_ray, sg[0], w_t, d["nH"], d["T"], **kw)
    target = torch.log10(U.urchin_trace_columns(bvh, x_t, dirs, w.l_ray, precision=U.F64))

    def loss_of(wv, grad):
        wv = wv.clone().requires_grad_(grad)
        x = UA.converged_x(wv, bvh, dirs, w.l_ray, sg[0], d["nH"], d["T"], solve_kw=kw,
                           vjp_kw=dict(tol=1e-12, max_iter=5000, gmres_m=40))
        tau = UA.columns(x, bvh, dirs, w.l_ray, precision=U.F64)
        L = ((torch.log10(tau) - target) ** 2).sum()
        if grad:
            L.backward()
            return L.item(), wv.grad.cpu().numpy()
        return L.item(), None

    L0, g = loss_of(sg[1], True)
    assert np.isfinite(g).all() and np.abs(g).max() > 0
    for b in np.sort(rng.choice(sg[1].numel(), size=4, replace=False)):
        dw = 1e-4 * float(sg[1][b])
        wp, wm = sg[1].clone(), sg[1].clone()
        wp[b] += dw
        wm[b] -= dw
        fd = (loss_of(wp, False)[0] - loss_of(wm, False)[0]) / (2 * dw)
        assert abs(g[b] - fd) <= 1e-4 * abs(fd) + 1e-6 * np.abs(g).max(), (b, g[b], fd)


def test_autograd_rate_gradient_in_x_matches_oracle():
    """d(sum_i a_i Gamma_i)/dx through columns and the spectral fold: the
    per-particle dGamma/dx products of the adjoint."""
    w = W.halo(n=2000, seed=31)
    bvh, d = build(w, torch)
    sg, so = spectra(w, torch)
    dirs = U.urchin_healpix_dirs(1)
    rng = np.random.default_rng(14)
    x0 = np.exp(rng.uniform(np.log(1e-3), 0.0, w.n))
    a = rng.standard_normal(w.n)
    x = torch.from_numpy(x0).cuda().requires_grad_(True)
    tau = UA.columns(x, bvh, dirs, w.l_ray, precision=U.F64)
    G, te = UA.shielded_rate(tau, sg[1], sg[0])
    (G * torch.from_numpy(a).cuda()).sum().backward()
    tau_o = O.columns(w, x0, O.healpix(1))
    dG_dtau, _ = O.gamma_partials(tau_o, so[0], so[1])
    ref = O.columns_vjp(w, O.healpix(1), a[:, None] * dG_dtau)
    mag = O.columns_vjp(w, O.healpix(1), np.abs(a[:, None] * dG_dtau))
    assert _rel(x.grad.cpu().numpy(), ref, mag, floor=1e-6) < 1e-9
