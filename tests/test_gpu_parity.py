"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.  Tolerances (stated per test):
  columns  FP64 mode rel 1e-11 (rounding order only); FP32 mode rel 1e-5
  Gamma    FP64 rel 1e-12; FP32 rel 2e-6 on identical FP32 columns (every
           bin's exponent s_j tau formed without rounding error)
  x        equilibrium on identical FP64 inputs rel 1e-12; end to end FP64
           rel 1e-9; FP32 sweeps per particle within check_sweep's error
           model (FP32 columns to 1e-6, fold to 2e-6 in ln Gamma, propagated
           through d ln x / d ln Gamma)
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import build, check_sweep, device_particles, rel_err, small_halo, spectra

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1304_4235_gb300 import urchin as U  # noqa: E402


@pytest.fixture(scope="module")
def lattice():
    w = W.lattice_box()
    bvh, d = build(w, torch)
    return w, bvh, d


@pytest.fixture(scope="module")
def halo_small():
    w = small_halo()
    bvh, d = build(w, torch)
    return w, bvh, d


def _x(w, seed=0, lo=1e-4, hi=1.0):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), w.n))


# --------------------------------------------------------------------------
# columns (Eq. colden)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kernel", [U.KERNEL_M4, U.KERNEL_GT])
def test_columns_lattice_fp64_all_origins(lattice, kernel):
    w, bvh, d = lattice
    x = _x(w, 1)
    dirs = U.urchin_healpix_dirs(1)
    tau = U.urchin_trace_columns(bvh, torch.from_numpy(x).cuda(), dirs, w.l_ray, kernel=kernel,
                                 precision=U.F64).cpu().numpy()
    ref = O.columns(w, x, O.healpix(1), kernel=kernel)
    assert rel_err(tau, ref).max() < 1e-11


@pytest.mark.parametrize("kernel", [U.KERNEL_M4, U.KERNEL_GT])
def test_columns_lattice_fp32_all_origins(lattice, kernel):
    w, bvh, d = lattice
    x = _x(w, 2)
    dirs = U.urchin_healpix_dirs(1)
    tau = U.urchin_trace_columns(bvh, torch.from_numpy(x).cuda(), dirs, w.l_ray, kernel=kernel,
                                 precision=U.F32).cpu().numpy()
    ref = O.columns(w, x, O.healpix(1), kernel=kernel)
    assert rel_err(tau, ref).max() < 1e-5


def test_columns_halo_fp32(halo_small):
    w, bvh, d = halo_small
    x = _x(w, 3)
    dirs = U.urchin_healpix_dirs(1)
    org = W.random_origins(w.n, 3000, 7)
    tau = U.urchin_trace_columns(bvh, torch.from_numpy(x).cuda(), dirs, w.l_ray,
                                 origins=torch.from_numpy(org).cuda()).cpu().numpy()
    ref = O.columns(w, x, O.healpix(1), origins=org)
    assert rel_err(tau, ref).max() < 1e-5
    tau64 = U.urchin_trace_columns(bvh, torch.from_numpy(x).cuda(), dirs, w.l_ray,
                                   origins=torch.from_numpy(org).cuda(), precision=U.F64).cpu().numpy()
    assert rel_err(tau64, ref).max() < 1e-11


@pytest.mark.parametrize("nside", [2, 4])
def test_columns_more_rays(halo_small, nside):
    w, bvh, d = halo_small
    x = _x(w, 4)
    org = W.random_origins(w.n, 400, 8)
    tau = U.urchin_trace_columns(bvh, torch.from_numpy(x).cuda(), U.urchin_healpix_dirs(nside), w.l_ray,
                                 origins=torch.from_numpy(org).cuda()).cpu().numpy()
    ref = O.columns(w, x, O.healpix(nside), origins=org)
    assert tau.shape == (400, 12 * nside * nside)
    assert rel_err(tau, ref).max() < 1e-5


def test_columns_full_size_halo_sampled():
    """262144-particle halo at its benchmark settings: all rays traced on the
    GPU, a seeded sample of origins recomputed by the oracle one by one."""
    w = W.halo()
    bvh, d = build(w, torch)
    x = _x(w, 5)
    dirs = U.urchin_healpix_dirs(1)
    tau = U.urchin_trace_columns(bvh, torch.from_numpy(x).cuda(), dirs, w.l_ray).cpu().numpy()
    org = W.random_origins(w.n, 256, 9)
    ref = O.columns(w, x, O.healpix(1), origins=org)
    assert rel_err(tau[org], ref).max() < 1e-5
    assert np.all(np.isfinite(tau)) and np.all(tau > 0)


def test_columns_edge_cases():
    dirs = U.urchin_healpix_dirs(1)
    od = O.healpix(1)
    # single particle: only its own half chord
    for n in (1, 2, 33, 1000):
        w = W.subset(small_halo(n=4000, seed=11), np.arange(n))
        bvh, d = build(w, torch)
        x = _x(w, n)
        tau = U.urchin_trace_columns(bvh, torch.from_numpy(x).cuda(), dirs, w.l_ray).cpu().numpy()
        ref = O.columns(w, x, od)
        assert rel_err(tau, ref).max() < 1e-5, n
    w = W.subset(small_halo(n=4000, seed=11), np.arange(500))
    bvh, d = build(w, torch)
    xg = torch.ones(w.n, dtype=torch.float64, device="cuda")
    # zero length and zero x give zero columns
    assert float(U.urchin_trace_columns(bvh, xg, dirs, 0.0).abs().max()) == 0.0
    assert float(U.urchin_trace_columns(bvh, torch.zeros_like(xg), dirs, w.l_ray).abs().max()) == 0.0
    # duplicated, unordered origins
    org = np.array([499, 3, 3, 250, 0, 499, 17], dtype=np.int32)
    tau = U.urchin_trace_columns(bvh, xg, dirs, w.l_ray, origins=torch.from_numpy(org).cuda()).cpu().numpy()
    ref = O.columns(w, np.ones(w.n), od, origins=org)
    assert rel_err(tau, ref).max() < 1e-5
    # empty origin list is a no-op
    out = U.urchin_trace_columns(bvh, xg, dirs, w.l_ray, origins=torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert out.shape == (0, 12)
    # out-of-range origin is an argument error
    with pytest.raises(U.UrchinError) as e:
        U.urchin_trace_columns(bvh, xg, dirs, w.l_ray, origins=torch.tensor([0, 500], dtype=torch.int32,
                                                                              device="cuda"))
    assert e.value.status == U.URCHIN_ERR_ARG


def test_columns_periodic_wrap_small_box():
    # spheres straddling the faces of a small periodic box; rays longer than
    # half the box so that several images of a particle are crossed
    w = W.lattice_box(n_side=6, box_kpc=100.0, n_ngb=32, seed=21)
    w.l_ray = 90.0
    bvh, d = build(w, torch)
    x = _x(w, 6)
    for prec, tol in ((U.F32, 1e-5), (U.F64, 1e-11)):
        tau = U.urchin_trace_columns(bvh, torch.from_numpy(x).cuda(), U.urchin_healpix_dirs(2), w.l_ray,
                                     precision=prec).cpu().numpy()
        ref = O.columns(w, x, O.healpix(2))
        assert rel_err(tau, ref).max() < tol


def test_build_rejects_nonfinite_and_bad_h():
    w = W.subset(small_halo(n=4000, seed=12), np.arange(100))
    d = device_particles(w, torch)
    d["px"][5] = float("nan")
    with pytest.raises(U.UrchinError) as e:
        U.urchin_build_bvh(d["px"], d["py"], d["pz"], d["h"], d["m"], False, 0.0, w.unit_cm)
    assert e.value.status == U.URCHIN_ERR_NONFINITE
    d = device_particles(w, torch)
    d["h"][3] = 0.0
    with pytest.raises(U.UrchinError) as e:
        U.urchin_build_bvh(d["px"], d["py"], d["pz"], d["h"], d["m"], False, 0.0, w.unit_cm)
    assert e.value.status == U.URCHIN_ERR_ARG


# --------------------------------------------------------------------------
# Gamma (Eq. gamma_shld) and equilibrium (App. C3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("R", [1, 12, 48])
@pytest.mark.parametrize("F", [1, 50, 200, 400])
@pytest.mark.parametrize("tau_max", [300.0, 3e4])
def test_gamma_random_columns(R, F, tau_max):
    rng = np.random.default_rng(R * 1000 + F)
    n = 777
    tau = np.exp(rng.uniform(np.log(1e-6), np.log(tau_max), (n, R))).astype(np.float32)
    tau[:5] = 0.0
    e, J = W.powerlaw_spectrum(F, 13.6, 54.4)
    s, wts = U.urchin_spectrum_weights(e, J, 1e-12)
    sg, wg = torch.from_numpy(s).cuda(), torch.from_numpy(wts).cuda()
    g_ref, te_ref = O.gamma(tau.astype(np.float64), s, wts)
    g32, te32 = U.urchin_gamma(torch.from_numpy(tau).cuda(), sg, wg)
    # identical FP32 columns on both sides: every bin's exponent is formed
    # without rounding, so the rate is within 2e-6 (the target is 1e-5) at
    # every tau; tau_eff = -ln(Gamma / Gamma_thin) within 2e-6 absolute plus
    # the rounding of the float32 output (an ulp, 1.2e-7 tau_eff)
    # (where exp(-s tau) underflows double both rates are 0)
    assert rel_err(g32.cpu().numpy(), g_ref, floor=1e-300).max() < 2e-6
    te32 = te32.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(te32 - te_ref) <= 2e-6 + 1.2e-7 * np.abs(te_ref))
    g64, te64 = U.urchin_gamma(torch.from_numpy(tau.astype(np.float64)).cuda(), sg, wg)
    assert rel_err(g64.cpu().numpy(), g_ref, floor=1e-300).max() < 1e-12
    assert np.all(g64.cpu().numpy()[:5] == pytest.approx(wts.sum(), rel=1e-14))


def test_gamma_deep_shielding_keeps_tau_eff_finite():
    # columns so large that Gamma underflows double: tau_eff still exact
    from scipy.special import logsumexp
    e, J = W.powerlaw_spectrum(100, 13.6, 54.4)
    s, wts = U.urchin_spectrum_weights(e, J, 1e-12)
    tau = np.array([[1e5] * 12, [1e3] * 6 + [1e6] * 6, [5e4] * 12])
    g, te = U.urchin_gamma(torch.from_numpy(tau).cuda(), torch.from_numpy(s).cuda(),
                           torch.from_numpy(wts).cuda())
    te = te.cpu().numpy()
    ref = np.array([-(logsumexp((np.log(wts / wts.sum())[None, :] - s[None, :] * t[:, None]).ravel())
                      - math.log(len(t))) for t in tau])
    assert np.all(np.isfinite(te))
    assert np.allclose(te, ref, rtol=1e-6)


@pytest.mark.parametrize("case_rule", [U.CASE_A, U.CASE_B, U.CASE_AUTO])
def test_equilibrium_matches_oracle(case_rule):
    rng = np.random.default_rng(case_rule + 40)
    n = 5000
    G = 10 ** rng.uniform(-22, -9, n)
    G[:7] = 0.0
    nH = 10 ** rng.uniform(-6, 2, n)
    T = 10 ** rng.uniform(3.5, 6.5, n)
    te = rng.uniform(0, 3, n).astype(np.float32)
    y = 0.05
    x = U.urchin_equilibrium(torch.from_numpy(G).cuda(), torch.from_numpy(te).cuda(),
                             torch.from_numpy(nH).cuda(), torch.from_numpy(T).cuda(), case_rule, y).cpu().numpy()
    caseB = np.full(n, case_rule == U.CASE_B) if case_rule != U.CASE_AUTO else te.astype(np.float64) >= 1
    ref = O.xeq(G, nH, T, y, caseB)
    assert rel_err(x, ref).max() < 1e-12


# --------------------------------------------------------------------------
# iteration driver (Sec. 4)
# --------------------------------------------------------------------------
def _solve_gpu(w, bvh, d, sw, precision, **kw):
    x, st = U.urchin_solve(bvh, U.urchin_healpix_dirs(w.nside), w.l_ray, sw[0], sw[1], d["nH"], d["T"],
                           precision=precision, raise_not_converged=False, **kw)
    return x.cpu().numpy(), st


@pytest.mark.parametrize("sweeps", [1, 2, 4])
def test_solve_lattice_fp64_step_matched(lattice, sweeps):
    w, bvh, d = lattice
    sg, so = spectra(w, torch)
    x, st = _solve_gpu(w, bvh, d, sg, U.F64, tol=1e-300, max_iter=sweeps)
    xr, fr, sr = O.solve(w, so[0], so[1], O.healpix(1), sweeps=sweeps)
    assert st["iterations"] == sweeps == sr["sweeps"]
    assert st["rays"] == sr["rays"]
    assert rel_err(x, xr).max() < 1e-9


def test_solve_lattice_fp64_converged(lattice):
    w, bvh, d = lattice
    sg, so = spectra(w, torch)
    x, st = _solve_gpu(w, bvh, d, sg, U.F64, tol=1e-3, max_iter=100)
    xr, fr, sr = O.solve(w, so[0], so[1], O.healpix(1), tol=1e-3, max_iter=100)
    assert st["converged"] and sr["converged"]
    assert st["iterations"] == sr["sweeps"]
    assert rel_err(x, xr).max() < 1e-9
    assert st["n_active"] == int((~fr).sum())


def _gpu_states(w, bvh, d, sg, sweeps, **kw):
    """x and the per-particle state (bit 0 case B latched, bit 1 frozen) after
    1..sweeps sweeps of the GPU solve (each a fresh, deterministic solve)."""
    out = []
    for k in range(1, sweeps + 1):
        state = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
        x, st = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-300, max_iter=k, state=state, **kw)
        assert st["iterations"] == k
        out.append((x, state.cpu().numpy()))
    return out


def _check_chain(w, so, states, org, nside=1, columns=None):
    """Every sweep of the chain against the oracle's update of the GPU's
    previous state (check_sweep's per-particle error model); sweep 0 from
    the oracle's x_thin."""
    x0 = O.xeq(so[1].sum(), w.nH, w.T, 0.0, False)
    worst = check_sweep(w, so, x0, None, states[0][0], org, nside, True, columns=columns)
    for (xp, sp), (xn, _) in zip(states[:-1], states[1:]):
        worst = max(worst, check_sweep(w, so, xp, sp, xn, org, nside, False, columns=columns))
    return worst


def test_solve_halo_small_fp32_step_matched(halo_small):
    """FP32 columns, FP64 equilibrium: sweeps 1-3, each checked at 4000
    seeded particles against the oracle's update of the GPU's previous state
    with the per-particle error model of check_sweep (no quantiles)."""
    w, bvh, d = halo_small
    sg, so = spectra(w, torch)
    states = _gpu_states(w, bvh, d, sg, 3)
    worst = _check_chain(w, so, states, W.random_origins(w.n, 4000, 31))
    assert worst <= 1.0
    _, st = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-300, max_iter=3)
    _, _, sr = O.solve(w, so[0], so[1], O.healpix(1), sweeps=3)
    assert st["rays"] == sr["rays"]


def test_solve_not_converged_and_bad_inputs(halo_small):
    w, bvh, d = halo_small
    sg, so = spectra(w, torch)
    with pytest.raises(U.UrchinError) as e:
        U.urchin_solve(bvh, U.urchin_healpix_dirs(1), w.l_ray, sg[0], sg[1], d["nH"], d["T"], tol=1e-12,
                       max_iter=2)
    assert e.value.status == U.URCHIN_ERR_NOT_CONVERGED
    bad = d["nH"].clone()
    bad[10] = -1.0
    with pytest.raises(U.UrchinError) as e:
        U.urchin_solve(bvh, U.urchin_healpix_dirs(1), w.l_ray, sg[0], sg[1], bad, d["T"])
    assert e.value.status == U.URCHIN_ERR_ARG


@pytest.mark.parametrize("segments", [U.SEG_RECOMPUTE, U.SEG_AUTO])
def test_solve_full_size_halo_one_sweep_sampled(segments):
    """Benchmark-size halo: sweeps 1-4 of the GPU at 256 seeded particles
    against the oracle's update of the GPU's previous state, per particle
    within check_sweep's error model.  With SEG_AUTO, sweep 0 traces every
    particle and keeps each ray's segment list (particle index, FP32 value)
    in linked chunks of 32 taken while tracing; sweeps 1-2 read their
    columns from the chunks and sweep 3 from the 7-byte rows (24-bit
    particle indices split into 16 + 8 bits) the chunks are copied into."""
    w = W.halo()
    bvh, d = build(w, torch)
    sg, so = spectra(w, torch)
    states = _gpu_states(w, bvh, d, sg, 4, segments=segments)
    _, st2 = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-300, max_iter=2, segments=segments)
    _, st4 = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-300, max_iter=4, segments=segments, profile=True)
    assert bool(st2["segments_stored"]) == bool(st4["segments_stored"]) == (segments == U.SEG_AUTO)
    assert st4["spmv_launches"] == (3 if segments == U.SEG_AUTO else 0)
    assert st4["trace_launches"] == (1 if segments == U.SEG_AUTO else 4)
    assert _check_chain(w, so, states, W.random_origins(w.n, 256, 10)) <= 1.0


# --------------------------------------------------------------------------
# stored segments and Newton-Krylov (same fixed point, same sweep semantics)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("sweeps", [1, 3])
def test_stored_segments_match_recompute_fp64(lattice, sweeps):
    w, bvh, d = lattice
    sg, so = spectra(w, torch)
    xr, sr = _solve_gpu(w, bvh, d, sg, U.F64, tol=1e-300, max_iter=sweeps)
    xs, ss = _solve_gpu(w, bvh, d, sg, U.F64, tol=1e-300, max_iter=sweeps, segments=U.SEG_STORE, profile=True)
    assert ss["segments_stored"] == 1 and sr["segments_stored"] == 0
    # the count and the fill pass each count every hit; each of the n R rays is
    # padded with fewer than 8 zero segments to a multiple of 8
    hits = ss["hits"] // 2
    assert ss["nnz"] % 8 == 0 and hits <= ss["nnz"] < hits + 8 * w.n * 12
    assert ss["iterations"] == sr["iterations"] == sweeps
    assert ss["rays"] == sr["rays"]
    assert rel_err(xs, xr).max() < 1e-11
    xo, fo, so_ = O.solve(w, so[0], so[1], O.healpix(1), sweeps=sweeps)
    assert rel_err(xs, xo).max() < 1e-9


def test_stored_segments_match_recompute_fp32(halo_small):
    """Four FP32 sweeps with stored segments: every sweep within
    check_sweep's error model of the oracle's update of the GPU's previous
    state, like the recomputed columns (test_solve_halo_small_fp32_step_matched)."""
    w, bvh, d = halo_small
    sg, so = spectra(w, torch)
    states = _gpu_states(w, bvh, d, sg, 4, segments=U.SEG_AUTO)
    _, ss = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-300, max_iter=4, segments=U.SEG_AUTO)
    assert ss["segments_stored"] == 1
    assert _check_chain(w, so, states, W.random_origins(w.n, 2000, 32)) <= 1.0


def test_newton_reaches_plain_fixed_point_lattice(lattice):
    w, bvh, d = lattice
    sg, so = spectra(w, torch)
    xp, sp = _solve_gpu(w, bvh, d, sg, U.F64, tol=1e-10, max_iter=300)
    xn, sn = _solve_gpu(w, bvh, d, sg, U.F64, tol=1e-10, max_iter=60, method=U.METHOD_NEWTON, gmres_m=20)
    assert sp["converged"] and sn["converged"]
    assert rel_err(xn, xp).max() < 1e-8
    xo, fo, st = O.solve(w, so[0], so[1], O.healpix(1), tol=1e-10, max_iter=300)
    assert rel_err(xn, xo).max() < 1e-8


@pytest.mark.parametrize("segments", [U.SEG_RECOMPUTE, U.SEG_STORE])
def test_newton_halo_small_fp32(halo_small, segments):
    """Plain sweeps then Newton-Krylov at the paper's dx_tol = 1e-3: converges
    in fewer evaluations than plain sweeps alone and lands closer to the
    fixed point (the step test stops plain sweeps early when they contract
    slowly)."""
    w, bvh, d = halo_small
    sg, so = spectra(w, torch)
    xt, st_ = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-6, max_iter=6000, segments=U.SEG_STORE)
    xp, sp = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-3, max_iter=3000, segments=U.SEG_STORE)
    xn, sn = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-3, max_iter=600, method=U.METHOD_NEWTON, gmres_m=20,
                        segments=segments)
    assert st_["converged"] and sp["converged"] and sn["converged"], (sp["iterations"], sn["iterations"])
    assert sn["newton_start"] > 0 and sn["iterations"] <= sp["iterations"]
    assert rel_err(xn, xt).max() <= rel_err(xp, xt).max()


def test_newton_full_halo_reaches_xstar_in_fewer_evaluations():
    """Benchmark-size halo: Newton-Krylov started once the sweeps are in
    their linear regime (at most 1 % of the particles moving by >= 1e-5),
    with GMRES(60) to relative residual 1e-4, converges quadratically and
    lands within rel 1e-5 of x* (plain sweeps to dx_tol 1e-6); plain sweeps
    need dx_tol 1e-5 and more evaluations to get within rel 1e-3 of x*."""
    w = W.halo()
    bvh, d = build(w, torch)
    sg, so = spectra(w, torch)
    xs, ss = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-6, max_iter=5000, segments=U.SEG_STORE)
    assert ss["converged"]
    xp, sp = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-5, max_iter=5000, segments=U.SEG_STORE)
    xn, sn = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-5, max_iter=1000, segments=U.SEG_STORE,
                        method=U.METHOD_NEWTON, gmres_m=60, newton_eta=1e-4, newton_switch=0.01)
    assert sp["converged"] and sn["converged"] and sn["newton_start"] > 0
    assert sn["iterations"] < sp["iterations"]
    assert rel_err(xn, xs).max() < 1e-4
    assert rel_err(xp, xs).max() < 1e-3


def test_memory_pool_keeps_and_trims(halo_small):
    """Work arrays come from a pool that keeps freed memory: a second solve
    reuses it (same result), and urchin_trim_memory returns it."""
    w, bvh, d = halo_small
    sg, so = spectra(w, torch)
    x1, s1 = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-300, max_iter=5, segments=U.SEG_STORE)
    torch.cuda.synchronize()
    held = U.urchin_trim_memory(-1)
    x2, s2 = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-300, max_iter=5, segments=U.SEG_STORE)
    torch.cuda.synchronize()
    assert held == 0 and s1["nnz"] == s2["nnz"] > 0
    np.testing.assert_allclose(x2, x1, rtol=1e-6, atol=0)
    assert U.urchin_trim_memory(torch.cuda.current_device()) == 0


def test_plain_solve_latched_case_matches_oracle(halo_small):
    """The latched case switch, step matched against the oracle on a halo
    where the unlatched rule would cycle."""
    w, bvh, d = halo_small
    sg, so = spectra(w, torch)
    x, st = _solve_gpu(w, bvh, d, sg, U.F64, tol=1e-300, max_iter=15, segments=U.SEG_STORE)
    xo, fo, so_ = O.solve(w, so[0], so[1], O.healpix(1), sweeps=15)
    assert rel_err(x, xo).max() < 1e-8


@pytest.mark.parametrize("blocks", [2, 8])
def test_density_ordered_blocks_match_oracle(halo_small, blocks):
    """The Sec. 4 high-to-low density update order, in blocks, step matched
    against the oracle (FP64, stored segments)."""
    w, bvh, d = halo_small
    sg, so = spectra(w, torch)
    x, st = _solve_gpu(w, bvh, d, sg, U.F64, tol=1e-300, max_iter=4, segments=U.SEG_STORE, blocks=blocks)
    xo, fo, so_ = O.solve(w, so[0], so[1], O.healpix(1), sweeps=4, blocks=blocks)
    assert st["iterations"] == 4 and st["rays"] == so_["rays"]
    assert rel_err(x, xo).max() < 1e-8


def test_density_ordered_blocks_converge_faster(halo_small):
    w, bvh, d = halo_small
    sg, so = spectra(w, torch)
    xj, sj = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-3, max_iter=3000, segments=U.SEG_STORE)
    xb, sb = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-3, max_iter=3000, segments=U.SEG_STORE, blocks=32)
    assert sj["converged"] and sb["converged"]
    assert sb["iterations"] < sj["iterations"]


# --------------------------------------------------------------------------
# tangent of the sweep map (what Newton-Krylov linearises)
# --------------------------------------------------------------------------
def _oracle_lnE(w, so, x, case_rule):
    g, te = O.gamma(O.columns(w, x, O.healpix(w.nside)), so[0], so[1])
    cb = np.full(w.n, case_rule == U.CASE_B)
    return np.log(O.xeq(g, w.nH, w.T, 0.0, cb))


@pytest.mark.parametrize("case_rule", [U.CASE_A, U.CASE_B])
def test_tangent_matches_finite_differences_fp64(lattice, case_rule):
    """d ln E / d ln x . v from the library against central differences of the
    library's own sweep map and of the FP64 oracle's (step 1e-4 in ln x)."""
    w, bvh, d = lattice
    sg, so = spectra(w, torch)
    dirs = U.urchin_healpix_dirs(1)
    # a partly shielded state: x_thin scaled by factors 0.5-2 (the lattice
    # turns fully neutral within two sweeps, where every derivative vanishes)
    rng = np.random.default_rng(31)
    x = O.xeq(so[1].sum(), w.nH, w.T, 0.0, case_rule == U.CASE_B) * rng.uniform(0.5, 2.0, w.n)
    v = rng.uniform(-1, 1, w.n)
    eps = 1e-4
    tg = lambda xx: U.urchin_tangent(bvh, dirs, w.l_ray, sg[0], sg[1], d["nH"], d["T"],
                                     torch.from_numpy(xx).cuda(), torch.from_numpy(v).cuda(),
                                     precision=U.F64, case_rule=case_rule)
    E0, dl = tg(x)
    dl = dl.cpu().numpy()
    Ep, _ = tg(x * np.exp(eps * v))
    Em, _ = tg(x * np.exp(-eps * v))
    fd = (np.log(Ep.cpu().numpy()) - np.log(Em.cpu().numpy())) / (2 * eps)
    scale = np.abs(fd).max()
    assert scale > 1e-3
    assert np.all(np.abs(dl - fd) <= 1e-6 * scale)
    fdo = (_oracle_lnE(w, so, x * np.exp(eps * v), case_rule) - _oracle_lnE(w, so, x * np.exp(-eps * v), case_rule)) / (2 * eps)
    assert np.all(np.abs(dl - fdo) <= 1e-6 * scale)
    xe = O.xeq(O.gamma(O.columns(w, x, O.healpix(1)), so[0], so[1])[0], w.nH, w.T, 0.0,
               np.full(w.n, case_rule == U.CASE_B))
    assert rel_err(E0.cpu().numpy(), xe).max() < 1e-9


def test_tangent_fp32_halo(halo_small):
    """The tangent d ln E / d ln x . v of one sweep (E the sweep's update),
    particle by particle, without quantiles.
    FP64: against central differences of the FP64 map, with the truncation
    error estimated by halving the step (|dl - fd(h/2)| ~ |fd(h) - fd(h/2)|/3).
    FP32 (columns of x and of x v in FP32, FP32 fold) against FP64 at 400
    seeded particles, within a first-order error model.  With
    dl = c sum_k g_k dtau_k (c = d ln x / d ln Gamma, g_k = d ln Gamma /
    d tau_k, dtau the column of x v), relative column errors <= eps_col in
    tau and errors <= eps_col tau_k(|x v|) in dtau move dl by at most
      eps_col sum_k |g_k| (|c| tau_k(|x v|) + |dtau_k| (|c| (s_max tau_k + D) + D))
    (g_k changes by s_max tau_k eps_col relative through its exponentials and
    by D eps_col through Gamma, D = sum_k tau_k |g_k|; c by at most D eps_col),
    and the FP32 fold adds eps_fold (|c| + 1) sum_k |g_k| |dtau_k|."""
    w, bvh, d = halo_small
    sg, so = spectra(w, torch)
    dirs = U.urchin_healpix_dirs(1)
    x, _ = _solve_gpu(w, bvh, d, sg, U.F32, tol=1e-300, max_iter=20, case_rule=U.CASE_A, segments=U.SEG_STORE)
    x = np.minimum(x, 0.9)           # keep x e^(eps v) inside (0, 1]
    rng = np.random.default_rng(32)
    v = rng.uniform(-1, 1, w.n)
    h = 1e-3
    tg = lambda xx, p=U.F64: U.urchin_tangent(bvh, dirs, w.l_ray, sg[0], sg[1], d["nH"], d["T"],
                                              torch.from_numpy(xx).cuda(), torch.from_numpy(v).cuda(),
                                              precision=p, case_rule=U.CASE_A)
    _, dl64 = tg(x)
    _, dl32 = tg(x, U.F32)
    dl64, dl32 = dl64.cpu().numpy(), dl32.cpu().numpy()
    lnE = lambda e: np.log(tg(x * np.exp(e * v))[0].cpu().numpy())
    fd1 = (lnE(h) - lnE(-h)) / (2 * h)
    fd2 = (lnE(h / 2) - lnE(-h / 2)) / h
    scale = np.abs(fd2).max()
    assert np.all(np.abs(dl64 - fd2) <= 1e-9 * scale + np.abs(fd1 - fd2))
    # FP32 against FP64 at seeded particles, with the oracle's columns and partials
    org = W.random_origins(w.n, 400, 33)
    od = O.healpix(1)
    tau = O.columns(w, x, od, origins=org)
    dtau = O.columns(w, x * np.maximum(v, 0), od, origins=org) - O.columns(w, x * np.maximum(-v, 0), od, origins=org)
    tabs = O.columns(w, x * np.abs(v), od, origins=org)
    G, _ = O.gamma(tau, so[0], so[1])
    # g_k = |dGamma/dtau_k| / Gamma from the oracle's partials, in log-sum-exp
    # form where Gamma underflows (fully shielded particles, whose c is 0)
    from scipy.special import logsumexp
    sb, wb = np.asarray(so[0], dtype=np.float64), np.asarray(so[1], dtype=np.float64)
    e = -tau[:, :, None] * sb[None, None, :]
    with np.errstate(divide="ignore"):
        g = np.exp(logsumexp(e + np.log(wb * sb)[None, None, :], axis=2)
                   - logsumexp((e + np.log(wb)[None, None, :]).reshape(len(org), -1), axis=1)[:, None])
    dG, _ = O.gamma_partials(tau[:4], so[0], so[1])
    assert np.allclose(g[:4] * G[:4, None], np.abs(dG), rtol=1e-12, atol=0)
    c = np.abs(G * O.xeq_dgamma(G, w.nH[org], w.T[org], 0.0, False) / O.xeq(G, w.nH[org], w.T[org], 0.0, False))
    D = (tau * g).sum(axis=1)
    smax = float(np.max(so[0]))
    eps_col, eps_fold = 1e-6, 2e-6
    bound = (eps_col * (g * (c[:, None] * tabs + np.abs(dtau) * (c[:, None] * (smax * tau + D[:, None])
                                                                   + D[:, None]))).sum(axis=1)
             + eps_fold * (c + 1) * (g * np.abs(dtau)).sum(axis=1) + 1e-12 * scale)
    err = np.abs(dl32[org] - dl64[org])
    assert np.all(err <= bound), (float(np.max(err / bound)), int(org[np.argmax(err / bound)]))
