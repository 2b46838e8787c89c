"""The paper's Test 2 in miniature: plane-parallel radiation onto uniform
isothermal SPH slabs (200 kpc, 16 lattice layers), one ray per particle
toward the lit surface, the near/far split with the numerical slab for the
binned spectrum, against the slice-by-slice slab solver NS of Test 1.  The
densities put the slab's neutral column from 10^17.8 to 10^20.3 cm^-2 (the
range where self-shielding sets in); the paper finds the SPH column within
0.05-0.1 dex of NS.  A power-law spectrum (nu^-1.5, 1-4 Ryd) stands in for
the HM01 background."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import build, spectra

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1304_4235_gb300 import urchin as U  # noqa: E402

DENSITIES = (1.0e-3, 1.1e-3, 1.2e-3, 1.3e-3, 1.4e-3)


def _columns(nH, near_far, two_sided=False):
    w = W.slab(nH=nH)
    bvh, d = build(w, torch)
    sg, so = spectra(w, torch)
    dirs = np.array([[0.0, 0.0, -1.0], [0.0, 0.0, 1.0]]) if two_sided else np.array([[0.0, 0.0, -1.0]])
    x, st = U.urchin_solve(bvh, dirs, w.l_ray, sg[0], sg[1], d["nH"], d["T"], tol=1e-6, max_iter=3000,
                           precision=U.F32, case_rule=U.CASE_A, near_far=near_far, segments=U.SEG_STORE)
    assert st["converged"]
    area = (w.box * w.unit_cm) ** 2
    sph = float((w.mass_H * x.cpu().numpy()).sum() / area)
    sth = O.sigma_th()
    if two_sided:
        _, t = O.ns_slab2(so[0], so[1], nH, 1e4, False, sth * nH * w.l_ray * w.unit_cm, 8000)
    else:
        _, t = O.ns_slab(so[0], so[1], nH, 1e4, False, sth * nH * w.l_ray * w.unit_cm, 40000)
    return np.log10(sph), np.log10(t / sth), st["iterations"]


def test_sph_slab_columns_match_the_slab_solver():
    """One-sided (Test 2): within 0.05 dex of NS with the numerical slab; the
    plain scheme, whose particles shield themselves through their
    neighbours, is printed beside it."""
    errs = []
    for nH in DENSITIES:
        ls, ln, it = _columns(nH, U.SLAB_SPECTRUM)
        lp, _, itp = _columns(nH, 0)
        errs.append(ls - ln)
        print(f"nH {nH:.2e}: log N_HI NS {ln:.3f} near/far {ls:.3f} ({it} sweeps) plain {lp:.3f} ({itp} sweeps)")
    assert np.max(np.abs(errs)) < 0.05, errs


def test_sph_slab_two_sided():
    """Two-sided (Test 3), two rays per particle: the slab of near particles
    sees one side at a time, so the intermediate columns carry the larger
    errors the paper reports (up to ~0.25 dex)."""
    errs = []
    for nH in DENSITIES + (1.6e-3,):
        ls, ln, it = _columns(nH, U.SLAB_SPECTRUM, two_sided=True)
        errs.append(ls - ln)
        print(f"two-sided nH {nH:.2e}: log N_HI NS {ln:.3f} near/far {ls:.3f} ({it} sweeps)")
    assert np.max(np.abs(errs)) < 0.3, errs
