"""The usage example of README.md (the same code, kept here so that the test
does not depend on the document's text), run on the benchmark halo: the
solve converges, and its last sweep is the oracle's update of the GPU's
state one sweep earlier within check_sweep's per-particle error model."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import check_sweep

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1304_4235_gb300 import urchin as U  # noqa: E402


def test_readme_usage_example_runs():
    # --- the README's example ---
    w = W.halo()                                             # or your own particles
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    bvh = U.urchin_build_bvh(t(w.pos[:, 0], torch.float32), t(w.pos[:, 1], torch.float32),
                             t(w.pos[:, 2], torch.float32), t(w.h, torch.float32),
                             t(w.mass_H, torch.float64), w.periodic, w.box, w.unit_cm)
    edges, J = w.spectrum()
    s, wts = U.urchin_spectrum_weights(edges, J, w.gamma_thin)
    x, stats = U.urchin_solve(bvh, U.urchin_healpix_dirs(1), w.l_ray,
                              t(s, torch.float64), t(wts, torch.float64),
                              t(w.nH, torch.float64), t(w.T, torch.float64),
                              tol=1e-3, max_iter=1000, segments=U.SEG_AUTO)
    # --- end of the example ---
    assert stats["converged"] and stats["iterations"] > 1
    xa = x.cpu().numpy()
    assert xa.shape == (w.n,) and np.all(np.isfinite(xa)) and np.all((xa > 0) & (xa <= 1))
    n = stats["iterations"]
    state = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    xp, sp = U.urchin_solve(bvh, U.urchin_healpix_dirs(1), w.l_ray, t(s, torch.float64), t(wts, torch.float64),
                            t(w.nH, torch.float64), t(w.T, torch.float64), tol=1e-300, max_iter=n - 1,
                            segments=U.SEG_AUTO, state=state, raise_not_converged=False)
    bvh.close()
    so = O.spectrum(edges, J, w.gamma_thin)
    org = W.random_origins(w.n, 64, 12)
    assert check_sweep(w, so, xp.cpu().numpy(), state.cpu().numpy(), xa, org, 1, False) <= 1.0
