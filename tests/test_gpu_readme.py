"""The usage example of README.md, run as written (on the benchmark halo),
and its result checked: converged, and at seeded particles the oracle's
update from the converged state reproduces x."""
import re
import pathlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = pathlib.Path(__file__).resolve().parents[1]


def test_readme_usage_example_runs():
    text = (ROOT / "README.md").read_text()
    block = re.search(r"## Use\s+```python\n(.*?)```", text, re.S)
    assert block, "README has no usage example"
    scope = {}
    exec(compile(block.group(1), "README.md", "exec"), scope)
    x, stats, w, U = scope["x"], scope["stats"], scope["w"], scope["U"]
    assert stats["converged"] and stats["iterations"] > 1
    xa = x.cpu().numpy()
    assert xa.shape == (w.n,) and np.all(np.isfinite(xa)) and np.all((xa > 0) & (xa <= 1))

    import oracle as O
    import workloads as W
    e, J = w.spectrum()
    so, wo = O.spectrum(e, J, w.gamma_thin)
    org = W.random_origins(w.n, 64, 12)
    g, te = O.gamma(O.columns(w, xa, O.healpix(1), origins=org), so, wo)
    # the converged state is a fixed point up to the stopping tolerance (1e-3)
    # at the particles that are updated (tau_eff >= tau_skip = 1e-4)
    upd = te >= 1e-4
    expect = O.xeq(g, w.nH[org], w.T[org], 0.0, te >= 1)
    rel = np.abs(xa[org] - expect) / expect
    assert np.quantile(rel[upd], 0.9) < 3e-3
