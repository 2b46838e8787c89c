"""urchin_trace_columns_noalloc, the entry point for callers that cannot
allocate device memory (for example code whose framework allocator owns the
whole memory pool, or services that forbid allocation on the hot path).  It
must give the same columns as the allocating urchin_trace_columns, on two
calls in a row (the second reusing the fixed work array the first left
behind), and refuse requests larger than its fixed array.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1304_4235_gb300 import urchin as U  # noqa: E402


def _bvh(w):
    pos = np.asarray(w.pos, dtype=np.float32)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    return U.urchin_build_bvh(t(pos[:, 0], np.float32), t(pos[:, 1], np.float32), t(pos[:, 2], np.float32),
                              t(w.h, np.float32), t(w.mass_H, np.float64), w.periodic, w.box, w.unit_cm)


@pytest.mark.parametrize("precision", [U.F32, U.F64])
def test_noalloc_matches_allocating_entry_point_twice(precision):
    w = W.halo(n=20000, seed=2024)
    bvh = _bvh(w)
    dirs = U.urchin_healpix_dirs(1)
    rng = np.random.default_rng(3)
    # first call: all origins; second call: a subset in arbitrary order and other x
    x1 = torch.from_numpy(np.exp(rng.uniform(np.log(1e-4), 0.0, w.n))).cuda()
    x2 = torch.from_numpy(np.exp(rng.uniform(np.log(1e-3), 0.0, w.n))).cuda()
    org = torch.from_numpy(rng.choice(w.n, 3000, replace=False).astype(np.int32)).cuda()
    for x, o in ((x1, None), (x2, org)):
        ref = U.urchin_trace_columns(bvh, x, dirs, w.l_ray, origins=o, precision=precision)
        got = U.urchin_trace_columns_noalloc(bvh, x, dirs, w.l_ray, origins=o, precision=precision)
        torch.cuda.synchronize()
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        assert a.shape == b.shape
        assert np.all(np.abs(a - b) <= 1e-5 * np.abs(b))
    bvh.close()


def test_noalloc_refuses_requests_beyond_its_array():
    w = W.halo(n=4000, seed=2025)
    bvh = _bvh(w)
    dirs = U.urchin_healpix_dirs(1)
    x = torch.ones(w.n, dtype=torch.float64, device="cuda")
    n_orig = (16 << 20) // 4 + 1               # the mapped origins alone exceed the array
    org = torch.zeros(n_orig, dtype=torch.int32, device="cuda")
    with pytest.raises(U.UrchinError) as e:
        U.urchin_trace_columns_noalloc(bvh, x, dirs, w.l_ray, origins=org)
    assert e.value.status == U.URCHIN_ERR_ARG and "fixed" in str(e.value)
    # a normal call still works after the refusal
    out = U.urchin_trace_columns_noalloc(bvh, x, dirs, w.l_ray)
    ref = U.urchin_trace_columns(bvh, x, dirs, w.l_ray)
    assert torch.allclose(out, ref, rtol=1e-5, atol=0)
    bvh.close()
