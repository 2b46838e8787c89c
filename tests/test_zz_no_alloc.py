"""urchin_trace_columns_noalloc, the entry point for callers that cannot
allocate device memory (for example code whose framework allocator owns the
whole memory pool, or services that forbid allocation on the hot path).  With
a preallocated output, two calls in a row (the second reusing the fixed work
array the first left behind) must change neither the device's free memory
nor torch's allocated bytes, give columns bit-equal to the allocating
urchin_trace_columns (a ray sums its hits in the tree's fixed depth-first
order in both), match the FP64 oracle at sampled origins, and refuse
requests larger than the fixed array.

This file is collected last so that a run stopping at the first failure has
already run every other test; it passes alone in a fresh process too (the
first call, which looks up the array's address and loads the kernels, is
made before the memory is measured)."""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1304_4235_gb300 import urchin as U  # noqa: E402


def _bvh(w):
    pos = np.asarray(w.pos, dtype=np.float32)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    return U.urchin_build_bvh(t(pos[:, 0], np.float32), t(pos[:, 1], np.float32), t(pos[:, 2], np.float32),
                              t(w.h, np.float32), t(w.mass_H, np.float64), w.periodic, w.box, w.unit_cm)


@pytest.mark.parametrize("precision,tol", [(U.F32, 1e-5), (U.F64, 1e-11)])
def test_noalloc_allocates_nothing_and_matches_twice(precision, tol):
    w = W.halo(n=20000, seed=2024)
    bvh = _bvh(w)
    dirs = U.urchin_healpix_dirs(1)
    R = dirs.shape[0]
    rng = np.random.default_rng(3)
    dt = torch.float64 if precision == U.F64 else torch.float32
    # first call: all origins; second call: a subset in arbitrary order and other x
    x1h = np.exp(rng.uniform(np.log(1e-4), 0.0, w.n))
    x2h = np.exp(rng.uniform(np.log(1e-3), 0.0, w.n))
    orgh = rng.choice(w.n, 3000, replace=False).astype(np.int32)
    x1, x2 = torch.from_numpy(x1h).cuda(), torch.from_numpy(x2h).cuda()
    org = torch.from_numpy(orgh).cuda()
    out1 = torch.empty((w.n, R), dtype=dt, device="cuda")
    out2 = torch.empty((orgh.size, R), dtype=dt, device="cuda")
    # set-up call (address lookup, kernel loading), then measure
    U.urchin_trace_columns_noalloc(bvh, x1, dirs, w.l_ray, precision=precision, out=out1)
    torch.cuda.synchronize()
    U.urchin_trim_memory(-1)
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    U.urchin_trace_columns_noalloc(bvh, x1, dirs, w.l_ray, precision=precision, out=out1)
    U.urchin_trace_columns_noalloc(bvh, x2, dirs, w.l_ray, origins=org, precision=precision, out=out2)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    for x, o, got in ((x1, None, out1), (x2, org, out2)):
        ref = U.urchin_trace_columns(bvh, x, dirs, w.l_ray, origins=o, precision=precision)
        assert torch.equal(got, ref)
    # and against the oracle at seeded origins of the second call
    pick = np.sort(rng.choice(orgh.size, 64, replace=False))
    oref = O.columns(w, x2h, O.healpix(1), origins=orgh[pick])
    a = out2.double().cpu().numpy()[pick]
    assert np.all(np.abs(a - oref) <= tol * np.abs(oref))
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
    assert torch.equal(out, ref)
    bvh.close()
