"""Seeded input generators: determinism and the stated shapes (CPU)."""
import numpy as np

import workloads as W


def test_lattice_box_shape_and_determinism():
    a = W.lattice_box()
    b = W.lattice_box()
    assert a.n == 4096 and a.pos.dtype == np.float32 and a.h.dtype == np.float32
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.h, b.h)
    assert a.periodic and a.box == 1000.0 and a.l_ray == 500.0 and a.F == 50
    assert np.all((a.pos >= 0) & (a.pos < a.box))
    # h from 32 neighbours on a 62.5 kpc lattice: ~ (3*33/(4 pi))^(1/3) * 62.5 kpc
    assert 110 < float(np.median(a.h)) < 140


def test_halo_density_law():
    w = W.halo(n=20000, seed=1)
    r = np.linalg.norm(w.pos.astype(np.float64), axis=1)
    assert r.min() >= 1.0 - 1e-5 and r.max() <= 100.0 + 1e-4
    # enclosed mass linear in r for n_H ~ r^-2
    hist, _ = np.histogram(r, bins=10, range=(1, 100))
    assert hist.min() > 0.85 * hist.mean()
    assert np.allclose(w.nH, 10.0 * r ** -2)
    assert not w.periodic and w.l_ray == 200.0 and w.F == 100


def test_lognormal_box_small():
    w = W.lognormal_box(n_side=16, box_kpc=500.0)
    assert w.n == 16 ** 3 and w.periodic
    # total hydrogen = mean n_H x volume; particles sit preferentially in dense cells
    assert np.isclose(w.mass_H.sum(), 1e-5 * (w.box * w.unit_cm) ** 3, rtol=1e-12)
    assert np.mean(w.nH) > 1e-5
    assert np.all(w.T > 0)


def test_spectrum_samples():
    edges, J = W.powerlaw_spectrum(50, 13.6, 54.4, 1.5)
    assert edges.shape == (51,) and J.shape == (50,)
    assert np.isclose(edges[0], 13.6) and np.isclose(edges[-1], 54.4)
    assert np.all(np.diff(J) < 0)
