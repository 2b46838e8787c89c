"""Seeded synthetic inputs for the reverse ray tracer.

This module builds the *inputs* of the method only: SPH particle sets
(positions, smoothing lengths, hydrogen masses, densities, temperatures) and
the sampled UV-background spectrum J_nu.  It holds none of the method's
arithmetic (no kernels, columns, cross sections, rates or ionisation
equilibrium), so the FP64 oracle and the CUDA library can both consume it
without sharing any of the computation they are compared on.

Workloads (all seeds are ``1304 + index``):

* ``lattice_box``   -- 16^3 jittered lattice in a periodic 1 Mpc box, uniform
  n_H = 1.5e-3 cm^-3, T = 1e4 K, h from 32 neighbours (uniform-gas tests of
  Sec. 5 use n_H = 1.5e-3 cm^-3, 500x the z=3 mean).
* ``halo``          -- 262144 particles sampling n_H = 10 (r/kpc)^-2 cm^-3 on
  r = 1..100 kpc, isotropic, T = 1e4 K, h from 48 neighbours (stand-in for the
  OWLS halo stacks of Sec. 5.4, which are not available).
* ``lognormal_box`` -- particles sampling a log-normal density field built
  from a Gaussian random field with P(k) ~ k^-2.5, periodic box, T ~ rho^0.6.

Units: positions and smoothing lengths in kpc (float32, the precision the
GPU consumes; both sides read the same float32 values), masses as the number
of hydrogen atoms m_i/m_p (float64), n_H in cm^-3, T in K.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

KPC_CM = 3.0856775814913673e21  # cm per kpc (IAU 2015 parsec x 1e3)


@dataclasses.dataclass
class Workload:
    name: str
    pos: np.ndarray        # float32 [n, 3], kpc
    h: np.ndarray          # float32 [n], kpc (kernel support radius)
    mass_H: np.ndarray     # float64 [n], hydrogen atoms per particle
    nH: np.ndarray         # float64 [n], cm^-3 (field value at the particle)
    T: np.ndarray          # float64 [n], K
    periodic: bool
    box: float             # kpc (box side if periodic, else 0)
    unit_cm: float         # cm per length unit
    nside: int             # HEALPix N_side of the ray set
    l_ray: float           # kpc
    F: int                 # frequency bins
    e_lo: float            # eV
    e_hi: float            # eV
    gamma_thin: float      # s^-1
    seed: int

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def R(self) -> int:
        return 12 * self.nside * self.nside

    def spectrum(self):
        return powerlaw_spectrum(self.F, self.e_lo, self.e_hi, alpha=1.5)


def smoothing_lengths(pos: np.ndarray, n_ngb: int, box: float | None) -> np.ndarray:
    """Distance to the n_ngb-th nearest *other* particle (periodic minimum
    image when ``box`` is given), computed in float64 from the float32
    positions and rounded to float32."""
    from scipy.spatial import cKDTree

    p = pos.astype(np.float64)
    if box:
        p = np.mod(p, box)
        tree = cKDTree(p, boxsize=box)
    else:
        tree = cKDTree(p)
    # only the (n_ngb + 1)-th nearest (the particle itself is the first)
    d, _ = tree.query(p, k=[n_ngb + 1], workers=-1)
    return d[:, 0].astype(np.float32)


def powerlaw_spectrum(F: int, e_lo: float, e_hi: float, alpha: float = 1.5):
    """F log-spaced bins between e_lo and e_hi (eV).  Returns the F+1 bin
    edges and J_nu ~ nu^-alpha sampled at the geometric bin centres (arbitrary
    amplitude: the solver normalises the spectrum to Gamma_thin)."""
    edges = np.exp(np.linspace(math.log(e_lo), math.log(e_hi), F + 1))
    centres = np.sqrt(edges[:-1] * edges[1:])
    J = (centres / e_lo) ** (-alpha)
    return edges, J


def lattice_box(n_side: int = 16, box_kpc: float = 1000.0, jitter: float = 0.1,
                nH: float = 1.5e-3, T: float = 1.0e4, n_ngb: int = 32,
                seed: int = 1304, nside: int = 1, l_ray: float | None = None,
                F: int = 50) -> Workload:
    rng = np.random.default_rng(seed)
    dx = box_kpc / n_side
    g = (np.arange(n_side) + 0.5) * dx
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    p = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    p += rng.uniform(-jitter * dx, jitter * dx, size=p.shape)
    p = np.mod(p, box_kpc).astype(np.float32)
    p[p >= np.float32(box_kpc)] = 0.0
    n = p.shape[0]
    h = smoothing_lengths(p, n_ngb, box_kpc)
    vol_cm3 = (box_kpc * KPC_CM) ** 3
    mass = np.full(n, nH * vol_cm3 / n, dtype=np.float64)
    return Workload("lattice_box", p, h, mass, np.full(n, nH), np.full(n, T),
                    True, box_kpc, KPC_CM, nside,
                    0.5 * box_kpc if l_ray is None else l_ray, F, 13.6, 54.4,
                    1.0e-12, seed)


def halo(n: int = 262144, r_min: float = 1.0, r_max: float = 100.0,
         n0: float = 10.0, T: float = 1.0e4, n_ngb: int = 48, seed: int = 1305,
         nside: int = 1, l_ray: float = 200.0, F: int = 100) -> Workload:
    """n_H = n0 (r/kpc)^-2: the enclosed mass grows linearly in r, so the
    radial inverse CDF is r = r_min + (r_max - r_min) u."""
    rng = np.random.default_rng(seed)
    u = rng.random(n)
    r = r_min + (r_max - r_min) * u
    cth = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sth = np.sqrt(1.0 - cth * cth)
    p = np.stack([r * sth * np.cos(phi), r * sth * np.sin(phi), r * cth], axis=1)
    p = p.astype(np.float32)
    h = smoothing_lengths(p, n_ngb, None)
    total_atoms = n0 * 4.0 * math.pi * (r_max - r_min) * KPC_CM ** 3
    mass = np.full(n, total_atoms / n, dtype=np.float64)
    rr = np.linalg.norm(p.astype(np.float64), axis=1)
    nH = n0 * rr ** -2
    return Workload("halo", p, h, mass, nH, np.full(n, T), False, 0.0, KPC_CM,
                    nside, l_ray, F, 13.6, 54.4, 1.0e-12, seed)


def gaussian_random_field(ng: int, slope: float, rng) -> np.ndarray:
    """Zero-mean unit-variance GRF on an ng^3 periodic grid with P(k) ~ k^slope."""
    kf = np.fft.fftfreq(ng) * ng
    kz = np.fft.rfftfreq(ng) * ng
    KX, KY, KZ = np.meshgrid(kf, kf, kz, indexing="ij")
    k = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = k[nz] ** (0.5 * slope)
    noise = rng.standard_normal((ng, ng, ng))
    field = np.fft.irfftn(np.fft.rfftn(noise) * amp, s=(ng, ng, ng), axes=(0, 1, 2))
    field -= field.mean()
    return field / field.std()


def lognormal_box(n_side: int = 128, box_kpc: float = 4000.0, sigma_ln: float = 2.0,
                  mean_nH: float = 1.0e-5, T0: float = 1.0e4, n_ngb: int = 32,
                  seed: int = 1306, nside: int = 2, l_ray: float = 100.0,
                  F: int = 200, e_hi: float = 54.4) -> Workload:
    """Cell-multinomial sampling of rho ~ exp(delta - sigma^2/2) with uniform
    positions inside each cell; T = T0 (rho/rho_mean)^0.6 of the cell."""
    rng = np.random.default_rng(seed)
    ng = n_side
    delta = sigma_ln * gaussian_random_field(ng, -2.5, rng)
    rho = np.exp(delta - 0.5 * sigma_ln ** 2)
    rho /= rho.mean()
    n = ng ** 3
    prob = (rho / rho.sum()).ravel()
    counts = rng.multinomial(n, prob)
    cell = np.repeat(np.arange(ng ** 3), counts)
    ci = np.stack(np.unravel_index(cell, (ng, ng, ng)), axis=1).astype(np.float64)
    dx = box_kpc / ng
    p = (ci + rng.random((n, 3))) * dx
    p = np.mod(p, box_kpc).astype(np.float32)
    p[p >= np.float32(box_kpc)] = 0.0
    h = smoothing_lengths(p, n_ngb, box_kpc)
    vol_cm3 = (box_kpc * KPC_CM) ** 3
    mass = np.full(n, mean_nH * vol_cm3 / n, dtype=np.float64)
    rc = rho.ravel()[cell]
    return Workload("lognormal_box", p, h, mass, mean_nH * rc, T0 * rc ** 0.6,
                    True, box_kpc, KPC_CM, nside, l_ray, F, 13.6, e_hi,
                    1.0e-12, seed)


def slab(n_z: int = 16, slab_kpc: float = 200.0, nH: float = 1.2e-3, T: float = 1.0e4, jitter: float = 0.1,
         n_ngb: int = 32, seed: int = 1307, F: int = 50, box_factor: int = 3) -> Workload:
    """Uniform isothermal slab z in [0, slab_kpc] (the SPH slabs of the
    paper's Tests 2-3): a jittered lattice of spacing slab_kpc / n_z, laterally
    periodic in a cubic box of side box_factor * slab_kpc (the rest of the box
    is empty, so a ray of length slab_kpc never wraps back into the slab).
    One ray per particle toward the lit surface z = 0 is the caller's choice
    of directions."""
    rng = np.random.default_rng(seed)
    d = slab_kpc / n_z
    box = box_factor * slab_kpc
    nxy = box_factor * n_z
    gx = (np.arange(nxy) + 0.5) * d
    gz = (np.arange(n_z) + 0.5) * d
    X, Y, Z = np.meshgrid(gx, gx, gz, indexing="ij")
    p = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    p += rng.uniform(-jitter * d, jitter * d, size=p.shape)
    p[:, :2] = np.mod(p[:, :2], box)
    p = p.astype(np.float32)
    p[p >= np.float32(box)] = 0.0
    n = p.shape[0]
    h = smoothing_lengths(p, n_ngb, box)
    vol_cm3 = (box * KPC_CM) ** 2 * (slab_kpc * KPC_CM)
    mass = np.full(n, nH * vol_cm3 / n, dtype=np.float64)
    return Workload("slab", p, h, mass, np.full(n, nH), np.full(n, T), True, box, KPC_CM, 1, slab_kpc, F,
                    13.6, 54.4, 1.0e-12, seed)


def subset(w: Workload, idx: np.ndarray, name: str | None = None) -> Workload:
    """Particles ``idx`` of a workload (e.g. a small isolated cut-out)."""
    return dataclasses.replace(
        w, name=name or (w.name + "_subset"), pos=w.pos[idx].copy(),
        h=w.h[idx].copy(), mass_H=w.mass_H[idx].copy(), nH=w.nH[idx].copy(),
        T=w.T[idx].copy())


def helium_fractions(w: Workload, seed: int):
    """Fixed He I and He II abundances per H atom for every particle (the
    paper iterates hydrogen only): n_He/n_H = 0.079 (X = 0.76) times seeded
    ion fractions, He I in [0, 0.3) and He II in [0, 0.5) of the rest."""
    rng = np.random.default_rng(seed)
    y = 0.079
    f1 = rng.uniform(0.0, 0.3, w.n)
    f2 = rng.uniform(0.0, 0.5, w.n) * (1 - f1)
    return y * f1, y * f2


def hei_cross_section_standin(edges: np.ndarray) -> np.ndarray:
    """A He I cross-section shape in units of sigma_th at the geometric bin
    centres, zero below the 24.59 eV edge and 1.2 (24.59 eV / E)^2 above it.
    The paper gives no He I fit; this stand-in only has to be the same input
    on every side that uses it."""
    centres = np.sqrt(edges[:-1] * edges[1:])
    return np.where(centres >= 24.59, 1.2 * (24.59 / centres) ** 2, 0.0)


def random_origins(n: int, count: int, seed: int) -> np.ndarray:
    """A seeded sample of ``count`` distinct particle indices (sorted)."""
    rng = np.random.default_rng(seed)
    count = min(count, n)
    return np.sort(rng.choice(n, size=count, replace=False)).astype(np.int32)


def cached(fn, cache_dir: str, **kw) -> Workload:
    """fn(**kw), stored under cache_dir as .npy arrays plus the scalar fields
    and reloaded on later calls with the same name and arguments (the
    generation of the largest boxes takes tens of seconds; the arrays are
    the same seeded values either way)."""
    import json
    import os
    key = fn.__name__ + "".join(f"_{k}{kw[k]}" for k in sorted(kw))
    d = os.path.join(cache_dir, key)
    arrays = ("pos", "h", "mass_H", "nH", "T")
    meta_path = os.path.join(d, "meta.json")
    if os.path.exists(meta_path):
        meta = json.load(open(meta_path))
        return Workload(**meta, **{a: np.load(os.path.join(d, a + ".npy")) for a in arrays})
    w = fn(**kw)
    tmp = d + f".tmp{os.getpid()}"
    os.makedirs(tmp, exist_ok=True)
    for a in arrays:
        np.save(os.path.join(tmp, a + ".npy"), getattr(w, a))
    meta = {f.name: getattr(w, f.name) for f in dataclasses.fields(w) if f.name not in arrays}
    json.dump(meta, open(os.path.join(tmp, "meta.json"), "w"))
    try:
        os.replace(tmp, d)
    except OSError:           # another process stored it first
        pass
    return w


CONFIGS = {
    "lattice_box": lattice_box,
    "halo": halo,
    "lognormal_box": lognormal_box,
    "slab": slab,
}
