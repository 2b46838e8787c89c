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
