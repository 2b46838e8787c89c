"""GB300-native reverse ray tracer for UV-background self-shielding
(Altay & Theuns, arXiv:1304.4235): C-ABI CUDA library (csrc/, include/urchin.h)
and its thin Python binding (urchin.py)."""
from .urchin import (  # noqa: F401
    Bvh, UrchinError, load, library_path, urchin_build_bvh, urchin_equilibrium, urchin_gamma,
    urchin_cross_section_ratio, urchin_equilibrium_vjp, urchin_gamma_he, urchin_gamma_nearfar, urchin_gamma_vjp, urchin_healpix_dirs, urchin_kernel_launches, urchin_solve,
    urchin_solve_vjp, urchin_spectrum_weights, urchin_tangent, urchin_trace_columns, urchin_trace_columns_noalloc,
    urchin_trace_columns_nearfar, urchin_trace_columns_vjp, urchin_version,
)
