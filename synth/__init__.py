"""Seeded synthetic inputs for the chi0 / epsilon^-1 path.

This package is the single source of inputs for both the CUDA library and the
CPU oracle.  It holds no arithmetic of the method itself (no oscillator
strengths, weights, contractions or Dyson steps): it only builds what a DFT
code would hand over -- a cubic cell, a Gamma-centred k grid, per-k
plane-wave spheres, orthonormal Bloch coefficients that obey time reversal,
band energies, occupations, q vectors and a frequency list.
"""
from .systems import (  # noqa: F401
    HA_EV,
    SystemSpec,
    System,
    make_system,
    make_closure_system,
    make_batching_system,
    make_plane_wave_system,
    truncate_bands,
    cfg_learned,
    cfg_large,
    large_energies,
    tr_partner,
    cfg_plain_fp64,
    cfg_precision,
    cfg_tiny,
    gauss_legendre_freqs,
    kgrid_fractions,
    sphere_miller,
)
