"""Plain FP64 CPU oracle for the chi0 / epsilon^-1 path -- TEST INFRASTRUCTURE.

This package exists to check the CUDA library, never to stand in for it.  Only
the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA path; its only
inputs come from the ``synth`` package (seeded synthetic systems).

Every routine follows the paper (Sangalli et al., "Many-body perturbation
theory calculations using the yambo code", J. Phys.: Condens. Matter 31,
325902 (2019), arXiv:1902.03837) in the most direct form available:

* oscillator strengths rho by direct plane-wave convolution (no FFT),
  Eq. (rhotw) of the Linear Response section;
* chi0 by explicit sums over k and band pairs, Eq. (X_IP) and the
  frequency/transition split of Appendix B;
* the Dyson step by Gauss-Jordan elimination with partial pivoting, and
  independently by the linear solve of Eq. (X_rpa_inv);
* the bare Coulomb interaction v(q+G) = 4 pi / |q+G|^2 of the Coulomb
  interaction subsection and the symmetric form of Eq. (W_def);
* the Bruneval-Gonze extrapolar correction of Eq. (X_term_def) and
  Appendix C through the closure relation over the bands at k;
* the Godby-Needs plasmon-pole fit of eps^-1 at w = 0 and w = i w_p (Full
  frequency GW subsection);
* the screened interaction W, its delta-like part and the self-energy kernel
  I of Eqs. (W_def), (W_delta), (I_c);
* the degenerate-pole grouping of Appendix B and the double-grid frequency
  factor.

Parity status: every function here is pinned by tests in tests/test_oracle_*.py
against invariants, closed forms or independent routes.
"""
from .geometry import kpair_map, response_gvectors, qg_norms  # noqa: F401
from .rho import rho_pair, rho_pair_shifted, rho_block, rho_transitions, rho_realspace_bruteforce  # noqa: F401
from .chi0 import (  # noqa: F401
    transitions_tr,
    weights_tr,
    chi0_all_pairs,
    chi0_tr,
    chi0_lindhard_plane_waves,
)
from .dyson import eps_tilde, eps_inv_gauss_jordan, eps_inv_rpa_route  # noqa: F401
from .bg_terminator import diag_density, extrapolar_weights, delta_chi_bg, chi0_bg  # noqa: F401
from .ppa import ppa_fit, ppa_eval  # noqa: F401
from .self_energy import screened_w, w_delta, i_kernel  # noqa: F401
from .poles import (  # noqa: F401
    pole_energies, pole_groups, weights_grouped, weights_double_grid, chi0_weighted, chi0_grouped,
    chi0_double_grid,
)
