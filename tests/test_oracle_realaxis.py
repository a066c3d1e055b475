"""Pins of the oracle on the real frequency axis (w > 0 with eta > 0), where
the weights are complex and chi0, eps~ are not Hermitian:

1. the time-reversal two-pole form equals the all-ordered-pairs form of
   Eq. (X_IP) (the paper's definition) at real frequencies;
2. absorption: for w > 0 the anti-Hermitian part (chi0 - chi0^H) / 2i is
   negative semidefinite (every transition absorbs), and it vanishes as
   eta -> 0 away from the transition energies;
3. Gauss-Jordan with partial pivoting inverts the general eps~ like LAPACK,
   and agrees with the RPA route of Eq. (X_rpa_inv);
4. causality: the real part of chi0 on the real axis is the Hilbert transform
   of its imaginary part (Kramers-Kronig, within 1e-4 of the largest value),
   and the advanced sign of eta fails that by order one.
"""
import numpy as np

import oracle as O
from synth import HA_EV, cfg_tiny, make_system


def _sys():
    return make_system(cfg_tiny(seed=5, kgrid=(3, 3, 2), n_occ=2, n_bands=5, npw_target=25,
                                q_frac=((1.0 / 3.0, 2.0 / 3.0, 0.5),), a=7.0))


REAL = np.array([0.05, 0.4, 1.3]) + 0j  # Ha


def test_tr_form_equals_all_pairs_on_real_axis():
    s = _sys()
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 8)
    eta = 0.1 / HA_EV
    a = O.chi0_all_pairs(s, 0, G, REAL, eta)
    b = O.chi0_tr(s, 0, G, REAL, eta)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    # genuinely non-Hermitian here
    assert np.abs(b - np.conj(np.transpose(b, (0, 2, 1)))).max() > 1e-3 * np.abs(b).max()


def test_absorption_sign():
    s = _sys()
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 8)
    chi = O.chi0_tr(s, 0, G, REAL, 0.05)
    for c in chi:
        anti = (c - c.conj().T) / 2j
        ev = np.linalg.eigvalsh(anti)
        assert ev.max() < 1e-14 * np.abs(ev).max()
        assert ev.min() < 0.0
    # far below every transition energy the absorptive part goes with eta
    lo = np.array([1e-3 + 0j])
    a1 = O.chi0_tr(s, 0, G, lo, 1e-4)[0]
    a2 = O.chi0_tr(s, 0, G, lo, 2e-4)[0]
    n1 = np.abs(a1 - a1.conj().T).max()
    n2 = np.abs(a2 - a2.conj().T).max()
    assert abs(n2 / n1 - 2.0) < 1e-3


def test_general_inverse_routes():
    s = _sys()
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 8)
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    for c in O.chi0_tr(s, 0, G, REAL, 0.05):
        e = O.eps_tilde(c, qg)
        gj = O.eps_inv_gauss_jordan(c, qg)
        assert np.abs(gj @ e - np.eye(len(G))).max() < 1e-12
        assert np.abs(gj - np.linalg.inv(e)).max() < 1e-12 * np.abs(gj).max()
        assert np.abs(gj - O.eps_inv_rpa_route(c, qg)).max() < 1e-12 * np.abs(gj).max()


def _pv_integral(x, f, x0):
    """Principal value of int f(x) / (x - x0) dx over the grid x (trapezoid on the
    subtracted, smooth integrand plus the closed form of the log term)."""
    fx0 = np.interp(x0, x, f)
    g = (f - fx0) / (x - x0)
    g[np.isclose(x, x0)] = np.gradient(f, x)[np.isclose(x, x0)]
    return np.trapezoid(g, x) + fx0 * np.log(abs((x[-1] - x0) / (x[0] - x0)))


def test_kramers_kronig():
    """Causality: with +i eta on both poles chi0 is analytic in the upper half
    plane, so on the real axis its real part is the Hilbert transform of its
    imaginary part, Re chi(w) = (1/pi) P int Im chi(w') / (w' - w) dw' (here
    for the head element, w' over the whole real line).  The advanced sign
    (-i eta) breaks the relation."""
    s = _sys()
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 2)
    eta = 0.2
    core = np.linspace(-20.0, 20.0, 4001)
    tail = np.geomspace(20.0, 4000.0, 400)[1:]
    x = np.concatenate([-tail[::-1], core, tail])
    for sign, ok in ((1.0, True), (-1.0, False)):
        chi = O.chi0_tr(s, 0, G, x + 0j, sign * eta)[:, 0, 0]
        for w0 in (0.3, 0.8, 1.2):
            re_kk = _pv_integral(x, chi.imag, w0) / np.pi
            re = np.interp(w0, x, chi.real)
            err = abs(re_kk - re) / np.abs(chi).max()
            assert (err < 1e-4) == ok, (sign, w0, err)
