"""Pins of the Bruneval-Gonze extrapolar correction in the oracle
(Eq. X_term_def, Appendix C), checked against facts the definition fixes:

1. the diagonal density rho~_m(0) = <m|m> = 1, and rho~_m(-d) = conj(rho~_m(d))
   (|u_m|^2 is real);
2. rho~ equals the real-space definition (1/N) sum_r |u_m(r)|^2 e^{i d.r},
   summed point by point on a small grid (no FFT);
3. the closure relation made exact: with a complete band basis at every k,
   occupied states on an inner sphere (so every product with a response
   vector stays inside the basis) and every omitted band at eps_bar, the
   truncated chi0 plus the correction equals the full-band chi0;
4. the correction is Hermitian on the imaginary axis.
"""
import numpy as np
import pytest

import oracle as O
from synth import HA_EV, cfg_tiny, make_closure_system, make_system, truncate_bands


def _small():
    return make_system(cfg_tiny(seed=31, kgrid=(2, 2, 2), n_occ=3, n_bands=8, npw_target=40, fft=(16, 16, 16),
                                ng=9, q_frac=((0.5, 0.0, 0.0),), freqs=(0.2j, 1.0j), eta=0.0, a=7.0))


def test_diag_density_normalised_and_hermitian():
    s = _small()
    ds = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [1, 2, -1], [-1, -2, 1], [0, -1, 2], [0, 1, -2]])
    for ik in range(s.nk):
        rt = O.diag_density(s, ik, range(s.nb), ds)
        assert np.allclose(rt[:, 0], 1.0, atol=1e-12)
        for a, b in ((1, 2), (3, 4), (5, 6)):
            assert np.allclose(rt[:, a], np.conj(rt[:, b]), atol=1e-13)


def test_diag_density_real_space_definition():
    s = _small()
    N = 12  # grid points per axis, enough for |u|^2 of these spheres without aliasing at the d used
    r = np.stack(np.meshgrid(*(np.arange(N) / N,) * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    ds = np.array([[0, 0, 0], [1, 0, 0], [0, 2, -1], [1, -1, 1]])
    ik = 1
    g = s.sphere(ik)
    for m in range(s.nb):
        c = s.coefs(ik)[m]
        u = np.exp(2j * np.pi * r @ g.T) @ c               # u_m(r) on the grid
        dens = np.abs(u) ** 2
        ref = np.array([np.mean(dens * np.exp(2j * np.pi * r @ d)) for d in ds])
        got = O.diag_density(s, ik, [m], ds)[0]
        assert np.allclose(got, ref, atol=1e-12), (m, got, ref)


def test_closure_exact_reproduces_full_band_sum():
    eps_bar = 45.0 / HA_EV
    nb_keep = 12
    full = make_closure_system(nb_keep=nb_keep, omitted_ev=(eps_bar * HA_EV, eps_bar * HA_EV))
    G = O.response_gvectors(full.spec.kgrid, full.q_frac[0], full.ng)
    assert np.abs(G).max() <= 1
    _, g0 = O.kpair_map(full.spec.kgrid, full.q_frac[0])
    assert np.abs(g0).max() <= 1
    ref = O.chi0_tr(full, 0, G, full.freqs, full.eta)
    trunc = truncate_bands(full, nb_keep)
    chi_t = O.chi0_tr(trunc, 0, G, full.freqs, full.eta)
    got = O.chi0_bg(trunc, 0, G, full.freqs, full.eta, eps_bar)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 1e-12, rel
    # the truncation alone is far off: the check is not trivial
    assert np.linalg.norm(chi_t - ref) / np.linalg.norm(ref) > 1e-2
    # a wrong extrapolar energy breaks it
    bad = O.chi0_bg(trunc, 0, G, full.freqs, full.eta, 1.5 * eps_bar)
    assert np.linalg.norm(bad - ref) / np.linalg.norm(ref) > 1e-3


def test_correction_hermitian_on_imaginary_axis():
    s = _small()
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    d = O.delta_chi_bg(s, 0, G, s.freqs, 0.0, eps_bar=40.0 / HA_EV)
    assert np.abs(d - np.conj(np.transpose(d, (0, 2, 1)))).max() < 1e-13 * np.abs(d).max()
    assert np.abs(d).max() > 0.0


def test_closure_exact_on_the_real_axis():
    """The closure form does not depend on the frequency factor: with every
    omitted band at eps_bar it reproduces the full-band chi0 at real
    frequencies with broadening too (complex weights, non-Hermitian chi0)."""
    eps_bar = 45.0 / HA_EV
    nb_keep = 12
    full = make_closure_system(nb_keep=nb_keep, omitted_ev=(eps_bar * HA_EV, eps_bar * HA_EV))
    G = O.response_gvectors(full.spec.kgrid, full.q_frac[0], full.ng)
    freqs, eta = np.array([0.2, 0.9, 1.7]) + 0j, 0.05
    ref = O.chi0_tr(full, 0, G, freqs, eta)
    got = O.chi0_bg(truncate_bands(full, nb_keep), 0, G, freqs, eta, eps_bar)
    assert np.abs(ref - np.conj(np.swapaxes(ref, 1, 2))).max() > 1e-3 * np.abs(ref).max()   # not Hermitian
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
