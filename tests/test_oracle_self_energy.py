"""Pins of the oracle's screened interaction and self-energy kernel
(Eqs. W_def, W_delta, I_c).

1. W in the symmetric form V eps~^-1 V equals the textbook W = eps^-1 v with
   eps = 1 - v chi0 (v = 4 pi / |q+G|^2 on the column index).
2. W^delta written term by term as printed equals (W - W^H)/(2i); it
   vanishes for a Hermitian W (imaginary axis) and is Hermitian.
3. A single plasmon pole: W^delta is the closed-form Lorentzian pair, and its
   integral over w > 0 tends to -pi R v (the pole's spectral weight).
4. On the real axis (w > 0, eta > 0) W^delta of the oracle's own eps~^-1 is
   negative semidefinite, and the diagonal of I is real and >= 0.
5. With W^delta = 1 on a G set that holds every Fourier component of the
   pair densities, Parseval's identity turns Eq. (I_c) into the cell average
   of conj(psi_a) psi_b |psi_m|^2, evaluated here on a real-space mesh from
   the plane-wave sums of the orbitals.
6. A rank-one W^delta = u u^H gives I_ab = -c (u^T rho_a) conj(u^T rho_b),
   which fixes the orientation of W^delta against (G, G').
"""
import itertools
import math

import numpy as np

import oracle as O
from synth import cfg_tiny, make_system


def _system(freqs=(0.3 + 0j,), eta=0.05, seed=31, ng=15):
    return make_system(cfg_tiny(seed=seed, kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),), fft=(16, 16, 16), ng=ng,
                                n_occ=3, n_bands=8, npw_target=20, a=6.0, freqs=freqs, eta=eta))


def _eps_inv(s, iw=0):
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    chi = O.chi0_tr(s, 0, G, s.freqs, s.eta)
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    return G, qg, chi[iw], O.eps_inv_gauss_jordan(chi[iw], qg)


def test_symmetric_w_equals_textbook_w():
    s = _system(freqs=(0.7 + 0j,))
    G, qg, chi, einv = _eps_inv(s)
    v = 4.0 * math.pi / qg ** 2
    eps = np.eye(s.ng) - v[:, None] * chi            # eps = 1 - v chi0
    W_textbook = np.linalg.solve(eps, np.diag(v))      # eps^-1 v
    W = O.screened_w(einv, qg)
    assert np.allclose(W, W_textbook, rtol=1e-12, atol=1e-12 * np.abs(W).max())


def test_w_delta_forms():
    rng = np.random.default_rng(3)
    W = rng.standard_normal((7, 7)) + 1j * rng.standard_normal((7, 7))
    Wd = O.w_delta(W)
    assert np.allclose(Wd, (W - W.conj().T) / 2j, rtol=0, atol=1e-15)
    assert np.allclose(Wd, Wd.conj().T, rtol=0, atol=0)
    H = W + W.conj().T
    assert np.abs(O.w_delta(H)).max() <= 1e-15


def test_single_pole_lorentzian_and_weight():
    R, wt, eta, v = -0.3, 0.8, 0.002, 2.5
    w = np.linspace(1e-4, 6.0, 600001)
    x = R * (1.0 / (w - wt + 1j * eta) - 1.0 / (w + wt + 1j * eta))
    Wd = np.array([O.w_delta(np.array([[v * (1.0 + xi)]]))[0, 0] for xi in x[::5000]])
    closed = v * R * (-eta / ((w - wt) ** 2 + eta ** 2) + eta / ((w + wt) ** 2 + eta ** 2))
    assert np.allclose(Wd, closed[::5000], rtol=1e-12, atol=1e-14)
    full = v * np.imag(x)                   # W^delta of the 1 x 1 case at every w
    assert np.allclose(full, closed, rtol=1e-9, atol=1e-12)
    weight = np.trapezoid(full, w)
    assert abs(weight - (-math.pi * R * v)) < 1e-2 * abs(math.pi * R * v)


def test_real_axis_sign_and_imaginary_axis_zero():
    s = _system(freqs=(0.4 + 0j, 1.2 + 0j, 0.5j), eta=0.05)
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    chi = O.chi0_tr(s, 0, G, s.freqs, s.eta)
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    for iw, w in enumerate(s.freqs):
        Wd = O.w_delta(O.screened_w(O.eps_inv_gauss_jordan(chi[iw], qg), qg))
        ev = np.linalg.eigvalsh(Wd)
        if w.real > 0:
            assert ev.max() <= 1e-12 * np.abs(ev).max() and ev.min() < 0
            I = O.i_kernel(s, 0, G, [2, 3], Wd)
            d = np.diagonal(I, axis1=2, axis2=3)
            assert np.abs(d.imag).max() <= 1e-12 * np.abs(d).max()
            assert d.real.min() >= -1e-12 * np.abs(d).max()
            assert np.allclose(I, np.conj(np.swapaxes(I, 2, 3)), rtol=0, atol=1e-13 * np.abs(I).max())
        else:
            assert np.abs(Wd).max() <= 1e-12 * np.abs(O.screened_w(np.eye(s.ng), qg)).max()


def _orbitals_on_mesh(s, ik, bands, n):
    """Periodic parts u(r) = sum_G c(G) e^{iG.r} on an n^3 mesh (reduced r)."""
    t = np.arange(n) / n
    r = np.stack(np.meshgrid(t, t, t, indexing="ij"), axis=-1).reshape(-1, 3)
    ph = np.exp(2j * np.pi * (r @ s.sphere(ik).astype(np.float64).T))      # (Nr, npw)
    return ph @ s.coefs(ik)[list(bands)].T                                   # (Nr, nbands)


def test_parseval_real_space():
    # a 3 x 2 x 2 grid: k points off the time-reversal invariant ones have
    # complex orbitals, so conj(psi_a) psi_b |psi_m|^2 is not symmetric in (a, b)
    s = make_system(cfg_tiny(seed=37, kgrid=(3, 2, 2), q_frac=((1.0 / 3.0, 0.0, 0.0),), fft=(16, 16, 16), ng=15,
                             n_occ=3, n_bands=6, npw_target=20, a=6.0, freqs=(0.3 + 0j,), eta=0.05))
    L = int(np.abs(s.gvec).max())
    _, g0 = O.kpair_map(s.spec.kgrid, s.q_frac[0])
    span = 2 * L + int(np.abs(g0).max())
    cube = np.array(list(itertools.product(range(-span, span + 1), repeat=3)), dtype=np.int64)
    qp = [1, 4]
    ks = [1, 4]
    I = O.i_kernel(s, 0, cube, qp, np.eye(cube.shape[0]), ks=ks)
    ikp, _ = O.kpair_map(s.spec.kgrid, s.q_frac[0])
    n = 2 * (2 * span) + 2          # the integrand's components reach +-2 span
    assert np.abs(I - np.swapaxes(I, 2, 3)).max() > 1e-3 * np.abs(I).max()   # not symmetric in (a, b)
    for j, ik in enumerate(ks):
        ua = _orbitals_on_mesh(s, ik, qp, n)
        um = _orbitals_on_mesh(s, int(ikp[ik]), range(s.nb), n)
        for m in range(s.nb):
            dens = np.abs(um[:, m]) ** 2
            want = -np.einsum("r,ra,rb->ab", dens, np.conj(ua), ua) / ua.shape[0] / (s.nk * s.omega_cell)
            assert np.allclose(I[j, m], want, rtol=1e-10, atol=1e-13 * np.abs(want).max()), (ik, m)


def test_rank_one_orientation():
    s = _system(freqs=(0.3 + 0j,))
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(s.ng) + 1j * rng.standard_normal(s.ng)
    I = O.i_kernel(s, 0, G, [0, 2, 5], np.outer(u, np.conj(u)), ks=[3])
    rho = O.rho_block(s, 0, G, 3, [0, 2, 5], np.arange(s.nb))                 # [a, m, G]
    p = np.einsum("g,amg->am", u, rho)                                        # u^T rho_a
    want = -np.einsum("am,bm->mab", p, np.conj(p)) / (s.nk * s.omega_cell)
    assert np.allclose(I[0], want, rtol=1e-12, atol=1e-14 * np.abs(want).max())
    # the transposed orientation differs
    It = O.i_kernel(s, 0, G, [0, 2, 5], np.outer(np.conj(u), u), ks=[3])
    assert np.abs(It[0] - want).max() > 1e-3 * np.abs(want).max()
