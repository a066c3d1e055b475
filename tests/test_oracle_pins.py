"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each check is chosen so that a plausible mistake in the oracle (a dropped
term, a wrong sign or index, a transposed operand, a wrong prefactor) fails
at least one of them:

P1  rho_nm(q=0, G=0) = delta_nm (orthonormality through Eq. rhotw)
P2  rho by direct plane-wave convolution == real-space Riemann sum of
    psi* e^{i(q+G)r} psi (a different route: explicit orbitals on a mesh)
P4  chi0 Hermitian and negative semidefinite (static w with the retarded
    eta under time reversal, and on the imaginary axis)
P5  all-ordered-pairs chi0 == time-reversal two-pole chi0 on TR inputs,
    and differs on inputs that break TR (the check has teeth)
P6  free-electron crystal: chi0 == discrete Lindhard sum (diagonal, closed
    form written from momenta without rho)
P7  gauge invariance (random phase per state)
P8  umklapp invariance (another reciprocal-lattice representative of k')
P9  Dyson: Gauss-Jordan == linear solve of Eq. (X_rpa_inv); eps~^-1
    Hermitian with spectrum in (0, 1]; Gauss-Jordan == LAPACK inverse
P10 high-frequency tail: w^2 chi0(iw) -> -f_s/(N_k Omega) sum_t 2|D_t| df rho rho^H
P13 absolute scale: the f-sum (Thomas-Reiche-Kuhn) rule of a free-electron
    crystal, nu^2 chi0_GG(i nu) -> -(N_el/Omega) |q+G|^2, with N_el counted
    from the occupations and Omega = a^3, so the prefactor f_s/(N_k Omega)
    and the 2 pi/a of the reciprocal lattice are fixed by physics, not by the
    oracle's own formula; |q+G| checked against values worked out by hand
G-set: the response G order for q = (1/4,0,0) written out by hand.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import (HA_EV, cfg_plain_fp64, cfg_tiny, make_plane_wave_system,
                   make_system)


@pytest.fixture(scope="module")
def tiny():
    return make_system(cfg_tiny(seed=11, kgrid=(2, 2, 2), n_occ=3, n_bands=6, npw_target=20,
                                q_frac=((0.5, 0.0, 0.0),)))


@pytest.fixture(scope="module")
def tiny3():
    # 3x3x1-like odd grid exercises non-self-partner k and umklapp along two axes
    return make_system(cfg_tiny(seed=5, kgrid=(3, 3, 2), n_occ=2, n_bands=5, npw_target=25,
                                q_frac=((1.0 / 3.0, 2.0 / 3.0, 0.5),), a=7.0))


# ---------------------------------------------------------------- inputs


def test_synth_orthonormal_and_time_reversal(tiny3):
    s = tiny3
    for ik in range(s.nk):
        c = s.coefs(ik)
        assert np.abs(c.conj() @ c.T - np.eye(s.nb)).max() < 1e-13
    kg = s.spec.kgrid
    for ik in range(s.nk):
        i, j, l = np.rint(s.kfrac[ik] * kg).astype(int)
        jk = ((-i) % kg[0] * kg[1] + (-j) % kg[1]) * kg[2] + (-l) % kg[2]
        g1 = np.rint(s.kfrac[ik] + s.kfrac[jk]).astype(int)
        where = {tuple(v): p for p, v in enumerate(s.sphere(ik).tolist())}
        for p, gp in enumerate(s.sphere(jk).tolist()):
            src = where[tuple((-np.array(gp) - g1).tolist())]
            assert np.abs(s.coefs(jk)[:, p] - np.conj(s.coefs(ik)[:, src])).max() < 1e-15
        assert np.array_equal(s.eps[ik], s.eps[jk])


def test_synth_deterministic():
    a = make_system(cfg_tiny(seed=3))
    b = make_system(cfg_tiny(seed=3))
    assert np.array_equal(a.coef, b.coef) and np.array_equal(a.eps, b.eps)


def test_plain_config_sizes():
    s = make_system(cfg_plain_fp64())
    assert s.nk == 64 and s.nb == 32
    assert 288 <= s.npw.min() and s.npw.max() <= 305
    assert abs(s.npw.mean() - 300.2) < 0.5


# ---------------------------------------------------------------- G set


def test_response_gvectors_by_hand():
    # |q+G|^2 for q = (1/4,0,0): 1/16; 9/16; 17/16 (x4, lex order); 25/16 (x5, lex order)
    want = [(0, 0, 0), (-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 1), (0, 1, 0),
            (-1, -1, 0), (-1, 0, -1), (-1, 0, 1), (-1, 1, 0), (1, 0, 0)]
    got = O.response_gvectors((4, 4, 4), (0.25, 0.0, 0.0), 11)
    assert [tuple(v) for v in got.tolist()] == want


def test_response_gvectors_shells():
    g = O.response_gvectors((4, 4, 4), (0.25, 0.0, 0.0), 65)
    d = ((g + np.array([0.25, 0.0, 0.0])) ** 2).sum(axis=1)
    assert np.all(np.diff(d) >= 0)
    # 59 vectors end inside the shell that starts at index 53 and closes at 65
    assert d[52] < d[53] and np.all(d[53:65] == d[53])


def test_kpair_map_umklapp():
    ikp, g0 = O.kpair_map((4, 4, 4), (0.25, 0.0, 0.0))
    # k = 0 minus q = (-1/4, 0, 0) = (3/4, 0, 0) + (-1, 0, 0)
    assert ikp[0] == 3 * 16 and tuple(g0[0]) == (-1, 0, 0)
    assert ikp[16] == 0 and tuple(g0[16]) == (0, 0, 0)


# ---------------------------------------------------------------- rho


def test_p1_rho_normalisation():
    s = make_system(cfg_tiny(seed=2, q_frac=((0.0, 0.0, 0.0),)))
    bands = np.arange(s.nb)
    for ik in range(s.nk):
        r = O.rho_block(s, 0, np.zeros((1, 3), dtype=int), ik, bands, bands)[:, :, 0]
        assert np.abs(r - np.eye(s.nb)).max() < 1e-14


@pytest.mark.parametrize("fixture", ["tiny", "tiny3"])
def test_p2_rho_direct_vs_realspace(fixture, request):
    s = request.getfixturevalue(fixture)
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 9)
    ngrid = 24
    for ik in range(s.nk):
        blk = O.rho_block(s, 0, G, ik, [0, s.nb - 1], [1, s.nb - 2])
        for a_, n in enumerate([0, s.nb - 1]):
            for b_, m in enumerate([1, s.nb - 2]):
                ref = O.rho_realspace_bruteforce(s, 0, G, ik, n, m, ngrid)
                assert np.abs(blk[a_, b_] - ref).max() < 1e-13


def test_rho_both_summation_orders(tiny3):
    s = tiny3
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 12)
    b = np.arange(s.nb)
    for ik in range(s.nk):
        r1 = O.rho_block(s, 0, G, ik, b, b)
        r2 = O.rho_block(s, 0, G, ik, b, b, shifted=True)
        assert np.abs(r1 - r2).max() < 1e-14


def test_p8_umklapp_representative(tiny3):
    s = tiny3
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 7)
    ikp, g0 = O.kpair_map(s.spec.kgrid, s.q_frac[0])
    shift = np.array([1, -2, 1])
    for ik in range(s.nk):
        jk = ikp[ik]
        ref = O.rho_pair(s.sphere(ik), s.coefs(ik), s.sphere(jk), s.coefs(jk), G, g0[ik])
        # the same states written about k'' = k' + shift: S'' = S - shift, G0'' = G0 - shift
        alt = O.rho_pair(s.sphere(ik), s.coefs(ik), s.sphere(jk) - shift, s.coefs(jk), G,
                         g0[ik] - shift)
        assert np.abs(ref - alt).max() < 1e-15
        assert np.abs(ref).max() > 1e-3


# ---------------------------------------------------------------- chi0


def _freqs():
    return np.array([0.0, 0.05j, 0.7j, 3.0j])


def test_p4_chi0_hermitian_nsd(tiny3):
    s = tiny3
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 8)
    # static with retarded eta (real weights under TR) and imaginary axis with eta = 0
    for freqs, eta in (([0j], s.eta), (_freqs()[1:], 0.0)):
        chi = O.chi0_all_pairs(s, 0, G, freqs, eta)
        for c in chi:
            scale = np.abs(c).max()
            assert np.abs(c - c.conj().T).max() < 1e-14 * scale
            ev = np.linalg.eigvalsh(0.5 * (c + c.conj().T))
            assert ev.max() < 1e-14 * scale and ev.min() < -1e-3 * scale


def test_p5_two_formulations_agree(tiny, tiny3):
    for s in (tiny, tiny3):
        G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 8)
        c3 = O.chi0_all_pairs(s, 0, G, _freqs(), 0.0)
        c4 = O.chi0_tr(s, 0, G, _freqs(), 0.0)
        assert np.abs(c3 - c4).max() < 1e-13 * np.abs(c3).max()
        c3 = O.chi0_all_pairs(s, 0, G, [0j], s.eta)
        c4 = O.chi0_tr(s, 0, G, [0j], s.eta)
        assert np.abs(c3 - c4).max() < 1e-13 * np.abs(c3).max()


def test_p5_teeth_broken_time_reversal(tiny3):
    s = make_system(tiny3.spec)
    rng = np.random.default_rng(0)
    n = s.npw[1]
    z = rng.standard_normal((n, s.nb)) + 1j * rng.standard_normal((n, s.nb))
    s.coef[1, :, :n] = np.linalg.qr(z)[0].T      # k index 1 loses its TR partner
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 8)
    c3 = O.chi0_all_pairs(s, 0, G, [0.3j], 0.0)
    c4 = O.chi0_tr(s, 0, G, [0.3j], 0.0)
    assert np.abs(c3 - c4).max() > 1e-3 * np.abs(c3).max()


def test_p6_lindhard_free_electrons():
    spec = cfg_tiny(kgrid=(2, 2, 2), n_bands=10, npw_target=40, q_frac=((0.5, 0.0, 0.0),),
                    eta=0.02)
    s = make_plane_wave_system(spec, e_fermi=0.3)
    assert 0 < s.occ.sum() < s.occ.size
    G = O.response_gvectors(spec.kgrid, s.q_frac[0], 7)
    freqs = [0j, 0.5j, 0.2 + 0j]
    chi = O.chi0_all_pairs(s, 0, G, freqs, spec.eta)
    ref = O.chi0_lindhard_plane_waves(s, 0, G, freqs, spec.eta, 0.3)
    assert np.abs(ref).max() > 1e-2
    assert np.abs(chi - ref).max() < 1e-14
    off = chi - np.einsum("wii->wi", chi)[:, :, None] * np.eye(len(G))[None]
    assert np.abs(off).max() == 0.0


def test_p7_gauge_invariance(tiny3):
    s = make_system(tiny3.spec)
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 8)
    ref3 = O.chi0_all_pairs(s, 0, G, _freqs(), 0.0)
    ref4 = O.chi0_tr(s, 0, G, _freqs(), 0.0)
    rng = np.random.default_rng(1)
    s.coef *= np.exp(1j * rng.uniform(0, 2 * np.pi, size=s.coef.shape[:2]))[:, :, None]
    assert np.abs(O.chi0_all_pairs(s, 0, G, _freqs(), 0.0) - ref3).max() < 1e-14 * np.abs(ref3).max()
    assert np.abs(O.chi0_tr(s, 0, G, _freqs(), 0.0) - ref4).max() < 1e-14 * np.abs(ref4).max()


def test_p7_degenerate_rotation(tiny3):
    s = make_system(tiny3.spec)
    # make bands 3 and 4 exactly degenerate everywhere, then rotate them at every k
    s.eps[:, 4] = s.eps[:, 3]
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 6)
    ref = O.chi0_all_pairs(s, 0, G, _freqs(), 0.0)
    th, ph = 0.7, 1.3
    u = np.array([[math.cos(th), -math.sin(th) * np.exp(-1j * ph)],
                  [math.sin(th) * np.exp(1j * ph), math.cos(th)]])
    s.coef[:, 3:5, :] = np.einsum("ab,kbg->kag", u, s.coef[:, 3:5, :])
    got = O.chi0_all_pairs(s, 0, G, _freqs(), 0.0)
    assert np.abs(got - ref).max() < 1e-14 * np.abs(ref).max()


def test_p10_frequency_tail(tiny3):
    s = tiny3
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 6)
    nu = 1.0e4
    chi = O.chi0_tr(s, 0, G, [1j * nu], 0.0)[0] * nu * nu
    trans = O.transitions_tr(s, 0)
    ikp, _ = O.kpair_map(s.spec.kgrid, s.q_frac[0])
    rho = O.rho_transitions(s, 0, G, trans)
    jk = ikp[trans[:, 0]]
    d = s.eps[jk, trans[:, 2]] - s.eps[trans[:, 0], trans[:, 1]]
    df = s.occ[jk, trans[:, 2]] - s.occ[trans[:, 0], trans[:, 1]]
    pref = s.spin_factor / (s.nk * s.omega_cell)
    tail = -pref * np.einsum("t,ti,tj->ij", 2 * np.abs(d) * df, rho, rho.conj())
    assert np.abs(chi - tail).max() < 1e-6 * np.abs(tail).max()


def test_weights_static_real_and_negative(tiny3):
    s = tiny3
    trans = O.transitions_tr(s, 0)
    w = O.weights_tr(s, 0, trans, [0j], s.eta)
    assert np.abs(w.imag).max() < 1e-15 * np.abs(w).max()
    assert np.all(w.real < 0)


# ---------------------------------------------------------------- Dyson


def test_gauss_jordan_vs_lapack():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((17, 17)) + 1j * rng.standard_normal((17, 17))
    assert np.abs(O.dyson.gauss_jordan_inverse(a) - np.linalg.inv(a)).max() < 1e-12


def test_p9_dyson_routes(tiny3):
    s = tiny3
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], 8)
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    chi = O.chi0_tr(s, 0, G, _freqs()[1:], 0.0)
    # scale chi0 up so that local fields matter
    for c in chi * 50.0:
        e1 = O.eps_inv_gauss_jordan(c, qg)
        e2 = O.eps_inv_rpa_route(c, qg)
        assert np.abs(e1 - e2).max() < 1e-12
        assert np.abs(e1 - e1.conj().T).max() < 1e-12
        ev = np.linalg.eigvalsh(0.5 * (e1 + e1.conj().T))
        assert ev.min() > 0 and ev.max() <= 1 + 1e-12 and ev.min() < 0.999
        assert np.abs(e1 @ O.eps_tilde(c, qg) - np.eye(len(G))).max() < 1e-12


# ---------------------------------------------------------------- absolute scale (P13)


def _fsum_system():
    """Free-electron crystal with few occupied plane waves and enough bands
    that every occupied momentum p has p + (q+G) and p - (q+G) in the band
    sets, for every G of the response set (checked below from momenta)."""
    spec = cfg_tiny(kgrid=(2, 2, 2), n_bands=40, npw_target=None, kc=3.0,
                    q_frac=((0.5, 0.0, 0.0),), eta=0.0)
    s = make_plane_wave_system(spec, e_fermi=0.15)
    G = O.response_gvectors(spec.kgrid, s.q_frac[0], 7)
    return s, G


def _band_momenta(s, ik):
    """Momentum k + G of every band (in units of 2 pi / a), doubled to integers
    (the k grid is 2x2x2 and q = (1/2, 0, 0))."""
    g = s.sphere(ik)[np.argmax(np.abs(s.coefs(ik)), axis=1)]
    return np.rint(2.0 * (s.kfrac[ik][None, :] + g)).astype(np.int64)


def _fsum_deviation(s, G, chi_fn):
    """max |nu^2 chi0_GG(i nu) + (N_el/Omega)|q+G|^2| / max |(N_el/Omega)|q+G|^2|
    and the largest off-diagonal |nu^2 chi0|, at nu = 1e5 Ha."""
    nu = 1.0e5
    chi = chi_fn(s, 0, G, [1j * nu], 0.0)[0] * nu * nu
    n_el = s.spin_factor * float(s.occ.sum()) / s.nk      # electrons per cell
    volume = s.spec.a ** 3                                # cubic cell (bohr^3)
    two_pi_a = 2.0 * math.pi / s.spec.a                   # reciprocal lattice step
    qg2 = (two_pi_a ** 2) * ((s.q_frac[0][None, :] + G) ** 2).sum(axis=1)
    expect = -(n_el / volume) * qg2
    dev = np.abs(np.diag(chi) - expect).max() / np.abs(expect).max()
    off = np.abs(chi - np.diag(np.diag(chi))).max() / np.abs(expect).max()
    return dev, off


def test_p13_fsum_preconditions():
    s, G = _fsum_system()
    held = set()
    for ik in range(s.nk):
        held |= {tuple(p) for p in _band_momenta(s, ik).tolist()}
    q2 = np.rint(2.0 * s.q_frac[0]).astype(np.int64)
    n_occ = 0
    for ik in range(s.nk):
        mom = _band_momenta(s, ik)
        for b in np.nonzero(s.occ[ik] > 0)[0]:
            n_occ += 1
            for Gv in G:
                Q = q2 + 2 * Gv
                assert tuple((mom[b] + Q).tolist()) in held
                assert tuple((mom[b] - Q).tolist()) in held
    assert 1 < n_occ < s.occ.size


@pytest.mark.parametrize("form", ["tr", "all_pairs"])
def test_p13_fsum_rule(form):
    s, G = _fsum_system()
    fn = O.chi0_tr if form == "tr" else O.chi0_all_pairs
    dev, off = _fsum_deviation(s, G, fn)
    assert dev < 1e-9 and off < 1e-12


def test_p13_fsum_teeth(monkeypatch):
    """The f-sum check fails on the plausible prefactor mistakes, planted in
    the oracle: the spin factor dropped, or Omega in place of N_k Omega."""
    import oracle.chi0 as oc
    s, G = _fsum_system()
    for wrong in (lambda sy: 1.0 / (sy.nk * sy.omega_cell),
                  lambda sy: sy.spin_factor / sy.omega_cell):
        monkeypatch.setattr(oc, "_prefactor", wrong)
        dev, _ = _fsum_deviation(s, G, O.chi0_tr)
        assert dev > 0.4


def _qg_literal_ok(qg_fn):
    """|q+G| in bohr^-1 for a = 10 bohr and q = (1/4, 0, 0), worked out by hand:
    G = 0: 2 pi/10 * 1/4 = 0.05 pi; G = (1,0,0): 2 pi/10 * 5/4 = 0.25 pi;
    G = (-1,0,0): 0.15 pi; G = (0,1,0): 0.2 pi * sqrt(17)/4; G = (1,1,1):
    0.2 pi * sqrt(57)/4."""
    G = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [1, 1, 1]])
    expect = math.pi * np.array([0.05, 0.25, 0.15, 0.05 * math.sqrt(17.0), 0.05 * math.sqrt(57.0)])
    got = qg_fn(10.0, np.array([0.25, 0.0, 0.0]), G)
    return np.abs(got - expect).max() < 1e-15


def test_p13_qg_norm_literal():
    assert _qg_literal_ok(O.qg_norms)
    # teeth: the reciprocal-lattice factor 2 pi/a dropped, or 1/a kept alone
    assert not _qg_literal_ok(lambda a, q, g: np.sqrt(((q[None, :] + g) ** 2).sum(axis=1)))
    assert not _qg_literal_ok(lambda a, q, g: np.sqrt(((q[None, :] + g) ** 2).sum(axis=1)) / a)
