"""Pins of the oracle's degenerate-pole grouping and double-grid frequency
factor (Appendix B; the dense-grid paragraph of the Bethe-Salpeter section).

1. The grouping rule on a hand-made list of pole energies, in any input order.
2. eps_thresh = 0 leaves every pole alone: the weights equal the plain
   two-pole weights exactly, and chi0 equals chi0_tr.
3. Poles that are exactly degenerate across k (every k with the same
   energies): grouping changes nothing, and the groups are the band pairs.
4. Degeneracies broken by less than eps_thresh: the grouped chi0 differs from
   the plain one by an amount linear in the splitting.
5. Double grid: one dense point equal to the coarse energies, or several
   copies of it, gives the plain weights; symmetric dense shifts +-delta move
   the weights by O(delta^2) (the mean of the factor is second-order accurate).
"""
import dataclasses

import numpy as np

import oracle as O
import oracle.poles as P
from synth import cfg_tiny, make_system


def _sys(freqs=(0.2j, 1.5j), seed=41):
    return make_system(cfg_tiny(seed=seed, kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),), fft=(16, 16, 16), ng=15,
                                n_occ=3, n_bands=7, npw_target=20, a=6.0, freqs=freqs, eta=0.0))


def test_grouping_rule():
    d = np.array([0.0, 0.4, 0.9, 1.2, 5.0, 5.05]) * 1e-5
    assert P.pole_groups(d, 1e-5).tolist() == [0, 0, 0, 3, 4, 4]
    assert P.pole_groups(d, 0.0).tolist() == [0, 1, 2, 3, 4, 5]
    rng = np.random.default_rng(1)
    perm = rng.permutation(d.size)
    rep = P.pole_groups(d[perm], 1e-5)
    # the same groups in any input order: perm[t] is the original index of t
    want = [0, 0, 0, 3, 4, 4]
    for t in range(d.size):
        assert perm[rep[t]] == want[perm[t]]


def test_zero_threshold_is_plain():
    s = _sys()
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    trans = O.transitions_tr(s, 0)
    assert np.array_equal(P.weights_grouped(s, 0, trans, s.freqs, s.eta, 0.0),
                          O.weights_tr(s, 0, trans, s.freqs, s.eta))
    a = P.chi0_grouped(s, 0, G, s.freqs, s.eta, 0.0)
    b = O.chi0_tr(s, 0, G, s.freqs, s.eta)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()


def _degenerate(s):
    eps = np.repeat(s.eps[:1], s.nk, axis=0)       # every k has the energies of k = 0
    return dataclasses.replace(s, eps=eps)


def test_exact_degeneracy_is_exact():
    s = _degenerate(_sys())
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    trans = O.transitions_tr(s, 0)
    rep = P.pole_groups(P.pole_energies(s, 0, trans), 1e-9)
    pairs = {(int(n), int(m)) for _, n, m in trans}
    assert np.unique(rep).size == len(pairs)        # one group per band pair
    a = P.chi0_grouped(s, 0, G, s.freqs, s.eta, 1e-9)
    b = O.chi0_tr(s, 0, G, s.freqs, s.eta)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_broken_degeneracy_linear():
    base = _degenerate(_sys())
    G = O.response_gvectors(base.spec.kgrid, base.q_frac[0], base.ng)
    rng = np.random.default_rng(2)
    pattern = rng.uniform(-1.0, 1.0, base.eps.shape)
    errs = []
    for delta in (1e-7, 2e-7):
        s = dataclasses.replace(base, eps=base.eps + delta * pattern)
        a = P.chi0_grouped(s, 0, G, s.freqs, s.eta, 1e-5)    # groups still the band pairs
        b = O.chi0_tr(s, 0, G, s.freqs, s.eta)
        errs.append(np.abs(a - b).max() / np.abs(b).max())
    assert errs[0] > 0 and 1.8 < errs[1] / errs[0] < 2.2


def test_double_grid_identities_and_order():
    s = _sys()
    trans = O.transitions_tr(s, 0)
    plain = O.weights_tr(s, 0, trans, s.freqs, s.eta)
    assert np.array_equal(P.weights_double_grid(s, 0, trans, s.freqs, s.eta, s.eps[:, None, :]), plain)
    three = np.repeat(s.eps[:, None, :], 3, axis=1)
    assert np.abs(P.weights_double_grid(s, 0, trans, s.freqs, s.eta, three) - plain).max() <= 1e-15 * np.abs(plain).max()
    rng = np.random.default_rng(3)
    pattern = rng.uniform(-1.0, 1.0, s.eps.shape)
    errs = []
    for delta in (2e-3, 1e-3):
        dense = np.stack([s.eps + delta * pattern, s.eps - delta * pattern], axis=1)
        w = P.weights_double_grid(s, 0, trans, s.freqs, s.eta, dense)
        errs.append(np.abs(w - plain).max() / np.abs(plain).max())
    assert errs[1] > 0 and 3.6 < errs[0] / errs[1] < 4.4
