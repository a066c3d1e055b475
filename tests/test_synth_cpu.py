"""The seeded batching workload follows its recipe: cell edge in [8, 14] bohr,
plane waves per state in [400, 4000] (within the rounding of a sphere), N_G in
[200, 1500], 4..20 distinct nonzero q vectors of the 4x4x4 grid, 8..64 imaginary
frequencies in (0, 100] eV, 64 bands in [-10, 30] eV sorted per k, Fermi-Dirac
occupations that hold 32 electrons per cell, an FFT grid of the form
2^a 3^b 5^c that is at least 4 n_max + 1; the same seed gives the same system."""
import numpy as np

from synth import HA_EV, make_batching_system


def _smooth(n):
    for f in (2, 3, 5):
        while n % f == 0:
            n //= f
    return n == 1


def test_batching_recipe():
    for s in (0, 5, 14):
        sy = make_batching_system(s)
        assert 8.0 <= sy.spec.a <= 14.0
        assert 200 <= sy.ng <= 1500
        assert 4 <= sy.q_frac.shape[0] <= 20
        q = {tuple(np.rint(4 * v).astype(int) % 4) for v in sy.q_frac}
        assert len(q) == sy.q_frac.shape[0] and (0, 0, 0) not in q
        assert np.all(np.isclose(4 * sy.q_frac, np.rint(4 * sy.q_frac)))
        assert 8 <= sy.freqs.size <= 64
        w = sy.freqs.imag * HA_EV
        assert np.all(sy.freqs.real == 0) and w.min() > 0 and w.max() < 100
        assert sy.nk == 64 and sy.nb == 64
        assert 0.8 * 400 <= sy.npw.min() and sy.npw.max() <= 1.2 * 4000
        e = sy.eps * HA_EV
        assert e.min() >= -10 and e.max() <= 30 and np.all(np.diff(sy.eps, axis=1) >= 0)
        assert abs(sy.spin_factor * sy.occ.sum() / sy.nk - 32.0) < 1e-6
        n_max = int(np.abs(sy.gvec).max())
        assert sy.fft[0] == sy.fft[1] == sy.fft[2] and _smooth(sy.fft[0]) and sy.fft[0] >= 4 * n_max + 1


def test_batching_seeded_and_q_cap():
    a = make_batching_system(3, nq_max=1)
    b = make_batching_system(3)
    assert a.q_frac.shape[0] == 1 and np.array_equal(a.q_frac[0], b.q_frac[0])
    assert np.array_equal(a.coef, b.coef) and np.array_equal(a.eps, b.eps)
