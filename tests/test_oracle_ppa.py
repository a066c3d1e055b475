"""Pins of the plasmon-pole fit in the oracle (Full frequency GW subsection):

1. a matrix whose elements are exactly single poles, x(w) = R [1/(w - wt) -
   1/(w + wt)], is recovered exactly (wt, R, and the values at any frequency);
2. for a general input (two poles per element) the model reproduces eps^-1 at
   the two fit frequencies exactly and differs elsewhere;
3. elements without a real pole (Re wt^2 <= 0, or no frequency dependence)
   are kept at their static value;
4. the Drude (free-electron) dielectric function: the fit recovers the
   plasma frequency for any second fit point and reproduces eps^-1 everywhere.
"""
import numpy as np

import oracle as O


def _single_pole(n, seed=0):
    rng = np.random.default_rng(seed)
    wt = rng.uniform(0.3, 2.0, (n, n)) * np.exp(1j * rng.uniform(-0.3, 0.3, (n, n)))
    R = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return wt, R


def _model(wt, R, w):
    return R * (1.0 / (w - wt) - 1.0 / (w + wt))


def test_single_pole_recovered_exactly():
    n, wp = 6, 1.0
    wt, R = _single_pole(n)
    eye = np.eye(n)
    e0 = eye + _model(wt, R, 0.0)
    ep = eye + _model(wt, R, 1j * wp)
    fwt, fR = O.ppa_fit(e0, ep, wp)
    assert np.allclose(fwt, wt, rtol=1e-12, atol=0)
    assert np.allclose(fR, R, rtol=1e-11, atol=0)
    freqs = np.array([0.4j, 2.5j, 0.7 + 0.05j])
    want = np.stack([eye + _model(wt, R, w) for w in freqs])
    got = O.ppa_eval(fwt, fR, freqs, 0.0)
    assert np.allclose(got, want, rtol=1e-11, atol=1e-12)


def test_two_fit_points_reproduced():
    n, wp = 5, 1.0
    a_wt, a_R = _single_pole(n, 1)
    b_wt, b_R = _single_pole(n, 2)
    eye = np.eye(n)
    ev = lambda w: eye + _model(a_wt, a_R, w) + 0.3 * _model(3.0 * b_wt, b_R, w)  # noqa: E731
    wt, R = O.ppa_fit(ev(0.0), ev(1j * wp), wp)
    fit = O.ppa_eval(wt, R, [0.0, 1j * wp, 3j], 0.0)
    static = wt == 0
    assert np.allclose(fit[0], ev(0.0), rtol=1e-12, atol=1e-12)
    assert np.allclose(fit[1][~static], ev(1j * wp)[~static], rtol=1e-11, atol=1e-12)
    assert np.abs(fit[2] - ev(3j)).max() > 1e-3


def test_elements_without_a_real_pole_stay_static():
    eye = np.eye(2)
    e0 = eye + np.array([[0.5, 0.2], [0.2, -0.1]])
    ep = eye + np.array([[0.5, 0.4], [0.1, -0.05]])  # (0,0): no change; (0,1): wt^2 < 0
    wt, R = O.ppa_fit(e0, ep, 1.0)
    assert wt[0, 0] == 0 and R[0, 0] == 0.5
    assert wt[0, 1] == 0 and R[0, 1] == 0.2
    assert wt[1, 0] != 0 and wt[1, 1] != 0
    out = O.ppa_eval(wt, R, [0.0, 2j], 0.0)
    assert out[0][0, 0] == 1.5 and out[1][0, 1] == 0.2



def test_drude_plasma_frequency_recovered():
    """The free-electron (Drude) dielectric function eps = 1 - Omega^2 / w^2 has
    eps^-1(i nu) = nu^2 / (nu^2 + Omega^2): one plasmon at the plasma frequency
    Omega.  With one Drude element per diagonal entry (and none off the
    diagonal), the two-point fit must return wt = Omega whatever the second
    point, keep the off-diagonal zeros static, and reproduce
    eps^-1 = 1 + Omega^2 / (w^2 - Omega^2) at any frequency."""
    Omega = np.array([0.35, 0.8, 1.3, 2.6])
    eye = np.eye(Omega.size)
    for wp in (0.5, 1.0, 3.0):
        e0 = np.zeros((Omega.size, Omega.size), complex)                 # eps^-1(0) = 0 on the diagonal
        ep = np.diag(wp ** 2 / (wp ** 2 + Omega ** 2)).astype(complex)   # eps^-1(i wp)
        wt, R = O.ppa_fit(e0, ep, wp)
        assert np.allclose(np.diag(wt), Omega, rtol=1e-12, atol=0)
        assert np.all(wt[~eye.astype(bool)] == 0) and np.all(R[~eye.astype(bool)] == 0)
        w = np.array([0.1, 0.9, 4.0, 0.6j]) + 1e-3j
        model = O.ppa_eval(wt, R, w, 0.0)
        for k, wk in enumerate(w):
            want = eye + np.diag(Omega ** 2 / (wk ** 2 - Omega ** 2))
            assert np.allclose(model[k], want, rtol=1e-10, atol=1e-12)
