"""Pins of the plasmon-pole fit in the oracle (Full frequency GW subsection):

1. a matrix whose elements are exactly single poles, x(w) = R [1/(w - wt) -
   1/(w + wt)], is recovered exactly (wt, R, and the values at any frequency);
2. for a general input (two poles per element) the model reproduces eps^-1 at
   the two fit frequencies exactly and differs elsewhere;
3. elements without a real pole (Re wt^2 <= 0, or no frequency dependence)
   are kept at their static value.
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
