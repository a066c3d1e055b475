"""Godby-Needs plasmon-pole model of eps^-1 (oracle; test infrastructure).

The Full frequency GW subsection fits a plasmon-pole model to eps^-1_GG'
at two frequencies, w = 0 and w = i w_p (PPAPntXp, default 1 Ha).  Per
element, with x(w) = eps^-1_GG'(w) - delta_GG', the single-pole form (in the
retarded convention of the rest of this oracle)

    x(w) = R [1/(w - wt + i eta) - 1/(w + wt + i eta)]

equals -2 R wt / (nu^2 + wt^2) at w = i nu (eta = 0), so the two fit
conditions give

    wt^2 = w_p^2 x(i w_p) / (x(0) - x(i w_p)),   R = -x(0) wt / 2,

wt the principal square root.  Where Re wt^2 <= 0 or x(0) = x(i w_p) the
model has no real pole; such an element is kept frequency independent,
marked by wt = 0 with R = x(0).
"""
from __future__ import annotations

import numpy as np


def ppa_fit(eps_inv_0, eps_inv_p, omega_p):
    """(wt, R) per element from eps^-1 at w = 0 and w = i omega_p (square matrices)."""
    e0 = np.asarray(eps_inv_0, dtype=np.complex128)
    ep = np.asarray(eps_inv_p, dtype=np.complex128)
    eye = np.eye(e0.shape[0])
    x0 = e0 - eye
    xp = ep - eye
    den = x0 - xp
    wt2 = np.zeros_like(x0)
    ok = den != 0
    wt2[ok] = omega_p ** 2 * xp[ok] / den[ok]
    ok &= wt2.real > 0
    wt = np.where(ok, np.sqrt(np.where(ok, wt2, 1.0)), 0.0)
    R = np.where(ok, -x0 * wt / 2.0, x0)
    return wt, R


def ppa_eval(wt, R, freqs, eta):
    """eps^-1[iw] of the model at complex frequencies freqs."""
    wt = np.asarray(wt, dtype=np.complex128)
    R = np.asarray(R, dtype=np.complex128)
    eye = np.eye(wt.shape[0])
    out = []
    static = wt == 0
    for w in np.asarray(freqs, dtype=np.complex128):
        with np.errstate(divide="ignore", invalid="ignore"):
            x = R * (1.0 / (w - wt + 1j * eta) - 1.0 / (w + wt + 1j * eta))
        out.append(eye + np.where(static, R, x))
    return np.stack(out)
