"""k-point bookkeeping, the response G set and |q+G| (oracle; test infrastructure).

* k - q is folded back to the grid: k - q = k' + G0 with k' in [0,1)^3
  (reduced coordinates) and G0 an integer vector (the umklapp shift).  States
  at k - q are taken in the periodic gauge psi_{k'+G0} = psi_{k'}, which is the
  reading of the paper's k - q labels in Eq. (rhotw).
* The response G set is the N_G vectors of smallest |q+G| (the "cutoff" of the
  response function, a convergence parameter of the linear-response
  runlevel).  Ties in |q+G| are broken by ascending (Gx, Gy, Gz); |q+G|^2 is
  compared in exact integer arithmetic.
* The bare Coulomb interaction is v(q+G) = 4 pi / |q+G|^2 (Coulomb
  interaction subsection); |q+G| is in bohr^-1 for a cubic cell of edge a.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def _grid_index(kfrac, kgrid):
    return tuple(int(round(kfrac[a] * kgrid[a])) for a in range(3))


def kpair_map(kgrid, q_frac):
    """For every k of the grid (ordered i-major), return (ik', G0) with
    k - q = k' + G0.  q must be a vector of the k grid."""
    n = [int(v) for v in kgrid]
    qi = []
    for a in range(3):
        x = q_frac[a] * n[a]
        if abs(x - round(x)) > 1e-9:
            raise ValueError("q is not a vector of the k grid")
        qi.append(int(round(x)))
    nk = n[0] * n[1] * n[2]
    ikp = np.zeros(nk, dtype=np.int64)
    g0 = np.zeros((nk, 3), dtype=np.int64)
    for i in range(n[0]):
        for j in range(n[1]):
            for l in range(n[2]):
                ik = (i * n[1] + j) * n[2] + l
                src = (i - qi[0], j - qi[1], l - qi[2])
                rep = [src[a] % n[a] for a in range(3)]
                # (src / n) = (rep / n) + G0  =>  G0 = (src - rep) / n
                g0[ik] = [(src[a] - rep[a]) // n[a] for a in range(3)]
                ikp[ik] = (rep[0] * n[1] + rep[1]) * n[2] + rep[2]
    return ikp, g0


def response_gvectors(kgrid, q_frac, ng):
    """The ng integer vectors G of smallest |q+G| (cubic cell), ties broken by
    ascending (Gx, Gy, Gz)."""
    qfr = [Fraction(round(q_frac[a] * kgrid[a]), int(kgrid[a])) for a in range(3)]
    radius = (3.0 * ng / (4.0 * math.pi)) ** (1.0 / 3.0) + 3.0
    m = int(math.ceil(radius))
    cands = []
    for gx in range(-m, m + 1):
        for gy in range(-m, m + 1):
            for gz in range(-m, m + 1):
                d = (qfr[0] + gx) ** 2 + (qfr[1] + gy) ** 2 + (qfr[2] + gz) ** 2
                cands.append((d, gx, gy, gz))
    cands.sort()
    chosen = cands[:ng]
    # every vector outside the searched cube has |q+G| >= m - 1 > the largest chosen
    assert chosen[-1][0] < (m - 1) ** 2
    return np.array([[c[1], c[2], c[3]] for c in chosen], dtype=np.int64)


def qg_norms(a, q_frac, gvecs):
    """|q+G| in bohr^-1 for a cubic cell of edge a."""
    v = (np.asarray(q_frac, dtype=np.float64)[None, :] + np.asarray(gvecs, dtype=np.float64))
    return (2.0 * math.pi / a) * np.sqrt((v * v).sum(axis=1))
