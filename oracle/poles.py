"""Degenerate-pole grouping and the double-grid frequency factor (oracle;
test infrastructure).

Appendix B splits chi0 into frequency factors F(w) of the pole energies and
frequency-independent R = rho rho^* terms (Eqs. X_IP_split, split1, split2),
and lets poles whose energies differ by less than eps_thresh share the factor
of one member of their group.  Grouping rule used here (greedy, on the pole
energies d_t = eps_{m,k-q} - eps_{n,k} of the contributing transitions):
sort them (stable in the transition order); a group opens at the smallest
pole not yet taken, which is its representative, and takes every following
pole with d_t - d_rep < eps_thresh.  eps_thresh = 0 leaves every pole alone.

The double grid (Bethe-Salpeter section, last paragraph on the dense grid)
replaces the frequency factor of each transition by the mean over the nd
transitions of the dense grid around it, F_t(w) -> 1/nd sum_j F(w; d_t^j),
d_t^j = eps^j_{m,k-q} - eps^j_{n,k} from the dense energies (sub-point j of
each coarse k); the occupation factor of R stays that of the coarse grid.
"""
from __future__ import annotations

import numpy as np

from .chi0 import _prefactor, transitions_tr
from .geometry import kpair_map
from .rho import rho_block


def pole_energies(system, iq, trans):
    """d_t = eps_{m,k-q} - eps_{n,k} for the transitions trans[t] = (ik, n, m)."""
    ikp, _ = kpair_map(system.spec.kgrid, system.q_frac[iq])
    trans = np.asarray(trans, dtype=np.int64)
    ik, n, m = trans[:, 0], trans[:, 1], trans[:, 2]
    return system.eps[ikp[ik], m] - system.eps[ik, n]


def pole_groups(d, eps_thresh):
    """rep[t]: the representative transition of t's group (see the module
    docstring).  Written as a plain loop over the sorted poles."""
    d = np.asarray(d, dtype=np.float64)
    order = np.argsort(d, kind="stable")
    rep = np.empty(d.size, dtype=np.int64)
    i = 0
    while i < d.size:
        r = order[i]
        rep[r] = r
        j = i + 1
        while j < d.size and d[order[j]] - d[r] < eps_thresh:
            rep[order[j]] = r
            j += 1
        i = j
    return rep


def _two_pole(freqs, d, eta):
    """The time-reversal two-pole frequency factor of the chi0 weights."""
    w = np.asarray(freqs, dtype=np.complex128)[:, None]
    return 1.0 / (w + d[None, :] + 1j * eta) - 1.0 / (w - d[None, :] + 1j * eta)


def weights_grouped(system, iq, trans, freqs, eta, eps_thresh):
    """w[iw, t] with the frequency factor of each transition's group representative."""
    ikp, _ = kpair_map(system.spec.kgrid, system.q_frac[iq])
    trans = np.asarray(trans, dtype=np.int64)
    ik, n, m = trans[:, 0], trans[:, 1], trans[:, 2]
    df = system.occ[ikp[ik], m] - system.occ[ik, n]
    d = pole_energies(system, iq, trans)
    rep = pole_groups(d, eps_thresh)
    return _prefactor(system) * df[None, :] * _two_pole(freqs, d[rep], eta)


def weights_double_grid(system, iq, trans, freqs, eta, eps_dense):
    """w[iw, t] with the frequency factor averaged over the dense grid:
    eps_dense[k, j, b] is band b at dense sub-point j of coarse k."""
    ikp, _ = kpair_map(system.spec.kgrid, system.q_frac[iq])
    trans = np.asarray(trans, dtype=np.int64)
    ik, n, m = trans[:, 0], trans[:, 1], trans[:, 2]
    jk = ikp[ik]
    df = system.occ[jk, m] - system.occ[ik, n]
    eps_dense = np.asarray(eps_dense, dtype=np.float64)
    nd = eps_dense.shape[1]
    F = np.zeros((np.asarray(freqs).size, trans.shape[0]), dtype=np.complex128)
    for j in range(nd):
        F += _two_pole(freqs, eps_dense[jk, j, m] - eps_dense[ik, j, n], eta)
    return _prefactor(system) * df[None, :] * (F / nd)


def chi0_weighted(system, iq, Gs, trans, w):
    """chi0[iw] = sum_t w[iw, t] rho_t rho_t^H over the transitions trans."""
    trans = np.asarray(trans, dtype=np.int64)
    w = np.asarray(w)
    chi = np.zeros((w.shape[0], len(Gs), len(Gs)), dtype=np.complex128)
    for ik in np.unique(trans[:, 0]):
        sel = np.nonzero(trans[:, 0] == ik)[0]
        ns = np.unique(trans[sel, 1])
        ms = np.unique(trans[sel, 2])
        blk = rho_block(system, iq, Gs, int(ik), ns, ms, shifted=True)
        rho = blk[np.searchsorted(ns, trans[sel, 1]), np.searchsorted(ms, trans[sel, 2]), :]
        for iw in range(w.shape[0]):
            chi[iw] += (rho.T * w[iw, sel][None, :]) @ np.conj(rho)
    return chi


def chi0_grouped(system, iq, Gs, freqs, eta, eps_thresh, occ_tol=0.0):
    trans = transitions_tr(system, iq, occ_tol)
    return chi0_weighted(system, iq, Gs, trans, weights_grouped(system, iq, trans, freqs, eta, eps_thresh))


def chi0_double_grid(system, iq, Gs, freqs, eta, eps_dense, occ_tol=0.0):
    trans = transitions_tr(system, iq, occ_tol)
    return chi0_weighted(system, iq, Gs, trans, weights_double_grid(system, iq, trans, freqs, eta, eps_dense))
