"""Bruneval-Gonze extrapolar correction to chi0, the X-terminator (oracle;
test infrastructure).

Eq. (X_term_def): chi0 = chi0^trunc + Delta chi(eps_bar), with Delta chi
given in Appendix C (Eqs. rhotw-term, F-term, X-term).  The bands that the
truncated sum leaves out are given one common energy eps_bar (the extrapolar
energy) and no occupation.  Their contribution then needs no wavefunctions:
by the closure relation over all bands at k,

    sum_{n >= nb} rho_nm(G) conj(rho_nm(G'))
        = rho~_m(G - G') - sum_{n < nb} rho_nm(G) conj(rho_nm(G')),

where rho~_{m,k'}(d) = < m k' | e^{i d.r} | m k' > is the diagonal density of
the state m at k' = k - q (Eq. rhotw-term; see the readings for the sign of
the argument).  Hence

    Delta chi_GG'(w) = sum_{k, m} wbar_{m,k-q}(w)
        [ rho~_{m,k-q}(G - G') - sum_{n < nb} rho_{nmk}(G) conj(rho_{nmk}(G')) ],

with wbar the two-pole frequency factor of chi0_tr for a transition from m
into a state at eps_bar (Eq. F-term, in the convention of weights_tr):

    wbar_{mk'}(w) = f_s/(N_k Omega) f_{mk'} [1/(w + dbar + i eta) - 1/(w - dbar + i eta)],
    dbar = eps_{mk'} - eps_bar.

The subtraction runs over every band n < nb at k, occupied ones included:
the closure relation sums over all of them.
"""
from __future__ import annotations

import numpy as np

from .chi0 import _prefactor, chi0_tr
from .geometry import kpair_map
from .rho import rho_block, rho_pair


def diag_density(system, ik, bands, ds):
    """rho~[b, i] = < m k | e^{i d_i.r} | m k > = sum_{G''} conj(c_m(G'' + d_i)) c_m(G'')
    for the states m = bands[b] at k = ik (Eq. rhotw-term; direct convolution)."""
    g = system.sphere(ik)
    c = system.coefs(ik)
    ds = np.asarray(ds, dtype=np.int64)
    out = np.zeros((len(bands), ds.shape[0]), dtype=np.complex128)
    for b, m in enumerate(bands):
        cm = c[[int(m)]]
        out[b] = rho_pair(g, cm, g, cm, ds, np.zeros(3, dtype=np.int64))[0, 0]
    return out


def extrapolar_weights(system, freqs, eta, eps_bar, occ_tol=0.0):
    """wbar[iw, k, m]: the frequency factor of a transition from m at k into an
    empty state at eps_bar (Eq. F-term), times f_s/(N_k Omega) f_mk; zero where
    f_mk <= occ_tol."""
    freqs = np.asarray(freqs, dtype=np.complex128)
    dbar = system.eps - eps_bar                                   # (nk, nb)
    f = np.where(system.occ > occ_tol, system.occ, 0.0)
    w = freqs[:, None, None]
    poles = 1.0 / (w + dbar[None] + 1j * eta) - 1.0 / (w - dbar[None] + 1j * eta)
    return _prefactor(system) * f[None] * poles


def delta_chi_bg(system, iq, Gs, freqs, eta, eps_bar, occ_tol=0.0):
    """Delta chi[iw, i, j] of Eq. (X-term) in the closure form above."""
    freqs = np.asarray(freqs, dtype=np.complex128)
    Gs = np.asarray(Gs, dtype=np.int64)
    nG = Gs.shape[0]
    ikp, _ = kpair_map(system.spec.kgrid, system.q_frac[iq])
    wbar = extrapolar_weights(system, freqs, eta, eps_bar, occ_tol)   # (nw, nk, nb)
    diff = Gs[:, None, :] - Gs[None, :, :]                            # G_i - G_j
    dchi = np.zeros((freqs.size, nG, nG), dtype=np.complex128)
    all_n = np.arange(system.nb)
    for ik in range(system.nk):
        jk = int(ikp[ik])
        ms = np.nonzero(system.occ[jk] > occ_tol)[0]
        if ms.size == 0:
            continue
        rt = diag_density(system, jk, ms, diff.reshape(-1, 3)).reshape(ms.size, nG, nG)
        rho = rho_block(system, iq, Gs, ik, all_n, ms, shifted=True)  # [n, m, i]
        inc = np.einsum("nmi,nmj->mij", rho, np.conj(rho))            # sum over all n < nb
        for iw in range(freqs.size):
            dchi[iw] += np.einsum("m,mij->ij", wbar[iw, jk, ms], rt - inc)
    return dchi


def chi0_bg(system, iq, Gs, freqs, eta, eps_bar, occ_tol=0.0):
    """chi0 with the extrapolar correction: Eq. (X_term_def)."""
    return (chi0_tr(system, iq, Gs, freqs, eta, occ_tol)
            + delta_chi_bg(system, iq, Gs, freqs, eta, eps_bar, occ_tol))
