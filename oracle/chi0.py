"""Independent-particle polarizability chi0_{GG'}(q,w) (oracle; test infrastructure).

Eq. (X_IP) of the Linear Response section gives chi0 as a sum over k and
band pairs of rho rho^* times a two-pole frequency factor, with prefactor
f_s / (N_k Omega) (f_s = 2 without spin polarisation).  Appendix B splits it
into frequency factors F_{nmk}(w) and frequency-independent matrices
R^{nmk}_{GG'}.  The band/k labels and the sign of i*eta differ between the
paper's equations; the oracle uses the self-consistent reading below (it
agrees with Eq. (rhotw): n at k, m at k - q):

all ordered pairs ("Adler-Wiser" form)
    chi0_ij(w) = f_s/(N_k Omega) sum_k sum_{n,m} rho_{nmk}(G_i) conj(rho_{nmk}(G_j))
                 (f_{m,k-q} - f_{n,k}) / (w + eps_{m,k-q} - eps_{n,k} + i eta)

time-reversal two-pole form (pairs with f_{m,k-q} > f_{n,k} only)
    w_t(w) = f_s/(N_k Omega) (f_m - f_n) [1/(w + D + i eta) - 1/(w - D + i eta)],
    D = eps_{m,k-q} - eps_{n,k},   chi0 = sum_t w_t rho_t rho_t^H.

+i eta on both poles is the retarded convention; on the imaginary axis
(eta = 0) every convention gives the same chi0.  The two forms agree when the
states obey time reversal (tests check this).
"""
from __future__ import annotations

import numpy as np

from .geometry import kpair_map
from .rho import rho_block


def _prefactor(system):
    return system.spin_factor / (system.nk * system.omega_cell)


def transitions_tr(system, iq, occ_tol=0.0):
    """Transitions t = (ik, n, m): n at k, m at k - q, f_{m,k-q} - f_{n,k} > occ_tol.
    Ordered by k, then n, then m."""
    ikp, _ = kpair_map(system.spec.kgrid, system.q_frac[iq])
    out = []
    for ik in range(system.nk):
        # df[n, m] = f_{m,k-q} - f_{n,k}
        df = system.occ[ikp[ik]][None, :] - system.occ[ik][:, None]
        n, m = np.nonzero(df > occ_tol)          # row-major: n, then m
        out.append(np.stack([np.full(n.size, ik), n, m], axis=1))
    return np.concatenate(out, axis=0).astype(np.int64).reshape(-1, 3)


def weights_tr(system, iq, trans, freqs, eta):
    """w[iw, t] of the time-reversal two-pole form (Appendix B frequency factor
    times the occupation factor and prefactor)."""
    ikp, _ = kpair_map(system.spec.kgrid, system.q_frac[iq])
    trans = np.asarray(trans, dtype=np.int64)
    ik, n, m = trans[:, 0], trans[:, 1], trans[:, 2]
    jk = ikp[ik]
    df = system.occ[jk, m] - system.occ[ik, n]
    d = system.eps[jk, m] - system.eps[ik, n]
    w = np.asarray(freqs, dtype=np.complex128)[:, None]
    poles = 1.0 / (w + d[None, :] + 1j * eta) - 1.0 / (w - d[None, :] + 1j * eta)
    return _prefactor(system) * df[None, :] * poles


def chi0_tr(system, iq, Gs, freqs, eta, occ_tol=0.0, ks=None):
    """chi0[iw, i, j] = sum_t w_t(w) rho_t(G_i) conj(rho_t(G_j)) over the
    time-reversal transitions (optionally only those with k in ks)."""
    freqs = np.asarray(freqs, dtype=np.complex128)
    ikp, _ = kpair_map(system.spec.kgrid, system.q_frac[iq])
    nG = len(Gs)
    chi = np.zeros((freqs.size, nG, nG), dtype=np.complex128)
    trans = transitions_tr(system, iq, occ_tol)
    klist = range(system.nk) if ks is None else ks
    for ik in klist:
        sel = trans[trans[:, 0] == ik]
        if sel.shape[0] == 0:
            continue
        ns = np.unique(sel[:, 1])
        ms = np.unique(sel[:, 2])
        blk = rho_block(system, iq, Gs, ik, ns, ms, shifted=True)
        rho = blk[np.searchsorted(ns, sel[:, 1]), np.searchsorted(ms, sel[:, 2]), :]  # (nt, nG)
        w = weights_tr(system, iq, sel, freqs, eta)                                   # (nw, nt)
        for iw in range(freqs.size):   # chi(w) += (w_t rho_t(G_i)) rho_t(G_j)^*
            chi[iw] += (rho.T * w[iw][None, :]) @ np.conj(rho)
    return chi


def chi0_all_pairs(system, iq, Gs, freqs, eta):
    """chi0 from the sum over all ordered band pairs (no occupation filter)."""
    freqs = np.asarray(freqs, dtype=np.complex128)
    ikp, _ = kpair_map(system.spec.kgrid, system.q_frac[iq])
    nG = len(Gs)
    bands = np.arange(system.nb)
    chi = np.zeros((freqs.size, nG, nG), dtype=np.complex128)
    for ik in range(system.nk):
        jk = ikp[ik]
        rho = rho_block(system, iq, Gs, ik, bands, bands)          # (nb, nb, nG): [n, m, i]
        df = system.occ[jk][None, :] - system.occ[ik][:, None]     # [n, m] = f_m - f_n
        de = system.eps[jk][None, :] - system.eps[ik][:, None]     # [n, m] = e_m - e_n
        for iw, w in enumerate(freqs):
            fac = df / (w + de + 1j * eta)                          # [n, m]
            chi[iw] += np.einsum("nm,nmi,nmj->ij", fac, rho, np.conj(rho))
    return chi * _prefactor(system)


def chi0_lindhard_plane_waves(system, iq, Gs, freqs, eta, e_fermi):
    """Closed form for a system whose every state is one plane wave
    (c_{nk}(G) = 1 on a single G, eps = |k+G|^2/2, f = 1 below e_fermi).

    Then rho_{nmk}(G) is 1 exactly when k+G_n = (k'+G_m) + q + G (umklapp
    included), so chi0 is diagonal and
        chi0_GG = f_s/(N_k Omega) sum_{p'} (f(p') - f(p'+q+G)) /
                  (w + |p'|^2/2 - |p'+q+G|^2/2 + i eta),
    p' running over the plane waves held at the k' points whose partner
    p'+q+G is held at k.  Evaluated from momenta only (no rho)."""
    freqs = np.asarray(freqs, dtype=np.complex128)
    a = system.spec.a
    b = 2.0 * np.pi / a
    ikp, _ = kpair_map(system.spec.kgrid, system.q_frac[iq])
    q = system.q_frac[iq]
    nG = len(Gs)
    chi = np.zeros((freqs.size, nG, nG), dtype=np.complex128)
    for ik in range(system.nk):
        jk = ikp[ik]
        # the plane wave of each band (the position of the unit coefficient)
        gk = system.sphere(ik)[np.argmax(np.abs(system.coefs(ik)), axis=1)]
        gkp = system.sphere(jk)[np.argmax(np.abs(system.coefs(jk)), axis=1)]
        held_k = {tuple((system.kfrac[ik] + g).round(9).tolist()) for g in gk.astype(np.float64)}
        for gm in gkp.astype(np.float64):
            pprime = system.kfrac[jk] + gm  # momentum of the state at k - q = k' + G0
            for i, G in enumerate(np.asarray(Gs, dtype=np.float64)):
                p = pprime + q + G          # momentum it is scattered to, held at k?
                if tuple(p.round(9).tolist()) not in held_k:
                    continue
                e1 = 0.5 * b * b * float((pprime ** 2).sum())
                e2 = 0.5 * b * b * float((p ** 2).sum())
                f1 = 1.0 if e1 < e_fermi else 0.0
                f2 = 1.0 if e2 < e_fermi else 0.0
                chi[:, i, i] += (f1 - f2) / (freqs + e1 - e2 + 1j * eta)
    return chi * _prefactor(system)
