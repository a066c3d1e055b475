"""Oscillator strengths rho_{nmk}(q,G) (oracle; test infrastructure).

Eq. (rhotw), Linear Response section:

    rho_{nmk}(q,G) = < n k | e^{i(q+G).r} | m k-q >.

With psi_{nk}(r) = Omega^-1/2 sum_{G in S_k} c_{nk}(G) e^{i(k+G).r}, the
integral over the cell keeps only the plane-wave pairs whose momenta match.
Writing k - q = k' + G0 (k' on the grid, G0 the umklapp vector) and using the
periodic gauge psi_{k'+G0} = psi_{k'}:

    rho_{nmk}(q,G) = sum_{G'' in S_k'} conj(c_{nk}(G + G'' - G0)) c_{mk'}(G''),

with c_{nk} = 0 outside S_k.  This is the "direct plane-wave convolution"
used here; there is no FFT anywhere in the oracle.  The substitution
g = G + G'' - G0 gives the equivalent sum over S_k,

    rho_{nmk}(q,G) = sum_{g in S_k} conj(c_{nk}(g)) c_{mk'}(g - G + G0),

which moves the index lookup onto the k' states (cheaper when there are fewer
of them); tests check that both orders agree.
"""
from __future__ import annotations

import numpy as np

from .geometry import kpair_map


class _SphereIndex:
    """Position of an integer vector inside a plane-wave sphere (or -1)."""

    def __init__(self, g):
        g = np.asarray(g, dtype=np.int64)
        self.lo = g.min(axis=0) - 1
        hi = g.max(axis=0) + 1
        self.shape = tuple((hi - self.lo + 1).tolist())
        self.table = -np.ones(self.shape, dtype=np.int64)
        p = g - self.lo
        self.table[p[:, 0], p[:, 1], p[:, 2]] = np.arange(g.shape[0])

    def find(self, v):
        v = np.asarray(v, dtype=np.int64)
        p = v - self.lo
        inside = np.all((p >= 0) & (p < np.array(self.shape)), axis=-1)
        out = -np.ones(v.shape[:-1], dtype=np.int64)
        pi = p[inside]
        out[inside] = self.table[pi[..., 0], pi[..., 1], pi[..., 2]]
        return out


def rho_pair(gn, cn, gm, cm, Gs, G0):
    """rho[n, m, i] = sum_{G'' in S_m} conj(c_n(G_i + G'' - G0)) c_m(G'').

    gn (npw_n,3), cn (Nn, npw_n): sphere and coefficients of the states at k;
    gm (npw_m,3), cm (Nm, npw_m): same at k'.  Direct convolution, one G at a
    time, with the lookup written out per plane wave G''."""
    gn = np.asarray(gn, dtype=np.int64)
    gm = np.asarray(gm, dtype=np.int64)
    cn = np.asarray(cn, dtype=np.complex128)
    cm = np.asarray(cm, dtype=np.complex128)
    G0 = np.asarray(G0, dtype=np.int64)
    where = {tuple(v): i for i, v in enumerate(gn.tolist())}
    out = np.zeros((cn.shape[0], cm.shape[0], len(Gs)), dtype=np.complex128)
    for i, G in enumerate(np.asarray(Gs, dtype=np.int64)):
        a = np.zeros((cn.shape[0], gm.shape[0]), dtype=np.complex128)
        for j, gpp in enumerate(gm):
            pos = where.get(tuple((G + gpp - G0).tolist()))
            if pos is not None:
                a[:, j] = np.conj(cn[:, pos])
        out[:, :, i] = a @ cm.T
    return out


def rho_pair_shifted(gn, cn, gm, cm, Gs, G0):
    """Same result as rho_pair, summed over g in S_n with the lookup of
    g - G + G0 in S_m (vectorised over g)."""
    gn = np.asarray(gn, dtype=np.int64)
    cn = np.asarray(cn, dtype=np.complex128)
    cm = np.asarray(cm, dtype=np.complex128)
    G0 = np.asarray(G0, dtype=np.int64)
    idx_m = _SphereIndex(gm)
    Gs = np.asarray(Gs, dtype=np.int64)
    nG = Gs.shape[0]
    # b[i, m, g] = c_m(g - G_i + G0) (zero outside S_m)
    pos = idx_m.find(gn[None, :, :] - Gs[:, None, :] + G0[None, None, :])  # (nG, npw_n)
    cm_pad = np.concatenate([cm, np.zeros((cm.shape[0], 1), dtype=np.complex128)], axis=1)
    b = cm_pad[:, np.where(pos >= 0, pos, cm.shape[1])]            # (Nm, nG, npw_n)
    # rho[n, m, i] = sum_g conj(c_n(g)) b[m, i, g]
    out = np.conj(cn) @ b.reshape(cm.shape[0] * nG, -1).T            # (Nn, Nm*nG)
    return out.reshape(cn.shape[0], cm.shape[0], nG)


def rho_block(system, iq, Gs, ik, n_bands, m_bands, shifted=False):
    """rho[n, m, i] for the states n (at k = ik) and m (at k - q)."""
    ikp, g0 = kpair_map(system.spec.kgrid, system.q_frac[iq])
    jk = int(ikp[ik])
    n_bands = np.asarray(n_bands, dtype=np.int64)
    m_bands = np.asarray(m_bands, dtype=np.int64)
    f = rho_pair_shifted if shifted else rho_pair
    return f(system.sphere(ik), system.coefs(ik)[n_bands], system.sphere(jk),
             system.coefs(jk)[m_bands], Gs, g0[ik])


def rho_transitions(system, iq, Gs, trans, shifted=True):
    """rho for an explicit list of transitions trans[t] = (ik, n, m); returns
    (nt, nG) complex128 in the order of trans."""
    trans = np.asarray(trans, dtype=np.int64)
    out = np.zeros((trans.shape[0], len(Gs)), dtype=np.complex128)
    for ik in np.unique(trans[:, 0]):
        sel = np.nonzero(trans[:, 0] == ik)[0]
        ns = np.unique(trans[sel, 1])
        ms = np.unique(trans[sel, 2])
        blk = rho_block(system, iq, Gs, int(ik), ns, ms, shifted=shifted)
        ni = np.searchsorted(ns, trans[sel, 1])
        mi = np.searchsorted(ms, trans[sel, 2])
        out[sel] = blk[ni, mi, :]
    return out


def rho_realspace_bruteforce(system, iq, Gs, ik, n, m, ngrid):
    """rho_{nmk}(q,G) as a Riemann sum of psi*_{nk} e^{i(q+G).r} psi_{m,k-q}
    over an ngrid^3 real-space mesh, with every orbital evaluated by its
    explicit plane-wave sum.  The integrand is cell periodic with integer
    frequencies bounded by the sphere radii, so the sum is exact once ngrid
    exceeds twice the largest frequency."""
    ikp, g0 = kpair_map(system.spec.kgrid, system.q_frac[iq])
    jk = int(ikp[ik])
    k = system.kfrac[ik]
    kp = system.kfrac[jk]
    q = system.q_frac[iq]
    t = np.arange(ngrid) / ngrid
    r = np.stack(np.meshgrid(t, t, t, indexing="ij"), axis=-1).reshape(-1, 3)  # reduced
    two_pi_i = 2j * np.pi

    def orbital(kvec, g, c):
        ph = np.exp(two_pi_i * (r @ (kvec[None, :] + g).T))  # (Nr, npw)
        return ph @ c

    psi_n = orbital(k, system.sphere(ik).astype(np.float64), system.coefs(ik)[n])
    psi_m = orbital(kp, system.sphere(jk).astype(np.float64), system.coefs(jk)[m])
    # the state at k - q is psi_{k'} (periodic gauge); q + G is taken literally
    out = np.zeros(len(Gs), dtype=np.complex128)
    for i, G in enumerate(np.asarray(Gs, dtype=np.float64)):
        ph = np.exp(two_pi_i * (r @ (q + G)))
        out[i] = np.mean(np.conj(psi_n) * ph * psi_m)
    return out
