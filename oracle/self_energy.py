"""Screened interaction W, its delta-like part W^delta and the self-energy
kernel I of the full-frequency GW step (oracle; test infrastructure).

Eq. (W_def): W_GG'(q,w) = eps^-1_GG'(q,w) 4 pi / (|q+G| |q+G'|).  The
matrix eps^-1 of that equation is the symmetric one: with V = diag(sqrt(4 pi)
/ |q+G|) it reads W = V eps~^-1 V, eps~^-1 = (1 - V chi0 V)^-1 (the Dyson
step of this oracle).

Eq. (W_delta): the delta-like part, built element by element from the real
and imaginary parts of W_GG' and W_G'G,

    W^d_GG' = 1/2 Im(W_GG' + W_G'G) - i/2 Re(W_GG' - W_G'G).

Eq. (I_c): for the states n, n' at k and every band m at k - q,

    I^{nn'k}_{mq}(w) = -1/(N_k Omega) sum_{G,G'} W^d_GG'(q,w) rho_{nmk}(q,G) rho*_{n'mk}(q,G'),

with rho of Eq. (rhotw) (n at k, m at k - q, as for chi0).
"""
from __future__ import annotations

import numpy as np

from .dyson import coulomb_sqrt
from .rho import rho_block


def screened_w(eps_inv, qg_norm):
    """W = V eps~^-1 V for one frequency (Eq. W_def, symmetric form)."""
    v = coulomb_sqrt(qg_norm)
    return v[:, None] * np.asarray(eps_inv, dtype=np.complex128) * v[None, :]


def w_delta(W):
    """Eq. (W_delta), term by term: real and imaginary parts of W and W^T."""
    W = np.asarray(W, dtype=np.complex128)
    Wt = W.T
    return 0.5 * (W.imag + Wt.imag) - 0.5j * (W.real - Wt.real)


def i_kernel(system, iq, Gs, qp_bands, Wd, ks=None, ms=None):
    """I[k, m, a, b] = I^{n_a n_b k}_{m q} of Eq. (I_c) for one frequency.

    qp_bands: the band indices n at k (n_a, n_b run over them); ks: the k
    indices (default all); ms: the bands m at k - q (default all).  Wd:
    W^delta on the G vectors Gs (N_G x N_G)."""
    ks = range(system.nk) if ks is None else ks
    qp_bands = np.asarray(qp_bands, dtype=np.int64)
    ms = np.arange(system.nb) if ms is None else np.asarray(ms, dtype=np.int64)
    Wd = np.asarray(Wd, dtype=np.complex128)
    pref = -1.0 / (system.nk * system.omega_cell)
    out = np.zeros((len(ks), ms.size, qp_bands.size, qp_bands.size), dtype=np.complex128)
    for j, ik in enumerate(ks):
        rho = rho_block(system, iq, Gs, int(ik), qp_bands, ms, shifted=True)      # [n, m, G]
        for jm in range(ms.size):
            r = rho[:, jm, :]                                                     # [n, G]
            out[j, jm] = pref * (r @ Wd @ np.conj(r).T)
    return out
