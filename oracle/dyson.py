"""Dyson step: symmetric dielectric matrix and its inverse (oracle; test infrastructure).

Local fields enter through Eq. (X_rpa): chi^RPA = chi0 + chi0 v chi^RPA with
the bare Coulomb interaction v(q+G) = 4 pi / |q+G|^2; Eq. (X_rpa_inv) writes
the solution as chi^RPA = [1 - chi0 v]^-1 chi0.  The symmetric dielectric
matrix uses V = diag(sqrt(4 pi) / |q+G_i|) (the same symmetrisation as
W = eps^-1 4 pi / (|q+G||q+G'|), Eq. (W_def)):

    eps~    = 1 - V chi0 V,
    eps~^-1 = 1 + V chi^RPA V.

Two independent routes are given: Gauss-Jordan inversion of eps~ with partial
pivoting (written out row by row), and the linear solve of Eq. (X_rpa_inv)
followed by the second identity.
"""
from __future__ import annotations

import math

import numpy as np


def coulomb_sqrt(qg_norm):
    """V_i = sqrt(4 pi) / |q+G_i| (bohr^-1 in, atomic units out)."""
    qg_norm = np.asarray(qg_norm, dtype=np.float64)
    if np.any(qg_norm == 0.0):
        raise ValueError("|q+G| = 0: the bare Coulomb interaction diverges")
    return math.sqrt(4.0 * math.pi) / qg_norm


def eps_tilde(chi0, qg_norm):
    """eps~ = 1 - V chi0 V for one frequency (chi0 is N x N)."""
    v = coulomb_sqrt(qg_norm)
    n = chi0.shape[0]
    return np.eye(n, dtype=np.complex128) - v[:, None] * chi0 * v[None, :]


def gauss_jordan_inverse(a):
    """Inverse of a square matrix by Gauss-Jordan elimination with partial
    pivoting on the augmented matrix [a | 1]."""
    a = np.array(a, dtype=np.complex128)
    n = a.shape[0]
    aug = np.concatenate([a, np.eye(n, dtype=np.complex128)], axis=1)
    for col in range(n):
        piv = col + int(np.argmax(np.abs(aug[col:, col])))
        if aug[piv, col] == 0:
            raise np.linalg.LinAlgError("singular matrix")
        if piv != col:
            aug[[col, piv]] = aug[[piv, col]]
        aug[col] = aug[col] / aug[col, col]
        for row in range(n):
            if row != col and aug[row, col] != 0:
                aug[row] = aug[row] - aug[row, col] * aug[col]
    return aug[:, n:]


def eps_inv_gauss_jordan(chi0, qg_norm):
    """eps~^-1 for one frequency by Gauss-Jordan inversion of eps~."""
    return gauss_jordan_inverse(eps_tilde(chi0, qg_norm))


def eps_inv_rpa_route(chi0, qg_norm):
    """eps~^-1 = 1 + V chi^RPA V with chi^RPA = [1 - chi0 v]^-1 chi0."""
    v = coulomb_sqrt(qg_norm)
    n = chi0.shape[0]
    vv = v * v  # 4 pi / |q+G|^2
    chi_rpa = np.linalg.solve(np.eye(n) - chi0 * vv[None, :], chi0)
    return np.eye(n, dtype=np.complex128) + v[:, None] * chi_rpa * v[None, :]
