"""Degenerate-pole grouping and the double-grid frequency factor on the GPU
(chi0_set_pole_grouping, chi0_set_double_grid; Appendix B and the dense-grid
paragraph) against the oracle.

1. Poles degenerate across k up to a splitting below the threshold: the
   grouped chi0 equals the oracle's within 1e-10 (FP64) / 1e-5 (mixed), on an
   imaginary- and real-axis frequency list; it differs from the plain chi0 by
   the amount the oracle gives.
2. The double grid with three dense points per k: chi0 and eps~^-1 equal the
   oracle's within the same tolerances.
3. Switching off restores the plain chi0 exactly; argument checks.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from synth import cfg_tiny, make_system

pytestmark = pytest.mark.gpu

FREQS = (0.05j, 0.6j, 0.4 + 0j)
ETA = 0.05


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0
    return chi0


def _sys(dtype):
    return make_system(cfg_tiny(seed=93, kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),), fft=(20, 20, 20), ng=45,
                                n_occ=5, n_bands=23, npw_target=90, a=8.0, freqs=FREQS, eta=ETA,
                                coef_dtype=dtype))


def _near_degenerate(s, split):
    rng = np.random.default_rng(4)
    eps = np.repeat(s.eps[:1], s.nk, axis=0) + split * rng.uniform(-1.0, 1.0, s.eps.shape)
    return dataclasses.replace(s, eps=eps)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _chi(lib, s, prec, thresh=0.0, dense=None, inv=False):
    import torch
    ctx = lib.Chi0.for_system(s, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    if thresh:
        ctx.set_pole_grouping(thresh)
    if dense is not None:
        ctx.set_double_grid(dense)
    ctx.compute_rho(0)
    chi = np.zeros((s.freqs.size, s.ng, s.ng), np.complex128)
    ctx.build_chi0(0, chi)
    out = chi
    if inv:
        e = np.zeros_like(chi)
        ctx.invert_eps(0, e)
        out = (chi, e)
    ctx.close()
    return out


@pytest.mark.parametrize("prec,dtype,tol", [(0, "c128", 1e-10), (1, "c64", 1e-5)])
def test_grouping_vs_oracle(lib, prec, dtype, tol):
    s = _near_degenerate(_sys(dtype), 4e-6)
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    got = _chi(lib, s, prec, thresh=1e-5)
    ref = O.chi0_grouped(s, 0, G, s.freqs, s.eta, 1e-5)
    plain = O.chi0_tr(s, 0, G, s.freqs, s.eta)
    for iw in range(s.freqs.size):
        assert _rel(got[iw], ref[iw]) < tol, iw
    if prec == 0:
        # the grouping moved chi0, and by the oracle's amount
        assert _rel(ref, plain) > 1e-8
        assert np.linalg.norm((got - plain) - (ref - plain)) <= 1e-3 * np.linalg.norm(ref - plain)


@pytest.mark.parametrize("prec,dtype,tol", [(0, "c128", 1e-10), (1, "c64", 1e-5)])
def test_double_grid_vs_oracle(lib, prec, dtype, tol):
    s = _sys(dtype)
    rng = np.random.default_rng(6)
    dense = s.eps[:, None, :] + 0.05 * rng.uniform(-1.0, 1.0, (s.nk, 3, s.nb))
    got, got_inv = _chi(lib, s, prec, dense=dense, inv=True)
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    ref = O.chi0_double_grid(s, 0, G, s.freqs, s.eta, dense)
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    for iw in range(s.freqs.size):
        assert _rel(got[iw], ref[iw]) < tol, iw
        ref_inv = O.eps_inv_gauss_jordan(ref[iw], qg)
        assert _rel(got_inv[iw], ref_inv) < tol, iw
    assert _rel(ref, O.chi0_tr(s, 0, G, s.freqs, s.eta)) > 1e-3


def test_switch_off_and_argument_checks(lib):
    import torch
    s = _near_degenerate(_sys("c64"), 4e-6)
    plain = _chi(lib, s, 1)
    ctx = lib.Chi0.for_system(s, precision=1, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    ctx.set_pole_grouping(1e-5)
    with pytest.raises(lib.Chi0Error, match="EINVAL"):
        ctx.set_double_grid(np.repeat(s.eps[:, None, :], 2, axis=1))
    with pytest.raises(lib.Chi0Error, match="EINVAL"):
        ctx.set_pole_grouping(-1.0)
    ctx.set_pole_grouping(0.0)
    bad = np.repeat(s.eps[:, None, :], 2, axis=1)
    bad[0, 0, 0] = np.nan
    with pytest.raises(lib.Chi0Error, match="EINVAL"):
        ctx.set_double_grid(bad)
    ctx.set_double_grid(np.repeat(s.eps[:, None, :], 2, axis=1))
    ctx.set_double_grid(None)
    ctx.compute_rho(0)
    chi = np.zeros_like(plain)
    ctx.build_chi0(0, chi)
    ctx.close()
    assert np.array_equal(chi, plain)


def _flat(dtype, split, seed=95):
    """64 k points whose poles repeat at every k up to +-split (Ha): 27 pole
    groups of 64 transitions, large enough for the grouped contraction."""
    s = make_system(cfg_tiny(seed=seed, kgrid=(4, 4, 4), q_frac=((0.25, 0.5, 0.0),), fft=(18, 18, 18), ng=40,
                             n_occ=3, n_bands=12, npw_target=50, a=8.0, freqs=(0.02j, 0.3j, 1.5j, 6.0j),
                             eta=0.0, coef_dtype=dtype))
    return _near_degenerate(s, split) if split > 0 else dataclasses.replace(
        s, eps=np.repeat(s.eps[:1], s.nk, axis=0))


def _chi_groups(lib, s, prec, thresh):
    import torch
    ctx = lib.Chi0.for_system(s, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    if thresh:
        ctx.set_pole_grouping(thresh)
    ctx.compute_rho(0)
    chi = torch.zeros((s.freqs.size, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    inv = torch.zeros_like(chi)
    ctx.build_invert(0, inv, chi)
    ctx.synchronize()
    groups = ctx.pole_groups()
    ctx.close()
    return chi.cpu().numpy(), inv.cpu().numpy(), groups


def test_grouped_contraction_vs_oracle(lib):
    """Large pole groups (splitting 1e-6 Ha below the 1e-4 Ha threshold): the
    mixed form builds chi0 from the frequency-independent group sums; chi0 and
    eps~^-1 equal the oracle's grouped result (1e-5) and the FP64 form's
    per-transition grouped weights (1e-5)."""
    s = _flat("c64", 1e-6)
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    chi, inv, (ngr, grouped) = _chi_groups(lib, s, 1, 1e-4)
    assert grouped and ngr == 27
    want = O.chi0_grouped(s, 0, G, s.freqs, s.eta, 1e-4)
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    want_inv = np.stack([O.eps_inv_gauss_jordan(c, qg) for c in want])
    assert _rel(chi, want) < 1e-5
    assert _rel(inv, want_inv) < 1e-5
    assert np.abs(chi - np.conj(np.transpose(chi, (0, 2, 1)))).max() == 0.0
    s64 = dataclasses.replace(s, coef=s.coef.astype(np.complex128))
    chi64, _, (ngr64, grouped64) = _chi_groups(lib, s64, 0, 1e-4)
    assert ngr64 == 27 and not grouped64
    assert _rel(chi, chi64) < 1e-5


def test_grouped_contraction_exact_degeneracy(lib):
    """Poles exactly degenerate across k: grouping changes no factor, so the
    grouped contraction reproduces the plain chi0 and the oracle."""
    s = _flat("c64", 0.0)
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    chi, _, (ngr, grouped) = _chi_groups(lib, s, 1, 1e-8)
    plain, _, (n0, g0) = _chi_groups(lib, s, 1, 0.0)
    assert grouped and ngr == 27 and n0 == 0 and not g0
    assert _rel(chi, plain) < 3e-6
    assert _rel(chi, O.chi0_tr(s, 0, G, s.freqs, s.eta)) < 1e-5
