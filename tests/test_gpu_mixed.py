"""Mixed form (FP32 rho, BF16x3 tensor-core contraction, FP64 Dyson) vs the
CPU oracle.

Tolerance: 1e-5 relative Frobenius for chi0 and eps~^-1 (the bar set for the
mixed form).  The error model: a BF16 hi/lo pair carries ~2^-17 of each
FP32 operand and the dropped lo*lo term is ~2^-18 of a product, so one
product is good to ~1e-5 in the worst case and the Frobenius error of a sum
of many such products lands near 1e-6; FP32 rho adds ~1e-7.
"""
import numpy as np
import pytest

import oracle as O
from synth import cfg_precision, cfg_tiny, make_system

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0
    return chi0


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _run(lib, s):
    import torch
    ctx = lib.Chi0.for_system(s, precision=lib.CHI0_MIXED_BF16X3,
                              stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    ctx.compute_rho(0)
    out = {"trans": ctx.get_transitions(), "rho": ctx.get_rho()}
    chi = np.zeros((s.freqs.size, s.ng, s.ng), np.complex128)
    ctx.build_chi0(0, chi)
    inv = np.zeros_like(chi)
    ctx.invert_eps(0, inv)
    ctx.synchronize()
    ctx.close()
    out["chi"], out["inv"] = chi, inv
    return out


@pytest.mark.parametrize("case", [
    # several 128 x 128 real tiles with a ragged edge, nt not a multiple of 64
    dict(kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),), fft=(20, 20, 20), ng=45, n_occ=5,
         n_bands=23, npw_target=90, a=8.0, freqs=(0.05j, 0.4j, 3.0j), eta=0.0),
    # more than one transition chunk (nt = 32 * 10 * 60 = 19200 > 8192), 3 x 3 tiles
    dict(kgrid=(4, 4, 2), q_frac=((0.25, 0.5, 0.0),), fft=(20, 20, 20), ng=130, n_occ=10,
         n_bands=70, npw_target=120, a=8.0, freqs=(0.1j, 1.0j), eta=0.0),
    # static with eta (real weights under time reversal), ng = 1
    dict(kgrid=(2, 2, 2), q_frac=((0.5, 0.5, 0.0),), fft=(16, 16, 16), ng=1, n_occ=2,
         n_bands=5, npw_target=25, freqs=(0j,), eta=0.01),
])
def test_mixed_small(lib, case):
    s = make_system(cfg_tiny(seed=41, coef_dtype="c64", **case))
    got = _run(lib, s)
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    trans = O.transitions_tr(s, 0)
    assert np.array_equal(got["trans"], trans)
    ref_rho = O.rho_transitions(s, 0, G, trans)
    assert np.abs(got["rho"] - ref_rho).max() / np.abs(ref_rho).max() < 1e-5
    ref = O.chi0_tr(s, 0, G, s.freqs, s.eta)
    e_chi = _rel(got["chi"], ref)
    assert e_chi < TOL, e_chi
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    ref_inv = np.stack([O.eps_inv_gauss_jordan(c, qg) for c in ref])
    e_inv = _rel(got["inv"], ref_inv)
    assert e_inv < TOL, e_inv
    # the result is exactly Hermitian by construction
    assert np.abs(got["chi"] - np.conj(np.transpose(got["chi"], (0, 2, 1)))).max() == 0.0


def _chi_only(lib, s):
    import torch
    ctx = lib.Chi0.for_system(s, precision=lib.CHI0_MIXED_BF16X3,
                              stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    ctx.compute_rho(0)
    nt = ctx.get_transitions().shape[0]
    chi = np.zeros((s.freqs.size, s.ng, s.ng), np.complex128)
    ctx.build_chi0(0, chi)
    ctx.synchronize()
    _, by, _, _ = ctx.get_stats()
    ctx.close()
    return chi, by["contract"], nt


def test_mixed_sign_weights(lib):
    """Imaginary-axis weights of one sign take the one-operand form
    chi0 = -S S^H with S = rho diag(sqrt|w|); weights of both signs (here: an
    occupied band lifted above every empty one at one k - q point, so its
    transitions get poles d = e_m - e_n > 0) take the two-operand form
    A = w rho, B = rho, which streams twice the operand bytes.  Both against
    the oracle."""
    case = dict(kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),), fft=(20, 20, 20), ng=45, n_occ=5,
                n_bands=23, npw_target=90, a=8.0, freqs=(0.05j, 0.4j, 3.0j), eta=0.0)
    s = make_system(cfg_tiny(seed=43, coef_dtype="c64", **case))
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    chi1, by1, nt = _chi_only(lib, s)
    ref1 = O.chi0_tr(s, 0, G, s.freqs, s.eta)
    e1 = _rel(chi1, ref1)
    assert e1 < TOL, e1
    # the one-operand split keeps the diagonal unbiased: without the lo'
    # correction every chi0_ii is low by about 3e-6 relative (sum of lo^2)
    for w in range(s.freqs.size):
        d = np.diagonal(chi1[w] - ref1[w]).real / np.diagonal(ref1[w]).real
        assert abs(d.mean()) < 1.5e-6, (w, d.mean())
    s.eps[3, 4] = s.eps.max() + 0.1
    w = O.weights_tr(s, 0, O.transitions_tr(s, 0), s.freqs, s.eta).real
    assert (w > 0).any() and (w < 0).any()
    chi2, by2, nt2 = _chi_only(lib, s)
    e2 = _rel(chi2, O.chi0_tr(s, 0, G, s.freqs, s.eta))
    assert e2 < TOL, e2
    # the two forms differ in the operand bytes the contraction streams:
    # 4 bytes (hi and lo BF16) per real row and transition for each extra operand
    assert nt2 == nt
    mpad = (2 * s.ng + 255) // 256 * 256
    kpad = (nt + 63) // 64 * 64
    assert by2 - by1 == s.freqs.size * 4.0 * mpad * kpad, (by1, by2)


@pytest.mark.slow
def test_precision_workload_full_size(lib):
    """8x8x8 k, 16+184 bands, ~2000 PW, FFT 48^3, N_G = 1000, 32 imaginary
    frequencies: the whole chi0 and eps~^-1 on the GPU in the benchmark's
    launch configuration; checked against the oracle on the 64 x 64 G
    sub-block (all transitions, all frequencies), on sampled rho rows, and
    through Hermiticity / sign / spectrum properties of the full matrices."""
    import torch
    s = make_system(cfg_precision())
    ctx = lib.Chi0.for_system(s, precision=lib.CHI0_MIXED_BF16X3,
                              stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    ctx.compute_rho(0)
    G = ctx.get_response_gvectors(0)
    assert np.array_equal(G, O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng))
    trans = ctx.get_transitions()
    assert trans.shape[0] == 512 * 184 * 16
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(trans.shape[0], size=24, replace=False))
    got_rho = ctx.get_rho_rows(rows)
    ref_rho = O.rho_transitions(s, 0, G, trans[rows])
    assert np.abs(got_rho - ref_rho).max() / np.abs(ref_rho).max() < 1e-5
    nw, ng = s.freqs.size, s.ng
    chi_d = torch.zeros((nw, ng, ng), dtype=torch.complex128, device="cuda")
    inv_d = torch.zeros_like(chi_d)
    ctx.build_chi0(0, chi_d)
    ctx.invert_eps(0, inv_d)
    ctx.synchronize()
    ctx.close()
    # the Dyson step alone at N_G = 1000: the GPU's eps~^-1 against the
    # oracle's Gauss-Jordan inversion of eps~ built from the GPU's own chi0
    # (same input, so the comparison isolates the FP64 elimination)
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    for iw in (0, nw - 1):
        want = O.eps_inv_gauss_jordan(chi_d[iw].cpu().numpy(), qg)
        e_d = _rel(inv_d[iw].cpu().numpy(), want)
        print(f"precision workload, eps~^-1 at N_G = 1000 vs oracle Gauss-Jordan (frequency {iw}): {e_d:.3e}")
        assert e_d < 1e-10, (iw, e_d)
    # properties of the full matrices (any size)
    herm = (chi_d - chi_d.conj().transpose(1, 2)).abs().max().item()
    assert herm == 0.0
    ev = torch.linalg.eigvalsh(chi_d[[0, nw // 2, nw - 1]]).cpu().numpy()
    scale = np.abs(ev).max()
    assert ev.max() < 1e-6 * scale  # negative semidefinite up to the mixed-precision error
    ev_inv = torch.linalg.eigvalsh(inv_d[[0, nw - 1]]).cpu().numpy()
    assert ev_inv.min() > 0.0 and ev_inv.max() < 1.0 + 1e-6
    # against the oracle (all transitions, all frequencies) on the G subset
    # G_0..G_63 (tile (0, 0) of the real 2 N_G grid) plus G_496..G_511 and
    # G_984..G_999: the entries among them fall in the diagonal tiles 0, 7 and
    # 15, in the off-diagonal tiles (7, 0), (15, 0), (15, 7) of the lower
    # triangle and in their Hermitian mirrors above the diagonal
    sub = np.concatenate([np.arange(0, 64), np.arange(496, 512), np.arange(984, 1000)])
    idx = torch.as_tensor(sub, device="cuda")
    got = chi_d[:, idx][:, :, idx].cpu().numpy()
    ref = O.chi0_tr(s, 0, G[sub], s.freqs, s.eta)
    e = _rel(got, ref)
    assert e < TOL, e
    per_w = [_rel(got[i], ref[i]) for i in range(nw)]
    print(f"precision workload, 96 x 96 G subset: chi0 relative Frobenius error {e:.3e} "
          f"(worst frequency {max(per_w):.3e})")
    assert max(per_w) < TOL, per_w
    # each block of the subset on its own (the small corner blocks carry
    # little of the Frobenius norm, so they are checked separately)
    parts = [np.arange(0, 64), np.arange(64, 80), np.arange(80, 96)]
    for a in parts:
        for b in parts:
            e_ab = _rel(got[:, a][:, :, b], ref[:, a][:, :, b])
            assert e_ab < TOL, (a[0], b[0], e_ab)
    # the plain FP64 form (the denominator of the mixed form's speed-up) at
    # full size, on the first two frequencies, against the same oracle values
    import dataclasses
    s2 = dataclasses.replace(s, freqs=s.freqs[:2])
    ctx = lib.Chi0.for_system(s2, precision=lib.CHI0_FP64, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s2)
    ctx.compute_rho(0)
    chi64 = torch.zeros((2, ng, ng), dtype=torch.complex128, device="cuda")
    ctx.build_chi0(0, chi64)
    ctx.synchronize()
    ctx.close()
    got64 = chi64[:, idx][:, :, idx].cpu().numpy()
    e64 = _rel(got64, ref[:2])
    print(f"precision workload, plain FP64 form, 96 x 96 G subset, 2 frequencies: {e64:.3e}")
    assert e64 < 1e-10, e64
    assert (chi64 - chi64.conj().transpose(1, 2)).abs().max().item() <= 1e-13 * chi64.abs().max().item()
