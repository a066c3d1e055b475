"""Real-axis frequencies (w > 0 with eta > 0) on the GPU: complex weights,
chi0 = H_r + i H_i from two Hermitian contractions per frequency, and the
Dyson step by a general (full-tile) Gauss-Jordan, against the oracle, in a
frequency list that mixes the imaginary and the real axis.

Tolerances: 1e-10 relative Frobenius per frequency in the FP64 form, 1e-5 in
the mixed form, for chi0 and for eps~^-1.
"""
import numpy as np
import pytest

import oracle as O
from synth import HA_EV, cfg_tiny, make_system

pytestmark = pytest.mark.gpu

FREQS = (0.1j, 0.3 + 0j, 2.0j, 1.0 + 0j, 3.5 + 0j)
ETA = 0.05


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0
    return chi0


def _sys(dtype, freqs=FREQS, eta=ETA):
    return make_system(cfg_tiny(seed=91, kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),), fft=(20, 20, 20), ng=45,
                                n_occ=5, n_bands=23, npw_target=90, a=8.0, freqs=freqs, eta=eta,
                                coef_dtype=dtype))


def _run(lib, s, prec, bg=None):
    import torch
    ctx = lib.Chi0.for_system(s, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    if bg is not None:
        ctx.set_bg_terminator(bg)
    ctx.compute_rho(0)
    shape = (s.freqs.size, s.ng, s.ng)
    chi = np.zeros(shape, np.complex128)
    inv = np.zeros(shape, np.complex128)
    ctx.build_chi0(0, chi)
    ctx.invert_eps(0, inv)
    ctx.close()
    return chi, inv


@pytest.mark.parametrize("prec,dtype,tol", [(0, "c128", 1e-10), (1, "c64", 1e-5)])
def test_real_axis_vs_oracle(lib, prec, dtype, tol):
    s = _sys(dtype)
    chi, inv = _run(lib, s, prec)
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    ref = O.chi0_tr(s, 0, G, s.freqs, s.eta)
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    for iw in range(s.freqs.size):
        e = np.linalg.norm(chi[iw] - ref[iw]) / np.linalg.norm(ref[iw])
        assert e < tol, (iw, e)
        ref_inv = O.eps_inv_gauss_jordan(ref[iw], qg)
        ei = np.linalg.norm(inv[iw] - ref_inv) / np.linalg.norm(ref_inv)
        assert ei < tol, (iw, ei)
    # the real-axis results are not Hermitian, the imaginary-axis ones exactly are
    for iw, w in enumerate(s.freqs):
        herm = np.abs(chi[iw] - chi[iw].conj().T).max()
        if w.real != 0.0:
            assert herm > 1e-3 * np.abs(chi[iw]).max()
        else:
            assert herm == 0.0


def test_real_axis_with_extrapolar_correction(lib):
    s = _sys("c128")
    eps_bar = 40.0 / HA_EV
    chi, _ = _run(lib, s, 0, bg=eps_bar)
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    ref = O.chi0_bg(s, 0, G, s.freqs, s.eta, eps_bar)
    assert np.linalg.norm(chi - ref) / np.linalg.norm(ref) < 1e-10


def test_real_axis_build_invert_and_batch(lib):
    import torch
    s = _sys("c64")
    stream = torch.cuda.current_stream().cuda_stream
    shape = (s.freqs.size, s.ng, s.ng)
    ctx = lib.Chi0.for_system(s, precision=1, stream=stream)
    ctx.load_system(s)
    ctx.compute_rho(0)
    chi_a = torch.zeros(shape, dtype=torch.complex128, device="cuda")
    inv_a = torch.zeros_like(chi_a)
    ctx.build_chi0(0, chi_a)
    ctx.invert_eps(0, inv_a)
    chi_b = torch.zeros_like(chi_a)
    inv_b = torch.zeros_like(chi_a)
    ctx.compute_rho(0)
    ctx.build_invert(0, inv_b, chi_b)
    ctx.synchronize()
    # build_invert runs the Dyson step in frequency groups beside the contraction
    assert torch.equal(chi_a, chi_b)
    assert (inv_b - inv_a).abs().max().item() <= 1e-13 * inv_a.abs().max().item()
    out = torch.zeros_like(chi_a)
    batch = lib.Batch([ctx], [0], [out], nstreams=1)
    batch.run(stream)
    torch.cuda.synchronize()
    ctx.synchronize()
    assert (out - inv_a).abs().max().item() <= 1e-13 * inv_a.abs().max().item()
    batch.close()
    ctx.close()


@pytest.mark.parametrize("freqs,eta", [((0.3 + 0j,), 0.0), ((-0.3 + 0j,), 0.05), ((0.3 + 0.1j,), 0.05)])
def test_rejected_frequencies(lib, freqs, eta):
    import torch
    s = _sys("c64", freqs=freqs, eta=eta)
    ctx = lib.Chi0.for_system(s, precision=1, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    ctx.compute_rho(0)
    with pytest.raises(lib.Chi0Error, match="EUNSUPPORTED"):
        ctx.build_chi0(0, None)
    ctx.close()
