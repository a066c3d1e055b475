"""Self-energy kernel I on the GPU (chi0_build_sigma_i; Eqs. W_def, W_delta,
I_c) against the oracle.

1. Two shapes that span several 64 x 64 tiles with ragged edges (N_G = 45 and
   137; 736 and 1656 transitions of the window, nqp = 4 and 9), and a
   one-band window: the GPU's I from the GPU's eps~^-1 equals the oracle's I
   from the same eps~^-1 within 1e-10 (FP64 form) / 1e-5 (mixed form),
   relative Frobenius per frequency; at an imaginary frequency eps~^-1 is
   Hermitian up to rounding and I vanishes (below 1e-12 of the real-axis I).
2. The FP64 form end to end (chi0, eps~^-1, I) against the oracle's own chain.
3. The plasmon-pole model as input (chi0_ppa_eval output on the real axis).
4. The 8x8x8 precision workload (N_G = 1000, a window of four bands around
   the gap, 409,600 transitions), sampled (k, m) blocks against the oracle.
5. Argument checks.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from synth import cfg_precision, cfg_tiny, make_system

pytestmark = pytest.mark.gpu

FREQS = (0.5j, 0.3 + 0j, 1.0 + 0j)
ETA = 0.05


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0
    return chi0


def _sys(dtype, ng=45, fft=20, freqs=FREQS, eta=ETA):
    return make_system(cfg_tiny(seed=91, kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),), fft=(fft, fft, fft), ng=ng,
                                n_occ=5, n_bands=23, npw_target=90, a=8.0, freqs=freqs, eta=eta,
                                coef_dtype=dtype))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _eps_inv_gpu(lib, s, prec):
    import torch
    ctx = lib.Chi0.for_system(s, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    ctx.compute_rho(0)
    inv = torch.zeros((s.freqs.size, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    ctx.build_chi0(0, None)
    ctx.invert_eps(0, inv)
    ctx.synchronize()
    return ctx, inv


def _oracle_i(s, inv_h, qp, ks=None, ms=None):
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    return np.stack([O.i_kernel(s, 0, G, qp, O.w_delta(O.screened_w(inv_h[iw], qg)), ks=ks, ms=ms)
                     for iw in range(inv_h.shape[0])])


@pytest.mark.parametrize("prec,dtype,tol", [(0, "c128", 1e-10), (1, "c64", 1e-5)])
@pytest.mark.parametrize("ng,fft,qp", [(45, 20, (3, 7)), (137, 24, (0, 9)), (45, 20, (4, 5))])
def test_sigma_i_vs_oracle(lib, prec, dtype, tol, ng, fft, qp):
    import torch
    s = _sys(dtype, ng=ng, fft=fft)
    ctx, inv = _eps_inv_gpu(lib, s, prec)
    nqp = qp[1] - qp[0]
    out = torch.zeros((s.freqs.size, s.nk, s.nb, nqp, nqp), dtype=torch.complex128, device="cuda")
    ctx.build_sigma_i(0, qp[0], qp[1], inv, out)
    ctx.synchronize()
    got = out.cpu().numpy()
    # the same call with a host output
    got_h = np.zeros_like(got)
    ctx.build_sigma_i(0, qp[0], qp[1], inv, got_h)
    ctx.close()
    assert np.array_equal(got, got_h)
    ref = _oracle_i(s, inv.cpu().numpy(), list(range(*qp)))
    scale = max(np.abs(got[iw]).max() for iw, w in enumerate(s.freqs) if w.real != 0.0)
    for iw, w in enumerate(s.freqs):
        if w.real == 0.0:
            # eps~^-1 Hermitian up to rounding on the imaginary axis: W^delta ~ 0
            assert np.abs(got[iw]).max() <= 1e-12 * scale
            continue
        e = _rel(got[iw], ref[iw])
        assert e < tol, (iw, e)
        # Hermitian in (a, b), non-negative diagonal (W^delta <= 0 for w > 0)
        herm = np.abs(got[iw] - np.conj(np.swapaxes(got[iw], 2, 3))).max()
        assert herm <= 10 * tol * np.abs(got[iw]).max()
        d = np.diagonal(got[iw], axis1=2, axis2=3).real
        assert d.min() >= -10 * tol * np.abs(d).max()


def test_sigma_i_fp64_end_to_end(lib):
    s = _sys("c128")
    ctx, inv = _eps_inv_gpu(lib, s, 0)
    qp = (3, 7)
    got = np.zeros((s.freqs.size, s.nk, s.nb, 4, 4), np.complex128)
    ctx.build_sigma_i(0, qp[0], qp[1], inv, got)
    ctx.close()
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    chi = O.chi0_tr(s, 0, G, s.freqs, s.eta)
    ref_inv = np.stack([O.eps_inv_gauss_jordan(chi[iw], qg) for iw in range(s.freqs.size)])
    ref = _oracle_i(s, ref_inv, list(range(*qp)))
    for iw, w in enumerate(s.freqs):
        if w.real != 0.0:
            assert _rel(got[iw], ref[iw]) < 1e-10


def test_sigma_i_from_plasmon_pole_model(lib):
    import torch
    s = _sys("c64", freqs=(0j, 1j))
    ctx, inv = _eps_inv_gpu(lib, s, 1)
    wt = torch.empty((s.ng, s.ng), dtype=torch.complex128, device="cuda")
    R = torch.empty_like(wt)
    stream = torch.cuda.current_stream().cuda_stream
    lib.ppa_fit(inv[0], inv[1], 1.0, wt, R, stream)
    freqs = [0.2, 0.7, 1.5]
    model = torch.empty((3, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    lib.ppa_eval(wt, R, freqs, 0.05, model, stream)
    got = np.zeros((3, s.nk, s.nb, 2, 2), np.complex128)
    ctx.build_sigma_i(0, 4, 6, model, got)
    ctx.close()
    ref = _oracle_i(s, model.cpu().numpy(), [4, 5])
    for iw in range(3):
        assert _rel(got[iw], ref[iw]) < 1e-5
        assert np.abs(got[iw]).max() > 0


def test_sigma_i_full_size_precision_workload(lib):
    """8x8x8 k, 16+184 bands, ~2000 PW, N_G = 1000; eps~^-1 at two real
    frequencies (eta = 0.1 eV); window [14, 18): 409,600 transitions."""
    import torch
    from synth import HA_EV
    spec = dataclasses.replace(cfg_precision(nw=2), freqs=(0.5 + 0j, 1.0 + 0j), eta=0.1 / HA_EV)
    s = make_system(spec)
    ctx, inv = _eps_inv_gpu(lib, s, 1)
    qp = (14, 18)
    out = torch.zeros((2, s.nk, s.nb, 4, 4), dtype=torch.complex128, device="cuda")
    ctx.build_sigma_i(0, qp[0], qp[1], inv, out)
    ctx.synchronize()
    ctx.close()
    inv_h = inv.cpu().numpy()
    ks, ms = [0, 137, 511], [0, 15, 16, 90, 199]
    ref = _oracle_i(s, inv_h, list(range(*qp)), ks=ks, ms=ms)
    got = out[:, ks][:, :, ms].cpu().numpy()
    e = _rel(got, ref)
    print(f"full-size I, sampled blocks: relative error {e:.2e}")
    assert e < 1e-5
    full = out.cpu().numpy()
    assert np.isfinite(full).all()
    d = np.diagonal(full, axis1=3, axis2=4).real
    assert d.min() >= -1e-5 * np.abs(d).max()


def test_sigma_i_argument_checks(lib):
    import torch
    s = _sys("c64")
    ctx, inv = _eps_inv_gpu(lib, s, 1)
    out = torch.zeros((s.freqs.size, s.nk, s.nb, 2, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(lib.Chi0Error, match="EINVAL"):
        ctx.build_sigma_i(0, 5, 5, inv, out)           # empty window
    with pytest.raises(lib.Chi0Error, match="EINVAL"):
        ctx.build_sigma_i(0, 22, 24, inv, out)         # beyond the last band
    ctx.close()
    fresh = lib.Chi0.for_system(s, precision=1, stream=torch.cuda.current_stream().cuda_stream)
    fresh.load_system(s)
    with pytest.raises(lib.Chi0Error, match="ESTATE"):
        fresh.build_sigma_i(0, 4, 6, inv, out)         # chi0_compute_rho first
    fresh.close()
