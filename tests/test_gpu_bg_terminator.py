"""Bruneval-Gonze extrapolar correction on the GPU (chi0_set_bg_terminator,
Eq. X_term_def with Appendix C) against the oracle.

1. Small insulator and metal, both precisions: the corrected chi0 equals the
   oracle's chi0_trunc + Delta chi within 1e-10 (FP64 form) and 1e-5 (mixed
   form), relative Frobenius.
2. A complete band basis with every omitted band at eps_bar: the corrected
   truncated chi0 equals the full-band chi0 (the closure relation is exact).
3. The same basis with the omitted bands spread over 35-70 eV: the correction
   takes the truncation error from ~0.9 to a few per cent.
4. The correction goes through chi0_build_invert (the term is added to each
   frequency as soon as it is reduced, ahead of that frequency's Dyson step)
   and through a batch.
5. Argument checks.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from synth import HA_EV, cfg_tiny, make_closure_system, make_system, truncate_bands

pytestmark = pytest.mark.gpu


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


def _insulator(dtype):
    return make_system(cfg_tiny(seed=81, kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),), fft=(20, 20, 20), ng=45,
                                n_occ=5, n_bands=23, npw_target=90, a=8.0, freqs=(0.05j, 0.4j, 3.0j), eta=0.0,
                                coef_dtype=dtype))


def _metal(dtype):
    spec = cfg_tiny(seed=82, kgrid=(2, 2, 2), q_frac=((0.5, 0.5, 0.0),), fft=(16, 16, 16), ng=30, n_occ=4,
                    n_bands=10, npw_target=40, a=7.0, freqs=(0.01j, 0.5j, 2.0j), eta=0.0, coef_dtype=dtype)
    spec = dataclasses.replace(spec, occ_ev=(-2.0, 0.5), emp_ev=(-0.5, 4.0), kT_ev=0.05, n_electrons=8)
    return make_system(spec)


def _chi_bg(lib, s, prec, eps_bar, iq=0):
    import torch
    ctx = lib.Chi0.for_system(s, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    ctx.set_bg_terminator(eps_bar)
    ctx.compute_rho(iq)
    chi = np.zeros((s.freqs.size, s.ng, s.ng), np.complex128)
    ctx.build_chi0(iq, chi)
    ctx.close()
    return chi


@pytest.mark.parametrize("prec,dtype,tol", [(0, "c128", 1e-10), (1, "c64", 1e-5)])
@pytest.mark.parametrize("make", [_insulator, _metal])
def test_bg_vs_oracle(lib, prec, dtype, tol, make):
    s = make(dtype)
    eps_bar = 40.0 / HA_EV
    got = _chi_bg(lib, s, prec, eps_bar)
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    ref = O.chi0_bg(s, 0, G, s.freqs, s.eta, eps_bar)
    assert _rel(got, ref) < tol, _rel(got, ref)
    # the correction is not negligible here, and the result is exactly Hermitian
    plain = O.chi0_tr(s, 0, G, s.freqs, s.eta)
    assert _rel(plain, ref) > 1e-3
    assert np.abs(got - np.conj(np.transpose(got, (0, 2, 1)))).max() == 0.0


@pytest.mark.parametrize("prec,dtype,tol", [(0, "c128", 1e-10), (1, "c64", 1e-5)])
def test_bg_closure_exact(lib, prec, dtype, tol):
    eps_bar = 45.0 / HA_EV
    full = make_closure_system(nb_keep=12, omitted_ev=(45.0, 45.0), coef_dtype=dtype)
    G = O.response_gvectors(full.spec.kgrid, full.q_frac[0], full.ng)
    ref = O.chi0_tr(full, 0, G, full.freqs, full.eta)
    got = _chi_bg(lib, truncate_bands(full, 12), prec, eps_bar)
    assert _rel(got, ref) < tol, _rel(got, ref)


def test_bg_gain_over_truncation(lib):
    full = make_closure_system(seed=9, nb_keep=20, omitted_ev=(35.0, 70.0), coef_dtype="c64")
    G = O.response_gvectors(full.spec.kgrid, full.q_frac[0], full.ng)
    ref = O.chi0_tr(full, 0, G, full.freqs, full.eta)
    trunc = truncate_bands(full, 20)
    e_trunc = _rel(O.chi0_tr(trunc, 0, G, full.freqs, full.eta), ref)
    e_bg = _rel(_chi_bg(lib, trunc, 1, 52.5 / HA_EV), ref)
    print(f"complete basis, omitted bands in 35-70 eV: truncated {e_trunc:.3f}, with the correction {e_bg:.4f}")
    assert e_trunc > 0.5 and e_bg < 0.05


def test_bg_through_build_invert_and_batch(lib):
    import torch
    s = _insulator("c64")
    eps_bar = 40.0 / HA_EV
    stream = torch.cuda.current_stream().cuda_stream
    shape = (s.freqs.size, s.ng, s.ng)
    ctx = lib.Chi0.for_system(s, precision=1, stream=stream)
    ctx.load_system(s)
    ctx.set_bg_terminator(eps_bar)
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


def test_bg_argument_checks(lib):
    import torch
    s = _insulator("c64")
    ctx = lib.Chi0.for_system(s, precision=1, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    with pytest.raises(lib.Chi0Error, match="EINVAL"):
        ctx.set_bg_terminator(float("nan"))
    ctx.compute_rho(0)
    ctx.set_bg_terminator(40.0 / HA_EV)
    with pytest.raises(lib.Chi0Error, match="ESTATE"):
        ctx.build_chi0(0, None)           # the transition block changed: compute_rho first
    params = torch.zeros(lib.mlp_nparams(), dtype=torch.float32, device="cuda")
    with pytest.raises(lib.Chi0Error, match="EINVAL"):
        ctx.set_terminator(params)
    ctx.set_bg_terminator(0.0, on=False)
    ctx.set_terminator(params)
    with pytest.raises(lib.Chi0Error, match="EINVAL"):
        ctx.set_bg_terminator(40.0 / HA_EV)
    ctx.set_terminator(None)
    ctx.close()
