"""chi0_build_invert: chi0 and eps~^-1 in one call, the Dyson step of each
frequency overlapping the tensor-core contraction of the later ones.  Its
results must equal those of chi0_build_chi0 followed by chi0_invert_eps (the
same kernels on the same data; the per-frequency Dyson launches take the same
arithmetic path as the batched one), with device and with host buffers, in
both precisions (FP64 runs the two steps one after the other), and agree with
the oracle."""
import numpy as np
import pytest

import oracle as O
from synth import cfg_tiny, make_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0
    return chi0


def _system(dtype):
    # ng = 77: three 32-wide pivot blocks with a ragged last one; 5 frequencies
    return make_system(cfg_tiny(seed=71, kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),), fft=(20, 20, 20),
                                ng=77, n_occ=5, n_bands=21, npw_target=90, a=8.0,
                                freqs=(0.02j, 0.1j, 0.4j, 1.5j, 6.0j), eta=0.0, coef_dtype=dtype))


@pytest.mark.parametrize("prec,dtype,tol", [(1, "c64", 1e-5), (0, "c128", 1e-10)])
def test_build_invert_matches_separate_calls(lib, prec, dtype, tol):
    import torch
    s = _system(dtype)
    stream = torch.cuda.current_stream().cuda_stream
    shape = (s.freqs.size, s.ng, s.ng)
    ctx = lib.Chi0.for_system(s, precision=prec, stream=stream)
    ctx.load_system(s)
    ctx.compute_rho(0)
    chi_a = torch.zeros(shape, dtype=torch.complex128, device="cuda")
    inv_a = torch.zeros_like(chi_a)
    ctx.build_chi0(0, chi_a)
    ctx.invert_eps(0, inv_a)
    # pipelined, device buffers, twice (the second run reuses the streams and events)
    for _ in range(2):
        chi_b = torch.full(shape, complex(float("nan"), 0.0), dtype=torch.complex128, device="cuda")
        inv_b = torch.full_like(chi_b, complex(float("nan"), 0.0))
        ctx.compute_rho(0)
        ctx.build_invert(0, inv_b, chi_b)
        ctx.synchronize()
        assert torch.equal(chi_a, chi_b)
        assert (inv_b - inv_a).abs().max().item() <= 1e-13 * inv_a.abs().max().item()
    # host buffers
    inv_h = np.zeros(shape, dtype=np.complex128)
    chi_h = np.zeros(shape, dtype=np.complex128)
    ctx.compute_rho(0)
    ctx.build_invert(0, inv_h, chi_h)
    assert np.array_equal(chi_h, chi_a.cpu().numpy())
    assert np.abs(inv_h - inv_a.cpu().numpy()).max() <= 1e-13 * np.abs(inv_h).max()
    # chi0 stays on the device for a later invert_eps
    inv_c = torch.zeros_like(chi_a)
    ctx.invert_eps(0, inv_c)
    ctx.synchronize()
    assert (inv_c - inv_a).abs().max().item() <= 1e-13 * inv_a.abs().max().item()
    ctx.close()
    # against the oracle
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    chi_o = O.chi0_tr(s, 0, G, s.freqs, s.eta)
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    inv_o = np.stack([O.eps_inv_gauss_jordan(c, qg) for c in chi_o])
    assert np.linalg.norm(inv_h - inv_o) / np.linalg.norm(inv_o) < tol
    assert np.linalg.norm(chi_h - chi_o) / np.linalg.norm(chi_o) < tol


def test_build_invert_validation(lib):
    import torch
    s = _system("c64")
    ctx = lib.Chi0.for_system(s, precision=1, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    out = torch.zeros((s.freqs.size, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    with pytest.raises(lib.Chi0Error, match="ESTATE"):
        ctx.build_invert(0, out)          # before compute_rho
    ctx.compute_rho(0)
    with pytest.raises(ValueError):
        ctx.build_invert(0, out, np.zeros((s.freqs.size, s.ng, s.ng), np.complex128))
    ctx.close()


def _fresh(lib, s, prec, stream):
    import torch
    ctx = lib.Chi0.for_system(s, precision=prec, stream=stream)
    ctx.load_system(s)
    ctx.compute_rho(0)
    inv = torch.zeros((s.freqs.size, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    chi = torch.zeros_like(inv)
    ctx.build_invert(0, inv, chi)
    ctx.synchronize()
    ctx.close()
    return chi, inv


@pytest.mark.parametrize("prec,dtype", [(1, "c64"), (0, "c128")])
def test_plans_reused_only_while_valid(lib, prec, dtype):
    """A context reuses its plans across steps whose inputs differ only in the
    coefficient values (same spheres, energies and occupations), and plans
    again when the spheres or the occupations change.  Every step must equal
    a fresh context on the same inputs, bit for bit."""
    import dataclasses
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    a = _system(dtype)
    b = make_system(dataclasses.replace(a.spec, seed=72))     # same spheres, new coefficients
    b.eps, b.occ = a.eps.copy(), a.occ.copy()                  # and the same energies
    c = make_system(dataclasses.replace(a.spec, seed=73, n_occ=4))            # other occupations
    d = make_system(dataclasses.replace(a.spec, seed=74, kc=a.spec.kc * 0.93))  # other spheres
    assert np.array_equal(a.gvec, b.gvec) and not np.array_equal(a.coef, b.coef)
    assert not np.array_equal(a.occ, c.occ) and not np.array_equal(a.npw, d.npw)
    ctx = lib.Chi0.for_system(a, precision=prec, stream=stream)
    shape = (a.freqs.size, a.ng, a.ng)
    for s in (a, b, b, c, a, d):
        ctx.load_system(s)
        ctx.compute_rho(0)
        inv = torch.full(shape, complex(float("nan"), 0.0), dtype=torch.complex128, device="cuda")
        chi = torch.full_like(inv, complex(float("nan"), 0.0))
        ctx.build_invert(0, inv, chi)
        ctx.synchronize()
        want_chi, want_inv = _fresh(lib, s, prec, stream)
        assert torch.equal(chi, want_chi)
        assert (inv - want_inv).abs().max().item() <= 1e-13 * want_inv.abs().max().item()
    ctx.close()
