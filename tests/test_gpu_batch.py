"""Batched problems (chi0_batch_*): several systems and q points, uneven in
grid size, response set, frequency count and transition count (one metal
with Fermi-Dirac occupations), run as one captured graph with a persistent
rho launch.  The batch must reproduce the one-problem-at-a-time results
exactly (the same kernels on the same data), on repeated replays, and the
metallic problem must agree with the oracle (1e-5, mixed form)."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from synth import HA_EV, cfg_tiny, make_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0
    return chi0


def _systems(coef_dtype):
    a = make_system(cfg_tiny(seed=61, kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),), fft=(20, 20, 20),
                             ng=45, n_occ=5, n_bands=23, npw_target=90, a=8.0,
                             freqs=(0.05j, 0.4j, 3.0j), eta=0.0, coef_dtype=coef_dtype))
    b = make_system(cfg_tiny(seed=62, kgrid=(4, 2, 2), q_frac=((0.25, 0.5, 0.0), (0.5, 0.0, 0.5)),
                             fft=(18, 18, 18), ng=70, n_occ=4, n_bands=12, npw_target=45, a=8.0,
                             freqs=(0.2j, 1.5j), eta=0.0, coef_dtype=coef_dtype))
    spec = cfg_tiny(seed=63, kgrid=(2, 2, 2), q_frac=((0.5, 0.5, 0.0),), fft=(16, 16, 16), ng=30,
                    n_occ=4, n_bands=10, npw_target=40, a=7.0, freqs=(0.01j, 0.1j, 0.5j, 2.0j),
                    eta=0.0, coef_dtype=coef_dtype)
    spec = dataclasses.replace(spec, occ_ev=(-2.0, 0.5), emp_ev=(-0.5, 4.0), kT_ev=0.05, n_electrons=8)
    metal = make_system(spec)
    return [(a, 0), (b, 0), (b, 1), (metal, 0)]


def _single(lib, s, iq, prec, stream):
    import torch
    ctx = lib.Chi0.for_system(s, precision=prec, stream=stream)
    ctx.load_system(s)
    ctx.compute_rho(iq)
    chi = torch.zeros((s.freqs.size, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    ctx.build_chi0(iq, chi)
    inv = torch.zeros_like(chi)
    ctx.invert_eps(iq, inv)
    ctx.synchronize()
    ctx.close()
    return chi, inv


@pytest.mark.parametrize("prec,dtype", [(1, "c64"), (0, "c128")])
def test_batch_matches_single_problems(lib, prec, dtype):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    probs = _systems(dtype)
    ref = [_single(lib, s, iq, prec, stream) for s, iq in probs]
    ctxs, outs = [], []
    for s, iq in probs:
        c = lib.Chi0.for_system(s, precision=prec, stream=stream)
        c.load_system(s)
        ctxs.append(c)
        outs.append(torch.full((s.freqs.size, s.ng, s.ng), complex(float("nan"), 0.0),
                               dtype=torch.complex128, device="cuda"))
    batch = lib.Batch(ctxs, [iq for _, iq in probs], outs, nstreams=3)
    assert batch.rho_width() in (1, 2, 4)
    for rep in range(2):
        for o in outs:
            o.fill_(complex(float("nan"), 0.0))
        batch.run(stream)
        torch.cuda.synchronize()
        for c in ctxs:
            c.synchronize()
        for (chi_r, inv_r), o in zip(ref, outs):
            assert torch.isfinite(o).all()
            assert (o - inv_r).abs().max().item() <= 1e-13 * inv_r.abs().max().item()
    batch.close()
    for c in ctxs:
        c.close()
    # the metallic problem (uneven transitions per k) against the oracle
    metal, iq = probs[3]
    assert np.any((metal.occ > 0.01) & (metal.occ < 0.99))  # partially filled bands
    G = O.response_gvectors(metal.spec.kgrid, metal.q_frac[iq], metal.ng)
    want = O.chi0_tr(metal, iq, G, metal.freqs, metal.eta)
    got = ref[3][0].cpu().numpy()
    tol = 1e-5 if prec == 1 else 1e-10
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol
