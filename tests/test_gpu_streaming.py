"""Band-block streaming (chi0_set_band_blocks): the transitions go through
rho, the weights and the contraction in blocks of k points x n bands, with
only the occupied-side mixed grids resident and chi0 summed over the blocks.
The blocks partition the transition set, so chi0 and eps~^-1 must agree with
the unstreamed path (up to the order of the additions) and with the oracle
(1e-5 mixed, 1e-10 FP64), on ragged k and band blocks, on the imaginary axis
and at a real frequency; a single block covering everything must reproduce
the unstreamed result bit for bit."""
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


def _system(dtype, real=False):
    freqs = (0.05j, 0.6j, 4.0j) if not real else (0.1j, 12.0 / HA_EV + 0j)
    return make_system(cfg_tiny(seed=81, kgrid=(4, 2, 2), q_frac=((0.25, 0.5, 0.0),), fft=(18, 18, 18),
                                ng=45, n_occ=4, n_bands=40, npw_target=60, a=8.0, freqs=freqs,
                                eta=(0.1 / HA_EV if real else 0.0), coef_dtype=dtype))


def _run(lib, s, prec, blocks):
    import torch
    ctx = lib.Chi0.for_system(s, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    if blocks is not None:
        ctx.set_band_blocks(*blocks)
    ctx.compute_rho(0)
    inv = torch.zeros((s.freqs.size, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    chi = torch.zeros_like(inv)
    ctx.build_invert(0, inv, chi)
    ctx.synchronize()
    if blocks is not None and blocks[0] > 0:
        with pytest.raises(lib.Chi0Error, match="ESTATE"):
            ctx.get_rho()
    ctx.close()
    return chi.cpu().numpy(), inv.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,dtype,tol", [(1, "c64", 1e-5), (0, "c128", 1e-10)])
@pytest.mark.parametrize("real", [False, True])
def test_streamed_equals_unstreamed_and_oracle(lib, prec, dtype, tol, real):
    s = _system(dtype, real)
    chi_u, inv_u = _run(lib, s, prec, None)
    # 36 n bands in blocks of 13 (13, 13, 10), 16 k points in blocks of 6 (6, 6, 4): 9 blocks
    chi_s, inv_s = _run(lib, s, prec, (13, 6))
    order_tol = 1e-6 if prec == 1 else 1e-13
    assert _rel(chi_s, chi_u) < order_tol
    assert _rel(inv_s, inv_u) < order_tol
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    want = O.chi0_tr(s, 0, G, s.freqs, s.eta)
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    want_inv = np.stack([O.eps_inv_gauss_jordan(c, qg) for c in want])
    assert _rel(chi_s, want) < tol
    assert _rel(inv_s, want_inv) < tol
    # one block holding every transition: the same arithmetic as unstreamed
    chi_1, inv_1 = _run(lib, s, prec, (1000, 0))
    assert np.array_equal(chi_1, chi_u)
    assert np.array_equal(inv_1, inv_u)


def test_streaming_settings_checked(lib):
    import torch
    s = _system("c64")
    ctx = lib.Chi0.for_system(s, precision=1, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    with pytest.raises(lib.Chi0Error, match="EINVAL"):
        ctx.set_band_blocks(-1, 0)
    ctx.set_band_blocks(8, 4)
    ctx.set_bg_terminator(1.5)
    with pytest.raises(lib.Chi0Error, match="EUNSUPPORTED"):
        ctx.compute_rho(0)
    ctx.set_bg_terminator(1.5, on=False)
    ctx.compute_rho(0)
    ctx.close()
