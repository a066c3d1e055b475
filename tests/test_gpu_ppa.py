"""Godby-Needs plasmon-pole model on the GPU (chi0_ppa_fit, chi0_ppa_eval;
Full frequency GW subsection) against the oracle.

1. Random matrices with prescribed poles, including elements without a real
   pole, a ragged element count, a single element and the response-set size
   of the 8x8x8 precision workload (N_G = 1000) with 100 frequencies: the
   static mask is identical and wt, R agree element by element within 1e-12
   (relative to each element's magnitude); the model values computed from
   the same parameters agree within 1e-11.
2. The path the paper describes: chi0 and eps~^-1 at w = 0 and w = i 1 Ha
   through chi0_build_chi0 / chi0_invert_eps, then the fit on the device.
   The GPU fit of the GPU eps~^-1 equals the oracle fit of the same matrices;
   in the FP64 form it also equals the oracle fit of the oracle's eps~^-1
   (model values within 1e-9); the model reproduces eps~^-1 at w = 0, and at
   i omega_p on every element with a real pole.
3. Argument checks.
"""
import numpy as np
import pytest

import oracle as O
from synth import cfg_tiny, make_system

pytestmark = pytest.mark.gpu

WP = 1.0   # omega_p, Ha (PPAPntXp default)


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0
    return chi0


def _pole_inputs(ng, seed):
    """eps^-1 at 0 and i WP whose elements are single poles with prescribed
    wt^2 (Re wt^2 of either sign, kept away from 0), plus exact static ones."""
    rng = np.random.default_rng(seed)
    x0 = (rng.standard_normal((ng, ng)) + 1j * rng.standard_normal((ng, ng))) * 0.1
    sgn = np.where(rng.random((ng, ng)) < 0.8, 1.0, -1.0)
    wt2 = sgn * rng.uniform(0.1, 4.0, (ng, ng)) + 1j * rng.uniform(-1.0, 1.0, (ng, ng))
    xp = x0 * wt2 / (WP ** 2 + wt2)
    same = rng.random((ng, ng)) < 0.05
    xp[same] = x0[same]
    eye = np.eye(ng)
    return eye + x0, eye + xp


def _close(a, b, tol):
    """|a - b| <= tol max(|b|, 1e-300) element by element."""
    return np.all(np.abs(a - b) <= tol * np.maximum(np.abs(b), 1e-300))


def _fit_gpu(lib, e0, ep, wp=WP):
    import torch
    d0 = e0 if torch.is_tensor(e0) else torch.from_numpy(np.ascontiguousarray(e0)).cuda()
    dp = ep if torch.is_tensor(ep) else torch.from_numpy(np.ascontiguousarray(ep)).cuda()
    wt = torch.empty_like(d0)
    R = torch.empty_like(d0)
    lib.ppa_fit(d0, dp, wp, wt, R, torch.cuda.current_stream().cuda_stream)
    return wt, R


def _eval_gpu(lib, wt, R, freqs, eta):
    import torch
    out = torch.empty((len(freqs),) + tuple(wt.shape), dtype=torch.complex128, device="cuda")
    lib.ppa_eval(wt, R, freqs, eta, out, torch.cuda.current_stream().cuda_stream)
    return out


@pytest.mark.parametrize("ng,nf", [(1, 3), (37, 5), (211, 40)])
def test_ppa_random_vs_oracle(lib, ng, nf):
    e0, ep = _pole_inputs(ng, seed=ng)
    wt, R = _fit_gpu(lib, e0, ep)
    rwt, rR = O.ppa_fit(e0, ep, WP)
    gwt, gR = wt.cpu().numpy(), R.cpu().numpy()
    assert np.array_equal(gwt == 0, rwt == 0)
    assert _close(gwt, rwt, 1e-12) and _close(gR, rR, 1e-12)
    rng = np.random.default_rng(7)
    freqs = np.where(rng.random(nf) < 0.5, 1j * rng.uniform(0, 5, nf), rng.uniform(0, 5, nf))
    got = _eval_gpu(lib, wt, R, freqs, 0.05).cpu().numpy()
    ref = O.ppa_eval(gwt, gR, freqs, 0.05)     # the evaluation alone, on the same parameters
    assert _close(got, ref, 1e-11)


def test_ppa_full_size_response_set(lib):
    """N_G = 1000 (the 8x8x8 precision workload's response set) with 100 real
    frequencies, the size of a real-axis frequency list; outputs sampled."""
    import torch
    ng, nf = 1000, 100
    e0, ep = _pole_inputs(ng, seed=1000)
    wt, R = _fit_gpu(lib, e0, ep)
    rwt, rR = O.ppa_fit(e0, ep, WP)
    gwt, gR = wt.cpu().numpy(), R.cpu().numpy()
    assert np.array_equal(gwt == 0, rwt == 0)
    assert _close(gwt, rwt, 1e-12) and _close(gR, rR, 1e-12)
    freqs = np.linspace(0.0, 100.0 / 27.211386, nf).astype(np.complex128)
    out = _eval_gpu(lib, wt, R, freqs, 0.1 / 27.211386)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    fi = rng.integers(0, nf, 4000)
    ii = rng.integers(0, ng, 4000)
    jj = rng.integers(0, ng, 4000)
    fi[:nf], ii[:nf], jj[:nf] = np.arange(nf), np.arange(nf) % ng, np.arange(nf) % ng   # some diagonals
    got = out[torch.from_numpy(fi).cuda(), torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()
    eye = (ii == jj).astype(np.float64)
    w = freqs[fi] + 1j * 0.1 / 27.211386
    t, r = gwt[ii, jj], gR[ii, jj]            # the evaluation alone, on the same parameters
    with np.errstate(divide="ignore", invalid="ignore"):
        ref = np.where(t == 0, r, r * (1.0 / (w - t) - 1.0 / (w + t))) + eye
    assert _close(got, ref, 1e-11)


def _two_point_eps_inv(lib, prec, dtype):
    import torch
    s = make_system(cfg_tiny(seed=95, kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),), fft=(20, 20, 20), ng=45,
                             n_occ=5, n_bands=23, npw_target=90, a=8.0, freqs=(0j, 1j * WP), eta=0.0,
                             coef_dtype=dtype))
    ctx = lib.Chi0.for_system(s, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    ctx.compute_rho(0)
    inv = torch.zeros((2, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    ctx.build_chi0(0, None)
    ctx.invert_eps(0, inv)
    ctx.synchronize()
    ctx.close()
    return s, inv


@pytest.mark.parametrize("prec,dtype", [(0, "c128"), (1, "c64")])
def test_ppa_from_dyson(lib, prec, dtype):
    s, inv = _two_point_eps_inv(lib, prec, dtype)
    wt, R = _fit_gpu(lib, inv[0], inv[1])
    h_inv = inv.cpu().numpy()
    rwt, rR = O.ppa_fit(h_inv[0], h_inv[1], WP)
    gwt, gR = wt.cpu().numpy(), R.cpu().numpy()
    assert np.array_equal(gwt == 0, rwt == 0)
    assert _close(gwt, rwt, 1e-12) and _close(gR, rR, 1e-12)
    # a physical screening: most elements get a real pole
    print(f"elements with a real pole: {(gwt != 0).mean():.3f}")
    assert (gwt != 0).mean() > 0.5
    # the model reproduces eps~^-1 at w = 0, and at i omega_p wherever it has a real pole
    back = _eval_gpu(lib, wt, R, [0j, 1j * WP], 0.0).cpu().numpy()
    pole = gwt != 0
    assert np.linalg.norm(back[0] - h_inv[0]) <= 1e-12 * np.linalg.norm(h_inv[0])
    assert np.linalg.norm((back[1] - h_inv[1])[pole]) <= 1e-12 * np.linalg.norm(h_inv[1][pole])
    if prec == 0:
        G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
        ref = O.chi0_tr(s, 0, G, s.freqs, s.eta)
        qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
        owt, oR = O.ppa_fit(O.eps_inv_gauss_jordan(ref[0], qg), O.eps_inv_gauss_jordan(ref[1], qg), WP)
        assert np.array_equal(gwt == 0, owt == 0)
        freqs = [0.5j, 3j, 0.4 + 0j, 2.0 + 0j]
        model = _eval_gpu(lib, wt, R, freqs, 0.05).cpu().numpy()
        want = O.ppa_eval(owt, oR, freqs, 0.05)
        for f in range(len(freqs)):
            assert np.linalg.norm(model[f] - want[f]) <= 1e-9 * np.linalg.norm(want[f])


def test_ppa_argument_checks(lib):
    import torch
    a = torch.zeros((4, 4), dtype=torch.complex128, device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(lib.Chi0Error, match="EINVAL"):
        lib.ppa_fit(a, a, 0.0, a, b)
    with pytest.raises(lib.Chi0Error, match="EINVAL"):
        lib.ppa_fit(a, a, float("nan"), a, b)
    with pytest.raises(lib.Chi0Error, match="EINVAL"):
        lib.ppa_eval(a, b, [1j], -1.0, torch.zeros((1, 4, 4), dtype=torch.complex128, device="cuda"))
    with pytest.raises(lib.Chi0Error, match="EINVAL"):
        lib.ppa_eval(a, b, [complex(np.nan, 0)], 0.0, torch.zeros((1, 4, 4), dtype=torch.complex128, device="cuda"))
    out = torch.full((1, 4, 4), 7.0, dtype=torch.complex128, device="cuda")
    lib.ppa_eval(a, b, [], 0.0, out)       # no frequencies: nothing written
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
