"""FP64 form on the GPU vs the CPU oracle, element by element.

Tolerance: 1e-10 relative (Frobenius for chi0 and eps~^-1, max-norm relative
to the largest element for rho), the bar set for the plain FP64 form.
"""
import numpy as np
import pytest

import oracle as O
from synth import cfg_plain_fp64, cfg_tiny, make_system

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0
    return chi0


def _run(lib, s, precision=0, rho=True):
    import torch
    ctx = lib.Chi0.for_system(s, precision=precision, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    ctx.compute_rho(0)
    out = {"G": ctx.get_response_gvectors(0), "trans": ctx.get_transitions()}
    if rho:
        out["rho"] = ctx.get_rho()
    chi = np.zeros((s.freqs.size, s.ng, s.ng), np.complex128)
    ctx.build_chi0(0, chi)
    inv = np.zeros_like(chi)
    ctx.invert_eps(0, inv)
    ctx.synchronize()
    out["chi"], out["inv"] = chi, inv
    out["stats"] = ctx.get_stats()
    ctx.close()
    return out


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _check_all(s, got, tol=TOL):
    G = O.response_gvectors(s.spec.kgrid, s.q_frac[0], s.ng)
    assert np.array_equal(got["G"], G)
    trans = O.transitions_tr(s, 0)
    assert np.array_equal(got["trans"], trans)
    if "rho" in got:
        ref_rho = O.rho_transitions(s, 0, G, trans)
        err = np.abs(got["rho"] - ref_rho).max() / np.abs(ref_rho).max()
        assert err < tol, err
    ref = O.chi0_tr(s, 0, G, s.freqs, s.eta)
    assert _rel(got["chi"], ref) < tol, _rel(got["chi"], ref)
    qg = O.qg_norms(s.spec.a, s.q_frac[0], G)
    ref_inv = np.stack([O.eps_inv_gauss_jordan(c, qg) for c in ref])
    assert _rel(got["inv"], ref_inv) < tol, _rel(got["inv"], ref_inv)


def test_plain_fp64_workload(lib):
    """4x4x4 k, 8+24 bands, ~300 PW, FFT 24^3, N_G = 59, q = (1/4,0,0), w = 0, eta = 0.1 eV."""
    s = make_system(cfg_plain_fp64())
    got = _run(lib, s)
    _check_all(s, got)


@pytest.mark.parametrize("case", [
    dict(kgrid=(3, 3, 2), q_frac=((1 / 3, 2 / 3, 0.5),), fft=(20, 18, 22), ng=45, n_occ=3,
         n_bands=11, npw_target=60, a=7.0, freqs=(0.02j, 0.3j, 2.0j), eta=0.0),
    dict(kgrid=(2, 2, 2), q_frac=((0.5, 0.5, 0.0),), fft=(16, 16, 16), ng=1, n_occ=2,
         n_bands=5, npw_target=25, freqs=(0j,), eta=0.01),
    dict(kgrid=(4, 2, 2), q_frac=((0.75, 0.5, 0.0),), fft=(18, 18, 18), ng=70, n_occ=5,
         n_bands=9, npw_target=45, a=8.0, freqs=(0.5j,), eta=0.0),
])
def test_ragged_shapes(lib, case):
    s = make_system(cfg_tiny(seed=31, **case))
    _check_all(s, _run(lib, s))


def test_no_transitions_gives_identity(lib):
    s = make_system(cfg_tiny(seed=3, n_occ=2, n_bands=5, freqs=(0.2j,), eta=0.0))
    s.occ[:] = 0.0  # an empty system: no transition has weight
    got = _run(lib, s, rho=False)
    assert np.abs(got["chi"]).max() == 0.0
    assert np.abs(got["inv"] - np.eye(s.ng)[None]).max() == 0.0


def test_alias_check(lib):
    import torch
    s = make_system(cfg_tiny(seed=3, fft=(6, 6, 6)))  # 6 <= 2 L + max|G - G0| = 6
    ctx = lib.Chi0.for_system(s, stream=torch.cuda.current_stream().cuda_stream)
    ctx.load_system(s)
    with pytest.raises(lib.Chi0Error) as ei:
        ctx.compute_rho(0)
    assert ei.value.status == -1 and "alias" in str(ei.value)
    ctx.close()


def test_repeat_is_bitwise_deterministic(lib):
    s = make_system(cfg_tiny(seed=8, freqs=(0.1j,), eta=0.0))
    a = _run(lib, s)
    b = _run(lib, s)
    assert np.array_equal(a["chi"], b["chi"]) and np.array_equal(a["inv"], b["inv"])
