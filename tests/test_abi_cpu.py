"""Host-side checks of libchi0 that need no GPU: the library loads, exports
every entry point that include/chi0.h declares, validates its arguments,
reports call-order errors, injects allocation failures on request, and
computes the response G set (host logic) exactly as the oracle does."""
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def binding():
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0
    return chi0


def _declared():
    txt = open(os.path.join(ROOT, "include", "chi0.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(chi0_[a-z_0-9]+)\s*\(", txt)))


def test_exports_match_header(binding):
    import ctypes
    lib = ctypes.CDLL(binding.LIB_PATH)
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(binding.EXPORTS)


def test_binding_declares_every_signature(binding):
    """Every entry point with arguments has ctypes argtypes: an undeclared
    pointer argument would be passed as a 32-bit int."""
    import re
    src = open(binding.__file__).read()
    for n in binding.EXPORTS:
        assert re.search(rf"lib\.{n}\.argtypes\s*=", src), n
        fn = getattr(binding._lib, n)
        assert fn.argtypes is not None, n


def _ctx(binding, **over):
    kw = dict(a=10.0, kgrid=(4, 4, 4), nbands=32, npw_max=305, fft=(24, 24, 24), ng=59,
              q_frac=[(0.25, 0, 0)], omega=[0j], eta=0.1 / 27.211386245988)
    kw.update(over)
    return binding.Chi0(**kw)


def test_create_validation(binding):
    for over, status in (({"ng": 0}, -1), ({"ng": 5000}, -1), ({"time_reversal": 0}, -8),
                         ({"q_frac": [(0.3, 0, 0)]}, -1), ({"precision": 7}, -1),
                         ({"eta": -1.0}, -1), ({"kgrid": (0, 4, 4)}, -1)):
        with pytest.raises(binding.Chi0Error) as ei:
            _ctx(binding, **over)
        assert ei.value.status == status, over


def test_call_order_and_arguments(binding):
    c = _ctx(binding)
    with pytest.raises(binding.Chi0Error) as ei:
        c.compute_rho(0)
    assert ei.value.status == -4  # ESTATE: no wavefunctions yet
    with pytest.raises(binding.Chi0Error) as ei:
        c.build_chi0(0, np.zeros((1, 59, 59), np.complex128))
    assert ei.value.status == -4
    with pytest.raises(binding.Chi0Error) as ei:
        c.compute_rho(3)
    assert ei.value.status == -1
    with pytest.raises(binding.Chi0Error) as ei:
        c.set_wavefunctions(64, np.zeros((3, 3), np.int32), np.zeros((32, 3), np.complex128))
    assert ei.value.status == -1
    with pytest.raises(binding.Chi0Error) as ei:
        c.set_energies(np.full((64, 32), np.nan), np.zeros((64, 32)))
    assert ei.value.status == -1
    with pytest.raises(binding.Chi0Error) as ei:
        c.set_energies(np.zeros((64, 32)), np.full((64, 32), 2.0))
    assert ei.value.status == -1
    c.close()


def test_new_entry_points_reject_bad_arguments(binding):
    """Argument and call-order checks of the plasmon-pole, self-energy,
    grouping and double-grid entry points; all of them return before any
    device memory is touched (the non-NULL pointers below are never read)."""
    import ctypes
    lib = binding._lib
    fake = ctypes.c_void_p(16)
    assert lib.chi0_ppa_fit(None, fake, 4, 1.0, fake, fake, None) == -1
    assert lib.chi0_ppa_fit(fake, fake, 0, 1.0, fake, fake, None) == -1
    assert lib.chi0_ppa_fit(fake, fake, 4, 0.0, fake, fake, None) == -1
    assert lib.chi0_ppa_fit(fake, fake, 4, float("nan"), fake, fake, None) == -1
    assert lib.chi0_ppa_eval(fake, fake, 4, None, 1, 0.0, fake, None) == -1      # nf > 0 needs frequencies
    f = (ctypes.c_double * 2)(0.3, float("inf"))
    assert lib.chi0_ppa_eval(fake, fake, 4, f, 1, 0.0, fake, None) == -1
    assert lib.chi0_ppa_eval(fake, fake, 4, f, 1, -1.0, fake, None) == -1
    c = _ctx(binding)
    h = c.h
    assert lib.chi0_build_sigma_i(h, 0, 5, 5, fake, 1, fake, 1) == -1            # empty window
    assert lib.chi0_build_sigma_i(h, 0, 30, 33, fake, 1, fake, 1) == -1          # beyond nbands = 32
    assert lib.chi0_build_sigma_i(h, 0, 0, 4, None, 1, fake, 1) == -1
    assert lib.chi0_build_sigma_i(h, 0, 0, 4, fake, 0, fake, 1) == -1
    assert lib.chi0_build_sigma_i(h, 1, 0, 4, fake, 1, fake, 1) == -1            # iq out of range
    assert lib.chi0_build_sigma_i(h, 0, 0, 4, fake, 1, fake, 1) == -4            # compute_rho first
    with pytest.raises(binding.Chi0Error) as ei:
        c.set_pole_grouping(-1e-5)
    assert ei.value.status == -1
    with pytest.raises(binding.Chi0Error) as ei:
        c.set_pole_grouping(float("nan"))
    assert ei.value.status == -1
    assert lib.chi0_set_double_grid(h, -1, None) == -1
    assert lib.chi0_set_double_grid(h, 2, None) == -1
    bad = np.zeros((64, 2, 32))
    bad[3, 1, 7] = np.inf
    with pytest.raises(binding.Chi0Error) as ei:
        c.set_double_grid(bad)
    assert ei.value.status == -1
    c.set_pole_grouping(1e-5)
    with pytest.raises(binding.Chi0Error) as ei:                               # the two exclude each other
        c.set_double_grid(np.zeros((64, 2, 32)))
    assert ei.value.status == -1
    c.set_pole_grouping(0.0)
    c.set_double_grid(None)
    with pytest.raises(binding.Chi0Error) as ei:
        c.set_bg_terminator(float("nan"))
    assert ei.value.status == -1
    c.close()


def test_noalloc_wrapper_rejects_mismatched_arguments(binding):
    """invert_eps_noalloc checks dtype, shape, contiguity and the length of
    v_sqrt before it calls the library (a short v_sqrt would be read past its
    end, a smaller out written past its end)."""
    import torch
    ok = torch.zeros((2, 5, 5), dtype=torch.complex128)
    v = np.ones(5)
    cases = [
        (ok.to(torch.complex64), v, ok),                 # wrong dtype of chi0
        (ok, v, ok.to(torch.complex64)),                 # wrong dtype of out
        (torch.zeros((2, 5, 4), dtype=torch.complex128), v, ok),   # not square
        (ok, v, torch.zeros((1, 5, 5), dtype=torch.complex128)),   # shapes differ
        (ok.transpose(1, 2), v, ok),                     # not contiguous
        (ok, np.ones(4), ok),                            # short v_sqrt
        (ok, v, ok),                                     # host tensors
    ]
    for c, vv, o in cases:
        with pytest.raises(ValueError):
            binding.invert_eps_noalloc(c, vv, o)


def test_injected_allocation_failure(binding, monkeypatch):
    c = _ctx(binding)
    monkeypatch.setenv("CHI0_FAULT", "alloc")
    with pytest.raises(binding.Chi0Error) as ei:
        c.set_wavefunctions(0, np.zeros((3, 3), np.int32), np.zeros((32, 3), np.complex128))
    assert ei.value.status == -2 and "injected" in str(ei.value)
    c.close()


@pytest.mark.parametrize("kgrid,q,ng", [((4, 4, 4), (0.25, 0, 0), 59), ((8, 8, 8), (0.25, 0, 0), 1000),
                                        ((3, 3, 2), (1 / 3, 2 / 3, 0.5), 77), ((6, 6, 6), (1 / 6, 0, 0), 500)])
def test_response_gvectors_match_oracle(binding, kgrid, q, ng):
    c = _ctx(binding, kgrid=kgrid, q_frac=[q], ng=ng)
    got = c.get_response_gvectors(0)
    want = O.response_gvectors(kgrid, q, ng)
    assert np.array_equal(got, want)
    c.close()
