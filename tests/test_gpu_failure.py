"""Failure detection on the GPU without a fault: every spin-wait of the
contraction is bounded, gives up after about two seconds, raises the
context's device error flag and returns.  chi0_check_bounded_wait queues one
such wait on a barrier that nothing completes; the next synchronising call
must report CHI0_ETIMEOUT, clear the flag, and leave the context usable (the
next chi0 equals that of a fresh context, which it would not if the flag had
stayed up: the contraction skips its work while the flag is set)."""
import time

import numpy as np
import pytest

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


def _chi(lib, ctx, s):
    ctx.compute_rho(0)
    chi = np.zeros((s.freqs.size, s.ng, s.ng), np.complex128)
    ctx.build_chi0(0, chi)
    return chi


def test_bounded_wait_gives_up_and_context_recovers(lib):
    import torch
    s = make_system(cfg_tiny(seed=97, kgrid=(2, 2, 2), q_frac=((0.5, 0.0, 0.0),), fft=(16, 16, 16), ng=30,
                             n_occ=4, n_bands=10, npw_target=40, a=7.0, freqs=(0.1j, 1.0j), eta=0.0,
                             coef_dtype="c64"))
    stream = torch.cuda.current_stream().cuda_stream
    ctx = lib.Chi0.for_system(s, precision=1, stream=stream)
    ctx.load_system(s)
    t0 = time.perf_counter()
    ctx.check_bounded_wait()
    with pytest.raises(lib.Chi0Error, match="ETIMEOUT"):
        ctx.synchronize()
    waited = time.perf_counter() - t0
    print(f"the bounded wait gave up after {waited:.2f} s")
    assert 0.2 < waited < 30.0
    ctx.synchronize()                      # the flag was cleared by the report
    got = _chi(lib, ctx, s)
    ctx.close()
    fresh = lib.Chi0.for_system(s, precision=1, stream=stream)
    fresh.load_system(s)
    ref = _chi(lib, fresh, s)
    fresh.close()
    assert np.array_equal(got, ref) and np.abs(ref).max() > 0
