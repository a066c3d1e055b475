"""The allocation-free Dyson entry point (chi0_invert_eps_noalloc).

Callers that cannot allocate device memory (memory owned by another
allocator that must account for every byte, or a service held to a fixed
device footprint) use this entry point; its scratch is a static device
array.  Two calls in a row
must agree with chi0_invert_eps, the allocating entry point, within the FP64
tolerance of the other GPU tests (1e-10 relative), which also shows that the
second call starts from a clean error flag and overwrites the first call's
scratch.  This file is collected last so that a run stopping at the first
failure has already run every other test."""
import math

import numpy as np
import pytest

from synth import cfg_tiny, make_system

pytestmark = pytest.mark.gpu


def test_noalloc_matches_invert_eps_twice():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0 as lib

    s = make_system(cfg_tiny(seed=19, kgrid=(3, 3, 2), q_frac=((1 / 3, 2 / 3, 0.5),), fft=(20, 18, 22),
                             ng=70, n_occ=3, n_bands=11, npw_target=60, a=7.0,
                             freqs=(0.02j, 0.3j, 2.0j), eta=0.0))
    stream = torch.cuda.current_stream()
    ctx = lib.Chi0.for_system(s, stream=stream.cuda_stream)
    ctx.load_system(s)
    ctx.compute_rho(0)
    nw, ng = s.freqs.size, s.ng
    chi = torch.zeros((nw, ng, ng), dtype=torch.complex128, device="cuda")
    ctx.build_chi0(0, chi)
    ref = torch.zeros_like(chi)
    ctx.invert_eps(0, ref)
    G = ctx.get_response_gvectors(0)
    ctx.synchronize()
    ctx.close()
    q = s.q_frac[0]
    qg = (2 * math.pi / s.spec.a) * np.sqrt(((G + q[None, :]) ** 2).sum(axis=1))
    v = math.sqrt(4 * math.pi) / qg
    ref_h = ref.cpu().numpy()
    scale = np.linalg.norm(ref_h)
    for _ in range(2):
        out = torch.full_like(chi, complex(float("nan"), 0.0))
        lib.invert_eps_noalloc(chi, v, out, stream.cuda_stream)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.linalg.norm(got - ref_h) / scale < 1e-10
    # sizes beyond the static scratch are refused with a clear status
    big = torch.zeros((1, 2049, 2049), dtype=torch.complex128, device="cuda")
    with pytest.raises(lib.Chi0Error) as ei:
        lib.invert_eps_noalloc(big, np.ones(2049), torch.zeros_like(big), stream.cuda_stream)
    assert ei.value.status == -8
