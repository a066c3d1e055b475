"""Learned band-sum terminator on the GPU.

1. The network kernels against the FP64 oracle (oracle/mlp.py, itself pinned
   by finite differences): loss, gradient, prediction and Adam step agree to
   2e-5 relative with FP32 operands; with BF16 operands (FP32 accumulation)
   the gradient agrees to the BF16 rounding level (3e-2 relative).
2. Trained on truncated/full-band chi0 pairs of seeded systems, the network
   reduces the error of the truncated chi0 against the full-band sum on
   held-out systems, and chi0_build_chi0 with the terminator set reproduces
   chi0_trunc + the Hermitised correction.
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from synth import cfg_learned, make_system, truncate_bands

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_1902_03837_gb300 import chi0
    return chi0


def _rand(seed, B):
    rng = np.random.default_rng(seed)
    p = omlp.init_params(seed) + 0.02 * rng.standard_normal(omlp.n_params())
    x = rng.standard_normal((B, 5))
    t = rng.standard_normal((B, 2)) * 0.3
    return p, x, t


@pytest.mark.parametrize("B", [1, 45, 200])
def test_loss_grad_predict_vs_oracle(lib, B):
    import torch
    p, x, t = _rand(B, B)
    L_ref, g_ref = omlp.loss_and_grad(p, x, t)
    dev = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda().contiguous()  # noqa: E731
    P, X, T = dev(p), dev(x), dev(t)
    G = torch.zeros_like(P)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = torch.empty(lib.mlp_workspace_floats(B), dtype=torch.float32, device="cuda")
    # operands as the GPU sees them (FP32): compare with the oracle on the same FP32 values
    p32, x32, t32 = (np.asarray(a, np.float32).astype(np.float64) for a in (p, x, t))
    L_ref, g_ref = omlp.loss_and_grad(p32, x32, t32)
    lib.mlp_loss_grad(P, X, T, G, loss, work, bf16=False)
    g = G.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - L_ref) < 2e-5 * abs(L_ref)
    assert np.abs(g - g_ref).max() < 2e-5 * np.abs(g_ref).max()
    Y = torch.zeros((B, 2), dtype=torch.float32, device="cuda")
    lib.mlp_predict(P, X, Y, bf16=False)
    y_ref = omlp.forward(p32, x32)
    assert np.abs(Y.cpu().numpy() - y_ref).max() < 2e-5 * max(1.0, np.abs(y_ref).max())
    # BF16 operands: same quantities to BF16 accuracy
    lib.mlp_loss_grad(P, X, T, G, loss, work, bf16=True)
    gb = G.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gb - g_ref) < 3e-2 * np.linalg.norm(g_ref)


def test_adam_vs_oracle(lib):
    import torch
    rng = np.random.default_rng(7)
    n = omlp.n_params()
    p = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    m = np.zeros(n)
    v = np.zeros(n)
    P = torch.from_numpy(p.astype(np.float32)).cuda()
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    for step in range(1, 4):
        g = rng.standard_normal(n).astype(np.float32).astype(np.float64)
        p, m, v = omlp.adam_step(p, g, m, v, step, lr=1e-2)
        lib.mlp_adam(P, torch.from_numpy(g.astype(np.float32)).cuda(), M, V, 1e-2, step)
    assert np.abs(P.cpu().numpy() - p).max() < 1e-5


def test_learned_terminator_gain_on_held_out_systems(lib):
    """Reduced learned-terminator case: 4x4x4 k, 8 occupied, truncated 24 vs
    full 96 bands, ~300 PW, FFT 24^3, N_G = 59, 8 imaginary frequencies;
    24 training systems, 8 held-out systems."""
    import torch
    from paper_1902_03837_gb300 import terminator as term
    stream = torch.cuda.current_stream().cuda_stream

    def system(seed):
        spec = cfg_learned(seed=seed, full_bands=96, n_occ=8, kgrid=(4, 4, 4), kc=2.6049,
                           fft=(24, 24, 24), ng=59, nw=8)
        full = make_system(spec)
        return full, truncate_bands(full, 24)

    X, T = [], []
    for seed in range(4000, 4024):
        full, trunc = system(seed)
        x, t, _, _, _ = term.pair(full, trunc, lib.CHI0_MIXED_BF16X3, stream)
        X.append(x)
        T.append(t)
    X = torch.cat(X)
    T = torch.cat(T)
    params, hist = term.train(X, T, steps=3000, batch=4096, lr=2e-3, seed=1, stream=stream, log_every=500)
    assert hist[-1][1] < hist[0][1]
    e_trunc, e_term = [], []
    for seed in range(5000, 5008):
        full, trunc = system(seed)
        _, chi_f = term.chi0_device(full, lib.CHI0_MIXED_BF16X3, stream)
        ctx_t, chi_t = term.chi0_device(trunc, lib.CHI0_MIXED_BF16X3, stream)
        ctx_c, chi_c = term.chi0_device(trunc, lib.CHI0_MIXED_BF16X3, stream, params=params)
        # chi_c must be chi_t plus an exactly Hermitian correction
        d = chi_c - chi_t
        assert (d - d.conj().transpose(1, 2)).abs().max().item() == 0.0
        nf = torch.linalg.norm(chi_f).item()
        e_trunc.append(torch.linalg.norm(chi_t - chi_f).item() / nf)
        e_term.append(torch.linalg.norm(chi_c - chi_f).item() / nf)
        for c in (ctx_t, ctx_c):
            c.close()
    e_trunc, e_term = np.array(e_trunc), np.array(e_term)
    print(f"held-out relative error: truncated {e_trunc.mean():.4f} +- {e_trunc.std():.4f}, "
          f"truncated + network {e_term.mean():.4f} +- {e_term.std():.4f}")
    assert e_term.mean() < 0.5 * e_trunc.mean()
    assert np.all(e_term < e_trunc)
