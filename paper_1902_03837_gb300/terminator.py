"""Learned band-sum terminator: training and use (kernels in libchi0).

A truncated chi0 (the first bands of a system) misses the contribution of the
higher bands; the paper's X-terminator (Eq. X_term_def, Appendix C) adds a
closure term for it.  Here a 5 -> 128 -> 128 -> 2 network predicts that term
entry by entry from (|q+G|, |q+G'|, |w|, chi0_trunc), trained on the GPU by
the library's own forward/backward and Adam kernels on pairs of truncated and
full-band chi0 of seeded systems.  The full-band sum remains the reference.
This module only moves device buffers between those library calls.
"""
from __future__ import annotations

import math

import numpy as np

from . import chi0 as lib


def init_params(seed: int):
    """Uniform(-1/sqrt(fan_in), +1/sqrt(fan_in)) weights, zero biases (host float32)."""
    rng = np.random.default_rng(seed)
    i, h, o = 5, 128, 2
    parts = [rng.uniform(-1, 1, (h, i)) / math.sqrt(i), np.zeros(h),
             rng.uniform(-1, 1, (h, h)) / math.sqrt(h), np.zeros(h),
             rng.uniform(-1, 1, (o, h)) / math.sqrt(h), np.zeros(o)]
    p = np.concatenate([a.ravel() for a in parts]).astype(np.float32)
    assert p.size == lib.mlp_nparams()
    return p


def chi0_device(system, precision, stream, params=None, bf16=True):
    """chi0 of `system` at q index 0 into a device tensor; returns (ctx, chi)."""
    import torch
    ctx = lib.Chi0.for_system(system, precision=precision, stream=stream)
    ctx.load_system(system)
    if params is not None:
        ctx.set_terminator(params, bf16)
    ctx.compute_rho(0)
    chi = torch.empty((system.freqs.size, system.ng, system.ng), dtype=torch.complex128, device="cuda")
    ctx.build_chi0(0, chi)
    return ctx, chi


def pair(full_system, truncated_system, precision, stream):
    """(features, targets, chi_trunc, chi_full, scale) of one system."""
    import torch
    ctx_f, chi_f = chi0_device(full_system, precision, stream)
    ctx_t, chi_t = chi0_device(truncated_system, precision, stream)
    n = chi_t.numel()
    x = torch.empty((n, 5), dtype=torch.float32, device="cuda")
    t = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    c = ctx_t.term_features(0, chi_t, x, chi_f, t)
    ctx_t.synchronize()
    ctx_f.close()
    ctx_t.close()
    return x, t, chi_t, chi_f, c


def train(X, T, steps=2000, batch=4096, lr=2e-3, seed=0, bf16=True, stream=None, log_every=0):
    """Adam on minibatches drawn uniformly from (X, T) (device tensors)."""
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    p = torch.from_numpy(init_params(seed)).cuda()
    g = torch.zeros_like(p)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = torch.empty(lib.mlp_workspace_floats(batch), dtype=torch.float32, device="cuda")
    hist = []
    for step in range(1, steps + 1):
        idx = torch.randint(0, X.shape[0], (batch,), device="cuda", generator=gen)
        xb = X.index_select(0, idx).contiguous()
        tb = T.index_select(0, idx).contiguous()
        lib.mlp_loss_grad(p, xb, tb, g, loss, work, bf16=bf16, stream=stream)
        lib.mlp_adam(p, g, m, v, lr, step, stream=stream)
        if log_every and step % log_every == 0:
            hist.append((step, float(loss.item())))
    return p, hist
