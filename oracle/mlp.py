"""FP64 reference of the band-sum terminator network (oracle; test infrastructure).

The paper corrects a band-truncated chi0 with the Bruneval-Gonze
X-terminator (Eq. X_term_def and Appendix C): chi0 = chi0^trunc + Delta chi.
Here Delta chi is predicted by a small network from per-entry features; this
module is the plain FP64 definition of that network, its loss gradient and
its Adam update, against which the GPU kernels are checked.  It is pinned by
central finite differences of the loss (tests/test_oracle_mlp.py).  The
accuracy of a *trained* network has no closed form: "parity unpinned" applies
to the terminator's prediction quality, which is judged against the
full-band sum on held-out systems.

Network (n_in = 5, n_hidden = 128, n_out = 2), parameters packed as
    W1[H][I], b1[H], W2[H][H], b2[H], W3[O][H], b3[O]:
    h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),  y = W3 h2 + b3;
loss L = 1/(2B) sum_b sum_o (y_bo - t_bo)^2 over a batch of B samples.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 5, 128, 2


def n_params(i=N_IN, h=N_HID, o=N_OUT):
    return h * i + h + h * h + h + o * h + o


def unpack(p, i=N_IN, h=N_HID, o=N_OUT):
    p = np.asarray(p, dtype=np.float64)
    k = 0
    W1 = p[k:k + h * i].reshape(h, i); k += h * i
    b1 = p[k:k + h]; k += h
    W2 = p[k:k + h * h].reshape(h, h); k += h * h
    b2 = p[k:k + h]; k += h
    W3 = p[k:k + o * h].reshape(o, h); k += o * h
    b3 = p[k:k + o]; k += o
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])


def init_params(seed, i=N_IN, h=N_HID, o=N_OUT):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (h, i)) / np.sqrt(i)
    W2 = rng.uniform(-1, 1, (h, h)) / np.sqrt(h)
    W3 = rng.uniform(-1, 1, (o, h)) / np.sqrt(h)
    return pack(W1, np.zeros(h), W2, np.zeros(h), W3, np.zeros(o))


def forward(p, x):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3.T + b3


def loss_and_grad(p, x, t):
    """L and dL/dp by backpropagation through the three layers."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    B = x.shape[0]
    W1, b1, W2, b2, W3, b3 = unpack(p)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    y = h2 @ W3.T + b3
    r = y - t
    L = 0.5 * float((r * r).sum()) / B
    dy = r / B
    dW3 = dy.T @ h2
    db3 = dy.sum(axis=0)
    dz2 = (dy @ W3) * (1.0 - h2 * h2)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    dW1 = dz1.T @ x
    db1 = dz1.sum(axis=0)
    return L, pack(dW1, db1, dW2, db2, dW3, db3)


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
