"""FP64 reference of the MADE proposal network -- TEST INFRASTRUCTURE ONLY.

The learned independence proposal is not in the paper (which samples by
MCMC, Sec. 7.1.1, without fixing a proposal); it is a masked autoregressive
network (Germain et al., MADE, ICML 2015).  This module restates it in plain
numpy float64 from that definition, independently of the CUDA library, so
that the GPU's BF16 forward and backward passes can be checked:

  degrees: input j -> j + 1; hidden unit h -> 1 + (h mod (M - 1));
  hidden unit h sees inputs/hidden units of degree <= its own;
  output j sees hidden units of degree <= j (so l_j depends on x_<j only);
  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3),
  l = W4 h3 + b4;  log q(x) = sum_j x_j log s(l_j) + (1 - x_j) log s(-l_j).

Parameter vector order (as the library's get/set): W1[H x M], b1, W2[H x H],
b2, W3[H x H], b3, W4[M x H], b4[M], row-major.
"""
from __future__ import annotations

import numpy as np


def degrees_hidden(M: int, H: int) -> np.ndarray:
    return 1 + (np.arange(H) % (M - 1))


def masks(M: int, H: int):
    """The four 0/1 weight masks, shapes [H x M], [H x H], [H x H], [M x H]."""
    din = np.arange(1, M + 1)
    dh = degrees_hidden(M, H)
    m1 = (dh[:, None] >= din[None, :]).astype(np.float64)
    m2 = (dh[:, None] >= dh[None, :]).astype(np.float64)
    m3 = m2.copy()
    m4 = (np.arange(1, M + 1)[:, None] > dh[None, :]).astype(np.float64)
    return [m1, m2, m3, m4]


def shapes(M: int, H: int):
    return [(H, M), (H,), (H, H), (H,), (H, H), (H,), (M, H), (M,)]


def unflatten(theta: np.ndarray, M: int, H: int):
    out, o = [], 0
    for shp in shapes(M, H):
        n = int(np.prod(shp))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(shp))
        o += n
    assert o == theta.size
    return out


def flatten(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def _log_sigmoid(z):
    return -np.logaddexp(0.0, -z)


def forward(theta, X, M, H):
    """logits (B x M) and the hidden activations, in float64."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(theta, M, H)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    h3 = np.maximum(h2 @ W3.T + b3, 0.0)
    logits = h3 @ W4.T + b4
    return logits, (X, h1, h2, h3)


def logq(theta, X, M, H):
    l, (X, *_) = forward(theta, X, M, H)
    return np.sum(X * _log_sigmoid(l) + (1.0 - X) * _log_sigmoid(-l), axis=1)


def loss_and_grad(theta, X, w, M, H):
    """L = -(sum_b w_b log q(x_b)) / sum_b w_b and dL/dtheta (flat), float64."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(theta, M, H)
    w = np.asarray(w, dtype=np.float64)
    wn = w / w.sum()
    l, (X, h1, h2, h3) = forward(theta, X, M, H)
    lq = np.sum(X * _log_sigmoid(l) + (1.0 - X) * _log_sigmoid(-l), axis=1)
    L = -np.sum(wn * lq)
    dl = wn[:, None] * (1.0 / (1.0 + np.exp(-l)) - X)          # dL/dlogits
    gW4, gb4 = dl.T @ h3, dl.sum(0)
    d3 = (dl @ W4) * (h3 > 0)
    gW3, gb3 = d3.T @ h2, d3.sum(0)
    d2 = (d3 @ W3) * (h2 > 0)
    gW2, gb2 = d2.T @ h1, d2.sum(0)
    d1 = (d2 @ W2) * (h1 > 0)
    gW1, gb1 = d1.T @ X, d1.sum(0)
    mk = masks(M, H)
    grads = [gW1 * mk[0], gb1, gW2 * mk[1], gb2, gW3 * mk[2], gb3, gW4 * mk[3], gb4]
    return L, flatten(grads)


def magnitude_logits(theta, X, M, H):
    """Forward pass of |W| and |x| (ReLU-gated like the real pass): the scale of
    each logit's sum of products, used to bound low-precision rounding."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(theta, M, H)
    l, (X, h1, h2, h3) = forward(theta, X, M, H)
    a1 = (np.abs(X) @ np.abs(W1).T + np.abs(b1)) * (h1 > 0)
    a2 = (a1 @ np.abs(W2).T + np.abs(b2)) * (h2 > 0)
    a3 = (a2 @ np.abs(W3).T + np.abs(b3)) * (h3 > 0)
    return a3 @ np.abs(W4).T + np.abs(b4)


def grad_magnitude(theta, X, w, M, H, dl_extra=None):
    """The backward pass run on magnitudes (|dL/dl|, |W|, |x|, ReLU gates of the
    real pass): the scale of each gradient entry's sum of products, used to
    bound low-precision rounding of the gradient.  dl_extra (B x M), if given,
    is added to |dL/dl| (an error already present in dL/dl, carried through)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(theta, M, H)
    w = np.asarray(w, dtype=np.float64)
    wn = w / w.sum()
    l, (X, h1, h2, h3) = forward(theta, X, M, H)
    dl = np.abs(wn[:, None] * (1.0 / (1.0 + np.exp(-l)) - X))
    if dl_extra is not None:
        dl = dl + dl_extra
    m3 = (dl @ np.abs(W4)) * (h3 > 0)
    m2 = (m3 @ np.abs(W3)) * (h2 > 0)
    m1 = (m2 @ np.abs(W2)) * (h1 > 0)
    parts = [m1.T @ np.abs(X), m1.sum(0), m2.T @ np.abs(h1), m2.sum(0), m3.T @ np.abs(h2), m3.sum(0),
             dl.T @ np.abs(h3), dl.sum(0)]
    return flatten(parts)


def preactivations(theta, X, M, H):
    """The three hidden layers' pre-activations (B x H each), float64."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(theta, M, H)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    z2 = np.maximum(z1, 0.0) @ W2.T + b2
    z3 = np.maximum(z2, 0.0) @ W3.T + b3
    return z1, z2, z3


def all_patterns(M: int) -> np.ndarray:
    return ((np.arange(1 << M)[:, None] >> np.arange(M)[None, :]) & 1).astype(np.float64)


def random_theta(M, H, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    mk = masks(M, H)
    for i, shp in enumerate(shapes(M, H)):
        p = rng.normal(0, scale / np.sqrt(shp[-1]), size=shp)
        if i % 2 == 0:
            p = p * mk[i // 2]
        parts.append(p)
    return flatten(parts)


def adam_step(theta, grad, m, v, t, lr, mask=None, b1=0.9, b2=0.999, eps=1e-8):
    """One masked Adam step (Kingma & Ba, ICLR 2015, Algorithm 1) in float64: t is the
    1-based step number; masked entries (mask 0) are not parameters: their gradient counts
    as zero and they stay at zero.  Returns (theta, m, v) after the step."""
    theta = np.asarray(theta, dtype=np.float64)
    mk = np.ones_like(theta) if mask is None else np.asarray(mask, dtype=np.float64)
    g = np.asarray(grad, dtype=np.float64) * mk
    m = b1 * np.asarray(m, dtype=np.float64) + (1.0 - b1) * g        # first moment
    v = b2 * np.asarray(v, dtype=np.float64) + (1.0 - b2) * g * g    # second moment
    m_hat = m / (1.0 - b1 ** t)                                       # bias corrections
    v_hat = v / (1.0 - b2 ** t)
    theta = (theta - lr * m_hat / (np.sqrt(v_hat) + eps)) * mk
    return theta, m, v
