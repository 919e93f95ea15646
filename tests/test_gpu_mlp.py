"""GPU tests of the MADE proposal network against the FP64 reference (oracle/made.py).

BF16 tolerance: each logit is a sum of products carried through three BF16
layers; every BF16 rounding (weights and activations, 8 significant bits) is
at most 2^-9 of the term's magnitude, so |error| <= 2^-6 * (the same forward
pass run on |W| and |x|), which the reference computes.  Gradients pass four
BF16 GEMMs and are checked per layer against the backward pass run on
magnitudes.
"""
import math

import numpy as np
import pytest
import torch

from oracle import made
from paper_2009_01177_gb300.tor import pack_patterns

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = cuda_lib.Context(0)
    yield c
    c.close()


def rand_patterns(B, M, seed, p=0.4):
    rng = np.random.default_rng(seed)
    return (rng.random((B, M)) < p).astype(np.float64)


def test_masks_match_reference(ctx, cuda_lib):
    M, H = 10, 32
    net = cuda_lib.MLP(ctx, M, H, seed=1)
    mk = net.get_params(2)
    ref = made.flatten([m if i % 2 == 0 else np.ones(s) for i, (m, s) in
                        enumerate(zip([made.masks(M, H)[i // 2] for i in range(8)], made.shapes(M, H)))])
    assert np.array_equal(mk, ref.astype(np.float32))
    th = net.get_params(0)
    assert np.all(th[ref == 0] == 0)
    net.close()


@pytest.mark.parametrize("M,H", [(8, 64), (20, 256), (60, 256)])
def test_forward_matches_reference(ctx, cuda_lib, M, H):
    net = cuda_lib.MLP(ctx, M, H, seed=2)
    th = made.random_theta(M, H, 5, scale=1.5)
    net.set_params(th)
    th32 = net.get_params(0).astype(np.float64)       # the FP32 master copy the GPU uses
    X = rand_patterns(100, M, 3)
    l_gpu = net.logits(pack_patterns(X, M).cuda())
    l_ref, _ = made.forward(th32, X, M, H)
    bound = 2.0 ** -6 * made.magnitude_logits(th32, X, M, H) + 1e-6
    assert np.all(np.abs(l_gpu - l_ref) <= bound)
    lq = net.logq(pack_patterns(X, M).cuda()).cpu().numpy()
    lq_ref = made.logq(th32, X, M, H)
    assert np.all(np.abs(lq - lq_ref) <= bound.sum(1) + 1e-5)
    net.close()


@pytest.mark.parametrize("M,H", [(8, 64), (20, 128)])
def test_gradients_match_reference(ctx, cuda_lib, M, H):
    net = cuda_lib.MLP(ctx, M, H, seed=3)
    th = made.random_theta(M, H, 9, scale=1.0)
    net.set_params(th)
    th32 = net.get_params(0).astype(np.float64)
    X = rand_patterns(256, M, 4)
    w = np.random.default_rng(5).random(256) + 0.05
    loss = net.grad(pack_patterns(X, M).cuda(), torch.tensor(w, dtype=torch.float32, device="cuda"))
    g = net.get_params(1).astype(np.float64)
    L_ref, g_ref = made.loss_and_grad(th32, X, w, M, H)
    assert abs(loss - L_ref) <= 2e-2 * max(1.0, abs(L_ref))
    # Four BF16 GEMMs deep: per layer, the error is within 2^-9 of the norm of the
    # backward pass run on magnitudes (measured: <= 6e-4 of it).  Single entries can
    # differ by a whole term where a ReLU gate sits within rounding of zero, so the
    # check is per layer, with the gradient's direction on top (a transposed operand
    # or a missing gate would turn it).
    mag = made.grad_magnitude(th32, X, w, M, H)
    o = 0
    for shp in made.shapes(M, H):
        n = int(np.prod(shp))
        a, b, m = g[o:o + n], g_ref[o:o + n], mag[o:o + n]
        o += n
        assert np.linalg.norm(a - b) <= 2.0 ** -9 * np.linalg.norm(m), shp
        assert a @ b >= 0.99 * np.linalg.norm(a) * np.linalg.norm(b), shp
    net.close()


def test_gradients_per_entry_with_all_units_active(ctx, cuda_lib):
    # small weights and positive hidden biases keep every pre-activation far from the ReLU
    # kink, so the GPU and the reference gate the same units and every entry can be bounded:
    # the logits carry at most 2^-6 of their magnitude sum (forward bound above), which
    # moves dL/dl by at most w/4 of that; four BF16 roundings (2^-9 each) on the way back
    # stay within 2^-6 of the backward pass on magnitudes seeded with that extra error.
    M, H, B = 12, 64, 256
    net = cuda_lib.MLP(ctx, M, H, seed=8)
    parts = made.unflatten(made.random_theta(M, H, 11, scale=0.3), M, H)
    for i in (1, 3, 5):
        parts[i] = np.full(H, 3.0)
    net.set_params(made.flatten(parts))
    th32 = net.get_params(0).astype(np.float64)
    X = rand_patterns(B, M, 12)
    assert min(z.min() for z in made.preactivations(th32, X, M, H)) > 1.0     # all active, with margin
    w = np.random.default_rng(13).random(B) + 0.05
    net.grad(pack_patterns(X, M).cuda(), torch.tensor(w, dtype=torch.float32, device="cuda"))
    g = net.get_params(1).astype(np.float64)
    _, g_ref = made.loss_and_grad(th32, X, w, M, H)
    wn = w / w.sum()
    dl_err = wn[:, None] * 2.0 ** -8 * made.magnitude_logits(th32, X, M, H)
    bound = 2.0 ** -6 * made.grad_magnitude(th32, X, w, M, H) + made.grad_magnitude(th32, X, w, M, H, dl_err) \
        - made.grad_magnitude(th32, X, w, M, H) + 1e-9
    assert np.all(np.abs(g - g_ref) <= bound)
    mk = net.get_params(2)
    assert np.all(g[mk == 0] == 0)                       # masked entries have no gradient
    net.close()


def test_adam_update_matches_reference(ctx, cuda_lib):
    # the optimizer arithmetic alone: each step's update of the FP32 master weights against
    # the FP64 masked Adam step of the oracle, given the gradient the GPU computed for it
    M, H, B, lr = 10, 64, 128, 1e-3
    net = cuda_lib.MLP(ctx, M, H, seed=9)
    net.set_params(made.random_theta(M, H, 14, scale=1.0))
    mask = net.get_params(2).astype(np.float64)
    X = pack_patterns(rand_patterns(B, M, 15), M).cuda()
    w = torch.rand(B, device="cuda", dtype=torch.float32) + 0.05
    theta = net.get_params(0).astype(np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    for t in range(1, 5):
        net.train_step(X, w, lr=lr)
        g = net.get_params(1).astype(np.float64)
        new = net.get_params(0).astype(np.float64)
        ref, m, v = made.adam_step(theta, g, m, v, t, lr, mask)
        # FP32 arithmetic: the update (about lr) to a few parts in 1e6, the weight to its rounding
        assert np.all(np.abs(new - ref) <= 1e-5 * lr + 2.0 ** -22 * np.abs(ref)), t
        assert np.all(new[mask == 0] == 0)
        theta = new
    net.close()


def test_sampling_matches_its_own_density(ctx, cuda_lib):
    M, H, B = 6, 64, 16384
    net = cuda_lib.MLP(ctx, M, H, seed=4)
    net.set_params(made.random_theta(M, H, 6, scale=1.5))
    pats, lq = net.sample(B, seed=99, step=1)
    lq2 = net.logq(pats)
    assert torch.allclose(lq, lq2, atol=1e-5)
    # empirical frequencies against q(x) over all 64 patterns
    codes = pats[:, 0].cpu().numpy()
    freq = np.bincount(codes, minlength=1 << M) / B
    allx = made.all_patterns(M)
    q = np.exp(net.logq(pack_patterns(allx, M).cuda()).cpu().numpy())
    assert abs(q.sum() - 1) < 1e-4                      # the network is normalised
    assert 0.5 * np.abs(freq - q).sum() < 0.03
    net.close()


def test_training_moves_q_toward_target(ctx, cuda_lib):
    # target: a correlated distribution over M = 8 patterns (weights = probabilities)
    M, H = 8, 128
    allx = made.all_patterns(M)
    score = allx @ np.linspace(-1, 1, M) + 1.5 * allx[:, 0] * allx[:, -1] - 0.8 * allx.sum(1)
    p = np.exp(score)
    p /= p.sum()
    net = cuda_lib.MLP(ctx, M, H, seed=7)
    P = pack_patterns(allx, M).cuda()
    w = torch.tensor(p, dtype=torch.float32, device="cuda")

    def kl():
        q = np.exp(net.logq(P).cpu().numpy())
        return float(np.sum(p * (np.log(p) - np.log(q))))

    k0 = kl()
    for _ in range(300):
        net.train_step(P, w, lr=3e-3)
    k1 = kl()
    assert k1 < 0.1 * k0 and k1 < 0.02, (k0, k1)
    net.close()
