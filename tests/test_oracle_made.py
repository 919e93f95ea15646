"""Pins for the FP64 MADE reference (oracle/made.py), CPU only.

Normalisation over all 2^M patterns and the autoregressive property follow
from the masks alone, and central finite differences check the analytic
gradient; a mistake in a mask, a sign or a layer of the backward pass fails
one of them.
"""
import numpy as np
import pytest

from oracle import made


@pytest.mark.parametrize("M,H,seed", [(3, 16, 1), (6, 32, 2), (8, 16, 3)])
def test_normalised_over_all_patterns(M, H, seed):
    th = made.random_theta(M, H, seed, scale=2.0)
    X = made.all_patterns(M)
    assert abs(np.exp(made.logq(th, X, M, H)).sum() - 1.0) < 1e-12


@pytest.mark.parametrize("M,H", [(5, 16), (9, 32)])
def test_autoregressive(M, H):
    th = made.random_theta(M, H, 7, scale=2.0)
    rng = np.random.default_rng(0)
    X = (rng.random((50, M)) < 0.5).astype(float)
    l0, _ = made.forward(th, X, M, H)
    for i in range(M):
        X2 = X.copy()
        X2[:, i] = 1 - X2[:, i]
        l1, _ = made.forward(th, X2, M, H)
        assert np.all(l1[:, :i + 1] == l0[:, :i + 1])     # l_j, j <= i, ignores x_i
    # and the masks are not trivially empty: the last logit depends on x_0
    X3 = X.copy()
    X3[:, 0] = 1 - X3[:, 0]
    assert np.any(made.forward(th, X3, M, H)[0][:, M - 1] != l0[:, M - 1])


def test_gradient_matches_finite_differences():
    M, H = 5, 16
    th = made.random_theta(M, H, 11, scale=1.5)
    rng = np.random.default_rng(3)
    X = (rng.random((40, M)) < 0.4).astype(float)
    w = rng.random(40) + 0.1
    L, g = made.loss_and_grad(th, X, w, M, H)
    mk = made.flatten([m if i % 2 == 0 else np.ones(s) for i, (m, s) in
                       enumerate(zip([made.masks(M, H)[i // 2] for i in range(8)], made.shapes(M, H)))])
    idx = rng.choice(th.size, 60, replace=False)
    for i in idx:
        if mk[i] == 0:
            assert g[i] == 0
            continue
        e = np.zeros_like(th)
        e[i] = 1e-6
        fd = (made.loss_and_grad(th + e, X, w, M, H)[0] - made.loss_and_grad(th - e, X, w, M, H)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_masks_follow_degree_rule():
    m1, m2, m3, m4 = made.masks(4, 6)
    # hidden degrees 1,2,3,1,2,3: unit 0 sees input 0 only, unit 2 sees inputs 0..2
    assert m1[0].tolist() == [1, 0, 0, 0] and m1[2].tolist() == [1, 1, 1, 0]
    # output 0 sees nothing, output 3 sees all hidden units (degrees <= 3)
    assert m4[0].sum() == 0 and m4[3].sum() == 6
