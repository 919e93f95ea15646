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


# ---------------------------------------------------------------- Adam step
def test_adam_two_step_worked_example():
    # worked by hand (Kingma & Ba, Algorithm 1; b1 = 0.9, b2 = 0.999, eps = 1e-8, lr = 0.1):
    # step 1, g = (0.1, -0.2): m = 0.1 g, v = 0.001 g^2, m_hat = g, v_hat = g^2, so each
    #   parameter moves by lr g / (|g| + eps): 1 - 0.1 / (1 + 1e-7), -2 + 0.1 / (1 + 5e-8);
    # step 2, g = (0.3, 0): m = 0.9 m + 0.1 g = (0.039, -0.018), v = 0.999 v + 0.001 g^2 =
    #   (9.999e-5, 3.996e-5), m_hat = m / 0.19, v_hat = v / 0.001999, and the step
    #   lr m_hat / (sqrt(v_hat) + eps) gives the values below (exact decimals, 40 digits);
    # the third parameter is masked: it stays 0 whatever its gradient.
    th, m, v = np.array([1.0, -2.0, 0.0]), np.zeros(3), np.zeros(3)
    mask = np.array([1.0, 1.0, 0.0])
    th, m, v = made.adam_step(th, [0.1, -0.2, 5.0], m, v, 1, 0.1, mask)
    assert th[0] == pytest.approx(0.90000000999999900000, abs=1e-15)
    assert th[1] == pytest.approx(-1.90000000499999975000, abs=1e-15)
    th, m, v = made.adam_step(th, [0.3, 0.0, 5.0], m, v, 2, 0.1, mask)
    assert m == pytest.approx([0.039, -0.018, 0.0], abs=1e-17)
    assert v == pytest.approx([9.999e-5, 3.996e-5, 0.0], abs=1e-19)
    assert th[0] == pytest.approx(0.80822190220558925578, abs=1e-15)
    assert th[1] == pytest.approx(-1.83299418432555796374, abs=1e-15)
    assert th[2] == 0.0


def test_adam_constant_gradient_moves_by_lr_each_step():
    # with a constant gradient g the bias-corrected moments are exactly g and g^2 at every
    # step, so every step moves a parameter by lr g / (|g| + eps) (about lr sign(g))
    rng = np.random.default_rng(3)
    g = rng.normal(size=50)
    th0 = rng.normal(size=50)
    th, m, v = th0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 31):
        th, m, v = made.adam_step(th, g, m, v, t, 1e-2)
        assert np.allclose(th, th0 - t * 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)


def test_adam_is_odd_in_the_gradient_and_ignores_masked_entries():
    rng = np.random.default_rng(4)
    th0, mask = rng.normal(size=40), (rng.random(40) < 0.7).astype(float)
    th0 *= mask
    gs = [rng.normal(size=40) for _ in range(4)]
    a = (th0.copy(), np.zeros(40), np.zeros(40))
    b = (th0.copy(), np.zeros(40), np.zeros(40))
    for t, g in enumerate(gs, 1):
        a = made.adam_step(a[0], g, a[1], a[2], t, 3e-3, mask)
        b = made.adam_step(b[0], -g, b[1], b[2], t, 3e-3, mask)
    assert np.allclose(a[0] - th0, -(b[0] - th0), atol=1e-15)    # the step is odd in g
    assert np.all(a[0][mask == 0] == 0) and np.all(a[1][mask == 0] == 0)
