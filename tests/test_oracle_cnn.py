"""Pins of the warm-start network oracle (oracle/cnn_oracle.py) against
brute force, adjoint identities, finite differences and closed forms."""
import numpy as np
import pytest

from oracle import cnn_oracle as C


def test_bf16_rounding_bit_patterns():
    f = np.float32
    # representable values pass unchanged
    for v in (1.0, -2.5, 0.0, 3.0 * 2.0 ** -20):
        assert C.bf16_round(f(v)) == f(v)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even (mantissa 0)
    assert C.bf16_round(f(1 + 2 ** -8)) == f(1.0)
    # 1 + 3 2^-8 is halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert C.bf16_round(f(1 + 3 * 2 ** -8)) == f(1 + 2 ** -6)
    # just above the midpoint rounds up; sign symmetric
    assert C.bf16_round(f(1 + 2 ** -8 + 2 ** -20)) == f(1 + 2 ** -7)
    assert C.bf16_round(f(-(1 + 2 ** -8 + 2 ** -20))) == f(-(1 + 2 ** -7))
    # the result always has 16 zero low bits
    x = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    assert np.all(C.bf16_round(x).view(np.uint32) & 0xFFFF == 0)
    assert np.abs(C.bf16_round(x) - x).max() <= np.abs(x).max() * 2.0 ** -8


def test_conv_matches_brute_force_loop():
    rng = np.random.default_rng(1)
    ci, co, H, W = 2, 3, 5, 4
    A = rng.standard_normal((ci, H, W))
    Wt = rng.standard_normal((co, 3, 3, ci))
    b = rng.standard_normal(co)
    Z = C.conv3x3(A, Wt, b)
    for o in range(co):
        for y in range(H):
            for x in range(W):
                s = b[o]
                for i in range(ci):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            s += Wt[o, dy + 1, dx + 1, i] * A[i, (y + dy) % H, (x + dx) % W]
                assert Z[o, y, x] == pytest.approx(s, abs=1e-12)


def test_conv_is_shift_equivariant():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((3, 7, 6))
    Wt = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    lhs = C.conv3x3(np.roll(A, (2, -3), axis=(1, 2)), Wt, b)
    rhs = np.roll(C.conv3x3(A, Wt, b), (2, -3), axis=(1, 2))
    assert np.abs(lhs - rhs).max() < 1e-12


def test_transpose_and_weight_gradient_are_adjoints():
    """<conv(A, W), G> = <A, conv^T(G, W)> = <W, wgrad(G, A)>."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, 6, 5))
    Wt = rng.standard_normal((4, 3, 3, 3))
    G = rng.standard_normal((4, 6, 5))
    lhs = np.sum(C.conv3x3(A, Wt, np.zeros(4)) * G)
    assert np.sum(A * C.conv3x3_transpose(G, Wt)) == pytest.approx(lhs, rel=1e-12)
    assert np.sum(Wt * C.conv3x3_wgrad(G, A)) == pytest.approx(lhs, rel=1e-12)


def test_zero_network_passes_the_state_through():
    params = [(np.zeros_like(W), np.zeros_like(b)) for W, b in C.init_params(0)]
    X = np.random.default_rng(4).standard_normal((3, 8, 8))
    Y, _ = C.forward(params, X)
    assert np.all(Y == 0)
    rho, T = np.full((8, 8), 3.4), np.full((8, 8), 0.41)
    X = C.encode(rho, T, 0.4, 3.5, 4 / 7)
    r2, T2 = C.decode(X, np.zeros((2, 8, 8)), 0.4, 3.5)
    assert np.allclose(r2, rho, rtol=1e-14) and np.allclose(T2, T, rtol=1e-14)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(5)
    params = C.init_params(7, scale=1.0)
    params[-1] = (params[-1][0] * 10, rng.standard_normal(2) * 0.1)
    X = rng.standard_normal((3, 6, 5))
    Xt = rng.standard_normal((2, 6, 5))
    L0, grads = C.loss_and_grads(params, X, Xt)
    h = 1e-6
    for l in range(len(params)):
        for j in range(2):                                   # weights, biases
            arr = params[l][j]
            idx = [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(6)]
            for ix in idx:
                def L_at(delta):
                    p2 = [(W.copy(), b.copy()) for W, b in params]
                    p2[l][j][ix] += delta
                    return C.loss_and_grads(p2, X, Xt)[0]
                fd = (L_at(h) - L_at(-h)) / (2 * h)
                an = grads[l][j][ix]
                assert an == pytest.approx(fd, rel=1e-5, abs=1e-9), (l, j, ix)


def test_adam_first_step_closed_form():
    """With zero moments the first bias-corrected step is
    w - lr g / (|g| + eps)."""
    W = np.array([[[[1.0, -2.0]]]]).repeat(3, 1).repeat(3, 2)
    b = np.array([0.5])
    g = (np.full_like(W, 0.25), np.array([-4.0]))
    st = {}
    (W1, b1), = C.adam_step([(W, b)], [g], st, lr=1e-3)
    assert np.allclose(W1, W - 1e-3 * 0.25 / (0.25 + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(b1, b + 1e-3 * 4.0 / (4.0 + 1e-8), rtol=0, atol=1e-15)
    # second step with the same gradient: still one lr per step (m/sqrt(v) = sign)
    (W2, _), = C.adam_step([(W1, b1)], [g], st, lr=1e-3)
    assert np.allclose(W2, W1 - 1e-3 * 0.25 / (0.25 + 1e-8), atol=1e-12)


def test_bf16_mode_stays_close_to_fp64():
    """The bfloat16 roundings perturb the output by O(2^-8) relative."""
    rng = np.random.default_rng(6)
    params = C.init_params(3)
    X = rng.standard_normal((3, 8, 8))
    Y64, _ = C.forward(params, X)
    Y16, _ = C.forward(params, X, bf16=True)
    assert np.abs(Y16 - Y64).max() <= 4 * 2.0 ** -8 * np.abs(Y64).max()
