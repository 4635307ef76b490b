"""Pins for the split oracle (bf16/tf32 rounding, block exponents, hi/lo
split) and the cost-model MLP oracle (forward, backward, Adam), each against a
library routine, a textbook restatement or a closed form."""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

import workloads as W
from oracle import mlp, split


def _special_values():
    f = np.float32
    vals = [0.0, -0.0, 1.0, -1.0, 1.00390625, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9,
            1.0 + 2 ** -8 + 2 ** -9, 65504.0, 3.3895314e38, -3.3895314e38,
            np.finfo(np.float32).max, np.finfo(np.float32).tiny, 2 ** -140, -2 ** -149,
            np.inf, -np.inf, 1e-39, 7.0e-45, 0.1, -0.3, 1.0 / 3.0]
    return np.array(vals, dtype=f)


def test_round_bf16_matches_torch_conversion():
    rng = np.random.default_rng(0)
    x = np.concatenate([_special_values(),
                        W.uniform(1, 5000, 3).ravel(),
                        W.wide_range(1, 5000, 4, lo=-126, hi=127).ravel(),
                        rng.standard_normal(5000).astype(np.float32) * 1e-38])
    ours = split.round_bf16(x)
    ref = torch.from_numpy(x.copy()).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))
    nan = split.round_bf16(np.array([np.nan], np.float32))
    assert np.isnan(nan).all()


def _tf32_textbook(x: float) -> float:
    """Round a normal float to 11 significant bits, ties to even (frexp form)."""
    if x == 0.0 or not math.isfinite(x):
        return x
    m, e = math.frexp(x)            # x = m * 2**e, 0.5 <= |m| < 1
    q = Fraction(m) * 2 ** 11       # 11 significant bits
    r = round(q)                    # Python rounds half to even
    return float(Fraction(r) / 2 ** 11 * Fraction(2) ** e)


def test_round_tf32_matches_textbook_rounding_on_normals():
    x = np.concatenate([W.uniform(1, 3000, 5).ravel(),
                        W.wide_range(1, 3000, 6, lo=-100, hi=100).ravel(),
                        np.array([1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11, 1.0 + 2 ** -11 + 2 ** -20,
                                  -(1.0 + 2 ** -11)], np.float32)])
    ours = split.round_tf32(x)
    ref = np.array([_tf32_textbook(float(v)) for v in x], np.float32)
    assert np.array_equal(ours, ref)
    assert not (ours.view(np.uint32) & 0x1FFF).any()


def test_block_exponent_closed_forms():
    # inside the safe range [2^-48, 2^48): no scaling
    for v in (1.0, 0.75, 8.0, 15.99, 2.0 ** -48, 2.0 ** 48 * 0.99):
        assert split.block_exponent(v) == 0
    # outside: floor(log2 max), clamped to [-126, 126]
    assert split.block_exponent(2.0 ** 48) == 48
    assert split.block_exponent(2.0 ** -49) == -49
    assert split.block_exponent(3.0 * 2.0 ** 60) == 61
    assert split.block_exponent(0.7 * 2.0 ** -100) == -101
    assert split.block_exponent(2.0 ** -130) == -126
    assert split.block_exponent(2.0 ** -126) == -126
    assert split.block_exponent(3.0e38) == 126
    assert split.block_exponent(0.0) == 0
    assert split.block_exponent(np.inf) == 0
    assert split.block_exponent(np.nan) == 0


@pytest.mark.parametrize("prec,bits", [("bf16", 8), ("tf32", 11)])
def test_split_reconstructs_within_bound(prec, bits):
    X = W.uniform(300, 77, 9)
    hi, lo, exps = split.split_rows(X, 300, 77, prec)
    assert exps.shape == (3,)
    assert (exps == 0).all()
    x = X.astype(np.float64)
    s = np.repeat(np.ldexp(1.0, -exps.astype(np.int64)), 128)[:300, None]
    xs = x * s
    # hi, lo representable in the target format
    mask = 0xFFFF if prec == "bf16" else 0x1FFF
    assert not (hi.view(np.uint32) & mask).any()
    assert not (lo.view(np.uint32) & mask).any()
    # |lo| <= half an ulp of hi; x' - hi - lo below 2^-(2*bits) relative
    err = np.abs(xs - hi.astype(np.float64) - lo.astype(np.float64))
    assert (err <= np.abs(xs) * 2.0 ** (-2 * bits) + 1e-45).all()
    nz = hi != 0
    ulp_hi = np.ldexp(1.0, np.frexp(hi[nz].astype(np.float64))[1] - bits)
    assert (np.abs(lo[nz]) <= ulp_hi / 2).all()


def test_split_of_integers_has_zero_low_part():
    X = W.integers(256, 40, 4)
    for prec in ("bf16", "tf32"):
        hi, lo, exps = split.split_rows(X, 256, 40, prec)
        assert (lo == 0).all()
        assert np.array_equal(hi, X)          # max |x| = 8 is in the safe range: e = 0
        assert (exps == 0).all()


def test_split_scaling_changes_nothing_in_the_safe_range():
    # a block near 2^60 (outside the safe range) is scaled by its exponent
    # 2^-59 and splits into exactly the planes of the unscaled block times 2
    X = W.uniform(128, 64, 10)
    hi0, lo0, e0 = split.split_rows(X, 128, 64, "bf16")
    big = W.scaled(X, 60)
    hi1, lo1, e1 = split.split_rows(big, 128, 64, "bf16")
    assert e0[0] == 0 and e1[0] == 59
    assert np.array_equal(hi1, hi0 * np.float32(2.0)) and np.array_equal(lo1, lo0 * np.float32(2.0))


def test_split_scaling_prevents_underflow_of_low_part():
    # entries near 2^-120: without scaling lo would be far below the fp32 normal range
    X = W.scaled(W.uniform(128, 64, 8), -120)
    hi, lo, exps = split.split_rows(X, 128, 64, "bf16")
    assert exps[0] == -121
    assert (np.abs(lo) > 0).mean() > 0.9
    rec = (hi.astype(np.float64) + lo) * 2.0 ** -121
    assert np.max(np.abs(rec - X) / np.abs(X)) < 2.0 ** -15


def test_split_non_finite():
    X = np.array([[1.0, np.inf, -2.0]], np.float32)
    hi, lo, exps = split.split_rows(X, 1, 3, "bf16")
    assert exps[0] == 0
    assert hi[0, 1] == np.inf and lo[0, 1] == 0.0
    assert hi[0, 0] == 1.0 and lo[0, 0] == 0.0


# ----------------------------------------------------------------- MLP oracle

def _rand_theta(F, H, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(mlp.param_count(F, H)) * 0.4


def test_mlp_tiny_closed_form():
    # F = 1, H = 1: y = w3*relu(W2*relu(W1*x + b1) + b2) + b3
    theta = mlp.pack([[2.0]], [-1.0], [[3.0]], [0.5], [-2.0], 0.25)
    X = np.array([[1.5], [0.2]])
    y, _ = mlp.forward(theta, X, H=1)
    # x=1.5: relu(2) = 2 -> relu(6.5) = 6.5 -> -13 + .25 ; x=0.2: relu(-0.6)=0 -> relu(.5) -> -1+.25
    assert np.array_equal(y, [-12.75, -0.75])
    t = np.array([-12.0, -1.0])
    loss, g = mlp.backward(theta, X, t, H=1)
    assert loss == ((-0.75) ** 2 + 0.25 ** 2) / 2
    # dy = (y - t) = [-0.75, 0.25]; gb3 = sum dy; gw3 = sum dy*h2
    W1, b1, W2, b2, w3, b3 = mlp.unpack(g, 1, 1)
    assert b3 == -0.5
    assert w3[0] == -0.75 * 6.5 + 0.25 * 0.5
    # dz2 = dy*w3 (both z2 > 0) = [1.5, -0.5]; gW2 = sum dz2*h1 = 1.5*2
    assert W2[0, 0] == 3.0 and b2[0] == 1.0
    # dz1 = dz2*W2 for the first sample only (z1 < 0 for the second): 4.5
    assert W1[0, 0] == 4.5 * 1.5 and b1[0] == 4.5


def test_mlp_backward_matches_finite_differences():
    F, H = 14, 64
    rng = np.random.default_rng(1)
    X = rng.standard_normal((40, F))
    t = rng.standard_normal(40)
    theta = _rand_theta(F, H, 2)
    loss, g = mlp.backward(theta, X, t, H)
    idx = list(rng.choice(theta.size, 300, replace=False)) + [theta.size - 1]
    # h = 1e-6: with h = 1e-3 some pre-activations lie within h of the ReLU kink
    # (|z| ~ 4e-4 here), where a central difference straddles the kink
    num = mlp.numeric_grad(theta, X, t, h=1e-6, H=H, idx=idx)
    for i in idx:
        assert abs(num[i] - g[i]) <= 1e-5 * max(abs(g[i]), 1e-2), (i, num[i], g[i])


def test_mlp_linear_regime_gradient_closed_form():
    # all weights/inputs positive -> every ReLU passes -> y is affine in x
    F, H = 3, 4
    rng = np.random.default_rng(3)
    W1 = rng.uniform(0.1, 1, (H, F)); b1 = rng.uniform(0.1, 1, H)
    W2 = rng.uniform(0.1, 1, (H, H)); b2 = rng.uniform(0.1, 1, H)
    w3 = rng.uniform(0.1, 1, H); b3 = 0.3
    theta = mlp.pack(W1, b1, W2, b2, w3, b3)
    X = rng.uniform(0.1, 1, (10, F))
    t = rng.uniform(0, 1, 10)
    y, _ = mlp.forward(theta, X, H)
    Weff = w3 @ W2 @ W1
    beff = w3 @ (W2 @ b1 + b2) + b3
    assert np.allclose(y, X @ Weff + beff, rtol=1e-13)
    _, g = mlp.backward(theta, X, t, H)
    gW1 = mlp.unpack(g, F, H)[0]
    dy = 2 * (y - t) / len(t)
    # dL/dW1[h][f] = sum_n dy_n * (w3 @ W2)[h] * X[n][f]
    expect = np.outer(w3 @ W2, X.T @ dy)
    assert np.allclose(gW1, expect, rtol=1e-12)


def test_adam_first_step_closed_form():
    theta = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.3, -4.0, 1e-3, 0.0])
    th1, m, v = mlp.adam_step(theta, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    # m_hat = g, v_hat = g^2  ->  step = lr * g / (|g| + eps)
    assert np.allclose(th1, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # second step with the same gradient: m_hat = g, v_hat = g^2 again
    th2, _, _ = mlp.adam_step(th1, g, m, v, 2, lr=0.01)
    assert np.allclose(th2, th1 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)


def test_split3_is_exact_and_extends_the_two_way_split():
    """BF16x6 split: three bf16 parts summing exactly to x' (normal values),
    each part at most half an ulp of the part before, and the first two
    parts are the two-way split."""
    from oracle import split
    import workloads as W
    x = np.concatenate([W.uniform(64, 64, 11).ravel(), W.wide_range(64, 64, 12, lo=-60, hi=60).ravel(),
                        np.array([1.0, -1.0, 3.0, 1.0 + 2 ** -23, 65504.0, 2 ** -100], np.float32)])
    hi, mid, lo = split.split3_values(x)
    for part in (hi, mid, lo):
        assert not (part.view(np.uint32) & 0xFFFF).any()          # representable in bf16
    assert np.array_equal(hi.astype(np.float64) + mid.astype(np.float64) + lo.astype(np.float64),
                          x.astype(np.float64))
    def ulp_bf16(v):
        e = np.floor(np.log2(np.abs(v.astype(np.float64)), where=v != 0, out=np.zeros(v.shape)))
        return np.where(v != 0, np.ldexp(1.0, (e - 7).astype(int)), 0.0)
    assert (np.abs(mid) <= ulp_bf16(hi) / 2).all()
    assert (np.abs(lo) <= ulp_bf16(mid) / 2 + (mid == 0)).all()
    h2, l2 = split.split_values(x, split.round_bf16)
    assert np.array_equal(h2, hi) and np.array_equal(l2, mid)
    # non-finite: hi carries it, the rest is zero
    h, m, l = split.split3_values(np.array([np.inf, -np.inf, np.nan], np.float32))
    assert np.isinf(h[:2]).all() and np.isnan(h[2]) and not m.any() and not l.any()
