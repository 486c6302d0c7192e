"""Pins of the FP64 MLP oracle used to check the surrogate's GPU kernels.

* GELU: gelu(x) - gelu(-x) = x exactly (the odd part of x Phi(x)), gelu(0) = 0,
  gelu -> x for large x and -> 0 for very negative x; its derivative matches
  central differences;
* backward: every weight and bias gradient matches central finite
  differences of the loss (double precision, no rounding);
* Adam: the first step moves every parameter by lr * sign(gradient) (the
  bias-corrected moments are g and g^2);
* bf16 rounding: round-to-nearest-even on the float32 bits, checked on
  exactly representable and halfway values.
"""
import numpy as np

from oracle import mlp


def test_gelu_identities():
    x = np.linspace(-6, 6, 241)
    np.testing.assert_allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-14)
    assert mlp.gelu(0.0) == 0.0
    assert abs(mlp.gelu(10.0) - 10.0) < 1e-15 and abs(mlp.gelu(-10.0)) < 1e-20
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(x), fd, atol=1e-8)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    params = mlp.init_params(5, 7, 3, 2, seed=4)
    for W, b in params:
        b += 0.1 * rng.standard_normal(b.shape)
    x = rng.standard_normal((6, 5))
    t = rng.standard_normal((6, 2))
    y, cache = mlp.forward(params, x)
    loss, dy = mlp.loss_and_grad_out(y, t)
    grads = mlp.backward(params, cache, dy)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for p, g in ((W, grads[li][0]), (b, grads[li][1])):
            flat, gflat = p.reshape(-1), g.reshape(-1)
            for k in range(0, flat.size, max(1, flat.size // 9)):
                old = flat[k]
                flat[k] = old + h
                lp = mlp.loss_and_grad_out(mlp.forward(params, x)[0], t)[0]
                flat[k] = old - h
                lm = mlp.loss_and_grad_out(mlp.forward(params, x)[0], t)[0]
                flat[k] = old
                assert abs((lp - lm) / (2 * h) - gflat[k]) <= 1e-6 * (1 + abs(gflat[k]))


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(5)
    params = mlp.init_params(3, 4, 1, 2, seed=6)
    before = [(W.copy(), b.copy()) for W, b in params]
    grads = [(rng.standard_normal(W.shape), rng.standard_normal(b.shape)) for W, b in params]
    st = mlp.adam_state(params)
    mlp.adam(params, grads, st, lr=0.01, eps=0.0)
    for (W0, b0), (W, b), (gW, gb) in zip(before, params, grads):
        np.testing.assert_allclose(W - W0, -0.01 * np.sign(gW), atol=1e-15)
        np.testing.assert_allclose(b - b0, -0.01 * np.sign(gb), atol=1e-15)


def test_bf16_rounding():
    exact = np.array([1.0, -2.5, 0.15625, 2.0 ** 100], np.float64)  # representable in bfloat16
    np.testing.assert_array_equal(mlp.bf16(exact), np.float32(exact).astype(np.float64))
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: ties to even -> 1 + 2^-6
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert mlp.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7


def test_wrong_elements_fall_outside_the_gpu_tolerance():
    """The per-element tolerances of the GPU parity test (tests/mlp_bounds.py)
    are tight enough to see a mistake: the oracle's own forward with one
    weight of a hidden layer 0.5 off (weights average 0.07), with one 64 x 64
    tile of a hidden layer's weights 5 % off or zeroed (one GEMM tile done
    wrong), with one bias dropped, or with two neighbouring hidden units
    swapped, fails the check; the unchanged forward passes it."""
    from mlp_bounds import forward_sigma, outside, setup

    params, x, t = setup(B=200, seed=4)
    p16 = [(mlp.bf16(W), np.float32(b).astype(np.float64)) for W, b in params]
    xb = mlp.bf16(x)
    yr, cache = mlp.forward(p16, xb, bf16_acts=True)
    _, _, sy = forward_sigma(p16, cache, yr)
    assert not outside(yr, yr, sy).any()

    def run(change):
        bad = [(W.copy(), b.copy()) for W, b in p16]
        change(bad)
        return mlp.forward(bad, xb, bf16_acts=True)[0]

    def w(bad):
        bad[1][0][7, 3] += 0.5

    def tile(bad):
        bad[2][0][64:128, 0:64] *= 1.05

    def zero_tile(bad):
        bad[2][0][64:128, 0:64] = 0.0

    def b(bad):
        bad[3][1][1] = 0.0

    def swap(bad):
        bad[2][0][[10, 11]] = bad[2][0][[11, 10]]

    assert outside(run(w), yr, sy).any()
    assert outside(run(tile), yr, sy).any()
    assert outside(run(zero_tile), yr, sy).mean() > 0.5
    assert outside(run(b), yr, sy)[:, 1].mean() > 0.9
    assert outside(run(swap), yr, sy).any()
