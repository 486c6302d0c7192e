"""The surrogate MLP's GPU kernels against the FP64 oracle (oracle/mlp.py).

The oracle runs on the same bfloat16-rounded weights and inputs and rounds
stored activations and gradients at the same points as the GPU, so the GPU
differs only by FP32 accumulation order and by bf16 ties that FP32 vs FP64
pre-rounding values can flip (one bf16 ulp = 2^-8 relative).  Asserted on
relative Frobenius norms: 1e-2 for outputs and gradients.  Adam: FP32 vs
FP64 arithmetic on identical gradients, 1e-5 relative.
"""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


def _setup(B=600, n_in=12, width=256, depth=3, n_out=2, seed=0):
    rng = np.random.default_rng(seed)
    params = ref.init_params(n_in, width, depth, n_out, seed=seed)
    for W, b in params:
        b += 0.05 * rng.standard_normal(b.shape)
    x = rng.standard_normal((B, n_in)).astype(np.float32)
    t = rng.standard_normal((B, n_out)).astype(np.float32)
    return params, x, t


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_forward_and_gradients_match_oracle():
    import torch

    from paper_2308_01241_gb300.surrogate_mlp import MLP

    params, x, t = _setup()
    net = MLP(params, 12, 256, 3, 2, max_batch=1024)
    dx, dt_ = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = torch.zeros((x.shape[0], 2), dtype=torch.float32, device="cuda")
    net.forward(dx, y)
    p16 = [(ref.bf16(W), np.float32(b).astype(np.float64)) for W, b in params]
    yr, cache = ref.forward(p16, ref.bf16(x), bf16_acts=True)
    assert _rel(y.cpu().numpy(), yr) < 1e-2
    grads, loss = net.gradients(dx, dt_)
    lr_, dy = ref.loss_and_grad_out(yr, t)
    gr = ref.backward(p16, cache, dy, bf16_acts=True)
    assert abs(loss - lr_) < 1e-2 * lr_
    for (gw, gb), (rw, rb) in zip(grads, gr):
        assert _rel(gw, rw) < 1e-2
        assert _rel(gb, rb) < 1e-2
    net.close()


def test_training_reduces_loss_on_a_smooth_target():
    import torch

    from paper_2308_01241_gb300.surrogate_mlp import MLP

    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, (8192, 12)).astype(np.float32)
    t = np.stack([np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2], np.tanh(x[:, 3] - x[:, 4])], 1).astype(np.float32)
    net = MLP(ref.init_params(12, 256, 3, 2, seed=2), 12, 256, 3, 2, max_batch=1024)
    dx, dt_ = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    losses = []
    for ep in range(30):
        for k in range(0, 8192, 1024):
            losses.append(net.train_step(dx[k:k + 1024], dt_[k:k + 1024], lr=2e-3))
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])
    net.close()


def test_adam_step_matches_oracle():
    import torch

    from paper_2308_01241_gb300.surrogate_mlp import MLP

    params, x, t = _setup(B=256, seed=3)
    net = MLP(params, 12, 256, 3, 2, max_batch=256)
    dx, dt_ = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    grads, _ = net.gradients(dx, dt_)
    net.train_step(dx, dt_, lr=1e-3)
    got = net.params()
    p = [(np.float32(W).astype(np.float64), np.float32(b).astype(np.float64)) for W, b in params]
    g64 = [(gw.astype(np.float64), gb.astype(np.float64)) for gw, gb in grads]
    st = ref.adam_state(p)
    ref.adam(p, g64, st, lr=1e-3)
    for (gw, gb), (rw, rb) in zip(got, p):
        np.testing.assert_allclose(gw, rw, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(gb, rb, rtol=1e-5, atol=1e-6)
    net.close()
