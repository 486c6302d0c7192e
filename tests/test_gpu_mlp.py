"""The surrogate MLP's GPU kernels against the FP64 oracle (oracle/mlp.py),
element by element.

The oracle runs on the same bfloat16-rounded weights and inputs and rounds
stored activations and gradients at the same points as the GPU, so the GPU
differs only by its FP32 arithmetic between those points.  Every output and
every weight and bias gradient element is checked against its own tolerance,
6 standard deviations of that FP32 arithmetic propagated through the network
(tests/mlp_bounds.py; its tightness is checked on the CPU in
test_oracle_mlp.py).  Adam: FP32 vs FP64 arithmetic on identical gradients,
1e-5 relative.
"""
import numpy as np
import pytest

from mlp_bounds import assert_within, backward_sigma, forward_sigma, output_grad_sigma, setup
from oracle import mlp as ref

pytestmark = pytest.mark.gpu


def test_forward_and_gradients_match_oracle():
    import torch

    from paper_2308_01241_gb300.surrogate_mlp import MLP

    params, x, t = setup()
    net = MLP(params, 12, 256, 3, 2, max_batch=1024)
    dx, dt_ = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = torch.zeros((x.shape[0], 2), dtype=torch.float32, device="cuda")
    net.forward(dx, y)
    p16 = [(ref.bf16(W), np.float32(b).astype(np.float64)) for W, b in params]
    yr, cache = ref.forward(p16, ref.bf16(x), bf16_acts=True)
    sa, sz, sy = forward_sigma(p16, cache, yr)
    assert_within(y.cpu().numpy(), yr, sy, "forward output")
    grads, loss = net.gradients(dx, dt_)
    lr_, dy = ref.loss_and_grad_out(yr, t)
    gr = ref.backward(p16, cache, dy, bf16_acts=True)
    assert abs(loss - lr_) < 1e-2 * lr_
    sig = backward_sigma(p16, cache, sa, sz, output_grad_sigma(sy, dy), ref.bf16(dy))
    for li, ((gw, gb), (rw, rb), (sw, sb)) in enumerate(zip(grads, gr, sig)):
        assert_within(gw, rw, sw, f"dW[{li}]")
        assert_within(gb, rb, sb, f"db[{li}]")
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

    params, x, t = setup(B=256, seed=3)
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
