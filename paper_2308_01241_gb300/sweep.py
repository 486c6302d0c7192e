"""In-degree sweep on one GPU: cost of one biological second versus synapses per neuron.

Section VII.C varies the input synapses per neuron from 100 to 1000 at a fixed
neuron count and reports the time of one simulated second. This is the
one-GPU counterpart: a fixed N (10M by default, the 20M network's voxel
structure at half size) and K in 100..1000, so that N x K stays within the
20M x 500 synapses of the full-size network.

For a fair comparison the operating point is held at one firing rate:
- all four receptor conductances are first scaled by 500 / K (same mean
  recurrent input per neuron), and the external drive's weight by K / 500
  (it enters through g_AMPA, so its product with g_AMPA stays fixed);
- the AMPA / NMDA gain is then bisected on the GPU until the mean rate over
  2,000 steps is within 2 % of the target.

Each K reports:
- the measured rate and the wall time per step, with CUDA events on the
  network's stream;
- wall-s per bio-s, synaptic events/s, and the per-kernel split from
  dtb_profile_steps.

    python -m paper_2308_01241_gb300.sweep [--neurons 10000000] [--K 100 200 500 1000] [--rate 15]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import dtb, netgen

K_REF = 500


def _log(*m):
    print(*m, file=sys.stderr, flush=True)


def _rate(net, tb, g, transient, window):
    net.set_hyperparams(g)
    net.reset()
    net.step(transient)
    _, s0, _ = net.counters()
    net.step(window)
    _, s1, _ = net.counters()
    return (s1 - s0) / (tb.n * window * float(tb.cfg["dt"]) * 1e-3)


def calibrate_gain(net, tb, g0, target, transient=1000, window=2000, lo=0.1, hi=8.0, iters=18, log=_log):
    """Bisects the factor on g_AMPA and g_NMDA of g0 [nv][4] for the target rate (log scale)."""
    def g_of(x):
        g = g0.copy()
        g[:, :2] *= x
        return g

    for _ in range(iters):
        m = float(np.sqrt(lo * hi))
        r = _rate(net, tb, g_of(m), transient, window)
        log(f"  gain {m:.4f} -> {r:.3f} Hz")
        if abs(r - target) <= 0.02 * target:
            return m, r
        if r < target:
            lo = m
        else:
            hi = m
    raise RuntimeError(f"no gain in [{lo:.4f}, {hi:.4f}] reaches {target} Hz")


def run_k(cfg, n, nv, K, target, steps, warmup, delivery, device="cuda:0", log=_log):
    import torch

    t0 = time.time()
    cfg = dict(cfg)
    cfg["w_ext"] = int(round(int(cfg["w_ext"]) * K / K_REF))
    tb = netgen.make_tables(cfg, n_neurons=n, n_vox=nv, K=K)
    csr = netgen.device_csr(tb, cfg["wfmt"], device=device)
    net = dtb.from_tables(tb, csr, device=device, bold_every=0, log_capacity=1 << 20, delivery=delivery)
    setup_s = time.time() - t0
    g0 = tb.vparams(1.0)[:, 6:10] * (K_REF / K)
    gain, _ = calibrate_gain(net, tb, g0, target, log=log)
    g = g0.copy()
    g[:, :2] *= gain
    net.set_hyperparams(g)
    net.reset()
    net.step(warmup)
    ev0, sp0, _ = net.counters()
    torch.cuda.synchronize(device)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(net.stream)
    net.step(steps)
    b.record(net.stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    ev1, sp1, _ = net.counters()
    prof = net.profile_steps(200)
    dt_s = float(cfg["dt"]) * 1e-3
    res = {
        "K": K, "w_ext": int(cfg["w_ext"]), "neurons": tb.n, "voxels": tb.nv, "synapses": tb.n * K, "gain": round(gain, 5),
        "rate_hz": (sp1 - sp0) / (tb.n * steps * dt_s), "ms_per_step": ms / steps,
        "wall_s_per_bio_s": (ms * 1e-3) / (steps * dt_s), "synaptic_events_per_s": (ev1 - ev0) / (ms * 1e-3),
        "kernel_ms": {nm: prof[k] / 200 for k, nm in enumerate(dtb.KERNELS)}, "setup_s": setup_s,
    }
    net.close()
    del net, csr
    torch.cuda.empty_cache()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c3_large_20m")
    ap.add_argument("--neurons", type=int, default=10_000_000)
    ap.add_argument("--voxels", type=int, default=1000)
    ap.add_argument("--K", type=int, nargs="+", default=[100, 200, 300, 500, 700, 1000])
    ap.add_argument("--rate", type=float, default=15.0)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=1000)
    ap.add_argument("--delivery", default="bins", choices=["ring", "queue", "bins"])
    a = ap.parse_args()
    cfg = netgen.load_config(a.config)
    if max(a.K) * a.neurons > 10_000_000_000:
        raise SystemExit("N x K above 1e10 synapses: beyond the memory plan of one GPU")
    out = []
    for K in a.K:
        _log(f"K = {K}")
        r = run_k(cfg, a.neurons, a.voxels, K, a.rate, a.steps, a.warmup, a.delivery)
        _log(json.dumps(r))
        out.append(r)
    print(json.dumps({"sweep": "in-degree", "target_rate_hz": a.rate, "delivery": a.delivery, "points": out}))


if __name__ == "__main__":
    main()
