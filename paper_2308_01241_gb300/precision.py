"""Reduced-precision synaptic weights on the 20M-neuron network.

The paper reports "mixed precision" (Performance Attributes table) without
detail.  Here the state stays FP32 and the sums stay exact int32; only the
stored weights shrink:
- int32 at 2^-16: the FP32-weight reference, 4 bytes per weight;
- BF16: 2 bytes;
- int8 with one power-of-two scale per row: 1 byte.

Each variant runs at the 7 / 15 / 30 Hz operating points for one
biological second. Against the reference it reports:
- the per-voxel firing-rate deviation (voxels at >= 1 Hz);
- the Pearson correlation of the BOLD signal (every voxel, sampled every
  10 ms);
- ms per step.

The network is chaotic, so the reference itself run with another drive seed
is reported too: deviations at that level are trajectory noise, not
precision loss.

    python -m paper_2308_01241_gb300.precision [--steps 10000] [--warmup 3000] [--delivery bins]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import dtb, netgen


def _run(tb, cfg, csr, wfmt, rates, warmup, steps, bold_every, seed=None, delivery="bins"):
    import torch

    kw = {}
    if seed is not None:
        kw["seed"] = seed
    wshift = 4 if wfmt == "int16" else 0
    net = dtb.Network(n=tb.n, voxel_start=tb.voxel_start, vparams=tb.vparams(1.0), delay_vv=tb.delay_vv,
                      d_max=tb.d_max, csr=csr, wfmt=wfmt, wshift=wshift, n_ch=int(cfg["n_ch"]), dt=float(cfg["dt"]),
                      nu_ext=float(cfg["nu_ext"]), w_ext=int(cfg["w_ext"]),
                      seed=kw.get("seed", int(cfg["seeds"]["drive"])), init_seed=int(cfg["seeds"]["init"]),
                      bold=cfg["bold"], bold_every=bold_every, log_capacity=1 << 16, delivery=delivery)
    out = {}
    dt_s = float(cfg["dt"]) * 1e-3
    sizes = np.diff(tb.voxel_start)
    for r in rates:
        net.set_hyperparams(tb.vparams(netgen.gain_for(cfg, r))[:, 6:10])
        net.reset()
        net.step(warmup)
        v0 = net.voxel_spikes()
        samples = []
        ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        done, ms = 0, 0.0
        chunk = 1000
        while done < steps:
            c = min(chunk, steps - done)
            ev[0].record(net.stream)
            try:
                net.step(c)
            except dtb.DtbError as e:
                if e.code != dtb.DTB_ETRUNC:
                    raise
            ev[1].record(net.stream)
            ev[1].synchronize()
            ms += ev[0].elapsed_time(ev[1])
            samples.append(net.get_bold_samples())
            done += c
        rate = (net.voxel_spikes() - v0) / (sizes * steps * dt_s)
        out[str(r)] = {"rate": rate, "bold": np.concatenate(samples), "ms_per_step": ms / steps}
    net.close()
    return out


def _compare(ref, var):
    res = {}
    for r, a in ref.items():
        b = var[r]
        act = a["rate"] >= 1.0
        dev = np.abs(b["rate"][act] - a["rate"][act]) / a["rate"][act]
        x, y = a["bold"].ravel(), b["bold"].ravel()
        pear = float(np.corrcoef(x, y)[0, 1])
        per_vox = [np.corrcoef(a["bold"][:, v], b["bold"][:, v])[0, 1] for v in range(a["bold"].shape[1])
                   if a["bold"][:, v].std() > 0 and b["bold"][:, v].std() > 0]
        res[r] = {"mean_rate_hz": float(a["rate"].mean()), "voxels_active": int(act.sum()),
                  "rate_dev_max": float(dev.max()), "rate_dev_p99": float(np.percentile(dev, 99)),
                  "rate_dev_mean": float(dev.mean()), "frac_voxels_within_2pct": float((dev <= 0.02).mean()),
                  "bold_pearson": pear, "bold_pearson_per_voxel_median": float(np.median(per_vox)),
                  "ms_per_step": b["ms_per_step"], "ref_ms_per_step": a["ms_per_step"]}
    return res


def main():
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c3_large_20m")
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=3000, help="steps before the measured second (the network settles in about 2,500)")
    ap.add_argument("--delivery", default="bins", choices=["ring", "queue", "bins"])
    ap.add_argument("--rates", type=int, nargs="+", default=[7, 15, 30])
    ap.add_argument("--bold-every", type=int, default=100)
    a = ap.parse_args()
    cfg = netgen.load_config(a.config)
    tb = netgen.make_tables(cfg)
    t0 = time.time()
    results = {}
    csr = netgen.device_csr(tb, "int32")
    ref = _run(tb, cfg, csr, "int32", a.rates, a.warmup, a.steps, a.bold_every, delivery=a.delivery)
    other_seed = _run(tb, cfg, csr, "int32", a.rates, a.warmup, a.steps, a.bold_every,
                      seed=int(cfg["seeds"]["drive"]) + 1000, delivery=a.delivery)
    results["int32, other drive seed (noise floor)"] = _compare(ref, other_seed)
    del csr
    torch.cuda.empty_cache()
    csr = netgen.device_csr(tb, "bf16")
    results["bf16"] = _compare(ref, _run(tb, cfg, csr, "bf16", a.rates, a.warmup, a.steps, a.bold_every, delivery=a.delivery))
    del csr
    torch.cuda.empty_cache()
    csr = netgen.device_csr_int8(tb)
    results["int8 + row scale"] = _compare(ref, _run(tb, cfg, csr, "int8", a.rates, a.warmup, a.steps, a.bold_every, delivery=a.delivery))
    del csr
    torch.cuda.empty_cache()
    print(json.dumps({"config": a.config, "steps": a.steps, "warmup": a.warmup, "delivery": a.delivery, "results": results,
                      "seconds": round(time.time() - t0, 1)}, indent=1))


if __name__ == "__main__":
    main()
