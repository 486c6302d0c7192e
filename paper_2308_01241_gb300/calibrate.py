"""Finds the excitatory gain that sets a network's mean firing rate.

The paper sets its 7 / 15 / 30 Hz operating points by scaling the AMPA and
NMDA conductances (section VII.A); here one global factor multiplies g_AMPA and
g_NMDA of every voxel and is bisected on the GPU: reset, run a transient,
measure the mean rate over a window, repeat.  The result is written into the
config's "gain" table, keyed by the target rate.

    python -m paper_2308_01241_gb300.calibrate c3_large_20m --rates 7 15 30 --write
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import netgen


def measure_rate(net, tb, gain: float, transient: int, window: int) -> float:
    g = tb.vparams(gain)[:, 6:10]
    net.set_hyperparams(g)
    net.reset()
    net.step(transient)
    _, sp0, _ = net.counters()
    net.step(window)
    _, sp1, _ = net.counters()
    dt_s = float(tb.cfg["dt"]) * 1e-3
    return (sp1 - sp0) / (tb.n * window * dt_s)


def calibrate(name: str, rates, transient=1500, window=2000, lo=0.9, hi=1.8, iters=14, device="cuda:0",
              log=print) -> dict:
    from . import dtb

    cfg = netgen.load_config(name)
    tb = netgen.make_tables(cfg)
    csr = netgen.device_csr(tb, cfg["wfmt"], device=device)
    net = dtb.from_tables(tb, csr, device=device, bold_every=0, log_capacity=1 << 20)
    out = {}
    for r in rates:
        a, b = lo, hi
        ra = measure_rate(net, tb, a, transient, window)
        rb = measure_rate(net, tb, b, transient, window)
        log(f"{name} target {r} Hz: gain {a} -> {ra:.2f} Hz, gain {b} -> {rb:.2f} Hz")
        if not (ra <= r <= rb):
            raise RuntimeError(f"target {r} Hz outside [{ra:.2f}, {rb:.2f}] Hz")
        g = None
        for _ in range(iters):
            m = 0.5 * (a + b)
            rm = measure_rate(net, tb, m, transient, window)
            log(f"  gain {m:.5f} -> {rm:.3f} Hz")
            if abs(rm - r) < 0.01 * r:
                g = round(m, 5)
                break
            if rm < r:
                a = m
            else:
                b = m
        if g is None:
            g = round(0.5 * (a + b), 5)
        out[str(r)] = g
        log(f"  {name} {r} Hz -> gain {g} (measured {measure_rate(net, tb, g, transient, window):.3f} Hz)")
    net.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("config")
    ap.add_argument("--rates", type=float, nargs="+", default=[7, 15, 30])
    ap.add_argument("--write", action="store_true")
    ap.add_argument("--transient", type=int, default=1500)
    ap.add_argument("--window", type=int, default=2000)
    a = ap.parse_args()
    t0 = time.time()
    rates = [int(r) if float(r).is_integer() else r for r in a.rates]
    gains = calibrate(a.config, rates, transient=a.transient, window=a.window)
    print(json.dumps({"config": a.config, "gain": gains, "seconds": round(time.time() - t0, 1)}))
    if a.write:
        path = os.path.join(netgen.CONFIG_DIR, a.config + ".json")
        cfg = json.load(open(path))
        cfg.setdefault("gain", {}).update(gains)
        with open(path, "w") as f:
            json.dump(cfg, f, indent=2)
            f.write("\n")


if __name__ == "__main__":
    main()
