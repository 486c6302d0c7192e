"""Writes c2_1m_15hz_10k.txt: digests of the FP32 oracle's run of the
heterogeneous 1M-neuron network (64 voxels, in-degree 500, int32 weights at
2^-16, delays 1-40 steps) at its 15 Hz operating point, for 10,000 steps
(1 s of biological time; the CPU-vs-GPU check of section VII.B runs 1 s).

Calls only oracle/ (and the seeded input generator).  Run from the repository
root:  python tests/golden/make_c2_golden.py   (about ten minutes, ~12 GB RAM)
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from helpers import array_digest, raster_digest, table_digest  # noqa: E402
from paper_2308_01241_gb300 import netgen as ng  # noqa: E402

CONFIG, RATE, STEPS, CHUNK = "c2_multi_voxel_1m", 15, 10_000, 100
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_1m_15hz_10k.txt")


def main():
    cfg = ng.load_config(CONFIG)
    tb = ng.make_tables(cfg)
    gain = ng.gain_for(cfg, RATE)
    t0 = time.time()
    pull = ng.host_pull(tb)
    net = oracle.OracleNet(ng.oracle_inputs(tb, pull, rate=RATE), "f32")
    del pull
    lines = [f"# {CONFIG} at the {RATE} Hz gain ({gain}), {STEPS} steps of the FP32 oracle in chunks of {CHUNK}",
             "# written by tests/golden/make_c2_golden.py (oracle only)",
             f"config {CONFIG} {RATE} {STEPS} {CHUNK}",
             f"inputs {table_digest(tb, gain)}"]
    total = 0
    for c in range(STEPS // CHUNK):
        ids, off = net.run(CHUNK)
        total += len(ids)
        lines.append(f"chunk{c:03d} {len(ids)} {raster_digest(ids, off)}")
        if c % 10 == 9:
            print(f"{(c + 1) * CHUNK} steps, {total} spikes, {time.time() - t0:.0f} s", flush=True)
    V, j, ref, ring, t = net.get_state()
    assert t == STEPS
    lines += [f"spikes {total}", f"events {net.events()}",
              f"V {array_digest(V)}", f"j {array_digest(j)}", f"ref {array_digest(ref)}",
              f"ring {array_digest(ring)}", f"ring_slot_sums {' '.join(str(int(x)) for x in ring.astype(np.int64).sum(axis=2).ravel())}"]
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"wrote {OUT}: {total} spikes in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
