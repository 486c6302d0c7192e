"""Bit-exact parity over one second of biological time on the heterogeneous
1M-neuron network: 64 voxels of log-normal size, in-degree 500 (half inside
the voxel, half from other voxels by the DTI-like matrix), int32 weights at
2^-16, delays 1-40 steps, at its 15 Hz operating point, 10,000 steps (the
CPU-vs-GPU comparison of section VII.B also runs 1 s).

The FP32 oracle takes minutes for this run, so its results are stored as
digests in tests/golden/c2_1m_15hz_10k.txt, written by
tests/golden/make_c2_golden.py, which calls only the oracle: per chunk of
100 steps the spike count and a sha256 of the raster (per-step counts, then
ascending ids), and after the last step sha256 digests of V, j, ref and the
dense delay ring and the ring's per-slot sums.  The GPU run is hashed the same
way (tests/helpers.py) and must match every line.  The inputs are checked
first: the generator's voxel-level tables must hash to the oracle run's.
"""
import numpy as np
import pytest

from helpers import array_digest, raster_digest, read_golden, table_digest
from paper_2308_01241_gb300 import netgen as ng

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = "c2_1m_15hz_10k.txt"


@pytest.mark.parametrize("delivery", ["bins", "queue", "ring"])
def test_c2_one_second_bit_exact(delivery):
    import torch

    from paper_2308_01241_gb300 import dtb

    gold = read_golden(GOLDEN)
    name, rate, steps, chunk = gold["config"][0], int(gold["config"][1]), int(gold["config"][2]), int(gold["config"][3])
    cfg = ng.load_config(name)
    tb = ng.make_tables(cfg)
    assert table_digest(tb, ng.gain_for(cfg, rate)) == gold["inputs"][0], "input tables differ from the oracle run's"
    csr = ng.device_csr(tb, cfg["wfmt"])
    net = dtb.from_tables(tb, csr, rate=rate, delivery=delivery, log_capacity=1 << 22)
    total = 0
    for c in range(steps // chunk):
        net.step(chunk)
        ids, off = net.get_spikes()
        want_n, want_h = gold[f"chunk{c:03d}"]
        assert (len(ids), raster_digest(ids, off)) == (int(want_n), want_h), \
            f"raster of steps {c * chunk}..{(c + 1) * chunk - 1} differs from the oracle's"
        total += len(ids)
    assert total == int(gold["spikes"][0])
    ev, sp, st = net.counters()
    assert (ev, sp, st) == (int(gold["events"][0]), total, steps)
    V, j, ref, ring, t = net.get_state()
    assert t == steps
    assert array_digest(V) == gold["V"][0]
    assert array_digest(j) == gold["j"][0]
    assert array_digest(ref) == gold["ref"][0]
    np.testing.assert_array_equal(ring.astype(np.int64).sum(axis=2).ravel(),
                                  np.array([int(x) for x in gold["ring_slot_sums"]], np.int64))
    assert array_digest(ring) == gold["ring"][0]
    net.close()
    del csr
    torch.cuda.empty_cache()
