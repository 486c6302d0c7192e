"""Parity at the benchmark's full size (20M neurons, 2,000 voxels, K = 500,
1e10 device-generated synapses), in the launch configuration bench.py times.

The oracle cannot run the whole network, so the checks are ones it computes
exactly from its own inputs:

* every step up to and including the first one with spikes, for all 20M
  neurons: the ring is empty until then, so V, j, ref and the spike sets
  depend only on the initial voltages and the drive, and a K = 0 oracle network
  with the same voxels computes them;
* the delivery of that first spiking step for 2,000 sampled targets: their
  pull rows (host generator) and the ORACLE's spikes give, through the
  oracle's pull-form delivery, every ring entry those targets then hold;
* over further steps, properties that hold at any size: the int64 sum that
  one step adds to the ring equals the summed outgoing weight of the step's
  spikes (from the device CSR), and each spiking neuron sits at V_reset with a
  full refractory count.
"""
import numpy as np
import pytest

import oracle
from paper_2308_01241_gb300 import netgen as ng

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", params=["bins", "queue", "ring"])
def big(request):
    import torch

    from paper_2308_01241_gb300 import dtb

    free, total = torch.cuda.mem_get_info()
    if free < 100e9:
        pytest.skip("needs ~90 GB of free device memory")
    cfg = ng.load_config("c3_large_20m")
    tb = ng.make_tables(cfg)
    csr = ng.device_csr(tb, "int16")
    net = dtb.from_tables(tb, csr, rate=15, log_capacity=1 << 25, delivery=request.param)
    yield cfg, tb, csr, net
    net.close()
    del csr
    torch.cuda.empty_cache()


def test_first_steps_all_neurons_and_sampled_delivery(big):
    cfg, tb, csr, net = big
    net.reset()
    # oracle: the same voxels and parameters, no synapses.  Until the first
    # spikes the ring is empty, so every neuron's trajectory depends only on its
    # initial voltage and its drive, and this K = 0 network is exact.
    d0 = ng.oracle_inputs(tb, (np.zeros((tb.n, 0), np.int32), np.zeros((tb.n, 0), np.uint8),
                                np.zeros((tb.n, 0), np.uint16)), rate=15)
    d0["K"], d0["d_max"] = 0, 1
    o = oracle.OracleNet(d0, "f32")
    t_f = None
    for t in range(200):
        net.step(1)
        ids, _ = net.get_spikes()
        rids, _ = o.run(1)
        np.testing.assert_array_equal(ids, rids)
        if len(rids):
            t_f = t
            break
    assert t_f is not None and len(rids) >= 1
    V, j, ref, _, _ = net.get_state(with_ring=False)
    RV, Rj, Rref = o.get_state()[:3]
    np.testing.assert_array_equal(V, RV)
    np.testing.assert_array_equal(j, Rj)
    np.testing.assert_array_equal(ref, Rref)
    del o
    # ring after step t_f for sampled targets, from the oracle's own spikes:
    # 1,000 random neurons plus up to 1,000 targets of those spikes (read from
    # the generator's CSR, an input), so that some sampled entries are nonzero
    rng = np.random.default_rng(7)
    row_ptr, word = csr[0].cpu(), csr[1]
    hit = []
    for s_ in rids[:16]:
        a, b = int(row_ptr[s_]), int(row_ptr[s_ + 1])
        hit.append((word[a:b].cpu().numpy().view(np.uint32) & 0x3FFFFFFF).astype(np.int64))
    hit = np.unique(np.concatenate(hit))[:1000]
    tgt = np.unique(np.concatenate([rng.choice(tb.n, size=1000, replace=False), hit]))
    rows = [ng.host_pull(tb, int(i), int(i) + 1) for i in tgt]
    pre = np.concatenate([r[0] for r in rows])
    cls = np.concatenate([r[1] for r in rows])
    wb = np.concatenate([r[2] for r in rows])
    fired = np.zeros(tb.n, np.uint8)
    fired[rids] = 1
    dd = ng.oracle_inputs(tb, (pre, cls, wb), rate=15)
    dd["K"] = tb.K
    acc = oracle.deliver_pull(dd, tgt, pre, cls, dd["w"], fired, t_f)  # [m][ch][D]
    got = net.get_ring_at(tgt).transpose(0, 2, 1).astype(np.int64)     # [m][D][ch] -> [m][ch][D]
    assert acc.sum() > 0
    np.testing.assert_array_equal(got, acc)


def test_ring_increment_conservation_over_steps(big):
    import torch

    cfg, tb, csr, net = big
    row_ptr, word, w = csr
    net.reset()
    net.step(300)
    vreset = np.float32(cfg["neuron"]["Vreset"])
    for _ in range(3):
        t = net.counters()[2]
        slot = t % net.D
        s0 = net.ring_slot_sums()
        net.step(1)
        ids, _ = net.get_spikes()
        s1 = net.ring_slot_sums()
        # slot t was consumed and cleared; every other slot only grew
        assert np.all(s1[slot] == 0)
        before = int(s0.sum()) - int(s0[slot].sum())
        added = int(s1.sum()) - before
        # summed outgoing weight (2^-16 units) of the neurons that fired
        sid = torch.from_numpy(ids.astype(np.int64)).to(w.device)
        lo, hi = row_ptr[sid], row_ptr[sid + 1]
        lens = hi - lo
        idx = torch.repeat_interleave(lo, lens) + (torch.arange(int(lens.sum().item()), device=w.device)
                                                   - torch.repeat_interleave(torch.cumsum(lens, 0) - lens, lens))
        expect = int((w[idx].to(torch.int64) * 16).sum().item())
        assert added == expect
        V1, _, ref1, _, _ = net.get_state(with_ring=False)
        assert np.all(V1[ids] == vreset)
        assert np.all(ref1[ids] == round(cfg["neuron"]["t_ref"] / cfg["dt"]))
        assert len(ids) > 100
