"""GPU edge cases through the C ABI, each against the C oracle or an exact
count: a network without synapses, a one-neuron network, compaction of an
all-zero bit set, a spike log too small for the call, and the two other step
entry points (dtb_step_timed, dtb_profile_steps) on the same steps as the
oracle."""
import ctypes

import numpy as np
import pytest

import oracle
from helpers import custom_net, params_row
from paper_2308_01241_gb300 import netgen as ng

pytestmark = pytest.mark.gpu

MODES = ["ring", "queue", "bins"]


@pytest.fixture(scope="module")
def dtb():
    from paper_2308_01241_gb300 import dtb as m

    return m


def _net_from_dict(dtb, d, delivery, **kw):
    """dtb.Network of an oracle input dict (pull form -> outgoing CSR)."""
    n, K = d["n"], d["K"]
    pre = np.asarray(d["pre"], np.int64).reshape(n, K)
    cls = np.asarray(d["cls"], np.uint32).reshape(n, K)
    w = np.asarray(d["w"]).reshape(n, K)
    tgt = np.repeat(np.arange(n, dtype=np.int64), K)
    src = pre.ravel()
    order = np.argsort(src, kind="stable")
    row_ptr = np.zeros(n + 1, np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(src, minlength=n))
    word = (tgt[order] | (cls.ravel()[order].astype(np.int64) << 30)).astype(np.uint32)
    csr = (row_ptr, word, np.ascontiguousarray(w.ravel()[order]))
    wfmt = {oracle.W_INT16: "int16", oracle.W_INT32: "int32"}[d["wfmt"]]
    return dtb.Network(n=n, voxel_start=d["voxel_start"], vparams=d["vparams"], delay_vv=d["delay_vv"],
                       d_max=d["d_max"], csr=csr, wfmt=wfmt, wshift=d["wshift"], n_ch=d["n_ch"], dt=d["dt"],
                       nu_ext=d["nu_ext"], w_ext=d["w_ext"], seed=d["seed"], init_seed=d["init_seed"],
                       bold=d["bold"], delivery=delivery, **kw)


def _same_run(net, ref, chunks):
    spikes = 0
    for c in chunks:
        net.step(c)
        ids, off = net.get_spikes()
        rids, roff = ref.run(c)
        np.testing.assert_array_equal(off, roff)
        np.testing.assert_array_equal(ids, rids)
        spikes += len(ids)
    V, j, r, ring, t = net.get_state()
    RV, Rj, Rr, Rring, Rt = ref.get_state()
    assert t == Rt
    np.testing.assert_array_equal(V, RV)
    np.testing.assert_array_equal(j, Rj)
    np.testing.assert_array_equal(r, Rr)
    np.testing.assert_array_equal(ring, Rring)
    return spikes


@pytest.mark.parametrize("delivery", MODES)
def test_network_without_synapses(dtb, delivery):
    """nnz = 0: 3,001 neurons in three voxels, driven only by the Poisson input;
    no delivery work exists, every counter of events stays 0."""
    cfg = ng.load_config("c2_multi_voxel_1m")
    cfg["gain"] = {"default": 1.3}
    tb = ng.make_tables(cfg, n_neurons=3001, n_vox=3, K=0)
    pull = ng.host_pull(tb)
    d = ng.oracle_inputs(tb, pull)
    assert d["pre"].size == 0
    d["w_ext"] = 8 * 65536  # enough drive that neurons fire without recurrent input
    net = _net_from_dict(dtb, d, delivery)
    ref = oracle.OracleNet(d, "f32")
    spikes = _same_run(net, ref, [1, 40, 300])
    assert spikes > 0
    ev, sp, st = net.counters()
    assert ev == 0 == ref.events() and sp == spikes and st == 341


@pytest.mark.parametrize("delivery", MODES)
def test_one_neuron_network(dtb, delivery):
    """n = 1 with one self-synapse (E class, delay 1): a single neuron in a
    single voxel, one update tile of 1,024 with 1,023 padding neurons."""
    d = custom_net(1, [[0]], [[0]], np.array([[40000]], np.int32),
                   params_row(g=(0.002, 0.00002, 0.01, 0.0005)), nu_ext=2000.0, w_ext=6 * 65536)
    net = _net_from_dict(dtb, d, delivery)
    ref = oracle.OracleNet(d, "f32")
    spikes = _same_run(net, ref, [1, 2, 64, 433])
    assert spikes > 3
    assert net.counters()[0] == ref.events() == spikes  # one synapse per spike


@pytest.mark.parametrize("n", [1, 1023, 1024, 65537, 3_000_001])
def test_compaction_of_an_all_zero_bit_set(dtb, n):
    """No bit set: count 0 and the id buffer untouched, through both
    compaction entry points."""
    import torch

    words = -(-n // 1024) * 32
    bits = torch.zeros(words, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for fn in (dtb.dtb_spike_compact, dtb.dtb_spike_compact_noalloc):
        ids = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        fn(bits, n, ids, cnt, stream)
        torch.cuda.synchronize()
        assert int(cnt.item()) == 0
        assert bool((ids == -7).all().item())


@pytest.mark.parametrize("delivery", ["bins", "ring"])
def test_spike_log_too_small(dtb, delivery):
    """A spike log of 500 ids over a call that fires more: dtb_get_spikes
    reports DTB_ETRUNC, *n_out is the log's capacity, the ids kept are the
    oracle's first 500 in step order, and the step offsets stop at 500.  A
    host buffer smaller than *n_out gives DTB_ETRUNC with nothing copied."""
    cfg = ng.load_config("c1_single_voxel_1k")
    tb = ng.make_tables(cfg)
    pull = ng.host_pull(tb)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull), delivery=delivery, log_capacity=500)
    ref = oracle.OracleNet(ng.oracle_inputs(tb, pull), "f32")
    steps = 400
    net.step(steps)
    rids, roff = ref.run(steps)
    assert len(rids) > 500
    lib = dtb._lib
    n_out = ctypes.c_int64(-1)
    off = np.full(steps + 1, -1, np.int64)
    ids = np.full(1000, -1, np.int32)
    r = lib.dtb_get_spikes(net.h, off.ctypes.data, ids.ctypes.data, ids.size, ctypes.byref(n_out))
    assert r == dtb.DTB_ETRUNC
    assert "overflowed" in dtb.dtb_last_error()
    assert n_out.value == 500
    np.testing.assert_array_equal(ids[:500], rids[:500])
    assert (ids[500:] == -1).all()
    np.testing.assert_array_equal(off, np.minimum(roff, 500))
    small = np.full(10, -1, np.int32)
    r = lib.dtb_get_spikes(net.h, None, small.ctypes.data, small.size, ctypes.byref(n_out))
    assert r == dtb.DTB_ETRUNC and n_out.value == 500
    assert (small == -1).all()
    # the state itself is unaffected by the log's size
    V, j, ref_, ring, t = net.get_state()
    RV, Rj, Rr, Rring, Rt = ref.get_state()
    np.testing.assert_array_equal(V, RV)
    np.testing.assert_array_equal(ring, Rring)


@pytest.mark.parametrize("delivery", MODES)
def test_timed_and_profiled_steps_match_the_oracle(dtb, delivery):
    """dtb_step_timed (the pipelined schedule without graphs, events around
    every kernel) and dtb_profile_steps (kernels one after the other) compute
    the same steps as dtb_step: rasters and state against the oracle."""
    tb = ng.make_tables(dict(ng.load_config("c2_multi_voxel_1m"), gain={"default": 1.35}), n_neurons=60013,
                        n_vox=8, K=80)
    pull = ng.host_pull(tb)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull), delivery=delivery)
    ref = oracle.OracleNet(ng.oracle_inputs(tb, pull), "f32")
    spikes = 0
    for k, how in [(70, "timed"), (33, "step"), (1, "timed"), (40, "profile"), (65, "timed")]:
        if how == "timed":
            ms, cnt = net.step_timed(k)
            assert cnt[0] == cnt[1] == cnt[2] == cnt[4] == k - 1
            assert cnt[3] == (0 if delivery == "ring" else k - 1)
            assert (ms[cnt > 0] > 0).all()
        elif how == "profile":
            ms = net.profile_steps(k)
            assert ms[0] > 0
        else:
            net.step(k)
        ids, off = net.get_spikes()
        rids, roff = ref.run(k)
        np.testing.assert_array_equal(off, roff)
        np.testing.assert_array_equal(ids, rids)
        spikes += len(ids)
    assert spikes > 1000
    V, j, r, ring, t = net.get_state()
    RV, Rj, Rr, Rring, Rt = ref.get_state()
    assert t == Rt == 209
    np.testing.assert_array_equal(V, RV)
    np.testing.assert_array_equal(j, Rj)
    np.testing.assert_array_equal(r, Rr)
    np.testing.assert_array_equal(ring, Rring)


@pytest.mark.parametrize("delivery", MODES)
@pytest.mark.parametrize("mode", [0, 1])
def test_both_schedules_match_the_oracle(dtb, delivery, mode):
    """The compaction after the update (0) and beside the next step's update
    (1, alternate copies of the spike bits and block counts): rasters and
    state against the oracle over calls of 1, 2, 33 (a graph chunk and a
    remainder), 70 and 5 steps, with the schedule switched after the 70."""
    tb = ng.make_tables(dict(ng.load_config("c2_multi_voxel_1m"), gain={"default": 1.35}), n_neurons=60013,
                        n_vox=8, K=80)
    pull = ng.host_pull(tb)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull), delivery=delivery)
    assert net.schedule_beside()  # 59 blocks: beside by size
    net.set_schedule(mode)
    assert net.schedule_beside() == (mode == 1)
    ref = oracle.OracleNet(ng.oracle_inputs(tb, pull), "f32")
    spikes = 0
    for k in [1, 2, 33, 70, 5]:
        net.step(k)
        ids, off = net.get_spikes()
        rids, roff = ref.run(k)
        np.testing.assert_array_equal(off, roff)
        np.testing.assert_array_equal(ids, rids)
        spikes += len(ids)
        if k == 70:
            net.set_schedule(1 - mode)
            assert net.schedule_beside() == (mode == 0)
    assert spikes > 1000
    V, j, r, ring, t = net.get_state()
    RV, Rj, Rr, Rring, Rt = ref.get_state()
    assert t == Rt == 111
    np.testing.assert_array_equal(V, RV)
    np.testing.assert_array_equal(j, Rj)
    np.testing.assert_array_equal(r, Rr)
    np.testing.assert_array_equal(ring, Rring)
    with pytest.raises(dtb.DtbError):
        net.set_schedule(2)
    net.set_schedule(-1)
    assert net.schedule_beside()


@pytest.mark.parametrize("delivery", MODES)
def test_voxel_wider_than_the_delivery_window(dtb, delivery):
    """One voxel of 300,000 neurons (74 regions of 4,096), in-degree 100, delay
    1: a source's targets lie up to 73 regions away, so about a fifth of the
    synapses fall outside the 64-region window of their delivery warp and, in
    bins mode, their runs reserve their own bin ranges.  Rasters and state
    against the oracle in every mode."""
    tb = ng.make_tables(ng.load_config("c1_single_voxel_1k"), n_neurons=300_000)
    pull = ng.host_pull(tb)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull), delivery=delivery)
    ref = oracle.OracleNet(ng.oracle_inputs(tb, pull), "f32")
    spikes = _same_run(net, ref, [1, 40, 60])
    assert spikes > 10_000
    assert net.counters()[0] == ref.events()


@pytest.mark.parametrize("delivery", MODES)
@pytest.mark.parametrize("wfmt", ["int16", "int32"])
def test_row_longer_than_255_work_items(dtb, delivery, wfmt):
    """A hub that every one of 140,000 neurons lists as an input: its row has
    140,000 synapses, 274 work items of 512, more than the per-neuron item
    byte holds, so the neuron update and the compaction count work items from
    the row bounds instead.  Rasters and state against the oracle."""
    n = 140_000
    rng = np.random.default_rng(11)
    pre = np.stack([np.zeros(n, np.int32), rng.integers(0, n, n, dtype=np.int32)], 1)
    cls = np.stack([np.zeros(n, np.uint8), rng.integers(0, 2, n, dtype=np.uint8)], 1)
    if wfmt == "int16":
        w = rng.integers(200, 2000, (n, 2)).astype(np.int16)
        d = custom_net(n, pre, cls, w, params_row(), nu_ext=2000.0, w_ext=6 * 65536, wfmt=oracle.W_INT16, wshift=4)
    else:
        w = rng.integers(3000, 30000, (n, 2)).astype(np.int32)
        d = custom_net(n, pre, cls, w, params_row(), nu_ext=2000.0, w_ext=6 * 65536, wfmt=oracle.W_INT32)
    net = _net_from_dict(dtb, d, delivery)
    ref = oracle.OracleNet(d, "f32")
    spikes = _same_run(net, ref, [1, 30, 50])
    assert spikes > 1000
    assert net.counters()[0] == ref.events()
