"""GPU parity: the CUDA path through the C ABI against the C oracle.

Bit-exact (FP32 state, int32 accumulators, ascending rasters): spike rasters,
V, j, ref and the whole delay ring, on seeded synthetic networks that span
several compaction tiles and a ragged tail, for every weight format and both
channel modes, across CUDA-graph chunks and remainders, checkpoints and
hyper-parameter changes.  BOLD (FP32 with powf/expf on the GPU, FP64 in the
oracle) is compared within a tolerance derived in the test.
"""
import numpy as np
import pytest

import oracle
from paper_2308_01241_gb300 import netgen as ng

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dtb():
    from paper_2308_01241_gb300 import dtb as m

    return m


def _tables(name, n=None, nv=None, K=None, **over):
    cfg = ng.load_config(name)
    cfg.update(over)
    return ng.make_tables(cfg, n_neurons=n, n_vox=nv, K=K)


def _net_kw(d):
    """Drive, time step and seeds of an oracle input dict, for dtb.Network."""
    return dict(dt=d["dt"], nu_ext=d["nu_ext"], w_ext=d["w_ext"], seed=d["seed"], init_seed=d["init_seed"],
                bold=d["bold"])


def _assert_state_equal(net, ref):
    V, j, r, ring, t = net.get_state()
    RV, Rj, Rr, Rring, Rt = ref.get_state()
    assert t == Rt
    np.testing.assert_array_equal(V, RV)
    np.testing.assert_array_equal(j, Rj)
    np.testing.assert_array_equal(r, Rr)
    np.testing.assert_array_equal(ring, Rring)


def _run_both(net, ref, chunks):
    total = 0
    for c in chunks:
        net.step(c)
        ids, off = net.get_spikes()
        rids, roff = ref.run(c)
        np.testing.assert_array_equal(off, roff)
        np.testing.assert_array_equal(ids, rids)
        total += len(ids)
    return total


MODES = ["ring", "queue", "bins"]


@pytest.mark.parametrize("delivery", MODES)
def test_c1_single_voxel_bit_exact(dtb, delivery):
    tb = _tables("c1_single_voxel_1k")
    pull = ng.host_pull(tb)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull), delivery=delivery)
    ref = oracle.OracleNet(ng.oracle_inputs(tb, pull), "f32")
    spikes = _run_both(net, ref, [1, 31, 32, 100, 836])  # graph chunks of 32 and remainders
    assert spikes > 500
    _assert_state_equal(net, ref)
    assert net.voxel_spikes().tolist() == [spikes]
    ev, sp, st = net.counters()
    assert (ev, sp, st) == (ref.events(), spikes, 1000)


@pytest.mark.parametrize("delivery", MODES)
@pytest.mark.parametrize("wfmt", ["int32", "int16"])
def test_multivoxel_tiles_and_ragged_tail(dtb, wfmt, delivery):
    # 200,003 neurons: 196 neuron blocks, 4 compaction tiles, ragged last block
    tb = _tables("c2_multi_voxel_1m", n=200003, nv=24, K=100, wfmt=wfmt, gain={"default": 1.35})
    pull = ng.host_pull(tb)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull), delivery=delivery)
    ref = oracle.OracleNet(ng.oracle_inputs(tb, pull), "f32")
    spikes = _run_both(net, ref, [64, 200, 7, 129])
    assert spikes > 2000
    _assert_state_equal(net, ref)
    net.reset()
    net.step(400)
    ids, _ = net.get_spikes()
    vox = np.searchsorted(tb.voxel_start, ids, side="right") - 1
    np.testing.assert_array_equal(net.voxel_spikes(), np.bincount(vox, minlength=tb.nv))
    assert net.counters()[0] == ref.events()


def _int8_csr(tb, pull, rng):
    """int8 weights with a per-source power-of-two scale (w_acc = q << (8 + s_row))."""
    pre, cls, wbin = pull
    q = ((wbin.astype(np.int32) % 120) + 1).astype(np.int8)
    row_shift = rng.integers(0, 4, size=tb.n).astype(np.uint8)
    row_ptr, word, wb = ng.host_push(tb, (pre, cls, q.view(np.uint8).astype(np.uint16)))
    w_push = wb.astype(np.uint8).view(np.int8)
    return q, row_shift, (row_ptr, word, w_push, row_shift)


@pytest.mark.parametrize("delivery", MODES)
@pytest.mark.parametrize("wfmt", ["bf16", "int8"])
def test_weight_formats(dtb, wfmt, delivery):
    tb = _tables("c2_multi_voxel_1m", n=50021, nv=10, K=80, gain={"default": 1.3})
    pull = ng.host_pull(tb)
    d = ng.oracle_inputs(tb, pull, wfmt="int16")
    if wfmt == "bf16":
        w = tb.wtable("bf16")[pull[2]]
        d.update(wfmt=oracle.W_BF16, w=w, wshift=0)
        row_ptr, word, wb = ng.host_push(tb, pull)
        csr = (row_ptr, word, tb.wtable("bf16")[wb])
        kw = dict(wfmt="bf16", wshift=0)
    else:
        q, rs, csr = _int8_csr(tb, pull, np.random.default_rng(5))
        d.update(wfmt=oracle.W_INT8, w=q, wshift=8, pre_shift=rs)
        kw = dict(wfmt="int8", wshift=8)
    net = dtb.Network(n=tb.n, voxel_start=tb.voxel_start, vparams=d["vparams"], delay_vv=tb.delay_vv,
                      d_max=tb.d_max, csr=csr, n_ch=2, delivery=delivery, **_net_kw(d), **kw)
    ref = oracle.OracleNet(d, "f32")
    assert _run_both(net, ref, [300, 45]) > 500
    _assert_state_equal(net, ref)


@pytest.mark.parametrize("delivery", MODES)
def test_four_channel_mode(dtb, delivery):
    tb = _tables("c2_multi_voxel_1m", n=30011, nv=6, K=60, gain={"default": 1.3})
    pre, cls, wbin = ng.host_pull(tb)
    cls = np.random.default_rng(9).integers(0, 4, size=cls.shape).astype(np.uint8)
    pull = (pre, cls, wbin)
    d = ng.oracle_inputs(tb, pull)
    d["n_ch"] = 4
    row_ptr, word, wb = ng.host_push(tb, pull)
    net = dtb.Network(n=tb.n, voxel_start=tb.voxel_start, vparams=d["vparams"], delay_vv=tb.delay_vv,
                      d_max=tb.d_max, csr=(row_ptr, word, tb.wtable("int32")[wb]), wfmt="int32", wshift=0, n_ch=4,
                      delivery=delivery, **_net_kw(d))
    ref = oracle.OracleNet(d, "f32")
    assert _run_both(net, ref, [250]) > 100
    _assert_state_equal(net, ref)


def test_bold_within_tolerance(dtb):
    # The oracle integrates BOLD in double on the identical raster (its FP32
    # build reproduces the GPU's spikes bit for bit); the GPU integrates in
    # float with powf/expf.  Per step each state update rounds by at most
    # 2^-24 of an O(1) state (f, v, q ~ 1), i.e. ~6e-8; the slowest mode decays
    # with rate kappa/2 = 0.625/s, i.e. over ~16,000 steps, so a random walk of
    # roundings stays near 6e-8 * sqrt(16000) ~ 8e-6.  Asserted: 3e-5 on s, f,
    # v, q and 3e-5 * V0 * (k1 + k2 + |k3|) on y.
    tb = _tables("c2_multi_voxel_1m", n=40009, nv=8, K=60, gain={"default": 1.35})
    pull = ng.host_pull(tb)
    d = ng.oracle_inputs(tb, pull)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull), bold_every=5000)
    ref = oracle.OracleNet(d, "f32")
    net.step(20000)
    ref.run(20000)
    y, st = net.get_bold()
    ry, rst = ref.get_bold()
    dev = np.abs(rst - np.array([[0.0], [1.0], [1.0], [1.0]]))
    assert dev.max() > 1e-3  # the voxels are active
    err = np.abs(st - rst)
    assert err.max() <= 3e-5, f"max |state err| {err.max():.3e} per row {err.max(1)}"
    b = d["bold"]
    ytol = 3e-5 * b["V0"] * (7 * b["E0"] + 2 + abs(2 * b["E0"] - 0.2))
    assert np.abs(y - ry).max() <= ytol, f"max |y err| {np.abs(y - ry).max():.3e}"
    samples = net.get_bold_samples()
    assert samples.shape == (4, tb.nv)
    np.testing.assert_array_equal(samples[-1], y)


@pytest.mark.parametrize("delivery", MODES)
def test_checkpoint_and_hyperparams(dtb, delivery):
    tb = _tables("c2_multi_voxel_1m", n=20011, nv=5, K=50, gain={"default": 1.3})
    pull = ng.host_pull(tb)
    d = ng.oracle_inputs(tb, pull)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull), delivery=delivery)
    ref = oracle.OracleNet(d, "f32")
    _run_both(net, ref, [150])
    blob = net.save_state()
    net.step(70)
    ids_a = net.get_spikes()[0].copy()
    ref.run(70)
    g = d["vparams"][:, 6:10].copy()
    g[:, 0] *= 1.1
    g[::2, 2] *= 0.9
    net.set_hyperparams(g)
    ref.set_g(g)
    _run_both(net, ref, [130])
    _assert_state_equal(net, ref)
    # restore and replay the 70 steps: bit-identical raster
    net.load_state(blob)
    net.set_hyperparams(d["vparams"][:, 6:10])
    net.step(70)
    np.testing.assert_array_equal(net.get_spikes()[0], ids_a)
    net.reset()
    net.step(10)
    ref2 = oracle.OracleNet(d, "f32")
    rids, _ = ref2.run(10)
    np.testing.assert_array_equal(net.get_spikes()[0], rids)


def test_device_philox_matches_oracle(dtb):
    import torch

    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(4096, 2), dtype=np.uint64).astype(np.uint32)
    dc = torch.from_numpy(ctr.view(np.int32)).cuda()
    dk = torch.from_numpy(key.view(np.int32)).cuda()
    out = torch.empty_like(dc)
    dtb.dtb_philox_device(dc, dk, out)
    got = out.cpu().numpy().view(np.uint32)
    for i in range(0, 4096, 97):
        np.testing.assert_array_equal(got[i], oracle.philox4x32_10(ctr[i], key[i]))


def test_device_philox_known_answers(dtb):
    """The device Philox on the published known-answer vectors."""
    import torch

    from helpers import philox_kat

    ctr, key, want = philox_kat()
    dc = torch.from_numpy(np.ascontiguousarray(ctr).view(np.int32)).cuda()
    dk = torch.from_numpy(np.ascontiguousarray(key).view(np.int32)).cuda()
    out = torch.empty_like(dc)
    dtb.dtb_philox_device(dc, dk, out)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), want)


def test_device_generator_matches_host():
    import torch

    tb = _tables("c3_large_20m", n=60013, nv=30, K=70)
    row_ptr, word, w = ng.device_csr(tb, "int16")
    pull = ng.host_pull(tb)
    hrp, hword, hwb = ng.host_push(tb, pull)
    np.testing.assert_array_equal(row_ptr.cpu().numpy(), hrp)
    dw = word.cpu().numpy().view(np.uint32)
    dwt = w.cpu().numpy()
    hwt = tb.wtable("int16")[hwb]
    src = np.repeat(np.arange(tb.n), np.diff(hrp))
    a = np.lexsort((dwt, dw, src))
    b = np.lexsort((hwt, hword, src))
    np.testing.assert_array_equal(dw[a], hword[b])
    np.testing.assert_array_equal(dwt[a], hwt[b])
    del torch


@pytest.mark.parametrize("n,density", [(1, 1.0), (1000, 0.5), (65536, 0.01), (65537, 0.3), (3_000_001, 0.002),
                                       (20_000_000, 0.0015)])
def test_standalone_compaction(dtb, n, density):
    """dtb_spike_compact: ascending ids of a random bit set, every tile size and a ragged tail."""
    import torch

    rng = np.random.default_rng(n)
    words = -(-n // 1024) * 32
    flags = rng.random(n) < density
    pad = np.zeros(words * 32, bool)
    pad[:n] = flags
    bits = np.packbits(pad, bitorder="little").view(np.uint32)  # bit b of word w = neuron 32w + b
    d_bits = torch.from_numpy(bits.view(np.int32)).cuda()
    ids = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    dtb.dtb_spike_compact(d_bits, n, ids, cnt, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    expect = np.flatnonzero(flags).astype(np.int32)
    c = int(cnt.item())
    assert c == expect.size
    np.testing.assert_array_equal(ids[:c].cpu().numpy(), expect)


@pytest.mark.parametrize("delivery", MODES)
def test_ring_diagnostics_match_dense_view(dtb, delivery):
    """ring_slot_sums and get_ring_at agree with the dense ring of get_state."""
    tb = _tables("c2_multi_voxel_1m", n=30011, nv=6, K=60, gain={"default": 1.35})
    pull = ng.host_pull(tb)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull), delivery=delivery)
    net.step(157)
    ring = net.get_state()[3]
    np.testing.assert_array_equal(net.ring_slot_sums(), ring.astype(np.int64).sum(axis=2))
    idx = np.random.default_rng(1).choice(tb.n, size=500, replace=False)
    np.testing.assert_array_equal(net.get_ring_at(idx), ring[:, :, idx].transpose(2, 0, 1))


@pytest.mark.parametrize("delivery,qcap,bcap,wfmt", [("queue", 1024, 0, "int16"), ("bins", 1024, 0, "int16"),
                                                     ("bins", 0, 256, "int16"), ("bins", 0, 256, "int32")])
def test_queue_overflow_spills_exactly(dtb, delivery, qcap, bcap, wfmt):
    """Queues (or, in bins mode, region bins of 4- or 8-byte events) far too
    small: events spill into the dense ring and the run stays bit-exact."""
    tb = _tables("c2_multi_voxel_1m", n=30011, nv=6, K=60, wfmt=wfmt, gain={"default": 1.45})
    pull = ng.host_pull(tb)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull), delivery=delivery, event_queue_capacity=qcap,
                          bin_capacity=bcap)
    ref = oracle.OracleNet(ng.oracle_inputs(tb, pull), "f32")
    assert _run_both(net, ref, [40, 160, 33]) > 1000
    _assert_state_equal(net, ref)
    blob = net.save_state()  # dense view with spilled entries round-trips
    net.load_state(blob)
    _run_both(net, ref, [50])
    _assert_state_equal(net, ref)


@pytest.mark.parametrize("delivery,wfmt", [("queue", "int16"), ("bins", "int16"), ("bins", "int32")])
def test_event_counters_cannot_wrap(dtb, delivery, wfmt):
    """Every queue and bin count preset (test hook) to 2^32 - 2, where a 32-bit
    counter would wrap at its next reservation and hand out positions over
    queued events, and then to 2^40: the events of the following steps all
    spill and the run stays bit-exact with the oracle."""
    tb = _tables("c2_multi_voxel_1m", n=30011, nv=6, K=60, wfmt=wfmt, gain={"default": 1.45})
    pull = ng.host_pull(tb)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull), delivery=delivery)
    ref = oracle.OracleNet(ng.oracle_inputs(tb, pull), "f32")
    _run_both(net, ref, [60])
    net.test_preset_counters((1 << 32) - 2)
    assert _run_both(net, ref, [45, 7]) > 100
    _assert_state_equal(net, ref)
    net.test_preset_counters(1 << 40)
    _run_both(net, ref, [33])
    _assert_state_equal(net, ref)
    with pytest.raises(dtb.DtbError) as e:
        net.test_preset_counters(5)  # below the capacity
    assert e.value.code == dtb.DTB_EINVAL


@pytest.mark.parametrize("M", [8, 64, 1024])
def test_enkf_analysis_matches_oracle(dtb, M):
    """dtb_enkf_analysis (FP32) vs the FP64 oracle.  Float moments over M members of
    O(1) values carry relative errors of about M * 2^-24 at worst (6e-5 at
    M = 1024); asserted |d theta| <= 1e-4 * (1 + |theta|)."""
    import torch

    rng = np.random.default_rng(M)
    C = 300
    theta = rng.standard_normal((C, M)) * 0.3
    hx = 0.8 * theta + 0.1 * rng.standard_normal((C, M)) + 0.05
    y = rng.standard_normal(C) * 0.2
    sd = rng.uniform(0.05, 0.3, C)
    eps = rng.standard_normal((C, M))
    expect = oracle.enkf(theta, hx, y, sd, eps, lam=1.05)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()  # noqa: E731
    th = t(theta)
    dtb.dtb_enkf_analysis(th, t(hx), t(y), t(sd), t(eps), inflation=1.05)
    got = th.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - expect) <= 1e-4 * (1 + np.abs(expect)))
    assert np.abs(expect - theta).max() > 0.01  # the analysis moved the ensemble


OU = dict(mu=0.1, sigma=0.15, tau=5.0)


@pytest.mark.parametrize("delivery,n_ch,nu_ext", [("ring", 2, None), ("queue", 2, None), ("queue", 2, 0.0),
                                                  ("ring", 4, None), ("bins", 2, None), ("bins", 4, 0.0)])
def test_ou_drive_bit_exact(dtb, delivery, n_ch, nu_ext):
    # OU background current on top of (or, nu_ext = 0, instead of) the Poisson drive
    tb = _tables("c2_multi_voxel_1m", n=60013, nv=8, K=60, gain={"default": 1.3})
    pre, cls, wbin = ng.host_pull(tb)
    if n_ch == 4:
        cls = np.random.default_rng(4).integers(0, 4, size=cls.shape).astype(np.uint8)
    pull = (pre, cls, wbin)
    d = ng.oracle_inputs(tb, pull)
    d["n_ch"] = n_ch
    ou = dict(OU)
    if nu_ext is not None:
        d["nu_ext"] = nu_ext
        ou.update(mu=0.45, sigma=0.2)  # mean drive V_inf = EL + mu/gL just below threshold
    d["ou"] = ou
    row_ptr, word, wb = ng.host_push(tb, pull)
    net = dtb.Network(n=tb.n, voxel_start=tb.voxel_start, vparams=d["vparams"], delay_vv=tb.delay_vv,
                      d_max=tb.d_max, csr=(row_ptr, word, tb.wtable("int32")[wb]), wfmt="int32", wshift=0,
                      n_ch=n_ch, delivery=delivery, ou=ou, **_net_kw(d))
    ref = oracle.OracleNet(d, "f32")
    np.testing.assert_array_equal(net.get_ou(), ref.get_ou())
    assert _run_both(net, ref, [33, 200, 64]) > 300
    _assert_state_equal(net, ref)
    np.testing.assert_array_equal(net.get_ou(), ref.get_ou())
    # checkpoint with OU currents: the restored run replays bit-exactly
    blob = net.save_state()
    net.step(50)
    ids_a, I_a = net.get_spikes()[0].copy(), net.get_ou()
    net.load_state(blob)
    net.step(50)
    np.testing.assert_array_equal(net.get_spikes()[0], ids_a)
    np.testing.assert_array_equal(net.get_ou(), I_a)
    # set_ou writes what get_ou reads; reset restores I = mu
    net.set_ou(np.full(tb.n, 0.25, np.float32))
    assert np.all(net.get_ou() == np.float32(0.25))
    net.reset()
    assert np.all(net.get_ou() == np.float32(ou["mu"]))


def test_ou_off_reports_state_error(dtb):
    tb = _tables("c1_single_voxel_1k")
    net = dtb.from_tables(tb, dtb.host_csr(tb, ng.host_pull(tb)))
    with pytest.raises(dtb.DtbError):
        net.get_ou()


@pytest.mark.parametrize("delivery", MODES)
def test_launch_shapes_do_not_change_results(dtb, delivery):
    # the pipelined step overlaps delivery with the next update differently for
    # every shape; the raster and the state must not depend on it
    tb = _tables("c2_multi_voxel_1m", n=70001, nv=12, K=80, gain={"default": 1.3})
    pull = ng.host_pull(tb)
    d = ng.oracle_inputs(tb, pull)
    ref = oracle.OracleNet(d, "f32")
    rids, roff = ref.run(260)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull), delivery=delivery)
    for shape in [(2, 1, 1), (4, 2, 3), (3, 0, 8), (2, 2, 2)]:
        net.set_shapes(*shape)
        net.reset()
        net.step(97)
        ids_a, off_a = net.get_spikes()
        net.step(163)
        ids_b, off_b = net.get_spikes()
        np.testing.assert_array_equal(np.concatenate([ids_a, ids_b]), rids)
        np.testing.assert_array_equal(np.diff(np.concatenate([off_a, off_b[1:] + off_a[-1]])), np.diff(roff))
    _assert_state_equal(net, ref)
    with pytest.raises(dtb.DtbError):
        net.set_shapes(5, 1, 1)
