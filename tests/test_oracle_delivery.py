"""Pins of the oracle's spike delivery (sections V.B, V.D: weighted sums of
presynaptic spikes arriving after a voxel-pair delay).

* brute force: on 10-neuron dense nets with explicit W, receptor classes and
  voxel-pair delays, a naive pull-form loop over a spike history (written
  here, independently of the oracle's outgoing lists and delay ring) gives the
  same rasters and bit-identical voltages;
* conservation: the int64 sum of everything one step adds to the delay ring
  equals the summed outgoing weight of the neurons that spiked, and the event
  count equals their summed out-degree.
"""
import numpy as np
import pytest

import oracle
from helpers import custom_net, params_row


def _brute_force(d, n_steps):
    """Pull-form reference: input of neuron i at step t is the sum over its
    inputs k of w[i,k] if pre[i,k] spiked at step t - delay(vox(pre), vox(i))."""
    f32 = np.float32
    n, K, nch = d["n"], d["K"], d["n_ch"]
    vs = d["voxel_start"]
    vox = np.searchsorted(vs, np.arange(n), side="right") - 1
    P = d["vparams"]
    kL = np.array([f32((0.1 * p[1]) / p[0]) for p in P])[vox]
    EL = P[vox, 2].astype(f32)
    Vth = P[vox, 3].astype(f32)
    Vr = P[vox, 4].astype(f32)
    kI = np.array([f32((0.1 * p[18]) / p[0]) for p in P])[vox]
    kU = np.array([[f32((0.1 * p[6 + u]) / p[0]) for u in range(4)] for p in P])[vox]
    dJ = np.array([[f32(1.0 - 0.1 / p[10 + u]) for u in range(4)] for p in P])[vox]
    E = P[vox, 14:18].astype(f32)
    refn = np.array([round(p[5] / 0.1) for p in P])[vox]
    lam = d["nu_ext"] * 0.1 / 1000.0
    # initial voltages the oracle draws (state read back, not recomputed)
    V = d["_V0"].astype(f32).copy()
    j = np.zeros((n, 4), f32)
    ref = np.zeros(n, np.int64)
    hist = np.zeros((n_steps, n), bool)
    raster = []
    SC = f32(1.0 / 65536.0)
    for t in range(n_steps):
        A = np.zeros((n, nch), np.int64)
        for i in range(n):
            for k in range(K):
                p = d["pre"][i, k]
                dd = int(d["delay_vv"][vox[p], vox[i]])
                if t - dd >= 0 and hist[t - dd, p]:
                    A[i, d["cls"][i, k]] += int(d["w"][i, k]) << d["wshift"]
        kk = oracle.drive_counts(d["seed"], lam, t, 0, n).astype(np.int64)
        if nch == 2:
            inp = np.stack([A[:, 0] + kk * d["w_ext"], A[:, 0], A[:, 1], A[:, 1]], 1)
        else:
            inp = np.stack([A[:, 0] + kk * d["w_ext"], A[:, 1], A[:, 2], A[:, 3]], 1)
        a = inp.astype(np.int32).astype(f32) * SC
        syn = np.zeros(n, f32)
        for u in range(4):
            x = V - E[:, u]
            y = kU[:, u] * j[:, u]
            syn = syn + y * x
        Vn = V - kL * (V - EL)
        Vn = Vn - syn
        Vn = Vn + kI
        j = dJ * j + a
        fired = []
        for i in range(n):
            if ref[i] > 0:
                ref[i] -= 1
                Vn[i] = Vr[i]
            elif Vn[i] >= Vth[i]:
                fired.append(i)
                Vn[i] = Vr[i]
                ref[i] = refn[i]
        V = Vn
        hist[t, fired] = True
        raster.append(fired)
    return raster, V, j


@pytest.mark.parametrize("nch", [2, 4])
@pytest.mark.parametrize("seed", [11, 12, 13])
def test_brute_force_dense_10(nch, seed):
    rng = np.random.default_rng(seed)
    n, d_max = 10, 6
    pre = np.tile(np.arange(n, dtype=np.int32), (n, 1))  # dense: input k of every neuron is neuron k
    cls = rng.integers(0, nch, size=(n, n)).astype(np.uint8)
    w = rng.integers(0, 1 << 17, size=(n, n)).astype(np.int32)
    P = np.stack([params_row(g=(0.002 * rng.uniform(1, 2), 0.00002, 0.01 * rng.uniform(0.5, 1), 0.0005),
                             I_ext=rng.uniform(0.0, 0.3)) for _ in range(n)])
    delay = rng.integers(1, d_max + 1, size=(n, n)).astype(np.uint8)
    np.fill_diagonal(delay, 1)
    d = custom_net(n, pre, cls, w, P, voxel_start=np.arange(n + 1), delay_vv=delay, d_max=d_max, n_ch=nch,
                   nu_ext=4000.0, seed=seed)
    net = oracle.OracleNet(d, "f32")
    d["_V0"] = net.get_state()[0]
    steps = 300
    ids, off = net.run(steps)
    raster, V, j = _brute_force(d, steps)
    got = [list(ids[off[t]:off[t + 1]]) for t in range(steps)]
    assert sum(len(r) for r in raster) > 10
    assert got == raster
    V_o, j_o = net.get_state()[:2]
    assert np.array_equal(V_o, V)
    assert np.array_equal(j_o, j.T)


def test_conservation_c1():
    from paper_2308_01241_gb300 import netgen as ng

    cfg = ng.load_config("c1_single_voxel_1k")
    tb = ng.make_tables(cfg)
    pull = ng.host_pull(tb)
    d = ng.oracle_inputs(tb, pull, rate="default")
    d["vparams"][:, 6:8] *= 1.8  # more spikes
    net = oracle.OracleNet(d, "f32")
    net.run(200)
    w_acc = d["w"].astype(np.int64) << d["wshift"]
    outsum = np.bincount(d["pre"].ravel(), weights=w_acc.ravel(), minlength=tb.n).astype(np.int64)
    outdeg = np.bincount(d["pre"].ravel(), minlength=tb.n)
    checked = 0
    for _ in range(150):
        V, j, ref, ring0, t = net.get_state()
        ev0 = net.events()
        ids, off = net.run(1)
        ring1 = net.get_state()[3]
        slot = t % net.D
        assert np.all(ring1[slot] == 0)  # consumed and cleared
        r0 = ring0.astype(np.int64).copy()
        r0[slot] = 0
        added = int(ring1.astype(np.int64).sum() - r0.sum())
        assert added == int(outsum[ids].sum())
        assert net.events() - ev0 == int(outdeg[ids].sum())
        checked += len(ids)
    assert checked > 20


# bf16 bit patterns and their accumulator values rne(float(w) * 2^16), worked
# out by hand: exact products, and the ties 0.5 -> 0, 1.5 -> 2, 2.5 -> 2, 3.5 -> 4
BF16_CASES = [(0x3F80, 65536), (0xBF00, -32768), (0x4120, 655360), (0x3E2A, 10880), (0x3FC0, 98304),
              (0x3780, 1), (0x3700, 0), (0x37C0, 2), (0x3820, 2), (0x3860, 4), (0xB7C0, -2), (0x8000, 0)]
# int8 codes q and the source rows' shifts: q * 2^(8 + row_shift[source])
INT8_CASES = [-128, -5, 1, 127, 64, -1]


def _two_sources_net(wfmt, codes, pre_shift=None):
    """Neurons 0, 1 (voxel 0, strong constant drive) feed six silent targets
    (voxel 1) through four inputs each; the sources' own inputs come from the
    targets with weight code 0.  Delay 1, no Poisson drive."""
    n, K = 8, 4
    pre = np.zeros((n, K), np.int32)
    cls = np.zeros((n, K), np.uint8)
    w = np.zeros((n, K), np.uint16 if wfmt == oracle.W_BF16 else np.int8)
    pre[0:2] = [2, 3, 4, 5]
    for t in range(6):
        for k in range(K):
            pre[2 + t, k] = (t + k) % 2
            cls[2 + t, k] = (t * K + k) // 3 % 2
            w[2 + t, k] = codes[(t * K + k) % len(codes)]
    P = [params_row(I_ext=2.0), params_row(I_ext=0.0)]
    d = custom_net(n, pre, cls, w, P, voxel_start=np.array([0, 2, 8]), delay_vv=np.ones((2, 2), np.uint8),
                   d_max=1, wfmt=wfmt, wshift=0 if wfmt == oracle.W_BF16 else 8)
    if pre_shift is not None:
        d["pre_shift"] = np.asarray(pre_shift, np.uint8)
    return d


def _check_increments(d, value_of):
    """Every step: the ring slot the step's spikes arrive in holds, per target
    and channel, the sum of value_of(code, source) over the spiking sources."""
    net = oracle.OracleNet(d, "f32")
    n, K = d["pre"].shape
    fired_sources = set()
    for _ in range(120):
        t = net.get_state()[4]
        ids, _ = net.run(1)
        ring = net.get_state()[3].astype(np.int64)
        want = np.zeros((2, n), np.int64)
        for i in range(n):
            for k in range(K):
                if d["pre"][i, k] in ids:
                    want[d["cls"][i, k], i] += value_of(int(d["w"][i, k]), int(d["pre"][i, k]))
        np.testing.assert_array_equal(ring[(t + 1) % net.D], want)
        fired_sources.update(int(s) for s in ids if s < 2)
    assert fired_sources == {0, 1}


def test_bf16_weights_decode_round_to_nearest_even():
    table = dict(BF16_CASES)
    d = _two_sources_net(oracle.W_BF16, [b for b, _ in BF16_CASES])
    _check_increments(d, lambda code, src: table[code])


def test_int8_weights_take_the_source_rows_shift():
    shift = np.array([3, 0, 5, 1, 2, 4, 6, 7], np.uint8)  # targets' shifts differ from both sources'
    d = _two_sources_net(oracle.W_INT8, INT8_CASES, pre_shift=shift)
    _check_increments(d, lambda code, src: (code if code < 128 else code - 256) * 2 ** (8 + int(shift[src])))
