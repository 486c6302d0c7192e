"""Pins of the oracle's neuron update (Eq. 1, explicit Euler) to closed forms.

* subthreshold relaxation: the Euler map V <- V - kL (V - EL) + kI has the
  closed form V_n = V_inf + (V_0 - V_inf)(1 - kL)^n, and tends to the
  continuous exponential with time constant C/gL as dt -> 0;
* interspike interval under constant suprathreshold current: the refractory
  steps plus the first n at which the closed form reaches threshold, and the
  continuous formula t_ref + tau_m ln((Vreset - V_inf) / (Vth - V_inf));
* gating variables: a single arrival w gives j_n = w (1 - dt/tau)^(n-1) on
  the receptors its class opens (a pair with two channels, one with four);
* refractoriness: V held at Vreset for round(t_ref/dt) steps, min ISI 21;
  arrivals during the hold still enter j; V exactly at threshold fires;
* Poisson drive: with j_AMPA frozen, it counts the drive's arrivals in units of
  w_ext 2^-16; their mean per step is lambda (the Poisson law), the other
  three receptors stay 0 in both channel modes;
* synaptic currents: with the gating variables frozen (tau so large that
  1 - dt/tau rounds to 1), V follows an affine map whose fixed point is the
  conductance-weighted mean of the reversal potentials, per receptor pair;
* FP64 bounds the FP32 one-step error at 1e-6 relative;
* initial state: V uniform on [Vreset, Vth) of each neuron's own voxel,
  independent across neurons; j, ref and the ring zero.
"""
import math

import numpy as np
import pytest

import oracle
from helpers import custom_net, lone_neurons, params_row

DT = 0.1
C, GL, EL, VTH, VRESET = 0.5, 0.025, -70.0, -50.0, -55.0
KL = DT * GL / C
TAU_M = C / GL


def _set_V(net, V0):
    V, j, ref, ring, t = net.get_state()
    V[:] = V0
    net.set_state(V, j, ref, ring, t)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_subthreshold_relaxation_closed_form(prec):
    I = 0.4  # nA -> V_inf = EL + I/gL = -54 mV, below threshold
    net = oracle.OracleNet(lone_neurons(4, I_ext=I), prec)
    V0 = np.array([-65.0, -70.0, -58.0, -54.5])
    _set_V(net, V0)
    kI = DT * I / C
    V_inf = EL + kI / KL
    trace = []
    for _ in range(50):
        net.run(100)
        trace.append(net.get_state()[0].astype(np.float64).copy())
    trace = np.array(trace)
    n = np.arange(1, 51)[:, None] * 100
    closed = V_inf + (V0[None, :] - V_inf) * (1.0 - KL) ** n
    tol = 1e-10 if prec == "f64" else 5e-3  # f32: per-step ulp error / kL
    np.testing.assert_allclose(trace, closed, rtol=0, atol=tol)
    # continuous solution of C dV/dt = -gL (V - EL) + I, within O(dt)
    cont = V_inf + (V0[None, :] - V_inf) * np.exp(-n * DT / TAU_M)
    assert np.max(np.abs(trace - cont)) < 0.02 * np.max(np.abs(V0 - V_inf))
    assert np.max(np.abs(trace - cont)) > 0  # Euler is not exact


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_isi_constant_drive(prec):
    I = 0.6  # V_inf = -46 mV
    net = oracle.OracleNet(lone_neurons(1, I_ext=I), prec)
    _set_V(net, [VRESET])
    ids, off = net.run(3000)
    steps = np.repeat(np.arange(3000), np.diff(off))
    isi = np.diff(steps)
    kI = DT * I / C
    V_inf = EL + kI / KL
    n = np.arange(1, 10000)
    Vn = V_inf + (VRESET - V_inf) * (1.0 - KL) ** n
    nstar = int(n[np.argmax(Vn >= VTH)])
    assert abs(Vn[nstar - 1] - VTH) > 1e-4 and abs(Vn[nstar - 2] - VTH) > 1e-4
    ref_steps = round(2.0 / DT)
    assert len(isi) > 5
    assert np.all(isi == ref_steps + nstar)
    # first spike from Vreset without a preceding refractory period
    assert steps[0] == nstar - 1
    T_cont = 2.0 + TAU_M * math.log((VRESET - V_inf) / (VTH - V_inf))
    assert abs(isi[0] * DT - T_cont) < 3 * DT


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nch,cls", [(2, 0), (2, 1), (4, 0), (4, 1), (4, 2), (4, 3)])
def test_gating_jump_and_decay(prec, nch, cls):
    w = 81920  # 1.25 in 2^-16 units
    tau = (2.0, 100.0, 6.0, 100.0)
    prm = params_row(g=(0, 0, 0, 0), tau=tau)
    # neuron 0 feeds neuron 1 (delay 1); neuron 0's own input has weight 0
    d = custom_net(2, [[1], [0]], [[0], [cls]], np.array([[0], [w]], np.int32), prm, n_ch=nch)
    net = oracle.OracleNet(d, prec)
    _set_V(net, [-40.0, -60.0])  # neuron 0 fires at step 0
    ids, off = net.run(1)
    assert list(ids) == [0]
    js = []
    for _ in range(40):
        net.run(1)
        js.append(net.get_state()[1][:, 1].astype(np.float64).copy())
    js = np.array(js)  # [step, receptor]
    n = np.arange(40)[:, None]
    decay = np.array([1.0 - DT / t for t in tau])[None, :]
    expect = (w / 65536.0) * decay ** n
    # two channels: an E synapse opens AMPA and NMDA, an I synapse GABAa and
    # GABAb; four channels: class c opens receptor c alone
    on = ([0, 1] if cls == 0 else [2, 3]) if nch == 2 else [cls]
    off_ = [u for u in range(4) if u not in on]
    rtol = 1e-12 if prec == "f64" else 2e-6
    np.testing.assert_allclose(js[:, on], expect[:, on], rtol=rtol)
    assert np.all(js[:, off_] == 0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_refractory_hold_and_min_isi(prec):
    net = oracle.OracleNet(lone_neurons(1, I_ext=30.0), prec)  # one step from reset reaches threshold
    _set_V(net, [VRESET])
    Vs, spikes = [], []
    for _ in range(200):
        ids, _ = net.run(1)
        spikes.append(len(ids))
        Vs.append(float(net.get_state()[0][0]))
    st = np.flatnonzero(spikes)
    assert np.all(np.diff(st) == 21)
    for s in st[:-1]:
        assert all(v == VRESET for v in Vs[s: s + 21])


def test_f64_bounds_f32_one_step():
    from paper_2308_01241_gb300 import netgen as ng

    cfg = ng.load_config("c1_single_voxel_1k")
    tb = ng.make_tables(cfg)
    d = ng.oracle_inputs(tb, ng.host_pull(tb))
    n32 = oracle.OracleNet(d, "f32")
    n64 = oracle.OracleNet(d, "f64")
    n32.run(400)
    V, j, ref, ring, t = n32.get_state()
    n64.set_state(V.astype(np.float64), j.astype(np.float64), ref, ring, t)
    n32.run(1)
    n64.run(1)
    V32, j32 = n32.get_state()[:2]
    V64, j64 = n64.get_state()[:2]
    relV = np.abs(V32 - V64) / np.abs(V64)
    assert relV.max() <= 1e-6
    mask = np.abs(j64) > 1e-30
    relj = np.abs(j32[mask] - j64[mask]) / np.abs(j64[mask])
    assert relj.max() <= 1e-6
    assert np.all(j32[~mask] == 0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("cls", [0, 1])
def test_frozen_conductance_relaxes_to_weighted_reversal_potential(prec, cls):
    w = 163840  # j = 2.5 on both receptors of the pair
    j = w / 65536.0
    g = (0.002, 0.001, 0.01, 0.0005)
    E = (0.0, -10.0, -70.0, -100.0)  # distinct within each pair, so a swapped receptor index shows
    I = 0.1
    prm = params_row(g=g, tau=(1e30,) * 4, E=E, I_ext=I)
    d = custom_net(2, [[1], [0]], [[0], [cls]], np.array([[0], [w]], np.int32), prm)
    net = oracle.OracleNet(d, prec)
    _set_V(net, [-40.0, -60.0])  # neuron 0 fires at step 0; its arrival is consumed at step 1
    net.run(2)
    jj = net.get_state()[1][:, 1].astype(np.float64)
    on = [0, 1] if cls == 0 else [2, 3]
    assert np.all(jj[on] == j) and np.all(np.delete(jj, on) == 0)
    V0 = -60.0
    _set_V(net, [VRESET - 20.0, V0])
    gsyn = sum(g[u] * j for u in on)
    V_star = (GL * EL + sum(g[u] * j * E[u] for u in on) + I) / (GL + gsyn)
    a = 1.0 - DT * (GL + gsyn) / C  # Euler factor of V - V_star per step
    trace = []
    for _ in range(40):
        ids, _ = net.run(50)
        assert 1 not in ids
        trace.append(float(net.get_state()[0][1]))
    n = np.arange(1, 41) * 50
    closed = V_star + (V0 - V_star) * a ** n
    tol = 1e-9 if prec == "f64" else 5e-3
    np.testing.assert_allclose(trace, closed, rtol=0, atol=tol)
    # the pair's reversal potentials pull V toward V_star: above EL for the
    # excitatory pair, below it for the inhibitory one
    assert (V_star > EL + I / GL) if cls == 0 else (V_star < EL + I / GL)
    # continuous solution with time constant C / (gL + g_syn j), within O(dt)
    cont = V_star + (V0 - V_star) * np.exp(-n * DT * (GL + gsyn) / C)
    assert np.max(np.abs(np.array(trace) - cont)) < 0.02 * abs(V0 - V_star)


@pytest.mark.parametrize("nch", [2, 4])
def test_poisson_drive_enters_ampa_only_in_units_of_w_ext(nch):
    n, steps, scale = 20000, 50, 3
    lam = (2000.0 * DT) / 1000.0
    prm = params_row(g=(0, 0, 0, 0), tau=(1e30, 100.0, 6.0, 100.0))
    d = custom_net(n, np.zeros((n, 0), np.int32), np.zeros((n, 0), np.uint8), np.zeros((n, 0), np.int32), prm,
                   n_ch=nch, nu_ext=2000.0, w_ext=scale * 65536, seed=7)
    net = oracle.OracleNet(d, "f32")
    net.run(steps)
    j = net.get_state()[1].astype(np.float64)
    assert np.all(j[1:] == 0)
    counts = j[0] / scale
    assert np.all(counts == np.round(counts)) and counts.min() >= 0
    # sum of n * steps independent Poisson(lambda) draws
    mean = counts.mean() / steps
    assert abs(mean - lam) < 4 * np.sqrt(lam / (n * steps))
    assert abs(counts.var() / steps - lam) < 0.1 * lam
    # the same draws as the drive's own counts
    want = sum(oracle.drive_counts(7, lam, t, 0, n).astype(np.int64) for t in range(steps))
    np.testing.assert_array_equal(counts.astype(np.int64), want)


def test_initial_state_uniform_between_reset_and_threshold():
    from scipy.stats import kstest

    n = 100003
    P = [params_row(Vth=-50.0, Vreset=-55.0), params_row(Vth=-45.0, Vreset=-65.0)]
    vs = np.array([0, 40000, n], np.int64)
    d = custom_net(n, np.zeros((n, 0), np.int32), np.zeros((n, 0), np.uint8), np.zeros((n, 0), np.int32), P,
                   voxel_start=vs, init_seed=11)
    V, j, ref, ring, t = oracle.OracleNet(d, "f64").get_state()
    assert t == 0 and not j.any() and not ref.any() and not ring.any()
    for v, (lo, hi) in enumerate([(-55.0, -50.0), (-65.0, -45.0)]):
        u = (V[vs[v]:vs[v + 1]] - lo) / (hi - lo)
        assert u.min() >= 0.0 and u.max() < 1.0
        assert kstest(u, "uniform").pvalue > 1e-3
        # neighbours draw different words of one Philox block, then new blocks
        for lag in (1, 2, 3, 4):
            assert abs(np.corrcoef(u[:-lag], u[lag:])[0, 1]) < 0.02
        assert np.unique(u).size > 0.99 * u.size
    # another seed, other voltages
    d["init_seed"] = 12
    V2 = oracle.OracleNet(d, "f64").get_state()[0]
    assert np.mean(V2 == V) < 1e-3


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gating_integrates_during_refractory_hold(prec):
    w = 98304  # 1.5
    tau = (2.0, 100.0, 6.0, 100.0)
    prm = params_row(tau=tau)
    d = custom_net(1, [[0]], [[0]], np.array([[w]], np.int32), prm)  # a self-synapse, delay 1
    net = oracle.OracleNet(d, prec)
    _set_V(net, [-40.0])
    ids, _ = net.run(1)
    assert list(ids) == [0]
    decay = np.array([1.0 - DT / t for t in tau])
    for n in range(15):  # inside the 20-step hold
        net.run(1)
        V, j, ref = net.get_state()[:3]
        assert float(V[0]) == VRESET and int(ref[0]) == 19 - n
        want = (w / 65536.0) * decay ** n
        rtol = 1e-12 if prec == "f64" else 2e-6
        np.testing.assert_allclose(j[:2, 0].astype(np.float64), want[:2], rtol=rtol)
        assert np.all(j[2:, 0] == 0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_voltage_equal_to_threshold_fires(prec):
    # EL = Vth and no current: the Euler map leaves V = Vth exactly
    net = oracle.OracleNet(lone_neurons(2, EL=VTH, g=(0, 0, 0, 0)), prec)
    _set_V(net, [VTH, np.nextafter(np.float32(VTH), np.float32(-100.0))])
    ids, _ = net.run(1)
    assert list(ids) == [0]

