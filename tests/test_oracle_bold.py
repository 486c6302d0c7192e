"""Pins of the oracle's Balloon-Windkessel BOLD model (section V.E cites
Friston 2000; the equations are that model's).

* rest: zero input keeps s = 0, f = v = q = 1 and y = 0 exactly;
* steady state under constant rate z: s = 0, f = 1 + eps z tau_f,
  v = f^alpha, q = v E(f)/E0 with E(f) = 1 - (1 - E0)^(1/f);
* the (s, f) subsystem is linear, so f - 1 after a step input is the damped
  oscillator x'' + x'/tau_s + x/tau_f = eps z, whose closed form the Euler
  trajectory must follow to O(dt);
* the network's input to the model: the voxel rate z = spikes / (n_v dt) in
  Hz, so one Euler step from rest sets s = eps * (the voxel's fraction of
  neurons that fired) and leaves f = v = q = 1.
"""
import math

import numpy as np

import oracle
from helpers import BOLD, custom_net, params_row


def test_rest_is_fixed_point():
    st, y = oracle.bold_integrate(BOLD, np.zeros(3), 10000, 1e-4)
    assert np.array_equal(st, np.array([[0.0] * 3, [1.0] * 3, [1.0] * 3, [1.0] * 3]))
    assert np.array_equal(y, np.zeros(3))


def test_steady_state_closed_form():
    z = np.array([2.0, 7.0, 15.0, 30.0])
    st, y = oracle.bold_integrate(BOLD, z, 600000, 1e-4)  # 60 s
    eps, tf, a, E0, V0 = BOLD["eps"], BOLD["tau_f"], BOLD["alpha"], BOLD["E0"], BOLD["V0"]
    f = 1 + eps * z * tf
    v = f ** a
    q = v * (1 - (1 - E0) ** (1 / f)) / E0
    yy = V0 * (7 * E0 * (1 - q) + 2 * (1 - q / v) + (2 * E0 - 0.2) * (1 - v))
    np.testing.assert_allclose(st[0], 0, atol=1e-6)
    np.testing.assert_allclose(st[1], f, rtol=1e-6)
    np.testing.assert_allclose(st[2], v, rtol=1e-5)
    np.testing.assert_allclose(st[3], q, rtol=1e-5)
    np.testing.assert_allclose(y, yy, rtol=1e-4)
    assert np.all(np.diff(y) > 0)  # more activity, more BOLD


def test_flow_step_response_closed_form():
    z = np.array([10.0])
    eps, ts, tf = BOLD["eps"], BOLD["tau_s"], BOLD["tau_f"]
    kap, gam = 1 / ts, 1 / tf
    om = math.sqrt(gam - kap * kap / 4)
    st = None
    t = 0.0
    for T in (0.25, 0.5, 1.0, 2.0, 4.0, 8.0):
        st, _ = oracle.bold_integrate(BOLD, z, int(round((T - t) / 1e-4)), 1e-4, st)
        t = T
        x = (eps * z[0] / gam) * (1 - math.exp(-kap * T / 2) * (math.cos(om * T) + kap / (2 * om) * math.sin(om * T)))
        assert abs((st[1][0] - 1) - x) < 2e-4 * eps * z[0] / gam + 1e-9
        s_exact = (eps * z[0] / om) * math.exp(-kap * T / 2) * math.sin(om * T)
        assert abs(st[0][0] - s_exact) < 2e-4 * eps * z[0]


def test_voxel_rate_input_from_spike_counts():
    sizes = [10, 37, 53, 8]
    fire = [3, 0, 11, 8]  # neurons of each voxel above threshold at step 0
    vs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(vs[-1])
    d = custom_net(n, np.zeros((n, 0), np.int32), np.zeros((n, 0), np.uint8), np.zeros((n, 0), np.int32),
                   params_row(), voxel_start=vs)
    for prec in ("f32", "f64"):
        net = oracle.OracleNet(d, prec)
        V, j, ref, ring, t = net.get_state()
        V[:] = -60.0
        for v in range(len(sizes)):
            V[vs[v]: vs[v] + fire[v]] = -40.0
        net.set_state(V, j, ref, ring, t)
        ids, _ = net.run(1)
        assert len(ids) == sum(fire)
        y, st = net.get_bold()
        frac = np.array(fire) / np.array(sizes)
        np.testing.assert_allclose(st[0], BOLD["eps"] * frac, rtol=1e-12, atol=0)
        assert np.array_equal(st[1:], np.ones((3, len(sizes))))
        assert np.array_equal(y, np.zeros(len(sizes)))

