"""Pins of the oracle's Ornstein-Uhlenbeck background current (section III.B).

The OU current I obeys tau dI = (mu - I) dt + sigma sqrt(2 tau) dW and adds
(dt/C) I to the membrane each step (Euler-Maruyama):

* starting at mu, the mean stays mu; the stationary variance of the AR(1) map
  I <- d I + c + s xi is s^2 / (1 - d^2), which tends to sigma^2 as dt -> 0;
* the lag-k autocorrelation is d^k, i.e. exp(-k dt / tau) to O(dt);
* the innovations xi recovered from consecutive currents have mean 0,
  variance 1, the Irwin-Hall(4) bound 2 sqrt 3 and excess kurtosis -0.3, and
  are uncorrelated between neurons and steps;
* with sigma = 0 the current stays mu and the membrane follows the closed
  form of the deterministic relaxation with I_ext + mu;
* a subthreshold neuron driven by OU noise: the stationary covariance of
  (V, I) is the solution of the discrete Lyapunov equation of the linear map
  (scipy), which pins the coupling dt/C and its step order.
"""
import numpy as np
import pytest
from scipy.linalg import solve_discrete_lyapunov

import oracle
from helpers import lone_neurons

DT = 0.1
C, GL, EL = 0.5, 0.025, -70.0
KL = DT * GL / C


def _ou_net(n, mu, sigma, tau, I_ext=0.0, seed=2):
    d = lone_neurons(n, I_ext=I_ext)
    d["ou"] = dict(mu=mu, sigma=sigma, tau=tau)
    d["seed"] = seed
    return d


def _trace(net, steps, every):
    out = []
    for _ in range(steps // every):
        net.run(every)
        out.append(net.get_ou().astype(np.float64).copy())
    return np.array(out)


def test_ou_off_reads_zero_and_starts_at_mu():
    net = oracle.OracleNet(lone_neurons(8), "f64")
    assert np.all(net.get_ou() == 0)
    net = oracle.OracleNet(_ou_net(8, 0.3, 0.1, 5.0), "f64")
    assert np.all(net.get_ou() == 0.3)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ou_stationary_mean_variance_autocorrelation(prec):
    mu, sigma, tau = 0.1, 0.05, 5.0
    n = 2048
    net = oracle.OracleNet(_ou_net(n, mu, sigma, tau), prec)
    net.run(1000)  # 20 tau
    lag = 25
    tr = []
    for _ in range(40):
        a = net.get_ou().astype(np.float64).copy()
        net.run(lag)
        b = net.get_ou().astype(np.float64).copy()
        tr.append((a, b))
        net.run(75)
    a = np.array([x for x, _ in tr]).ravel()
    b = np.array([y for _, y in tr]).ravel()
    d = 1.0 - DT / tau
    s = sigma * np.sqrt(2.0 * DT / tau)
    var_exact = s * s / (1.0 - d * d)
    N = a.size
    assert abs(a.mean() - mu) < 5 * np.sqrt(var_exact / N * 3)
    assert abs(a.var() / var_exact - 1.0) < 0.03
    assert abs(var_exact / sigma ** 2 - 1.0) < 0.02  # Euler-Maruyama is O(dt/tau)
    rho = np.corrcoef(a, b)[0, 1]
    assert abs(rho - d ** lag) < 0.02
    assert abs(d ** lag - np.exp(-lag * DT / tau)) < 0.01


def test_ou_innovations_are_standard_irwin_hall():
    mu, sigma, tau = -0.2, 0.3, 3.0
    n, steps = 512, 400
    net = oracle.OracleNet(_ou_net(n, mu, sigma, tau, seed=7), "f64")
    I = [net.get_ou().copy()]
    for _ in range(steps):
        net.run(1)
        I.append(net.get_ou().copy())
    I = np.array(I)
    d = 1.0 - DT / tau
    c = mu * DT / tau
    s = sigma * np.sqrt(2.0 * DT / tau)
    xi = (I[1:] - (d * I[:-1] + c)) / s
    x = xi.ravel()
    assert abs(x.mean()) < 5 / np.sqrt(x.size)
    assert abs(x.var() - 1.0) < 0.02
    assert np.max(np.abs(x)) <= 2 * np.sqrt(3) + 1e-9
    kurt = np.mean((x - x.mean()) ** 4) / x.var() ** 2 - 3.0
    assert abs(kurt + 0.3) < 0.05  # Irwin-Hall(4): -6/(5*4)
    # neighbours in index and in time are independent draws
    assert abs(np.corrcoef(xi[:, :-1].ravel(), xi[:, 1:].ravel())[0, 1]) < 0.02
    assert abs(np.corrcoef(xi[:-1].ravel(), xi[1:].ravel())[0, 1]) < 0.02
    # another seed gives other draws
    net2 = oracle.OracleNet(_ou_net(n, mu, sigma, tau, seed=8), "f64")
    net2.run(1)
    assert not np.array_equal(net2.get_ou(), I[1])


def test_ou_deterministic_limit_is_constant_current():
    mu = 0.15
    net = oracle.OracleNet(_ou_net(3, mu, 0.0, 4.0, I_ext=0.1), "f64")
    V, j, ref, ring, t = net.get_state()
    V0 = np.array([-65.0, -60.0, -52.0])
    V[:] = V0
    net.set_state(V, j, ref, ring, t)
    net.run(2000)
    np.testing.assert_allclose(net.get_ou(), mu, rtol=0, atol=1e-12)
    kI = DT * (0.1 + mu) / C  # V_inf = EL + (I_ext + mu)/gL = -60 mV
    V_inf = EL + kI / KL
    closed = V_inf + (V0 - V_inf) * (1.0 - KL) ** 2000
    np.testing.assert_allclose(net.get_state()[0], closed, rtol=0, atol=1e-9)


def test_ou_membrane_covariance_matches_lyapunov():
    mu, sigma, tau = 0.0, 0.06, 5.0  # V stays far below threshold
    n = 2048
    net = oracle.OracleNet(_ou_net(n, mu, sigma, tau, seed=11), "f64")
    net.run(4000)  # 20 membrane time constants
    Vs, Is = [], []
    for _ in range(40):
        net.run(200)
        Vs.append(net.get_state()[0].astype(np.float64).copy())
        Is.append(net.get_ou().astype(np.float64).copy())
    V, I = np.array(Vs).ravel(), np.array(Is).ravel()
    assert V.max() < -60.0
    d = 1.0 - DT / tau
    s = sigma * np.sqrt(2.0 * DT / tau)
    A = np.array([[1.0 - KL, DT / C], [0.0, d]])
    P = solve_discrete_lyapunov(A, np.diag([0.0, s * s]))
    assert abs(V.mean() - EL) < 5 * np.sqrt(P[0, 0] / V.size * 10)
    assert abs(V.var() / P[0, 0] - 1.0) < 0.06
    cov = np.mean((V - V.mean()) * (I - I.mean()))
    assert abs(cov / P[0, 1] - 1.0) < 0.08
    # a coupling of dt (not dt/C) or one step late changes these moments
    P_wrong = solve_discrete_lyapunov(np.array([[1.0 - KL, DT], [0.0, d]]), np.diag([0.0, s * s]))
    assert abs(P_wrong[0, 0] / P[0, 0] - 1.0) > 0.5
