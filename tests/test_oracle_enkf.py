"""Pins of the oracle's ensemble-Kalman analysis (the hierarchical data
assimilation of section V.E, read as a stochastic EnKF with perturbed
observations, local per voxel parameter).

* linear-Gaussian case: with h = a theta + b exactly, a Gaussian prior and a
  large ensemble, the analysis ensemble's mean and variance converge to the
  Kalman posterior mu0 + K (y - a mu0 - b), (1 - K a) s0^2 with
  K = a s0^2 / (a^2 s0^2 + sd^2);
* no information: with constant predictions (zero spread) the gain is zero
  and theta only changes by the inflation of its anomalies, exactly;
* huge observation noise leaves theta (nearly) unchanged;
* a two-member case worked by hand.
"""
import numpy as np

import oracle


def test_linear_gaussian_converges_to_kalman_posterior():
    rng = np.random.default_rng(0)
    M, C = 40000, 3
    mu0, s0 = np.array([0.0, 1.0, -2.0]), np.array([1.0, 0.5, 2.0])
    a, b, sd = np.array([2.0, -1.0, 0.5]), np.array([0.3, 0.0, 1.0]), np.array([0.5, 0.2, 1.5])
    y = np.array([1.7, -0.4, 0.0])
    theta = mu0[:, None] + s0[:, None] * rng.standard_normal((C, M))
    hx = a[:, None] * theta + b[:, None]
    eps = rng.standard_normal((C, M))
    post = oracle.enkf(theta, hx, y, sd, eps)
    K = a * s0 ** 2 / (a ** 2 * s0 ** 2 + sd ** 2)
    mu = mu0 + K * (y - a * mu0 - b)
    var = (1 - K * a) * s0 ** 2
    se_mu = np.sqrt(var / M)
    assert np.all(np.abs(post.mean(1) - mu) < 5 * se_mu + 1e-12)
    assert np.all(np.abs(post.var(1, ddof=1) / var - 1) < 5 * np.sqrt(2.0 / M))


def test_zero_spread_only_inflates():
    rng = np.random.default_rng(1)
    theta = rng.standard_normal((4, 16))
    hx = np.ones((4, 16)) * 3.0
    eps = rng.standard_normal((4, 16))
    post = oracle.enkf(theta, hx, np.zeros(4), np.ones(4), eps, lam=1.3)
    m = theta.mean(1, keepdims=True)
    np.testing.assert_allclose(post, m + 1.3 * (theta - m), rtol=0, atol=1e-14)


def test_huge_noise_leaves_theta():
    rng = np.random.default_rng(2)
    theta = rng.standard_normal((2, 32))
    hx = theta * 2.0
    post = oracle.enkf(theta, hx, np.array([5.0, -5.0]), np.array([1e9, 1e9]), rng.standard_normal((2, 32)))
    np.testing.assert_allclose(post, theta, atol=1e-6)


def test_two_members_by_hand():
    # theta = (0, 2), hx = (1, 3): mean theta 1, mean h 2, cov 2, var 2; sd = 1 -> K = 2/3
    # y = 4, eps = (0, 1): theta_0 = 0 + 2/3 (4 - 1) = 2; theta_1 = 2 + 2/3 (4 + 1 - 3) = 10/3
    post = oracle.enkf([[0.0, 2.0]], [[1.0, 3.0]], [4.0], [1.0], [[0.0, 1.0]])
    np.testing.assert_allclose(post, [[2.0, 10.0 / 3.0]], rtol=1e-15)
