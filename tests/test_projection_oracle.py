"""Pins of the oracle's learned warp (App. F, learning h from the integrand)."""
import numpy as np
import pytest


def test_uniform_table_reproduces_the_plain_warp(oracle):
    T, n = 10.0, 4
    tabs = oracle.gf_tables(1.0, 0.2, T, 4096)
    sh = oracle.shift_words(5, 2, n)
    cdf = np.tile(np.linspace(0.0, 1.0, 1025), (n, 1))
    S1, n1 = oracle.estimate(n, 1024, sh, T, 1.0, tabs, T)
    S2, n2 = oracle.estimate_proj(n, 1024, sh, T, 1.0, cdf, tabs, T)
    assert np.array_equal(n1, n2)
    assert np.array_equal(S1, S2)


def test_order1_with_a_skewed_table_matches_adaptive_quadrature(oracle):
    """Importance sampling with any positive density is unbiased: Q_1 through an arbitrary
    table equals the 1-D quadrature of the same order-1 integrand."""
    from scipy.integrate import quad
    from paper_2002_12372_gb300 import workloads as W

    t = 10.0
    tabs = oracle.gf_tables(1.0, 0.5, t, 4096)
    f = lambda u: (-2j * oracle.integrand(1, np.array([u]), t, tabs, t)[0]).real
    knots = list(oracle.table_nodes(t, 4096)[2048:][::64]) + [t]
    exact, lo = 0.0, 0.0
    for hi in knots:
        if hi > lo:
            exact += quad(f, lo, hi, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
            lo = hi
    cdf = W.synthetic_projection(3, 1, 512)
    S, _ = oracle.estimate_proj(1, 2 ** 16, oracle.shift_words(9, 8, 1), t, 0.95, cdf, tabs, t)
    m, e = oracle.shift_statistics(oracle.q_from_sums(S).real)
    assert abs(m - exact) < 5 * e + 1e-9
    assert e < 1e-5


@pytest.mark.slow
def test_learned_table_lowers_the_error_bar_and_keeps_the_mean(oracle):
    T, n, N, K = 10.0, 5, 2 ** 12, 16
    tabs = oracle.gf_tables(1.0, 0.0, T, 4096)
    cdf = oracle.learn_projection(n, 20000, 2002123720, T, 1.0, tabs, T)
    assert np.all(np.diff(cdf, axis=1) > 0) and np.all(cdf[:, -1] == 1.0)
    sh = oracle.shift_words(2002123720, K, n)
    m0, e0 = oracle.shift_statistics(oracle.q_from_sums(oracle.estimate(n, N, sh, T, 1.0, tabs, T)[0]).real)
    m1, e1 = oracle.shift_statistics(
        oracle.q_from_sums(oracle.estimate_proj(n, N, sh, T, 1.0, cdf, tabs, T)[0]).real)
    assert e1 < e0
    assert abs(m1 - m0) < 4 * np.hypot(e0, e1)


@pytest.mark.parametrize("lam", [0.05, 0.1])
def test_projection_of_a_separable_density_is_its_smoothed_marginal(oracle, lam):
    """Samples on Sobol' points with the separable value g(x_1) g(x_2), g(x) = 1 + a cos(2 pi x):
    the projection onto x_d is g (the other factor integrates to 1), and smoothing with the
    kernel exp(-d^2 / lam^2) attenuates the cosine by exp(-pi^2 lam^2), so away from the edges
    the learned CDF is z + a exp(-pi^2 lam^2) sin(2 pi z) / (2 pi) up to a constant offset.
    A wrong kernel width, a half-bin shift of the centres or a dropped factor fails this."""
    M, a = 2 ** 16, 0.8
    V = oracle.sobol_direction_numbers(2)
    x = oracle.sobol_points(2, 0, M, V).astype(np.float64) * 2.0 ** -32
    g = lambda v: 1.0 + a * np.cos(2 * np.pi * v)
    vals = g(x[:, 0]) * g(x[:, 1]) / M
    cdf = oracle.projection_cdf(x, vals, n_bins=100, lam=lam, floor_frac=1e-3, cells=1024)
    z = np.arange(1025) / 1024.0
    want = z + a * np.exp(-(np.pi * lam) ** 2) * np.sin(2 * np.pi * z) / (2 * np.pi)
    inner = (z > 3 * lam) & (z < 1 - 3 * lam)
    for d in range(2):
        dev = cdf[d, inner] - want[inner]
        assert np.max(np.abs(dev - np.mean(dev))) < 1e-3, (d, np.max(np.abs(dev - np.mean(dev))))
    # a plainly wrong width is detected at the same bar
    wrong = z + a * np.exp(-(np.pi * 2 * lam) ** 2) * np.sin(2 * np.pi * z) / (2 * np.pi)
    dev = cdf[0, inner] - wrong[inner]
    assert np.max(np.abs(dev - np.mean(dev))) > 1e-3
