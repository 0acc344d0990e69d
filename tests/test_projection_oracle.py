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
