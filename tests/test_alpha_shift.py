"""Quadratic shift alpha of the interaction (App. E): U n_up n_down is written
U (n_up - alpha)(n_down - alpha), which moves every vertex diagonal of the
Keldysh matrices from g^<(0) to g^<(0) - i alpha and leaves the measurement
pair alone.

CPU pins of the oracle against things other than itself, then parity of the
CUDA path with the oracle at alpha != 0.
"""
import math

import numpy as np
import pytest


# ------------------------------------------------------------ oracle pins ---

@pytest.mark.parametrize("eps", [0.0, 0.7])
def test_alpha_at_the_occupation_removes_order_one(oracle, eps):
    """alpha = <n_sigma> = Im g^<(0): the shifted vertex density vanishes, so the
    one-vertex spin-down determinant is zero and c_1(u) = 0 at every u."""
    T = 10.0
    tabs = oracle.gf_tables(1.0, eps, T, 4096)
    n0 = float(np.imag(tabs[2]))
    u = np.linspace(0.0, T, 257).reshape(-1, 1)
    c0 = oracle.integrand(1, u, T, tabs, T)
    c = oracle.integrand(1, u, T, tabs, T, alpha=n0)
    assert np.max(np.abs(c0)) > 1e-3
    assert np.max(np.abs(c)) <= 1e-15


def _q1_quadrature(oracle, tabs, t, alpha):
    """-2i int_0^t c_1(u) du by Gauss-Legendre on panels graded towards u = t."""
    x, w = np.polynomial.legendre.leggauss(20)
    edges = np.unique(np.concatenate([np.linspace(0.0, t - 4.0, 27), t - 4.0 + np.linspace(0.0, 4.0, 129)]))
    pts, wts = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        pts.append(0.5 * (b - a) * x + 0.5 * (a + b))
        wts.append(0.5 * (b - a) * w)
    pts, wts = np.concatenate(pts), np.concatenate(wts)
    c = oracle.integrand(1, pts.reshape(-1, 1), t, tabs, t, alpha=alpha)
    return float(np.sum(wts * (-2j * c).real))


@pytest.mark.parametrize("eps,gamma,alpha", [(0.0, 1.0, 0.3), (0.8, 1.0, -0.45), (-0.5, 0.7, 0.5)])
def test_alpha_moves_q1_by_the_static_charge_susceptibility(oracle, eps, gamma, alpha):
    """U (n_up - a)(n_down - a) = U n_up n_down - U a (n_up + n_down) + const: at first
    order in U the shift is a level shift eps_d -> eps_d - U a, so in the steady state
    Q_1(a) - Q_1(0) = -a dQ_0/d eps_d = 2 a / (pi Gamma (1 + (eps_d / Gamma)^2)) with
    Q_0 = 1 - 2 arctan(eps_d / Gamma) / pi.  At t = 30 / Gamma the transient is below 1e-6."""
    t = 30.0 / gamma
    tabs = oracle.gf_tables(gamma, eps, t, 65536)
    d = _q1_quadrature(oracle, tabs, t, alpha) - _q1_quadrature(oracle, tabs, t, 0.0)
    exact = 2.0 * alpha / (math.pi * gamma * (1.0 + (eps / gamma) ** 2))
    assert abs(d - exact) < 2e-5 * abs(exact), (d, exact)


def test_alpha_is_linear_in_the_keldysh_sum_at_order_one(oracle):
    """At order 1 the alpha^2 term of det M_up det M_down does not depend on the Keldysh
    index and cancels in the signed sum: c_1 is affine in alpha."""
    T = 10.0
    tabs = oracle.gf_tables(1.0, 0.3, T, 4096)
    u = np.linspace(0.05, T, 61).reshape(-1, 1)
    c = [oracle.integrand(1, u, T, tabs, T, alpha=a) for a in (0.0, 0.5, 1.0)]
    second = c[2] - 2.0 * c[1] + c[0]
    assert np.max(np.abs(second)) <= 1e-14 * np.max(np.abs(c[0]))


# ------------------------------------------------------------- GPU parity ---

@pytest.fixture(scope="module")
def Q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2002_12372_gb300 import build as b
    b.build()
    from paper_2002_12372_gb300 import qqmc
    qqmc.load()
    return qqmc


def _problem(Q, seed, T, alpha, L=4096):
    from paper_2002_12372_gb300 import workloads as W
    gl, gg, g0, _ = W.synthetic_tables(seed, L, T)
    p = Q.make_params(t_max=T, n_table=L, alpha=alpha)
    return Q.qqmc_create_problem_tables(p, gl, gg, g0), (gl, gg, g0)


@pytest.mark.gpu
@pytest.mark.parametrize("order,count", [(1, 64), (2, 64), (4, 32), (6, 16), (9, 6), (12, 2)])
def test_integrand_with_alpha_matches_oracle(Q, oracle, order, count):
    from paper_2002_12372_gb300 import workloads as W
    T, alpha = 10.0, 0.37
    pr, tabs = _problem(Q, 500 + order, T, alpha)
    try:
        u = W.ordered_times(600 + order, count, order, T)
        gpu = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_FP64)
        mixed = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_MIXED)
    finally:
        Q.qqmc_destroy_problem(pr)
    ref, scale = oracle.integrand(order, u, T, tabs, T, return_abs=True, alpha=alpha)
    assert np.all(np.abs(gpu - ref) <= 1e-12 * scale), np.max(np.abs(gpu - ref) / scale)
    assert np.all(np.abs(mixed - ref) <= 2.0 ** -20 * scale), np.max(np.abs(mixed - ref) / scale)


@pytest.mark.gpu
@pytest.mark.parametrize("lane", [False, True])
def test_integration_with_alpha_matches_oracle(Q, oracle, lane):
    """Both determinant kernels (cooperative warp and one point per lane) at alpha != 0."""
    from paper_2002_12372_gb300 import autotune
    from paper_2002_12372_gb300 import workloads as W
    T, K, alpha = 10.0, 3, -0.6
    pr, tabs = _problem(Q, 81, T, alpha)
    try:
        for n in range(1, 5):
            Q.qqmc_set_tuning(Q.QQMC_PREC_FP64, n, 2, 1 if lane else 2)
        for n, N in [(1, 2049), (3, 1000), (4, 777), (7, 200)]:
            sw = W.shift_words(700 + n, K, n)
            res, S = Q.qqmc_integrate(pr, n, N, K, Q.QQMC_PREC_FP64, sw)
            S0, nin = oracle.estimate(n, N, sw, T, 1.0, tabs, T, alpha=alpha)
            assert res.n_in_domain == int(nin.sum())
            assert np.all(np.abs(S - S0) <= 1e-10 * np.abs(S0)), (n, S, S0)
    finally:
        Q.qqmc_destroy_problem(pr)
        autotune.reset()


# ------------------------------------------------- alpha at the occupation ---
# alpha = Im g^<(0), the App. E choice that cancels the Hartree term, makes every vertex diagonal
# of M_down zero.  At particle-hole symmetry (eps_d = 0, alpha = 1/2) M_down is moreover skew-
# symmetric for every Keldysh index vector (g^>(tau) = conj g^<(tau)), so every odd leading minor
# vanishes and det M_down = 0 at odd orders: c_n = 0 there, and both sides return rounding.
# Bars per point: FP64 1e-12 sum_a |term_a| (the standard bar) plus 1e-14 times the summed
# Hadamard bounds of both determinants, which bound the rounding of a determinant that vanishes
# (n eps_64 < 1e-14 up to order 22); mixed precision 2^-20 (charge) or 2^-18 (current) of
# sum_a |term_a| plus 2^-20 of the Hadamard sum (n eps_32 < 2^-20 up to order 12).

OFFSETS = [0.0, 1e-6, -1e-6, 1e-3, -1e-3]


def _check_point_bars(gpu, mixed, ref, scale, had, mixed_rel=2.0 ** -20):
    assert np.all(np.isfinite(gpu)) and np.all(np.isfinite(mixed))
    dev = np.abs(gpu - ref)
    assert np.all(dev <= 1e-12 * scale + 1e-14 * had), np.max(dev / (scale + had))
    dm = np.abs(mixed - ref)
    assert np.all(dm <= mixed_rel * scale + 2.0 ** -20 * had), np.max(dm / (scale + had))


@pytest.mark.gpu
@pytest.mark.parametrize("order,count", [(1, 64), (2, 64), (3, 48), (4, 32), (5, 24), (6, 16), (7, 12), (8, 8),
                                         (9, 6), (10, 4), (12, 2)])
def test_integrand_at_the_occupation_matches_oracle(Q, oracle, order, count):
    from paper_2002_12372_gb300 import workloads as W
    T = 10.0
    gl, gg, g0, _ = W.synthetic_tables(500 + order, 4096, T)
    u = W.ordered_times(600 + order, count, order, T)
    for off in OFFSETS:
        alpha = float(np.imag(g0)) + off
        pr = Q.qqmc_create_problem_tables(Q.make_params(t_max=T, n_table=4096, alpha=alpha), gl, gg, g0)
        try:
            gpu = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_FP64)
            mixed = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_MIXED)
        finally:
            Q.qqmc_destroy_problem(pr)
        ref, scale, had = oracle.integrand(order, u, T, (gl, gg, g0), T, return_abs=True, return_had=True,
                                           alpha=alpha)
        _check_point_bars(gpu, mixed, ref, scale, had)
        if order == 1 and off == 0.0:  # the one-vertex det M_down is exactly zero
            assert np.all(gpu == 0.0) and np.all(mixed == 0.0)


@pytest.mark.gpu
@pytest.mark.parametrize("order,count", [(1, 32), (2, 32), (3, 32), (4, 24), (5, 16), (6, 12), (7, 8), (8, 6),
                                         (9, 4), (11, 2)])
def test_integrand_at_particle_hole_symmetry_matches_oracle(Q, oracle, order, count):
    """The wide-band dot at eps_d = 0 (tables from the oracle's closed form on both sides) with
    alpha = <n> = 1/2 and next to it."""
    from paper_2002_12372_gb300 import workloads as W
    T, L = 10.0, 4096
    gl, gg, g0 = oracle.gf_tables(1.0, 0.0, T, L)
    u = W.ordered_times(700 + order, count, order, T)
    for off in [0.0, 1e-6, -1e-3]:
        alpha = float(np.imag(g0)) + off
        pr = Q.qqmc_create_problem_tables(Q.make_params(t_max=T, n_table=L, alpha=alpha), gl, gg, g0)
        try:
            gpu = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_FP64)
            mixed = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_MIXED)
        finally:
            Q.qqmc_destroy_problem(pr)
        ref, scale, had = oracle.integrand(order, u, T, (gl, gg, g0), T, return_abs=True, return_had=True,
                                           alpha=alpha)
        _check_point_bars(gpu, mixed, ref, scale, had)


@pytest.mark.gpu
@pytest.mark.parametrize("order,count", [(1, 64), (2, 64), (3, 48), (5, 32), (7, 12), (10, 4)])
def test_current_integrand_at_the_occupation_matches_oracle(Q, oracle, order, count):
    from paper_2002_12372_gb300 import workloads as W
    T, L = 10.0, 4096
    gl, gg, g0, _ = W.synthetic_tables(800 + order, L, T)
    cl, cg, c0 = W.synthetic_column_tables(1800 + order, L, T)
    u = W.ordered_times(900 + order, count, order, T)
    for off in OFFSETS:
        alpha = float(np.imag(g0)) + off
        pr = Q.qqmc_create_problem_tables(Q.make_params(t_max=T, n_table=L, alpha=alpha), gl, gg, g0)
        try:
            Q.qqmc_set_current_tables(pr, cl, cg, c0)
            gpu = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_FP64)
            mixed = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_MIXED)
        finally:
            Q.qqmc_destroy_problem(pr)
        ref, scale, had = oracle.integrand(order, u, T, (gl, gg, g0), T, return_abs=True, return_had=True,
                                           alpha=alpha, col=(cl, cg, c0))
        _check_point_bars(gpu, mixed, ref, scale, had, mixed_rel=2.0 ** -18)


@pytest.mark.gpu
@pytest.mark.parametrize("lane", [False, True])
@pytest.mark.parametrize("off", [0.0, 1e-6, -1e-3])
@pytest.mark.parametrize("current", [False, True])
def test_integration_at_the_occupation_matches_oracle(Q, oracle, lane, off, current):
    """Per-shift sums at alpha = Im g^<(0) and next to it, with the cooperative warp kernel and the
    one-point-per-lane kernel (orders <= 4), for the charge and the current."""
    from paper_2002_12372_gb300 import autotune
    from paper_2002_12372_gb300 import workloads as W
    T, K, L = 10.0, 3, 4096
    gl, gg, g0, _ = W.synthetic_tables(81, L, T)
    col = W.synthetic_column_tables(1081, L, T) if current else None
    alpha = float(np.imag(g0)) + off
    pr = Q.qqmc_create_problem_tables(Q.make_params(t_max=T, n_table=L, alpha=alpha), gl, gg, g0)
    try:
        if current:
            Q.qqmc_set_current_tables(pr, *col)
        for n in range(1, 5):
            Q.qqmc_set_tuning(Q.QQMC_PREC_FP64, n, 2, 1 if lane else 2)
        for n, N in [(1, 2049), (2, 1000), (3, 1000), (4, 777), (7, 200), (10, 64)]:
            sw = W.shift_words(700 + n, K, n)
            res, S = Q.qqmc_integrate(pr, n, N, K, Q.QQMC_PREC_FP64, sw)
            S0, nin = oracle.estimate(n, N, sw, T, 1.0, (gl, gg, g0), T, alpha=alpha, col=col)
            assert res.n_in_domain == int(nin.sum())
            assert np.all(np.isfinite(S))
            assert np.all(np.abs(S - S0) <= 1e-10 * np.abs(S0)), (n, S, S0)
    finally:
        Q.qqmc_destroy_problem(pr)
        autotune.reset()


@pytest.mark.gpu
@pytest.mark.parametrize("ph", [False, True])
@pytest.mark.parametrize("order,count", [(3, 32), (4, 24), (5, 16), (7, 8), (9, 4)])
def test_single_vertex_tree_at_the_auto_threshold(Q, oracle, ph, order, count):
    """QQMC_ELIM_AUTO keeps the single-vertex tree while |g^<(0) - i alpha| is at least 0.01
    (FP64) or 0.25 (mixed) of max(|g^<(0)|, |g^>(0)|).  Just above those thresholds, where its
    first pivot (and at particle-hole symmetry every odd pivot) is that small, it still holds the
    bars: synthetic tables, and the wide-band dot at eps_d = 0."""
    from paper_2002_12372_gb300 import workloads as W
    T, L = 10.0, 4096
    if ph:
        gl, gg, g0 = oracle.gf_tables(1.0, 0.0, T, L)
    else:
        gl, gg, g0, _ = W.synthetic_tables(950 + order, L, T)
    u = W.ordered_times(960 + order, count, order, T)
    scale = max(abs(g0), abs(g0 - 1j))
    for prec, frac, rel in [(Q.QQMC_PREC_FP64, 0.01, 1e-12), (Q.QQMC_PREC_MIXED, 0.25, 2.0 ** -20)]:
        alpha = float(np.imag(g0)) + 1.02 * frac * scale
        pr = Q.qqmc_create_problem_tables(Q.make_params(t_max=T, n_table=L, alpha=alpha), gl, gg, g0)
        try:
            assert Q.qqmc_elimination(pr, prec) == Q.QQMC_ELIM_SINGLE
            got = Q.qqmc_integrand(pr, order, u, prec)
        finally:
            Q.qqmc_destroy_problem(pr)
        ref, sc, had = oracle.integrand(order, u, T, (gl, gg, g0), T, return_abs=True, return_had=True,
                                        alpha=alpha)
        floor = 1e-14 if prec == Q.QQMC_PREC_FP64 else 2.0 ** -20
        dev = np.abs(got - ref)
        assert np.all(np.isfinite(got))
        assert np.all(dev <= rel * sc + floor * had), (prec, np.max(dev / sc))


@pytest.mark.gpu
def test_auto_elimination_picks_pairs_near_the_occupation(Q):
    """The auto rule itself: pairs within the thresholds, single vertices outside them."""
    from paper_2002_12372_gb300 import workloads as W
    gl, gg, g0, _ = W.synthetic_tables(5, 256, 10.0)
    scale = max(abs(g0), abs(g0 - 1j))
    for prec, frac in [(Q.QQMC_PREC_FP64, 0.01), (Q.QQMC_PREC_MIXED, 0.25)]:
        for off, want in [(0.0, Q.QQMC_ELIM_PAIRS), (0.98 * frac * scale, Q.QQMC_ELIM_PAIRS),
                          (-0.98 * frac * scale, Q.QQMC_ELIM_PAIRS), (1.02 * frac * scale, Q.QQMC_ELIM_SINGLE)]:
            pr = Q.qqmc_create_problem_tables(
                Q.make_params(t_max=10.0, n_table=256, alpha=float(np.imag(g0)) + off), gl, gg, g0)
            try:
                assert Q.qqmc_elimination(pr, prec) == want, (prec, off)
                Q.qqmc_set_elimination(pr, Q.QQMC_ELIM_SINGLE)
                assert Q.qqmc_elimination(pr, prec) == Q.QQMC_ELIM_SINGLE
                Q.qqmc_set_elimination(pr, Q.QQMC_ELIM_PAIRS)
                assert Q.qqmc_elimination(pr, prec) == Q.QQMC_ELIM_PAIRS
            finally:
                Q.qqmc_destroy_problem(pr)


# -------------------------------------------------- the oracle's rounding scale ---

def test_hadamard_scale_bounds_every_keldysh_term(oracle):
    """Hadamard's inequality |det A| <= prod_rows ||row|| holds for each of the two determinants, so
    the summed bounds dominate sum_a |term_a|; every bound is homogeneous of degree 2n + 1 in the
    Green functions (n + 1 rows of M_up, n of M_down, one factor each)."""
    from paper_2002_12372_gb300 import workloads as W
    T = 10.0
    gl, gg, g0, _ = W.synthetic_tables(5, 512, T)
    for n in (1, 2, 3, 5):
        u = W.ordered_times(40 + n, 16, n, T)
        _, scale, had = oracle.integrand(n, u, T, (gl, gg, g0), T, return_abs=True, return_had=True, alpha=0.2)
        assert np.all(had >= scale) and np.all(had > 0.0)
        lam = 1.7
        _, had2 = oracle.integrand(n, u, T, (lam * gl, lam * gg, lam * g0), T, return_had=True, alpha=lam * 0.2)
        assert np.allclose(had2, lam ** (2 * n + 1) * had, rtol=1e-12)
    # one vertex at alpha = Im g^<(0): M_down = (0), so both its bound and the term vanish
    u = W.ordered_times(49, 8, 1, T)
    c, scale, had = oracle.integrand(1, u, T, (gl, gg, g0), T, return_abs=True, return_had=True,
                                     alpha=float(np.imag(g0)))
    assert np.all(had == 0.0) and np.all(scale == 0.0) and np.all(c == 0.0)
