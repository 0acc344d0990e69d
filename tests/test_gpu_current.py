"""Current observable and finite-bandwidth leads on the CUDA path, against the oracle.

* Lead tables: the device quadrature (composite Gauss-Legendre in w = D sin theta)
  against the oracle's adaptive quadrature at sampled nodes.
* Integrand and integration with the measurement column on lead site 1: byte-
  identical synthetic tables on both sides, both determinant kernels, FP64 and mixed.
* End to end from physical parameters: each side builds its own tables.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def W():
    from paper_2002_12372_gb300 import workloads
    return workloads


@pytest.mark.parametrize("gam,Ed,D,V,T,L", [(1.0, 0.3, 10.0, 0.6, 15.0, 1024), (0.1, 0.09, 2.0, 0.6 / 7, 100.0, 4096),
                                           (1.0, -0.8, 6.0, 0.0, 8.0, 512), (0.5, 0.2, 3.0, 7.0, 10.0, 256)])
def test_lead_tables_match_oracle(Q, oracle, gam, Ed, D, V, T, L):
    p = Q.make_params(gamma=gam, eps_d=Ed, t_max=T, n_table=L, observable=Q.QQMC_OBS_CURRENT, half_bandwidth=D,
                      bias=V)
    pr = Q.qqmc_create_problem(p)
    try:
        gl, gg, g0 = Q.qqmc_problem_tables(pr, L)
        cl, cg, c0 = Q.qqmc_problem_current_tables(pr, L)
    finally:
        Q.qqmc_destroy_problem(pr)
    nodes = oracle.table_nodes(T, L)
    rng = np.random.default_rng(L)
    k_dot = np.concatenate([[L // 2 - 1, L // 2, L - 1], rng.integers(L // 2, L, 29)])
    k_col = np.concatenate([[0, L // 2 - 1, L // 2], rng.integers(0, L // 2, 29)])
    F = oracle.lead_functions(np.concatenate([nodes[k_dot], nodes[k_col], [0.0]]), gam, Ed, D, V)
    m = k_dot.size
    assert np.max(np.abs(gl[k_dot] - F[0, :m])) < 1e-12
    assert np.max(np.abs(gg[k_dot] - F[1, :m])) < 1e-12
    assert np.max(np.abs(cl[k_col] - F[2, m:2 * m])) < 1e-12
    assert np.max(np.abs(cg[k_col] - F[3, m:2 * m])) < 1e-12
    assert abs(g0 - F[0, -1]) < 1e-12 and abs(c0 - F[2, -1]) < 1e-12


def _current_problem(Q, W, seed, T, L=4096, alpha=0.0):
    gl, gg, g0, _ = W.synthetic_tables(seed, L, T)
    cl, cg, c0 = W.synthetic_column_tables(seed + 1000, L, T)
    pr = Q.qqmc_create_problem_tables(Q.make_params(t_max=T, n_table=L, alpha=alpha), gl, gg, g0)
    Q.qqmc_set_current_tables(pr, cl, cg, c0)
    return pr, (gl, gg, g0), (cl, cg, c0)


@pytest.mark.parametrize("order,count", [(1, 64), (2, 64), (3, 48), (5, 32), (7, 12), (10, 4), (12, 2)])
def test_current_integrand_matches_oracle(Q, W, oracle, order, count):
    T = 10.0
    pr, tabs, col = _current_problem(Q, W, 800 + order, T, alpha=0.21)
    try:
        u = W.ordered_times(900 + order, count, order, T)
        gpu = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_FP64)
        mixed = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_MIXED)
    finally:
        Q.qqmc_destroy_problem(pr)
    ref, scale = oracle.integrand(order, u, T, tabs, T, return_abs=True, alpha=0.21, col=col)
    assert np.all(np.abs(gpu - ref) <= 1e-12 * scale), np.max(np.abs(gpu - ref) / scale)
    # FP32: 2^-18 of the Keldysh-sum scale.  Inside det M_up the measurement-pair product d dv and
    # the column products r_a c_a cancel partially (up to 4.5x at order 1 on these inputs), which
    # sum_a |term_a| does not see; the charge column (g_00 itself) stays within 2^-20.
    assert np.all(np.abs(mixed - ref) <= 2.0 ** -18 * scale), np.max(np.abs(mixed - ref) / scale)


@pytest.mark.parametrize("lane", [False, True])
def test_current_integration_matches_oracle(Q, W, oracle, lane):
    from paper_2002_12372_gb300 import autotune
    T, K = 10.0, 3
    pr, tabs, col = _current_problem(Q, W, 91, T)
    try:
        for n in range(1, 5):
            Q.qqmc_set_tuning(Q.QQMC_PREC_FP64, n, 2, 1 if lane else 2)
        for n, N in [(1, 2049), (2, 1000), (4, 777), (6, 300), (9, 64)]:
            sw = W.shift_words(1100 + n, K, n)
            res, S = Q.qqmc_integrate(pr, n, N, K, Q.QQMC_PREC_FP64, sw)
            S0, nin = oracle.estimate(n, N, sw, T, 1.0, tabs, T, col=col)
            assert res.n_in_domain == int(nin.sum())
            assert np.all(np.abs(S - S0) <= 1e-10 * np.abs(S0)), (n, S, S0)
            I0 = oracle.i_from_sums(S0)
            assert res.q_mean == pytest.approx(np.mean(I0), rel=1e-10, abs=1e-14)
    finally:
        Q.qqmc_destroy_problem(pr)
        autotune.reset()


def test_current_from_physical_parameters_end_to_end(Q, W, oracle):
    """Semicircular leads under bias with alpha: the device builds its tables, the oracle
    its own; I_n per shift agree to the table difference (1e-12) propagated (1e-9)."""
    gam, Ed, D, V, T, L, alpha = 1.0, 0.3, 10.0, 0.6, 8.0, 2048, 0.25
    p = Q.make_params(gamma=gam, eps_d=Ed, t_max=T, tau=1.5, n_table=L, observable=Q.QQMC_OBS_CURRENT,
                      half_bandwidth=D, bias=V, alpha=alpha)
    pr = Q.qqmc_create_problem(p)
    tabs, col = oracle.lead_tables(gam, Ed, D, V, T, L)
    try:
        for n, N in [(1, 4096), (3, 1024), (5, 256)]:
            sw = W.shift_words(1200 + n, 4, n)
            res, S = Q.qqmc_integrate(pr, n, N, 4, Q.QQMC_PREC_FP64, sw)
            S0, nin = oracle.estimate(n, N, sw, T, 1.5, tabs, T, alpha=alpha, col=col)
            assert res.n_in_domain == int(nin.sum())
            assert np.all(np.abs(S - S0) <= 1e-9 * np.max(np.abs(S0))), (n, S, S0)
    finally:
        Q.qqmc_destroy_problem(pr)


def test_served_current_series(Q, oracle):
    """A served current request: q[0] is the Landauer current, q[n] the direct integration."""
    import time
    p = Q.make_params(gamma=1.0, eps_d=0.3, t_max=8.0, tau=1.5, n_table=1024, observable=Q.QQMC_OBS_CURRENT,
                      half_bandwidth=10.0, bias=0.6)
    r = Q.qqmc_request()
    r.params = p
    r.n_max = 3
    r.n_shifts = 3
    r.n_points = 2048
    r.U = 0.5
    srv = Q.qqmc_server_create(Q.qqmc_server_opts(device_memory_limit=1 << 30, precision=0))
    try:
        h = Q.qqmc_submit(srv, r)
        t0 = time.time()
        while True:
            rc, out = Q.qqmc_poll(srv, h)
            if rc != Q.QQMC_PENDING:
                break
            assert time.time() - t0 < 120
            time.sleep(0.002)
    finally:
        Q.qqmc_server_destroy(srv)
    assert rc == Q.QQMC_OK
    assert out.q[0] == pytest.approx(oracle.landauer_current(1.0, 0.3, 10.0, 0.6), rel=1e-11)
    pr = Q.qqmc_create_problem(p)
    try:
        for n in range(1, 4):
            res, _ = Q.qqmc_integrate(pr, n, 2048, 3, 0, None)
            assert res.q_mean == out.q[n]
    finally:
        Q.qqmc_destroy_problem(pr)
