"""Learned warp on the GPU against the oracle (identical seeded inputs)."""
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


def _problem(Q, W, seed, T=10.0, L=4096):
    gl, gg, g0, _ = W.synthetic_tables(seed, L, T)
    return Q.qqmc_create_problem_tables(Q.make_params(t_max=T, n_table=L), gl, gg, g0), (gl, gg, g0)


@pytest.mark.parametrize("order,N,lane", [(2, 3000, True), (3, 2049, False), (5, 1000, False), (7, 300, False)])
def test_installed_table_integration_matches_oracle(Q, W, oracle, order, N, lane):
    from paper_2002_12372_gb300 import autotune
    T, K = 10.0, 3
    pr, tabs = _problem(Q, W, 81 + order, T)
    cdf = W.synthetic_projection(order, order, 512)
    sw = W.shift_words(4000 + order, K, order)
    try:
        if lane:
            Q.qqmc_set_tuning(0, order, 2, 1)
        Q.qqmc_set_projection(pr, order, cdf)
        res, S = Q.qqmc_integrate(pr, order, N, K, Q.QQMC_PREC_FP64, sw)
        res32, S32 = Q.qqmc_integrate(pr, order, N, K, Q.QQMC_PREC_MIXED, sw)
        S0, nin = oracle.estimate_proj(order, N, sw, T, 1.0, cdf, tabs, T)
        assert res.n_in_domain == int(nin.sum())
        assert np.all(np.abs(S - S0) <= 1e-10 * np.abs(S0))
        assert np.all(np.abs(S32 - S0) <= 1e-4 * np.abs(S0))
        # removing the table restores the plain warp
        Q.qqmc_set_projection(pr, order, None)
        resp, Sp = Q.qqmc_integrate(pr, order, N, K, Q.QQMC_PREC_FP64, sw)
        S0p, _ = oracle.estimate(order, N, sw, T, 1.0, tabs, T)
        assert np.all(np.abs(Sp - S0p) <= 1e-10 * np.abs(S0p))
    finally:
        Q.qqmc_destroy_problem(pr)
        autotune.reset()


@pytest.mark.parametrize("order", [1, 4, 6])
def test_learned_tables_match_oracle_learning(Q, W, oracle, order):
    T = 10.0
    pr, tabs = _problem(Q, W, 91 + order, T)
    try:
        cdf = Q.qqmc_learn_projection(pr, order, M=8000, n_bins=100, lam=0.05, floor_frac=1e-3, cells=512)
        ref = oracle.learn_projection(order, 8000, 2002123720, T, 1.0, tabs, T, n_bins=100, lam=0.05,
                                      floor_frac=1e-3, cells=512)
        assert np.max(np.abs(cdf - ref)) < 1e-10
        # the installed learned table drives the next integration; the oracle integrates with
        # its own learned table (the two agree to < 1e-10, see above)
        sw = W.shift_words(17, 2, order)
        res, S = Q.qqmc_integrate(pr, order, 512, 2, Q.QQMC_PREC_FP64, sw)
        S0, _ = oracle.estimate_proj(order, 512, sw, T, 1.0, ref, tabs, T)
        assert np.all(np.abs(S - S0) <= 1e-8 * np.abs(S0))
    finally:
        Q.qqmc_destroy_problem(pr)
