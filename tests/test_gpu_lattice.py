"""Rank-1 lattice point set on the CUDA path against the oracle: point words and
warp bit-exact, integrations in both determinant kernels, mixed-precision bound,
and the lattice bounds."""
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


M = 16


def _korobov(a: int, dims: int) -> np.ndarray:
    """Test generating vector (1, a, a^2, ...) mod 2^M: a fixed input both sides receive."""
    return np.array([pow(a, d, 1 << M) for d in range(dims)], dtype=np.uint32)


def _lattice_problem(Q, W, oracle, seed, T=10.0, L=4096, dims=12, bakers=False):
    gl, gg, g0, _ = W.synthetic_tables(seed, L, T)
    pr = Q.qqmc_create_problem_tables(Q.make_params(t_max=T, n_table=L), gl, gg, g0)
    z = _korobov(17797, dims)
    Q.qqmc_set_lattice(pr, M, z, bakers)
    return pr, (gl, gg, g0), z


@pytest.mark.parametrize("order,bakers", [(1, False), (4, False), (9, False), (12, False), (3, True), (10, True)])
def test_lattice_warp_points_match_oracle(Q, W, oracle, order, bakers):
    T = 10.0
    pr, _, z = _lattice_problem(Q, W, oracle, 40 + order, T=T, bakers=bakers)
    try:
        sh = W.shift_words(41 + order, 1, order)[0]
        u, w, ins = Q.qqmc_warp_points(pr, order, 1000, 20000, sh)
    finally:
        Q.qqmc_destroy_problem(pr)
    u0, w0, ins0 = oracle.warp(order, 1000, 20000, None, sh, T, 1.0, lattice=(z, M, bakers))
    assert np.array_equal(ins, ins0)
    assert np.max(np.abs(u - u0)) <= 1e-13 * T
    assert np.max(np.abs(w / w0 - 1.0)) < 1e-13


@pytest.mark.parametrize("lane,bakers", [(False, False), (True, False), (False, True)])
def test_lattice_integration_matches_oracle(Q, W, oracle, lane, bakers):
    from paper_2002_12372_gb300 import autotune
    T, K = 10.0, 3
    pr, tabs, z = _lattice_problem(Q, W, oracle, 51, T=T, bakers=bakers)
    try:
        for n in range(1, 5):
            Q.qqmc_set_tuning(Q.QQMC_PREC_FP64, n, 2, 1 if lane else 2)
        for n, N, first in [(1, 4096, 0), (3, 2049, 100), (4, 1000, 0), (7, 300, 65000), (10, 64, 0)]:
            sw = W.shift_words(1300 + n, K, n)
            plan = Q.Plan([(pr, n, K, N, sw, first)], Q.QQMC_PREC_FP64)
            plan.launch()
            (res, S), = plan.results()
            plan.close()
            S0, nin = oracle.estimate(n, N, sw, T, 1.0, tabs, T, i0=first, lattice=(z, M, bakers))
            assert res.n_in_domain == int(nin.sum())
            assert np.all(np.abs(S - S0) <= 1e-10 * np.abs(S0)), (n, S, S0)
    finally:
        Q.qqmc_destroy_problem(pr)
        autotune.reset()


def test_lattice_mixed_within_bound_of_fp64(Q, W, oracle):
    T, K, n, N = 10.0, 4, 6, 4096
    pr, _, _ = _lattice_problem(Q, W, oracle, 61, T=T)
    try:
        sw = W.shift_words(1400, K, n)
        r64, S64 = Q.qqmc_integrate(pr, n, N, K, Q.QQMC_PREC_FP64, sw)
        r32, S32 = Q.qqmc_integrate(pr, n, N, K, Q.QQMC_PREC_MIXED, sw)
    finally:
        Q.qqmc_destroy_problem(pr)
    assert r32.n_in_domain == r64.n_in_domain
    assert abs(r32.q_mean - r64.q_mean) < 0.05 * r64.q_err


def test_items_outside_the_lattice_are_rejected(Q, W, oracle):
    pr, _, _ = _lattice_problem(Q, W, oracle, 71, dims=4)
    try:
        with pytest.raises(Q.QQMCError) as e:
            Q.qqmc_integrate(pr, 5, 64, 2, 0, None)  # order above the lattice dimension
        assert e.value.code == Q.QQMC_E_INVAL
        with pytest.raises(Q.QQMCError) as e:
            Q.Plan([(pr, 3, 2, 100, W.shift_words(1, 2, 3), (1 << M) - 50)], Q.QQMC_PREC_FP64)
        assert e.value.code == Q.QQMC_E_INVAL
        Q.qqmc_set_lattice(pr, M, None)  # back to Sobol'
        res, _ = Q.qqmc_integrate(pr, 5, 64, 2, 0, None)
        assert res.n_points == 64
    finally:
        Q.qqmc_destroy_problem(pr)
