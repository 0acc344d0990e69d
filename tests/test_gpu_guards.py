"""Non-finite integrand sums are reported, never returned as valid coefficients.

Every work unit flags a partial sum that is NaN or infinite, the reduction
counts the flagged units per shift, and the host returns QQMC_E_NONFINITE
(results still filled; qqmc_result.n_nonfinite holds the count) from
qqmc_integrate, qqmc_plan_results and, per request, from the server.  The
NaN is planted in a caller table on the host: the kernels read it as data,
nothing faults on the device.
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


def _problems(Q, T=10.0, L=4096):
    from paper_2002_12372_gb300 import workloads as W
    gl, gg, g0, _ = W.synthetic_tables(3, L, T)
    bad = gl.copy()
    bad[L // 2 + L // 8] = np.nan  # tau ~ T / 4: read by most points
    p = Q.make_params(t_max=T, n_table=L)
    return Q.qqmc_create_problem_tables(p, gl, gg, g0), Q.qqmc_create_problem_tables(p, bad, gg, g0)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("lane", [False, True])
def test_nan_in_a_table_is_reported(Q, precision, lane):
    from paper_2002_12372_gb300 import autotune
    from paper_2002_12372_gb300 import workloads as W
    ok, bad = _problems(Q)
    try:
        for n in range(1, 5):
            Q.qqmc_set_tuning(precision, n, 2, 1 if lane else 2)
        for order in (1, 3, 7):
            sw = W.shift_words(40 + order, 2, order)
            with pytest.raises(Q.QQMCError) as e:
                Q.qqmc_integrate(bad, order, 1000, 2, precision, sw)
            assert e.value.code == Q.QQMC_E_NONFINITE
            res, S = Q.qqmc_integrate(ok, order, 1000, 2, precision, sw)
            assert res.n_nonfinite == 0 and np.all(np.isfinite(S))
            # one plan holding a clean and a poisoned item: only the poisoned one is flagged
            plan = Q.Plan([(ok, order, 2, 1000, sw), (bad, order, 2, 1000, sw)], precision)
            try:
                plan.launch()
                with pytest.raises(Q.QQMCError) as e:
                    plan.results()
                assert e.value.code == Q.QQMC_E_NONFINITE
                (r0, S0), (r1, S1) = plan.results(check=False)
                assert r0.n_nonfinite == 0 and np.all(np.isfinite(S0))
                assert np.array_equal(S0, S)  # the clean item is unaffected, bit for bit
                assert r1.n_nonfinite > 0 and not np.all(np.isfinite(S1))
            finally:
                plan.close()
    finally:
        Q.qqmc_destroy_problem(ok)
        Q.qqmc_destroy_problem(bad)
        autotune.reset()
