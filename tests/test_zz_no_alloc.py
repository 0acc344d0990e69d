"""The allocation-free entry point against the regular one.

qqmc_integrate_noalloc serves callers that cannot allocate device memory
where they integrate (a framework that owns the device through its own pool,
a real-time loop that must stay out of the allocator).  It takes device
buffers from the caller and keeps its scratch in a static array inside the
library.  Two calls in a row must each reproduce qqmc_integrate within the
FP64 tolerance of the parity tests (relative 1e-10 per shift); the second
call also checks that the scratch left behind by the first does not leak in.
The mixed precision, in-domain counts left in the library's scratch
(d_counts = NULL) and a high FP64 order (its whole tree stack in shared
memory) are covered too.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_integrate_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2002_12372_gb300 import build as b
    b.build()
    from paper_2002_12372_gb300 import qqmc as Q
    from paper_2002_12372_gb300 import workloads as W

    torch.cuda.set_device(0)
    T, L = 10.0, 4096
    gl, gg, g0, _ = W.synthetic_tables(31, L, T)
    pr = Q.qqmc_create_problem_tables(Q.make_params(t_max=T, n_table=L), gl, gg, g0)
    try:
        for order, N, K in [(5, 3000, 4), (3, 777, 3)]:
            sw = W.shift_words(500 + order, K, order)
            res, S_ref = Q.qqmc_integrate(pr, order, N, K, Q.QQMC_PREC_FP64, sw)
            d_sw = torch.from_numpy(sw.view(np.int32).copy()).cuda()
            d_sums = torch.full((K, 2), float("nan"), dtype=torch.float64, device="cuda")
            d_counts = torch.zeros(K, dtype=torch.int64, device="cuda")
            stream = torch.cuda.current_stream().cuda_stream
            Q.qqmc_integrate_noalloc(pr, order, N, K, Q.QQMC_PREC_FP64, d_sw.data_ptr(), d_sums.data_ptr(),
                                     d_counts.data_ptr(), stream)
            torch.cuda.synchronize()
            S = (d_sums[:, 0] + 1j * d_sums[:, 1]).cpu().numpy() / N
            assert np.all(np.abs(S - S_ref) <= 1e-10 * np.abs(S_ref)), (S, S_ref)
            assert int(d_counts.sum().item()) == res.n_in_domain
    finally:
        Q.qqmc_destroy_problem(pr)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2002_12372_gb300 import qqmc as Q
    from paper_2002_12372_gb300 import workloads as W

    gl, gg, g0, _ = W.synthetic_tables(31, 64, 10.0)
    pr = Q.qqmc_create_problem_tables(Q.make_params(t_max=10.0, n_table=64), gl, gg, g0)
    try:
        d = torch.zeros(64, dtype=torch.float64, device="cuda")
        with pytest.raises(Q.QQMCError) as e:
            Q.qqmc_integrate_noalloc(pr, 3, 2 ** 24, 1024, Q.QQMC_PREC_FP64, d.data_ptr(), d.data_ptr())
        assert e.value.code == Q.QQMC_E_INVAL
        assert "static scratch" in str(e.value)
    finally:
        Q.qqmc_destroy_problem(pr)


def test_noalloc_mixed_high_order_and_internal_counts():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2002_12372_gb300 import qqmc as Q
    from paper_2002_12372_gb300 import workloads as W

    torch.cuda.set_device(0)
    T, L = 10.0, 4096
    gl, gg, g0, _ = W.synthetic_tables(33, L, T)
    pr = Q.qqmc_create_problem_tables(Q.make_params(t_max=T, n_table=L), gl, gg, g0)
    stream = torch.cuda.current_stream().cuda_stream
    try:
        # (order, N, K, precision): the same per-point arithmetic as qqmc_integrate, whose plan may
        # cut the items into finer work units (a different grouping of the FP64 sums), so the
        # parity tests' relative 1e-10 per shift; order 14 in FP64 runs with its whole tree stack
        # in shared memory, where qqmc_integrate keeps the wide levels in device memory
        for order, N, K, prec in [(6, 2000, 3, Q.QQMC_PREC_MIXED), (9, 512, 2, Q.QQMC_PREC_MIXED),
                                  (14, 256, 2, Q.QQMC_PREC_FP64)]:
            sw = W.shift_words(900 + order, K, order)
            res, S_ref = Q.qqmc_integrate(pr, order, N, K, prec, sw)
            d_sw = torch.from_numpy(sw.view(np.int32).copy()).cuda()
            for _ in range(2):
                d_sums = torch.full((K, 2), float("nan"), dtype=torch.float64, device="cuda")
                Q.qqmc_integrate_noalloc(pr, order, N, K, prec, d_sw.data_ptr(), d_sums.data_ptr(), None, stream)
                torch.cuda.synchronize()
                S = (d_sums[:, 0] + 1j * d_sums[:, 1]).cpu().numpy() / N
                assert np.all(np.abs(S - S_ref) <= 1e-10 * np.abs(S_ref)), (order, S, S_ref)
                assert res.n_in_domain > 0
    finally:
        Q.qqmc_destroy_problem(pr)
