"""Serving loop: continuous batching gives each request the same result alone
and in a mix, and the host-side failure paths report their error codes.

Failures are made on the host (a cancelled request, a full queue, a request
that times out in the queue, malformed parameters); nothing here faults or
hangs the GPU.
"""
import time

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
    torch.cuda.set_device(0)
    return qqmc


def _req(Q, eps, t, n_max, N, U=2.0, K=4):
    r = Q.qqmc_request()
    r.params = Q.make_params(eps_d=eps, t_max=t, n_table=1024)
    r.n_max = n_max
    r.n_shifts = K
    r.n_points = N
    r.U = U
    return r


def _wait(Q, srv, h, timeout=120.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        rc, out = Q.qqmc_poll(srv, h)
        if rc != Q.QQMC_PENDING:
            return rc, out
        time.sleep(0.002)
    raise AssertionError("request did not complete")


@pytest.mark.parametrize("precision", [0, 1])
def test_each_result_is_the_same_alone_and_in_the_mix(Q, precision):
    reqs = [(-2.0, 5.0, 4, 3000), (0.5, 10.0, 6, 1000), (2.5, 20.0, 3, 5000), (0.0, 10.0, 5, 2048),
            (-0.7, 5.0, 7, 600)]
    opts = Q.qqmc_server_opts(device_memory_limit=1 << 30, max_queue=64, max_batch_items=64, precision=precision,
                              use_graph=0, request_timeout_s=0.0)
    srv = Q.qqmc_server_create(opts)
    try:
        alone = []
        for eps, t, nm, N in reqs:
            h = Q.qqmc_submit(srv, _req(Q, eps, t, nm, N))
            rc, out = _wait(Q, srv, h)
            assert rc == Q.QQMC_OK
            alone.append(out)
        hs = [Q.qqmc_submit(srv, _req(Q, eps, t, nm, N)) for eps, t, nm, N in reqs]
        mixed = [_wait(Q, srv, h) for h in hs]
    finally:
        Q.qqmc_server_destroy(srv)
    for (eps, t, nm, N), a, (rc, m) in zip(reqs, alone, mixed):
        assert rc == Q.QQMC_OK
        for n in range(nm + 1):
            assert a.q[n] == m.q[n], (n, a.q[n], m.q[n])
            assert a.q_err[n] == m.q_err[n]
        assert a.n_in_domain == m.n_in_domain
        assert a.series_sum == m.series_sum
        assert a.latency_ms > 0 and m.latency_ms > 0


def test_served_coefficients_equal_direct_integration(Q):
    opts = Q.qqmc_server_opts(device_memory_limit=1 << 30, precision=0)
    srv = Q.qqmc_server_create(opts)
    try:
        h = Q.qqmc_submit(srv, _req(Q, 0.3, 10.0, 4, 4096, U=1.5, K=3))
        rc, out = _wait(Q, srv, h)
    finally:
        Q.qqmc_server_destroy(srv)
    assert rc == Q.QQMC_OK
    pr = Q.qqmc_create_problem(Q.make_params(eps_d=0.3, t_max=10.0, n_table=1024))
    try:
        total = out.q[0]
        for n in range(1, 5):
            res, _ = Q.qqmc_integrate(pr, n, 4096, 3, 0, None)
            assert res.q_mean == out.q[n]
            assert res.q_err == out.q_err[n]
            total += res.q_mean * 1.5 ** n
    finally:
        Q.qqmc_destroy_problem(pr)
    assert out.series_sum == pytest.approx(total, rel=1e-14)
    assert out.q[0] == pytest.approx(1.0 - 2.0 * np.arctan(0.3) / np.pi, rel=1e-15)


def _wait_state(Q, srv, h, state, timeout=60.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        st = Q.qqmc_request_state(srv, h)
        if st == state:
            return
        assert st in (Q.QQMC_PENDING, Q.QQMC_RUNNING), st
        time.sleep(0.0005)
    raise AssertionError("request never reached state %d" % state)


@pytest.mark.parametrize("precision", [0, 1])
def test_rounds_admitted_while_another_runs_execute_with_it(Q, precision):
    """Continuous batching: a long request is admitted and running; requests submitted then are
    admitted in a later round, and that round's kernels execute on the device while the long
    round's are still running (their device-clock spans overlap).  Every result equals its
    alone result bit for bit."""
    short = [(-2.0, 5.0, 4, 3000), (0.5, 10.0, 6, 1000), (2.5, 20.0, 3, 5000), (0.0, 10.0, 5, 2048)]
    long_N = 2 ** 17 if precision == 0 else 2 ** 19
    opts = Q.qqmc_server_opts(device_memory_limit=1 << 30, max_queue=64, max_batch_items=64, precision=precision,
                              use_graph=0, request_timeout_s=0.0)
    srv = Q.qqmc_server_create(opts)
    try:
        alone = []
        for eps, t, nm, N in short:
            rc, out = _wait(Q, srv, Q.qqmc_submit(srv, _req(Q, eps, t, nm, N)))
            assert rc == Q.QQMC_OK
            alone.append(out)
        h_long = Q.qqmc_submit(srv, _req(Q, 0.2, 10.0, 10, long_N, K=16))
        _wait_state(Q, srv, h_long, Q.QQMC_RUNNING)
        hs = [Q.qqmc_submit(srv, _req(Q, eps, t, nm, N)) for eps, t, nm, N in short]
        mixed = [_wait(Q, srv, h) for h in hs]
        rcl, outl = _wait(Q, srv, h_long)
    finally:
        Q.qqmc_server_destroy(srv)
    assert rcl == Q.QQMC_OK
    assert outl.device_end_ns > outl.device_start_ns > 0
    overlapped = 0
    for (eps, t, nm, N), a, (rc, m) in zip(short, alone, mixed):
        assert rc == Q.QQMC_OK
        for n in range(nm + 1):
            assert a.q[n] == m.q[n], (n, a.q[n], m.q[n])
            assert a.q_err[n] == m.q_err[n]
        assert a.n_in_domain == m.n_in_domain
        assert a.series_sum == m.series_sum
        assert m.batch > outl.batch  # admitted in a later round than the running request
        overlapped += m.device_start_ns < outl.device_end_ns and m.device_end_ns > outl.device_start_ns
    assert overlapped >= 1, "no later round executed while the long round ran"


def test_served_series_matches_the_oracle(Q, oracle):
    """One served request against the oracle: each side builds its own tables (device contour
    quadrature, oracle closed form; 1e-13 apart), shift words from the request's seed."""
    eps, T, L, nm, N, K, U = 0.3, 10.0, 1024, 4, 4096, 3, 1.5
    srv = Q.qqmc_server_create(Q.qqmc_server_opts(device_memory_limit=1 << 30, precision=0))
    try:
        req = _req(Q, eps, T, nm, N, U=U, K=K)
        rc, out = _wait(Q, srv, Q.qqmc_submit(srv, req))
    finally:
        Q.qqmc_server_destroy(srv)
    assert rc == Q.QQMC_OK
    tabs = oracle.gf_tables(1.0, eps, T, L)
    total = out.q[0]
    for n in range(1, nm + 1):
        sw = oracle.shift_words(req.params.seed, K, n)
        S0, _ = oracle.estimate(n, N, sw, T, 1.0, tabs, T)
        q = oracle.q_from_sums(S0).real
        assert out.q[n] == pytest.approx(np.mean(q), rel=1e-9, abs=1e-13)
        assert out.q_err[n] == pytest.approx(np.std(q, ddof=1) / np.sqrt(K), rel=1e-7, abs=1e-13)
        total += out.q[n] * U ** n
    assert out.series_sum == pytest.approx(total, rel=1e-14)


def test_failure_paths_report_codes(Q):
    """Every host-side failure code, deterministically: a 1-byte memory budget holds the queue
    behind a running request and a queue of one makes the next submission E_BUSY."""
    srv = Q.qqmc_server_create(Q.qqmc_server_opts(device_memory_limit=1, precision=0, max_queue=1,
                                                  request_timeout_s=0.05))
    try:
        bad = _req(Q, 0.0, 10.0, Q.QQMC_MAX_ORDER + 1, 1024)
        with pytest.raises(Q.QQMCError) as e:
            Q.qqmc_submit(srv, bad)
        assert e.value.code == Q.QQMC_E_RANGE
        bad = _req(Q, 0.0, -1.0, 3, 1024)
        with pytest.raises(Q.QQMCError) as e:
            Q.qqmc_submit(srv, bad)
        assert e.value.code == Q.QQMC_E_INVAL
        rc, _ = Q.qqmc_poll(srv, 987654321)
        assert rc == Q.QQMC_E_NOTFOUND
        assert Q.qqmc_request_state(srv, 987654321) == Q.QQMC_E_NOTFOUND
        # a long request runs (~1 s); one request waits behind it and fills the queue
        h_long = Q.qqmc_submit(srv, _req(Q, 0.0, 10.0, 10, 2 ** 17, K=16))
        _wait_state(Q, srv, h_long, Q.QQMC_RUNNING)
        h1 = Q.qqmc_submit(srv, _req(Q, 0.1, 10.0, 3, 1024))
        with pytest.raises(Q.QQMCError) as e:
            Q.qqmc_submit(srv, _req(Q, 0.3, 10.0, 2, 64))
        assert e.value.code == Q.QQMC_E_BUSY
        # it cannot be admitted while the long one holds the budget: it times out in the queue
        rc1, out1 = _wait(Q, srv, h1)
        assert rc1 == Q.QQMC_E_TIMEOUT and out1.status == Q.QQMC_E_TIMEOUT
        assert Q.qqmc_request_state(srv, h_long) == Q.QQMC_RUNNING
        rcl, _ = _wait(Q, srv, h_long)
        assert rcl == Q.QQMC_OK
    finally:
        Q.qqmc_server_destroy(srv)
    # cancellation of a queued request
    srv = Q.qqmc_server_create(Q.qqmc_server_opts(device_memory_limit=1, precision=0))
    try:
        h_long = Q.qqmc_submit(srv, _req(Q, 0.0, 10.0, 10, 2 ** 17, K=16))
        _wait_state(Q, srv, h_long, Q.QQMC_RUNNING)
        h2 = Q.qqmc_submit(srv, _req(Q, 0.2, 10.0, 3, 1024))
        assert Q.qqmc_request_state(srv, h2) == Q.QQMC_PENDING
        Q.qqmc_cancel(srv, h2)
        rc2, out2 = _wait(Q, srv, h2)
        assert rc2 == Q.QQMC_E_CANCELLED
        assert _wait(Q, srv, h_long)[0] == Q.QQMC_OK
    finally:
        Q.qqmc_server_destroy(srv)


def test_destroy_cancels_pending_requests(Q):
    srv = Q.qqmc_server_create(Q.qqmc_server_opts(precision=0, device_memory_limit=1))
    hs = [Q.qqmc_submit(srv, _req(Q, 0.0, 10.0, 8, 2 ** 15, K=8)) for _ in range(3)]
    Q.qqmc_server_destroy(srv)  # returns after in-flight work; the rest is cancelled
    assert len(hs) == 3
