"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Inputs are seeded and shared byte for byte (``workloads``): synthetic
Keldysh tables, shift words, vertex times.  Bars:
  * integers (Sobol' words, in-domain counts): bit-exact;
  * FP64 integrand per point: |c_gpu - c_oracle| <= 1e-12 * sum_a |term_a|
    (the oracle's own scale of the Keldysh sum: both sides round at ~1e-16
    relative to the largest terms, times the O(2^n) additions);
  * FP64 coefficients per shift: relative 1e-10 (the stated target);
  * mixed precision: the bound stated in each test.
"""
import os

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


def _problem(Q, W, seed=7, T=10.0, L=4096, tau=1.0, elim=0):
    """elim: the Keldysh-sum tree (QQMC_ELIM_AUTO = 0, _PAIRS = 1, _SINGLE = 2)."""
    gl, gg, g0, _ = W.synthetic_tables(seed, L, T)
    p = Q.make_params(t_max=T, tau=tau, n_table=L)
    pr = Q.qqmc_create_problem_tables(p, gl, gg, g0)
    Q.qqmc_set_elimination(pr, elim)
    return pr, (gl, gg, g0)


TREES = [1, 2]  # both Keldysh-sum trees: vertex pairs, single vertices


# ------------------------------------------------------------------ points ---

@pytest.mark.parametrize("order", [1, 3, 7, 12])
def test_sobol_points_bit_exact(Q, W, oracle, order):
    V = oracle.sobol_direction_numbers(12)
    sh = W.shift_words(3, 1, order)[0]
    for first, count in [(0, 4096), (2 ** 20 - 5, 77), (3_000_001, 33)]:
        gpu = Q.qqmc_sobol_points(order, first, count, sh)
        ref = oracle.sobol_points(order, first, count, V) ^ sh[None, :order]
        assert np.array_equal(gpu, ref)


@pytest.mark.parametrize("order,tau,t", [(1, 1.0, 10.0), (4, 0.95, 10.0), (10, 1.0, 10.0), (12, 1.5, 5.0)])
def test_warp_points_match_oracle(Q, W, oracle, order, tau, t):
    pr, _ = _problem(Q, W, T=t, tau=tau)
    try:
        sh = W.shift_words(5, 1, order)[0]
        u, w, ins = Q.qqmc_warp_points(pr, order, 1000, 20000, sh)
    finally:
        Q.qqmc_destroy_problem(pr)
    V = oracle.sobol_direction_numbers(12)
    u0, w0, ins0 = oracle.warp(order, 1000, 20000, V, sh, t, tau)
    assert np.array_equal(ins, ins0)
    assert np.max(np.abs(u - u0)) <= 1e-13 * t
    assert np.max(np.abs(w / w0 - 1.0)) < 1e-13


# -------------------------------------------------------------- integrand ---

@pytest.mark.parametrize("elim", TREES)
@pytest.mark.parametrize("order,count", [(1, 64), (2, 64), (3, 64), (5, 48), (6, 32), (8, 16), (10, 6), (12, 2)])
def test_integrand_fp64_matches_oracle(Q, W, oracle, order, count, elim):
    T = 10.0
    pr, tabs = _problem(Q, W, seed=100 + order, T=T, elim=elim)
    try:
        u = W.ordered_times(200 + order, count, order, T)
        gpu = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_FP64)
    finally:
        Q.qqmc_destroy_problem(pr)
    ref, scale = oracle.integrand(order, u, T, tabs, T, return_abs=True)
    assert np.all(np.abs(gpu - ref) <= 1e-12 * scale), np.max(np.abs(gpu - ref) / scale)


@pytest.mark.parametrize("elim", TREES)
@pytest.mark.parametrize("order,count", [(2, 64), (5, 32), (6, 16), (7, 16), (8, 12), (10, 6), (12, 2)])
def test_integrand_mixed_within_fp32_bound(Q, W, oracle, order, count, elim):
    """FP32 Schur updates: deviation bounded by 2^-20 (~1e-6) of the Keldysh-sum scale.  With the
    single-vertex tree, orders >= 7 resolve their sibling leaves in one paired flat phase (two
    choice paths per lane), order 6 its lone leaf one path per lane."""
    T = 10.0
    pr, tabs = _problem(Q, W, seed=300 + order, T=T, elim=elim)
    try:
        u = W.ordered_times(400 + order, count, order, T)
        gpu = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_MIXED)
    finally:
        Q.qqmc_destroy_problem(pr)
    ref, scale = oracle.integrand(order, u, T, tabs, T, return_abs=True)
    assert np.all(np.abs(gpu - ref) <= 2.0 ** -20 * scale), np.max(np.abs(gpu - ref) / scale)


# ------------------------------------------------------------- integration ---

@pytest.mark.parametrize("elim", TREES)
@pytest.mark.parametrize("order,N,K", [(1, 4096, 4), (2, 1000, 3), (3, 2049, 3), (4, 4096, 2), (6, 517, 2),
                                       (8, 97, 2), (1, 1, 1), (2, 31, 2), (3, 33, 2)])
def test_integration_fp64_matches_oracle(Q, W, oracle, order, N, K, elim):
    T = 10.0
    pr, tabs = _problem(Q, W, seed=order, T=T, elim=elim)
    sw = W.shift_words(1000 + order, K, order)
    try:
        res, S = Q.qqmc_integrate(pr, order, N, K, Q.QQMC_PREC_FP64, sw)
    finally:
        Q.qqmc_destroy_problem(pr)
    S0, nin = oracle.estimate(order, N, sw, T, 1.0, tabs, T)
    assert res.n_in_domain == int(nin.sum())
    rel = np.abs(S - S0) / np.maximum(np.abs(S0), 1e-300)
    assert np.all(rel < 1e-10), rel
    q0 = oracle.q_from_sums(S0).real
    assert res.q_mean == pytest.approx(np.mean(q0), rel=1e-10, abs=1e-14)


def test_batched_plan_equals_single_runs(Q, W, oracle):
    """Uneven orders and point counts in one persistent launch: the same sums
    (bit-identical when every order runs the same kernel shape, as with the
    built-in tuning here; to rounding otherwise)."""
    T = 10.0
    pr, tabs = _problem(Q, W, seed=21, T=T)
    try:
        items = [(pr, n, 2, N, W.shift_words(50 + n, 2, n)) for n, N in [(2, 3000), (5, 700), (3, 1), (7, 64)]]
        plan = Q.Plan(items, Q.QQMC_PREC_FP64)
        plan.launch()
        batched = plan.results()
        plan.launch(use_graph=True)
        graphed = plan.results()
        plan.close()
        for (pr_, n, K, N, sw), (res, S), (res_g, S_g) in zip(items, batched, graphed):
            res1, S1 = Q.qqmc_integrate(pr, n, N, K, Q.QQMC_PREC_FP64, sw)
            assert np.array_equal(S, S1)
            assert np.array_equal(S_g, S1)
            assert res.n_in_domain == res1.n_in_domain
    finally:
        Q.qqmc_destroy_problem(pr)


# ------------------------------------------------------------------ tables ---

@pytest.mark.parametrize("eps,T", [(0.0, 10.0), (-1.0, 10.0), (1.0, 10.0), (2.5, 20.0)])
def test_gf_table_kernel_matches_oracle(Q, oracle, eps, T):
    L = 4096
    p = Q.make_params(eps_d=eps, t_max=T, n_table=L)
    pr = Q.qqmc_create_problem(p)
    try:
        gl, gg, g0 = Q.qqmc_problem_tables(pr, L)
    finally:
        Q.qqmc_destroy_problem(pr)
    rl, rg, r0 = oracle.gf_tables(1.0, eps, T, L)
    assert abs(g0 - r0) < 1e-15
    assert np.max(np.abs(gl - rl)) < 1e-13
    assert np.max(np.abs(gg - rg)) < 1e-13


# ------------------------------------------------- physics, end to end ---

def test_end_to_end_q_coefficients_match_oracle(Q, W, oracle):
    """Each side with its own tables (GPU contour quadrature vs oracle E1 closed
    form, agreeing to ~1e-14): Q_1..Q_4 at Gamma=1, eps_d=0, t=10, N=2^14, K=16."""
    T, L, K, N = 10.0, 4096, 16, 2 ** 14
    p = Q.make_params(eps_d=0.0, t_max=T, n_table=L)
    pr = Q.qqmc_create_problem(p)
    tabs = oracle.gf_tables(1.0, 0.0, T, L)
    try:
        for n in range(1, 5):
            sw = oracle.shift_words(2002123720, K, n)
            res, S = Q.qqmc_integrate(pr, n, N, K, Q.QQMC_PREC_FP64, None)
            S0, nin = oracle.estimate(n, N, sw, T, 1.0, tabs, T)
            assert res.n_in_domain == int(nin.sum())
            assert np.max(np.abs(S - S0) / np.abs(S0)) < 1e-9
    finally:
        Q.qqmc_destroy_problem(pr)


def test_single_level_flat_occupation_cancels_at_every_order(Q, W, oracle):
    """One Lorentzian level with a flat occupation is an infinite-temperature
    state: every interaction correction vanishes, on both sides, to roundoff."""
    T, L = 10.0, 4096
    gl, gg, g0, _ = W.synthetic_tables(9, L, T, components=1)
    p = Q.make_params(t_max=T, n_table=L)
    pr = Q.qqmc_create_problem_tables(p, gl, gg, g0)
    try:
        for n in (1, 2, 5):
            u = W.ordered_times(n, 16, n, T)
            c = Q.qqmc_integrand(pr, n, u, Q.QQMC_PREC_FP64)
            ref, scale = oracle.integrand(n, u, T, (gl, gg, g0), T, return_abs=True)
            assert np.all(np.abs(c) <= 1e-13 * scale)
            assert np.all(np.abs(ref) <= 1e-13 * scale)
    finally:
        Q.qqmc_destroy_problem(pr)


def test_one_long_shift_reduces_like_the_oracle(Q, W, oracle):
    """One shifted sequence of N = 2^20 points: 32768 chunk partials, 128 per thread of the
    reduction block, summed with two-sum per thread and across the block; the per-shift sum
    matches the oracle's (Neumaier per chunk, exactly rounded across chunks) to 1e-10."""
    T, order, N = 10.0, 2, 2 ** 20
    pr, tabs = _problem(Q, W, seed=17, T=T)
    try:
        sw = W.shift_words(19, 1, order)
        res, S = Q.qqmc_integrate(pr, order, N, 1, Q.QQMC_PREC_FP64, sw)
    finally:
        Q.qqmc_destroy_problem(pr)
    S0, nin = oracle.estimate(order, N, sw, T, 1.0, tabs, T)
    assert res.n_in_domain == int(nin.sum())
    assert np.all(np.abs(S - S0) <= 1e-10 * np.abs(S0)), (S, S0)


@pytest.mark.parametrize("order,N", [(3, 4096), (6, 2048), (9, 512)])
def test_integration_mixed_within_stated_bound_of_fp64(Q, W, oracle, order, N):
    """Mixed precision (FP32 tables and Schur updates, compensated FP32 leaf sums,
    FP64 point and shift sums) against the FP64 path on the same shifts:
    per-shift sums within 1e-4 relative, the shift mean within 5% of its error bar."""
    T, K = 10.0, 8
    pr, tabs = _problem(Q, W, seed=40 + order, T=T)
    sw = W.shift_words(2000 + order, K, order)
    try:
        r64, S64 = Q.qqmc_integrate(pr, order, N, K, Q.QQMC_PREC_FP64, sw)
        r32, S32 = Q.qqmc_integrate(pr, order, N, K, Q.QQMC_PREC_MIXED, sw)
    finally:
        Q.qqmc_destroy_problem(pr)
    assert np.all(np.abs(S32 - S64) <= 1e-4 * np.abs(S64)), np.abs(S32 - S64) / np.abs(S64)
    assert abs(r32.q_mean - r64.q_mean) <= 0.05 * r64.q_err


@pytest.mark.parametrize("flat", [2, 3, 4, 5])
def test_mixed_every_flat_depth_within_bound_of_fp64(Q, W, oracle, flat):
    """Every flat depth of the mixed kernel, with the breadth-first levels above it (the first one
    built as both children of the leaf in one pass), against the FP64 path on the same shifts:
    equal in-domain counts, per-shift sums within 1e-4 of the shifts' scale (the largest |S_k|:
    a shift sum that cancels between points keeps the absolute FP32 error of the others) and the
    shift mean within 5% of its error bar."""
    from paper_2002_12372_gb300 import autotune
    T, K = 10.0, 8
    pr, tabs = _problem(Q, W, seed=90, T=T)
    try:
        for n, N in [(6, 1024), (7, 1024), (10, 256)]:
            Q.qqmc_set_tuning(Q.QQMC_PREC_MIXED, n, 2, flat)
            sw = W.shift_words(4000 + n, K, n)
            r64, S64 = Q.qqmc_integrate(pr, n, N, K, Q.QQMC_PREC_FP64, sw)
            r32, S32 = Q.qqmc_integrate(pr, n, N, K, Q.QQMC_PREC_MIXED, sw)
            assert r32.n_in_domain == r64.n_in_domain
            scale = np.max(np.abs(S64))
            assert np.all(np.abs(S32 - S64) <= 1e-4 * scale), (n, np.abs(S32 - S64) / scale)
            assert abs(r32.q_mean - r64.q_mean) <= 0.05 * r64.q_err
    finally:
        Q.qqmc_destroy_problem(pr)
        autotune.reset()


@pytest.mark.parametrize("precision", [0, 1])
def test_two_points_per_warp_match_oracle(Q, W, oracle, precision):
    """Orders whose single-vertex tree fills at most half a warp per point (n <= 5, and n = 6 in mixed
    precision at flat 5) run two points per warp, one per half-warp, with both points' breadth-first
    levels built together; an odd in-domain count leaves a lone last point on the one-point path.
    Every order 1..6 at every flat depth, with 16384 and 8191 points x 4 shifts (work units of 4 and
    2 points: the plan cuts small items into point groups, so a unit holds pairs, odd counts and lone
    points): FP64 within 1e-10 of the oracle per shift; mixed within 1e-4 of the FP64 path's shift
    scale."""
    from paper_2002_12372_gb300 import autotune
    T, K = 10.0, 4
    pr, tabs = _problem(Q, W, seed=77, T=T, elim=2)
    try:
        for n in range(1, 7):
            sw = W.shift_words(8000 + n, K, n)
            for N in (16384, 8191):
                ref = oracle.estimate(n, N, sw, T, 1.0, tabs, T) if precision == Q.QQMC_PREC_FP64 else None
                for flat in (2, 3, 4, 5):
                    Q.qqmc_set_tuning(precision, n, 2, flat)
                    res, S = Q.qqmc_integrate(pr, n, N, K, precision, sw)
                    if precision == Q.QQMC_PREC_FP64:
                        S0, nin = ref
                        assert res.n_in_domain == int(nin.sum())
                        rel = np.abs(S - S0) / np.maximum(np.abs(S0), 1e-300)
                        assert np.all(rel < 1e-10), (n, flat, N, rel)
                    else:
                        Q.qqmc_set_tuning(Q.QQMC_PREC_FP64, n, 2, 2)
                        r64, S64 = Q.qqmc_integrate(pr, n, N, K, Q.QQMC_PREC_FP64, sw)
                        assert res.n_in_domain == r64.n_in_domain
                        assert np.all(np.abs(S - S64) <= 1e-4 * np.max(np.abs(S64))), (n, flat, N)
    finally:
        Q.qqmc_destroy_problem(pr)
        autotune.reset()


@pytest.mark.slow
def test_full_size_bench_launch_sampled_chunks(Q, W, oracle):
    """The benchmark's launch shape at full size (three problems, n = 1..10, N = 2^20 x 32 shifts,
    one persistent launch with the installed tuning) on identical synthetic tables: the in-domain
    counts are exact, and sampled chunks of 32 points match the oracle's sums over the same
    indices (FP64, relative 1e-10)."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    from paper_2002_12372_gb300 import autotune
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    t = autotune.load(os.path.join(root, "paper_2002_12372_gb300", "tuning_gb300.json"))
    if t:
        autotune.install(t)
    N, K, T, L = 2 ** 20, 32, 10.0, 4096
    tables = [W.synthetic_tables(51 + j, L, T) for j in range(3)]
    probs = [Q.qqmc_create_problem_tables(Q.make_params(t_max=T, n_table=L), gl, gg, g0)
             for gl, gg, g0, _ in tables]
    rng = np.random.default_rng(5)
    V = oracle.sobol_direction_numbers(12)
    try:
        items, shifts = [], {}
        for j, pr in enumerate(probs):
            for n in range(1, 11):
                sw = W.shift_words(7000 + 16 * j + n, K, n)
                shifts[(j, n)] = sw
                items.append((pr, n, K, N, sw))
        plan = Q.Plan(items, Q.QQMC_PREC_FP64)
        plan.launch()
        res = plan.results()
        for idx, (r, S) in enumerate(res):
            j, n = divmod(idx, 10)
            n += 1
            sw = shifts[(j, n)]
            if j == 0 and n in (6, 10):
                with ThreadPoolExecutor(16) as ex:
                    cnt = ex.map(lambda k: int(oracle.warp(n, 0, N, V, sw[k], T, 1.0)[2].sum()), range(K))
                assert r.n_in_domain == sum(cnt)
            gl, gg, g0, _ = tables[j]
            k = int(rng.integers(K))
            chunks = rng.integers(0, N // 32, size=2 if n >= 9 else 4)
            got = plan.chunk_sums(idx, k, chunks)
            for c, g in zip(chunks, got):
                S0, _ = oracle.estimate(n, 32, sw[k:k + 1], T, 1.0, (gl, gg, g0), T, i0=int(c) * 32, threads=1)
                ref = S0[0] * 32
                assert abs(g - ref) <= 1e-10 * abs(ref), (n, c, g, ref)
        plan.close()
    finally:
        for pr in probs:
            Q.qqmc_destroy_problem(pr)
        autotune.reset()


@pytest.mark.parametrize("precision", [0, 1])
def test_one_point_per_lane_mode_matches(Q, W, oracle, precision):
    """Orders <= 4 tuned to one point per lane run in their own kernel: FP64 within 1e-10 of the
    oracle per shift, mixed within 1e-4 of FP64; a plan mixing both kernels returns the same sums
    as single runs."""
    from paper_2002_12372_gb300 import autotune
    T, K = 10.0, 4
    pr, tabs = _problem(Q, W, seed=61, T=T)
    try:
        for n in range(1, 5):
            Q.qqmc_set_tuning(precision, n, 2, 1)
        ref = {}
        for n, N in [(1, 3001), (2, 2048), (3, 999), (4, 1500)]:
            sw = W.shift_words(3000 + n, K, n)
            res, S = Q.qqmc_integrate(pr, n, N, K, precision, sw)
            S0, nin = oracle.estimate(n, N, sw, T, 1.0, tabs, T)
            if precision == 0:
                assert res.n_in_domain == int(nin.sum())
                assert np.all(np.abs(S - S0) <= 1e-10 * np.abs(S0))
            else:
                assert np.all(np.abs(S - S0) <= 1e-4 * np.abs(S0))
            ref[n] = (N, sw, S)
        items = [(pr, n, K, ref[n][0], ref[n][1]) for n in (4, 2)] + [(pr, 6, K, 300, W.shift_words(77, K, 6))]
        plan = Q.Plan(items, precision)
        assert plan.kernel_count() == 3
        plan.launch()
        out = plan.results()
        plan.close()
        for (_, n, _, _, _), (r, S) in zip(items[:2], out[:2]):
            assert np.allclose(S, ref[n][2], rtol=1e-12, atol=0)
    finally:
        Q.qqmc_destroy_problem(pr)
        autotune.reset()


def test_checkpoint_resume_by_index_cursor(Q, W, oracle):
    """A run split at an index cursor (first_index) adds up to the uninterrupted run: the
    per-(order, shift) sums plus the cursor are a complete checkpoint."""
    T, K, N = 10.0, 3, 4096
    pr, tabs = _problem(Q, W, seed=71, T=T)
    try:
        for n in (2, 7):
            sw = W.shift_words(90 + n, K, n)
            plan = Q.Plan([(pr, n, K, N, sw, 0)], Q.QQMC_PREC_FP64)
            plan.launch()
            (r_full, S_full), = plan.results()
            plan.close()
            parts, n_in = [], 0
            for first, cnt in [(0, 1536), (1536, 2560)]:
                p2 = Q.Plan([(pr, n, K, cnt, sw, first)], Q.QQMC_PREC_FP64)
                p2.launch()
                (r, S), = p2.results()
                p2.close()
                parts.append(S * cnt)
                n_in += r.n_in_domain
            assert n_in == r_full.n_in_domain
            assert np.allclose((parts[0] + parts[1]) / N, S_full, rtol=1e-12, atol=0)
    finally:
        Q.qqmc_destroy_problem(pr)


def test_cut_work_units_match_oracle(Q, W, oracle):
    """Few points at a high order: the plan cuts each 32-point chunk into single-point units and
    each point's Keldysh tree into subtrees (order 13, 64 points, 1 shift: 2 chunks -> 64 point
    units -> 512 subtree units).  Each chunk's sum (over its units), the per-shift sum and the
    in-domain count match the oracle over the same points (FP64, relative 1e-10)."""
    T, n, N = 10.0, 13, 64
    pr, tabs = _problem(Q, W, seed=313, T=T)
    try:
        sw = W.shift_words(1313, 1, n)
        plan = Q.Plan([(pr, n, 1, N, sw)], Q.QQMC_PREC_FP64)
        plan.launch()
        (res, S), = plan.results()
        got = plan.chunk_sums(0, 0, [0, 1])
        plan.close()
    finally:
        Q.qqmc_destroy_problem(pr)
    refs, nin = [], 0
    for c in range(2):
        S0, cnt = oracle.estimate(n, 32, sw, T, 1.0, tabs, T, i0=32 * c)
        refs.append(S0[0] * 32)
        nin += int(cnt.sum())
    assert res.n_in_domain == nin
    for g, ref in zip(got, refs):
        assert abs(g - ref) <= 1e-10 * abs(ref), (g, ref)
    assert abs(S[0] - (refs[0] + refs[1]) / N) <= 1e-10 * abs(S[0])


@pytest.mark.parametrize("order", [13, 14, 16, 17, 18])
def test_high_orders_match_oracle(Q, W, oracle, order):
    """Orders beyond the benchmark table (the paper reaches 22): integrand parity at a few points
    and, at order 13, a small integration against the oracle."""
    T = 10.0
    pr, tabs = _problem(Q, W, seed=200 + order, T=T)
    try:
        u = W.ordered_times(300 + order, 2 if order < 16 else 1, order, T)
        gpu = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_FP64)
        ref, scale = oracle.integrand(order, u, T, tabs, T, return_abs=True)
        assert np.all(np.abs(gpu - ref) <= 1e-12 * scale), np.max(np.abs(gpu - ref) / scale)
        if order == 13:
            sw = W.shift_words(13, 1, order)
            res, S = Q.qqmc_integrate(pr, order, 48, 1, Q.QQMC_PREC_FP64, sw)
            S0, nin = oracle.estimate(order, 48, sw, T, 1.0, tabs, T)
            assert res.n_in_domain == int(nin.sum())
            assert np.all(np.abs(S - S0) <= 1e-10 * np.abs(S0))
    finally:
        Q.qqmc_destroy_problem(pr)


def _golden_high_orders():
    rows = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "high_order_integrand.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, re, im, sc = line.split()
                rows[int(n)] = (complex(float(re), float(im)), float(sc))
    return rows


@pytest.mark.parametrize("order", [19, 20, 21, 22])
def test_orders_19_to_22_match_stored_oracle_values(Q, W, order):
    """Orders 19..22 against oracle values stored by tests/golden/make_high_order_integrand.py
    (the oracle needs 10 s to 2 min per point there).  From order 21 the FP64 tree stack lives in
    device memory; the mixed path keeps it in shared memory."""
    c_ref, scale = _golden_high_orders()[order]
    T = 10.0
    pr, _ = _problem(Q, W, seed=200 + order, T=T)
    try:
        u = W.ordered_times(300 + order, 1, order, T)
        gpu = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_FP64)[0]
        mixed = Q.qqmc_integrand(pr, order, u, Q.QQMC_PREC_MIXED)[0]
    finally:
        Q.qqmc_destroy_problem(pr)
    assert abs(gpu - c_ref) <= 1e-12 * scale, abs(gpu - c_ref) / scale
    assert abs(mixed - c_ref) <= 2.0 ** -20 * scale, abs(mixed - c_ref) / scale


def test_order_22_plan_equals_its_points(Q, W):
    """A batched FP64 plan at order 22 (tree stack in device memory) returns the weighted sum of
    the integrand at its own warped points."""
    T, n, N = 10.0, 22, 40
    pr, _ = _problem(Q, W, seed=222, T=T, tau=0.35)
    try:
        sw = W.shift_words(2222, 1, n)
        plan = Q.Plan([(pr, n, 1, N, sw)], Q.QQMC_PREC_FP64)
        plan.launch()
        (res, S), = plan.results()
        plan.close()
        u, w, ins = Q.qqmc_warp_points(pr, n, 0, N, sw[0])
        c = Q.qqmc_integrand(pr, n, u[ins], Q.QQMC_PREC_FP64)
    finally:
        Q.qqmc_destroy_problem(pr)
    assert res.n_in_domain == int(ins.sum()) > 0
    ref = np.sum(w[ins] * c) / N
    # The two kernels round differently (separately compiled), and at order 22 the Keldysh sum
    # cancels to |c| ~ 1e-11 of its terms, so an FP64 c is good to ~1e-4 relative; a bookkeeping
    # error (wrong point, weight or stack slice) would be O(1).
    assert abs(S[0] - ref) <= 1e-3 * np.sum(np.abs(w[ins] * c)) / N


@pytest.mark.parametrize("precision", [0, 1])
def test_split_stack_is_bit_identical(Q, W, precision):
    """The split tree stack (wide levels in device memory, qqmc_set_stack_policy) runs the same
    arithmetic as the shared-memory stack: the same per-shift sums bit for bit."""
    T = 10.0
    pr, _ = _problem(Q, W, seed=91, T=T)
    items = [(pr, n, 2, N, W.shift_words(90 + n, 2, n)) for n, N in [(6, 700), (9, 130), (12, 33)]]
    try:
        Q.qqmc_set_stack_policy(precision, Q.QQMC_MAX_ORDER + 1)
        plan = Q.Plan(items, precision)
        plan.launch()
        ref = plan.results()
        plan.close()
        Q.qqmc_set_stack_policy(precision, 1)
        plan = Q.Plan(items, precision)
        plan.launch()
        out = plan.results()
        plan.close()
    finally:
        Q.qqmc_set_stack_policy(precision, 0)
        Q.qqmc_destroy_problem(pr)
    for (r0, S0), (r1, S1) in zip(ref, out):
        assert r0.n_in_domain == r1.n_in_domain
        assert np.array_equal(S0, S1)


def test_stack_policy_change_after_plan_creation(Q, W):
    """A plan keeps the device-memory stack it was sized for: changing the stack policy between
    creating and launching it leaves the sums unchanged (the split and the shared-memory stacks run
    the same arithmetic)."""
    T = 10.0
    pr, _ = _problem(Q, W, seed=93, T=T)
    items = [(pr, n, 2, N, W.shift_words(190 + n, 2, n)) for n, N in [(6, 700), (9, 130), (12, 33)]]
    try:
        Q.qqmc_set_stack_policy(0, Q.QQMC_MAX_ORDER + 1)
        ref = Q.Plan(items, 0)
        ref.launch()
        ref_out = ref.results()
        Q.qqmc_set_stack_policy(0, 1)  # after creation: the plan was sized without a split stack
        ref.launch()
        out1 = ref.results()
        ref.close()
        split = Q.Plan(items, 0)  # sized with the split stack for every group
        Q.qqmc_set_stack_policy(0, Q.QQMC_MAX_ORDER + 1)
        split.launch()
        out2 = split.results()
        split.close()
    finally:
        Q.qqmc_set_stack_policy(0, 0)
        Q.qqmc_destroy_problem(pr)
    for (r0, S0), (r1, S1), (r2, S2) in zip(ref_out, out1, out2):
        assert r0.n_in_domain == r1.n_in_domain == r2.n_in_domain
        assert np.array_equal(S0, S1) and np.array_equal(S0, S2)
