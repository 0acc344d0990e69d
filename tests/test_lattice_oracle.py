"""Pins of the oracle's rank-1 lattice point family (the lattice rules the paper
cites as the other low-discrepancy family) and of its component-by-component
construction, against closed forms, the character sum that defines a lattice
rule, and brute force."""
import math

import numpy as np
import pytest


def test_lattice_rule_character_sum(oracle):
    """(1/N) sum_i exp(2 pi i h.x_i) = exp(2 pi i h.Delta) if h.z = 0 mod N, else 0."""
    m, n = 8, 3
    N = 1 << m
    z = np.array([1, 37, 91], dtype=np.uint32)
    S = np.array([0x12345678, 0x9abcdef0, 0x0f0f0f0f], dtype=np.uint32)
    x = oracle.lattice_points(n, 0, N, z, m, S).astype(np.float64) * 2.0 ** -32
    delta = S.astype(np.float64) * 2.0 ** -32
    rng = np.random.default_rng(1)
    hs = [rng.integers(-40, 41, n) for _ in range(30)]
    hs += [np.array([37, -1, 0]), np.array([91, 0, -1]), np.array([N, 0, 0]), np.array([0, 0, 0])]  # dual lattice
    for h in hs:
        val = np.mean(np.exp(2j * math.pi * (x @ h)))
        on_dual = int(np.dot(h, z.astype(np.int64))) % N == 0
        ref = np.exp(2j * math.pi * float(np.dot(h, delta))) if on_dual else 0.0
        assert abs(val - ref) < 1e-12, (h, val, ref)


def test_lattice_is_periodic_and_distinct(oracle):
    m, n = 6, 4
    N = 1 << m
    z = np.array([1, 5, 13, 27], dtype=np.uint32)
    S = np.zeros(n, dtype=np.uint32)
    a = oracle.lattice_points(n, 0, 2 * N, z, m, S)
    assert np.array_equal(a[:N], a[N:])
    assert len({tuple(r) for r in a[:N]}) == N
    assert np.array_equal(a[:, 0], (np.arange(2 * N) % N << (32 - m)).astype(np.uint32))


def test_cbc_criterion_one_dimension_closed_form(oracle):
    """One dimension, z = 1: e^2 = gamma 2 pi^2 (1/N) sum_k B_2(k/N) = gamma pi^2 / (3 N^2)."""
    for m in (3, 7, 10):
        N = 1 << m
        assert oracle.lattice_cbc_criterion(np.array([1]), m, np.array([0.7])) == pytest.approx(
            0.7 * math.pi ** 2 / (3 * N * N), rel=1e-10)


def test_cbc_matches_brute_force_on_a_small_lattice(oracle):
    m, dims = 6, 4
    N = 1 << m
    gamma = np.array([1.0, 0.5, 0.25, 0.125])
    z = oracle.lattice_cbc(m, dims, gamma)
    assert z[0] == 1
    for d in range(1, dims):
        best, arg = None, None
        for c in range(1, N // 2 + 1, 2):  # brute force over every admissible component
            e = oracle.lattice_cbc_criterion(np.concatenate([z[:d], [c]]), m, gamma)
            if best is None or e < best - 1e-12 * abs(best):  # equal up to rounding: keep the smaller
                best, arg = e, c
        assert z[d] == arg, (d, z[d], arg)
    # the construction beats a plain Korobov vector (1, 3, 9, 27) on its own criterion
    assert oracle.lattice_cbc_criterion(z, m, gamma) < oracle.lattice_cbc_criterion(
        np.array([1, 3, 9, 27]), m, gamma)


@pytest.mark.parametrize("n", [2, 4])
def test_lattice_warp_gives_simplex_volume(oracle, n):
    """With f = 1 the lattice estimate converges to the ordered-simplex volume t^n / n!."""
    t, tau, m = 3.0, 1.0, 14
    N = 1 << m
    gamma = np.array([0.9 ** d for d in range(n)])
    z = oracle.lattice_cbc(m, n, gamma)
    vals = []
    for k in range(8):
        S = oracle.shift_words(77 + k, 1, n)[0]
        u, w, ins = oracle.warp(n, 0, N, None, S, t, tau, lattice=(z, m))
        vals.append(np.sum(w[ins]) / N)
    mean, err = oracle.shift_statistics(np.array(vals))
    exact = t ** n / math.factorial(n)
    assert abs(mean - exact) < 5 * err + 1e-12 * exact
    assert err < 3e-3 * exact


def test_bakers_transform_preserves_the_measure_and_raises_the_rate(oracle):
    """x -> 1 - |2x - 1| is 2-to-1 and piecewise measure preserving: on an unshifted lattice
    {k/N} it gives every even multiple of 1/N twice (0 and 1 - 2^-32 once each).  For a smooth
    non-periodic f the 1-D lattice error falls as N^-2 after the transform, N^-1 before."""
    for m in (4, 9):
        N = 1 << m
        w = oracle.lattice_points(1, 0, N, np.array([1]), m, np.zeros(1, dtype=np.uint32), tent=True)[:, 0]
        expect = sorted([2 * k << (32 - m) for k in range(N // 2)] + [2 * k << (32 - m) for k in range(1, N // 2)]
                        + [0xFFFFFFFF])
        assert sorted(int(x) for x in w) == expect
    f = lambda x: np.exp(x)  # integral e - 1
    errs = {}
    for tent in (False, True):
        for m in (8, 12):
            x = oracle.lattice_points(1, 0, 1 << m, np.array([1]), m, np.array([0x1234567], dtype=np.uint32),
                                      tent=tent)[:, 0].astype(np.float64) * 2.0 ** -32
            errs[(tent, m)] = abs(np.mean(f(x)) - (math.e - 1.0))
    assert errs[(False, 8)] / errs[(False, 12)] < 40      # ~16 = N ratio
    assert errs[(True, 8)] / errs[(True, 12)] > 150       # ~256 = N^2 ratio
