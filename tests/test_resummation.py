"""Series resummation (parabola conformal map): the oracle against closed forms,
and the C-ABI host routine against the oracle.  No GPU needed."""
import math


import numpy as np
import pytest

pytest.importorskip("sympy")  # the oracle expands the map symbolically


def test_oracle_resummation_inside_radius_is_exact(oracle):
    a = [(-1.0) ** n for n in range(17)]  # 1/(1+U), radius 1
    assert oracle.resum_parabola(a, -1.0, 0.3) == pytest.approx(1 / 1.3, rel=1e-7)


def test_oracle_resummation_converges_beyond_radius(oracle):
    errs = []
    for N in (4, 8, 12, 16):
        a = [(-1.0) ** n for n in range(N + 1)]
        errs.append(abs(oracle.resum_parabola(a, -1.0, 2.0) - 1 / 3.0))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-3
    # the plain partial sum diverges there
    assert abs(sum((-2.0) ** n for n in range(17)) - 1 / 3.0) > 1e3
    # log(1+U)/U, a branch point instead of a pole
    a = [(-1.0) ** n / (n + 1) for n in range(17)]
    assert abs(oracle.resum_parabola(a, -1.0, 3.0) - math.log1p(3.0) / 3.0) < 5e-3


def test_oracle_resummation_of_the_inverse(oracle):
    a = [1.0, 1.0] + [0.0] * 14  # F = 1 + U: 1/F has radius 1, F itself is exact
    assert oracle.resum_parabola(a, -1.0, 2.0, invert=True) == pytest.approx(3.0, rel=2e-3)


@pytest.fixture(scope="module")
def Q():
    from paper_2002_12372_gb300 import build as b
    b.build()
    from paper_2002_12372_gb300 import qqmc
    qqmc.load()
    return qqmc


@pytest.mark.parametrize("N,p,U,invert", [(6, -1.0, 2.5, False), (12, -0.7, 4.0, False), (16, -3.0, 1.0, False),
                                          (10, -1.5, 3.0, True)])
def test_library_resummation_matches_oracle(Q, oracle, N, p, U, invert):
    rng = np.random.default_rng(N)
    a = rng.normal(size=N + 1) / (1.0 + np.arange(N + 1)) ** 2
    a[0] = 1.0 + abs(a[0])
    v, err, tail = Q.qqmc_resum_parabola(a, p, U, a_err=np.full(N + 1, 1e-6), invert=invert)
    assert v == pytest.approx(oracle.resum_parabola(a, p, U, invert=invert), rel=1e-11, abs=1e-13)
    assert err > 0 and tail >= 0


def test_library_resummation_rejects_bad_arguments(Q):
    with pytest.raises(Q.QQMCError):
        Q.qqmc_resum_parabola([1.0, 2.0], 1.0, 2.0)   # p must be negative
    with pytest.raises(Q.QQMCError):
        Q.qqmc_resum_parabola([0.0, 2.0], -1.0, 2.0, invert=True)


def _atanh_sq_coeffs(N):
    """c_m of atanh(sqrt W)^2 = sum_m c_m W^m from the Cauchy product of atanh x = sum_k x^(2k+1)/(2k+1):
    c_m = sum_{j+k=m-1} 1 / ((2j+1)(2k+1))  (1, 2/3, 23/45, 44/105, ...)."""
    return [0.0] + [sum(1.0 / ((2 * j + 1) * (2 * (m - 1 - j) + 1)) for j in range(m)) for m in range(1, N + 1)]


@pytest.mark.parametrize("p,U", [(-1.0, 0.7), (-2.5, 3.0)])
def test_oracle_parabola_map_expansion(oracle, p, U):
    """F(U) = U re-expanded in W is U(W) = |p| atanh(sqrt W)^2 truncated at the input order: its
    value at W(U) = tanh(sqrt(U/|p|))^2 is |p| sum_{m<=N} c_m W^m, and F(U) = U^2 gives the square
    of that series, truncated."""
    N = 8
    c = np.array(_atanh_sq_coeffs(N)) * abs(p)
    assert c[1] == pytest.approx(abs(p)) and c[2] == pytest.approx(2 * abs(p) / 3)
    assert c[3] == pytest.approx(23 * abs(p) / 45) and c[4] == pytest.approx(44 * abs(p) / 105)
    W = math.tanh(math.sqrt(U / abs(p))) ** 2
    a1 = [0.0, 1.0] + [0.0] * (N - 1)
    assert oracle.resum_parabola(a1, p, U) == pytest.approx(np.polynomial.polynomial.polyval(W, c), rel=1e-12)
    a2 = [0.0, 0.0, 1.0] + [0.0] * (N - 2)
    sq = np.polynomial.polynomial.polymul(c, c)[: N + 1]
    assert oracle.resum_parabola(a2, p, U) == pytest.approx(np.polynomial.polynomial.polyval(W, sq), rel=1e-12)


def test_oracle_parabola_map_inverts_the_transform(oracle):
    """U(W(U)) = U: the resummed series of F(U) = U converges to U as the order grows (W < 1)."""
    p, U = -1.0, 2.0
    errs = [abs(oracle.resum_parabola([0.0, 1.0] + [0.0] * (N - 1), p, U) - U) for N in (4, 8, 16, 24)]
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 0.02 * U
