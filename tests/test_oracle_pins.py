"""Pins of the CPU oracle against things other than itself.

Each test fixes one piece of the oracle with a value the paper prints, a
closed form, an invariant of the Keldysh formalism, a library routine used
as an independent check, or brute force.  None of them needs a GPU.
"""
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _bethe():
    out = {}
    with open(os.path.join(HERE, "golden", "bethe_q.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, v = line.split()
                out[int(n)] = float(v)
    return out


# ----------------------------------------------------------------- fixtures ---

def test_bethe_golden_matches_printed_closed_forms():
    """The 25-digit column of the paper's Bethe table agrees with its closed forms."""
    q = _bethe()
    pi = math.pi
    assert q[1] == pytest.approx(-1 / pi, rel=1e-15)
    assert q[2] == pytest.approx(1 / pi ** 2, rel=1e-15)
    assert q[3] == pytest.approx((pi ** 2 - 9) / (3 * pi ** 3), rel=1e-13)
    assert q[4] == pytest.approx((90 - 11 * pi ** 2) / (6 * pi ** 4), rel=1e-13)
    assert q[6] == pytest.approx(945 / pi ** 6 - 3185 / (27 * pi ** 4) + 137 / (60 * pi ** 2), rel=1e-12)


# ------------------------------------------------------------------- points ---

def test_sobol_bit_exact_vs_scipy_and_torch(oracle):
    from scipy.stats import qmc
    import torch

    V = oracle.sobol_direction_numbers(12)
    pts = oracle.sobol_points(12, 0, 4096, V)
    ref = np.rint(qmc.Sobol(12, scramble=False, bits=32).random(4096) * 2.0 ** 32)
    assert np.array_equal(ref.astype(np.uint64).astype(np.uint32), pts)
    tp = torch.quasirandom.SobolEngine(12, scramble=False).draw(4096, dtype=torch.float64).numpy()
    assert np.array_equal(np.rint(tp * 2.0 ** 32).astype(np.uint64).astype(np.uint32), pts)
    eng = qmc.Sobol(12, scramble=False, bits=32)
    eng.fast_forward(3_000_001)
    far = np.rint(eng.random(7) * 2.0 ** 32).astype(np.uint64).astype(np.uint32)
    assert np.array_equal(far, oracle.sobol_points(12, 3_000_001, 7, V))


def test_splitmix64_published_outputs(oracle):
    """First outputs of splitmix64 seeded with 0 (the generator's published reference run)."""
    g = 0x9E3779B97F4A7C15
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(g) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64((2 * g) % 2 ** 64) == 0x06C45D188009454F


def test_shift_is_xor(oracle):
    V = oracle.sobol_direction_numbers(5)
    S = oracle.shift_words(7, 1, 5)[0]
    x = oracle.sobol_points(5, 0, 1024, V)
    u, w, ins = oracle.warp(5, 0, 1024, V, S, 1e9, 1.0)
    # with t huge every point is inside; recover x from v = u_{m-1} - u_m
    v = -np.diff(np.concatenate([np.full((1024, 1), 1e9), u], axis=1), axis=1)
    xs = ((x ^ S).astype(np.float64)) * 2.0 ** -32
    assert np.allclose(v, -np.log1p(-xs), rtol=1e-6, atol=1e-6)


# ---------------------------------------------------------- Green functions ---

def _mp_contour(tau, eps, gamma, which):
    """30-digit g^< / g^> by the App. E deformed contour (vertical ray + segment)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    eps, gamma, tau = mp.mpf(eps), mp.mpf(gamma), mp.mpf(tau)
    A = lambda w: 2 * gamma / ((w - eps) ** 2 + gamma ** 2)
    sgn = 1 if tau > 0 else -1
    if which == "lesser":   # i Int_{-inf}^0 dw/2pi e^{-iw tau} A
        wm = min(eps, 0) - 2
        f = lambda w: mp.exp(-1j * w * tau) * A(w)
        ray = mp.quad(lambda y: f(wm - sgn * 1j * y) * (-sgn * 1j), [mp.inf, 0])
        seg = mp.quad(f, mp.linspace(wm, 0, 20))
        return complex(1j / (2 * mp.pi) * (ray + seg))
    wp = max(eps, 0) + 2     # -i Int_0^inf dw/2pi e^{-iw tau} A
    f = lambda w: mp.exp(-1j * w * tau) * A(w)
    seg = mp.quad(f, mp.linspace(0, wp, 20))
    ray = mp.quad(lambda y: f(wp - sgn * 1j * y) * (-sgn * 1j), [0, mp.inf])
    return complex(-1j / (2 * mp.pi) * (seg + ray))


@pytest.mark.parametrize("eps", [-1.0, 0.0, 1.0])
def test_gf_against_30_digit_quadrature(oracle, eps):
    for tau in [0.01, 0.7, 3.3, 9.5, -2.0]:
        gl, gg = oracle.gf_exact(tau, 1.0, eps)
        assert abs(gl[0] - _mp_contour(tau, eps, 1.0, "lesser")) < 1e-14
        assert abs(gg[0] - _mp_contour(tau, eps, 1.0, "greater")) < 1e-14


@pytest.mark.parametrize("eps,gamma", [(0.0, 1.0), (-2.3, 1.0), (1.7, 0.5)])
def test_gf_exact_identities(oracle, eps, gamma):
    tau = np.linspace(-12, 12, 997)
    gl, gg = oracle.gf_exact(tau, gamma, eps)
    # spectral sum rule: g^> - g^< = -i Int dw/2pi e^{-iw tau} A(w) = -i e^{-i eps tau - Gamma |tau|}
    assert np.max(np.abs(gg - gl + 1j * np.exp(-1j * eps * tau - gamma * np.abs(tau)))) < 1e-14
    # g(-tau) = -conj g(tau)
    gl2, gg2 = oracle.gf_exact(-tau, gamma, eps)
    assert np.max(np.abs(gl2 + np.conj(gl))) < 1e-15
    assert np.max(np.abs(gg2 + np.conj(gg))) < 1e-15
    # equal time: g^<(0) = i(1/2 - arctan(eps/Gamma)/pi), approached continuously
    g0 = 1j * (0.5 - math.atan(eps / gamma) / math.pi)
    glt, _ = oracle.gf_exact(np.array([1e-10, -1e-10]), gamma, eps)
    assert np.max(np.abs(glt - g0)) < 1e-8
    # |g^<| <= <n> and |g^>| <= 1 - <n> (positive spectral weight)
    n0 = g0.imag
    assert np.all(np.abs(gl) <= n0 + 1e-13) and np.all(np.abs(gg) <= 1 - n0 + 1e-13)


def test_table_interpolation_vs_numpy(oracle):
    T, L = 10.0, 4096
    tab = oracle.gf_tables(1.0, 0.4, T, L)[0]
    x = oracle.table_nodes(T, L)
    rng = np.random.default_rng(3)
    tau = rng.uniform(-T, T, 5000)
    ref = np.interp(tau, x, tab.real) + 1j * np.interp(tau, x, tab.imag)
    assert np.max(np.abs(oracle.table_at(tab, T, tau) - ref)) < 4e-15  # a few ulps of |g| <= 1/2


# --------------------------------------------------------------- integrand ---

def test_det_lu_vs_library_and_leibniz(oracle):
    from itertools import permutations

    rng = np.random.default_rng(11)
    for m in [1, 2, 3, 5, 8, 13]:
        A = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
        assert abs(oracle.det(A) - np.linalg.det(A)) < 1e-12 * max(1.0, abs(np.linalg.det(A)))
    A = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    leib = 0
    for p in permutations(range(4)):
        sgn = np.linalg.det(np.eye(4)[list(p)])
        leib += sgn * np.prod([A[i, p[i]] for i in range(4)])
    assert abs(oracle.det(A) - leib) < 1e-13
    # a matrix that needs pivoting (zero leading entry)
    B = np.array([[0, 1], [1, 0]], dtype=complex)
    assert oracle.det(B) == -1


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_causality_vertex_after_measurement_cancels(oracle, n):
    """A vertex later than the measurement time drops out of the Keldysh sum."""
    t = 5.0
    tabs = oracle.gf_tables(1.0, 0.3, 2 * t, 4096)
    rng = np.random.default_rng(n)
    for _ in range(5):
        u = rng.uniform(0, t, n)
        u[rng.integers(n)] = rng.uniform(t + 0.05, 1.8 * t)
        val, ab = oracle.integrand(n, u, t, tabs, 2 * t, return_abs=True)
        assert abs(val[0]) < 1e-13 * ab[0]
        # and a generic point does not cancel
        u2 = rng.uniform(0, t, n)
        val2, ab2 = oracle.integrand(n, u2, t, tabs, 2 * t, return_abs=True)
        assert abs(val2[0]) > 1e-6 * ab2[0]


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_charge_integrand_is_real(oracle, n):
    """Q-integrand -2i c(u) is real point by point (c purely imaginary)."""
    t = 10.0
    tabs = oracle.gf_tables(1.0, -0.7, t, 4096)
    rng = np.random.default_rng(100 + n)
    u = np.sort(rng.uniform(0, t, (20, n)), axis=1)[:, ::-1]
    val, ab = oracle.integrand(n, u, t, tabs, t, return_abs=True)
    assert np.all(np.abs(val.real) < 1e-14 * ab)


def test_integrand_symmetric_in_vertex_labels(oracle):
    t = 10.0
    tabs = oracle.gf_tables(1.0, 0.0, t, 4096)
    rng = np.random.default_rng(5)
    u = rng.uniform(0, t, 4)
    a = oracle.integrand(4, u, t, tabs, t)[0]
    b = oracle.integrand(4, u[[2, 0, 3, 1]], t, tabs, t)[0]
    assert abs(a - b) < 1e-14


def _wick_brute(n, u, t, alpha, vals, meas, meas_col):
    """App. E Eq. (integral_gf) at 50 digits, assembled point by point on the Keldysh contour:
    g[(x,u,a),(x',u',a')] is the 2x2 matrix (g^T, g^<; g^>, g^Tbar)_{a a'} at u - u', with
    g^T = g^> for u > u' (g^< otherwise) and g^Tbar the reverse.  Vertex diagonals are the
    equal-time lesser value shifted by -i alpha; the measurement entry is not shifted.
    vals(x, tau) -> (g^<, g^>) between site 0 and site x; meas: g^<_{0x}(0); meas_col: x of
    the measurement column (0: charge, 1: current)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50

    def g(A, B):
        (xa, ua, aa), (xb, ub, ab) = A, B
        lt, gt = vals(xb, ua - ub)
        if (aa, ab) == (0, 1):
            return lt
        if (aa, ab) == (1, 0):
            return gt
        later = ua > ub
        return (gt if later else lt) if aa == 0 else (lt if later else gt)

    total = mp.mpc(0)
    for conf in range(1 << n):
        a = [(conf >> k) & 1 for k in range(n)]
        U = [(0, float(u[k]), a[k]) for k in range(n)]
        rows = [(0, t, 0)] + U
        cols = [(meas_col, t, 1)] + U
        up = mp.matrix(n + 1, n + 1)
        for r in range(n + 1):
            for c in range(n + 1):
                if r == 0 and c == 0:
                    up[r, c] = meas
                elif r == c:
                    up[r, c] = vals(0, 0.0)[0] - 1j * alpha
                else:
                    up[r, c] = g(rows[r], cols[c])
        dn = mp.matrix(n, n)
        for r in range(n):
            for c in range(n):
                dn[r, c] = vals(0, 0.0)[0] - 1j * alpha if r == c else g(U[r], U[c])
        total += (-1) ** sum(a) * mp.det(up) * mp.det(dn)
    return complex(mp.mpc(1j) ** n * total)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("current", [False, True])
def test_integrand_assembly_against_50_digit_wick_sum(oracle, n, current):
    """The oracle's integrand against the Wick-determinant sum of App. E assembled independently
    (contour points, 2x2 Keldysh blocks, mpmath determinants), on the same table values: charge
    and current, alpha != 0, vertices in any time order, one later than t."""
    t, T, L, alpha = 6.0, 12.0, 512, 0.37
    tabs = oracle.gf_tables(1.0, 0.4, T, L)
    # any tables serve for the dot-lead column: the assembly is a polynomial in the entries
    other = oracle.gf_tables(0.6, -0.9, T, L)
    col = (0.3 * other[0], -0.2j * other[1], 0.3 * other[2]) if current else None

    def vals(x, tau):
        if tau == 0.0 and x == 0:
            return complex(tabs[2]), None
        src = col if x == 1 else tabs
        return complex(oracle.table_at(src[0], T, tau)[0]), complex(oracle.table_at(src[1], T, tau)[0])

    meas = complex(col[2]) if current else complex(tabs[2])
    rng = np.random.default_rng(40 + n + 10 * current)
    pts = [rng.uniform(0, t, n) for _ in range(3)]
    pts[0][-1] = t + 1.3  # a vertex after the measurement time
    for u in pts:
        got, ab = oracle.integrand(n, u, t, tabs, T, return_abs=True, alpha=alpha, col=col)
        ref = _wick_brute(n, u, t, alpha, vals, meas, 1 if current else 0)
        assert abs(got[0] - ref) <= 1e-13 * ab[0] + 1e-300, (u, got[0], ref)


# ------------------------------------------------------------ warp & estimate ---

@pytest.mark.parametrize("n,tau", [(1, 1.0), (2, 0.6), (3, 1.0), (4, 0.95), (3, 1.7)])
def test_warp_weight_gives_simplex_volume(oracle, n, tau):
    """With f = 1 the warped estimator integrates the ordered simplex: t^n / n!."""
    t, N, K = 3.0, 2 ** 14, 8
    V = oracle.sobol_direction_numbers(n)
    vals = []
    for S in oracle.shift_words(42, K, n):
        u, w, ins = oracle.warp(n, 0, N, V, S, t, tau)
        vals.append(np.sum(w * ins) / N)
        assert np.all((u[:, -1] > 0) == ins)
    m, e = oracle.shift_statistics(np.array(vals))
    exact = t ** n / math.factorial(n)
    assert abs(m - exact) < 5 * e + 1e-12 * exact
    assert e < 3e-3 * exact  # the domain indicator is discontinuous: plain MC-like rate


def test_order1_against_adaptive_quadrature(oracle):
    """Q_1 by QMC equals the 1-D adaptive quadrature of the same order-1 integrand."""
    from scipy.integrate import quad

    t = 10.0
    tabs = oracle.gf_tables(1.0, 0.5, t, 4096)
    f = lambda u: (-2j * oracle.integrand(1, np.array([u]), t, tabs, t)[0]).real
    knots = list(oracle.table_nodes(t, 4096)[2048:][::64]) + [t]
    exact = 0.0
    lo = 0.0
    for hi in knots:
        if hi > lo:
            exact += quad(f, lo, hi, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
            lo = hi
    S, _ = oracle.estimate(1, 2 ** 16, oracle.shift_words(9, 8, 1), t, 0.95, tabs, t)
    m, e = oracle.shift_statistics(oracle.q_from_sums(S).real)
    assert abs(m - exact) < 5 * e + 1e-9
    assert e < 1e-6


def test_order2_against_nested_gauss_legendre(oracle):
    """Q_2 by QMC equals nested Gauss-Legendre over 0 < u_2 < u_1 < t."""
    t = 4.0
    tabs = oracle.gf_tables(1.0, 0.0, t, 4096)
    x, wq = np.polynomial.legendre.leggauss(24)
    panels = np.linspace(0, t, 17)
    U1, W1 = [], []
    for a, b in zip(panels[:-1], panels[1:]):
        U1.append(0.5 * (b - a) * x + 0.5 * (a + b))
        W1.append(0.5 * (b - a) * wq)
    U1, W1 = np.concatenate(U1), np.concatenate(W1)
    pts, wts = [], []
    for u1, w1 in zip(U1, W1):
        sub = np.linspace(0, u1, 9)
        for a, b in zip(sub[:-1], sub[1:]):
            u2 = 0.5 * (b - a) * x + 0.5 * (a + b)
            pts.append(np.stack([np.full_like(u2, u1), u2], axis=1))
            wts.append(w1 * 0.5 * (b - a) * wq)
    pts, wts = np.concatenate(pts), np.concatenate(wts)
    vals = (-2j * oracle.integrand(2, pts, t, tabs, t)).real
    gauss = float(np.sum(wts * vals))
    S, _ = oracle.estimate(2, 2 ** 16, oracle.shift_words(10, 8, 2), t, 1.3, tabs, t)
    m, e = oracle.shift_statistics(oracle.q_from_sums(S).real)
    assert abs(m - gauss) < 5 * e + 2e-8


@pytest.mark.slow
def test_bethe_coefficients_at_long_time(oracle):
    """Q_1..Q_5 at t = 30 match the paper's Bethe-ansatz table (fine table, 8 shifts)."""
    q = _bethe()
    t = 30.0
    tabs = oracle.gf_tables(1.0, 0.0, t, 65536)
    sh = oracle.shift_words(2002123720, 8, 5)
    for n in range(1, 6):
        S, _ = oracle.estimate(n, 2 ** 14, sh, t, 1.0, tabs, t)
        Q = oracle.q_from_sums(S)
        m, e = oracle.shift_statistics(Q.real)
        assert np.max(np.abs(Q.imag)) < 1e-12
        assert abs(m - q[n]) < 6 * e + 1e-5 * abs(q[n]), (n, m, q[n], e)


def test_q0_is_one(oracle):
    """Q_0 = -2i g^<(0) = 1 at eps_d = 0 (particle-hole symmetric, non-interacting)."""
    gl0 = oracle.gf_tables(1.0, 0.0, 10.0, 16)[2]
    assert abs(-2j * gl0 - 1.0) < 1e-15


def test_shift_statistics_definition(oracle):
    m, e = oracle.shift_statistics(np.array([1.0, 2.0, 4.0, 5.0]))
    assert m == 3.0
    assert e == pytest.approx(math.sqrt(10.0 / 3.0) / 2.0)
