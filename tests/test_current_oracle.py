"""Pins of the oracle's current observable (App. E, i = 1: the measurement
column on lead site 1) and of its finite-bandwidth lead tables.

Each pin compares with something other than the oracle's own formulas: a
30-digit mpmath quadrature, the wide-band closed form, equal-time identities of
the operators, the Landauer formula, and the first-order (Hartree) relation.
"""

import numpy as np
import pytest

GAM, ED, D, V = 1.0, 0.3, 10.0, 0.6


def test_lead_functions_against_30_digit_quadrature(oracle):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30

    def spec(th, j):
        w = D * mp.sin(th)
        G = GAM * mp.cos(th)
        delta = GAM * (mp.sin(th) - 1j * mp.cos(th))
        gR = 1 / (w - ED - delta)
        fL = 1 if w < V / 2 else 0
        fR = 1 if w < -V / 2 else 0
        a2 = abs(gR) ** 2
        gl = 1j * G * a2 * (fL + fR)
        gg = -1j * G * a2 * (2 - fL - fR)
        vals = [gl, gg, 1j * fR * G * gR + mp.conj(delta) / 2 * gl,
                -1j * (1 - fR) * G * gR + mp.conj(delta) / 2 * gg]
        return vals[j] * D * mp.cos(th) / (2 * mp.pi)

    br = [-mp.pi / 2, mp.asin(-V / (2 * D)), mp.asin(V / (2 * D)), mp.pi / 2]
    tau = -5.2
    F = oracle.lead_functions(np.array([tau]), GAM, ED, D, V)
    for j in range(4):
        tot = 0
        for a, b in zip(br[:-1], br[1:]):
            tot += mp.quad(lambda th: spec(th, j) * mp.exp(-1j * D * mp.sin(th) * tau), mp.linspace(a, b, 16))
        assert abs(complex(tot) - F[j, 0]) < 1e-14


def test_equal_time_identities_and_landauer(oracle):
    """tau = 0: g^>_00 - g^<_00 = -i (spectral weight 1); g^<_00 = i<n> with <n> from
    Int A f; gamma g^>_01 = gamma g^<_01 ({c_0, c_1^+} = 0); -4 Re gamma g^<_01 is the
    Landauer current (1/pi) Int_{-V/2}^{V/2} Gamma(w)^2 |g^R|^2 dw, zero at V = 0."""
    for v in (V, 0.0, 2.5):
        gl, gg, cl, cg = oracle.lead_functions(np.array([0.0]), GAM, ED, D, v)[:, 0]
        assert abs(gg - gl + 1j) < 1e-13
        assert abs(gl - 1j * oracle.lead_occupation(GAM, ED, D, v)) < 1e-13
        assert abs(cg - cl) < 1e-13
        assert abs(-4.0 * cl.real - oracle.landauer_current(GAM, ED, D, v)) < 1e-12
    assert oracle.landauer_current(GAM, ED, D, 2.5) > 0.5


def test_wide_band_limit_of_the_dot_tables(oracle):
    """Delta -> -i Gamma as D -> infinity: the finite-D tables approach the closed form
    (errors O(Gamma/D); linear extrapolation from D = 200, 400)."""
    taus = np.array([0.5, 2.0, 4.0, -1.3])
    ex = oracle.gf_exact(taus, GAM, ED)
    F1 = oracle.lead_functions(taus, GAM, ED, 200.0, 0.0)
    F2 = oracle.lead_functions(taus, GAM, ED, 400.0, 0.0)
    for j in range(2):
        assert np.max(np.abs(2 * F2[j] - F1[j] - ex[j])) < 1e-5


@pytest.mark.parametrize("n", [1, 2, 3])
def test_current_causality_vertex_after_measurement_cancels(oracle, n):
    t = 5.0
    tabs, col = oracle.lead_tables(GAM, ED, D, V, 2 * t, 2048)
    rng = np.random.default_rng(40 + n)
    for _ in range(4):
        u = rng.uniform(0, t, n)
        u[rng.integers(n)] = rng.uniform(t + 0.05, 1.8 * t)
        val, ab = oracle.integrand(n, u, t, tabs, 2 * t, return_abs=True, col=col)
        assert abs(val[0]) < 1e-13 * ab[0]
        u2 = rng.uniform(0, t, n)
        val2, ab2 = oracle.integrand(n, u2, t, tabs, 2 * t, return_abs=True, col=col)
        assert abs(val2[0]) > 1e-6 * ab2[0]


def _first_order(oracle, tabs, col, t, alpha):
    x, w = np.polynomial.legendre.leggauss(20)
    edges = np.unique(np.concatenate([np.linspace(0, t - 3, 61), t - 3 + np.linspace(0, 3, 241)]))
    pts = np.concatenate([0.5 * (b - a) * x + 0.5 * (a + b) for a, b in zip(edges[:-1], edges[1:])])
    wts = np.concatenate([0.5 * (b - a) * w for a, b in zip(edges[:-1], edges[1:])])
    cq = oracle.integrand(1, pts.reshape(-1, 1), t, tabs, t, alpha=alpha)
    ci = oracle.integrand(1, pts.reshape(-1, 1), t, tabs, t, alpha=alpha, col=col)
    return float(np.sum(wts * oracle.q_from_sums(cq).real)), float(np.sum(wts * oracle.i_from_sums(ci)))


@pytest.mark.parametrize("alpha", [0.0, 0.2])
def test_first_order_is_the_hartree_level_shift(oracle, alpha):
    """At first order in U the interaction U (n_up - a)(n_dn - a) acts as the static level
    shift U (<n> - a), so in the steady state Q_1 = (<n> - a) dQ_0/dE_d and
    I_1 = (<n> - a) dI_0/dE_d, with Q_0 = 2 <n> and I_0 the Landauer current (derivatives
    by central differences of their 1-D integrals).  t = 15 / Gamma: transient < 1e-6."""
    t, L = 15.0, 8192
    tabs, col = oracle.lead_tables(GAM, ED, D, V, t, L)
    Q1, I1 = _first_order(oracle, tabs, col, t, alpha)
    n0 = tabs[2].imag
    h = 1e-4
    dQ = 2 * (oracle.lead_occupation(GAM, ED + h, D, V) - oracle.lead_occupation(GAM, ED - h, D, V)) / (2 * h)
    dI = (oracle.landauer_current(GAM, ED + h, D, V) - oracle.landauer_current(GAM, ED - h, D, V)) / (2 * h)
    assert Q1 == pytest.approx((n0 - alpha) * dQ, rel=3e-5)
    assert I1 == pytest.approx((n0 - alpha) * dI, rel=3e-5)
    assert abs(I1) > 1e-3
