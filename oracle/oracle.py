"""ORACLE -- test infrastructure only.

Plain, slow CPU restatement of the QQMC estimator for the perturbative
coefficients of the Anderson single-level dot at T = 0: the charge Q_n
(wide-band or semicircular leads) and the current I_n (semicircular leads of
half-bandwidth D under a symmetric bias V).
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA path
and imports nothing from the product package; inputs (shift words, synthetic
tables) are passed in by the caller.

Pieces and the passages they follow:

* ``gf_exact`` / ``gf_tables`` -- the non-interacting lesser/greater Green
  functions of the dot in the time domain, App. E Eq. (lesser_greater_freq)
  specialised to V = 0, T = 0 and the flat band Delta = -i Gamma (App. E,
  "universal regime"), Fourier transformed.  The convention is the textbook
  one, g^<(0) = i<n>, with the Lorentzian spectral function
  A(w) = 2 Gamma / ((w - eps_d)^2 + Gamma^2):

      g^<(tau) =  i Int dw/2pi e^{-i w tau} A(w) theta(-w)
      g^>(tau) = -i Int dw/2pi e^{-i w tau} A(w) theta(+w)

  Each half-line Fourier integral is written in closed form with the
  exponential integral E1 (partial fractions of the Lorentzian, then the
  Laplace-transform identity Int_0^inf e^{-p s}/(s+b) ds = e^{pb} E1(pb)),
  continued onto the sheet the integration path selects.  The App. E
  contour-deformation quadrature is a different route to the same numbers;
  this closed form is pinned against 30-digit quadrature in the tests.
* ``sobol_direction_numbers`` -- direction words of the unscrambled Sobol'
  sequence (main text below Eq. (warped_int2)), read off scipy's generator.
* ``sobol_points`` / ``warp`` / ``estimate`` -- C routines in qqmc_oracle.c
  (Gray-code Sobol' with a digital shift, App. H; product-model warp,
  Eq. (warper1d) with App. F Eq. (hi_expo); estimator Eq. (warped_int2)).
* ``integrand`` -- App. E Eq. (integral_gf): naive sum over all 2^n Keldysh
  index vectors of det M_up * det M_down, each by pivoted LU.
* ``lead_functions`` / ``lead_tables`` -- finite-bandwidth leads, App. E
  (semicircular hybridisation Delta(w), bias V, Eq. (lesser_greater_freq) for
  g_00 and the dot-lead function gamma g_01), Fourier transformed by adaptive
  quadrature; ``landauer_current`` and ``lead_occupation`` are independent 1-D
  integrals used by the pins.
* ``q_from_sums`` / ``i_from_sums`` / ``shift_statistics`` -- readouts
  Q_n = -2i c_n and I_n = -4 Re c_n (measurement column on lead site 1, App. E
  "i = 1"), and the randomised-QMC error bar (App. G, App. H: standard
  deviation over the K shifted sequences divided by sqrt(K)).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qqmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

_lib = None
_lib_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is not None:
        return _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i64 = ctypes.c_int64
        L.oracle_integrand.argtypes = [ctypes.c_int, i64, dp, ctypes.c_double, dp, dp, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_double,
                                       dp, dp]
        L.oracle_sobol.argtypes = [ctypes.c_int, i64, i64, u32p, u32p]
        L.oracle_estimate.argtypes = [ctypes.c_int, i64, i64, u32p, u32p, ctypes.c_double,
                                      ctypes.c_double, dp, dp, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, dp, ctypes.POINTER(i64), ctypes.c_double,
                                      dp, ctypes.c_int]
        L.oracle_warp.argtypes = [ctypes.c_int, i64, i64, u32p, u32p, ctypes.c_double,
                                  ctypes.c_double, dp, dp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int]
        L.oracle_points.argtypes = [ctypes.c_int, i64, i64, u32p, u32p, ctypes.c_int, u32p]
        L.oracle_det.argtypes = [ctypes.c_int, dp, dp]
        L.oracle_estimate_proj.argtypes = [ctypes.c_int, i64, i64, u32p, u32p, ctypes.c_double, ctypes.c_double,
                                           dp, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, dp, ctypes.POINTER(i64),
                                           ctypes.c_double, dp, ctypes.c_int]
        L.oracle_table_at.argtypes = [dp, ctypes.c_int, ctypes.c_double, i64, dp, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


# --------------------------------------------------------------------------
# Green functions (App. E)
# --------------------------------------------------------------------------

def _half_line_ft(eps: float, gamma: float, tau: np.ndarray) -> np.ndarray:
    """I(tau) = Int_0^inf e^{i s tau} 2Gamma/((s+eps)^2+Gamma^2) ds for tau > 0.

    With beta = eps + i Gamma the Lorentzian is -i [1/(s+beta*) - 1/(s+beta)],
    and F(b) = Int_0^inf e^{i s tau}/(s+b) ds = e^{w} E1(w) with w = -i b tau.
    For b = beta the argument has Re w = Gamma tau > 0 (principal E1).  For
    b = beta* it is w = -Gamma tau - i eps tau, reached from the lower half
    plane (eps > 0); for eps <= 0 the path crosses the negative real axis
    and E1 is continued past its cut: E1 + 2 pi i above the axis, the lower
    boundary value on it.
    """
    from scipy.special import exp1

    tau = np.asarray(tau, dtype=np.float64)
    beta = complex(eps, gamma)
    w_plus = -1j * beta * tau
    w_minus = -1j * np.conj(beta) * tau
    F_plus = np.exp(w_plus) * exp1(w_plus)
    if eps > 0:
        E = exp1(w_minus)
    else:
        on_axis = np.imag(w_minus) == 0.0
        wm = np.where(on_axis, np.real(w_minus) + 0j, w_minus)
        E = exp1(wm) + 2j * np.pi
        # on the axis itself take the boundary value from below
        below = np.conj(exp1(np.real(w_minus) + 0j))
        E = np.where(on_axis, below, E)
    F_minus = np.exp(w_minus) * E
    return -1j * (F_minus - F_plus)


def gf_exact(tau, gamma: float, eps_d: float):
    """Exact g^<(tau), g^>(tau) of the wide-band dot at T = 0, V = 0.

    tau = 0 gives g^<(0) = i(1/2 - arctan(eps_d/Gamma)/pi) and
    g^>(0) = g^<(0) - i.  Negative tau uses g(-tau) = -conj g(tau).
    """
    tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
    a = np.abs(tau)
    pos = a > 0
    gl = np.empty(tau.shape, dtype=np.complex128)
    gg = np.empty(tau.shape, dtype=np.complex128)
    gl0 = 1j * (0.5 - math.atan(eps_d / gamma) / math.pi)
    gl[~pos] = gl0
    gg[~pos] = gl0 - 1j
    if np.any(pos):
        ap = a[pos]
        # g^<(tau) = (i/2pi) Int_0^inf e^{i s tau} A(-s) ds      (w = -s)
        gl_p = 1j / (2 * math.pi) * _half_line_ft(eps_d, gamma, ap)
        # g^>(tau) = (-i/2pi) Int_0^inf e^{-i w tau} A(w) dw = (-i/2pi) conj(I_{-eps})
        gg_p = -1j / (2 * math.pi) * np.conj(_half_line_ft(-eps_d, gamma, ap))
        neg = tau[pos] < 0
        gl_p = np.where(neg, -np.conj(gl_p), gl_p)
        gg_p = np.where(neg, -np.conj(gg_p), gg_p)
        gl[pos] = gl_p
        gg[pos] = gg_p
    return gl, gg


def table_nodes(T: float, L: int) -> np.ndarray:
    """Uniform nodes tau_k = -T + k * 2T/(L-1), k = 0..L-1 (both ends included)."""
    h = 2.0 * T / (L - 1)
    return -T + np.arange(L, dtype=np.float64) * h


def gf_tables(gamma: float, eps_d: float, T: float, L: int = 4096):
    """(g^< table, g^> table, g^<(0)) on ``table_nodes(T, L)``."""
    gl, gg = gf_exact(table_nodes(T, L), gamma, eps_d)
    gl0 = 1j * (0.5 - math.atan(eps_d / gamma) / math.pi)
    return gl, gg, gl0


# --------------------------------------------------------------------------
# Semicircular leads at finite half-bandwidth D and symmetric bias V (App. E)
# --------------------------------------------------------------------------
#
# Hybridisation of both leads, App. E: inside the band |w| < D,
#     Delta(w) = (Gamma / D) (w - i sqrt(D^2 - w^2)),  Gamma(w) = -Im Delta(w),
# g^R = 1 / (w - E_d - Delta); each lead carries Delta / 2.  Lead L has Fermi
# level +V/2, lead R (the one holding site 1) -V/2; T = 0 Fermi functions
# f_L = theta(V/2 - w), f_R = theta(-V/2 - w).  Keldysh functions in the
# textbook normalisation of the charge tables (g^< = i A f; the paper's
# Eq. (lesser_greater_freq) differs by an overall factor, see the reading in
# the design notes):
#     g^<_00 =  i Gamma(w) |g^R|^2 (f_L + f_R)
#     g^>_00 = -i Gamma(w) |g^R|^2 (2 - f_L - f_R)
# and, from the Dyson equation G_01 = G_00 gamma g_11 with the Langreth rule
# (AB)^< = A^R B^< + A^< B^A and gamma^2 g_11 = Delta / 2:
#     gamma g^<_01 =  i f_R Gamma(w) g^R + (Delta^* / 2) g^<_00
#     gamma g^>_01 = -i (1 - f_R) Gamma(w) g^R + (Delta^* / 2) g^>_00.
# Outside the band Gamma(w) = 0 and all four vanish (no bound state exists for
# |E_d| < D - Gamma).  Time domain: g(tau) = Int dw/2pi e^{-i w tau} g(w).
# With w = D sin(theta) the square root becomes Gamma cos(theta) and every
# integrand is smooth in theta between the Fermi steps.

def _lead_spectra(theta, gamma: float, Ed: float, D: float, V: float):
    """[g^<_00, g^>_00, gamma g^<_01, gamma g^>_01](w(theta)) * (dw/dtheta) / 2pi, and w."""
    theta = np.asarray(theta, dtype=np.float64)
    w = D * np.sin(theta)
    G = gamma * np.cos(theta)
    delta = gamma * (np.sin(theta) - 1j * np.cos(theta))
    gR = 1.0 / (w - Ed - delta)
    fL = (w < 0.5 * V).astype(np.float64)
    fR = (w < -0.5 * V).astype(np.float64)
    a2 = np.abs(gR) ** 2
    gl = 1j * G * a2 * (fL + fR)
    gg = -1j * G * a2 * (2.0 - fL - fR)
    cl = 1j * fR * G * gR + 0.5 * np.conj(delta) * gl
    cg = -1j * (1.0 - fR) * G * gR + 0.5 * np.conj(delta) * gg
    jac = D * np.cos(theta) / (2.0 * np.pi)
    return w, np.stack([gl, gg, cl, cg]) * jac


def _theta_breaks(D: float, V: float):
    b = [-0.5 * math.pi]
    if 0.5 * V < D:
        b += sorted({math.asin(-0.5 * V / D), math.asin(0.5 * V / D)})
    return b + [0.5 * math.pi]


def lead_functions(tau, gamma: float, Ed: float, D: float, V: float = 0.0, epsabs: float = 1e-13):
    """[4, len(tau)] complex: g^<_00, g^>_00, gamma g^<_01, gamma g^>_01 at tau, by adaptive
    vector quadrature (scipy quad_vec) of the Fourier integral in theta, split at the Fermi steps."""
    from scipy.integrate import quad_vec

    tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))

    def f(th):
        w, S = _lead_spectra(th, gamma, Ed, D, V)
        z = S[:, None] * np.exp(-1j * w * tau)[None, :]
        return np.concatenate([z.real.ravel(), z.imag.ravel()])

    br = _theta_breaks(D, V)
    tot = np.zeros(8 * tau.size)
    for a, b in zip(br[:-1], br[1:]):
        if b > a:
            val, _err = quad_vec(f, a, b, epsabs=epsabs, epsrel=1e-13, norm="max", limit=200000)
            tot += val
    m = 4 * tau.size
    return (tot[:m] + 1j * tot[m:]).reshape(4, tau.size)


def lead_tables(gamma: float, Ed: float, D: float, V: float, T: float, L: int):
    """Tables of the finite-bandwidth dot on ``table_nodes(T, L)``:
    ((g^<_00, g^>_00, g^<_00(0)), (gamma g^<_01, gamma g^>_01, gamma g^<_01(0)))."""
    nodes = np.concatenate([table_nodes(T, L), [0.0]])
    F = lead_functions(nodes, gamma, Ed, D, V)
    return (F[0, :L], F[1, :L], complex(F[0, L])), (F[2, :L], F[3, :L], complex(F[2, L]))


def landauer_current(gamma: float, Ed: float, D: float, V: float) -> float:
    """Non-interacting current, both spins: (1/pi) Int_{-V/2}^{V/2} Gamma(w)^2 |g^R(w)|^2 dw."""
    from scipy.integrate import quad

    def T(w):
        s = math.sqrt(max(D * D - w * w, 0.0))
        G = gamma / D * s
        den = complex(w - Ed - gamma / D * w, G)
        return G * G / abs(den) ** 2

    a = 0.5 * min(V, 2 * D)
    return quad(T, -a, a, epsabs=1e-15, epsrel=1e-13, limit=500, points=[Ed] if -a < Ed < a else None)[0] / math.pi


def lead_occupation(gamma: float, Ed: float, D: float, V: float) -> float:
    """<n_sigma> = Int dw/2pi Gamma(w) |g^R|^2 (f_L + f_R), by quadrature in w."""
    from scipy.integrate import quad

    def A(w):
        s = math.sqrt(max(D * D - w * w, 0.0))
        G = gamma / D * s
        den = complex(w - Ed - gamma / D * w, G)
        return G / abs(den) ** 2 / (2.0 * math.pi)

    tot = 0.0
    for mu in (0.5 * V, -0.5 * V):
        hi = min(mu, D)
        if hi > -D:
            pts = [Ed] if -D < Ed < hi else None
            tot += quad(A, -D, hi, epsabs=1e-15, epsrel=1e-13, limit=500, points=pts)[0]
    return tot


# --------------------------------------------------------------------------
# Sobol' direction numbers (library primitive: scipy's unscrambled generator)
# --------------------------------------------------------------------------

_V_CACHE: dict = {}


def sobol_direction_numbers(n_dims: int, n_bits: int = 26) -> np.ndarray:
    """uint32 [n_dims, 32]: V[d, j] = X_{2^j, d}, the natural-order point 2^j.

    scipy emits points in Gray-code order, where consecutive outputs differ
    by one direction word: output p XOR output p+1 = V[ctz(p+1)].  So
    V[:, j] = out[2^j - 1] XOR out[2^j].  Words j >= n_bits are left zero
    (the callers never index points at or beyond 2^n_bits).
    """
    key = (n_dims, n_bits)
    if key in _V_CACHE:
        return _V_CACHE[key]
    from scipy.stats import qmc

    V = np.zeros((n_dims, 32), dtype=np.uint32)
    eng = qmc.Sobol(n_dims, scramble=False, bits=32)
    pos = 0
    for j in range(n_bits):
        target = (1 << j) - 1
        if target < pos:
            eng = qmc.Sobol(n_dims, scramble=False, bits=32)
            pos = 0
        if target > pos:
            eng.fast_forward(target - pos)
        pts = np.rint(eng.random(2) * 2.0 ** 32).astype(np.uint64)
        pos = target + 2
        V[:, j] = (pts[0] ^ pts[1]).astype(np.uint32)
    _V_CACHE[key] = V
    return V


def sobol_points(n: int, i0: int, count: int, V: np.ndarray) -> np.ndarray:
    """Unshifted Sobol' integers, Gray-code order: uint32 [count, n]."""
    Vc = np.ascontiguousarray(V[:n], dtype=np.uint32)
    out = np.zeros((count, n), dtype=np.uint32)
    lib().oracle_sobol(n, i0, count, _u32p(Vc), _u32p(out))
    return out


def _family(n: int, V, lattice):
    """(generator words, family code): Sobol' direction numbers V [n, 32] with code 0, or a rank-1
    lattice given as (z [>= n], m) or (z, m, tent) for N = 2^m points: code m, or 64 + m when the
    baker's transform follows the shift."""
    if lattice is None:
        return np.ascontiguousarray(V[:n], dtype=np.uint32), 0
    z, m = lattice[0], int(lattice[1])
    tent = len(lattice) > 2 and bool(lattice[2])
    return np.ascontiguousarray(np.asarray(z, dtype=np.uint32)[:n]), m + (64 if tent else 0)


def warp(n: int, i0: int, count: int, V: np.ndarray, shift: np.ndarray, t: float, tau: float, lattice=None):
    """Warped points: (u [count, n], weight C/p_n [count], in-domain flag [count])."""
    Vc, lm = _family(n, V, lattice)
    S = np.ascontiguousarray(shift[:n], dtype=np.uint32)
    u = np.zeros((count, n))
    w = np.zeros(count)
    ins = np.zeros(count, dtype=np.int32)
    lib().oracle_warp(n, i0, count, _u32p(Vc), _u32p(S), t, tau, _dp(u), _dp(w),
                      ins.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), lm)
    return u, w, ins.astype(bool)


def lattice_points(n: int, i0: int, count: int, z: np.ndarray, m: int, shift: np.ndarray,
                   tent: bool = False) -> np.ndarray:
    """Shifted rank-1 lattice words uint32 [count, n]: ((i z_d mod 2^m) << (32 - m)) + S_d mod 2^32,
    then the baker's transform if tent."""
    Vc, lm = _family(n, None, (z, m, tent))
    S = np.ascontiguousarray(np.asarray(shift, dtype=np.uint32)[:n])
    out = np.zeros((count, n), dtype=np.uint32)
    if lib().oracle_points(n, i0, count, _u32p(Vc), _u32p(S), lm, _u32p(out)) != 0:
        raise ValueError("oracle_points rejected its arguments")
    return out


def lattice_cbc_criterion(z: np.ndarray, m: int, gamma: np.ndarray) -> float:
    """Shift-averaged worst-case error squared of the rank-1 lattice (N = 2^m, generating vector z)
    in the Korobov-type space with smoothness 2 and product weights gamma:
        e^2(z) = -1 + (1/N) sum_{k=0}^{N-1} prod_d (1 + gamma_d 2 pi^2 B_2({k z_d / N})),
    B_2(x) = x^2 - x + 1/6 (the criterion minimised by component-by-component constructions)."""
    N = 1 << m
    k = np.arange(N, dtype=np.int64)
    prod = np.ones(N)
    for d, zd in enumerate(np.asarray(z, dtype=np.int64)):
        x = ((k * zd) % N) / N
        prod *= 1.0 + gamma[d] * 2.0 * math.pi ** 2 * (x * x - x + 1.0 / 6.0)
    return float(prod.mean() - 1.0)


def lattice_cbc(m: int, dims: int, gamma: np.ndarray) -> np.ndarray:
    """Component-by-component construction: z_1 = 1, then each z_d the odd number in [1, N/2]
    (z and N - z give the same points up to reflection) minimising e^2 given z_1..z_{d-1};
    ties (equal up to rounding: e.g. z and its inverse mod N give the same point set) go to the
    smallest z.  Plain O(dims N^2) evaluation (small N only)."""
    N = 1 << m
    k = np.arange(N, dtype=np.int64)
    cand = np.arange(1, N // 2 + 1, 2, dtype=np.int64) if N > 2 else np.array([1], dtype=np.int64)
    z = [1]
    prod = 1.0 + gamma[0] * 2.0 * math.pi ** 2 * ((k / N) ** 2 - k / N + 1.0 / 6.0)
    for d in range(1, dims):
        x = ((k[None, :] * cand[:, None]) % N) / N
        vals = (prod[None, :] * (1.0 + gamma[d] * 2.0 * math.pi ** 2 * (x * x - x + 1.0 / 6.0))).mean(axis=1)
        lo = float(np.min(vals))
        best = int(cand[np.nonzero(vals <= lo + 1e-12 * abs(lo))[0][0]])
        z.append(best)
        xb = ((k * best) % N) / N
        prod = prod * (1.0 + gamma[d] * 2.0 * math.pi ** 2 * (xb * xb - xb + 1.0 / 6.0))
    return np.array(z, dtype=np.uint32)


# --------------------------------------------------------------------------
# Integrand and estimator
# --------------------------------------------------------------------------

def _tab(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64)


def _col(col, L: int):
    """Packed dot-lead tables for the current (None for the charge):
    col = (gamma g^<_01 [L], gamma g^>_01 [L], gamma g^<_01(0))."""
    if col is None:
        return None
    cl, cg, c0 = col
    cl, cg = _tab(cl), _tab(cg)
    if cl.size != 2 * L or cg.size != 2 * L:
        raise ValueError("dot-lead tables must be on the same mesh as the dot tables")
    return np.ascontiguousarray(np.concatenate([cl, cg, [float(np.real(c0)), float(np.imag(c0))]]))


def _cp(a):
    return None if a is None else _dp(a)


def integrand(n: int, u: np.ndarray, t: float, tables, T: float, return_abs: bool = False, alpha: float = 0.0,
              col=None, return_had: bool = False):
    """c(u) of App. E Eq. (integral_gf) at each row of u ([count, n], any time order);
    alpha: quadratic shift of the vertex diagonals (App. E); col: dot-lead tables
    (gamma g^<_01, gamma g^>_01, gamma g^<_01(0)) for the current, None for the charge.
    return_abs adds sum_a |term_a|; return_had adds sum_a of the Hadamard bounds
    prod_rows ||row|| of det M_up and det M_down (finite where det M_down vanishes)."""
    gl, gg, gl0 = tables
    u = np.ascontiguousarray(np.atleast_2d(np.asarray(u, dtype=np.float64)).reshape(-1, n))
    count = u.shape[0]
    gl_t, gg_t = _tab(gl), _tab(gg)
    L = gl_t.size // 2
    out = np.zeros(2 * count)
    ab = np.zeros(count)
    hd = np.zeros(count)
    cp = _col(col, L)
    rc = lib().oracle_integrand(n, count, _dp(u), t, _dp(gl_t), _dp(gg_t), L, T,
                                float(np.real(gl0)), float(np.imag(gl0)), _dp(out), _dp(ab), float(alpha),
                                _cp(cp), _dp(hd) if return_had else None)
    if rc != 0:
        raise ValueError("oracle_integrand rejected its arguments")
    val = out[0::2] + 1j * out[1::2]
    ret = (val,) + ((ab,) if return_abs else ()) + ((hd,) if return_had else ())
    return ret if len(ret) > 1 else val


def det(A: np.ndarray) -> complex:
    """Determinant by the oracle's pivoted LU (for the pins)."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.complex128))
    out = np.zeros(2)
    if lib().oracle_det(A.shape[0], _dp(A.view(np.float64)), _dp(out)) != 0:
        raise ValueError("matrix too large for the oracle")
    return complex(out[0], out[1])


def table_at(table: np.ndarray, T: float, tau: np.ndarray) -> np.ndarray:
    """Linear interpolation of a table on ``table_nodes(T, L)`` at tau."""
    tab = _tab(table)
    tau = np.ascontiguousarray(np.atleast_1d(np.asarray(tau, dtype=np.float64)))
    out = np.zeros(2 * tau.size)
    lib().oracle_table_at(_dp(tab), tab.size // 2, T, tau.size, _dp(tau), _dp(out))
    return out[0::2] + 1j * out[1::2]


def _estimate_chunk(args):
    n, i0, i1, Vc, S, t, tau, gl_t, gg_t, L, T, gl0, alpha, cp, lm = args
    res = np.zeros(4)
    n_in = ctypes.c_int64(0)
    rc = lib().oracle_estimate(n, i0, i1, _u32p(Vc), _u32p(S), t, tau, _dp(gl_t), _dp(gg_t), L, T,
                               float(np.real(gl0)), float(np.imag(gl0)), _dp(res), ctypes.byref(n_in),
                               float(alpha), _cp(cp), lm)
    if rc != 0:
        raise ValueError("oracle_estimate rejected its arguments")
    return res, n_in.value


def estimate(n: int, N: int, shifts: np.ndarray, t: float, tau: float, tables, T: float,
             V: np.ndarray | None = None, threads: int | None = None, i0: int = 0,
             chunk: int = 4096, alpha: float = 0.0, col=None, lattice=None):
    """Per-shift estimates S_k = (1/N) sum_{i=i0}^{i0+N-1} w_i c(u_i), Eq. (warped_int2).
    lattice = (z, m): a rank-1 lattice of 2^m points instead of Sobol' (shifts added mod 2^32).

    shifts: uint32 [K, >= n] digital-shift words.  Returns (S [K] complex,
    n_in [K] int).  Point ranges are split into chunks run on a thread pool
    (the C call releases the GIL); each chunk is a Neumaier sum and the
    chunk totals are combined with math.fsum (exact rounding).
    """
    if V is None and lattice is None:
        V = sobol_direction_numbers(max(n, 1))
    Vc, lm = _family(n, V, lattice)
    gl, gg, gl0 = tables
    gl_t, gg_t = _tab(gl), _tab(gg)
    L = gl_t.size // 2
    cp = _col(col, L)
    shifts = np.atleast_2d(np.asarray(shifts, dtype=np.uint32))
    K = shifts.shape[0]
    jobs = []
    for k in range(K):
        S = np.ascontiguousarray(shifts[k, :n])
        for a in range(i0, i0 + N, chunk):
            b = min(a + chunk, i0 + N)
            jobs.append((k, (n, a, b, Vc, S, t, tau, gl_t, gg_t, L, T, gl0, alpha, cp, lm)))
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(max_workers=threads) as ex:
        results = list(ex.map(_estimate_chunk, [j[1] for j in jobs]))
    re_parts = [[] for _ in range(K)]
    im_parts = [[] for _ in range(K)]
    n_in = np.zeros(K, dtype=np.int64)
    for (k, _), (res, cnt) in zip(jobs, results):
        re_parts[k].extend([res[0], res[2]])
        im_parts[k].extend([res[1], res[3]])
        n_in[k] += cnt
    S = np.array([complex(math.fsum(re_parts[k]), math.fsum(im_parts[k])) / N for k in range(K)])
    return S, n_in


def q_from_sums(S: np.ndarray) -> np.ndarray:
    """Q_n^{(k)} = -2i * S_k (readout of the charge from G^<(t,t) = i<n_up>)."""
    return -2j * np.asarray(S)


def i_from_sums(S: np.ndarray) -> np.ndarray:
    """I_n^{(k)} = -4 Re S_k: current from the dot into lead site 1, both spins.

    Per spin dN_R/dt = i[H, N_R] = -2 gamma Im<c_0^+ c_1>, and with the
    textbook G^<_{01}(t,t) = i<c_1^+ c_0> this is -2 Re(gamma G^<_{01}(t,t));
    S carries gamma G^<_{01} because the measurement column holds gamma g_01."""
    return -4.0 * np.real(np.asarray(S))


def shift_statistics(values: np.ndarray):
    """Mean over shifts and the RQMC error bar std_{ddof=1}/sqrt(K) (App. H)."""
    v = np.asarray(values, dtype=np.float64)
    K = v.size
    return float(np.mean(v)), float(np.std(v, ddof=1) / math.sqrt(K))


def splitmix64(x: int) -> int:
    """One output of the splitmix64 generator for state x (Steele, Lea & Flood 2014)."""
    M = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def shift_words(seed: int, K: int, n_dims: int) -> np.ndarray:
    """Digital-shift words S[k, d] = high 32 bits of splitmix64(seed XOR (k*2^16 + d))."""
    out = np.zeros((K, n_dims), dtype=np.uint32)
    for k in range(K):
        for d in range(n_dims):
            out[k, d] = splitmix64((seed ^ (k * 65536 + d)) & ((1 << 64) - 1)) >> 32
    return out


# --------------------------------------------------------------------------
# Series resummation (App. H): parabola conformal map
# --------------------------------------------------------------------------

def resum_parabola(a, p: float, U: float, invert: bool = False):
    """Conformal resummation of F(U) = sum_n a_n U^n with the parabola transform
    W = -tan^2(sqrt(U/p)), p < 0 (App. H), i.e. W = tanh^2(sqrt(U/|p|)) for U >= 0.

    The inverse map U(W) = |p| atanh(sqrt W)^2 is expanded symbolically (sympy),
    F(U(W)) is re-expanded in W and truncated at the order N of the input, and the
    truncated series is evaluated at W(U).  invert: resum 1/F and return its
    reciprocal.  Returns the value.
    """
    import sympy as sp

    a = [float(x) for x in a]
    N = len(a) - 1
    if invert:  # power series of 1/F by long division
        f = [1.0 / a[0]]
        for k in range(1, N + 1):
            f.append(-sum(a[j] * f[k - j] for j in range(1, k + 1)) / a[0])
    else:
        f = list(a)
    Wsym = sp.Symbol("W", positive=True)
    ser = sp.series(sp.atanh(sp.sqrt(Wsym)) ** 2, Wsym, 0, N + 1).removeO()
    poly = sp.Poly(sp.expand(ser), Wsym)
    c = np.zeros(N + 1)
    for (deg,), coef in poly.terms():
        if deg <= N:
            c[deg] = float(coef) * abs(p)
    b = np.zeros(N + 1)
    power = np.zeros(N + 1)
    power[0] = 1.0
    for k in range(N + 1):
        b += f[k] * power
        power = np.polynomial.polynomial.polymul(power, c)[: N + 1]
        power = np.pad(power, (0, N + 1 - power.size))
    W = math.tanh(math.sqrt(U / abs(p))) ** 2
    val = float(np.polynomial.polynomial.polyval(W, b))
    return 1.0 / val if invert else val


# --------------------------------------------------------------------------
# Learned warp (App. F: learning h from the integrand)
# --------------------------------------------------------------------------

def learn_projection(n: int, M: int, seed: int, t: float, tau: float, tables, T: float, n_bins: int = 100,
                     lam: float = 0.05, floor_frac: float = 1e-3, cells: int = 1024, V=None) -> np.ndarray:
    """Per-dimension CDF tables [n, cells + 1] of the learned warp.

    Samples: the first M Sobol' points shifted by shift_words(seed, 65536, n)[65535]
    (the learning sequence), plain exponential warp; value |w c_n(u)| of the
    in-domain points.  Projection onto each w_m: histogram with n_bins bins
    (sum of values / M per bin).  Smoothing: Gaussian kernel
    exp(-(w - w_l)^2 / lam^2) over the bin centres w_l, evaluated at the cell
    centres; floor at floor_frac x maximum; CDF by cumulative sum.
    """
    if V is None:
        V = sobol_direction_numbers(max(n, 1))
    S = np.array([splitmix64((seed ^ (65535 * 65536 + d)) & ((1 << 64) - 1)) >> 32 for d in range(n)],
                 dtype=np.uint32)
    u, w, ins = warp(n, 0, M, V, S, t, tau)
    x = ((sobol_points(n, 0, M, V) ^ S[None, :]).astype(np.float64)) * 2.0 ** -32
    vals = np.zeros(M)
    if ins.any():
        c = integrand(n, u[ins], t, tables, T)
        vals[ins] = w[ins] * np.abs(c) / M
    return projection_cdf(x, vals, n_bins, lam, floor_frac, cells)


def projection_cdf(x: np.ndarray, vals: np.ndarray, n_bins: int = 100, lam: float = 0.05,
                   floor_frac: float = 1e-3, cells: int = 1024) -> np.ndarray:
    """The projection step of the learned warp (App. F) for samples x [M, n] in [0, 1)^n with
    values vals [M]: per dimension d, the histogram of vals over n_bins equal bins of x_d
    (centres (l + 1/2) / n_bins), smoothed by the Gaussian kernel exp(-(z - w_l)^2 / lam^2)
    normalised over the bin centres, evaluated at the centres z of `cells` equal cells, floored
    at floor_frac x its maximum; returns the cumulative sums [n, cells + 1], 0 .. 1."""
    n = x.shape[1]
    centers = (np.arange(n_bins) + 0.5) / n_bins
    z = (np.arange(cells) + 0.5) / cells
    K = np.exp(-((z[:, None] - centers[None, :]) ** 2) / lam ** 2)
    out = np.zeros((n, cells + 1))
    for d in range(n):
        b = np.clip((x[:, d] * n_bins).astype(np.int64), 0, n_bins - 1)
        hist = np.bincount(b, weights=vals, minlength=n_bins)
        h = (K @ hist) / K.sum(axis=1)
        hmax = h.max()
        h = np.ones(cells) if hmax <= 0 else np.maximum(h, floor_frac * hmax)
        cdf = np.concatenate([[0.0], np.cumsum(h) / h.sum()])
        cdf[-1] = 1.0
        out[d] = cdf
    return out


def _estimate_proj_chunk(args):
    n, i0, i1, Vc, S, t, tau, cdf, cells, gl_t, gg_t, L, T, gl0, alpha, cp = args
    res = np.zeros(4)
    n_in = ctypes.c_int64(0)
    rc = lib().oracle_estimate_proj(n, i0, i1, _u32p(Vc), _u32p(S), t, tau, _dp(cdf), cells, _dp(gl_t), _dp(gg_t),
                                    L, T, float(np.real(gl0)), float(np.imag(gl0)), _dp(res), ctypes.byref(n_in),
                                    float(alpha), _cp(cp), 0)
    if rc != 0:
        raise ValueError("oracle_estimate_proj rejected its arguments")
    return res, n_in.value


def estimate_proj(n: int, N: int, shifts: np.ndarray, t: float, tau: float, cdf: np.ndarray, tables, T: float,
                  V: np.ndarray | None = None, threads: int | None = None, chunk: int = 4096, alpha: float = 0.0,
                  col=None):
    """Per-shift estimates with the learned warp (same contract as ``estimate``)."""
    if V is None:
        V = sobol_direction_numbers(max(n, 1))
    Vc = np.ascontiguousarray(V[:n], dtype=np.uint32)
    cdf = np.ascontiguousarray(np.asarray(cdf, dtype=np.float64)[:n])
    cells = cdf.shape[1] - 1
    gl, gg, gl0 = tables
    gl_t, gg_t = _tab(gl), _tab(gg)
    L = gl_t.size // 2
    cp = _col(col, L)
    shifts = np.atleast_2d(np.asarray(shifts, dtype=np.uint32))
    K = shifts.shape[0]
    jobs = []
    for k in range(K):
        S = np.ascontiguousarray(shifts[k, :n])
        for a in range(0, N, chunk):
            jobs.append((k, (n, a, min(a + chunk, N), Vc, S, t, tau, cdf, cells, gl_t, gg_t, L, T, gl0, alpha,
                             cp)))
    with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
        results = list(ex.map(_estimate_proj_chunk, [j[1] for j in jobs]))
    re_parts = [[] for _ in range(K)]
    im_parts = [[] for _ in range(K)]
    n_in = np.zeros(K, dtype=np.int64)
    for (k, _), (res, cnt) in zip(jobs, results):
        re_parts[k].extend([res[0], res[2]])
        im_parts[k].extend([res[1], res[3]])
        n_in[k] += cnt
    S = np.array([complex(math.fsum(re_parts[k]), math.fsum(im_parts[k])) / N for k in range(K)])
    return S, n_in
