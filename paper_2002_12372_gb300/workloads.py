"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module holds no arithmetic of the QQMC method: it only draws seeded
inputs (shift words, vertex times, request sweeps) and builds one synthetic
Green-function table from a closed form, so that the CUDA path and the CPU
oracle can be fed byte-identical inputs.

Workload shapes follow the paper's single-level-dot calculations (App. C, E,
H): Gamma = 1 (or 0.1), eps_d of a few Gamma, measurement times 5..30 /
Gamma, exponential warp decay tau ~ 1 / Gamma, 2^14..2^22 Sobol' points and
10..32 digitally shifted sequences.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED = 2002123720


@dataclass
class DotConfig:
    """One single-level-dot workload (a row of the benchmark table)."""
    name: str
    gamma: float = 1.0
    eps_d: tuple = (0.0,)
    t_max: float = 10.0
    tau: float = 1.0
    n_table: int = 4096
    orders: tuple = (1, 2, 3, 4)
    n_points: dict = field(default_factory=dict)   # order -> N
    n_shifts: int = 16
    precision: str = "fp64"


def plain_small() -> DotConfig:
    """Plain QQMC, wide band: Gamma=1, eps_d=0, t=10, L=4096, n=1..4, N=2^14, K=16."""
    return DotConfig("plain-n1-4-N2^14-K16", orders=(1, 2, 3, 4), n_points={n: 2 ** 14 for n in range(1, 5)},
                     n_shifts=16)


def plain_scale() -> DotConfig:
    """Plain method at scale: eps_d in {-1,0,1}, n=1..10, N=2^20, K=32, FP64."""
    return DotConfig("plain-eps{-1,0,1}-n1-10-N2^20-K32", eps_d=(-1.0, 0.0, 1.0), orders=tuple(range(1, 11)),
                     n_points={n: 2 ** 20 for n in range(1, 11)}, n_shifts=32)


def batched_uneven() -> DotConfig:
    """One launch over n=2..12 with N_n = 2^max(14, 24-n), K=16, FP64."""
    return DotConfig("batched-n2-12-N2^22..2^14-K16", orders=tuple(range(2, 13)),
                     n_points={n: 2 ** max(14, 24 - n) for n in range(2, 13)}, n_shifts=16)


def precision_mixed() -> DotConfig:
    """n=6..12, N=2^22, K=16, FP32 tables and Schur updates, FP64 sums."""
    return DotConfig("mixed-n6-12-N2^22-K16", orders=tuple(range(6, 13)), n_points={n: 2 ** 22 for n in range(6, 13)},
                     n_shifts=16, precision="mixed")


def shift_words(seed: int, n_shifts: int, n_dims: int) -> np.ndarray:
    """Seeded digital-shift words, uint32 [n_shifts, n_dims] (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2 ** 32, size=(n_shifts, n_dims), dtype=np.uint64).astype(np.uint32)


def ordered_times(seed: int, count: int, n: int, t: float) -> np.ndarray:
    """count x n vertex times with t > u_1 > ... > u_n > 0 (uniform on the simplex)."""
    rng = np.random.default_rng(seed)
    u = np.sort(rng.uniform(0.0, t, size=(count, n)), axis=1)[:, ::-1]
    return np.ascontiguousarray(u)


def synthetic_tables(seed: int, L: int, T: float, components: int = 3):
    """A seeded Keldysh Green function on the mesh tau_k = -T + k 2T/(L-1).

    A mixture of Lorentzian levels j (energy e_j, width gam_j, weight a_j,
    sum a_j = 1) each with its own flat occupation f_j:
        g^<(tau) =  i sum_j a_j f_j     e^{-i e_j tau - gam_j |tau|}
        g^>(tau) = -i sum_j a_j (1-f_j) e^{-i e_j tau - gam_j |tau|}
    i.e. a positive spectral function with an energy-dependent distribution,
    a valid non-interacting Keldysh function out of equilibrium.  (A single
    component is an infinite-temperature state in which every interaction
    correction vanishes; the mixture is not.)  Values are computed on the
    nodes with tau > 0 and mirrored exactly, g(-tau) = -conj g(tau).
    Returns (g_lesser [L], g_greater [L], g0 = g^<(0), parameters).
    """
    rng = np.random.default_rng(seed)
    e = rng.uniform(-1.5, 1.5, components)
    gam = rng.uniform(0.05, 0.3, components)
    f = rng.uniform(0.05, 0.95, components)
    a = rng.uniform(0.2, 1.0, components)
    a = a / a.sum()
    h = 2.0 * T / (L - 1)
    tau = -T + np.arange(L, dtype=np.float64) * h
    pos = np.arange(L // 2, L)
    z = np.exp(-1j * e[None, :] * tau[pos, None] - gam[None, :] * np.abs(tau[pos, None]))
    gl = np.empty(L, dtype=np.complex128)
    gg = np.empty(L, dtype=np.complex128)
    gl[pos] = 1j * (z * (a * f)[None, :]).sum(axis=1)
    gg[pos] = -1j * (z * (a * (1.0 - f))[None, :]).sum(axis=1)
    mirror = L - 1 - pos
    gl[mirror] = -np.conj(gl[pos])
    gg[mirror] = -np.conj(gg[pos])
    g0 = 1j * float(np.sum(a * f))
    return gl, gg, g0, (e, gam, f, a)


@dataclass
class Request:
    arrival_s: float
    gamma: float
    eps_d: float
    U: float
    t_max: float
    n_max: int
    n_points: int
    n_shifts: int


def serving_sweep(seed: int = SEED, n_requests: int = 256, rate_hz: float = 50.0, log2_min: int = 16,
                  log2_max: int = 22, n_shifts: int = 16) -> list:
    """Gate/interaction sweep: eps_d ~ U[-3,3], U/Gamma in {1,2,4}, t_max in {5,10,20},
    n_max ~ U{4..10}, N = 2^floor(U[log2_min, log2_max]), Poisson arrivals at rate_hz."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += float(rng.exponential(1.0 / rate_hz))
        out.append(Request(arrival_s=t, gamma=1.0, eps_d=float(rng.uniform(-3.0, 3.0)),
                           U=float(rng.choice([1.0, 2.0, 4.0])), t_max=float(rng.choice([5.0, 10.0, 20.0])),
                           n_max=int(rng.integers(4, 11)),
                           n_points=int(2 ** math.floor(rng.uniform(log2_min, log2_max + 1e-9))),
                           n_shifts=n_shifts))
    return out


def synthetic_projection(seed: int, n: int, cells: int = 1024) -> np.ndarray:
    """Seeded warp tables [n, cells + 1]: per dimension the cumulative sums of a
    positive smooth density on `cells` equal cells (1 + a sin(2 pi (f z + phi))
    with a in [0.3, 0.9]), normalised to end at 1."""
    rng = np.random.default_rng(seed)
    z = (np.arange(cells) + 0.5) / cells
    out = np.zeros((n, cells + 1))
    for d in range(n):
        a, f, phi = rng.uniform(0.3, 0.9), rng.uniform(0.5, 3.0), rng.uniform(0.0, 1.0)
        h = 1.0 + a * np.sin(2 * np.pi * (f * z + phi))
        out[d, 1:] = np.cumsum(h) / h.sum()
        out[d, -1] = 1.0
    return out


def synthetic_column_tables(seed: int, L: int, T: float, components: int = 3):
    """Seeded dot-lead tables for the current on the mesh tau_k = -T + k 2T/(L-1):
    c^<(tau) = sum_j b_j e^{-i e_j tau - gam_j |tau|} and c^> likewise with its own
    complex amplitudes (|b| ~ 0.1), a smooth complex function with the decay
    scales of the dot tables.  Returns (c_lesser [L], c_greater [L], c0 = c^<(0))."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(-1.5, 1.5, components)
    gam = rng.uniform(0.05, 0.3, components)
    bl = 0.1 * (rng.normal(size=components) + 1j * rng.normal(size=components))
    bg = 0.1 * (rng.normal(size=components) + 1j * rng.normal(size=components))
    tau = -T + np.arange(L, dtype=np.float64) * (2.0 * T / (L - 1))
    z = np.exp(-1j * e[None, :] * tau[:, None] - gam[None, :] * np.abs(tau[:, None]))
    return z @ bl, z @ bg, complex(bl.sum())


@dataclass
class CurrentConfig:
    """Finite-bias current through the dot with semicircular leads (App. C/E current
    calculations): D = 2, Gamma = 0.1, t = 10 / Gamma, exponential warp tau = 1.5 / Gamma,
    orders 1..10, V = U / 7 at U = 6 Gamma. E_d and alpha are chosen so that the Hartree term
    vanishes: alpha is the level's occupation Im g^<(0), about 0.27 at this E_d (the value kept
    here); the current benchmark reads the exact one from the problem's own tables."""
    name: str = "current-D2-Gamma0.1-t100-n1-10"
    gamma: float = 0.1
    half_bandwidth: float = 2.0
    E_d: float = 0.09
    alpha: float = 0.27
    U: float = 0.6
    bias: float = 0.6 / 7.0
    t_max: float = 100.0
    tau: float = 15.0
    n_table: int = 4096
    orders: tuple = tuple(range(1, 11))
    n_shifts: int = 10
