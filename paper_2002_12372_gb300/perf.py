"""Work accounting for the roofline of the determinant kernel.

``flops_per_point(n, F)`` counts the real floating-point operations the
kernel executes for one in-domain point of order n (complex FMA c - a*b = 8,
complex product = 6, complex reciprocal = 6, the two-sum accumulation of a
leaf term = 8), following the kernel's loops exactly: level 0 (vertex 1
eliminated), the depth-first Schur tree over a_2.., and the per-lane flat
phase over the last F vertices.  ``w_naive`` is the cost of the plain form
(one LU per Keldysh configuration of M_up and of M_down), for an
algorithm-independent "effective" rate.

Peaks of the GB300 CUDA cores (the path is not a dense contraction and does
not use tensor cores): 152 SMs at up to 2070 MHz; per SM and clock 128 FP32
FMA lanes and 2 FP64 FMA lanes (the FP64 rate measured by an FMA-chain
microbenchmark on this part, 1.20 TFLOP/s at ~1.97 GHz, fixes the latter).
"""
from __future__ import annotations

SMS = 152
SM_MAX_MHZ = 2070.0
FP32_LANES = 128
FP64_LANES = 2


def peak_tflops(precision: str, mhz: float = SM_MAX_MHZ) -> float:
    lanes = FP64_LANES if precision == "fp64" else FP32_LANES
    return SMS * lanes * 2.0 * mhz * 1e6 / 1e12


CFMS, CMUL, CRCP, ACC = 8, 6, 6, 8


TREE_LEAF = 5


def _flat_lane(Rf: int) -> float:
    """One lane resolving Rf vertices of a node along one choice path."""
    if Rf == 0:
        return 2 * CMUL + 2 + ACC
    M = Rf + 1
    fl = CRCP + CMUL + M * CMUL + (M * M - 2) * CFMS
    for q in range(1, Rf):
        p = q + 1
        rows = 2 + (M - 1 - p)
        fl += CRCP + CMUL + rows * CMUL + (rows * rows - 2) * CFMS
    return fl + 2 * CMUL + 2 + ACC


def flops_per_point(n: int, RF: int = 2) -> float:
    """Real flops per in-domain point of order n with RF vertices per lane."""
    R0 = n - 1
    S0 = 2 * n
    fl = 0.0
    # pair interpolation: 2 complex lerps + position arithmetic
    fl += (n * (n + 1) // 2) * 12
    # level 0: one cfms per entry, the right factors M(1, .) / d once per block index
    # (2 cmul each), one reciprocal
    fl += S0 * S0 * CFMS + 2 * n * CMUL + CRCP
    levels = R0 - TREE_LEAF if R0 > TREE_LEAF else 0
    Rleaf = R0 - levels
    # depth-first tree: level l -> l+1 computed 2^(l+1) times in the walk; children wider
    # than a warp (S2 > 32) take the general step, which skips the never-read entries that
    # join a row to its other copy (S2 of the S2^2)
    for l in range(levels):
        S2 = 2 * (R0 - l)
        upd = S2 * (S2 - 1) if S2 > 32 else S2 * S2
        fl += 2 ** (l + 1) * (S2 * CMUL + upd * CFMS + CRCP + CMUL)
    # below each tree leaf: breadth-first levels (the general step, S2 (S2 - 1) updates),
    # then the per-lane flat phase
    B = Rleaf - RF if Rleaf > RF else 0
    Rf = Rleaf - B
    leaf = 0.0
    for lb in range(B):
        S2 = 2 * (Rleaf - lb)
        leaf += 2 ** (lb + 1) * (CRCP + CMUL + S2 * CMUL + S2 * (S2 - 1) * CFMS)
    leaf += 2 ** Rleaf * _flat_lane(Rf)
    return fl + 2 ** levels * leaf


def w_naive(n: int) -> float:
    """2^n (8/3)(n^3 + (n+1)^3): one LU of M_down (n x n) and of M_up per configuration."""
    return 2.0 ** n * (8.0 / 3.0) * (n ** 3 + (n + 1) ** 3)
