"""Work accounting for the roofline of the determinant kernel.

``flops_per_point(n, F, pairs, precision)`` counts the real floating-point operations
the kernel executes for one in-domain point of order n (complex FMA c -/+ a*b
= 8, complex product = 6, complex reciprocal = 6, the accumulation of a leaf
term = 8), following the kernel's loops exactly, for either Keldysh-sum tree:
the single-vertex tree (level 0 with vertex 1 eliminated, a depth-first tree
over a_2.., breadth-first levels below each leaf, the per-lane flat phase over
the last F vertices) or the pair-block tree (a root per a_2 with vertices 1
and 2 eliminated by their 2x2 pivot block, a depth-first tree of vertex pairs,
breadth-first pair levels, the per-lane flat phase).  ``w_naive`` is the cost of the plain form
(one LU per Keldysh configuration of M_up and of M_down), for an
algorithm-independent "effective" rate.

Peaks of the GB300 CUDA cores (the path is not a dense contraction and does
not use tensor cores): 152 SMs at up to 2070 MHz; per SM and clock 128 FP32
FMA lanes and 2 FP64 FMA lanes.  The roofline divides by the FMA throughput
measured on this part with the library's own register-resident microbenchmark
(qqmc_fma_peak): 1.2558 TFLOP/s FP64 (99.8 % of the unit-count figure) and
77.32 TFLOP/s FP32 (96 %).
"""
from __future__ import annotations

SMS = 152
SM_MAX_MHZ = 2070.0
FP32_LANES = 128
FP64_LANES = 2


# Measured FMA throughput on GB300 (qqmc_fma_peak: register-resident FMA chains on 64 warps per SM,
# best of three ~1 s runs, SM clock 2070 MHz throughout, no throttle reason), from
#   python bench.py --config peaks --steps 3
MEASURED_TFLOPS = {"fp64": 1.2558, "mixed": 77.32}


def derived_tflops(precision: str, mhz: float = SM_MAX_MHZ) -> float:
    """Unit count x clock: SMs x FMA lanes x 2 flops x clock."""
    lanes = FP64_LANES if precision == "fp64" else FP32_LANES
    return SMS * lanes * 2.0 * mhz * 1e6 / 1e12


def peak_tflops(precision: str) -> float:
    """The roofline denominator: the measured FMA throughput of the pipe that bounds the kernel."""
    return MEASURED_TFLOPS["fp64" if precision == "fp64" else "mixed"]


CFMS, CMUL, CRCP, ACC = 8, 6, 6, 8
CFMA, CSUB = 8, 2

LEAF_MAX = 6


def _tree_shape(n: int):
    """(R_r, depth-first pair levels, leaf vertices, both roots in one group?) of order n."""
    Rr = n - 2
    dfl = (Rr - LEAF_MAX + 1) // 2 if Rr > LEAF_MAX else 0
    return Rr, dfl, Rr - 2 * dfl, Rr <= 4


def _bfs_levels(Rleaf: int, RF: int) -> int:
    return (Rleaf - RF + 1) // 2 if Rleaf > RF else 0


# leaf formulas: lone last vertex (no reciprocal) and last vertex pair (no reciprocal)
LEAF_TERM = 2 * CMUL + CFMS + CSUB + CFMS + 3 * CMUL
LEAF_PAIR = (CMUL + CFMS) + 4 * (CMUL + CFMS) + 2 * (CMUL + CFMA) + 2 * CSUB + CFMS + 3 * CMUL
PIVOT = CMUL + CFMS + CRCP  # det of a 2x2 block and its reciprocal
W_COL = 2 * (CMUL + CFMS + CMUL)  # B^-1 (e_p; e_q) for one column, adjugate form


def _flat_term(F: int) -> float:
    """One lane, one choice path over F vertices (first pair fused with the gather)."""
    if F == 1:
        return LEAF_TERM
    if F == 2:
        return LEAF_PAIR
    M = F
    fl = PIVOT + CMUL + M * W_COL + (M * M - 2) * 2 * CFMS
    if M == 3:
        return fl + LEAF_TERM
    if M == 4:
        return fl + LEAF_PAIR
    return fl + PIVOT + CMUL + 3 * W_COL + 7 * 2 * CFMS + LEAF_TERM  # M == 5


def _root(n: int) -> float:
    nb = n - 1
    return PIVOT + nb * 4 * (CMUL + CFMS + CMUL) + (2 * nb + 4 * (nb * nb - nb)) * 2 * CFMS


NODE_PIVOTS = 4 * (PIVOT + 4 * CMUL)  # B^-1 and det B of a node's four children, once per node
W_BINV = 2 * (CMUL + CFMA)  # (W0; W1) = B^-1 (e_p; e_q) for one column from a stored B^-1


def _child_lanecol(S2: int) -> float:
    """Depth-first pair step, one child of S2 rows (every entry formed), pivot data stored."""
    return CMUL + S2 * W_BINV + S2 * S2 * 2 * CFMS


def _child_general(S2: int, stored_pivot: bool = False) -> float:
    """General pair step, per child: pivot (unless stored), scaled pivot rows, the used entries."""
    return (0 if stored_pivot else PIVOT + 4 * CMUL) + CMUL + S2 * W_BINV + S2 * (S2 - 1) * 2 * CFMS


def _flops_pairs(n: int, RF: int) -> float:
    """Pair-block tree: root (vertices 1, 2) per a_2, depth-first pair levels, then
    per leaf group the breadth-first pair levels and the per-lane flat phase."""
    fl = (n * (n + 1) // 2) * 12  # pair interpolation: 2 complex lerps + position arithmetic
    if n == 1:
        return fl + 3 * CMUL + CSUB + ACC
    if n == 2:
        return fl + 2 * LEAF_PAIR + CSUB + ACC
    Rr, dfl, Rleaf, g = _tree_shape(n)
    fl += 2 * _root(n)
    for l in range(1, dfl + 1):  # level l is built 2 * 4^(l-1) * 4 times per point
        S2 = 2 * (Rr - 2 * l) + 2
        per = _child_lanecol(S2) if S2 <= 32 else _child_general(S2, stored_pivot=True)
        fl += 2 * 4 ** (l - 1) * (NODE_PIVOTS + 4 * per)
    B = _bfs_levels(Rleaf, RF)
    F = Rleaf - 2 * B
    nodes = 2 if g else 1
    leaf = 0.0
    for b in range(1, B + 1):
        nodes *= 4
        leaf += nodes * _child_general(2 * (Rleaf - 2 * b) + 2)
    leaf += (nodes << F) * (_flat_term(F) + ACC)
    groups = 1 if g else 2 * 4 ** dfl
    return fl + groups * leaf


TREE_LEAF = 5


def _flat_lane_single(Rf: int) -> float:
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


def _flat_pair_single(Rf: int) -> float:
    """One lane resolving Rf vertices of a node along the two choice paths that differ only
    in the last vertex: both of its rows and columns ride through the first Rf - 1
    eliminations (the entries joining its two copies, like those joining the measurement
    copies, are skipped), then one leaf term per path."""
    M = Rf + 2
    fl = CRCP + CMUL + M * CMUL + (M * M - 4) * CFMS
    for q in range(1, Rf - 1):
        rows = M - q
        fl += CRCP + CMUL + rows * CMUL + (rows * rows - 4) * CFMS
    return fl + 2 * (LEAF_TERM + 2 + ACC)


def _flops_single(n: int, RF: int, paired: bool = False) -> float:
    """Single-vertex tree: level 0 (vertex 1 eliminated), the depth-first tree over a_2..,
    the breadth-first levels below each leaf and the per-lane flat phase.  paired: the
    FP32 kernel's sibling leaves at flat depth 5, resolved together by the two half-warps
    with two choice paths per lane."""
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
    if paired and levels >= 1 and B == 0 and Rf == TREE_LEAF:
        leaf += 2 ** (Rleaf - 1) * _flat_pair_single(Rf)
    else:
        leaf += 2 ** Rleaf * _flat_lane_single(Rf)
    return fl + 2 ** levels * leaf


def flops_per_point(n: int, RF: int = 2, pairs: bool = False, precision: str = "fp64") -> float:
    """Real flops per in-domain point of order n with tuned flat depth RF, on the
    single-vertex tree or (pairs) the pair-block tree, in the given precision's kernel."""
    if pairs:
        return _flops_pairs(n, RF)
    return _flops_single(n, RF, paired=precision != "fp64")


def w_naive(n: int) -> float:
    """2^n (8/3)(n^3 + (n+1)^3): one LU of M_down (n x n) and of M_up per configuration."""
    return 2.0 ** n * (8.0 / 3.0) * (n ** 3 + (n + 1) ** 3)
