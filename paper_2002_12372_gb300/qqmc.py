"""Thin ctypes binding of the QQMC C ABI (``include/qqmc.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library ``_build/libqqmc.so``.  If the library is missing, importing the
functions raises -- there is no CPU fallback.

The functions keep the C names (``qqmc_create_problem``, ``qqmc_integrate``,
``qqmc_submit``, ``qqmc_poll`` ...); a few helpers at the bottom wrap them
with numpy buffers.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libqqmc.so")

QQMC_OK = 0
QQMC_PENDING = 1
QQMC_RUNNING = 2
QQMC_E_INVAL = -1
QQMC_E_RANGE = -2
QQMC_E_NOMEM = -3
QQMC_E_CUDA = -4
QQMC_E_BUSY = -5
QQMC_E_TIMEOUT = -6
QQMC_E_CANCELLED = -7
QQMC_E_NOTFOUND = -8
QQMC_E_NONFINITE = -9
QQMC_MAX_ORDER = 22
QQMC_PREC_FP64 = 0
QQMC_PREC_MIXED = 1
QQMC_TUNE_PAIRS = 16
QQMC_ELIM_AUTO = 0
QQMC_ELIM_PAIRS = 1
QQMC_ELIM_SINGLE = 2
QQMC_OBS_CHARGE = 0
QQMC_OBS_CURRENT = 1

# Every symbol the header declares (checked by the tests against the library).
EXPORTED = [
    "qqmc_create_problem", "qqmc_create_problem_tables", "qqmc_destroy_problem", "qqmc_problem_tables",
    "qqmc_integrate", "qqmc_plan_create", "qqmc_plan_launch", "qqmc_plan_results", "qqmc_plan_destroy",
    "qqmc_plan_kernel_count", "qqmc_plan_timing", "qqmc_set_tuning", "qqmc_get_tuning", "qqmc_direction_numbers",
    "qqmc_shift_words", "qqmc_sobol_points", "qqmc_warp_points", "qqmc_integrand", "qqmc_server_create",
    "qqmc_submit", "qqmc_poll", "qqmc_cancel", "qqmc_server_destroy", "qqmc_last_error",
    "qqmc_integrate_noalloc", "qqmc_plan_chunk_sums", "qqmc_resum_parabola", "qqmc_set_projection",
    "qqmc_learn_projection", "qqmc_set_current_tables", "qqmc_problem_current_tables", "qqmc_set_lattice",
    "qqmc_lattice_cbc", "qqmc_set_stack_policy", "qqmc_plan_device_span", "qqmc_request_state",
    "qqmc_set_elimination", "qqmc_elimination", "qqmc_fma_peak",
]


class qqmc_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("eps_d", ctypes.c_double), ("t_max", ctypes.c_double),
                ("tau", ctypes.c_double), ("n_table", ctypes.c_int32), ("observable", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("alpha", ctypes.c_double), ("half_bandwidth", ctypes.c_double),
                ("bias", ctypes.c_double)]


class qqmc_result(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("n_shifts", ctypes.c_int32), ("n_points", ctypes.c_uint64),
                ("q_mean", ctypes.c_double), ("q_err", ctypes.c_double), ("q_imag_absmax", ctypes.c_double),
                ("n_in_domain", ctypes.c_uint64), ("device_ms", ctypes.c_double), ("n_nonfinite", ctypes.c_uint64)]


class qqmc_item(ctypes.Structure):
    _fields_ = [("problem", ctypes.c_void_p), ("order", ctypes.c_int32), ("n_shifts", ctypes.c_int32),
                ("n_points", ctypes.c_uint64), ("first_index", ctypes.c_uint64),
                ("shift_words", ctypes.POINTER(ctypes.c_uint32))]


class qqmc_server_opts(ctypes.Structure):
    _fields_ = [("device_memory_limit", ctypes.c_uint64), ("max_queue", ctypes.c_int32),
                ("max_batch_items", ctypes.c_int32), ("precision", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("request_timeout_s", ctypes.c_double)]


class qqmc_request(ctypes.Structure):
    _fields_ = [("params", qqmc_params), ("n_max", ctypes.c_int32), ("n_shifts", ctypes.c_int32),
                ("n_points", ctypes.c_uint64), ("U", ctypes.c_double)]


class qqmc_series(ctypes.Structure):
    _fields_ = [("n_max", ctypes.c_int32), ("status", ctypes.c_int32),
                ("q", ctypes.c_double * (QQMC_MAX_ORDER + 1)), ("q_err", ctypes.c_double * (QQMC_MAX_ORDER + 1)),
                ("series_sum", ctypes.c_double), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("n_in_domain", ctypes.c_uint64), ("batch", ctypes.c_uint64), ("device_start_ns", ctypes.c_uint64),
                ("device_end_ns", ctypes.c_uint64)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libqqmc.so (built by ``paper_2002_12372_gb300.build``).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libqqmc.so not found at %s: build it with paper_2002_12372_gb300.build.build() "
                           "(the QQMC path has no CPU fallback)" % path)
    L = ctypes.CDLL(path)
    vp, dp, u32p, i32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint32), \
        ctypes.POINTER(ctypes.c_int32)
    P = ctypes.POINTER
    sig = {
        "qqmc_create_problem": [P(qqmc_params), P(vp)],
        "qqmc_create_problem_tables": [P(qqmc_params), dp, dp, ctypes.c_double, ctypes.c_double, P(vp)],
        "qqmc_destroy_problem": [vp],
        "qqmc_problem_tables": [vp, dp, dp, dp],
        "qqmc_integrate": [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, u32p, dp, P(qqmc_result)],
        "qqmc_plan_create": [P(qqmc_item), ctypes.c_int, ctypes.c_int, P(vp)],
        "qqmc_plan_launch": [vp, vp, ctypes.c_int],
        "qqmc_plan_results": [vp, P(qqmc_result), dp],
        "qqmc_plan_destroy": [vp],
        "qqmc_plan_kernel_count": [vp],
        "qqmc_plan_timing": [vp, dp, dp],
        "qqmc_set_tuning": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
        "qqmc_get_tuning": [ctypes.c_int, ctypes.c_int, i32p, i32p],
        "qqmc_direction_numbers": [ctypes.c_int, u32p],
        "qqmc_shift_words": [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, u32p],
        "qqmc_sobol_points": [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, u32p, u32p],
        "qqmc_warp_points": [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, u32p, dp, dp, i32p],
        "qqmc_integrand": [vp, ctypes.c_int, ctypes.c_uint64, dp, ctypes.c_int, dp],
        "qqmc_server_create": [P(qqmc_server_opts), P(vp)],
        "qqmc_submit": [vp, P(qqmc_request), P(ctypes.c_uint64)],
        "qqmc_poll": [vp, ctypes.c_uint64, P(qqmc_series)],
        "qqmc_cancel": [vp, ctypes.c_uint64],
        "qqmc_server_destroy": [vp],
        "qqmc_last_error": [ctypes.c_char_p, ctypes.c_size_t],
        "qqmc_integrate_noalloc": [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp],
        "qqmc_plan_chunk_sums": [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, dp],
        "qqmc_resum_parabola": [dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp, dp],
        "qqmc_set_projection": [vp, ctypes.c_int, dp, ctypes.c_int],
        "qqmc_learn_projection": [vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_int, dp],
        "qqmc_set_current_tables": [vp, dp, dp, ctypes.c_double, ctypes.c_double],
        "qqmc_set_lattice": [vp, ctypes.c_int, u32p, ctypes.c_int, ctypes.c_int],
        "qqmc_set_stack_policy": [ctypes.c_int, ctypes.c_int],
        "qqmc_lattice_cbc": [ctypes.c_int, ctypes.c_int, dp, u32p],
        "qqmc_problem_current_tables": [vp, dp, dp, dp],
        "qqmc_plan_device_span": [vp, P(ctypes.c_uint64), P(ctypes.c_uint64)],
        "qqmc_request_state": [vp, ctypes.c_uint64],
        "qqmc_set_elimination": [vp, ctypes.c_int],
        "qqmc_elimination": [vp, ctypes.c_int],
        "qqmc_fma_peak": [ctypes.c_int, ctypes.c_double, dp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    _lib = L
    return L


class QQMCError(RuntimeError):
    def __init__(self, code: int, where: str):
        buf = ctypes.create_string_buffer(512)
        load().qqmc_last_error(buf, 512)
        super().__init__("%s failed (%d): %s" % (where, code, buf.value.decode(errors="replace")))
        self.code = code


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise QQMCError(rc, where)
    return rc


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


# ----------------------------------------------------------------- C names

def qqmc_create_problem(params: qqmc_params) -> int:
    out = ctypes.c_void_p()
    _check(load().qqmc_create_problem(ctypes.byref(params), ctypes.byref(out)), "qqmc_create_problem")
    return out.value


def qqmc_create_problem_tables(params: qqmc_params, g_lesser: np.ndarray, g_greater: np.ndarray, g0: complex) -> int:
    gl = np.ascontiguousarray(np.asarray(g_lesser, dtype=np.complex128)).view(np.float64)
    gg = np.ascontiguousarray(np.asarray(g_greater, dtype=np.complex128)).view(np.float64)
    if gl.size != 2 * params.n_table or gg.size != 2 * params.n_table:
        raise ValueError("tables must have n_table entries")
    out = ctypes.c_void_p()
    _check(load().qqmc_create_problem_tables(ctypes.byref(params), _ptr(gl, ctypes.c_double),
                                             _ptr(gg, ctypes.c_double), float(np.real(g0)), float(np.imag(g0)),
                                             ctypes.byref(out)), "qqmc_create_problem_tables")
    return out.value


def qqmc_destroy_problem(pr: int) -> None:
    load().qqmc_destroy_problem(ctypes.c_void_p(pr))


def qqmc_problem_tables(pr: int, L: int):
    gl = np.zeros(2 * L)
    gg = np.zeros(2 * L)
    g0 = np.zeros(2)
    _check(load().qqmc_problem_tables(ctypes.c_void_p(pr), _ptr(gl, ctypes.c_double), _ptr(gg, ctypes.c_double),
                                      _ptr(g0, ctypes.c_double)), "qqmc_problem_tables")
    return gl.view(np.complex128), gg.view(np.complex128), complex(g0[0], g0[1])


def qqmc_set_current_tables(pr: int, c_lesser: np.ndarray, c_greater: np.ndarray, c0: complex) -> None:
    """Dot-lead tables gamma g^<_01, gamma g^>_01 on the problem's full mesh (L complex values each)."""
    cl = np.ascontiguousarray(np.asarray(c_lesser, dtype=np.complex128)).view(np.float64)
    cg = np.ascontiguousarray(np.asarray(c_greater, dtype=np.complex128)).view(np.float64)
    if cl.size != cg.size or cl.size % 4:
        raise ValueError("dot-lead tables must have the problem's n_table entries")
    _check(load().qqmc_set_current_tables(ctypes.c_void_p(pr), _ptr(cl, ctypes.c_double), _ptr(cg, ctypes.c_double),
                                          float(np.real(c0)), float(np.imag(c0))), "qqmc_set_current_tables")


def qqmc_set_lattice(pr: int, log2_n: int, z: np.ndarray | None, bakers: bool = False) -> None:
    """Rank-1 lattice of 2^log2_n points with generating vector z (None: back to Sobol');
    bakers: apply the baker's transform after the shift."""
    if z is None:
        _check(load().qqmc_set_lattice(ctypes.c_void_p(pr), 0, None, 0, 0), "qqmc_set_lattice")
        return
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.uint32))
    _check(load().qqmc_set_lattice(ctypes.c_void_p(pr), log2_n, _ptr(zz, ctypes.c_uint32), zz.size, int(bakers)),
           "qqmc_set_lattice")


def qqmc_set_stack_policy(precision: int, min_order: int) -> None:
    """Split tree stack from order min_order (<= 0: built-in default)."""
    _check(load().qqmc_set_stack_policy(precision, min_order), "qqmc_set_stack_policy")


def qqmc_lattice_cbc(log2_n: int, dims: int, gamma) -> np.ndarray:
    g = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64)[:dims])
    z = np.zeros(dims, dtype=np.uint32)
    _check(load().qqmc_lattice_cbc(log2_n, dims, _ptr(g, ctypes.c_double), _ptr(z, ctypes.c_uint32)),
           "qqmc_lattice_cbc")
    return z


def qqmc_problem_current_tables(pr: int, L: int):
    """(gamma g^<_01, gamma g^>_01 at nodes 0..L/2, gamma g^<_01(0))."""
    cl = np.zeros(2 * (L // 2 + 1))
    cg = np.zeros(2 * (L // 2 + 1))
    c0 = np.zeros(2)
    _check(load().qqmc_problem_current_tables(ctypes.c_void_p(pr), _ptr(cl, ctypes.c_double),
                                              _ptr(cg, ctypes.c_double), _ptr(c0, ctypes.c_double)),
           "qqmc_problem_current_tables")
    return cl.view(np.complex128), cg.view(np.complex128), complex(c0[0], c0[1])


def qqmc_integrate(pr: int, order: int, n_points: int, n_shifts: int, precision: int = QQMC_PREC_FP64,
                   shift_words: np.ndarray | None = None):
    """Returns (qqmc_result, per_shift S_k as complex array [n_shifts])."""
    sw = None if shift_words is None else np.ascontiguousarray(np.asarray(shift_words, dtype=np.uint32)[:, :order])
    per = np.zeros(2 * n_shifts)
    res = qqmc_result()
    _check(load().qqmc_integrate(ctypes.c_void_p(pr), order, n_points, n_shifts, precision,
                                 _ptr(sw, ctypes.c_uint32), _ptr(per, ctypes.c_double), ctypes.byref(res)),
           "qqmc_integrate")
    return res, per.view(np.complex128)


class Plan:
    """Batched device-resident execution (qqmc_plan_*)."""

    def __init__(self, items, precision: int = QQMC_PREC_FP64):
        """items: list of (problem, order, n_shifts, n_points[, shift_words[, first_index]])."""
        self._keep = []
        arr = (qqmc_item * len(items))()
        self.n_shifts = []
        for i, it in enumerate(items):
            pr, order, K, N = it[:4]
            sw = it[4] if len(it) > 4 else None
            first = it[5] if len(it) > 5 else 0
            arr[i].problem = pr
            arr[i].order = order
            arr[i].n_shifts = K
            arr[i].n_points = N
            arr[i].first_index = first
            if sw is not None:
                sw = np.ascontiguousarray(np.asarray(sw, dtype=np.uint32)[:, :order])
                self._keep.append(sw)
                arr[i].shift_words = sw.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
            self.n_shifts.append(K)
        self.n_items = len(items)
        out = ctypes.c_void_p()
        _check(load().qqmc_plan_create(arr, len(items), precision, ctypes.byref(out)), "qqmc_plan_create")
        self.handle = out.value

    def launch(self, stream: int = 0, use_graph: bool = False) -> None:
        _check(load().qqmc_plan_launch(ctypes.c_void_p(self.handle), ctypes.c_void_p(stream or None),
                                       int(use_graph)), "qqmc_plan_launch")

    def results(self, check: bool = True):
        """[(qqmc_result, S_k per shift)] per item.  check=False returns the results of a
        plan whose sums hit NaN or infinity (QQMC_E_NONFINITE) instead of raising; the
        affected items carry n_nonfinite > 0."""
        res = (qqmc_result * self.n_items)()
        per = np.zeros(2 * sum(self.n_shifts))
        rc = load().qqmc_plan_results(ctypes.c_void_p(self.handle), res, _ptr(per, ctypes.c_double))
        if check or rc != QQMC_E_NONFINITE:
            _check(rc, "qqmc_plan_results")
        S = per.view(np.complex128)
        out, o = [], 0
        for i in range(self.n_items):
            out.append((res[i], S[o:o + self.n_shifts[i]].copy()))
            o += self.n_shifts[i]
        return out

    def timing(self):
        """(determinant-kernel ms, whole-launch ms) of the last launch."""
        k, a = ctypes.c_double(), ctypes.c_double()
        _check(load().qqmc_plan_timing(ctypes.c_void_p(self.handle), ctypes.byref(k), ctypes.byref(a)),
               "qqmc_plan_timing")
        return k.value, a.value

    def device_span(self):
        """(start_ns, end_ns) of the last launch's determinant kernels on the device clock."""
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().qqmc_plan_device_span(ctypes.c_void_p(self.handle), ctypes.byref(a), ctypes.byref(b)),
               "qqmc_plan_device_span")
        return a.value, b.value

    def chunk_sums(self, item: int, shift: int, chunks) -> np.ndarray:
        """Complex per-chunk sums (sum + compensation) of the last launch."""
        ch = np.ascontiguousarray(np.asarray(chunks, dtype=np.int64))
        out = np.zeros(4 * ch.size)
        _check(load().qqmc_plan_chunk_sums(ctypes.c_void_p(self.handle), item, shift,
                                           ch.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ch.size,
                                           _ptr(out, ctypes.c_double)), "qqmc_plan_chunk_sums")
        o = out.reshape(-1, 4)
        return (o[:, 0] + o[:, 2]) + 1j * (o[:, 1] + o[:, 3])

    def kernel_count(self) -> int:
        return load().qqmc_plan_kernel_count(ctypes.c_void_p(self.handle))

    def close(self) -> None:
        if self.handle:
            load().qqmc_plan_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qqmc_integrate_noalloc(pr: int, order: int, n_points: int, n_shifts: int, precision: int,
                           d_shift_words: int, d_sums: int, d_counts: int = 0, stream: int = 0) -> None:
    """Allocation-free integration: every pointer is a device address (e.g. a
    torch tensor's data_ptr()); d_sums receives the per-shift sums not divided
    by N.  Enqueues on `stream` and returns."""
    _check(load().qqmc_integrate_noalloc(ctypes.c_void_p(pr), order, n_points, n_shifts, precision,
                                         ctypes.c_void_p(d_shift_words), ctypes.c_void_p(d_sums),
                                         ctypes.c_void_p(d_counts or None), ctypes.c_void_p(stream or None)),
           "qqmc_integrate_noalloc")


def qqmc_set_elimination(pr: int, mode: int) -> None:
    """QQMC_ELIM_AUTO (default), QQMC_ELIM_PAIRS or QQMC_ELIM_SINGLE for this problem's Keldysh sums."""
    _check(load().qqmc_set_elimination(ctypes.c_void_p(pr), mode), "qqmc_set_elimination")


def qqmc_elimination(pr: int, precision: int) -> int:
    """The elimination order the problem's sums use at this precision (QQMC_ELIM_PAIRS or _SINGLE)."""
    rc = load().qqmc_elimination(ctypes.c_void_p(pr), precision)
    _check(rc if rc < 0 else 0, "qqmc_elimination")
    return rc


def qqmc_fma_peak(precision: int, seconds: float = 1.0) -> float:
    """Measured FMA throughput (TFLOP/s, 2 flops per FMA) of the FP64 or FP32 pipes."""
    t = ctypes.c_double()
    _check(load().qqmc_fma_peak(precision, seconds, ctypes.byref(t)), "qqmc_fma_peak")
    return t.value


def qqmc_set_tuning(precision: int, order: int, warps_per_block: int, flat_vertices: int) -> None:
    _check(load().qqmc_set_tuning(precision, order, warps_per_block, flat_vertices), "qqmc_set_tuning")


def qqmc_get_tuning(precision: int, order: int):
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(load().qqmc_get_tuning(precision, order, ctypes.byref(a), ctypes.byref(b)), "qqmc_get_tuning")
    return a.value, b.value


def qqmc_direction_numbers(n_dims: int) -> np.ndarray:
    out = np.zeros((n_dims, 32), dtype=np.uint32)
    _check(load().qqmc_direction_numbers(n_dims, _ptr(out, ctypes.c_uint32)), "qqmc_direction_numbers")
    return out


def qqmc_shift_words(seed: int, n_shifts: int, n_dims: int) -> np.ndarray:
    out = np.zeros((n_shifts, n_dims), dtype=np.uint32)
    _check(load().qqmc_shift_words(seed, n_shifts, n_dims, _ptr(out, ctypes.c_uint32)), "qqmc_shift_words")
    return out


def qqmc_sobol_points(order: int, first_index: int, count: int, shift: np.ndarray | None = None) -> np.ndarray:
    out = np.zeros((count, order), dtype=np.uint32)
    sh = None if shift is None else np.ascontiguousarray(np.asarray(shift, dtype=np.uint32)[:order])
    _check(load().qqmc_sobol_points(order, first_index, count, _ptr(sh, ctypes.c_uint32),
                                    _ptr(out, ctypes.c_uint32)), "qqmc_sobol_points")
    return out


def qqmc_warp_points(pr: int, order: int, first_index: int, count: int, shift: np.ndarray | None = None):
    u = np.zeros((count, order))
    w = np.zeros(count)
    ins = np.zeros(count, dtype=np.int32)
    sh = None if shift is None else np.ascontiguousarray(np.asarray(shift, dtype=np.uint32)[:order])
    _check(load().qqmc_warp_points(ctypes.c_void_p(pr), order, first_index, count, _ptr(sh, ctypes.c_uint32),
                                   _ptr(u, ctypes.c_double), _ptr(w, ctypes.c_double), _ptr(ins, ctypes.c_int32)),
           "qqmc_warp_points")
    return u, w, ins.astype(bool)


def qqmc_integrand(pr: int, order: int, u: np.ndarray, precision: int = QQMC_PREC_FP64) -> np.ndarray:
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, order))
    out = np.zeros(2 * u.shape[0])
    _check(load().qqmc_integrand(ctypes.c_void_p(pr), order, u.shape[0], _ptr(u, ctypes.c_double), precision,
                                 _ptr(out, ctypes.c_double)), "qqmc_integrand")
    return out.view(np.complex128)


def qqmc_resum_parabola(a, p: float, U: float, a_err=None, invert: bool = False):
    """Returns (value, propagated error, last-term size) of the parabola-map resummation."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    e = None if a_err is None else np.ascontiguousarray(np.asarray(a_err, dtype=np.float64))
    v, er, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().qqmc_resum_parabola(_ptr(a, ctypes.c_double), _ptr(e, ctypes.c_double), a.size - 1, p, U,
                                      int(invert), ctypes.byref(v), ctypes.byref(er), ctypes.byref(t)),
           "qqmc_resum_parabola")
    return v.value, er.value, t.value


def qqmc_set_projection(pr: int, order: int, cdf=None) -> None:
    """Install a learned warp (cdf [order, cells + 1]) or, with None, restore the plain warp."""
    if cdf is None:
        _check(load().qqmc_set_projection(ctypes.c_void_p(pr), order, None, 0), "qqmc_set_projection")
        return
    c = np.ascontiguousarray(np.asarray(cdf, dtype=np.float64))
    _check(load().qqmc_set_projection(ctypes.c_void_p(pr), order, _ptr(c, ctypes.c_double), c.shape[1] - 1),
           "qqmc_set_projection")


def qqmc_learn_projection(pr: int, order: int, M: int = 20000, n_bins: int = 100, lam: float = 0.05,
                          floor_frac: float = 1e-3, cells: int = 1024) -> np.ndarray:
    """Learn, install and return the warp table [order, cells + 1]."""
    out = np.zeros((order, cells + 1))
    _check(load().qqmc_learn_projection(ctypes.c_void_p(pr), order, M, n_bins, lam, floor_frac, cells,
                                        _ptr(out, ctypes.c_double)), "qqmc_learn_projection")
    return out


def qqmc_server_create(opts: qqmc_server_opts) -> int:
    out = ctypes.c_void_p()
    _check(load().qqmc_server_create(ctypes.byref(opts), ctypes.byref(out)), "qqmc_server_create")
    return out.value


def qqmc_submit(server: int, req: qqmc_request) -> int:
    h = ctypes.c_uint64()
    _check(load().qqmc_submit(ctypes.c_void_p(server), ctypes.byref(req), ctypes.byref(h)), "qqmc_submit")
    return h.value


def qqmc_poll(server: int, handle: int):
    """Returns (status, qqmc_series or None)."""
    out = qqmc_series()
    rc = load().qqmc_poll(ctypes.c_void_p(server), handle, ctypes.byref(out))
    if rc == QQMC_PENDING:
        return rc, None
    return rc, out


def qqmc_request_state(server: int, handle: int) -> int:
    """QQMC_PENDING (queued), QQMC_RUNNING (admitted) or the final status; the handle stays."""
    return load().qqmc_request_state(ctypes.c_void_p(server), handle)


def qqmc_cancel(server: int, handle: int) -> int:
    return load().qqmc_cancel(ctypes.c_void_p(server), handle)


def qqmc_server_destroy(server: int) -> None:
    load().qqmc_server_destroy(ctypes.c_void_p(server))


def make_params(gamma=1.0, eps_d=0.0, t_max=10.0, tau=1.0, n_table=4096, seed=2002123720,
                alpha=0.0, observable=QQMC_OBS_CHARGE, half_bandwidth=0.0, bias=0.0) -> qqmc_params:
    return qqmc_params(gamma, eps_d, t_max, tau, n_table, observable, seed, alpha, half_bandwidth, bias)
