"""C-ABI checks that need no GPU: the library builds, loads, exports every
declared symbol, and its host-side generators and argument checks behave."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def Q():
    from paper_2002_12372_gb300 import build as b
    b.build()
    from paper_2002_12372_gb300 import qqmc
    qqmc.load()
    return qqmc


def declared_symbols():
    with open(os.path.join(ROOT, "include", "qqmc.h")) as f:
        txt = f.read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qqmc_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(Q):
    import ctypes
    lib = ctypes.CDLL(Q.LIB_PATH)
    decl = declared_symbols()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(Q.EXPORTED) == decl


def test_direction_numbers_match_scipy_sobol(Q):
    from scipy.stats import qmc
    D = Q.QQMC_MAX_ORDER
    V = Q.qqmc_direction_numbers(D)
    # natural-order point 2^j is V[:, j]; scipy emits Gray order: out[2^j-1] ^ out[2^j] = V[:, j]
    pts = np.rint(qmc.Sobol(D, scramble=False, bits=32).random(2 ** 14) * 2.0 ** 32).astype(np.uint64)
    for j in range(14):
        assert np.array_equal((pts[(1 << j) - 1] ^ pts[1 << j]).astype(np.uint32), V[:, j]), j
    # Gray-code points from V reproduce scipy exactly
    i = np.arange(2 ** 14, dtype=np.uint64)
    g = i ^ (i >> np.uint64(1))
    X = np.zeros((2 ** 14, D), dtype=np.uint32)
    for j in range(14):
        bit = ((g >> np.uint64(j)) & np.uint64(1)).astype(bool)
        X[bit] ^= V[:, j]
    assert np.array_equal(X, pts.astype(np.uint32))


def test_shift_words_match_oracle_splitmix(Q):
    from oracle import oracle as O
    assert np.array_equal(Q.qqmc_shift_words(2002123720, 5, 12), O.shift_words(2002123720, 5, 12))


def test_argument_errors_without_device(Q):
    with pytest.raises(Q.QQMCError) as e:
        Q.qqmc_sobol_points(Q.QQMC_MAX_ORDER + 1, 0, 4)
    assert e.value.code == Q.QQMC_E_RANGE
    with pytest.raises(Q.QQMCError) as e:
        Q.qqmc_direction_numbers(0)
    assert e.value.code == Q.QQMC_E_INVAL
    with pytest.raises(Q.QQMCError):
        Q.qqmc_set_tuning(0, 5, 99, 4)
    Q.qqmc_set_tuning(0, 5, 3, 4)
    assert Q.qqmc_get_tuning(0, 5) == (3, 4)
    Q.qqmc_set_tuning(0, 5, 0, 0)
    lib = Q.load()
    import ctypes
    res = Q.qqmc_result()
    assert lib.qqmc_integrate(None, 3, 1024, 4, 0, None, None, ctypes.byref(res)) == Q.QQMC_E_INVAL
    assert "problem" in str(Q.QQMCError(-1, "x"))
