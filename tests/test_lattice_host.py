"""The library's host-side lattice construction (FFT-based component-by-component
search) against the oracle's plain O(N^2) construction.  No GPU needed."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def Q():
    from paper_2002_12372_gb300 import build as b
    b.build()
    from paper_2002_12372_gb300 import qqmc
    qqmc.load()
    return qqmc


@pytest.mark.parametrize("m,dims", [(3, 3), (6, 4), (10, 8), (12, 6)])
def test_fast_cbc_matches_plain_cbc(Q, oracle, m, dims):
    g = np.array([0.9 ** d for d in range(dims)])
    z = Q.qqmc_lattice_cbc(m, dims, g)
    zo = oracle.lattice_cbc(m, dims, g)
    # the minimised criterion is unique; the argument can differ only between candidates equal up to rounding
    assert oracle.lattice_cbc_criterion(z, m, g) == pytest.approx(oracle.lattice_cbc_criterion(zo, m, g), rel=1e-12)
    assert np.all(z % 2 == 1) and np.all(z <= (1 << m) // 2)


def test_cbc_arguments(Q):
    with pytest.raises(Q.QQMCError) as e:
        Q.qqmc_lattice_cbc(2, 3, [1.0, 1.0, 1.0])
    assert e.value.code == Q.QQMC_E_INVAL
    with pytest.raises(Q.QQMCError):
        Q.qqmc_lattice_cbc(8, 3, [1.0, 0.0, 1.0])
