"""Writes high_order_integrand.txt: the oracle's integrand c_n(u) (App. E
Eq. (integral_gf), naive sum of 2^n pivoted-LU determinant products) at one
seeded point for each order 19..22, on the seeded synthetic tables the GPU
tests use.  These orders take the oracle 10 s to 2 min per point, so the
values are stored instead of recomputed in the test.  Calls only the oracle
and the seeded input generators.

    python tests/golden/make_high_order_integrand.py
"""
import os
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2002_12372_gb300 import workloads as W  # noqa: E402

T, L = 10.0, 4096
ORDERS = (19, 20, 21, 22)


def one(n):
    tabs = W.synthetic_tables(200 + n, L, T)[:3]
    u = W.ordered_times(300 + n, 1, n, T)
    c, scale = O.integrand(n, u, T, tabs, T, return_abs=True)
    return n, c[0], scale[0]


def main():
    O.build()
    with ThreadPoolExecutor(max_workers=len(ORDERS)) as ex:
        rows = list(ex.map(one, ORDERS))
    with open(os.path.join(HERE, "high_order_integrand.txt"), "w") as f:
        f.write("# oracle integrand c_n(u) at u = workloads.ordered_times(300 + n, 1, n, 10.0),\n")
        f.write("# tables workloads.synthetic_tables(200 + n, 4096, 10.0); written by make_high_order_integrand.py\n")
        f.write("# n  re(c)  im(c)  sum_a |term_a|\n")
        for n, c, s in rows:
            f.write("%d %.17e %.17e %.17e\n" % (n, c.real, c.imag, s))


if __name__ == "__main__":
    main()
