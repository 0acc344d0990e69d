"""Autotuner of the determinant kernel's launch shape.

A plan groups its items by their orders' tuned flat depth and launches each
group with the shape of the group's highest order.  For each order n the tuner
times a batch holding every order 1..n of the plain dot (the shape of the
benchmark batch and of a served request) with the candidate shape installed
for n and the shapes already chosen for 1..n-1, so n's choice is measured in
the launch it will share.  The candidates
are warps per block (points in flight per block) and vertices resolved per
lane in the flat phase (a lane's Keldysh chunk: one of 2^flat choice paths of
the last vertices).  The fastest shape is installed with ``qqmc_set_tuning``
and the table can be stored as JSON keyed by the GPU name.  Each Keldysh-sum
tree has its own table: the single-vertex tree under the precision code (0, 1),
the pair-block tree under precision | QQMC_TUNE_PAIRS (16, 17); the tuning
problem is set to the tree being tuned.

    python -m paper_2002_12372_gb300.autotune [--orders 1-12] [--tree single|pairs|both] [--out tuning.json]
"""
from __future__ import annotations

import argparse
import json
import os
import time

from . import qqmc as Q

CANDIDATES = {
    Q.QQMC_PREC_FP64: [(w, f) for w in (1, 2, 3, 4) for f in (2, 3, 4, 5)],
    Q.QQMC_PREC_MIXED: [(w, f) for w in (2, 4, 6, 8) for f in (2, 3, 4, 5)],
}
# flat 1 = one point per lane (orders <= 4)
LANE_CANDIDATES = {
    Q.QQMC_PREC_FP64: [(w, 1) for w in (1, 2, 4)],
    Q.QQMC_PREC_MIXED: [(w, 1) for w in (2, 4, 8)],
}


def _precision(code: int) -> int:
    return code & ~Q.QQMC_TUNE_PAIRS


def _points_for(order: int, precision: int) -> int:
    # Large enough that the grid drains the way a full batch does (tens of
    # chunks per resident warp), small enough to time each shape in ~0.1 s.
    base = 2 ** 17 if precision == Q.QQMC_PREC_MIXED else 2 ** 15
    return max(2 ** 12, base >> max(0, order - 7))


def time_shape(pr: int, order: int, code: int, wpb: int, flat: int, reps: int = 2) -> float:
    """Kernel time of the batch 1..order with (wpb, flat) installed for `order` in table `code`."""
    Q.qqmc_set_tuning(code, order, wpb, flat)
    precision = _precision(code)
    Q.qqmc_set_elimination(pr, Q.QQMC_ELIM_PAIRS if code & Q.QQMC_TUNE_PAIRS else Q.QQMC_ELIM_SINGLE)
    N = _points_for(order, precision)
    plan = Q.Plan([(pr, m, 16, N) for m in range(1, order + 1)], precision)
    try:
        plan.launch()
        plan.results()
        best = float("inf")
        for _ in range(reps):
            plan.launch()
            plan.results()
            k, _a = plan.timing()
            best = min(best, k)
        return best
    finally:
        plan.close()


def tune(orders=range(1, Q.QQMC_MAX_ORDER + 1), precisions=(Q.QQMC_PREC_FP64, Q.QQMC_PREC_MIXED), verbose=False):
    """Returns {table code: {order: (wpb, flat, ms)}} and installs the winners; a code is a
    precision, or a precision | QQMC_TUNE_PAIRS for the pair-block tree."""
    pr = Q.qqmc_create_problem(Q.make_params(eps_d=0.0, t_max=10.0))
    table = {}
    try:
        for prec in precisions:
            table[prec] = {}
            for n in orders:
                results = []
                cands = CANDIDATES[_precision(prec)] + (LANE_CANDIDATES[_precision(prec)] if n <= 4 else [])
                for wpb, flat in cands:
                    try:
                        ms = time_shape(pr, n, prec, wpb, flat)
                    except Q.QQMCError:
                        continue  # shape does not fit (shared memory)
                    results.append((ms, wpb, flat))
                    if verbose:
                        print("prec=%d n=%2d wpb=%d flat=%d  %.3f ms" % (prec, n, wpb, flat, ms), flush=True)
                ms, wpb, flat = min(results)
                table[prec][n] = (wpb, flat, ms)
                Q.qqmc_set_tuning(prec, n, wpb, flat)
    finally:
        Q.qqmc_destroy_problem(pr)
    return table


def install(table) -> None:
    for prec, rows in table.items():
        for n, (wpb, flat, _ms) in rows.items():
            Q.qqmc_set_tuning(int(prec), int(n), int(wpb), int(flat))


def reset() -> None:
    """Restore the built-in defaults for every (precision, order)."""
    for prec in (Q.QQMC_PREC_FP64, Q.QQMC_PREC_MIXED):
        for tree in (0, Q.QQMC_TUNE_PAIRS):
            for n in range(1, Q.QQMC_MAX_ORDER + 1):
                Q.qqmc_set_tuning(prec | tree, n, 0, 0)


def save(table, path: str) -> None:
    import torch
    name = torch.cuda.get_device_name(0)
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    merged = data.setdefault(name, {})  # orders not tuned this time keep their rows
    for p, rows in table.items():
        merged.setdefault(str(p), {}).update({str(n): list(v) for n, v in rows.items()})
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


def load(path: str):
    import torch
    if not os.path.exists(path):
        return None
    with open(path) as f:
        data = json.load(f)
    rows = data.get(torch.cuda.get_device_name(0))
    if rows is None:
        return None
    return {int(p): {int(n): tuple(v) for n, v in r.items()} for p, r in rows.items()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--orders", default="1-12")
    ap.add_argument("--out", default=None)
    ap.add_argument("--precision", choices=["fp64", "mixed", "both"], default="both")
    ap.add_argument("--tree", choices=["single", "pairs", "both"], default="both")
    args = ap.parse_args()
    lo, hi = (int(x) for x in args.orders.split("-"))
    precs = {"fp64": (Q.QQMC_PREC_FP64,), "mixed": (Q.QQMC_PREC_MIXED,),
             "both": (Q.QQMC_PREC_FP64, Q.QQMC_PREC_MIXED)}[args.precision]
    trees = {"single": (0,), "pairs": (Q.QQMC_TUNE_PAIRS,), "both": (0, Q.QQMC_TUNE_PAIRS)}[args.tree]
    precs = tuple(p | t for t in trees for p in precs)
    from . import build
    build.build()
    t0 = time.time()
    table = tune(range(lo, hi + 1), precs, verbose=True)
    print(json.dumps({str(p): {str(n): v for n, v in r.items()} for p, r in table.items()}))
    print("tuning took %.1f s" % (time.time() - t0))
    if args.out:
        save(table, args.out)


if __name__ == "__main__":
    main()
