"""Writes tests/golden/c2_error_table.json: the oracle's accuracy table of the N = 8192
algebraic-decay configuration (a_ij = (|i-j|+1)^-3 s_ij, A and B independent, leaf 64) over
tau = 1e-1 .. 1e-7 and every precision mode.

TEST INFRASTRUCTURE ONLY (see the package docstring).  It calls only oracle/ and the seeded
generators.  For each tau: S, the valid ratio, the skipped bound bound2 / (||A|| ||B||), the
pruning error of the exact pruned product, and per mode the relative error
||C_mode - AB||_F / (||A||_F ||B||_F) of the FP64 evaluation of that mode's rounded operands
(oracle.precision.emulated_multiply; the split modes flag by the dominant-triple rule at target
1e-5) with its a-priori bound.  AB is the dense FP64 product.  Minutes of CPU time.

Usage: python -m oracle.c2_error_table [--out tests/golden/c2_error_table.json]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

from . import precision as OP
from . import spamm as S
from . import tau as OT

TAUS = (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7)
MODES = (("bf16", OP.BF16), ("fp16", OP.FP16), ("bf16_split", OP.BF16_SPLIT),
         ("fp16_split", OP.FP16_SPLIT), ("tf32x3", OP.TF32X3))
TARGET = 1e-5


def table(a, b, leaf: int = 64, taus=TAUS, log=print) -> dict:
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    na, nb = OT.frobenius_from_normmap(nA), OT.frobenius_from_normmap(nB)
    ab = na * nb
    dense = S.dense_reference(a, b)
    rows = []
    for tau in taus:
        surv = S.flat_survivors(nA, nB, tau)
        _, b2 = S.skipped_bounds(nA, nB, surv)
        pruned = S.multiply_with_skipset(a, b, leaf, surv)
        row = {"tau": tau, "S": int(surv.sum()), "valid_ratio": S.valid_ratio(surv),
               "bound2_rel": b2 / ab, "pruning_rel": S.frobenius(pruned - dense) / ab, "modes": {}}
        for name, mode in MODES:
            flags = None
            if mode in (OP.BF16_SPLIT, OP.FP16_SPLIT):
                m = OP.flag_exponent(nA, nB, surv, OP.mode_format(mode), TARGET, b2, na, nb)
                flags = OP.flag_mask(nA, nB, surv, m, na, nb)
            c = OP.emulated_multiply(a, b, leaf, surv, mode, flags)
            row["modes"][name] = {
                "rel_err": S.frobenius(c - dense) / ab,
                "rounding_rel": S.frobenius(c - pruned) / ab,
                "apriori_rel": OP.apriori_bound(nA, nB, surv, mode, leaf, flags) / ab,
                "flagged": int(flags.sum()) if flags is not None else None}
        rows.append(row)
        log(f"tau {tau:g}: S = {row['S']}, pruning {row['pruning_rel']:.3e}, " +
            ", ".join(f"{k} {v['rel_err']:.3e}" for k, v in row["modes"].items()))
    return {"workload": "algebraic decay (|i-j|+1)^-3 * (+-1), N=8192, A and B independent, leaf 64",
            "norm_ab": ab, "target_rel_err_split_flags": TARGET, "rows": rows,
            "command": "python -m oracle.c2_error_table"}


def main(argv=None):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(root, "tests", "golden", "c2_error_table.json"))
    ap.add_argument("--n", type=int, default=8192)
    args = ap.parse_args(argv)
    a, b = synth.workload_c2(args.n)
    res = table(a, b)
    res["n"] = args.n
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1)
    print(args.out)


if __name__ == "__main__":
    main()
