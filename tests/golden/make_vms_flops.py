#!/usr/bin/env python3
"""Writes vms_flops.json: the oracle's operation count per element of the VMS
residual, the Jacobian apply and both at one state (oracle/flops.cpp: every
FP64 operation of the oracle's element computation, constants folded, common
subexpressions merged within the element), plus the assembly additions on the
64^3 and 128^3 grids.  Calls only oracle/.  Run from the repository root:

    python tests/golden/make_vms_flops.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import flops  # noqa: E402


def counts():
    out = {"how": "oracle/flops.cpp: the oracle's FP64 operations per element (+ - * / sqrt), "
                  "operations on constants folded, x+0 / x*1 / x*0 free, common "
                  "subexpressions merged within one element; the oracle evaluates fields "
                  "and projects test functions by dense sums over the element's 8 nodes",
           "per_element": {}, "assembly_per_element": {}}
    for what in ("residual", "jacobian", "fused"):
        total, parts = flops.vms_flops(what, N=3)
        local = parts["evaluation"] + parts["weak_form"]
        out["per_element"][what] = {"element": local, "evaluation": parts["evaluation"],
                                    "weak_form": parts["weak_form"]}
    for N in (8, 64, 128):
        E, n = N ** 3, (N + 1) ** 3
        out["assembly_per_element"][str(N)] = (32.0 * E - 4.0 * n) / E
    return out


if __name__ == "__main__":
    path = os.path.join(HERE, "vms_flops.json")
    with open(path, "w") as f:
        json.dump(counts(), f, indent=1)
        f.write("\n")
    print(open(path).read())
