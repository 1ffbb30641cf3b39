"""Operation count of the oracle's VMS operators per element (flops.cpp).

TEST AND MEASUREMENT INFRASTRUCTURE ONLY.  The benchmark does not call this
module: ``tests/golden/make_vms_flops.py`` runs it and stores the counts in
``tests/golden/vms_flops.json``, which the benchmark reads as data, and
``tests/test_oracle_flops.py`` checks that the stored counts are current.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flops.cpp")
_LIB = os.path.join(_HERE, "_build", "libflops.so")


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    deps = (_SRC, os.path.join(_HERE, "fsi_oracle.c"))
    if force or not os.path.exists(_LIB) or any(
            os.path.getmtime(_LIB) < os.path.getmtime(d) for d in deps):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-w",
                               f"-I{_HERE}", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def vms_flops(what: str, N: int = 4, driver: bool = False):
    """(operations per element, {evaluation, weak form, assembly}) of the
    residual ("residual"), the Jacobian apply ("jacobian") or both at one
    state ("fused") on an N^3 grid; driver=True counts the oracle's own
    assembled operators instead (parts then zero)."""
    L = ctypes.CDLL(build())
    f = L.or_count_vms_flops
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_double
    parts = (ctypes.c_double * 3)()
    total = f(int(N), {"residual": 0, "jacobian": 1, "fused": 2}[what], int(driver), parts)
    return total, {"evaluation": parts[0], "weak_form": parts[1], "assembly": parts[2]}
