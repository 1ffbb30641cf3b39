"""The oracle's operation count (oracle/flops.cpp) that the benchmark's
roofline divides by a kernel's time.

Checks that the count means what it says: on a single element (where the
oracle's own assembled operators and the element computation coincide) the
count of the oracle's drivers equals the per-element count; the per-element
count does not depend on the grid; the residual and the Jacobian apply share
exactly the evaluation of the fields; and the values stored in
tests/golden/vms_flops.json (read by the benchmark) are current.
"""
import json
import os

import pytest

from oracle import flops

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("what", ["residual", "jacobian", "fused"])
def test_single_element_driver_equals_element_count(what):
    assert flops.vms_flops(what, N=1)[0] == flops.vms_flops(what, N=1, driver=True)[0]


def test_per_element_count_is_grid_independent():
    for what in ("residual", "jacobian", "fused"):
        a = flops.vms_flops(what, N=1)[1]
        b = flops.vms_flops(what, N=3)[1]
        assert a["evaluation"] == b["evaluation"] and a["weak_form"] == b["weak_form"]


def test_fused_shares_the_evaluation_only():
    r = flops.vms_flops("residual", N=2)[1]
    j = flops.vms_flops("jacobian", N=2)[1]
    f = flops.vms_flops("fused", N=2)[1]
    assert f["evaluation"] == r["evaluation"] == j["evaluation"]
    # the weak forms share tau, the strong residuals and the fine scales
    assert max(r["weak_form"], j["weak_form"]) < f["weak_form"] < r["weak_form"] + j["weak_form"]


def test_stored_counts_are_current():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_vms_flops", os.path.join(HERE, "golden", "make_vms_flops.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    with open(os.path.join(HERE, "golden", "vms_flops.json")) as f:
        stored = json.load(f)
    assert stored == mk.counts()
