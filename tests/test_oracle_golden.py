"""Regression of the oracle against its stored trace summary.

tests/golden/water32_trace_seed1.json is written by
tests/golden/make_golden.py, which calls only the oracle.  The oracle is
built without fused multiply-add, so x86-64 and aarch64 hosts must agree:
integer fields exactly, the energy sum to rounding.
"""
import json
import os

import pytest

from tests.golden.make_golden import water32_trace_summary

HERE = os.path.dirname(os.path.abspath(__file__))


def test_water32_trace_matches_stored_summary():
    with open(os.path.join(HERE, "golden", "water32_trace_seed1.json")) as f:
        want = json.load(f)
    got = water32_trace_summary(want["first"], want["count"])
    for k in ("fates", "n_virtual", "n_real", "n_compton", "n_draws", "events"):
        assert got[k] == want[k], k
    assert got["e_final_sum_kev"] == pytest.approx(want["e_final_sum_kev"], rel=1e-12)
