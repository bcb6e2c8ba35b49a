"""Writes the stored expected values under tests/golden/.

Calls only the CPU oracle (and the seeded input generator).  Run from the
repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2105_13324_gb300 import phantoms as P  # noqa: E402


def water32_trace_summary(first=0, count=50_000):
    w = P.workload("water32")
    pr = oracle.Problem(w.phantom, w.geometry)
    rec = oracle.trace(pr, w.seed, first, count)
    det = np.nonzero(rec["n_events"])[0]
    return {
        "workload": "water32", "seed": w.seed, "first": first, "count": count,
        "fates": np.bincount(rec["fate"], minlength=4).tolist(),
        "n_virtual": int(rec["n_virtual"].sum()), "n_real": int(rec["n_real"].sum()),
        "n_compton": int(rec["n_compton"].sum()), "n_draws": int(rec["n_draws"].sum()),
        "e_final_sum_kev": float(rec["e_final_kev"].sum()),
        "events": [[int(first + h), int(rec["n_events"][h])] + [int(r) for r in rec["event_row"][h][:rec["n_events"][h]]]
                   for h in det],
    }


if __name__ == "__main__":
    out = os.path.join(HERE, "water32_trace_seed1.json")
    with open(out, "w") as f:
        json.dump(water32_trace_summary(), f, indent=1)
    print("wrote", out)
