"""Writes closed_form_counts.json from oracle/counts.py (calls only oracle/).

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.counts import closed_form_sizes  # noqa: E402

SHAPES = {
    "tiny: n0=8, 4 unary (sq sqrt exp log), 5 binary slots (+ - * a/b b/a), rung 2": (8, 4, 5, 2),
    "medium: n0=20, 6 unary, 6 binary, rung 2": (20, 6, 6, 2),
    "precision: n0=12, 6 unary, 6 binary, rung 3": (12, 6, 6, 3),
    "large: n0=40, 6 unary, 6 binary, rung 2": (40, 6, 6, 2),
}

out = {"cite": "Unpruned |Phi_r| of the rung construction (Software Description): "
               "|new_r| = U*m + S*(m(m-1)/2 + m*o) with m = |new_{r-1}|, o = |Phi_{r-2}|.",
       "sizes": {k: closed_form_sizes(*v) for k, v in SHAPES.items()}}
with open(os.path.join(HERE, "closed_form_counts.json"), "w") as f:
    json.dump(out, f, indent=1)
    f.write("\n")
