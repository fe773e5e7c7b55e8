"""Write tests/golden/highdim_mc.json: Monte Carlo prices of the high-dimensional
calls on the maximum (inputs.high_dim_problem(d, "max"), d = 20, 50, 100), the
only reference at these d (random correlation: no one-factor form, no grid sum).

    python tests/golden/make_highdim_golden.py

Calls only oracle/closed_forms.mc_price (exact terminal sampling, Eq. mc with the
GBM law), 8e6 paths, seed 7 + d; stores mean and standard error.
"""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "highdim_mc.json")
PATHS = 8_000_000


def main():
    from oracle import closed_forms
    from paper_2203_02804_gb300 import inputs

    out = {"paths": PATHS, "generator": "paper_2203_02804_gb300.inputs.high_dim_problem(d, 'max')", "prices": {}}
    for d in (20, 50, 100):
        p = inputs.high_dim_problem(d, "max")
        m, se = closed_forms.mc_price(p.spot, p.cov, p.strike, p.rate, p.maturity, "max", PATHS, 7 + d)
        out["prices"][str(d)] = {"mean": m, "se": se}
        print(d, m, se, flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
