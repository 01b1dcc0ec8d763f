"""Writes tests/golden/closed_form.json from the oracle alone (oracle/reduced.py).

The stored values are the closed form of Sec. II (Eqs. 5-6: P = sin^2((2k+1)
theta), marked amplitude sin((2k+1)theta)/sqrt(M), unmarked amplitude
cos((2k+1)theta)/sqrt(N-M), theta = arcsin sqrt(M/N)) and the exact Schmidt
spectrum at a few cuts, for the workloads the GPU tests and bench use.
Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import reduced  # noqa: E402
from paper_2601_03832_gb300 import inputs  # noqa: E402


def entry(inst, cuts):
    P, aw, ar = reduced.closed_form(inst.n, inst.M, inst.k)
    return {
        "n": inst.n, "M": inst.M, "k": inst.k, "marked": inst.marked,
        "theta": reduced.theta(inst.n, inst.M),
        "P": P, "amp_marked": aw, "amp_unmarked": ar,
        "schmidt": {str(c): [float(x) for x in reduced.schmidt_values(inst.n, inst.marked, inst.k, c)[:4]]
                    for c in cuts},
    }


def main():
    out = {
        "source": "closed form, Sec. II Eqs. 5-6; Schmidt values from the invariant-plane model",
        "n12_M1_k50": entry(inputs.config_small(), [1, 6, 11]),
        "n29_M1_k18198": entry(inputs.config_n29(), [1, 14, 28]),
        "n40_M32_k1000": entry(inputs.config_multi_marked(1000), [1, 20, 39]),
    }
    with open(os.path.join(HERE, "closed_form.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
