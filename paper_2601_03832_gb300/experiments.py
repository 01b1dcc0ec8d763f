"""The paper's experiments, run on this package's iterative MPS path.

Sec. IV measures the iterative Grover simulation for M = 1 marked item with
k = round(pi/4 sqrt(N)) iterations (Eq. 8) over a range of qubit counts:
  * runtime against n (Fig. 2),
  * the marked ("target") probability in FP32 against FP64 (Fig. 3): here
    the complex64 form (FP32 tensors, FP64 QR/SVD) beside plain FP64,
  * shot counts from the final state (Fig. 4): perfect sampling with
    1 ... 4096 shots; the raw marked count is reported (the paper's own
    estimator is not described, so it is not reproduced).
Everything below runs on the CUDA library through the binding; nothing here
computes a reference value.  The marked string for n qubits is drawn from
seed 1000 + n (SplitMix64, `inputs.marked_strings`).

Run: python -m paper_2601_03832_gb300.experiments [--ns 10-29] [--shots-ns 2-29]
"""
from __future__ import annotations

import argparse
import json
import math
import sys

from . import binding, inputs

SHOT_COUNTS = (1, 8, 64, 512, 4096)


def k_paper(n: int) -> int:
    """Iterations of the paper's experiments for M = 1: round(pi/4 sqrt(2^n)) (Eq. 8)."""
    return int(round(math.pi / 4 * math.sqrt(2.0 ** n)))


def marked_for(n: int) -> int:
    return inputs.marked_strings(n, 1, seed=1000 + n)[0]


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def precision_sweep(ns, dtypes=("c128", "c64"), chi_max=4, apply="fused"):
    """Marked probability after k_paper(n) iterations in each form, with the
    device time of the iterations (CUDA events on the handle's stream)."""
    import torch
    stream = torch.cuda.current_stream()
    rows = []
    for n in ns:
        w, k = marked_for(n), k_paper(n)
        row = {"n": n, "k": k, "marked": w}
        for dt in dtypes:
            g = binding.GroverMPS(n, [w], dtype=dt, apply=apply, chi_max=chi_max, stream=stream.cuda_stream)
            a, b = _events()
            a.record(stream)
            g.iterate(k)
            b.record(stream)
            torch.cuda.synchronize()
            sec = a.elapsed_time(b) / 1000.0
            row[dt] = {"P_marked": g.prob_marked(), "seconds": sec,
                       "iterations_per_s": k / sec if sec > 0 else None,
                       "max_bond": g.stats()["max_bond"]}
            g.close()
        rows.append(row)
    return rows


def shot_sweep(ns, shots=SHOT_COUNTS, sample_seed=2, dtype="c128", chi_max=4, apply="fused"):
    """Marked count among `s` perfect-sampling shots of the final state, for
    each s in `shots` (independent draws: seed sample_seed + index)."""
    rows = []
    for n in ns:
        w, k = marked_for(n), k_paper(n)
        g = binding.GroverMPS(n, [w], dtype=dtype, apply=apply, chi_max=chi_max)
        g.iterate(k)
        counts = {}
        for i, s in enumerate(shots):
            bits = g.sample(s, sample_seed + i)
            counts[str(s)] = int((bits == w).sum())
        rows.append({"n": n, "k": k, "P_marked": g.prob_marked(), "marked_counts": counts})
        g.close()
    return rows


def _range(text: str):
    lo, _, hi = text.partition("-")
    return list(range(int(lo), int(hi or lo) + 1))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--ns", default="10-29", help="qubit counts of the precision and runtime sweep")
    ap.add_argument("--shots-ns", default="2-29", help="qubit counts of the shot sweep")
    ap.add_argument("--out", default=None, help="write the results as JSON")
    args = ap.parse_args(argv)
    binding.load()
    res = {"precision": precision_sweep(_range(args.ns)), "shots": shot_sweep(_range(args.shots_ns))}
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
    print("| n | k | P FP64 | P complex64 | FP64 iterations/s |")
    print("|---|---|---|---|---|")
    for r in res["precision"]:
        print(f"| {r['n']} | {r['k']} | {r['c128']['P_marked']:.12f} | {r['c64']['P_marked']:.8f} | "
              f"{r['c128']['iterations_per_s']:.0f} |")
    print()
    print("| n | " + " | ".join(f"{s} shots" for s in SHOT_COUNTS) + " |")
    print("|---|" + "---|" * len(SHOT_COUNTS))
    for r in res["shots"]:
        print(f"| {r['n']} | " + " | ".join(str(r["marked_counts"][str(s)]) for s in SHOT_COUNTS) + " |")
    return 0


if __name__ == "__main__":
    sys.exit(main())
