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

It also compares the iterative MPS path with the iterative statevector path
(grover_sv_*, Sec. III-B-1) over n -- the crossover of Sec. IV-1 --, the
gate-level "Common" and "Iterative" methods of Sec. III-A (Fig. 1), and runs
single instances for profiling.

Run: python -m paper_2601_03832_gb300.experiments [--ns 10-29] [--shots-ns 2-29]
     python -m paper_2601_03832_gb300.experiments crossover [--ns 12-31] [--sv-max-iters 400]
     python -m paper_2601_03832_gb300.experiments circuits [--ns 10-29] [--kmax K]
     python -m paper_2601_03832_gb300.experiments batched [--count 512] [--kcap K] [--dtype c64]
     python -m paper_2601_03832_gb300.experiments differentiable [--vectors 64]
     python -m paper_2601_03832_gb300.experiments single --n 29 --k 50 [--M 1] [--dtype c128] [--apply fused]
         [--path mps|sv]
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


def crossover_sweep(ns, sv_max_iters=400, mps_max_iters=4000, chi_max=4):
    """Iterations/s of the iterative MPS path (FP64, fused) and of the
    iterative statevector path (complex128) for M = 1 at each n, each timed
    with CUDA events on a slice of min(k, max_iters) iterations of the
    k_paper(n) run (a statevector pass costs the same at every iteration),
    and the predicted full-run seconds.  The statevector path is skipped
    where its 2^n x 16 bytes do not fit the device."""
    import torch
    stream = torch.cuda.current_stream()
    free, _ = torch.cuda.mem_get_info()
    rows = []
    for n in ns:
        w, k = marked_for(n), k_paper(n)
        row = {"n": n, "k": k}
        km = min(k, mps_max_iters)
        g = binding.GroverMPS(n, [w], dtype="c128", apply="fused", chi_max=chi_max, stream=stream.cuda_stream)
        g.iterate(2)
        g.reset()
        a, b = _events()
        a.record(stream)
        g.iterate(km)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1000.0
        row["mps"] = {"iterations_per_s": km / sec, "timed_iterations": km, "full_run_s": k * sec / km}
        g.close()
        if (16 << n) < 0.8 * free:
            ks = min(k, sv_max_iters)
            v = binding.GroverSV(n, [w], dtype="c128", stream=stream.cuda_stream)
            v.iterate(min(ks, 70))        # warm-up: graph instantiation
            v.reset()
            a, b = _events()
            a.record(stream)
            v.iterate(ks)
            b.record(stream)
            torch.cuda.synchronize()
            sec = a.elapsed_time(b) / 1000.0
            row["sv"] = {"iterations_per_s": ks / sec, "timed_iterations": ks, "full_run_s": k * sec / ks,
                         "hbm_gbs": 32.0 * (1 << n) * ks / sec / 1e9}
            v.close()
        rows.append(row)
    cross = None
    for r in rows:
        if "sv" in r and r["mps"]["iterations_per_s"] > r["sv"]["iterations_per_s"]:
            cross = r["n"]
            break
    return rows, cross


def common_vs_iterative(ns, chi_max=4, kmax=None):
    """The paper's two gate-level methods (Sec. III-A, Fig. 1) on this GPU for
    M = 1 and k = k_paper(n) (capped at kmax): "Common" builds the whole
    k-iteration circuit (H, X and multi-controlled Z gates) and applies it
    once; "Iterative" builds one iteration's gates and applies them k times
    to the state it keeps.  Both run gate by gate through
    grover_mps_apply_circuit; wall seconds include building the gate list on
    the host and copying it to the device.  The fused direct-sum iteration
    (one sweep pair per Grover gate) is timed beside them."""
    import time

    import torch
    rows = []
    for n in ns:
        w, k = marked_for(n), k_paper(n)
        if kmax:
            k = min(k, kmax)
        row = {"n": n, "k": k}
        for method in ("iterative", "common"):
            g = binding.GroverMPS(n, [w], dtype="c128", apply="mpo", chi_max=chi_max)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            gates = binding.grover_gates(n, [w], 1 if method == "iterative" else k)
            g.apply_circuit(gates, repeat=k if method == "iterative" else 1)
            p = g.prob_marked()
            sec = time.perf_counter() - t0
            row[method] = {"seconds": sec, "P_marked": p, "gates": len(gates),
                           "gate_list_bytes": len(gates) * 72}
            g.close()
        g = binding.GroverMPS(n, [w], dtype="c128", apply="fused", chi_max=chi_max)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.iterate(k)
        row["fused"] = {"seconds": time.perf_counter() - t0, "P_marked": g.prob_marked()}
        g.close()
        row["common_over_iterative"] = row["common"]["seconds"] / row["iterative"]["seconds"]
        rows.append(row)
    return rows


def batched(count=512, kcap=None, dtype="c64", threads=256):
    """The batched workload (the first `count` of the 512 instances, k_i
    capped at kcap) in one persistent launch; returns the wall seconds and
    the largest |P - closed form| is left to the caller (no reference here)."""
    import time

    import torch
    insts = inputs.config_batched(count=512)[:count]
    if kcap:
        for i in insts:
            i.k = min(i.k, kcap)
    b = binding.GroverBatch(insts, dtype=dtype, apply="fused")
    b.set_threads(threads)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run(use_graph=False)
    p, st, rc = b.result()
    sec = time.perf_counter() - t0
    b.close()
    return {"count": count, "kcap": kcap, "seconds": sec, "iterations": int(sum(i.k for i in insts)),
            "instances_with_status": int((st != 0).sum()), "P_marked": [float(x) for x in p]}


def differentiable(vectors=64):
    """The differentiable workload (n = 20, M = 4, K = 64, checkpoint every 8)
    for `vectors` phase vectors through grover_mps_diff_batch_run."""
    import time

    import torch

    from . import autograd
    di, phi, psi = inputs.config_differentiable(B=vectors)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L, gphi, gpsi = autograd.loss_and_grad_batch(di.n, di.marked, phi, psi)
    torch.cuda.synchronize()
    return {"vectors": vectors, "seconds": time.perf_counter() - t0, "loss": [float(x) for x in L]}


def single(n, M, k, dtype="c128", apply="fused", chi_max=None, path="mps", seed=None):
    """One instance (marked strings from seed 1000 + n unless `seed`): k
    iterations on the MPS or statevector path, P_marked printed.  A small,
    fixed case for profiling the kernels."""
    marked = inputs.marked_strings(n, M, seed=1000 + n if seed is None else seed)
    if path == "sv":
        g = binding.GroverSV(n, marked, dtype=dtype)
    else:
        g = binding.GroverMPS(n, marked, dtype=dtype, apply=apply, chi_max=chi_max or M + 3)
    g.iterate(k)
    p = g.prob_marked()
    g.close()
    return {"n": n, "M": M, "k": k, "dtype": dtype, "path": path, "P_marked": p}


def _range(text: str):
    lo, _, hi = text.partition("-")
    return list(range(int(lo), int(hi or lo) + 1))


def main(argv=None):
    argv = list(sys.argv[1:] if argv is None else argv)
    if argv and argv[0] == "crossover":
        ap = argparse.ArgumentParser(description="iterative MPS against iterative statevector over n")
        ap.add_argument("--ns", default="12-31")
        ap.add_argument("--sv-max-iters", type=int, default=400)
        args = ap.parse_args(argv[1:])
        binding.load()
        rows, cross = crossover_sweep(_range(args.ns), sv_max_iters=args.sv_max_iters)
        print(json.dumps({"rows": rows, "mps_faster_from_n": cross}))
        return 0
    if argv and argv[0] == "circuits":
        ap = argparse.ArgumentParser(description="gate-level Common against Iterative")
        ap.add_argument("--ns", default="10-29")
        ap.add_argument("--kmax", type=int, default=None)
        args = ap.parse_args(argv[1:])
        binding.load()
        print(json.dumps({"rows": common_vs_iterative(_range(args.ns), kmax=args.kmax)}))
        return 0
    if argv and argv[0] == "batched":
        ap = argparse.ArgumentParser(description="the batched workload (subset)")
        ap.add_argument("--count", type=int, default=512)
        ap.add_argument("--kcap", type=int, default=None)
        ap.add_argument("--dtype", default="c64")
        args = ap.parse_args(argv[1:])
        binding.load()
        r = batched(args.count, args.kcap, args.dtype)
        r.pop("P_marked")
        print(json.dumps(r))
        return 0
    if argv and argv[0] == "differentiable":
        ap = argparse.ArgumentParser(description="the differentiable workload")
        ap.add_argument("--vectors", type=int, default=64)
        args = ap.parse_args(argv[1:])
        binding.load()
        r = differentiable(args.vectors)
        r.pop("loss")
        print(json.dumps(r))
        return 0
    if argv and argv[0] == "single":
        ap = argparse.ArgumentParser(description="one instance")
        ap.add_argument("--n", type=int, required=True)
        ap.add_argument("--M", type=int, default=1)
        ap.add_argument("--k", type=int, required=True)
        ap.add_argument("--dtype", default="c128")
        ap.add_argument("--apply", default="fused")
        ap.add_argument("--chi-max", type=int, default=None)
        ap.add_argument("--path", default="mps", choices=["mps", "sv"])
        args = ap.parse_args(argv[1:])
        binding.load()
        print(json.dumps(single(args.n, args.M, args.k, args.dtype, args.apply, args.chi_max, args.path)))
        return 0
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
