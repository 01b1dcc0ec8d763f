"""Benchmark: MPS Grover iterations/s on one GB300.

Workload (one step): the n = 29, M = 1 plain-Grover instance (marked string
from seed 3), k = 18198 = floor(pi/4 * 2^14.5) iterations on an MPS with
chi_max = 4, in IEEE FP64 (complex128): reset to |+>^n, all k iterations
(operator contraction + QR sweep + truncated SVD sweep per iteration), the
marked probability and amplitude, and 4096 + 1 perfect-sampling shots.
`value` = k / (device time per step).

Run: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica of the
workload (a single instance does not shard); `value` counts all ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SITES, K_ITERS, CHI_MAX, SHOTS = 29, 18198, 4, (4096, 1)
APPLY = "fused"
SAMPLE_SEED = 2
# Counters of the iterate kernel on this instance from one ncu capture (k = 50;
# the DRAM traffic is the chain's load and store and the code, independent of
# k): DRAM bytes (read + write) per launch, and the FP64 pipe busy share of the
# SM running the instance (sm__pipe_fp64_cycles_active, summed over its four
# sub-partitions).  None until a capture of the current kernel is recorded.
CAPTURE = {"traffic_bytes": 209152, "fp64_pipe_share": 4 * 0.15512}


def flops_per_iter_parts(n: int, chi: int, M: int, apply: str):
    """Algorithmic real flops of one iteration at bond chi (complex = 4x the
    real counts), split into (QR + SVD, contractions).

    Per operator contraction + sweep pair with expanded bond X:
      contraction  R (r x X) . B_l: 2 r X chi complex MACs (8 flops each),
                   plus the absorption of U S into the left neighbour, 2 r chi chi
      Householder QR of the (2r) x X matrix and its thin Q:
                   2 * 4 (2 m n^2 - 2 n^3 / 3), m = 2r, n = X
      SVD of the r x 2 chi matrix (Golub & Van Loan thin-SVD count):
                   4 (14 m n^2 + 8 n^3), m = max, n = min
    summed over the n - 1 site steps; interior bonds r = X (after the QR sweep).
    """
    if apply == "fused":
        ops = [chi + M + 1]
    elif apply == "split":
        ops = [chi + M, chi + 1]
    else:
        ops = [(M + 1) * chi, 2 * chi]
    linalg = contr = 0.0
    for X in ops:
        r = X
        m_, n_ = 2 * r, X
        qr = 2 * 4 * (2 * m_ * n_ ** 2 - 2 * n_ ** 3 / 3)
        a, b = max(r, 2 * chi), min(r, 2 * chi)
        svd = 4 * (14 * a * b ** 2 + 8 * b ** 3)
        linalg += (n - 1) * (qr + svd)
        contr += (n - 1) * (8 * (2 * r * X * chi) + 8 * (2 * r * chi * chi))
    return linalg, contr


def executed_flops_per_iter(n: int, chi: int, M: int, apply: str) -> float:
    """Real flops of one iteration as the rank-revealing sweeps execute it at
    steady state (bond chi at every cut; the iterate stays in span{sum_w |w>,
    |s>}, so every QR step factors a matrix of 2 chi rows and stops after
    chi reflectors): per sweep pair with expanded bond X and per site
      contraction of R (chi rows) into the expanded site: chi x 2 x X chi/.. MACs
      Householder QR of the 2chi x X matrix, chi reflectors: for step j the
        X-j-1 trailing columns take a dot, an update (16 flops per element of
        rows >= j) and a norm update (4 flops)
      thin Q (2 chi x chi) from the reflectors
      SVD of the chi x 2 chi matrix (Golub & Van Loan thin-SVD count)
      absorption of U S into the left neighbour: chi x 2chi x chi MACs.
    The nominal count below (algorithmic_flops_per_iter) assumes a full-rank
    QR of the 2X x X expanded matrix instead; for the generic MPO of bond
    M + 1 (X = (M+1) chi) it exceeds this by orders of magnitude."""
    if apply == "fused":
        ops = [(chi + M + 1, chi * chi + M + 1)]
    elif apply == "split":
        ops = [(chi + M, chi * chi + M), (chi + 1, chi * chi + 1)]
    else:
        ops = [((M + 1) * chi, (M + 1) * chi * chi), (2 * chi, 2 * chi * chi)]
    total = 0.0
    for X, macs_per_row in ops:
        m, p = 2 * chi, chi
        qr = sum((X - j - 1) * (m - j) * 20 for j in range(p))
        q = sum((p - j - 1) * (m - j) * 16 + 8 * (m - j) for j in range(p))
        svd = 4 * (14 * (2 * chi) * chi ** 2 + 8 * chi ** 3)
        contr = 8 * chi * 2 * macs_per_row + 8 * chi * 2 * chi * chi
        total += (n - 1) * (qr + q + svd + contr)
    return total


def algorithmic_flops_per_iter(n: int, chi: int, M: int, apply: str) -> float:
    """Total algorithmic real flops of one iteration (flops_per_iter_parts summed)."""
    a, b = flops_per_iter_parts(n, chi, M, apply)
    return a + b


def roofline_alu(flops: float, seconds: float, peak_tflops: float, peak_name: str, sms_used: int, sms: int,
                 nominal_flops: float = None):
    """ALU roofline entry: achieved TFLOP/s (flops: the executed count of
    executed_flops_per_iter) against the measured chip peak, and against the
    share of it that the SMs the work ran on hold; with nominal_flops, the
    same time against the nominal full-rank count beside it."""
    ach = flops / seconds / 1e12
    out = {"bound": "alu", "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s", "frac": ach / peak_tflops,
           "peak_source": f"measured {peak_name} (libgmps_peaks.so, this run)",
           "sms_used": sms_used, "frac_of_sms_used": ach / (peak_tflops * sms_used / sms),
           "flop_model": "executed (rank-revealing QR on 2 chi rows, chi reflectors; thin SVD of chi x 2 chi)"}
    if nominal_flops is not None:
        out["nominal"] = {"flops": nominal_flops, "achieved": nominal_flops / seconds / 1e12,
                          "model": "full-rank QR of the 2X x X expanded matrix (Golub-Van Loan counts)"}
    return out


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def replica_rate(local_ms: float, steps: int, k: int):
    """Whole-job rate of independent replicas, one per rank.  The slowest
    rank's total time (max over ranks) sets ms per step; every rank ran k
    iterations per step, so value = world_size * k / (ms per step).  Returns
    (ms_per_step, value); without an initialised process group it is the
    single-rank rate."""
    import torch
    ws = 1
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        ws = torch.distributed.get_world_size()
        dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
        t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.barrier()
        local_ms = t.item()
    ms_per_step = local_ms / steps
    return ms_per_step, ws * k / (ms_per_step / 1000.0)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(seconds_budget: float = 12.0):
    """The oracle (plain NumPy FP64 MPS, same contraction mode) timed on one host
    core for a bounded slice of the workload."""
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
from oracle import mps
from paper_2601_03832_gb300 import inputs
inst = inputs.config_n29()
st = mps.plus_state(inst.n)
t0 = time.perf_counter(); done = 0
while time.perf_counter() - t0 < {seconds_budget}:
    st = mps.grover_iterate(st, inst.marked, 100, inst.chi_max, 0.0, mode={APPLY!r})
    done += 100
dt = time.perf_counter() - t0
print(json.dumps({{"iters": done, "seconds": dt}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    res = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": res["iters"] / res["seconds"], "unit": "iterations/s", "cores": 1, "kind": "oracle",
            "sample": f"first {res['iters']} of the {K_ITERS} iterations of the same n=29 instance "
                      f"({APPLY} contraction, NumPy FP64, OMP_NUM_THREADS=1), {res['seconds']:.1f} s"}


def _oracle_batched_slice(task):
    """One instance of the batched workload on the oracle (process-pool task)."""
    n, marked, k, chi_max = task
    from oracle import mps
    t0 = time.perf_counter()
    mps.grover_iterate(mps.plus_state(n), marked, k, chi_max, 0.0, mode=APPLY)
    return k, time.perf_counter() - t0


def _oracle_adjoint_vector(task):
    """Forward and adjoint of one phase vector on the oracle (process-pool task)."""
    n, marked, phi, psi = task
    from oracle import statevector
    t0 = time.perf_counter()
    statevector.adjoint(n, marked, phi, psi)
    return time.perf_counter() - t0


def _oracle_pool(fn, tasks, workers):
    """Run oracle tasks on `workers` spawned processes with one BLAS thread
    each; returns (results, wall seconds)."""
    import multiprocessing
    from concurrent.futures import ProcessPoolExecutor
    keep = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for v in keep:
        os.environ[v] = "1"
    try:
        t0 = time.perf_counter()
        with ProcessPoolExecutor(max_workers=workers, mp_context=multiprocessing.get_context("spawn")) as ex:
            res = list(ex.map(fn, tasks))
        wall = time.perf_counter() - t0
    finally:
        for v, x in keep.items():
            if x is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = x
    return res, wall


def cpu_baseline_batched(insts, kslice: int = 10, count: int = 64):
    """The oracle on a bounded sample of the batched workload: the first
    `count` instances, `kslice` iterations each, spread over all host cores."""
    cores = os.cpu_count() or 1
    tasks = [(x.n, list(x.marked), min(x.k, kslice), x.chi_max) for x in insts[:count]]
    res, wall = _oracle_pool(_oracle_batched_slice, tasks, cores)
    its = sum(r[0] for r in res)
    return {"value": its / wall, "unit": "iterations/s", "cores": cores, "kind": "oracle",
            "sample": f"first {len(tasks)} of the 512 instances, min(k_i, {kslice}) iterations each "
                      f"({its} in all), NumPy FP64 MPS, {cores} spawned processes with one BLAS thread, "
                      f"{wall:.1f} s wall including process start-up"}


def cpu_baseline_differentiable(di, phi, psi, vectors: int = 4):
    """The oracle's forward + adjoint (dense FP64 statevector, n = 20) on a
    bounded sample of the phase vectors, one process per vector."""
    workers = min(vectors, os.cpu_count() or 1)
    tasks = [(di.n, list(di.marked), phi[b], psi[b]) for b in range(vectors)]
    res, wall = _oracle_pool(_oracle_adjoint_vector, tasks, workers)
    return {"value": 1000.0 * wall / vectors, "unit": "ms per vector (forward + backward)", "cores": workers,
            "kind": "oracle",
            "sample": f"{vectors} of the 64 phase vectors, dense FP64 statevector forward and adjoint, "
                      f"{workers} spawned processes, {wall:.1f} s wall (per-vector CPU {max(res):.1f} s)"}


def extra_workloads(B, inputs, sptr, peaks):
    """The other forms and workloads, each measured once outside the headline's
    timed region (CUDA events on the handle's stream), each with its error
    against the closed form and its roofline against the measured peaks."""
    import numpy as np
    import torch

    from oracle import reduced
    out = {}
    stream = torch.cuda.current_stream()
    sms = peaks["sms"]
    fp64, fp32 = peaks["fp64_fma_tflops"], peaks["fp32_fma_tflops"]

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1000.0, r

    # precision forms at the full n = 29 workload (errors vs the closed form)
    inst = inputs.config_n29()
    Pc, awc, _ = reduced.closed_form(inst.n, inst.M, inst.k)
    for dt in ("c64", "dw"):
        g = B.GroverMPS(inst.n, inst.marked, dtype=dt, apply=APPLY, chi_max=inst.chi_max, stream=sptr)
        sec, _ = timed(lambda: g.iterate(inst.k))
        p = g.prob_marked()
        a = g.amplitude(inst.marked[0])
        bits = g.sample(4096, SAMPLE_SEED)
        chi = g.stats()["max_bond"]
        ex = inst.k * executed_flops_per_iter(inst.n, chi, inst.M, APPLY)
        nom = inst.k * algorithmic_flops_per_iter(inst.n, chi, inst.M, APPLY)
        ent = {"iterations_per_s": inst.k / sec, "P_marked": p, "P_err": p - Pc, "amp_err": abs(a - awc),
               "shots_4096_marked": int(np.sum(bits == inst.marked[0])), "max_bond": chi}
        if dt == "c64":
            ent["dtype"] = "c64 storage and contraction, FP64 QR/SVD and bookkeeping"
            ent["roofline"] = roofline_alu(ex, sec, fp64, "FP64 FMA", 1, sms, nom)
            ent["roofline"]["note"] = "the FP64 QR/SVD set the bound; the contraction runs on the FP32 pipes"
        else:
            ent["dtype"] = "f32x2 double-word on the FP32 pipes"
            ent["roofline"] = roofline_alu(ex, sec, fp32, "FP32 FMA", 1, sms, nom)
            ent["roofline"]["note"] = "each double-word flop costs several FP32 instructions"
        out[f"n29_{dt}"] = ent
        g.close()
    # batched: the 512-instance workload with its full k_i = min(floor(pi/4
    # sqrt(2^n/M)), 4000); the autotuner's timed slices (k_i capped at 10) are
    # the warm-up, and the one timed run includes the CUDA-graph capture
    from paper_2601_03832_gb300 import autotune
    insts = inputs.config_batched(count=512)
    thr, rec = autotune.tune_batch(insts, dtype="c64", apply=APPLY, kslice=10, stream=sptr)
    bt = B.GroverBatch(insts, dtype="c64", apply=APPLY, stream=sptr)
    bt.set_threads(thr)
    sec, _ = timed(lambda: bt.run(use_graph=True))
    p, st, rc = bt.result()
    errs, rel = [], []
    flops = nflops = 0.0
    busy, t0s, t1s, longest = {}, [], [], 0.0
    bad_bonds = 0
    for i, x in enumerate(insts):
        P = reduced.closed_form(x.n, x.M, x.k)[0]
        errs.append(abs(p[i] - P))
        rel.append(abs(p[i] - P) / P)
        s_ = bt.stats(i)
        flops += x.k * executed_flops_per_iter(x.n, s_["max_bond"], x.M, APPLY)
        nflops += x.k * algorithmic_flops_per_iter(x.n, s_["max_bond"], x.M, APPLY)
        d = (s_["t_end_ns"] - s_["t_begin_ns"]) / 1e9
        busy[s_["sm_id"]] = busy.get(s_["sm_id"], 0.0) + d
        t0s.append(s_["t_begin_ns"])
        t1s.append(s_["t_end_ns"])
        longest = max(longest, d)
        if s_["max_bond"] > x.M + 1:
            bad_bonds += 1
    span = (max(t1s) - min(t0s)) / 1e9
    tot = sum(x.k for x in insts)
    rl = roofline_alu(flops, sec, fp64, "FP64 FMA", sms, sms, nflops)
    out["batched_512_c64"] = {
        "iterations_per_s": tot / sec, "seconds": sec, "total_iterations": tot,
        "k": "full, min(floor(pi/4 sqrt(2^n/M)), 4000)", "threads": thr, "autotune": rec, "graph": True,
        "max_P_err": max(errs), "median_P_err": float(np.median(errs)), "max_P_rel_err": max(rel),
        "instances_with_status": int((st != 0).sum()), "instances_above_rank_M_plus_1": bad_bonds,
        "sm_busy": {"launch_span_s": span, "sms_used": len(busy),
                    "mean_busy_frac": sum(busy.values()) / (sms * span),
                    "longest_instance_s": longest,
                    "total_instance_s": sum(busy.values())},
        "roofline": rl}
    bt.close()
    out["batched_512_c64"]["cpu_baseline"] = cpu_baseline_batched(insts)
    # multi-marked n = 40, M = 32, chi_max = 128, tol = 1e-12, full k = 1000,
    # in the plain FP64 form and in the two precision forms
    mi = inputs.config_multi_marked(k=1000)
    Pm = reduced.closed_form(mi.n, mi.M, mi.k)[0]
    for dt, peak, pname in (("c128", fp64, "FP64 FMA"), ("c64", fp64, "FP64 FMA"), ("dw", fp32, "FP32 FMA")):
        g = B.GroverMPS(mi.n, mi.marked, dtype=dt, apply=APPLY, chi_max=mi.chi_max, tol=mi.tol, stream=sptr)
        g.iterate(1)                                                   # warm-up iteration
        g.reset()
        sec, _ = timed(lambda: g.iterate(mi.k))
        p = g.prob_marked()
        st_ = g.stats()
        chi = st_["max_bond"]
        out["n40_M32_" + dt] = {
            "iterations_per_s": mi.k / sec, "k": mi.k, "seconds": sec, "P_marked": p, "P_closed_form": Pm,
            "P_rel_err": (p - Pm) / Pm, "max_bond": chi,
            "jacobi_sweeps_per_svd": st_["jacobi_sweeps"] / max(1, st_["svd_count"]),
            "roofline": roofline_alu(mi.k * executed_flops_per_iter(mi.n, chi, mi.M, APPLY), sec, peak, pname, 1, sms,
                                     mi.k * algorithmic_flops_per_iter(mi.n, chi, mi.M, APPLY))}
        g.close()
    # the same instance with the oracle as a generic MPO of bond M + 1 = 33
    # (expanded bond 33 x 35 = 1155; QR matrices in the device work area),
    # a k = 5 slice
    mg = inputs.config_multi_marked(k=5)
    g = B.GroverMPS(mg.n, mg.marked, dtype="c128", apply="mpo", chi_max=mg.chi_max, tol=mg.tol, stream=sptr)
    g.iterate(1)                                                   # warm-up iteration
    g.reset()
    sec, _ = timed(lambda: g.iterate(mg.k))
    p = g.prob_marked()
    Pm = reduced.closed_form(mg.n, mg.M, mg.k)[0]
    gst = g.stats()
    chi = gst["max_bond"]
    # QR at the expanded bond X = (M+1) chi_l for the oracle, 2 chi_l for the
    # diffusion, on matrices of 2 r_l rows with r_l <= chi + M the rank the
    # QR reveals; SVD at the kept bonds
    out["n40_M32_generic_mpo_c128"] = {
        "iterations_per_s": mg.k / sec, "k_slice": mg.k, "seconds": sec, "P_rel_err": (p - Pm) / Pm, "max_bond": chi,
        "expanded_bond": (mg.M + 1) * 35, "ctas": gst["ctas"],
        "roofline": roofline_alu(mg.k * executed_flops_per_iter(mg.n, chi, mg.M, "mpo"), sec, fp64, "FP64 FMA",
                                 gst["ctas"], sms, mg.k * algorithmic_flops_per_iter(mg.n, chi, mg.M, "mpo"))}
    g.close()
    # differentiable: n = 20, M = 4, K = 64, the batch of 64 phase vectors,
    # forward + backward of all 64
    from paper_2601_03832_gb300 import autograd as AG
    di, phi, psi = inputs.config_differentiable(B=64)
    AG.loss_and_grad_batch(di.n, di.marked, phi[:2], psi[:2])          # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Ls, gphis, gpsis = AG.loss_and_grad_batch(di.n, di.marked, phi, psi)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    worst = 0.0
    for b in range(len(phi)):
        L, rphi, rpsi = reduced.loss_and_grad(di.n, di.M, phi[b], psi[b])
        worst = max(worst, abs(Ls[b] - L), float(np.abs(gphis[b] - rphi).max()), float(np.abs(gpsis[b] - rpsi).max()))
    # forward K iterations, segment recompute K iterations, costate K steps
    dflops = len(phi) * 3 * di.k * executed_flops_per_iter(di.n, di.M + 1, di.M, APPLY)
    dnom = len(phi) * 3 * di.k * algorithmic_flops_per_iter(di.n, di.M + 1, di.M, APPLY)
    out["differentiable_n20_M4_K64"] = {"fwd_bwd_ms_per_vector": 1000 * sec / len(phi), "vectors": len(phi),
                                        "wall_s": sec, "max_err_vs_reduced_model": worst,
                                        "roofline": roofline_alu(dflops, sec, fp64, "FP64 FMA",
                                                                 min(len(phi), sms), sms, dnom),
                                        "cpu_baseline": cpu_baseline_differentiable(di, phi, psi)}
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    budget = max(3.0, 60.0 / max(1, args.steps + args.warmup))
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(budget)
        if i >= args.warmup:
            vals.append(cb["value"])
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": "MPS Grover iterations/s (n=29, M=1, FP64)", "value": v,
            "unit": "iterations/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * K_ITERS / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "n29_M1_k18198 plain Grover MPS, chi_max=4, FP64", "n": N_SITES, "M": 1,
                       "k": K_ITERS, "chi_max": CHI_MAX, "apply": APPLY},
            "cpu_baseline": {"value": v, "unit": "iterations/s", "cores": 1, "kind": "oracle",
                             "sample": f"per step a {budget:.0f} s slice of the n=29 iterations (NumPy FP64 MPS oracle, "
                                       "1 thread); ms_per_step extrapolates the slice to k=18198"},
            "ms_per_step_extrapolated": True,
            "e2e": {"value": v, "unit": "iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other forms and workloads")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    from paper_2601_03832_gb300 import binding as B
    from paper_2601_03832_gb300 import inputs

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    B.load()
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    from paper_2601_03832_gb300 import peaks as PK
    peaks = PK.measure()
    inst = inputs.config_n29()
    k = inst.k
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    g = B.GroverMPS(inst.n, inst.marked, dtype="c128", apply=APPLY, chi_max=inst.chi_max, stream=sptr)

    def step(record=None):
        g.reset()
        if record is not None:
            record[0].record(stream)
        g.iterate(k)
        if record is not None:
            record[1].record(stream)
        p = g.prob_marked()
        a = g.amplitude(inst.marked[0])
        bits = [g.sample(s, SAMPLE_SEED) for s in SHOTS]
        return p, a, bits

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = B.launch_count()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for i in range(args.steps):
            flush.zero_()                      # L2 flush between timed steps (outside the events)
            ev[i][0].record(stream)
            res = step(kev[i])
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    launches = B.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = [a.elapsed_time(b) for a, b in kev]
    ms_per_step, value = replica_rate(sum(step_ms), args.steps, k)

    # ---- end to end through the C ABI with host buffers (create .. destroy)
    e2e_ms = []
    h2d = 8 * inst.M                                         # marked strings
    d2h = 16 * inst.M + 16 + 8 * sum(SHOTS)                  # amplitudes, P, shots
    for i in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ge = B.GroverMPS(inst.n, inst.marked, dtype="c128", apply=APPLY, chi_max=inst.chi_max, stream=sptr)
        ge.iterate(k)
        pe = ge.prob_marked()
        ae = ge.amplitude(inst.marked[0])
        be = [ge.sample(s, SAMPLE_SEED) for s in SHOTS]
        ge.close()
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    _, e2e_val = replica_rate(sum(e2e_ms), len(e2e_ms), k)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    from oracle import reduced
    p, a, bits = res
    Pc, awc, arc = reduced.closed_form(inst.n, inst.M, k)
    st = g.stats()
    chi = max(st["chi"])
    flops = k * executed_flops_per_iter(inst.n, chi, inst.M, APPLY)
    kern_s = statistics.mean(kern_ms) / 1000.0
    roof = roofline_alu(flops, kern_s, peaks["fp64_fma_tflops"], "FP64 FMA", 1, peaks["sms"],
                        k * algorithmic_flops_per_iter(inst.n, chi, inst.M, APPLY))
    roof.update({"traffic": CAPTURE["traffic_bytes"], "kernel": "iterate_kernel<double,double2,double>",
                 "algorithmic_flops_per_launch": flops, "kernel_ms": statistics.mean(kern_ms)})
    if CAPTURE["fp64_pipe_share"] is not None:
        roof["chain_bound"] = {"model": "FP64 issue bound: the instance's FP64 warp instructions back to back "
                                        "on one SM sub-partition's pipe, as a share of the launch",
                               "frac": CAPTURE["fp64_pipe_share"],
                               "source": "ncu capture of the iterate kernel at n=29, k=50"}
    line = {
        "metric": "MPS Grover iterations/s (n=29, M=1, FP64)",
        "value": value, "unit": "iterations/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "n29_M1_k18198 plain Grover MPS, chi_max=4, FP64 (complex128), "
                               "G applied as one direct-sum contraction + QR sweep + truncated SVD sweep",
                   "n": inst.n, "M": inst.M, "k": k, "chi_max": inst.chi_max, "apply": APPLY,
                   "shots": list(SHOTS), "marked_seed": 3, "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "flushed between timed steps (256 MiB write outside the events)"},
        "results": {"P_marked": p, "P_closed_form": Pc, "P_err": p - Pc, "amp_marked": [a.real, a.imag],
                    "amp_closed_form": awc, "shots_4096_marked": int(np.sum(bits[0] == inst.marked[0])),
                    "shot_1": int(bits[1][0]), "max_bond": chi, "jacobi_sweeps_max": st["max_jacobi_sweeps"],
                    "discarded_weight": st["discarded_weight"]},
        "roofline": roof,
        "peaks": peaks,
        "e2e": {"value": e2e_val, "unit": "iterations/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": statistics.mean(e2e_ms)},
        "gpu_launches": launches,
    }
    clk_sum = clk.summary()
    line["clocks"] = clk_sum
    if not args.no_extras and ws == 1:
        line["workloads"] = extra_workloads(B, inputs, sptr, peaks)
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline()
    g.close()
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
