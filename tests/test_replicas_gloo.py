"""The multi-GPU form of the benchmark is N independent replicas (a single
instance's sweep is a site-sequential chain and does not shard).  Its host
logic -- max over ranks of the timed region, whole-job value = N k / time --
is checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r's timed region took 1000 (r + 1) ms over 2 steps of k = 100 iterations
        ms, value = bench.replica_rate(1000.0 * (rank + 1), 2, 100)
        q.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_replica_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, value in got:
        assert ms == pytest.approx(1000.0)      # slowest rank: 2000 ms / 2 steps
        assert value == pytest.approx(200.0)    # 2 replicas x 100 iterations / 1 s


def test_replica_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    ms, value = bench.replica_rate(500.0, 5, 50)
    assert ms == pytest.approx(100.0) and value == pytest.approx(500.0)


def test_flop_model_matches_the_stated_counts():
    """The roofline's algorithmic flops per iteration (Householder QR + thin Q
    2*4(2mn^2 - 2n^3/3), thin SVD 4(14mn^2 + 8n^3), 8 flops per complex MAC)
    at the n = 12 and n = 29 workloads: ~1.8e5 (MPO form) and ~8.6e4 (direct
    sum) at n = 12, 2.27e5 for the fused n = 29 headline."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.algorithmic_flops_per_iter(12, 2, 1, "mpo") == pytest.approx(1.8e5, rel=0.02)
    assert bench.algorithmic_flops_per_iter(12, 2, 1, "fused") == pytest.approx(8.6e4, rel=0.05)
    assert bench.algorithmic_flops_per_iter(29, 2, 1, "fused") == pytest.approx(2.27e5, rel=0.01)


def test_executed_flop_model_hand_count():
    """The executed count at n = 2, chi = 1, M = 1 (fused, X = chi + M + 1 = 3,
    one site step), worked by hand: Householder QR of the 2 x 3 matrix with one
    reflector, (3 - 1) trailing columns x 2 rows x 20 flops = 80; thin Q from
    it, 8 x 2 = 16; thin SVD of 1 x 2, 4 (14 * 2 * 1 + 8) = 144; contraction
    8 * 1 * 2 * 3 = 48 plus the absorption 8 * 1 * 2 * 1 = 16: 304 in all.  At
    every workload it stays below the nominal full-rank count."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.executed_flops_per_iter(2, 1, 1, "fused") == 304
    for n, chi, M, apply in ((29, 2, 1, "fused"), (40, 33, 32, "fused"), (40, 33, 32, "mpo"), (20, 5, 4, "split")):
        assert bench.executed_flops_per_iter(n, chi, M, apply) < bench.algorithmic_flops_per_iter(n, chi, M, apply)


def test_oracle_pool_baselines_run_on_cpu():
    """The batched and differentiable CPU baselines of the bench run the
    oracle in spawned processes (one BLAS thread each) and report the cores
    they used; a tiny sample of each finishes on the CPU alone."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2601_03832_gb300 import inputs
    insts = inputs.config_batched(count=512)
    rec = bench.cpu_baseline_batched(insts, kslice=1, count=2)
    assert rec["kind"] == "oracle" and rec["value"] > 0 and rec["cores"] >= 1
    assert "first 2 of the 512 instances" in rec["sample"]
    di, phi, psi = inputs.config_differentiable(B=64)
    small = type(di)(n=10, marked=[3, 700], k=4, chi_max=di.chi_max, tag="small")
    rec = bench.cpu_baseline_differentiable(small, phi[:, :4], psi[:, :4], vectors=1)
    assert rec["value"] > 0 and rec["cores"] == 1
