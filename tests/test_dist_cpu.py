"""The multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1)
agree on the whole-job rate (the slowest rank's time, world x the units of
one rank), and the oracle reference arm runs on rank 0 only."""
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [100.0, 250.0][rank]
        q.put((rank, bench.whole_job_rate(local_ms, world, 1e12, 10, torch.device("cpu"))))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        max_ms, value = res[r]
        assert max_ms == 250.0
        assert value == pytest.approx(2 * 1e12 * 10 / 0.25 / 1e12)


def test_single_rank_rate_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(50.0, 1, 2e12, 5, torch.device("cpu")) == (50.0, pytest.approx(2e12 * 5 / 0.05 / 1e12))


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_class_rooflines_cover_every_contraction_class():
    """The bench line's per-class rooflines: each contraction class present in
    the profile gets TFLOP/s against the sustained peak; absent ones are left
    out; the attention forward also gets its exponential bound."""
    import bench
    prof = {n: {"flops": 2e12, "ms": 10.0, "bytes": 1e9, "launches": 4}
            for n in ("gemm_tc", "attn_fwd_tc", "attn_bwd_tc", "tri_einsum", "opm_outer", "mlp_fused")}
    prof["ln_fwd"] = {"flops": 0.0, "ms": 1.0, "bytes": 1e9, "launches": 2}
    peaks = {"bf16_sus": 1000.0, "hbm": 5000.0}
    out = bench.class_rooflines(prof, peaks, {"sm_mhz": 2000.0}, {"f32": 1e13})
    assert set(out) == {"gemm_tc", "attn_fwd_tc", "attn_bwd_tc", "tri_einsum", "opm_outer", "mlp_fused"}
    for e in out.values():
        assert abs(e["tflops"] - 200.0) < 1e-9 and abs(e["tensor_frac"] - 0.2) < 1e-12
        assert abs(e["hbm_frac_of_operand_bytes"] - 0.02) < 1e-12
    assert abs(out["attn_fwd_tc"]["exp_bound_ms"] - 1e3 * 2e12 / 128.0 / 1e13) < 1e-9
    del prof["mlp_fused"]
    assert "mlp_fused" not in bench.class_rooflines(prof, peaks, None, None)
