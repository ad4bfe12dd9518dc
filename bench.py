#!/usr/bin/env python
"""Benchmark of one Evoformer block forward + backward on GB300.

Workload: the paper's initial-training crop (Table "model settings":
N_seq=128, N_res=256; C_m=256, C_z=128, 8 MSA heads as in the per-layer
timing table), BF16 activations with FP32 accumulation, 5% padded residues,
seeded synthetic inputs.  One step = BF16 copy of the parameters, block
forward, block backward (which recomputes the forward: per-block recompute)
through the C ABI of libevo.so.

Metric: algorithmic TFLOP/s = 3 x (forward contraction flops) / time, the
backward counted as twice the forward and the recompute not counted.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead (on host cores, rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Evoformer block fwd+bwd ms & TFLOP/s, BF16 vs FP32, GB300, N_res=256 N_seq=128"
L2_BYTES = 129 * 2 ** 20


def block_fwd_flops(d) -> float:
    """Algorithmic forward flops of one block (2 flops per multiply-add of every contraction)."""
    S, R, Cm, Cz = d.n_seq, d.n_res, d.c_m, d.c_z
    Mm, Mz = S * R, R * R
    HCm, HCt = d.h_msa * d.c_msa, d.h_tri * d.c_tri
    f = 0.0
    # MSA row attention with pair bias
    f += 2 * Mm * Cm * 4 * HCm + 2 * Mz * Cz * d.h_msa + 4 * S * d.h_msa * R * R * d.c_msa + 2 * Mm * HCm * Cm
    # MSA column attention (global column attention in the extra-MSA block)
    if d.msa_col_mode == 0:
        f += 2 * Mm * Cm * 4 * HCm + 4 * R * d.h_msa * S * S * d.c_msa + 2 * Mm * HCm * Cm
    else:
        f += 2 * Mm * Cm * (2 * HCm + 2 * d.c_msa) + 4 * S * R * HCm + 2 * Mm * HCm * Cm
    # MSA transition
    f += 2 * 2 * Mm * Cm * d.trans_n * Cm
    # outer product mean
    co = d.c_opm
    f += 2 * Mm * Cm * 2 * co + 2 * (R * co) ** 2 * S + 2 * Mz * co * co * Cz
    # triangle multiplication x2
    f += 2 * (2 * Mz * Cz * (4 * d.c_mul + Cz) + 2 * d.c_mul * R ** 3 + 2 * Mz * d.c_mul * Cz)
    # triangle attention x2
    f += 2 * (2 * Mz * Cz * d.h_tri + 2 * Mz * Cz * 4 * HCt + 4 * R * d.h_tri * R * R * d.c_tri + 2 * Mz * HCt * Cz)
    # pair transition
    f += 2 * 2 * Mz * Cz * d.trans_n * Cz
    return float(f)


def pair_block_fwd_flops(d) -> float:
    """Algorithmic forward flops of one template pair stack block (the pair steps alone)."""
    R, Cz = d.n_res, d.c_z
    Mz, HCt = R * R, d.h_tri * d.c_tri
    f = 2 * (2 * Mz * Cz * (4 * d.c_mul + Cz) + 2 * d.c_mul * R ** 3 + 2 * Mz * d.c_mul * Cz)
    f += 2 * (2 * Mz * Cz * d.h_tri + 2 * Mz * Cz * 4 * HCt + 4 * R * d.h_tri * R * R * d.c_tri + 2 * Mz * HCt * Cz)
    f += 2 * 2 * Mz * Cz * d.trans_n * Cz
    return float(f)


def step_flops(d) -> float:
    return 3.0 * block_fwd_flops(d)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return dict(hbm=j["hbm_gbs"], bf16=j["bf16_tflops"], bf16_sus=j["bf16_tflops_sustained"], src="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, src="fallback")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if len(r) > 5 + k and "Active" in r[5 + k]
                          and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def whole_job_rate(local_ms, world, flops_per_unit, units, device):
    """Weak-scaling whole-job rate: every rank processed `units` units of
    `flops_per_unit` in `local_ms`; the job takes the slowest rank's time
    (max over ranks) and processed world x units.  Returns (max_ms, TFLOP/s)."""
    import torch
    t = torch.tensor([local_ms], device=device, dtype=torch.float64)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    max_ms = float(t.item())
    return max_ms, world * flops_per_unit * units / (max_ms / 1e3) / 1e12


def run_oracle_step(d, prob):
    from oracle import evoformer as O
    from paper_2207_05477_gb300 import synth
    p = synth.unpack_params(d, prob["params"])
    t0 = time.perf_counter()
    O.block_forward_backward(prob["m"], prob["z"], prob["msa_mask"], prob["pair_mask"], p, d, prob["gm"], prob["gz"])
    return time.perf_counter() - t0


def cpu_baseline(d, seed):
    """The FP64 oracle timed once on the host cores: one full block fwd+bwd of the workload."""
    import torch
    from paper_2207_05477_gb300 import synth
    prob = synth.make_problem(d, seed, pad_frac=0.05)
    t = run_oracle_step(d, prob)
    return {"value": step_flops(d) / t / 1e12, "unit": "TFLOP/s", "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"one FP64 block fwd+bwd at N_seq={d.n_seq} N_res={d.n_res} (the full step), {t:.1f} s",
            "seconds": t}


# ---------------------------------------------------------------- reference arm
def reference_arm(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import torch
    from paper_2207_05477_gb300 import synth
    full = synth.Dims(n_seq=args.n_seq, n_res=args.n_res)
    # Each step is the whole workload (one FP64 block fwd+bwd, about 7.5 s on
    # 16 host cores at the training crop) when the run stays within about
    # four minutes; otherwise a bounded sample: the same block on a
    # 128-residue crop (about 1.2 s)
    whole = (args.steps + args.warmup) * 7.5 * (full.n_seq * full.n_res ** 2) / (128 * 256 ** 2) <= 240.0
    d = full if whole else full.replace(n_res=min(128, args.n_res))
    prob = synth.make_problem(d, 32, pad_frac=0.05)
    for _ in range(args.warmup):
        run_oracle_step(d, prob)
    ts = [run_oracle_step(d, prob) for _ in range(args.steps)]
    tot = sum(ts)
    v = step_flops(d) * args.steps / tot / 1e12
    sample = (f"one FP64 block fwd+bwd per step, the whole workload (N_seq={d.n_seq}, N_res={d.n_res})" if whole else
              f"one FP64 block fwd+bwd per step on an N_seq={d.n_seq}, N_res={d.n_res} crop of the workload")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"Evoformer block fwd+bwd, N_seq={full.n_seq} N_res={full.n_res}, c_m=256 c_z=128",
                       "sample": sample},
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
SFU_EX2_PER_CLK_SM = 16  # nominal special-function-unit ex2 rate of one SM
N_SM = 152


def measure_ex2_rate(evo, dev):
    """The special-function unit's exponential throughput on this GPU (the
    library's probe kernel, CUDA events, best of five launches): ex2 results
    per second for ex2.approx.f32 and ex2.approx.bf16x2."""
    import torch
    blocks, iters = N_SM * 8, 1024
    sink = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    out = {}
    for variant, name in ((0, "f32"), (1, "bf16x2")):
        evo.probe_ex2(variant, blocks, iters, sink)
        best = None
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            evo.probe_ex2(variant, blocks, iters, sink)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        out[name] = blocks * 256 * 8 * iters * (variant + 1) / (best / 1e3)
    return out


def class_rooflines(prof, peaks, clk, ex2_rate=None):
    """Per kernel class of the step: achieved TFLOP/s and fraction of the
    sustained BF16 tensor peak for the contractions (attention forward and
    backward, triangle einsum, outer-product contraction, the fused
    transition MLP, every other GEMM),
    and for the attention forward also against the exponential bound: one
    ex2 per (query, key) pair and 4 c flops per pair at head dim c = 32, so
    its flops / 128 exponentials at 16 per clock per SM."""
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    nominal = SFU_EX2_PER_CLK_SM * N_SM * mhz * 1e6
    rate = (ex2_rate or {}).get("f32") or nominal
    out = {}
    for name in ("gemm_tc", "attn_fwd_tc", "attn_bwd_tc", "tri_einsum", "opm_outer", "mlp_fused"):
        v = prof.get(name)
        if not v or not v["flops"] or not v["ms"]:
            continue
        tf = v["flops"] / (v["ms"] / 1e3) / 1e12
        e = {"tflops": tf, "tensor_frac": tf / peaks["bf16_sus"], "ms": v["ms"], "launches": v["launches"]}
        if v["bytes"]:
            e["hbm_frac_of_operand_bytes"] = v["bytes"] / (v["ms"] / 1e3) / 1e9 / peaks["hbm"]
        if name == "attn_fwd_tc":
            t_exp = v["flops"] / 128.0 / rate
            e["exp_bound_ms"] = 1e3 * t_exp
            e["exp_frac"] = 1e3 * t_exp / v["ms"]
            e["exp_rate"] = {"per_s": rate, "source": "measured (ex2.approx.f32 probe)" if ex2_rate else
                             f"nominal {SFU_EX2_PER_CLK_SM} ex2/clk/SM x {N_SM} SMs at {mhz:.0f} MHz",
                             "nominal_per_s": nominal}
        out[name] = e
    return out
PROFILE_EVERY = 10
TUNE_PASSES = 12  # at least the largest candidate count of a GEMM shape


def autotune(evo, run_once, passes):
    """GEMM tile autotuning before the warm-up: `passes` untimed runs of the
    workload cycle every GEMM shape through its candidate tile widths (and
    split counts); the library keeps the fastest per shape."""
    import torch
    torch.cuda.synchronize()
    evo.tune_begin()
    for _ in range(passes):
        run_once()
    n = evo.tune_end()
    ents = evo.tune_entries()
    changed = [f"{e['M']}x{e['N']}x{e['K']}*{e['batch']}: n{e['default_bn']}s{e['default_splits']}"
               f"->n{e['bn']}s{e['splits']}" for e in ents
               if (e["bn"], e["splits"]) != (e["default_bn"], e["default_splits"])]
    return {"shapes": n, "changed": len(changed), "choices": changed}


def ours_arm(args):
    import torch
    from paper_2207_05477_gb300 import evo, synth
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    evo.lib()

    d = synth.Dims(n_seq=args.n_seq, n_res=args.n_res)
    act = evo.EVO_BF16 if args.dtype == "bf16" else evo.EVO_F32
    tdt = torch.bfloat16 if act == evo.EVO_BF16 else torch.float32
    cd = evo.cdims(d, act)
    seed = 32 + rank
    prob = synth.make_problem(d, seed, pad_frac=0.05)

    # device-resident inputs
    params = torch.tensor(prob["params"], device=dev)
    p16 = torch.empty(evo.param_count(cd), dtype=torch.bfloat16, device=dev) if act == evo.EVO_BF16 else None
    m = torch.tensor(prob["m"], device=dev).to(tdt)
    z = torch.tensor(prob["z"], device=dev).to(tdt)
    mm = torch.tensor(prob["msa_mask"], device=dev)
    pm = torch.tensor(prob["pair_mask"], device=dev)
    gm = torch.tensor(prob["gm"], device=dev).to(tdt)
    gz = torch.tensor(prob["gz"], device=dev).to(tdt)
    m_out, z_out = torch.empty_like(m), torch.empty_like(z)
    dm, dz = torch.empty_like(m), torch.empty_like(z)
    dparams = torch.zeros_like(params)
    ws_f = evo.workspace(cd, evo.EVO_MODE_FWD, dev)
    ws_b = evo.workspace(cd, evo.EVO_MODE_BWD, dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # training-mode dropout (--dropout): the seeded scales of the five AF2
    # sites, device-resident like the other inputs
    drop = {k: torch.tensor(v, device=dev) for k, v in synth.make_dropout(d, seed).items()} if args.dropout else None

    def step(mi, zi, mmi, pmi, gmi, gzi, prm, out=None, dr=None):
        # out: (m_out, z_out, dm, dz, dparams) of this step (default: the timed buffers)
        mo, zo, dmo, dzo, dpo = out if out is not None else (m_out, z_out, dm, dz, dparams)
        dr = drop if dr is None else dr
        if p16 is not None:
            evo.params_to_bf16(cd, prm, p16)
        if dr is None:
            evo.block_fwd(cd, prm, p16, mi, zi, mo, zo, mmi, pmi, ws_f)
            evo.block_bwd(cd, prm, p16, mi, zi, mmi, pmi, gmi, gzi, dmo, dzo, dpo, ws_b)
        else:
            evo.block_fwd_dropout(cd, prm, p16, mi, zi, mo, zo, mmi, pmi, dr, ws_f)
            evo.block_bwd_dropout(cd, prm, p16, mi, zi, mmi, pmi, dr, gmi, gzi, dmo, dzo, dpo, ws_b)

    tuned = autotune(evo, lambda: step(m, z, mm, pm, gm, gz, params), TUNE_PASSES) \
        if act == evo.EVO_BF16 and not args.no_tune else None
    for _ in range(args.warmup):
        step(m, z, mm, pm, gm, gz, params)
    torch.cuda.synchronize()
    if evo.get_error() != evo.EVO_OK:
        raise RuntimeError("device error word set during warm-up")

    graph = None
    if args.graph:
        # the whole step (parameter copy, forward, backward) as one CUDA graph; the
        # library's per-kernel event records are captured with it and hold the
        # times of the last replay
        gstream = torch.cuda.Stream()
        gstream.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gstream):
            step(m, z, mm, pm, gm, gz, params)
        stream.wait_stream(gstream)
        graph.replay()
        torch.cuda.synchronize()

    # one profiled eager step before the timed region names the dominant kernel class
    torch.cuda.synchronize()
    evo.profile_begin()
    step(m, z, mm, pm, gm, gz, params)
    pre = evo.profile_end()
    dom_name = max(pre.items(), key=lambda kv: kv[1]["ms"])[0]

    # ---- timed region: K steps, L2 flushed between steps (outside each step's events).
    # In every PROFILE_EVERY-th eager step one event pair brackets each launch
    # of the dominant kernel class (its live per-launch times for the
    # roofline); the other steps run untouched, since an event between two
    # launches stops the next one from starting early.  A graph replay cannot
    # time launches inside it.
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    if graph is None:
        evo.profile_only(dom_name)
        evo.profile_begin()
        evo.profile_pause(True)
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        if graph is None:
            sampled = i % PROFILE_EVERY == PROFILE_EVERY - 1 or args.steps < PROFILE_EVERY
            if sampled:
                evo.profile_pause(False)
            step(m, z, mm, pm, gm, gz, params)
            if sampled:
                evo.profile_pause(True)
        else:
            graph.replay()
        ev[i][1].record(stream)
    dom_live = evo.profile_end() if graph is None else None
    torch.cuda.synchronize()
    if graph is not None:
        # launches inside a graph replay cannot be timed one by one: the
        # dominant class's live per-launch times come from eager steps after the
        # timed region, only that class bracketed by events (as in eager timing)
        evo.profile_only(dom_name)
        evo.profile_begin()
        for i in range(max(1, min(args.steps, PROFILE_EVERY))):
            flush.fill_(float(i))
            step(m, z, mm, pm, gm, gz, params)
        dom_live = evo.profile_end()
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = sorted(a.elapsed_time(b) for a, b in ev)
    dev_ms = sum(step_ms)
    pick = lambda q: step_ms[min(len(step_ms) - 1, int(q * (len(step_ms) - 1) + 0.5))]
    step_stats = {"p10": pick(0.1), "median": pick(0.5), "p90": pick(0.9)}
    if evo.get_error() != evo.EVO_OK:
        raise RuntimeError("device error word set during the timed steps")
    max_ms, value = whole_job_rate(dev_ms, world, step_flops(d), args.steps, dev)

    # ---- end to end through the C ABI with host buffers: H2D of the step's inputs, D2H of its results.
    # A training loop's pipelining: two device buffer sets (A, the timed one,
    # and B) alternate between steps, so that step k + 1's inputs are uploaded
    # and step k's results read back on two copy streams while the GPU
    # computes; every step's copies are inside the timed region (the first
    # upload after its start event, the last read-back before its end event).
    host = {k: torch.tensor(prob[k]).to(tdt if k in ("m", "z", "gm", "gz") else torch.float32).pin_memory()
            for k in ("m", "z", "msa_mask", "pair_mask", "gm", "gz", "params")}
    host_drop = {k: v.cpu().pin_memory() for k, v in drop.items()} if drop is not None else {}
    # the step's results: the forward outputs and every gradient
    res_names = ("m_out", "z_out", "dm", "dz", "dparams")
    out_a = (m_out, z_out, dm, dz, dparams)
    out_host = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in zip(res_names, out_a)}
    h2d = sum(v.numel() * v.element_size() for v in list(host.values()) + list(host_drop.values()))
    d2h = sum(v.numel() * v.element_size() for v in out_host.values())
    in_a = {"m": m, "z": z, "msa_mask": mm, "pair_mask": pm, "gm": gm, "gz": gz, "params": params}
    in_b = {k: torch.empty_like(v) for k, v in in_a.items()}
    out_b = tuple(torch.zeros_like(v) for v in out_a)
    drop_b = {k: torch.empty_like(v) for k, v in drop.items()} if drop is not None else None
    graph_b = None
    if graph is not None:  # a graph reads fixed device buffers: one per buffer set
        gstream = torch.cuda.Stream()
        gstream.wait_stream(stream)
        graph_b = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph_b, stream=gstream):
            step(in_b["m"], in_b["z"], in_b["msa_mask"], in_b["pair_mask"], in_b["gm"], in_b["gz"], in_b["params"],
                 out=out_b, dr=drop_b)
        stream.wait_stream(gstream)
    sets = [(in_a, out_a, drop, graph), (in_b, out_b, drop_b, graph_b)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    in_ready = [torch.cuda.Event(), torch.cuda.Event()]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    read = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(si):
        dst, _, dr, _ = sets[si]
        with torch.cuda.stream(up):
            for k in host:
                dst[k].copy_(host[k], non_blocking=True)
            for k in host_drop:  # the dropout draw of the step is an input too
                dr[k].copy_(host_drop[k], non_blocking=True)
            in_ready[si].record(up)

    e2e_steps = max(1, min(args.steps, 50))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    up.wait_event(e0)
    upload(0)
    for i in range(e2e_steps):
        si = i & 1
        din, dout, dr, g = sets[si]
        stream.wait_event(in_ready[si])
        if i >= 2:
            stream.wait_event(read[si])  # step i - 2's results have left this set's outputs
        if g is None:
            step(din["m"], din["z"], din["msa_mask"], din["pair_mask"], din["gm"], din["gz"], din["params"],
                 out=dout, dr=dr)
        else:
            g.replay()
        done[si].record(stream)
        if i + 1 < e2e_steps:
            if i >= 1:
                up.wait_event(done[si ^ 1])  # step i - 1 has read the other set's inputs
            upload(si ^ 1)
        down.wait_event(done[si])
        with torch.cuda.stream(down):
            for k, v in zip(res_names, dout):
                out_host[k].copy_(v, non_blocking=True)
            read[si].record(down)
    stream.wait_stream(down)
    stream.wait_stream(up)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_max_ms, e2e_value = whole_job_rate(e2e_ms, world, step_flops(d), 1, dev)

    # ---- plain FP32 path, same workload (the comparison the target names)
    fp32 = None
    if act == evo.EVO_BF16 and not args.no_fp32:
        cd32 = evo.cdims(d, evo.EVO_F32)
        m32, z32 = torch.tensor(prob["m"], device=dev), torch.tensor(prob["z"], device=dev)
        g32m, g32z = torch.tensor(prob["gm"], device=dev), torch.tensor(prob["gz"], device=dev)
        mo32, zo32, dm32, dz32 = (torch.empty_like(x) for x in (m32, z32, m32, z32))
        w32f, w32b = evo.workspace(cd32, evo.EVO_MODE_FWD, dev), evo.workspace(cd32, evo.EVO_MODE_BWD, dev)
        dp32 = torch.zeros_like(params)

        def step32():
            if drop is None:
                evo.block_fwd(cd32, params, None, m32, z32, mo32, zo32, mm, pm, w32f)
                evo.block_bwd(cd32, params, None, m32, z32, mm, pm, g32m, g32z, dm32, dz32, dp32, w32b)
            else:
                evo.block_fwd_dropout(cd32, params, None, m32, z32, mo32, zo32, mm, pm, drop, w32f)
                evo.block_bwd_dropout(cd32, params, None, m32, z32, mm, pm, drop, g32m, g32z, dm32, dz32, dp32, w32b)

        step32()
        torch.cuda.synchronize()
        n32 = 3
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n32):
            step32()
        b.record(stream)
        torch.cuda.synchronize()
        ms32 = a.elapsed_time(b) / n32
        fp32 = {"ms_per_step": ms32, "tflops": step_flops(d) / (ms32 / 1e3) / 1e12,
                "bf16_speedup": ms32 / (max_ms / args.steps)}
        del w32f, w32b

    # ---- per-kernel profile: eager steps after the timed region, every launch timed
    torch.cuda.synchronize()
    prof_steps = max(1, min(args.steps, 10))
    evo.profile_begin()
    for i in range(prof_steps):
        flush.fill_(float(i))
        step(m, z, mm, pm, gm, gz, params)
    prof = evo.profile_end()
    launches = int(round(sum(v["launches"] for v in prof.values()) / prof_steps)) * args.steps

    # ---- roofline of the dominant kernel class: live event times of the timed
    # steps (eager), else of the profiled steps (graph replay)
    peaks = load_peaks()
    dom = (dom_live or prof)[dom_name]
    dom_src = ("eager steps after the timed graph replays" if graph is not None
               else f"every {PROFILE_EVERY}th timed step" if args.steps >= PROFILE_EVERY else "timed steps")
    dom_ms_per_launch = dom["ms"] / max(dom["launches"], 1)
    # the bound a class is judged against: the contractions (every class with
    # algorithmic flops) against the tensor peak, the rest against HBM; the
    # other fraction is reported beside it
    if dom["flops"]:
        achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12
        roof = {"kernel": dom_name, "bound": "tensor", "achieved": achieved, "peak": peaks["bf16_sus"],
                "unit": "TFLOP/s", "frac": achieved / peaks["bf16_sus"],
                "peak_kind": f"bf16 dense sustained, {peaks['src']}"}
        if dom["bytes"]:
            gbs = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
            roof["hbm_of_operand_bytes"] = {"achieved_gbs": gbs, "frac": gbs / peaks["hbm"],
                                            "note": "operand bytes of each launch as issued (every materialised "
                                                    "intermediate counted), against the HBM copy peak"}
    else:
        achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
        roof = {"kernel": dom_name, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm"], "unit": "GB/s",
                "frac": achieved / peaks["hbm"], "peak_kind": f"HBM copy, {peaks['src']}"}
    roof["ms_per_launch"] = dom_ms_per_launch
    roof["launches_timed"] = int(dom["launches"])
    roof["times_from"] = dom_src
    roof["algorithmic"] = {"flops_per_launch": dom["flops"] / max(dom["launches"], 1),
                           "bytes_per_launch": dom["bytes"] / max(dom["launches"], 1)}
    roof["share_of_step"] = prof[dom_name]["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-9)
    roof["traffic"] = None
    tfile = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if os.path.exists(tfile):
        with open(tfile) as f:
            tr = json.load(f)
        ent = tr.get(dom_name, {})
        # the capture's figure holds for its own workload shape only
        same = ent.get("n_seq") == d.n_seq and ent.get("n_res") == d.n_res and not args.dropout
        if ent.get("valid", False) and same:
            roof["traffic"] = ent["bytes_per_launch"]

    ex2 = measure_ex2_rate(evo, dev)
    roof["classes"] = class_rooflines(prof, peaks, clk, ex2)
    roof["ex2_rate_per_s"] = ex2

    kernels = {k: {"ms_per_step": v["ms"] / prof_steps, "launches_per_step": v["launches"] / prof_steps,
                   "share": v["ms"] / max(sum(x["ms"] for x in prof.values()), 1e-9),
                   "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12) if v["flops"] else None,
                   "gbs": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["bytes"] else None}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(d, 32)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": f"Evoformer block fwd+bwd (per-block recompute), N_seq={d.n_seq} N_res={d.n_res}, "
                                   f"c_m=256 c_z=128, 5% padded residues",
                       "n_seq": d.n_seq, "n_res": d.n_res, "flops_per_step": step_flops(d),
                       "l2": "flushed between timed steps (258 MB write outside the step events)",
                       "parallelism": f"replicas x{world}", "cuda_graph": bool(args.graph),
                       "dropout": "training mode, AF2 rates (0.15 MSA row, 0.25 pair), seeded draws as inputs"
                       if args.dropout else "evaluation mode (none)",
                       "gemm_tiles": ("autotuned before the warm-up: " + json.dumps(tuned)) if tuned else "built-in"},
            "clocks": clk, "gpu_launches": launches, "step_ms": step_stats,
            "e2e": {"value": e2e_value, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_max_ms, "steps": e2e_steps,
                    "how": "pinned host inputs copied in and every result copied out each step, on two copy "
                           "streams overlapping the previous / next step's compute (two device buffer sets); "
                           "no L2 flush: each step's inputs arrive by copy from the host"},
            "roofline": roof, "cpu_baseline": cpu, "fp32_plain": fp32, "kernels": kernels,
            "paper_context": {"ms_per_layer_fwd_bwd": 32.47, "hardware": "A100 40G, FP16, PPFold DAP=1 BP=1"},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------- other workloads
def other_workload(args):
    """The paper's other shapes, one JSON line each (not the headline):
    small_fp32_fwd  one block forward, plain FP32 path, N_seq=16 N_res=64
    extra_msa       extra-MSA block fwd+bwd (global column attention), N_extra=1024 N_res=256 c_e=64
    stack48         48-block stack fwd+bwd, N_seq=512 N_res=384, per-block recompute (block inputs kept)
    long2048        one block forward at N_res=2048, N_seq=128
    long4096        one block forward at N_res=4096, N_seq=128 in the inference workspace plan
    long4096_slab   the same with the pair stack subbatched in i-slabs of 512 rows (Sec. 3.4.4)
    long8192_slab   one block forward at N_res=8192, N_seq=128, i-slabs of 1024 rows
    batch16         16 proteins (N_res ~ U[64,1024], N_seq ~ U[32,512], seeded), 48-block forward each
    template_pair   template pair stack block fwd+bwd (AF2 Alg. 16), N_res=256, c_t=64, dropout
    adam48          fused training update (global-norm clip, Adam, EMA, BF16 copy) over the flat
                    parameter buffer of the 48-block stack at the paper's dims (Sec. 3.2 tensor fusion)
    """
    import numpy as np
    import torch
    from paper_2207_05477_gb300 import evo, synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    evo.lib()
    stream = torch.cuda.current_stream()
    peaks = load_peaks()

    def buffers(d, act, seed, n_params=1):
        cd = evo.cdims(d, act)
        tdt = torch.bfloat16 if act == evo.EVO_BF16 else torch.float32
        prob = synth.make_problem(d, seed, pad_frac=0.05)
        n = evo.param_count(cd)
        stride = (n + 127) // 128 * 128  # per-block sets start 256-byte aligned in both copies
        if n_params == 1:
            params = torch.tensor(prob["params"], device=dev)
        else:
            params = torch.zeros(n_params * stride, device=dev)
            for b in range(n_params):
                params[b * stride:b * stride + n] = torch.tensor(synth.make_params(d, seed + 1000 + b), device=dev)
        p16 = None
        if act == evo.EVO_BF16:
            p16 = torch.empty(params.numel(), dtype=torch.bfloat16, device=dev)
            for b in range(n_params):
                evo.params_to_bf16(cd, params[b * stride:b * stride + n], p16[b * stride:b * stride + n])
        return dict(cd=cd, stride=stride, params=params, p16=p16,
                    m=torch.tensor(prob["m"], device=dev).to(tdt), z=torch.tensor(prob["z"], device=dev).to(tdt),
                    mm=torch.tensor(prob["msa_mask"], device=dev), pm=torch.tensor(prob["pair_mask"], device=dev),
                    gm=torch.tensor(prob["gm"], device=dev).to(tdt), gz=torch.tensor(prob["gz"], device=dev).to(tdt))

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        if evo.get_error() != evo.EVO_OK:
            raise RuntimeError("device error word set")
        return a.elapsed_time(b) / steps, clocks.stop()

    torch.cuda.reset_peak_memory_stats()
    w = args.workload
    extra = {}
    if w == "template_pair":
        # template pair stack block fwd+bwd (AF2 Alg. 16) at the template dims,
        # N_res = 256 crop, one template, training-mode dropout
        d = synth.DIMS_TEMPLATE
        cd = evo.cdims(d, evo.EVO_BF16)
        prob = synth.make_problem(d, 32, pad_frac=0.05)
        params = torch.tensor(prob["params"], device=dev)
        p16 = evo.pair_bf16_params(cd, params)
        z = torch.tensor(prob["z"], device=dev).to(torch.bfloat16)
        pm = torch.tensor(prob["pair_mask"], device=dev)
        gz = torch.tensor(prob["gz"], device=dev).to(torch.bfloat16)
        drop = {k: torch.tensor(v, device=dev) for k, v in synth.make_dropout(d, 32).items()}
        zo, dz, dp = torch.empty_like(z), torch.empty_like(z), torch.zeros_like(params)
        wsf, wsb = evo.pair_workspace(cd, evo.EVO_MODE_FWD, dev), evo.pair_workspace(cd, evo.EVO_MODE_BWD, dev)

        def fn():
            evo.pair_block_fwd(cd, params, p16, z, zo, pm, wsf, drop)
            evo.pair_block_bwd(cd, params, p16, z, pm, gz, dz, dp, wsb, drop)

        if not args.no_tune:
            extra["gemm_tiles"] = autotune(evo, fn, TUNE_PASSES)
        ms, clk = timed(fn, args.steps, max(3, args.warmup))
        flops = 3.0 * pair_block_fwd_flops(d)
        desc = "template pair stack block fwd+bwd, N_res=256 c_t=64 (4 heads x 16, c_mul 64), BF16, dropout"
        line = {"workload": w, "metric": desc, "value": flops / (ms / 1e3) / 1e12, "unit": "TFLOP/s",
                "ms_per_step": ms, "steps": args.steps, "flops_per_step": flops,
                "peak_mem_gb": torch.cuda.max_memory_allocated() / 1e9, "clocks": clk, "data": "synthetic"}
        line.update(extra)
        print(json.dumps(line), flush=True)
        return 0
    if w == "adam48":
        # one fused update over 48 blocks x 1,830,016 floats (87.8 M parameters;
        # 1.8 GB of FP32 state, far above L2, so no flush is needed between steps)
        cd = evo.cdims(synth.DIMS_TRAIN_CROP, evo.EVO_BF16)
        stride = (evo.param_count(cd) + 127) // 128 * 128
        n = 48 * stride
        st = {k: torch.tensor(v, device=dev) for k, v in synth.make_adam_state(n, 32).items()}
        pb = torch.empty(n, dtype=torch.bfloat16, device=dev)
        gn = torch.zeros(1, device=dev)
        ws = torch.empty(evo.adam_workspace_size(n), dtype=torch.uint8, device=dev)
        h = evo.adam_hyper(1)

        def fn():
            evo.adam_step(h, st["params"], st["grad"], st["exp_avg"], st["exp_avg_sq"], ws, ema=st["ema"],
                          params_bf16=pb, grad_norm=gn)

        ms, clk = timed(fn, args.steps, max(3, args.warmup))
        algo = 42.0 * n  # norm: g (4 B); update: p, g, m, v, e read, p, m, v, e written, BF16 copy (38 B)
        pk = load_peaks()
        gbs = algo / (ms / 1e3) / 1e9
        line = {"workload": w, "metric": "fused training update over the 48-block flat parameter buffer "
                "(clip by global norm, Adam, EMA, BF16 copy), 87.8 M parameters",
                "value": gbs, "unit": "GB/s", "ms_per_step": ms, "steps": args.steps, "n_params": n,
                "gpu_launches_per_step": 2, "bytes_per_step": algo,
                "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk["hbm"], "unit": "GB/s",
                             "frac": gbs / pk["hbm"], "peak_kind": f"HBM copy, {pk['src']}"},
                "clocks": clk, "data": "synthetic", "l2": "state 1.8 GB > L2, no flush"}
        print(json.dumps(line), flush=True)
        return 0
    if w in ("long4096_slab", "long8192_slab"):
        # inputs drawn on the device (N(0, 1) activations, 5 % padded residues):
        # the host generator would need 8 bytes per element of z
        R = 4096 if w == "long4096_slab" else 8192
        d = synth.Dims(n_seq=128, n_res=R)
        slab = R // 8
        cd = evo.cdims(d, evo.EVO_BF16, pair_slab=slab)
        params = torch.tensor(synth.make_params(d, 32), device=dev)
        p16 = evo.bf16_params(cd, params)
        gen = torch.Generator(device=dev)
        gen.manual_seed(32)

        def normal_bf16(*shape):
            t = torch.empty(*shape, dtype=torch.bfloat16, device=dev)
            for i in range(0, shape[0], 256):
                t[i:i + 256] = torch.randn(t[i:i + 256].shape, generator=gen, device=dev).to(torch.bfloat16)
            return t

        m, z = normal_bf16(d.n_seq, R, d.c_m), normal_bf16(R, R, d.c_z)
        mmask, pmask = synth.make_masks(d, 32, 0.05)
        mm, pm = torch.tensor(mmask, device=dev), torch.tensor(pmask, device=dev)
        mo, zo = torch.empty_like(m), torch.empty_like(z)
        wsf = evo.workspace(cd, evo.EVO_MODE_INFER, dev)
        extra["workspace_gb"] = wsf.numel() / 1e9
        extra["unsliced_workspace_gb"] = evo.workspace_size(evo.cdims(d, evo.EVO_BF16), evo.EVO_MODE_INFER) / 1e9
        extra["plan"] = f"inference workspace plan, pair stack in i-slabs of {slab} rows (evo_block_fwd_infer)"
        extra["device_gb_held"] = torch.cuda.memory_allocated(dev) / 1e9

        def fn():
            evo.block_fwd_infer(cd, params, p16, m, z, mo, zo, mm, pm, wsf)

        if not args.no_tune:
            extra["gemm_tiles"] = autotune(evo, fn, 1)
        ms, clk = timed(fn, args.steps, max(3, args.warmup))
        flops = block_fwd_flops(d)
        desc = f"N_seq={d.n_seq} N_res={R} c_m={d.c_m} fwd BF16, i-slabs of {slab} rows"
    elif w in ("small_fp32_fwd", "long2048", "long4096", "extra_msa"):
        infer = w == "long4096"
        if w == "small_fp32_fwd":
            d, act, bwd = synth.DIMS_SMALL_FP32, evo.EVO_F32, False
        elif w == "long2048":
            d, act, bwd = synth.Dims(n_seq=128, n_res=2048), evo.EVO_BF16, False
        elif w == "long4096":
            d, act, bwd = synth.Dims(n_seq=128, n_res=4096), evo.EVO_BF16, False
        else:
            d, act, bwd = synth.DIMS_EXTRA_MSA, evo.EVO_BF16, True
        B = buffers(d, act, 32)
        cd = B["cd"]
        mo, zo = torch.empty_like(B["m"]), torch.empty_like(B["z"])
        wsf = evo.workspace(cd, evo.EVO_MODE_INFER if infer else evo.EVO_MODE_FWD, dev)
        wsb = evo.workspace(cd, evo.EVO_MODE_BWD, dev) if bwd else None
        dm, dz, dp = torch.empty_like(B["m"]), torch.empty_like(B["z"]), torch.zeros_like(B["params"])
        if infer:
            extra["workspace_gb"] = wsf.numel() * wsf.element_size() / 1e9
            extra["plan"] = "inference workspace plan (evo_block_fwd_infer)"

        def fn():
            if infer:
                evo.block_fwd_infer(cd, B["params"], B["p16"], B["m"], B["z"], mo, zo, B["mm"], B["pm"], wsf)
            else:
                evo.block_fwd(cd, B["params"], B["p16"], B["m"], B["z"], mo, zo, B["mm"], B["pm"], wsf)
            if bwd:
                evo.block_bwd(cd, B["params"], B["p16"], B["m"], B["z"], B["mm"], B["pm"], B["gm"], B["gz"], dm, dz,
                              dp, wsb)

        if act == evo.EVO_BF16 and not args.no_tune:
            extra["gemm_tiles"] = autotune(evo, fn, TUNE_PASSES)
        ms, clk = timed(fn, args.steps, max(3, args.warmup))
        flops = step_flops(d) if bwd else block_fwd_flops(d)
        desc = f"N_seq={d.n_seq} N_res={d.n_res} c_m={d.c_m} {'fwd+bwd' if bwd else 'fwd'} " \
               f"{'BF16' if act else 'FP32 plain'}{' global column attention' if d.msa_col_mode else ''}"
    elif w == "stack48":
        d = synth.Dims(n_seq=512, n_res=384)
        nb = 48
        B = buffers(d, evo.EVO_BF16, 32, n_params=nb)
        cd, stride = B["cd"], B["stride"]
        wsf = evo.workspace(cd, evo.EVO_MODE_FWD, dev)
        wsb = evo.workspace(cd, evo.EVO_MODE_BWD, dev)
        ms_in = [torch.empty_like(B["m"]) for _ in range(nb + 1)]  # block inputs: the only saved activations
        zs_in = [torch.empty_like(B["z"]) for _ in range(nb + 1)]
        dm, dz = B["gm"].clone(), B["gz"].clone()
        dm2, dz2 = torch.empty_like(dm), torch.empty_like(dz)
        dp = torch.zeros_like(B["params"])

        def fn():
            ms_in[0].copy_(B["m"])
            zs_in[0].copy_(B["z"])
            for b in range(nb):
                p = B["params"][b * stride:(b + 1) * stride]
                p16 = B["p16"][b * stride:(b + 1) * stride]
                evo.block_fwd(cd, p, p16, ms_in[b], zs_in[b], ms_in[b + 1], zs_in[b + 1], B["mm"], B["pm"], wsf)
            g_m, g_z, o_m, o_z = B["gm"], B["gz"], dm, dz
            for b in reversed(range(nb)):
                p = B["params"][b * stride:(b + 1) * stride]
                p16 = B["p16"][b * stride:(b + 1) * stride]
                evo.block_bwd(cd, p, p16, ms_in[b], zs_in[b], B["mm"], B["pm"], g_m, g_z, o_m, o_z,
                              dp[b * stride:(b + 1) * stride], wsb)
                g_m, g_z, o_m, o_z = o_m, o_z, (dm2 if o_m is dm else dm), (dz2 if o_z is dz else dz)

        if not args.no_tune:  # one pass launches each GEMM shape at least 48 times
            extra["gemm_tiles"] = autotune(evo, fn, 1)
        ms, clk = timed(fn, args.steps, 1)
        flops = nb * step_flops(d)
        desc = f"48-block stack fwd+bwd, N_seq=512 N_res=384, BF16, per-block recompute"
        extra["saved_block_inputs_gb"] = sum(t.numel() * t.element_size() for t in ms_in + zs_in) / 1e9
    else:  # batch16
        rng = np.random.default_rng(32)
        prot = [(int(rng.integers(32, 513)), int(rng.integers(64, 1025))) for _ in range(16)]
        nb = 48
        flops = 0.0
        jobs = []
        for i, (S, R) in enumerate(prot):
            d = synth.Dims(n_seq=S, n_res=R)
            B = buffers(d, evo.EVO_BF16, 100 + i, n_params=1)
            jobs.append((d, B))
            flops += nb * block_fwd_flops(d)
        # proteins run concurrently on NSTREAMS CUDA streams (largest first onto
        # the least-loaded stream), each stream with its own workspace, so the
        # small proteins fill the SMs the large ones leave idle
        NSTREAMS = max(1, args.streams)
        order = sorted(range(len(jobs)), key=lambda i: -block_fwd_flops(jobs[i][0]))
        load = [0.0] * NSTREAMS
        lanes = [[] for _ in range(NSTREAMS)]
        for i in order:
            k = min(range(NSTREAMS), key=lambda q: load[q])
            lanes[k].append(i)
            load[k] += block_fwd_flops(jobs[i][0])
        streams = [torch.cuda.Stream() for _ in range(NSTREAMS)]
        wss = [torch.empty(max([evo.workspace_size(jobs[i][1]["cd"], evo.EVO_MODE_FWD) for i in lane] or [1]),
                           dtype=torch.uint8, device=dev) for lane in lanes]
        work = {i: (jobs[i][1]["m"].clone(), jobs[i][1]["z"].clone()) for i in range(len(jobs))}

        def run_lanes(base):
            # fork from `base` onto the lanes' streams, join back into `base`
            start = torch.cuda.Event()
            start.record(base)
            for k, lane in enumerate(lanes):
                st = streams[k]
                st.wait_event(start)
                with torch.cuda.stream(st):
                    for i in lane:
                        d, B = jobs[i]
                        m, z = work[i]
                        m.copy_(B["m"])
                        z.copy_(B["z"])
                        for _ in range(nb):
                            evo.block_fwd(B["cd"], B["params"], B["p16"], m, z, m, z, B["mm"], B["pm"], wss[k],
                                          stream=st)
            for st in streams:
                done = torch.cuda.Event()
                done.record(st)
                base.wait_event(done)

        def fn():
            run_lanes(torch.cuda.current_stream())

        def tune_once():  # each protein's shapes, one protein at a time on one stream
            wst = torch.empty(max(evo.workspace_size(B["cd"], evo.EVO_MODE_FWD) for _, B in jobs),
                              dtype=torch.uint8, device=dev)
            for d, B in jobs:
                m, z = B["m"].clone(), B["z"].clone()
                for _ in range(TUNE_PASSES):
                    evo.block_fwd(B["cd"], B["params"], B["p16"], m, z, m, z, B["mm"], B["pm"], wst)

        if not args.no_tune:
            tuned = autotune(evo, tune_once, 1)
            extra["gemm_tiles"] = {"shapes": tuned["shapes"], "changed": tuned["changed"]}

        def as_graph(body):
            # the whole batch (all proteins, all blocks, every stream) as one CUDA graph
            body()  # first run outside capture: lazy kernel set-up
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            cap = torch.cuda.Stream()
            cap.wait_stream(torch.cuda.current_stream())
            with torch.cuda.graph(g, stream=cap):
                body()
            torch.cuda.current_stream().wait_stream(cap)
            torch.cuda.synchronize()
            return g.replay

        ms, clk = timed(as_graph(fn) if args.graph else fn, args.steps, 1)
        desc = (f"16 proteins (seeded N_res~U[64,1024], N_seq~U[32,512]), 48-block forward each, BF16, "
                f"{NSTREAMS} concurrent CUDA streams{', one CUDA graph replay per step' if args.graph else ''}")
        extra["proteins"] = prot
        extra["streams"] = NSTREAMS
        extra["cuda_graph"] = bool(args.graph)

        # the same batch through the batched C ABI: one evo_stack_fwd over the
        # padded [16, Smax, Rmax, c] buffers, proteins one after another on one
        # stream, each staged at its own sizes (no work on the padding)
        for i in range(len(jobs)):
            work[i] = None
        del wss
        Smax, Rmax = max(S for S, _ in prot), max(R for _, R in prot)
        dpad = synth.Dims(n_seq=Smax, n_res=Rmax)
        cdp = evo.cdims(dpad, evo.EVO_BF16)
        npar = evo.param_count(cdp)
        pstride = (npar + 127) // 128 * 128
        p32 = torch.zeros(nb * pstride, device=dev)
        p32[:npar] = jobs[0][1]["params"][:npar]
        p16b = torch.zeros(nb * pstride, dtype=torch.bfloat16, device=dev)
        p16b[:npar] = jobs[0][1]["p16"][:npar]
        for k in range(1, nb):  # the first protein's block, repeated (the shapes are what is timed)
            p32[k * pstride:k * pstride + npar] = p32[:npar]
            p16b[k * pstride:k * pstride + npar] = p16b[:npar]
        Bn = len(jobs)
        m0 = torch.zeros(Bn, Smax, Rmax, dpad.c_m, dtype=torch.bfloat16, device=dev)
        z0 = torch.zeros(Bn, Rmax, Rmax, dpad.c_z, dtype=torch.bfloat16, device=dev)
        mm0 = torch.zeros(Bn, Smax, Rmax, device=dev)
        pm0 = torch.zeros(Bn, Rmax, Rmax, device=dev)
        for i, (S, R) in enumerate(prot):
            B = jobs[i][1]
            m0[i, :S, :R], z0[i, :R, :R] = B["m"], B["z"]
            mm0[i, :S, :R], pm0[i, :R, :R] = B["mm"], B["pm"]
        mB, zB = m0.clone(), z0.clone()
        wsB = evo.workspace(cdp, evo.EVO_MODE_FWD, dev, batch=Bn)

        def fnb():
            mB.copy_(m0)
            zB.copy_(z0)
            evo.stack_fwd(cdp, nb, p32, p16b, pstride, mB, zB, mm0, pm0, wsB,
                          n_seq_b=[S for S, _ in prot], n_res_b=[R for _, R in prot])

        msb, _ = timed(as_graph(fnb) if args.graph else fnb, args.steps, 1)
        extra["batched_abi"] = {"ms_per_step": msb, "tflops": flops / (msb / 1e3) / 1e12,
                                "how": "one evo_stack_fwd over the padded batch, one stream" +
                                       (", one CUDA graph replay per step" if args.graph else "")}
    line = {"workload": w, "metric": desc, "value": flops / (ms / 1e3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
            "steps": args.steps, "flops_per_step": flops, "frac_of_bf16_peak": flops / (ms / 1e3) / 1e12 / peaks["bf16_sus"],
            "peak_mem_gb": torch.cuda.max_memory_allocated() / 1e9, "clocks": clk, "data": "synthetic"}
    line.update(extra)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--n-seq", type=int, default=128)
    ap.add_argument("--n-res", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the built-in GEMM tile choice")
    ap.add_argument("--dropout", action="store_true", help="training-mode dropout (AF2 sites and rates)")
    ap.add_argument("--streams", type=int, default=8, help="concurrent CUDA streams of the 16-protein batch")
    ap.add_argument("--graph", action="store_true",
                    help="replay the step as one captured CUDA graph (the default; kept for older command lines)")
    ap.add_argument("--eager", action="store_true", help="time eager launches instead of a CUDA graph replay")
    ap.add_argument("--workload", default="train_crop",
                    choices=["train_crop", "small_fp32_fwd", "extra_msa", "stack48", "long2048", "batch16",
                             "template_pair", "adam48", "long4096", "long4096_slab", "long8192_slab"])
    args = ap.parse_args()
    args.graph = not args.eager
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload != "train_crop":
        return other_workload(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
