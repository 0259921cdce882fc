#!/usr/bin/env python
"""Benchmark of the SCALE local-energy hot path on GB300.

One step = one chain step over B resident walkers of the 16x16 Hubbard workload
(U = 8, 112+112 electrons, 6 layers of 32 channels, mixed precision):
  * low-rank local energies of every walker (device-side enumeration of the connected
    configurations, incremental receptive-field update, rank-r determinants);
  * one Woodbury commit per walker (a proposed nearest-neighbour hop, drawn on the host
    beforehand with a seeded generator and uploaded once);
  * the FP64 re-factorisation of the walkers whose commit counter reaches 64 (counters are
    staggered, so 1/64 of the batch per step).
value = local energies per second (walkers x steps / device time), max over ranks.

Also reported (rank 0): the cold path (load = forward + FP64 inverse + projector, then
E_loc), the full-recompute path on a subset of the same walkers (same GPU, same precision
mode), per-sample gradients, the roofline of the dominant kernel, GPU clocks during the
timed region, and the FP64 CPU oracle timed on the host cores on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl scale|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_25775_gb300 import inputs as I  # noqa: E402

FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz
FP64_PEAK_TFLOPS = 1.196  # DFMA loop measured on this machine's GB300 (profiles/peaks_fp32_fp64.txt)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", default="scale", choices=["scale", "reference"])
    ap.add_argument("--workload", default="hubbard16x16")
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--full-samples", type=int, default=128)
    ap.add_argument("--cpu-samples", type=int, default=48)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--precision", default=None, choices=list(PRECISIONS),
                    help="site-wise layers as three TF32 (mixed), FP16 (mixed_fp16) or BF16 (mixed_bf16) "
                         "tensor-core products; default: the workload's mode (hubbard16x16: mixed_fp16)")
    ap.add_argument("--lowrank-kernel", default="warp", choices=["warp", "batched"],
                    help="low-rank local-energy kernel of the timed chain step")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--sweep-steps", type=int, default=64)
    ap.add_argument("--sym-walkers", type=int, default=1024)
    ap.add_argument("--ace-walkers", type=int, default=16)
    ap.add_argument("--wide-walkers", type=int, default=8)
    return ap.parse_args()


# DRAM traffic of the local-energy kernel per walker, from the ncu capture summarised in
# this file; used only while the kernel sources still hash to the value recorded there.
ELOC_PROFILE = os.path.join(ROOT, "profiles", "k_eloc_hubbard16x16.md")
ELOC_SOURCES = ["lowrank.cu", "eloc_common.cuh", "move.cuh", "mlp_mma.cuh", "scale_internal.cuh"]


# The shared header contributes only its device part (geometry, parameter view, activation
# functions); the context struct and launch declarations below the marker do not reach the
# kernel's code.
HEADER_DEVICE_END = b"\n// The context (opaque to callers)."


def eloc_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in ELOC_SOURCES:
        with open(os.path.join(ROOT, "paper_2604_25775_gb300", "csrc", name), "rb") as f:
            data = f.read()
        if name == "scale_internal.cuh":
            data = data.split(HEADER_DEVICE_END, 1)[0]
        h.update(data)
    return h.hexdigest()


def profiled_traffic_per_walker():
    """(bytes per walker, note) from the profile summary, or (None, reason)."""
    try:
        fields = {}
        with open(ELOC_PROFILE) as f:
            for line in f:
                if ":" in line and line.split(":", 1)[0].strip() in ("dram_bytes_per_walker", "sources_sha256"):
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip().strip("`")
        if fields.get("sources_sha256") != eloc_sources_sha256():
            return None, "kernel sources changed since the capture"
        return float(fields["dram_bytes_per_walker"]), "ncu capture at 512 walkers, scaled per walker"
    except (OSError, KeyError, ValueError):
        return None, "no capture summary"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# The headline metric: the low-rank local-energy rate is the value; the full-recompute rate on
# the same GPU and the serving latencies are reported beside it.
METRIC = "local energies/s, low-rank vs full-det at 16×16 same GPU; p50/p99 serve latency"


def workload_config(pb, name: str, walkers: int, world: int) -> dict:
    """The workload both arms run, named by its sizes (the reference arm times a bounded
    sample of its walkers)."""
    bc = {(1, 1): "torus", (1, 0): "cylinder", (0, 1): "cylinder", (0, 0): "open"}[(pb.pbc_x, pb.pbc_y)]
    n_conv = sum(1 for k in pb.ksize if k > 1)
    k0 = pb.ksize[0]
    binv_gb = walkers * (pb.n_up + pb.n_dn) ** 2 * 4 / 1e9
    return {"workload": f"{name}: {pb.Lx}x{pb.Ly} {bc}, U={pb.U:g}, {pb.n_up}+{pb.n_dn}, SCALE {n_conv} conv "
                        f"{k0}x{k0} + {pb.n_layers - n_conv} site-wise, h={pb.h}",
            "walkers": walkers, "refresh_every": pb.refresh_every,
            "l2": f"inputs larger than L2 (cached inverses {binv_gb:.1f} GB)", "parallelism": f"replicas x{world}"}


def replica_plan(rank: int, world: int, walkers: int) -> dict:
    """Replicas only: every rank runs the whole step on its own walkers (weak scaling)."""
    pseed, cseed = I.workload_seeds("hubbard16x16")
    return {"walkers": walkers, "param_seed": pseed, "config_seed": cseed + 1000 * rank,
            "move_seed": 777 + 1000 * rank, "world": world}


def max_over_ranks(t_ms: float, dist=None, device="cuda") -> float:
    """Slowest rank's time (the job's time)."""
    if dist is None:
        return t_ms
    import torch
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(walkers: int, steps: int, world: int, t_max_ms: float) -> float:
    """Whole-job local energies per second over all ranks."""
    return world * walkers * steps / (t_max_ms / 1e3)


def move_schedule(pb, occ, n_steps, seed):
    """Valid nearest-neighbour hop proposals for n_steps consecutive commits (host, seeded)."""
    cur = occ
    out = []
    for k in range(n_steps):
        mv = I.random_hop_moves(pb, cur, seed + k)
        out.append(mv)
        cur = I.apply_moves(cur, mv)
    return np.stack(out)


def lowrank_flops_per_sample(pb, occ, n=32):
    """Algorithmic FLOPs of one low-rank E_loc per walker, counted from the configurations:
    per connected move, |S| sites x (L-1) site-wise layers x 2h^2, the moved electron's
    features against the projector (2 r h; its (M0 + proj_b) . Phi^-1 part is read from the
    cache that every commit keeps current), the Delta H . P block (2 r^2 h) and the r x r LU
    (2/3 r^3); r = electrons on the affected sites after the move, S = union of the 3x3
    stencils."""
    N, h, L = pb.N, pb.h, pb.n_layers
    r0 = (pb.ksize[0] - 1) // 2
    tot = 0.0
    for b in range(min(n, occ.shape[0])):
        x = occ[b].astype(np.int64)
        for i in range(N):
            for (dx, dy) in ((1, 0), (0, 1)):
                xx, yy = (i % pb.Lx + dx) % pb.Lx, (i // pb.Lx + dy) % pb.Ly
                j = yy * pb.Lx + xx
                for s in (0, 1):
                    a, c = (x[i] >> s) & 1, (x[j] >> s) & 1
                    if a == c:
                        continue
                    src, dst = (i, j) if a else (j, i)
                    S = set()
                    for t in (src, dst):
                        for ey in range(-r0, r0 + 1):
                            for ex in range(-r0, r0 + 1):
                                S.add(((t // pb.Lx + ey) % pb.Ly) * pb.Lx + (t % pb.Lx + ex) % pb.Lx)
                    y = x.copy()
                    y[src] &= ~(1 << s)
                    y[dst] |= 1 << s
                    r = int(sum(((y[q] & 1) + ((y[q] >> 1) & 1)) for q in S))
                    tot += len(S) * (L - 1) * 2 * h * h + 2 * r * h + 2 * r * r * h + 2 * r ** 3 / 3
    return tot / min(n, occ.shape[0])


# --precision: the mode of the site-wise tensor-core layers (everything else as in mixed mode)
PRECISIONS = {"mixed": I.PREC_MIXED, "mixed_fp16": I.PREC_MIXED_FP16, "mixed_bf16": I.PREC_MIXED_BF16}
DTYPES = {I.PREC_MIXED: "f32 (rank-r, network; site-wise layers as 3 tf32 tensor-core products) + f64 (LU refresh, accumulation)",
          I.PREC_MIXED_FP16: "f32 (rank-r, network; site-wise layers as 3 f16 tensor-core products) + f64 (LU refresh, accumulation)",
          I.PREC_MIXED_BF16: "f32 (rank-r, network; site-wise layers as 3 bf16 tensor-core products) + f64 (LU refresh, accumulation)"}


def run_reference(args, world, rank):
    """The oracle (FP64 CPU, full recompute), as it stands, on the host cores: each step a
    bounded sample of walkers of the same workload."""
    if rank != 0:
        return
    from oracle import oracle as O
    pb = I.workload(args.workload)
    pseed, cseed = I.workload_seeds(args.workload)
    params = I.random_params(pb, pseed)
    M0 = I.plane_wave_M0(pb)
    m = O.Model(pb, params, M0)
    per_step = max(1, O.num_threads() // 2)
    occ = I.random_configs(pb, per_step * (args.steps + args.warmup), cseed)
    for k in range(args.warmup):
        m.local_energy(occ[k * per_step:(k + 1) * per_step])
    t0 = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        m.local_energy(occ[k * per_step:(k + 1) * per_step])
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "E_loc/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(pb, args.workload, args.batch, world),
            "step": f"E_loc of {per_step} of the workload's walkers by full recompute (FP64 CPU oracle)",
            "cpu_baseline": {"value": value, "unit": "E_loc/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{per_step} walkers per step x {args.steps} steps"},
            "e2e": {"value": value, "unit": "E_loc/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, world, rank)
        return
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2604_25775_gb300 import binding as Bd
    Bd.load_library(build=True)

    pb = I.workload(args.workload)
    if args.precision:
        pb = pb.replace(precision=PRECISIONS[args.precision])
    if args.lowrank_kernel == "batched":
        pb = pb.replace(lowrank_kernel=I.LOWRANK_BATCHED)
    B, K, W = args.batch, args.steps, args.warmup
    plan = replica_plan(rank, world, B)
    params = I.random_params(pb, plan["param_seed"])
    M0 = I.plane_wave_M0(pb)
    occ = I.random_configs(pb, B, plan["config_seed"])
    stream = torch.cuda.Stream()
    ctx = Bd.make_context(pb, params, M0, B, stream=stream)
    moves = move_schedule(pb, occ, K + W, plan["move_seed"])
    moves_d = torch.from_numpy(moves).cuda()
    occ_d = torch.from_numpy(occ).cuda()
    eloc = torch.empty(B, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        ctx.scale_load(occ_d)
    stream.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up
    for k in range(W):
        ctx.scale_local_energy(eloc)
        ctx.scale_commit(moves_d[k])
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(K):
            ev[k][0].record(stream)
            ctx.scale_local_energy(eloc)
            ev[k][1].record(stream)
            ctx.scale_commit(moves_d[W + k])
            ev[k][2].record(stream)
        t_end.record(stream)
        barrier()
    total_ms = t_start.elapsed_time(t_end)
    eloc_ms = float(np.mean([a.elapsed_time(b) for a, b, c in ev]))
    commit_ms = float(np.mean([b.elapsed_time(c) for a, b, c in ev]))
    t_max = max_over_ranks(total_ms, dist)
    value = aggregate_rate(B, K, world, t_max)
    assert torch.isfinite(eloc).float().mean().item() > 0.99

    # end-to-end through the public API: proposals from pinned host memory, E_loc back
    E2E_STEPS = min(K, 10)
    mv_host = torch.from_numpy(move_schedule(pb, ctx.get_occ().cpu().numpy(), E2E_STEPS, 999 + rank)).pin_memory()
    e_host = torch.empty((E2E_STEPS, B), dtype=torch.float64).pin_memory()
    mv_dev = torch.empty((B, 4), dtype=torch.int32, device="cuda")
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    with torch.cuda.stream(stream):
        for k in range(E2E_STEPS):
            mv_dev.copy_(mv_host[k], non_blocking=True)
            ctx.scale_local_energy(eloc)
            ctx.scale_commit(mv_dev)
            e_host[k].copy_(eloc, non_blocking=True)
    t1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(t0.elapsed_time(t1), dist)
    e2e_val = aggregate_rate(B, E2E_STEPS, world, e2e_ms)

    line = {
        "metric": METRIC,
        "value": value, "unit": "E_loc/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES.get(pb.precision, "f64"), "data": "synthetic",
        "config": workload_config(pb, args.workload, B, world),
        "step": "E_loc (low-rank) + 1 Woodbury commit per walker + staggered FP64 refresh",
        "precision": {v: k for k, v in PRECISIONS.items()}.get(pb.precision, "fp64"),
        "e2e": {"value": e2e_val, "unit": "E_loc/s", "h2d_bytes_per_step": B * 4 * 4,
                "d2h_bytes_per_step": B * 8},
        "stage_ms": {"eloc_lowrank": eloc_ms, "commit_and_refresh": commit_ms},
        "clocks": clk.summary(),
    }
    stats = ctx.scale_get_stats()
    line["stats"] = {k: stats[k] for k in ("n_commits", "n_refresh", "n_drift_refresh", "drift_max")}

    if rank == 0 and not args.no_extras:
        flops = lowrank_flops_per_sample(pb, occ)
        achieved = flops * B / (eloc_ms / 1e3) / 1e12
        tpw, tnote = profiled_traffic_per_walker()
        line["roofline"] = {"kernel": "k_eloc (low-rank E_loc)", "bound": "alu", "achieved": achieved,
                            "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                            "traffic": None if tpw is None else tpw * B, "traffic_note": tnote,
                            "flops_per_walker": flops,
                            "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 x 2.07 GHz (derived)"}
        # cold path: load (forward, FP64 Gauss-Jordan inverse, projector) + E_loc
        ctx2 = Bd.make_context(pb, params, M0, B)
        ctx2.scale_load(occ_d)
        ctx2.scale_local_energy(eloc)
        torch.cuda.synchronize()
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ctx2.scale_load(occ_d)
        mid = torch.cuda.Event(enable_timing=True)
        mid.record()
        ctx2.scale_local_energy(eloc)
        b2.record()
        torch.cuda.synchronize()
        load_ms, cold_eloc_ms = a.elapsed_time(mid), mid.elapsed_time(b2)
        line["cold"] = {"load_ms": load_ms, "eloc_ms": cold_eloc_ms,
                        "eloc_per_s": B / ((load_ms + cold_eloc_ms) / 1e3)}
        ctx2.close()
        # the same local energies with the batched tensor-core kernel (site-wise layers of all
        # moves on tcgen05; arch.lowrank_kernel = SCALE_LOWRANK_BATCHED), which runs the TF32x3
        # products of SCALE_PREC_MIXED, beside the per-warp kernel in that mode
        pb_t = pb.replace(precision=I.PREC_MIXED)
        alt_ms = {}
        for key, pbx in (("batched", pb_t.replace(lowrank_kernel=I.LOWRANK_BATCHED)), ("warp_tf32x3", pb_t)):
            ctxb = Bd.make_context(pbx, params, M0, B)
            ctxb.scale_load(occ_d)
            eb = torch.empty(B, dtype=torch.float64, device="cuda")
            ctxb.scale_local_energy(eb)
            torch.cuda.synchronize()
            a.record()
            ctxb.scale_local_energy(eb)
            b2.record()
            torch.cuda.synchronize()
            alt_ms[key] = a.elapsed_time(b2)
            ctxb.close()
        bt_ms = alt_ms["batched"]
        line["lowrank_batched_kernel"] = {"eloc_ms": bt_ms, "eloc_per_s": B / (bt_ms / 1e3),
                                          "warp_kernel_tf32x3_eloc_ms": alt_ms["warp_tf32x3"],
                                          "warp_kernel_eloc_ms": eloc_ms,
                                          "note": "same walkers as the cold load; the batched kernel runs the TF32x3 "
                                                  "products (SCALE_PREC_MIXED), compare it with the per-warp kernel in "
                                                  "that mode; the default is the per-warp kernel with the workload's "
                                                  "products"}
        # Metropolis sweep on the same walkers: hop proposal, rank-r ratio, accept, Woodbury
        # commit of the accepted moves (random numbers generated on the host beforehand). The
        # first --sweep-steps are timed; the sweep then continues untimed to 2.5 N steps per
        # walker, so that the walkers are drawn from |psi|^2 for the comparison below.
        steps_per_sample = int(2.5 * pb.N)
        occ_cmp, cmp_from = occ_d, "uniformly random walkers of the workload"
        if args.sweep_steps > 0:
            S = args.sweep_steps
            ctxs = Bd.make_context(pb, params, M0, B)
            ctxs.scale_load(occ_d)
            pk, dr, uu = I.metropolis_randoms(pb, B, 4 + max(S, steps_per_sample), 77)
            pk_d, dr_d, uu_d = (torch.from_numpy(x).cuda() for x in (pk, dr, uu))
            ctxs.sweep(pk_d[:4].contiguous(), dr_d[:4].contiguous(), uu_d[:4].contiguous())
            pk_t, dr_t, uu_t = pk_d[4:4 + S].contiguous(), dr_d[4:4 + S].contiguous(), uu_d[4:4 + S].contiguous()
            torch.cuda.synchronize()
            a.record()
            acc_s = ctxs.sweep(pk_t, dr_t, uu_t)
            b2.record()
            torch.cuda.synchronize()
            sw_ms = a.elapsed_time(b2)
            line["sweep"] = {"walkers": B, "steps": S, "ms": sw_ms,
                             "walker_steps_per_s": B * S / (sw_ms / 1e3),
                             "acceptance": float(acc_s.double().mean().item() / S),
                             "ms_per_sweep_2.5N": sw_ms / S * steps_per_sample,
                             "steps_per_sweep": steps_per_sample}
            if steps_per_sample > S:
                ctxs.sweep(pk_d[4 + S:4 + steps_per_sample].contiguous(), dr_d[4 + S:4 + steps_per_sample].contiguous(),
                           uu_d[4 + S:4 + steps_per_sample].contiguous())
            occ_cmp = ctxs.get_occ()
            cmp_from = f"walkers after {max(S, steps_per_sample)} Metropolis steps each (|psi|^2-distributed)"
            torch.cuda.synchronize()
            del pk_d, dr_d, uu_d, pk_t, dr_t, uu_t
            ctxs.close()
        # full-recompute path (psi(n) and every psi(n') by a fresh forward and FP64 LU) against
        # the low-rank path on the same walkers, same GPU and precision mode
        nf = args.full_samples
        ctxf = Bd.make_context(pb, params, M0, nf)
        ctxf.scale_load(occ_cmp[:nf].contiguous())
        ef = torch.empty(nf, dtype=torch.float64, device="cuda")
        el = torch.empty(nf, dtype=torch.float64, device="cuda")
        ctxf.scale_local_energy(ef, Bd.PATH_FULL)
        torch.cuda.synchronize()
        a.record()
        ctxf.scale_local_energy(ef, Bd.PATH_FULL)
        b2.record()
        torch.cuda.synchronize()
        full_ms = a.elapsed_time(b2)
        ctxf.scale_local_energy(el, Bd.PATH_LOWRANK)
        torch.cuda.synchronize()
        diff = ((ef - el).abs() / ef.abs().clamp(min=1.0)).cpu().numpy()
        full_rate = nf / (full_ms / 1e3)
        lowrank_rate = B / (eloc_ms / 1e3)
        line["full_recompute"] = {"walkers": nf, "walkers_from": cmp_from, "ms": full_ms, "eloc_per_s": full_rate,
                                  "chunk": int(ctxf.scale_get_stats()["full_chunk"]),
                                  "determinants": "FP64 LU of the mode-precision Slater matrices",
                                  "lowrank_eloc_per_s": lowrank_rate, "speedup_lowrank_vs_full": lowrank_rate / full_rate,
                                  "max_rel_diff_vs_lowrank": float(diff.max()),
                                  "median_rel_diff_vs_lowrank": float(np.median(diff)),
                                  "frac_within_1e-4": float(np.mean(diff <= 1e-4))}
        ctxf.close()
        # per-sample gradients on a subset
        ng = 1024
        ctxg = Bd.make_context(pb, params, M0, ng)
        ctxg.scale_load(occ_d[:ng].contiguous())
        g = torch.empty((ng, ctxg.P), dtype=torch.float64, device="cuda")
        ctxg.scale_grad_logpsi(g)
        torch.cuda.synchronize()
        a.record()
        ctxg.scale_grad_logpsi(g)
        b2.record()
        torch.cuda.synchronize()
        line["grad"] = {"walkers": ng, "ms": a.elapsed_time(b2), "params": ctxg.P}
        del g
        ctxg.close()
        # per-sample gradients at the gradient workload: 16x4 cylinder, 12 residual 3x3 layers
        from paper_2604_25775_gb300 import next_bench as NB
        line["grad_cylinder16x4"] = NB.run_grad(2048)
        # symmetry projection over the lattice translations: |G| fresh amplitudes per walker;
        # ACE (no cached update: every psi(n') of a local energy is a fresh forward + LU)
        from paper_2604_25775_gb300 import next_bench
        if args.sym_walkers > 0:
            line["symmetry"] = next_bench.run_symmetry(args.sym_walkers)
        if args.ace_walkers > 0:
            line["ace"] = next_bench.run_ace(args.ace_walkers)
        if args.wide_walkers > 0:  # Table tab:model SCALE-L / SCALE-XL shapes: full recompute and cached update
            line["wide"] = next_bench.run_wide(args.wide_walkers)
        # the cached update with SCALE-L's plus stencil (bench network otherwise)
        line["plus_stencil"] = next_bench.run_plus(B)
        # serving: open-loop Poisson local-energy requests over mixed chains (8x8, 16x16, 32x32,
        # Hubbard and t-J, 64..4096 walkers), continuous batching, at 0.3 / 0.6 / 0.9 of the
        # measured capacity
        if args.serve_requests > 0:
            from paper_2604_25775_gb300 import serve_bench
            line["serve"] = serve_bench.run(requests_per_load=args.serve_requests)
        # CPU oracle baseline on a bounded sample
        from oracle import oracle as O
        m = O.Model(pb, params, M0)
        n_cpu = args.cpu_samples
        t0c = time.perf_counter()
        m.local_energy(occ[:n_cpu])
        dt = time.perf_counter() - t0c
        line["cpu_baseline"] = {"value": n_cpu / dt, "unit": "E_loc/s", "cores": O.num_threads(), "kind": "oracle",
                                "sample": f"{n_cpu} walkers of the same workload, FP64 full recompute"}
    # per step, as an ncu launch list of the chain step shows: k_eloc, k_commit, k_mark_refresh,
    # and the refresh of the due samples: k_slots, k_layer, k_mlp_fwd, k_phi, k_gj, k_project
    line["gpu_launches"] = K * 9
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
