#!/usr/bin/env python
"""Throughput benchmark of the GPU partitioned-network-expansion path.

Default workload: 2D random-tensor networks, 16x16 open lattice, bond
dimension D=4, entries U[0,1)+0.1 (SplitMix64 seeds), expansion order K=8 in
LOOP mode; one step = one full pass (BP partition, gauge, cluster and term
enumeration, cluster contractions, FP64 term sums) over a batch of 32
networks.  Metric: PNE terms contracted per second (whole job, all ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pne|reference]
                  [--dtype f64|f32|tf32|bf16] [--workload random16|ising4|ising3d]

Under torchrun each rank works on its own 32 networks (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2512_10910_gb300 import inputs as I  # noqa: E402

BP_ARITH = {"fp64": 0, "ff": 1}

WORKLOADS = {
    "random16": dict(desc="2D random-tensor network 16x16 open, D=4, U[0,1)+0.1, K=8 LOOP, 32 networks per step",
                     kind="random2d", L=16, D=4, K=8, batch=32, mode=0),
    "ising4": dict(desc="2D Ising 4x4 open, D=2, beta=0.40, full order K=24 LOOP, 32 copies per step",
                   kind="ising2d", L=4, D=2, K=24, batch=32, mode=0, beta=0.40),
    "ising3d": dict(desc="3D Ising 8x8x8 open, D=2, beta in {0.20,0.2217,0.25}, K=8 LOOP",
                    kind="ising3d", L=8, D=2, K=8, batch=3, mode=0),
    "batched": dict(desc="4096 independent 2D networks LxL, L~U{6..24}, D~U{2..6}, half random U[0,1)+0.1, "
                         "half Ising beta~U[0.3,0.5] (D=2), seed 1234, K=8 LOOP, one persistent fused launch "
                         "replayed from a CUDA graph", kind="batched", n=4096, K=8, mode=0),
    "serve": dict(desc="served: Poisson arrivals mean 2000 req/s, seed 7; 1/2 AKLT norm networks LxL, L~U{8..32} "
                       "(D=4), 1/2 3D random networks L^3, L~U{6..12}, D~U{2..4}, N(1,0.3^2); K~U{4..8}; "
                       "continuous batching with memory admission", kind="serve", rate=2000.0, mode=0),
}


def make_networks(wl, rank):
    if wl["kind"] == "random2d":
        g = I.square_lattice(wl["L"], wl["L"], wl["D"])
        seeds = range(rank * wl["batch"], (rank + 1) * wl["batch"])
        return g, [I.random_tensors(g, s) for s in seeds]
    if wl["kind"] == "ising2d":
        g = I.square_lattice(wl["L"], wl["L"], 2)
        return g, [I.ising_tensors(g, wl["beta"]) for _ in range(wl["batch"])]
    if wl["kind"] == "ising3d":
        g = I.cubic_lattice(wl["L"], wl["L"], wl["L"], 2)
        return g, [I.ising_tensors(g, b) for b in (0.20, 0.2217, 0.25)]
    raise ValueError(wl["kind"])


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle baseline
def oracle_step(wl, net):
    """The oracle as it stands on one network of the workload; returns
    (n_terms, seconds, result)."""
    from oracle import enumerate as E
    from oracle import expansion as X
    t0 = time.perf_counter()
    r = X.pne(net, wl["K"], E.LOOP if wl["mode"] == 0 else E.ALL)
    return r.n_terms, time.perf_counter() - t0, r


def hbm_peak():
    """Measured copy bandwidth of the GB300s (GB/s), else the fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (of fallback)"


def algorithmic_bp_flops(g, iters):
    """FP64 flops of one BP sweep-set: per site and sweep, the two half
    contractions touch every tensor entry once with one multiply-add each
    (4 flops per entry); times the sweeps each tensor set took."""
    per_sweep = 0
    for v in range(g.n_sites):
        per_sweep += 4 * int(np.prod(g.leg_dims(v)))
    return per_sweep * float(sum(iters))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="pne", choices=["pne", "reference"])
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "tf32", "bf16"])
    ap.add_argument("--workload", default="random16", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--bp", default="ff", choices=["fp64", "ff"],
                    help="BP sweep arithmetic: FP64, or float-float pairs on the FP32 pipes")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, wl, rank, world)
    if wl["kind"] == "batched":
        return run_batched(args, wl, rank, world, local_rank)
    if wl["kind"] == "serve":
        return run_serve(args, wl, rank, world, local_rank)

    import torch
    import torch.distributed as dist
    from paper_2512_10910_gb300 import pne

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    sh = ctypes_stream = stream.cuda_stream

    g, nets = make_networks(wl, rank)
    B = len(nets)
    flat = np.concatenate([n.flat_data()[0] for n in nets])
    data_dev = torch.from_numpy(flat).to(dev)
    data_host = torch.from_numpy(flat).pin_memory()
    ctx = pne.Context(local_rank)
    K, mode = wl["K"], wl["mode"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > 129 MB L2

    enum_cache = [0]      # the headline recomputes the enumeration every step
    # the enumeration is geometry-only: it runs on a second stream while BP runs
    # on the first (the partition is built without waiting for its convergence
    # record, which pne_sum reads); the contraction waits for both
    # the enumeration is the longer chain: its stream gets the higher priority,
    # so its small level launches are scheduled ahead of BP's blocks
    side = torch.cuda.Stream(dev, priority=-1)
    side_h = side.cuda_stream
    joined = torch.cuda.Event()

    # the network description (geometry arrays, tensor pointer) is marshalled
    # once per input buffer, as a caller stepping one geometry would; the
    # library still reads and checks it on every call
    structs = {}
    popts = pne.PartitionOpts(1e-13, 10000, 0.0, BP_ARITH[args.bp], 1)

    def step(data, dtype):
        if id(data) not in structs:
            structs[id(data)] = pne.network_struct(g, data=data, n_batch=B)
        ns, keep = structs[id(data)]
        part, _ = pne.pne_build_partition(ctx.h, ns, popts, ctypes_stream)
        try:
            terms, nc, nt = pne.pne_enumerate_terms(ctx.h, part, pne.EnumOpts(K, mode, enum_cache[0]), side_h)
            try:
                joined.record(side)
                stream.wait_event(joined)
                pne.pne_contract_terms(ctx.h, terms, dtype, ctypes_stream)
                res = pne.pne_sum(ctx.h, terms, ctypes_stream)
            finally:
                pne.pne_terms_destroy(terms)
        finally:
            pne.pne_partition_destroy(part)
        return res

    def timed(data, dtype, steps, warmup, profile=False):
        for _ in range(warmup):
            step(data, dtype)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        if profile:
            pne.pne_ctx_profile(ctx.h, True)
        total = 0.0
        res = None
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            res = step(data, dtype)
            b.record(stream)
            b.synchronize()
            total += a.elapsed_time(b)
        torch.cuda.synchronize(dev)
        prof = pne.pne_ctx_profile_read(ctx.h) if profile else None
        if profile:
            pne.pne_ctx_profile(ctx.h, False)
        if world > 1:
            t = torch.tensor([total], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total = float(t.item())
        return total, res, prof

    dtype = pne.DTYPES[args.dtype]
    clocks = ClockSampler(local_rank)
    clocks.start()
    total_ms, res, _ = timed(data_dev, dtype, args.steps, args.warmup)
    clk = clocks.stop()
    # per-kernel event timings come from a separate pass, so that the timed
    # steps carry no profiling events
    prof_steps = max(5, args.steps // 4)
    _, _, prof_all = timed(data_dev, dtype, prof_steps, 1, profile=True)
    prof = {k: v for k, v in prof_all.items() if not k.startswith("host:")}
    host_ms = {k[5:]: round(v[1] / prof_steps, 4) for k, v in prof_all.items() if k.startswith("host:")}
    n_terms = res[0]["n_terms"]
    terms_per_step = n_terms * B
    ms_per_step = total_ms / args.steps
    value = terms_per_step * world / (ms_per_step * 1e-3)

    # end to end: host (pinned) input copied inside the call, results read back
    e2e_ms, _, _ = timed(data_host, dtype, max(5, args.steps // 5), 2)
    e2e_ms /= max(5, args.steps // 5)
    geom_bytes = 2 * ((g.n_sites + 1) * 8 + (3 * g.n_bonds + g.n_sites + 1 + len(g.site_bonds) + 2 * g.n_bonds
                                              + len(g.site_bonds) + 64 * g.n_sites) * 4)
    h2d = int(flat.nbytes + geom_bytes)
    d2h = int(B * (K + 1) * 2 * 8 + B * 3 * 8 + B * 12 + 64)

    # variants in the other precisions (fewer steps)
    variants = {}
    if not args.no_variants:
        for dn in ("f64", "f32", "tf32", "bf16"):
            if dn == args.dtype:
                continue
            tv, rv, _ = timed(data_dev, pne.DTYPES[dn], max(5, args.steps // 5), 2)
            msv = tv / max(5, args.steps // 5)
            variants[dn] = {"value": terms_per_step * world / (msv * 1e-3), "ms_per_step": msv,
                            "log_abs_first": rv[0]["log_abs"], "err_bound_first": rv[0]["err_bound"]}
        # context only: the same step with the enumeration taken from the
        # context's cache (geometry-only work done once, as a user stepping many
        # tensor sets of one geometry would); not the headline
        enum_cache[0] = 1
        tv, rv, _ = timed(data_dev, dtype, max(5, args.steps // 5), 2)
        enum_cache[0] = 0
        msv = tv / max(5, args.steps // 5)
        variants[args.dtype + "_enumeration_cached"] = {"value": terms_per_step * world / (msv * 1e-3),
                                                        "ms_per_step": msv}

    # roofline of the dominant kernel (largest event-timed share of the step)
    fam, (launches, tot) = max(prof.items(), key=lambda kv: kv[1][1])
    avg_ms = tot / max(launches, 1)
    # the launch sequence of a step is fixed for a given network: launches per
    # profiled step times the timed steps
    gpu_launches = int(round(sum(v[0] for v in prof.values()) / prof_steps)) * args.steps
    peak_f64 = pne.pne_measure_fma_peak(ctx.h, pne.PNE_F64, ctypes_stream)
    peak_f32 = pne.pne_measure_fma_peak(ctx.h, pne.PNE_F32, ctypes_stream)
    roof = {"kernel": fam, "bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s",
            "frac": None, "traffic": None}
    if fam == "bp_sweeps":
        iters = [r["bp_iters"] for r in res[:B]]
        flops = algorithmic_bp_flops(g, iters)
        if args.bp == "ff":
            # float-float sweeps: a multiply-add costs 16 FP32 instructions (8 for the
            # error-free product, 8 for the compensated accumulation), so the ALU
            # roof for this work is the FP32 FMA-chain rate / 16
            roof.update(achieved=flops / (avg_ms * 1e-3) / 1e12, peak=peak_f32 / 16 / 1e12,
                        peak_source="measured FP32 FMA-chain kernel (pne_measure_fma_peak) / 16 FP32 "
                                    "instructions per float-float multiply-add",
                        work=f"4 flops per tensor entry per site per sweep; {sum(iters)} sweeps over {B} sets")
        else:
            roof.update(achieved=flops / (avg_ms * 1e-3) / 1e12, peak=peak_f64 / 1e12,
                        peak_source="measured FP64 FMA-chain kernel (pne_measure_fma_peak)",
                        work=f"4 flops per tensor entry per site per sweep; {sum(iters)} sweeps over {B} sets")
    elif fam == "contract":
        ns, keep = pne.network_struct(g, data=data_dev, n_batch=B)
        part, _ = pne.pne_build_partition(ctx.h, ns, pne.PartitionOpts(1e-13, 10000, 0.0, BP_ARITH[args.bp]), ctypes_stream)
        terms, _, _ = pne.pne_enumerate_terms(ctx.h, part, pne.EnumOpts(K, mode, 0), ctypes_stream)
        fma = pne.pne_terms_work(ctx.h, terms, ctypes_stream)
        pne.pne_terms_destroy(terms); pne.pne_partition_destroy(part)
        pk = peak_f64 if args.dtype == "f64" else peak_f32
        roof.update(achieved=2.0 * fma * B / (avg_ms * 1e-3) / 1e12, peak=pk / 1e12,
                    peak_source="measured FMA-chain kernel (pne_measure_fma_peak)",
                    work=f"2 flops per plan multiply-add; {fma} multiply-adds per network")
    elif fam in ("enum_expand", "enum_dfs"):
        # the cluster search is integer work bound by latency; its algorithmic
        # traffic is the cluster lists it writes (edges, sorted vertices, size)
        n_cl = res[0]["n_clusters"]
        per_cluster = 4 * K + 4 * (K + 1) + 4
        per_search_ms = tot / prof_steps
        peak_gbs, src = hbm_peak()
        roof.update(bound="hbm", unit="GB/s", achieved=n_cl * per_cluster / (per_search_ms * 1e-3) / 1e9,
                    peak=peak_gbs, peak_source=src,
                    work=f"{n_cl} clusters x {per_cluster} B written per search "
                         f"({launches // prof_steps} launches per search, timed together)")
    if roof["achieved"] is not None and roof["peak"]:
        roof["frac"] = roof["achieved"] / roof["peak"]
    roof["avg_launch_ms"] = avg_ms
    roof["kernel_shares"] = {k: round(v[1] / sum(x[1] for x in prof.values()), 4) for k, v in prof.items()}
    # context beside the dominant kernel: the contraction and BP sweeps against
    # their own arithmetic roofs (event-timed in the same profiled steps)
    others = {}
    if "contract" in prof and fam != "contract":
        ns, keep = pne.network_struct(g, data=data_dev, n_batch=B)
        part, _ = pne.pne_build_partition(ctx.h, ns, pne.PartitionOpts(1e-13, 10000, 0.0, BP_ARITH[args.bp]), ctypes_stream)
        terms, _, _ = pne.pne_enumerate_terms(ctx.h, part, pne.EnumOpts(K, mode, 0), ctypes_stream)
        if mode == pne.PNE_MODE_LOOP:
            fma = pne.pne_terms_work(ctx.h, terms, ctypes_stream)
            c_ms = prof["contract"][1] / prof_steps
            pk = peak_f64 if args.dtype == "f64" else peak_f32
            ach = 2.0 * fma * B / (c_ms * 1e-3) / 1e12
            others["contract"] = {"bound": "alu", "unit": "TFLOP/s", "achieved": ach, "peak": pk / 1e12,
                                  "frac": ach / (pk / 1e12), "ms_per_step": c_ms,
                                  "work": f"2 flops per plan multiply-add; {fma} multiply-adds per network",
                                  "peak_source": "measured FMA-chain kernel (pne_measure_fma_peak)"}
        pne.pne_terms_destroy(terms); pne.pne_partition_destroy(part)
    if "bp_sweeps" in prof and fam != "bp_sweeps" and args.bp == "ff":
        iters = [r["bp_iters"] for r in res[:B]]
        b_ms = prof["bp_sweeps"][1] / prof_steps
        ach = algorithmic_bp_flops(g, iters) / (b_ms * 1e-3) / 1e12
        others["bp_sweeps"] = {"bound": "alu", "unit": "TFLOP/s", "achieved": ach, "peak": peak_f32 / 16 / 1e12,
                               "frac": ach / (peak_f32 / 16 / 1e12), "ms_per_step": b_ms,
                               "work": f"4 flops per tensor entry per site per sweep; {sum(iters)} sweeps over {B} sets",
                               "peak_source": "measured FP32 FMA-chain kernel / 16 FP32 instructions per "
                                              "float-float multiply-add"}
    if others:
        roof["others"] = others

    out = {
        "metric": "PNE terms contracted/sec",
        "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": wl["desc"], "networks_per_step_per_gpu": B, "terms_per_network": n_terms,
                   "clusters_per_network": res[0]["n_clusters"], "K": K,
                   "l2": "flushed between timed steps (256 MB write)",
                   "enumeration": "recomputed every step (cache off)",
                   "parallelism": f"independent networks per GPU x{world}"},
        "e2e": {"value": terms_per_step * world / (e2e_ms * 1e-3), "unit": "terms/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": gpu_launches,
        "host_ms_per_step": host_ms,
        "roofline": roof,
        "clocks": clk,
        "variants": variants,
        "peaks_measured": {"fp64_tflops": peak_f64 / 1e12, "fp32_tflops": peak_f32 / 1e12},
    }

    # CPU baseline: the oracle on a bounded sample (rank 0, single GPU only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # whole networks of the step, in order, until about 10 s of CPU work
        nt, secs, r = oracle_step(wl, nets[0])
        used = 1
        while secs < 10.0 and used < B:
            nt_i, secs_i, _ = oracle_step(wl, nets[used])
            nt += nt_i; secs += secs_i; used += 1
        out["cpu_baseline"] = {"value": nt / secs, "unit": "terms/s", "cores": 1, "kind": "oracle",
                               "sample": f"networks 0..{used - 1} of the {B} per step, full oracle pipeline "
                                         f"({nt} terms in {secs:.1f} s, single thread)"}
        # time to 1e-6: cheapest dtype whose result is within 1e-6 of the oracle
        ttt = {}
        for dn in ("bf16", "tf32", "f32", "f64"):
            (rr,) = ctx.expand(nets[0], K, mode, pne.DTYPES[dn])
            err = abs(math.expm1(rr["log_abs"] - r.log_abs))
            ms = ms_per_step if dn == args.dtype else variants.get(dn, {}).get("ms_per_step")
            ttt[dn] = {"rel_err_vs_oracle": err, "ms_per_step": ms, "reached_1e-6": bool(err <= 1e-6)}
        ok = [d for d in ("bf16", "tf32", "f32", "f64") if ttt[d]["reached_1e-6"]]
        out["time_to_1e-6"] = {"cheapest_dtype": ok[0] if ok else None,
                               "ms_per_step": ttt[ok[0]]["ms_per_step"] if ok else None, "by_dtype": ttt}
    if rank == 0:
        print(json.dumps(out))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def run_batched(args, wl, rank, world, local_rank):
    """cfg4: networks grouped by geometry; one partition and one enumeration
    per group (enumeration is geometry-only and built once), one batch over all
    groups.  A step re-runs every partition on its tensors (BP, gauge) and
    replays the batch's graph (conversion, fused contraction + term sums,
    per-order reduction, copy-back)."""
    import torch
    import torch.distributed as dist
    from paper_2512_10910_gb300 import pne
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    dtype = pne.DTYPES[args.dtype]
    t0 = time.time()
    work = I.batched_workload(wl["n"], 1234 + 1000003 * rank)
    groups = {}
    for kind, L, D, beta, net in work:
        groups.setdefault((L, D), []).append(net)
    ctx = pne.Context(local_rank)
    parts, terms, datas, keep = [], [], [], []
    for (L, D), nets in sorted(groups.items()):
        g = nets[0]
        flat = np.concatenate([n.flat_data()[0] for n in nets])
        data = torch.from_numpy(flat).to(dev)
        ns, kp = pne.network_struct(g, data=data, n_batch=len(nets))
        p, _ = pne.pne_build_partition(ctx.h, ns, pne.PartitionOpts(1e-13, 10000, 0.0, BP_ARITH[args.bp]), sh)
        t, _, _ = pne.pne_enumerate_terms(ctx.h, p, pne.EnumOpts(wl["K"], wl["mode"], 1), sh)
        parts.append(p); terms.append(t); datas.append(data); keep.append((ns, kp))
    batch = pne.pne_batch_create(ctx.h, terms, dtype, None, sh)
    wpb, bps, tuned = pne.pne_batch_config(batch)
    setup_s = time.time() - t0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # the geometry groups' partitions are independent: their updates run on
    # several streams without waiting for their convergence records (the
    # batch run reads them all at once), joined into the batch's stream
    side = [torch.cuda.Stream(dev) for _ in range(8)]
    uopts = pne.PartitionOpts(1e-13, 10000, 0.0, BP_ARITH[args.bp], 1)

    def step():
        for st in side:
            st.wait_stream(stream)
        for i, (p, d) in enumerate(zip(parts, datas)):
            pne.pne_partition_update(ctx.h, p, d, uopts, side[i % len(side)].cuda_stream)
        for st in side:
            stream.wait_stream(st)
        return pne.pne_batch_run(ctx.h, batch, sh)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local_rank)
    clocks.start()
    pne.pne_ctx_profile(ctx.h, True)
    total = 0.0
    res = None
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True); e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res = step()
        e.record(stream); e.synchronize()
        total += a.elapsed_time(e)
    prof = {k: v for k, v in pne.pne_ctx_profile_read(ctx.h).items() if not k.startswith("host:")}
    pne.pne_ctx_profile(ctx.h, False)
    clk = clocks.stop()
    if world > 1:
        tt = torch.tensor([total], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total = float(tt.item())
    ms = total / args.steps
    n_terms = sum(r["n_terms"] for r in res)
    n_clusters = sum(r["n_clusters"] for r in res)
    fam, (launches, tot) = max(prof.items(), key=lambda kv: kv[1][1])
    out = {"metric": "PNE terms contracted/sec", "value": n_terms * world / (ms * 1e-3), "unit": "terms/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
           "config": {"workload": wl["desc"], "networks": len(work), "geometry_groups": len(groups),
                      "terms_per_step": n_terms, "clusters_per_step": n_clusters,
                      "launch_shape": {"warps_per_block": wpb, "blocks_per_sm": bps, "tuned_ms": tuned},
                      "setup_s": setup_s, "enumeration": "per geometry, built once at setup",
                      "l2": "flushed between timed steps (256 MB write)"},
           "gpu_launches": int(sum(v[0] for v in prof.values())),
           "kernel_shares": {k: round(v[1] / sum(x[1] for x in prof.values()), 4) for k, v in prof.items()},
           "kernel_ms_per_step": {k: round(v[1] / args.steps, 3) for k, v in prof.items()},
           "clocks": clk}
    if rank == 0:
        print(json.dumps(out))
    pne.pne_batch_destroy(batch)
    for t in terms:
        pne.pne_terms_destroy(t)
    for p in parts:
        pne.pne_partition_destroy(p)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    del fam, launches, tot


def serve_trace(n, rate, seed):
    """Arrival times and request descriptors of the served workload."""
    u = I.splitmix64_uniform(seed, 6 * n).reshape(n, 6)
    gaps = -np.log(1.0 - u[:, 0]) / rate
    t = np.cumsum(gaps)
    reqs = []
    for i in range(n):
        K = 4 + min(4, int(u[i, 1] * 5))
        if u[i, 2] < 0.5:
            reqs.append(("aklt", 8 + min(24, int(u[i, 3] * 25)), 4, K, None))
        else:
            reqs.append(("rand3d", 6 + min(6, int(u[i, 3] * 7)), 2 + min(2, int(u[i, 4] * 3)), K,
                         seed * 1000003 + i))
    return t, reqs


def run_serve(args, wl, rank, world, local_rank):
    """cfg5: requests replayed in real time against the library's server.
    Geometries (and their enumerations) are warmed once before the trace."""
    import torch
    from paper_2512_10910_gb300 import pne
    torch.cuda.set_device(local_rank)
    duration = max(0.5, args.steps / 10.0)            # --steps 20 -> a 2 s trace
    n = int(wl["rate"] * duration)
    t_arr, reqs = serve_trace(n, wl["rate"], 7 + rank)
    geoms, flats = {}, {}

    def build(kind, L, D, K, seed):
        key = (kind, L, D)
        if key not in geoms:
            g = I.square_lattice(L, L, 4) if kind == "aklt" else I.cubic_lattice(L, L, L, D)
            if kind == "aklt":
                flats[key] = I.aklt_tensors(g).flat_data()[0]
            geoms[key] = g
        g = geoms[key]
        if kind == "aklt":
            flat = flats[key]
        else:
            size = int(sum(np.prod(g.leg_dims(v)) for v in range(g.n_sites))) if key not in flats else flats[key]
            flats[key] = size
            flat = I.splitmix64_normal(seed, size, 1.0, 0.3)     # the random_tensors layout, sites in order
        return pne.network_struct(g, data=flat)

    t0 = time.time()
    structs = [build(*r) for r in reqs]
    build_s = time.time() - t0
    dtype = pne.DTYPES[args.dtype]
    ctx = pne.Context(local_rank)
    opts = pne.ServerOpts(64 << 30, 512, 12, 512, dtype, 0, 0)
    srv = pne.pne_server_create(ctx.h, opts)
    # warm the geometry cache: one request per distinct (geometry, K)
    seen, warm = set(), []
    for (ns, keep), r in zip(structs, reqs):
        key = (r[0], r[1], r[2], r[3])
        if key not in seen:
            seen.add(key)
            warm.append(pne.pne_server_submit(srv, ns, r[3]))
    pne.pne_server_drain(srv)
    warm_failed = {}
    for rid in warm:
        st, _, _ = pne.pne_server_poll(srv, rid)
        if st != pne.PNE_OK:
            warm_failed[int(st)] = warm_failed.get(int(st), 0) + 1
    if warm_failed:
        # a failed warm-up request is reported, and the trace is not run on a
        # context that may have lost its device
        print(json.dumps({"error": "warm-up requests failed", "failed_by_status": warm_failed,
                          "first_error": pne.pne_server_first_error(srv)}), file=sys.stderr)
        pne.pne_server_destroy(srv)
        ctx.close()
        return 1
    clocks = ClockSampler(local_rank)
    clocks.start()
    ids = []
    start = time.perf_counter()
    for (ns, keep), r, ta in zip(structs, reqs, t_arr):
        delay = ta - (time.perf_counter() - start)
        if delay > 0:
            time.sleep(delay)
        ids.append(pne.pne_server_submit(srv, ns, r[3]))
    pne.pne_server_drain(srv)
    wall = time.perf_counter() - start
    clk = clocks.stop()
    lat, terms, batch, first, last = [], 0, [], None, None
    failed = {}
    for rid in ids:
        st, res, info = pne.pne_server_poll(srv, rid)
        if st != pne.PNE_OK:
            failed[int(st)] = failed.get(int(st), 0) + 1
            continue
        lat.append(info["t_done"] - info["t_arrival"])
        terms += res["n_terms"]
        batch.append(info["batch_size"])
        first = info["t_arrival"] if first is None else min(first, info["t_arrival"])
        last = info["t_done"] if last is None else max(last, info["t_done"])
    peak, _ = pne.pne_server_stats(srv)
    first_error = pne.pne_server_first_error(srv)
    pne.pne_server_destroy(srv)
    ctx.close()
    lat = np.array(lat)
    if not len(lat):
        print(json.dumps({"error": "no request completed", "failed_by_status": failed, "first_error": first_error}),
              file=sys.stderr)
        return 1
    span = last - first
    out = {"metric": "PNE terms contracted/sec", "value": terms / span, "unit": "terms/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * span, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
           "config": {"workload": wl["desc"], "requests": len(ids), "completed": int(len(lat)),
                      "failed_by_status": failed, "first_error": first_error,
                      "offered_rate_req_s": wl["rate"], "trace_s": float(t_arr[-1]),
                      "served_req_s": len(lat) / span, "geometries_warmed": len(seen),
                      "device_budget_bytes": int(opts.device_budget_bytes), "peak_admitted_bytes": peak,
                      "input_build_s": build_s},
           "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99)),
                          "mean": 1e3 * float(lat.mean()), "max": 1e3 * float(lat.max())},
           "batch_size": {"mean": float(np.mean(batch)), "max": int(np.max(batch))},
           "wall_s": wall, "clocks": clk}
    if rank == 0:
        print(json.dumps(out))


def run_reference(args, wl, rank, world):
    """The oracle as the reference arm, on this arm's workload and metric.
    Each step is a bounded sample: the full oracle pipeline on one network;
    the run stops early when the steps would exceed about three minutes."""
    if rank != 0:
        return 0
    g, nets = make_networks(wl, rank)
    for i in range(min(args.warmup, 1)):
        oracle_step(wl, nets[i % len(nets)])
    total_terms, total_s, steps = 0, 0.0, 0
    budget = 180.0
    for i in range(args.steps):
        nt, secs, _ = oracle_step(wl, nets[i % len(nets)])
        total_terms += nt; total_s += secs; steps += 1
        if total_s + secs > budget:
            break
    value = total_terms / total_s
    out = {"impl": "reference", "metric": "PNE terms contracted/sec", "value": value, "unit": "terms/s",
           "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl["desc"], "sample_per_step": "one network, full oracle pipeline"},
           "cpu_baseline": {"value": value, "unit": "terms/s", "cores": 1, "kind": "oracle",
                            "sample": f"{steps} networks, one per step, single thread"},
           "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main() or 0)
