#!/usr/bin/env python3
"""Benchmark of the SIS screening hot path on GB300.

Default workload (the largest single-GPU configuration; the one on which the
metric's comparison with the plain FP64 GPU path is defined): N = 20000
samples, 40 primaries of mixed distributions (uniform, lognormal, signed
normal), units over 5 base dimensions, the full operator library, rung 2
(19.2 M candidate ids), 16 residual targets, top-10000 per target.  One step
= one pass of the whole hot path over it: build the feature space (rung 1
materialised on the device, masks, summaries), then the SIS screen of every
candidate against the 16 targets (unit check, a-priori and realised masks;
a*b, a/b, b/a, a+b, a-b from the multi-target Gram contraction on the
tensor cores, BF16x3 with FP32 bounds; stored, unary and |a-b| candidates
evaluated in FP32 on the CUDA cores; streaming top-k, exact selection with
the FP32-pair / FP64 re-score of the boundary).  Inputs are resident in HBM when the timed region starts; L2 is
flushed (256 MiB write) between steps.

Metric: SIS-screened candidate features per second (valid candidates, each
scored on all N samples against every target), with evals/s (candidate x
sample) and the plain FP64 GPU path on the same workload beside it.  Prints
one JSON line (rank 0).  With N > 1 ranks (torchrun) the candidate ids are
split into one contiguous block per rank and the per-target top-k lists are
merged after one NCCL all-gather (strong scaling: the total work is fixed).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dse|reference]
    python bench.py --workload medium      # N=1000 residual loop D=1..3 (separate line)
    python bench.py --workload batched     # 256-problem batched screen (separate line)
    python bench.py --workload gmt_small   # the default workload's first 4096 samples,
                                           # screen only (a small case for profiling)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SIS-screened candidate features/sec and evals/sec vs plain FP64 GPU path"
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP32_LANES = 128
# algorithmic FP32 lane operations per (valid candidate, sample) at one target:
# evaluation, sum w, sum w^2 (FMA), sum w*y (FMA)
OPS_PER_EVAL = 4
# Gram path of the product/quotient slots (one FP32 target, 16 <= N <= 2048):
# per pair and sample, 5 contraction entries x 3 slots x 3 BF16 products x 2
# flops of tensor work
GRAM_FLOPS_PER_PAIR_SAMPLE = 5 * 3 * 3 * 2


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            m = json.load(f)
        mhz = float(m.get("sm_max_mhz", SM_MAX_MHZ))
        return mhz, "measured max SM clock (MEASURED_PEAKS.json sm_max_mhz)"
    except Exception:
        return SM_MAX_MHZ, "nominal max SM clock (fallback)"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


_PROBED = {}


def probed_peaks(dse):
    """The library's issue-rate probe (dse_measure_peaks), run once per
    process: FP32 FMA, MUFU and FP64 FMA lane operations per second."""
    if not _PROBED:
        _PROBED.update(dse.measure_peaks())
    return dict(_PROBED)


def alu_peak(dse):
    """FP32 ALU roofline denominator in T lane-ops/s (an FMA is one lane
    operation) and its source."""
    p = probed_peaks(dse)
    return p["fp32_fma_per_s"] / 1e12, "FP32 FMA issue rate measured on this GPU (dse_measure_peaks)"


def measured_bf16(key):
    """A bf16 tensor peak (TFLOP/s) from MEASURED_PEAKS.json, else the
    recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), f"{key} (MEASURED_PEAKS.json)"
    except Exception:
        return (1900.0 if key == "bf16_tflops" else 1700.0), f"fallback {key}"


def profiled_traffic(name="k_pair_mul_medium.txt"):
    """DRAM bytes (read + write) per launch of the dominant kernel from the
    committed ncu summary of the same kernel and workload, or None."""
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    try:
        tot = 0.0
        found = 0
        with open(os.path.join(ROOT, "profiles", name)) as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 4 and parts[0] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                    tot += float(parts[2]) * scale[parts[3]]
                    found += 1
        return tot if found == 2 else None
    except Exception:
        return None


def workload(seed):
    from paper_2602_06986_gb300 import workloads as W

    return W.medium(seed)


def count_step_evals(stats_list, N):
    cands = sum(s["evaluated"] for s in stats_list)
    return cands, cands * N


def run_step_device(torch, dse, w, Xd, yd, k, D, stream, precision, timing="main"):
    """One step with device-resident inputs: space build, then the residual
    loop D = 1..3 on the device (dse_residual_loop).  timing: "main" times
    the product/quotient kernel group only (two CUDA events per screen),
    "all" every group, None nothing.  Returns (per-screen stats, chosen
    ids)."""
    sp = dse.Space(Xd, w["units"], w["op_mask"], w["max_rung"], unit_check_addsub=w["unit_check_addsub"],
                   explog_dimensionless=w["explog_dimensionless"], stream=stream)
    flags = {"main": dse.FLAG_TIMING_MAIN, "all": dse.FLAG_TIMING, None: 0}[timing]
    out = sp.residual_loop(yd, D, k, precision=precision, stream=stream, flags=flags)
    sp.free()
    return out["stats"], out["chosen"]


def run_step_host(dse, w, k, D):
    """One step through the public API with host buffers: the primaries and
    the target are copied to the device inside the step, the SIS subspaces,
    the final residual and the picks come back to host memory."""
    X = w["X"]
    y = np.ascontiguousarray(w["Y"][0])
    sp = dse.Space(X, w["units"], w["op_mask"], w["max_rung"], unit_check_addsub=w["unit_check_addsub"],
                   explog_dimensionless=w["explog_dimensionless"])
    sis = np.zeros((D, k), np.uint64)
    resid = np.zeros(len(y))
    out = sp.residual_loop(y, D, k, sis_ids=sis, residual=resid)
    sp.free()
    h2d = X.nbytes + w["units"].nbytes + y.nbytes
    d2h = sis.nbytes + resid.nbytes + ctypes_sizeof_loop_result(dse)
    return out["stats"], h2d, d2h


def ctypes_sizeof_loop_result(dse):
    import ctypes

    return ctypes.sizeof(dse.LoopResult)


def cpu_oracle_step(w, k, D):
    import oracle

    t0 = time.perf_counter()
    S = oracle.Space(w["X"], w["units"], w["op_mask"], w["max_rung"], unit_check_addsub=w["unit_check_addsub"],
                     explog_dimensionless=w["explog_dimensionless"])
    out = S.residual_loop(w["Y"][0], D, k)
    dt = time.perf_counter() - t0
    # valid candidates scored by one screen of the full space, per screen
    slots, rs = S.rung_counts(w["max_rung"])
    per_screen = S.n_features + rs["valid"]
    return dt, per_screen * D, out


def bench_batched(args):
    """The batched workload: 256 problems (32 base data sets x 5 CV folds + 3
    bootstrap resamples, N in [50, 5000], 10-30 primaries, rung 2, top-200
    each).  Spaces are built once (untimed); a step is one screen of every
    problem with fresh targets: eager (plan reused) and CUDA-graph
    replay, targets device resident."""
    import torch

    from paper_2602_06986_gb300 import _build
    from paper_2602_06986_gb300 import workloads as W

    _build.build()
    from paper_2602_06986_gb300 import dse

    w = W.batched(0)
    kw = dict(unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    Xd = [torch.from_numpy(b["X"]).cuda() for b in w["bases"]]
    t0 = time.perf_counter()
    spaces = [dse.Space(Xd[p["base"]], w["bases"][p["base"]]["units"], w["op_mask"], w["max_rung"],
                        sample_idx=p["samples"], **kw) for p in w["problems"]]
    build_s = time.perf_counter() - t0
    targets = [w["bases"][p["base"]]["y"][p["samples"]] for p in w["problems"]]
    Ycat = torch.from_numpy(np.concatenate(targets)).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # job size of the batched plan, tuned on the device (untimed)
    from paper_2602_06986_gb300 import autotune as at

    def one_batch():
        bt0 = dse.Batch(spaces, targets, w["k"])
        bt0.fetch(0)
        bt0.free()

    entry = at.tune("batched", max(len(t) for t in targets), 1, one_batch, reps=2)
    dse.set_tuning(entry["config"] or None)
    tuning = {"chosen": entry["config"] or "defaults", "in_effect": dse.get_tuning(),
              "tried_ms": [[t["config"], round(t["seconds"] * 1e3, 2)] for t in entry["tried"]]}
    res = {}
    for mode in ("eager", "graph"):
        bt = dse.Batch(spaces, targets, w["k"], graph=(mode == "graph"))
        for _ in range(args.warmup):
            bt.rescreen(Ycat)
            bt.fetch(0)
        ms, cands = [], 0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            bt.rescreen(Ycat)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            st = [bt.stats(i) for i in range(len(spaces))]
            cands += sum(s["evaluated"] for s in st)
        tot = sum(ms)
        res[mode] = {"value": cands / (tot * 1e-3), "ms_per_step": tot / args.steps,
                     "reruns": max(s["reruns"] for s in st), "kernel_launches": st[0]["kernel_launches"]}
        bt.free()
    n_total = sum(sp.n_total for sp in spaces)
    # roofline over the whole batched screen (every kernel group; the batch
    # has no per-group events): 4 FP32 lane operations per valid
    # candidate-sample against the measured FP32 FMA rate
    bt = dse.Batch(spaces, targets, w["k"])
    bt.fetch(0)
    st = [bt.stats(i) for i in range(len(spaces))]
    bt.free()
    lane_ops = sum(s["evaluated"] * len(t) for s, t in zip(st, targets)) * OPS_PER_EVAL
    pk, pk_src = alu_peak(dse)
    ach = lane_ops / (res["graph"]["ms_per_step"] * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": "the whole batched screen (k_feature_batched, k_pair<float,..,BATCH>, "
                                          "k_pairlist_batched, selection)",
                "achieved": ach, "peak": pk, "unit": "T fp32-lane-ops/s", "frac": ach / pk, "traffic": None,
                "peak_source": pk_src, "ops_per_candidate_sample": OPS_PER_EVAL,
                "note": "time of the whole step: a lower bound of the dominant kernel's fraction"}
    # the plain FP64 GPU path on the same problems (one eager batch)
    ms64 = []
    for _ in range(2):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b64 = dse.Batch(spaces, targets, w["k"], precision=dse.PREC_FP64)
        b64.fetch(0)
        e1.record()
        torch.cuda.synchronize()
        ms64.append(e0.elapsed_time(e1))
        c64 = sum(b64.stats(i)["evaluated"] for i in range(len(spaces)))
        b64.free()
    fp64 = {"value": c64 / (min(ms64) * 1e-3), "unit": "candidates/s", "ms_per_step": min(ms64),
            "speedup_of_fp32_path": res["graph"]["value"] / (c64 / (min(ms64) * 1e-3)),
            "note": "plan, screen and fetch of every problem in FP64 (best of 2)"}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        # the oracle's full screens of the first problems (about 15 s of CPU
        # work), rate per valid candidate
        c_sum, t_sum, n_done = 0, 0.0, 0
        for p, t in zip(w["problems"], targets):
            b = w["bases"][p["base"]]
            S = oracle.Space(np.ascontiguousarray(b["X"][:, p["samples"]]), b["units"], w["op_mask"], w["max_rung"],
                             **kw)
            t0 = time.perf_counter()
            _, _, cnt = S.screen(t[None, :], w["k"])
            t_sum += time.perf_counter() - t0
            c_sum += cnt["valid"]
            n_done += 1
            if t_sum > 15.0:
                break
        cpu = {"value": c_sum / t_sum, "unit": "candidates/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"full screens of the first {n_done} of {len(spaces)} problems ({c_sum} valid candidates, "
                         f"{t_sum:.1f} s)"}
    line = {"metric": "batched SIS-screened candidate features/sec", "value": res["graph"]["value"],
            "unit": "candidates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["graph"]["ms_per_step"], "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": {"workload": w["name"], "problems": len(spaces), "k": w["k"],
                                            "candidate_slots": n_total, "l2": "flushed between steps"},
            "eager": res["eager"], "graph": res["graph"], "roofline": roofline, "fp64_plain": fp64,
            "cpu_baseline": cpu, "space_build_s_total": build_s, "tuning": tuning}
    print(json.dumps(line))


def bench_multi_target(args, which):
    """Multi-target screens on the tensor-core path (BF16x3 tcgen05): the
    precision workload (N=500, rung 3, one 2^30-id block, 64 targets,
    top-1000 each) or the large one (N=20000, rung 2, 16 targets, top-10000
    each).  The space is built once (untimed); a step is one screen, targets
    resident; L2 flushed between steps."""
    import torch

    from paper_2602_06986_gb300 import _build
    from paper_2602_06986_gb300 import workloads as W

    _build.build()
    from paper_2602_06986_gb300 import dse

    w = W.precision(0, n_targets=64) if which in ("precision", "tc_small") else W.large(0, n_targets=16)
    if which == "tc_small":  # the precision primaries at rung 2: a small case of the same kernels
        w = dict(w, max_rung=2, name="precision_primaries_rung2_T64_top1000")
    if which == "gmt_small":  # the large workload's first 4096 samples: a small case of its kernels
        w = dict(w, X=np.ascontiguousarray(w["X"][:, :4096]), Y=np.ascontiguousarray(w["Y"][:, :4096]),
                 name="large_first4096_samples_rung2_T16_top10000")
    Xd = torch.from_numpy(w["X"]).cuda()
    sp = dse.Space(Xd, w["units"], w["op_mask"], w["max_rung"],
                   unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    Yd = torch.from_numpy(w["Y"]).cuda()
    T, N = w["Y"].shape
    if which == "precision":
        b0 = sp.n_stored + 6 * sp.n_stored + w["block_seed"]
        b1 = min(b0 + w["block_len"], sp.n_total)
    else:
        b0, b1 = 0, 0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        r = sp.screen(Yd, w["k"], id_begin=b0, id_end=b1, precision=dse.PREC_AUTO, flags=dse.FLAG_TIMING)
        r.stats()
        r.free()
    ms, stats = [], []
    clocks = Clocks(0)
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r = sp.screen(Yd, w["k"], id_begin=b0, id_end=b1, precision=dse.PREC_AUTO, flags=dse.FLAG_TIMING)
        st = r.stats()
        e1.record()
        torch.cuda.synchronize()
        r.free()
        ms.append(e0.elapsed_time(e1))
        stats.append(st)
    clk = clocks.stop()
    tot = sum(ms)
    cands = sum(s["evaluated"] for s in stats)
    tc_ms = sum(s["kernel_ms"][1] + s["kernel_ms"][2] for s in stats)
    tc_valid = sum(s["valid_by_group"][1] + s["valid_by_group"][2] for s in stats)
    flops = 6.0 * T * N * tc_valid  # BF16x3: three products of 2 flops per candidate, sample, target
    achieved = flops / (tc_ms * 1e-3) / 1e12 if tc_ms > 0 else None
    peak, peak_src = 1688.5, "bf16_tflops_sustained (MEASURED_PEAKS.json)"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops_sustained"])
    except Exception:
        peak, peak_src = 1700.0, "fallback sustained bf16"
    alu_pk, _ = alu_peak(dse)
    alu = 6.0 * N * tc_valid / (tc_ms * 1e-3) / 1e12 if tc_ms > 0 else None
    roofline = {"bound": "tensor", "kernel": "k_pair_tc (BF16x3 tcgen05)", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak if achieved else None,
                "traffic": None, "peak_source": peak_src, "flops_per_candidate_sample": 6 * T,
                "launch_ms_total_per_step": tc_ms / args.steps,
                "alu_lane_ops_tps": alu, "alu_frac": alu / alu_pk if alu else None}
    if stats[0]["binary_path"] == dse.PATH_GRAM_MT:
        roofline = gmt_roofline(dse, w, Xd, None, sum(s["kernel_ms"][1] for s in stats) / len(stats),
                                tot / args.steps, peak, peak_src)
        roofline["traffic"] = None
    line = {"metric": f"{which}: SIS-screened candidate features/sec (multi-target, tensor cores)",
            "value": cands / (tot * 1e-3), "unit": "candidates/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot / args.steps, "higher_is_better": True, "dtype": "f32+bf16x3",
            "data": "synthetic", "config": {"workload": w["name"], "targets": T, "N": N, "k": w["k"],
                                            "screened_ids": stats[0]["screened"], "l2": "flushed between steps"},
            "evals_per_s": cands * N / (tot * 1e-3), "precision_used": stats[0]["precision_used"],
            "binary_path": stats[0]["binary_path"], "roofline": roofline,
            "per_screen": {k2: sum(s[k2] for s in stats) / len(stats)
                           for k2 in ("evaluated", "buffered", "escalated", "rescored", "reruns")},
            "kernel_group_ms_per_step": [sum(s["kernel_ms"][g] for s in stats) / len(stats) for g in range(4)],
            "clocks": clk}
    print(json.dumps(line))


def bench_l0(args):
    """Exhaustive L0 search over the union of the SIS subspaces of the medium
    workload's residual loop (3 x top-1000): every pair (D = 2) and every
    triple (D = 3) of the union, FP64 on the device.  The subspace is found
    once (untimed); a step is one search per dimension."""
    import math

    import torch

    from paper_2602_06986_gb300 import _build
    from paper_2602_06986_gb300 import workloads as W

    _build.build()
    from paper_2602_06986_gb300 import dse

    w = W.medium(0)
    sp = dse.Space(torch.from_numpy(w["X"]).cuda(), w["units"], w["op_mask"], w["max_rung"],
                   unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    y = np.ascontiguousarray(w["Y"][0])
    D, k = w["D"], w["k"]
    sis = np.zeros((D, k), np.uint64)
    sp.residual_loop(y, D, k, sis_ids=sis)
    ids = np.unique(sis[sis != np.iinfo(np.uint64).max])
    n = len(ids)
    yd = torch.from_numpy(y).cuda()
    idd = torch.from_numpy(ids.astype(np.int64)).cuda()
    res = {}
    for dim in (2, 3):
        for _ in range(args.warmup):
            sp.l0_search(yd, idd, dim, n_top=8)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            pos, rm, cf = sp.l0_search(yd, idd, dim, n_top=8)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = sum(ms) / len(ms)
        subsets = math.comb(n, dim)
        res[f"D{dim}"] = {"ms": t, "subsets": subsets, "subsets_per_s": subsets / (t * 1e-3),
                          "best_rmse": float(rm[0]), "best_ids": [int(ids[p]) for p in pos[0]]}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        orc = oracle.Space(w["X"], w["units"], w["op_mask"], w["max_rung"], unit_check_addsub=w["unit_check_addsub"],
                           explog_dimensionless=w["explog_dimensionless"])
        sub = ids[:400]
        t0 = time.perf_counter()
        orc.l0_search(y, sub, 2, 8)
        dt = time.perf_counter() - t0
        cpu = {"value": math.comb(len(sub), 2) / dt, "unit": "subsets/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": f"D=2 over the first {len(sub)} ids of the union ({dt:.1f} s)"}
    line = {"metric": "exhaustive L0 search: least-squares subsets evaluated per second",
            "value": res["D3"]["subsets_per_s"], "unit": "subsets/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["D3"]["ms"], "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "medium_n1000 SIS-subspace union", "n_ids": n,
                                            "dims": [2, 3]},
            "per_dim": res, "cpu_baseline": cpu}
    print(json.dumps(line))


# ---------------------------------------------------------------- headline

# FP32 lane operations per (valid candidate, sample) that the tensor-core
# multi-target kernel issues on the CUDA cores: the evaluation, sum w and
# sum w^2, and the BF16 hi/lo split (conversion, difference, conversion);
# the T numerators go to the tensor pipe (3 BF16 products of 2 flops each per
# target).
TC_ALU_OPS_PER_EVAL = 6


def large_space(dse, w, X, stream=None):
    return dse.Space(X, w["units"], w["op_mask"], w["max_rung"], unit_check_addsub=w["unit_check_addsub"],
                     explog_dimensionless=w["explog_dimensionless"], stream=stream)


def large_step_device(dse, w, Xd, Yd, k, precision, id_range, stream, flags, group=None):
    """One step with device-resident inputs: space build, then the screen of
    this rank's id block against every target.  With a process group the
    per-target lists of all ranks are merged after one all-gather.  Returns
    the screen's statistics."""
    from paper_2602_06986_gb300 import shard

    sp = large_space(dse, w, Xd, stream)
    b, e = id_range(sp.n_total)
    if group is not None:
        lists, st = shard.sharded_screen(sp, Yd, k, group=group, precision=precision, stream=stream, flags=flags)
        st = st or {"evaluated": 0, "kernel_ms": [0.0] * 4, "valid_by_group": [0, 0, 0], "kernel_launches": 0}
    else:
        r = sp.screen(Yd, k, precision=precision, id_begin=b, id_end=e, stream=stream, flags=flags)
        st = r.stats()
        r.free()
    sp.free()
    return st


def large_step_host(dse, w, k):
    """One step through the public API with host buffers: primaries, units
    and the 16 targets go to the device inside the step, every list (id,
    score, bound) comes back to host memory."""
    X, Y = w["X"], np.ascontiguousarray(w["Y"])
    sp = large_space(dse, w, X)
    r = sp.screen(Y, k, precision=dse.PREC_AUTO)
    d2h = 0
    for t in range(r.n_lists):
        ids, sc, eb = r.fetch(t)
        d2h += ids.nbytes + sc.nbytes + eb.nbytes
    st = r.stats()
    r.free()
    sp.free()
    h2d = X.nbytes + w["units"].nbytes + Y.nbytes
    return st, h2d, d2h


def oracle_large_block(w, S, begin, n_ids):
    """The oracle's screen of ids [begin, begin + n_ids) of the large
    workload: (valid candidates, seconds)."""
    t0 = time.perf_counter()
    _, _, cnt = S.screen(w["Y"], w["k"], id_begin=begin, id_end=begin + n_ids)
    return cnt["valid"], time.perf_counter() - t0


def oracle_large_space(w):
    import oracle

    oracle.build()
    return oracle.Space(w["X"], w["units"], w["op_mask"], w["max_rung"], unit_check_addsub=w["unit_check_addsub"],
                        explog_dimensionless=w["explog_dimensionless"])


def binary_pairs(sp, max_rung):
    """Pairs (i, j), j < i, of the binary block of the last rung: i among the
    features of rung max_rung - 1 (ids from o), j any stored feature."""
    n = sp.n_stored
    o = sum(sp.counts(r)[1]["valid"] for r in range(max_rung - 1))
    return n * (n - 1) // 2 - o * (o - 1) // 2


# contraction entries per ordered pair and sample of the multi-target Gram
# kernel at T targets: H (q y_t of x and of 1/x) and G (p q, p q^2, p^2 q,
# p^2 q^2 of both families); 2 flops each, 3 BF16 products each (BF16x3)
def gmt_flops_per_ordered_pair_sample(T):
    return (2 * T + 8) * 2 * 3


def gmt_roofline(dse, w, Xd, stream, launch_ms, step_ms, tc_peak, tc_src):
    """Roofline of k_pair_gmt: algorithmic flops = the contraction entries
    the method needs for every ordered pair of the binary block (both orders:
    a/b and b/a) x N samples; time = the kernel's CUDA events in the timed
    steps."""
    T, N = w["Y"].shape
    sp = large_space(dse, w, Xd, stream)
    pairs = binary_pairs(sp, w["max_rung"])
    sp.free()
    fl = gmt_flops_per_ordered_pair_sample(T)
    flops = 2.0 * pairs * N * fl
    achieved = flops / (launch_ms * 1e-3) / 1e12 if launch_ms > 0 else None
    return {"bound": "tensor",
            "kernel": "k_pair_gmt (multi-target Gram contraction, BF16x3 tcgen05: a/b, b/a, a*b, a+b, a-b)",
            "achieved": achieved, "peak": tc_peak, "unit": "TFLOP/s",
            "frac": achieved / tc_peak if achieved else None,
            "traffic": profiled_traffic("k_pair_gmt_large.txt"),
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch "
                              "(profiles/k_pair_gmt_large.txt)",
            "peak_source": tc_src + " (of measured, sustained: the kernel runs inside a long step)",
            "flops_per_ordered_pair_sample": fl, "ordered_pairs": 2 * pairs, "flops_per_launch": flops,
            "launch_ms": launch_ms, "share_of_step": launch_ms / step_ms}


def tc_roofline(dse, T, N, mul_ms, mul_valid, step_ms, stats, tc_peak, tc_src):
    """Roofline of k_pair_tc (sample-by-sample generation on the FP32 pipes,
    numerators on the tensor cores): the FP32 ALU bound, with the tensor
    fraction beside it."""
    alu_pk, alu_src = alu_peak(dse)
    ntp = 16 if T <= 16 else 32 if T <= 32 else 64
    alu = TC_ALU_OPS_PER_EVAL * N * mul_valid / (mul_ms * 1e-3) / 1e12 if mul_ms > 0 else None
    tc_flops = 6.0 * ntp * N * mul_valid / (mul_ms * 1e-3) / 1e12 if mul_ms > 0 else None
    return {"bound": "alu", "kernel": f"k_pair_tc<KIND_MUL,{ntp}> (a*b, a/b, b/a; BF16x3 tcgen05 numerators)",
            "achieved": alu, "peak": alu_pk, "unit": "T fp32-lane-ops/s",
            "frac": alu / alu_pk if alu else None,
            "traffic": profiled_traffic("k_pair_tc_large.txt"),
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch "
                              "(profiles/k_pair_tc_large.txt)",
            "peak_source": alu_src,
            "ops_per_candidate_sample": TC_ALU_OPS_PER_EVAL, "valid_candidates_per_launch": mul_valid / len(stats),
            "launch_ms": mul_ms / len(stats), "share_of_step": mul_ms / sum(step_ms),
            "tensor": {"achieved": tc_flops, "peak": tc_peak, "unit": "TFLOP/s",
                       "frac": tc_flops / tc_peak if tc_flops else None,
                       "flops_per_candidate_sample": 6 * ntp, "peak_source": tc_src + " (of measured)"}}


def bench_large(args):
    from paper_2602_06986_gb300 import workloads as W

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    w = W.large(0)
    k = w["k"]
    T, N = w["Y"].shape
    config = {"workload": w["name"], "N": N, "n_primary": int(w["X"].shape[0]), "max_rung": w["max_rung"],
              "targets": T, "k": k, "precision": "AUTO: binary slots from BF16x3 tcgen05 Gram contractions (FP32 bounds), "
                                                 "stored/unary and |a-b| on FP32 CUDA cores",
              "l2": "flushed between steps (256 MiB write); stored FP32 rows 0.2 GB > L2",
              "parallelism": ("one GPU" if world == 1 else
                              f"id-range split over {world} ranks + NCCL all-gather of the top-k lists")}

    if args.impl == "reference":
        # the reference arm is the CPU FP64 oracle, timed on the host cores
        # on bounded contiguous id blocks of the same workload
        if rank != 0:
            return
        import oracle

        S = oracle_large_space(w)
        rng = np.random.Generator(np.random.PCG64(77))
        n_ids = args.ref_ids
        offs = rng.integers(0, S.total_candidates - n_ids, size=args.warmup + args.steps)
        for i in range(args.warmup):
            oracle_large_block(w, S, int(offs[i]), n_ids)
        tot, cands = 0.0, 0
        for i in range(args.steps):
            c, dt = oracle_large_block(w, S, int(offs[args.warmup + i]), n_ids)
            tot += dt
            cands += c
        v = cands / tot
        sample = (f"{args.steps} contiguous blocks of {n_ids} candidate ids at seeded offsets, one per step, "
                  f"screened against all {T} targets (the oracle's space build, 1% of the work, excluded)")
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "candidates/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": v, "unit": "candidates/s", "cores": oracle.num_threads(),
                                 "kind": "oracle", "sample": sample},
                "e2e": {"value": v, "unit": "candidates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch

    torch.cuda.set_device(local)
    group = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        group = dist.group.WORLD
    from paper_2602_06986_gb300 import _build

    if rank == 0:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    _build.build()
    from paper_2602_06986_gb300 import dse

    stream = torch.cuda.current_stream().cuda_stream
    Xd = torch.from_numpy(w["X"]).cuda()
    Yd = torch.from_numpy(np.ascontiguousarray(w["Y"])).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    whole = lambda n: (0, 0)  # noqa: E731  (the whole space; sharding goes through the group)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    # the planner's tile settings for this workload class, tuned on the
    # device (untimed; coordinate descent from the defaults, 2 runs each)
    tuning = None
    if not args.no_tune:
        from paper_2602_06986_gb300 import autotune as at

        sp_t = large_space(dse, w, Xd, stream)
        r_t = sp_t.screen(Yd, k, precision=dse.PREC_AUTO, stream=stream)
        kclass = "screen_gmt" if r_t.stats()["binary_path"] == dse.PATH_GRAM_MT else "screen_tc"
        r_t.free()
        entry = at.tune(kclass, N, T, lambda: sp_t.screen(Yd, k, precision=dse.PREC_AUTO, stream=stream).free(),
                        reps=2)
        sp_t.free()
        chosen = entry["config"]
        if world > 1:  # every rank uses rank 0's choice
            obj = [chosen]
            torch.distributed.broadcast_object_list(obj, src=0)
            chosen = obj[0]
        dse.set_tuning(chosen or None)
        tuning = {"kernel_class": at.key(kclass, N, T), "chosen": chosen or "defaults",
                  "in_effect": dse.get_tuning(),
                  "tried_ms": [[t["config"], round(t["seconds"] * 1e3, 2)] for t in entry["tried"]]}
    for _ in range(args.warmup):
        large_step_device(dse, w, Xd, Yd, k, dse.PREC_AUTO, whole, stream, dse.FLAG_TIMING_MAIN, group)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    L0 = dse.lib().dse_kernel_launches()
    step_ms, stats = [], []
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.cuda.nvtx.range_push("timed_step")
        st = large_step_device(dse, w, Xd, Yd, k, dse.PREC_AUTO, whole, stream, dse.FLAG_TIMING_MAIN, group)
        torch.cuda.nvtx.range_pop()
        e1.record()
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stats.append(st)
    launches = dse.lib().dse_kernel_launches() - L0
    barrier()
    clk = clocks.stop()
    tot_ms = sum(step_ms)
    cands_local = sum(s["evaluated"] for s in stats)
    if world > 1:
        t = torch.tensor([tot_ms, float(cands_local)], dtype=torch.float64, device="cuda")
        tmax = t.clone()
        torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
        tot_ms, cands = float(tmax[0].item()), int(t[1].item())
    else:
        cands = cands_local
    value = cands / (tot_ms * 1e-3)

    # dominant kernel: the binary slots' group on the tensor cores, live
    # CUDA events in the timed steps
    mul_ms = sum(s["kernel_ms"][1] for s in stats)
    mul_valid = sum(s["valid_by_group"][1] for s in stats)
    tc_peak, tc_src = measured_bf16("bf16_tflops_sustained")
    if stats[0].get("binary_path") == dse.PATH_GRAM_MT:
        roofline = gmt_roofline(dse, w, Xd, stream, mul_ms / len(stats), sum(step_ms) / len(stats), tc_peak, tc_src)
    else:
        roofline = tc_roofline(dse, T, N, mul_ms, mul_valid, step_ms, stats, tc_peak, tc_src)
    # the kernel groups' device times from one more (untimed) step with an
    # event at every group boundary
    flush.zero_()
    barrier()
    st_all = large_step_device(dse, w, Xd, Yd, k, dse.PREC_AUTO, whole, stream, dse.FLAG_TIMING, group)
    group_ms = st_all["kernel_ms"]

    # the plain FP64 GPU path on the same workload (same step, FP64 kernels)
    fp64_ms, fp64_c = [], 0
    for _ in range(args.fp64_steps):
        flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st64 = large_step_device(dse, w, Xd, Yd, k, dse.PREC_FP64, whole, stream, 0, group)
        e1.record()
        torch.cuda.synchronize()
        fp64_ms.append(e0.elapsed_time(e1))
        fp64_c += st64["evaluated"]
    fp64_tot = sum(fp64_ms)
    if world > 1:
        t = torch.tensor([fp64_tot, float(fp64_c)], dtype=torch.float64, device="cuda")
        tmax = t.clone()
        torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
        fp64_tot, fp64_c = float(tmax[0].item()), int(t[1].item())
    fp64 = None
    if fp64_ms:
        fp64_value = fp64_c / (fp64_tot * 1e-3)
        # FP64 lane operations of the plain path: evaluation, sum w, sum w^2
        # and one FMA per target, per valid candidate and sample
        fp64_rate = fp64_c * N * (3 + T) / (fp64_tot * 1e-3)  # all ranks' candidates over the slowest rank's time
        pk = probed_peaks(dse)["fp64_fma_per_s"]
        fp64 = {"value": fp64_value, "unit": "candidates/s", "ms_per_step": fp64_tot / len(fp64_ms),
                "steps": len(fp64_ms), "speedup_of_fp32_path": value / fp64_value,
                "fp64_lane_ops_per_s": fp64_rate, "fp64_peak_lane_ops_per_s": pk * world,
                "fp64_frac": fp64_rate / (pk * world) if pk else None,
                "fp64_peak_source": "FP64 FMA issue rate measured on this GPU (dse_measure_peaks)"}

    # end to end through the public API with host buffers (rank 0's GPU; the
    # whole workload on one device)
    e2e = None
    if rank == 0 and not args.no_e2e:
        e2e_ms, e2e_c = [], 0
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st_h, h2d, d2h = large_step_host(dse, w, k)
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            e2e_c += st_h["evaluated"]
        e2e = {"value": e2e_c / (sum(e2e_ms) * 1e-3), "unit": "candidates/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": sum(e2e_ms) / len(e2e_ms),
               "note": "host buffers through the C ABI on one GPU, copies inside the timed region"}
    if world > 1:
        torch.distributed.barrier()
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        S = oracle_large_space(w)
        rng = np.random.Generator(np.random.PCG64(76))
        n_ids = min(args.cpu_ids, S.total_candidates)
        b0 = int(rng.integers(0, S.total_candidates - n_ids + 1))
        c, dt = oracle_large_block(w, S, b0, n_ids)
        cpu = {"value": c / dt, "unit": "candidates/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"ids [{b0}, {b0 + n_ids}) of the same workload ({n_ids} contiguous ids, {c} valid, all "
                         f"{T} targets, top-{k}), {dt:.1f} s; rate extrapolated to the whole space"}
    line = {
        "metric": METRIC, "value": value, "unit": "candidates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
        "evals_per_s": value * N,
        "fp64_plain": fp64,
        "roofline": roofline,
        "kernel_group_ms_per_step": {"stored_unary": group_ms[0], "pair_mul": group_ms[1], "pair_add": group_ms[2],
                                     "select": group_ms[3], "source": "one untimed step with an event per group"},
        "per_screen": {key: sum(s[key] for s in stats) / len(stats)
                       for key in ("screened", "evaluated", "buffered", "escalated", "rescored", "reruns",
                                   "kernel_launches")},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "tuning": tuning,
        "measured_peaks": {"fp32_fma_per_s": probed_peaks(dse)["fp32_fma_per_s"],
                           "sfu_per_s": probed_peaks(dse)["sfu_per_s"],
                           "fp64_fma_per_s": probed_peaks(dse)["fp64_fma_per_s"],
                           "source": "dse_measure_peaks on this GPU (lane operations per second)"},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dse", choices=["dse", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="large",
                    choices=["large", "medium", "batched", "precision", "large_screen", "tc_small", "gmt_small", "l0"])
    ap.add_argument("--cpu-ids", type=int, default=1_000_000,
                    help="contiguous candidate ids the oracle screens for the cpu_baseline of the large workload")
    ap.add_argument("--ref-ids", type=int, default=100_000,
                    help="candidate ids per step of the reference (oracle) arm on the large workload")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the plain FP64 GPU path (0: skip)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) leg")
    ap.add_argument("--no-tune", action="store_true", help="keep the planner's default tile settings")
    args = ap.parse_args()
    if args.workload == "large":
        return bench_large(args)
    if args.workload == "batched":
        return bench_batched(args)
    if args.workload in ("precision", "large_screen", "tc_small", "gmt_small"):
        return bench_multi_target(args, "large" if args.workload == "large_screen" else args.workload)
    if args.workload == "l0":
        return bench_l0(args)
    return bench_medium(args)


def bench_medium(args):

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    w = workload(rank)
    k, D = w["k"], w["D"]
    N = w["X"].shape[1]
    config = {"workload": w["name"], "N": N, "n_primary": int(w["X"].shape[0]), "max_rung": w["max_rung"],
              "k": k, "D": D, "targets": 1, "l2": "flushed between steps (256 MiB write)",
              "parallelism": f"replicas x{world} (independent workloads, no collective)"}

    if args.impl == "reference":
        # the reference arm is the CPU FP64 oracle, timed on the host cores
        if rank != 0:
            return
        import oracle

        oracle.build()
        for _ in range(args.warmup):
            cpu_oracle_step(w, k, D)
        times, cands = [], 0
        for _ in range(args.steps):
            dt, c, _ = cpu_oracle_step(w, k, D)
            times.append(dt)
            cands += c
        tot = sum(times)
        v = cands / tot
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "candidates/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": v, "unit": "candidates/s", "cores": oracle.num_threads(),
                                 "kind": "oracle", "sample": "the full workload per step (space build + 3 screens "
                                                             "+ refits)"},
                "e2e": {"value": v, "unit": "candidates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2602_06986_gb300 import _build

    _build.build()
    from paper_2602_06986_gb300 import dse

    stream = torch.cuda.current_stream().cuda_stream
    Xd = torch.from_numpy(w["X"]).cuda()
    yd = torch.from_numpy(w["Y"][0].copy()).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    for _ in range(args.warmup):
        run_step_device(torch, dse, w, Xd, yd, k, D, stream, dse.PREC_FP32)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    L0 = dse.lib().dse_kernel_launches()
    step_ms, all_stats = [], []
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.cuda.nvtx.range_push("timed_step")  # lets a profiler select the timed steps' kernels
        stats, picks = run_step_device(torch, dse, w, Xd, yd, k, D, stream, dse.PREC_FP32)
        torch.cuda.nvtx.range_pop()
        e1.record()
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        all_stats.append(stats)
    launches = dse.lib().dse_kernel_launches() - L0
    barrier()
    clk = clocks.stop()
    tot_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([tot_ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        tot_ms = float(t.item())
    cands = sum(count_step_evals(s, N)[0] for s in all_stats)
    value = world * cands / (tot_ms * 1e-3)
    evals_per_s = value * N

    # dominant kernel: the product/quotient pair kernel (live CUDA-event time)
    mul_ms = sum(s["kernel_ms"][1] for st in all_stats for s in st)
    mul_valid = sum(s["valid_by_group"][1] for st in all_stats for s in st)
    mul_launches = sum(1 for st in all_stats for s in st)
    mhz, peak_src = peaks()
    # the kernel groups' device times from one more (untimed) step with an
    # event at every group boundary
    flush.zero_()
    barrier()
    st_all, _ = run_step_device(torch, dse, w, Xd, yd, k, D, stream, dse.PREC_FP32, timing="all")
    group_ms = [sum(s["kernel_ms"][g] for s in st_all) for g in range(4)]
    launch_ms = mul_ms / max(mul_launches, 1)
    if 16 <= N <= 2048:
        # the Gram contraction on the tensor cores: every pair of the binary
        # block (i in the newest stored rung, j < i) is contracted
        sp = dse.Space(Xd, w["units"], w["op_mask"], w["max_rung"], unit_check_addsub=w["unit_check_addsub"],
                       explog_dimensionless=w["explog_dimensionless"])
        o = sp.counts(0)[1]["valid"]
        m = sp.n_stored - o
        pairs = m * (m - 1) // 2 + m * o
        sp.free()
        flops = GRAM_FLOPS_PER_PAIR_SAMPLE * pairs * N
        peak, tc_src = measured_bf16("bf16_tflops")
        achieved = flops / (launch_ms * 1e-3) / 1e12 if launch_ms > 0 else None
        roofline = {"bound": "tensor", "kernel": "k_pair_gram (BF16x3 tcgen05 Gram contraction: a*b, a/b, b/a, a+b, a-b)",
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": (achieved / peak) if achieved else None,
                    # (the committed capture predates the kernel's a+b / a-b slots: no
                    # counters of the current kernel, so no traffic figure)
                    "traffic": None,
                    "traffic_source": "none: profiles/k_pair_gram_medium.txt was captured before the kernel "
                                      "took the a+b and a-b slots",
                    "peak_source": tc_src + " (of measured, burst: the kernel runs ~0.06 ms at a time inside a short step)",
                    "flops_per_launch": flops, "flops_per_pair_sample": GRAM_FLOPS_PER_PAIR_SAMPLE,
                    "pairs": pairs, "launch_ms": launch_ms, "share_of_step": mul_ms / tot_ms}
    else:
        peak, alu_src = alu_peak(dse)  # T lane-ops/s
        achieved = mul_valid * N * OPS_PER_EVAL / (mul_ms * 1e-3) / 1e12 if mul_ms > 0 else None
        roofline = {"bound": "alu", "kernel": "k_pair<float,MUL,1,2,2> (a*b, a/b, b/a slots)",
                    "achieved": achieved, "peak": peak, "unit": "T fp32-lane-ops/s",
                    "frac": (achieved / peak) if achieved else None, "traffic": None,
                    "peak_source": alu_src,
                    "ops_per_eval": OPS_PER_EVAL, "launch_ms": launch_ms, "share_of_step": mul_ms / tot_ms}

    # the plain FP64 GPU path on the same workload (same step, FP64 kernels)
    fp64_ms, fp64_c = [], 0
    for _ in range(2):
        flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st64, _ = run_step_device(torch, dse, w, Xd, yd, k, D, stream, dse.PREC_FP64, timing=None)
        e1.record()
        torch.cuda.synchronize()
        fp64_ms.append(e0.elapsed_time(e1))
        fp64_c += count_step_evals(st64, N)[0]
    fp64_value = fp64_c / (sum(fp64_ms) * 1e-3)

    # end to end through the public API with host buffers
    e2e_ms, e2e_c = [], 0
    for _ in range(3):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        st_h, h2d, d2h = run_step_host(dse, w, k, D)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e_c += count_step_evals(st_h, N)[0]
    e2e_value = e2e_c / (sum(e2e_ms) * 1e-3)

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        oracle.build()
        dt, c, _ = cpu_oracle_step(w, k, D)
        cpu = {"value": c / dt, "unit": "candidates/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "one full step of the same workload (space build + 3 screens + refits), "
                         f"{dt:.1f} s"}
    line = {
        "metric": METRIC, "value": value, "unit": "candidates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
        "evals_per_s": evals_per_s,
        "fp64_plain": {"value": fp64_value, "unit": "candidates/s", "ms_per_step": sum(fp64_ms) / len(fp64_ms),
                       "speedup_of_fp32_path": value / world / fp64_value},
        "roofline": roofline,
        "kernel_group_ms_per_step": {"stored_unary": group_ms[0], "pair_mul": group_ms[1], "pair_add": group_ms[2],
                                     "select": group_ms[3], "source": "one untimed step with an event per group"},
        "per_screen": {key: sum(s[key] for st in all_stats for s in st) / max(1, sum(len(st) for st in all_stats))
                       for key in ("evaluated", "buffered", "escalated", "rescored", "reruns", "kernel_launches")},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "candidates/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
