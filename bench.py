#!/usr/bin/env python3
"""Benchmark of the stage-1 ANLS sweep on GB300.

Headline workload: synthetic PDF-like data, n = 3000 rows, m = 2000 time
columns, k = 4, 1e-3 relative noise.  A step is one whole run of the
mixed-precision form (FP32 M; FP32 sweeps, then chunks of a compensated
sweep and incremental sweeps; FP64 NNLS, Grams and KKT) from the U[0,1]
start until the relative KKT error is <= 1e-8; the value is seconds per run
(lower is better).  L2 is flushed (256 MB write) before every timed run.

Also reported: the plain FP64 form's time to the same target, the converged
runs against the oracle's own run from the same start, per-pass device times
and the incremental M pass's bandwidth against the measured HBM peak, single
sweeps of every pass, an end-to-end figure through the C ABI with host
buffers, the rank-16 tensor-core pass at n = 8192, m = 16384, the batched and
serving forms, and the CPU oracle timed on the host cores (one core and all).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank solves its own problem (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to rel. KKT 1e-8 (s); ANLS sweeps/s; HBM GB/s — mixed vs FP64 on 1 GB300"
N_ROWS, M_COLS, RANK_K, NOISE = 3000, 2000, 4, 1e-3
FLUSH_BYTES = 256 << 20
PRECOND = 400     # sweeps from the U[0,1] start before timing: steady-state sweeps are timed
WORKLOAD = ("PDF-like streaming NMF n=3000 m=2000 k=4 (1e-3 rel. noise): the mixed form from the U[0,1] start "
            "to relative KKT 1e-8")
YPASS_SOURCES = ["paper_2101_08431_gb300/csrc/nmf_sweep.cuh", "paper_2101_08431_gb300/csrc/nmf_nnls.cuh",
                 "paper_2101_08431_gb300/csrc/nmf_common.cuh", "paper_2101_08431_gb300/csrc/nmf_arith.cuh"]
TRAFFIC_FILES = {"f32": "profiles/ypass_f32_n3000_m2000_k4.md", "inc": "profiles/ypass_inc_n3000_m2000_k4.md"}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def kernel_hash():
    h = hashlib.sha256()
    for f in YPASS_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(which):
    """DRAM bytes per M-pass launch from the committed ncu summary, if it was
    taken on the current kernel source (else null)."""
    path = os.path.join(ROOT, TRAFFIC_FILES[which])
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    mh = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    mb = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not mh or not mb or mh.group(1) != kernel_hash():
        return None
    return float(mb.group(1))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) > 8 for i in range(4)
                          if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def make_data(seed):
    import synth
    M, _, _ = synth.pdf_like(N_ROWS, M_COLS, RANK_K, noise=NOISE, relative=True, seed=seed)
    X0, Y0 = synth.init_factors(N_ROWS, M_COLS, RANK_K, seed=seed)
    return np.asfortranarray(M.astype(np.float32)), np.asfortranarray(M), X0, Y0


def cpu_sweep_rate(M64, X0, Y0, budget_s=12.0, min_sweeps=3):
    """The oracle as it stands, single-threaded, on a bounded sample: whole
    sweeps of the same problem until budget_s has elapsed."""
    import oracle
    oracle.build()
    X, Y = X0, Y0
    t0 = time.perf_counter()
    n = 0
    while n < min_sweeps or time.perf_counter() - t0 < budget_s:
        X, Y, _, _, st = oracle.sweep(M64, X, Y)
        n += 1
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def oracle_reference_run():
    """The oracle's own run of the workload to relative KKT 1e-8 from the
    same start, stored by tests/golden/make_cfg2_reference.py (its sweep
    count scales the oracle's per-sweep time to a time to the target)."""
    path = os.path.join(ROOT, "tests", "golden", "cfg2_oracle_run.json")
    try:
        return json.load(open(path))
    except Exception:
        return None


def cpu_time_to_target(M64, X0, Y0, budget_s, openmp=False):
    """The oracle as it stands on the host cores: whole sweeps of the
    workload from the U[0,1] start until budget_s has elapsed, scaled by the
    number of sweeps the oracle needs to reach relative KKT 1e-8 from that
    start (its stored reference run).  Returns (seconds to the target,
    seconds per sweep, sweeps timed, threads, sweeps to the target)."""
    import oracle
    oracle.build(openmp=openmp)
    ref = oracle_reference_run()
    need = ref["sweeps"] if ref else None
    X, Y = X0, Y0
    oracle.sweep(M64, X, Y, openmp=openmp)            # warm (thread pool, caches)
    t0 = time.perf_counter()
    n = 0
    while n < 3 or time.perf_counter() - t0 < budget_s:
        X, Y, _, _, _ = oracle.sweep(M64, X, Y, openmp=openmp)
        n += 1
    per = (time.perf_counter() - t0) / n
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)) if openmp else 1
    return (per * need if need else None), per, n, threads, need


def run_reference(args):
    """The reference arm: the oracle on the host cores, same workload, metric
    and direction; each step is one oracle sweep of the workload (a bounded
    sample), and the value scales the mean sweep time by the sweeps the
    oracle needs to reach the target from the same start."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    _, M64, X0, Y0 = make_data(0)
    import oracle
    oracle.build()
    ref = oracle_reference_run()
    X, Y = X0, Y0
    for _ in range(args.warmup):
        X, Y, _, _, _ = oracle.sweep(M64, X, Y)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        X, Y, _, _, _ = oracle.sweep(M64, X, Y)
    dt = time.perf_counter() - t0
    per = dt / args.steps
    need = ref["sweeps"] if ref else None
    v = per * need if need else None
    sample = ("%d oracle sweeps of the workload (after %d untimed), %.1f ms each, times the %s sweeps the "
              "oracle needs from the same start to relative KKT 1e-8" % (args.steps, args.warmup, 1e3 * per, need))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * per,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": N_ROWS, "m": M_COLS, "k": RANK_K},
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2101_08431_gb300 import NMF_PREC_FP64, NMF_PREC_MIXED, StreamingNMF, build

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)          # a real stream handle (the default stream is 0)
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    M32, M64, X0, Y0 = make_data(rank)
    flush_buf = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def flush():
        flush_buf.fill_(1.0)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def timed_sweeps(h, steps, warmup, precond=0):
        """steps single sweeps, L2 flushed before each; CUDA events."""
        if precond:
            h.sweep(precond, want_stats=False)
        for _ in range(warmup):
            flush()
            h.sweep(1, want_stats=False)
        h.set_timing(True)
        l0 = h.launches
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        for e0, e1 in ev:
            flush()
            e0.record(stream)
            h.sweep(1, want_stats=False)
            e1.record(stream)
        barrier()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
        launches = h.launches - l0
        tm = h.get_timing()
        h.set_timing(False)
        return ms, launches, tm

    def run_to_target(h, X, Y, timing=False):
        """One run from (X, Y) to relative KKT 1e-8: L2 flushed, then
        nmf_sweep(0) between CUDA events on the handle's stream."""
        h.set_factors(X, Y)
        h.set_pass_mode(-1)
        if timing:
            h.set_timing(True)
        flush()
        barrier()
        l0 = h.launches
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        st = h.sweep(0, allow_notconv=True)
        e1.record(stream)
        barrier()
        wall = time.perf_counter() - t0
        return {"seconds": e0.elapsed_time(e1) / 1e3, "wall_s": wall, "sweeps": st["sweeps"],
                "fp64_sweeps": st["fp64_sweeps"], "kkt_rel": st["kkt_rel"], "converged": bool(st["converged"]),
                "f": st["f"], "launches": h.launches - l0}

    out = {}
    peak, peak_kind = peaks()
    hm = StreamingNMF(N_ROWS, RANK_K, M_COLS, prec=NMF_PREC_MIXED, kkt_target=1e-8, max_sweeps=60000,
                      stream=sptr)
    hm.append_columns(M32)
    hf = StreamingNMF(N_ROWS, RANK_K, M_COLS, prec=NMF_PREC_FP64, kkt_target=1e-8, max_sweeps=60000,
                      stream=sptr)
    hf.append_columns(M64)
    # ---- the headline: mixed form, seconds to relative KKT 1e-8 from the U[0,1] start
    for _ in range(args.warmup):
        run_to_target(hm, X0, Y0)
    runs = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            runs.append(run_to_target(hm, X0, Y0))
    secs = max_over_ranks(sum(r["seconds"] for r in runs) / len(runs))
    out["value"] = secs
    out["ms_per_step"] = 1e3 * secs
    out["gpu_launches"] = sum(r["launches"] for r in runs)
    out["clocks"] = clk.summary()
    last = runs[-1]
    # ---- per-pass device times inside one more run (events around every sweep's two kernels)
    tr = run_to_target(hm, X0, Y0, timing=True)
    passes = {}
    for name in ("f32", "df", "inc"):
        t = hm.get_pass_timing(name)
        if t["sweeps"]:
            passes[name] = {"sweeps": t["sweeps"], "ypass_avg_ms": t["ypass_ms"] / t["sweeps"],
                            "xpass_avg_ms": t["xpass_ms"] / t["sweeps"]}
    hm.set_timing(False)
    # the dominant kernel of the run: the incremental M pass (most sweeps)
    alg_inc = N_ROWS * M_COLS * 4 + 4 * M_COLS * RANK_K * 8 + N_ROWS * RANK_K * 4
    inc = passes.get("inc", {})
    y_inc = inc.get("ypass_avg_ms")
    out["roofline"] = {"bound": "hbm", "achieved": (alg_inc / (y_inc / 1e3) / 1e9) if y_inc else None,
                       "peak": peak, "unit": "GB/s",
                       "frac": (alg_inc / (y_inc / 1e3) / 1e9 / peak) if y_inc else None,
                       "traffic": measured_traffic("inc"), "peak_kind": peak_kind,
                       "kernel": "ypass_kernel<float, ArInc, 4> (incremental M pass)",
                       "alg_bytes_per_launch": alg_inc, "avg_launch_ms": y_inc,
                       "where": "inside a run to the target: M (24 MB) stays in L2 between sweeps",
                       "per_pass": passes, "timed_run_sweeps": tr["sweeps"]}
    out["time_to_kkt"] = {"mixed": {"runs": len(runs), "seconds_mean": secs,
                                    "seconds_min": min(r["seconds"] for r in runs),
                                    "sweeps": last["sweeps"], "refinement_sweeps": last["fp64_sweeps"],
                                    "kkt_rel": last["kkt_rel"], "f": last["f"], "converged": last["converged"]}}
    # ---- the plain FP64 form beside it
    fr = [run_to_target(hf, X0, Y0) for _ in range(max(1, min(3, args.steps)))]
    out["time_to_kkt"]["fp64"] = {"runs": len(fr), "seconds_mean": sum(r["seconds"] for r in fr) / len(fr),
                                  "sweeps": fr[-1]["sweeps"], "kkt_rel": fr[-1]["kkt_rel"], "f": fr[-1]["f"],
                                  "converged": fr[-1]["converged"]}
    out["time_to_kkt"]["fp64_over_mixed"] = out["time_to_kkt"]["fp64"]["seconds_mean"] / secs
    # agreement of the two converged runs with the oracle's own run from the same start
    ref = oracle_reference_run()
    if ref:
        Xm, Ym, xmm, ymm = hm.get_factors()
        Xq, Yq, xmq, ymq = hf.get_factors()
        out["time_to_kkt"]["oracle_run"] = {
            "sweeps": ref["sweeps"], "f": ref["f"],
            "mixed_f_rel_diff": abs(last["f"] - ref["f"]) / ref["f"],
            "fp64_f_rel_diff": abs(fr[-1]["f"] - ref["f"]) / ref["f"],
            "mixed_mask_differences": int(mask_differences(ymm, xmm, ref)),
            "fp64_mask_differences": int(mask_differences(ymq, xmq, ref))}
    # ---- single sweeps of each pass in steady state, L2 flushed before each
    hm.set_factors(X0, Y0)
    hm.sweep(PRECOND, want_stats=False)
    alg32 = N_ROWS * M_COLS * 4 + 2 * M_COLS * RANK_K * 8 + N_ROWS * RANK_K * 4
    out["pass_sweeps"] = {}
    for mode, name, alg in ((0, "fp32", alg32), (3, "incremental_chunk", alg_inc), (2, "compensated", alg32)):
        hm.set_pass_mode(mode)
        nr = max(10, args.steps)
        if mode == 3:
            # a chunk of 32 sweeps (1 compensated + 31 incremental) per step
            hm.sweep(64, want_stats=False)
            hm.set_timing(True)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(max(2, nr // 8)):
                flush()
                hm.sweep(32, want_stats=False)
            e1.record(stream)
            barrier()
            nsw = 32 * max(2, nr // 8)
            ms_r = e0.elapsed_time(e1)
            ti = hm.get_pass_timing("inc")
            hm.set_timing(False)
            yr = ti["ypass_ms"] / max(ti["sweeps"], 1)
            out["pass_sweeps"][name] = {"sweeps_per_s": world * nsw / (max_over_ranks(ms_r) / 1e3),
                                        "inc_ypass_avg_ms": yr, "inc_xpass_avg_ms": ti["xpass_ms"] / max(ti["sweeps"], 1),
                                        "inc_ypass_gbs": alg / (yr / 1e3) / 1e9,
                                        "l2": "flushed before every chunk of 32 sweeps"}
            continue
        ms_r, launches, tm_r = timed_sweeps(hm, nr, 3)
        yr = tm_r["ypass_ms"] / max(tm_r["ypass_launches"], 1)
        xr = tm_r["xpass_ms"] / max(tm_r["xpass_launches"], 1)
        gbs = alg / (yr / 1e3) / 1e9
        out["pass_sweeps"][name] = {"sweeps_per_s": world * nr / (max_over_ranks(ms_r) / 1e3), "ypass_avg_ms": yr,
                                    "xpass_avg_ms": xr, "ypass_gbs": gbs, "ypass_hbm_frac": gbs / peak,
                                    "l2": "flushed before every sweep"}
        if mode == 0:
            out["pass_sweeps"][name]["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                                    "frac": gbs / peak, "traffic": measured_traffic("f32"),
                                                    "alg_bytes_per_launch": alg}
    hf.set_factors(X0, Y0)
    hf.sweep(PRECOND, want_stats=False)
    nf = max(10, args.steps // 2)
    ms_f, _, tm_f = timed_sweeps(hf, nf, 3)
    yf = tm_f["ypass_ms"] / max(tm_f["ypass_launches"], 1)
    fbytes = N_ROWS * M_COLS * 8 + 2 * M_COLS * RANK_K * 8 + N_ROWS * RANK_K * 8
    # the FP64 form's M pass against the measured FP64 FMA rate (4 n m k flops:
    # the two contractions; an ALU roofline, the same kernel's HBM bytes beside)
    from paper_2101_08431_gb300 import measure_fma_peaks
    alu = measure_fma_peaks(sptr)
    out["alu_peaks"] = dict(alu, how="independent FMA chains on every SM, CUDA events (nmf_measure_fma_peaks)")
    f64_tfl = 4.0 * N_ROWS * M_COLS * RANK_K / (yf / 1e3) / 1e12
    out["pass_sweeps"]["fp64_form"] = {"sweeps_per_s": world * nf / (max_over_ranks(ms_f) / 1e3), "ypass_avg_ms": yf,
                                       "xpass_avg_ms": tm_f["xpass_ms"] / max(tm_f["xpass_launches"], 1),
                                       "ypass_gbs": fbytes / (yf / 1e3) / 1e9,
                                       "ypass_fp64_tflops": f64_tfl,
                                       "roofline": {"bound": "alu", "achieved": f64_tfl, "peak": alu["fp64_tflops"],
                                                    "unit": "TFLOP/s", "frac": f64_tfl / alu["fp64_tflops"],
                                                    "traffic": None, "peak_kind": "measured FP64 FMA rate"}}
    # ---- end to end through the C ABI with host buffers: every step copies M
    # (pinned), X0 and Y0 in, runs to the target, and copies X, Y and the
    # passive sets out
    pinned = torch.empty((M_COLS, N_ROWS), dtype=torch.float32, pin_memory=True)
    pinned.numpy()[:] = M32.T
    pin_view = pinned.t()            # n x m, column-major view for the ABI
    he = StreamingNMF(N_ROWS, RANK_K, M_COLS, prec=NMF_PREC_MIXED, kkt_target=1e-8, max_sweeps=60000,
                      stream=sptr)
    ne = max(2, min(5, args.steps))

    def e2e_step():
        he.append_columns(pin_view)
        he.set_factors(X0, Y0)
        st = he.sweep(0)
        return he.get_factors(), st

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(ne):
        (Xe, Ye, xme, yme), st = e2e_step()
    barrier()
    dt_e = max_over_ranks(time.perf_counter() - t0)
    he.close()
    out["e2e"] = {"value": dt_e / ne, "unit": "s",
                  "h2d_bytes_per_step": N_ROWS * M_COLS * 4 + (N_ROWS + M_COLS) * RANK_K * 8,
                  "d2h_bytes_per_step": (N_ROWS + M_COLS) * (RANK_K * 8 + 4),
                  "step": "append all m columns from pinned host memory, set the U[0,1] factors from host "
                          "memory, run to relative KKT 1e-8, copy X, Y and the passive sets to the host",
                  "sweeps": st["sweeps"], "kkt_rel": st["kkt_rel"]}
    hm.close()
    hf.close()
    # ---- mixed precision at scale: rank 16 on the tensor cores
    if not args.skip_k16:
        out["rank16"] = rank16_leg(args, sptr, barrier)
    # ---- batched persistent form: 256 uneven problems
    if not args.skip_batch:
        out["batched"] = batched_leg(args, rank, sptr, barrier, max_over_ranks, world)
        if not args.skip_batch_ttk and world == 1:
            out["batched"]["time_to_kkt_subset"] = batched_ttk_leg(args, sptr)
    # ---- the paper's chain warm start against the parallel one
    if not args.skip_paper and rank == 0:
        out["chain_warm_start"] = chain_leg(args, sptr)
    # ---- the paper's experiment shapes, to its absolute stopping rule
    if not args.skip_paper and rank == 0:
        out["paper_shapes"] = paper_shapes_leg(args, sptr)
    # ---- streaming serving: 32 streams, Poisson chunk arrivals
    if not args.skip_serve:
        out["serving"] = serving_leg(args, rank, sptr)
    # ---- CPU baseline (rank 0 at N = 1 only): the oracle on one core and,
    # its -fopenmp build, on all host cores
    if rank == 0 and world == 1 and not args.skip_cpu:
        v1, per1, n1, _, need = cpu_time_to_target(M64, X0, Y0, 10.0)
        vN, perN, nN, thr, _ = cpu_time_to_target(M64, X0, Y0, 6.0, openmp=True)
        out["cpu_baseline"] = {"value": v1, "unit": "s", "cores": 1, "kind": "oracle",
                               "host_nproc": os.cpu_count(),
                               "sample": "%d oracle sweeps of the workload from the U[0,1] start, %.1f ms each, "
                                         "times the %s sweeps the oracle needs from that start to relative KKT 1e-8"
                                         % (n1, 1e3 * per1, need),
                               "all_cores": {"value": vN, "unit": "s", "cores": thr, "kind": "oracle (-fopenmp)",
                                             "sample": "%d sweeps, %.1f ms each" % (nN, 1e3 * perN)}}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": out["value"], "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["ms_per_step"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N_ROWS, "m": M_COLS, "k": RANK_K,
                       "step": "one run of the mixed form from the U[0,1] start to relative KKT 1e-8",
                       "l2": "flushed (256 MB write) before every timed run; M (24 MB) stays in L2 within a run",
                       "parallelism": "independent problem per GPU" if world > 1 else "single GPU"}}
    for key in ("roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks", "time_to_kkt", "pass_sweeps",
                "alu_peaks", "rank16", "batched", "chain_warm_start", "paper_shapes", "serving"):
        if key in out:
            line[key] = out[key]
    print(json.dumps(line), flush=True)
    return 0


def mask_differences(ym, xm, ref):
    """Passive-set entries that differ from the oracle run's (stored as hex)."""
    ymo = np.array([int(v, 16) for v in ref["ymask_hex"]], dtype=np.uint64)
    xmo = np.array([int(v, 16) for v in ref["xmask_hex"]], dtype=np.uint64)
    d = np.bitwise_xor(ym.astype(np.uint64), ymo)
    e = np.bitwise_xor(xm.astype(np.uint64), xmo)
    return sum(bin(int(v)).count("1") for v in d) + sum(bin(int(v)).count("1") for v in e)


K16_N, K16_M, K16_K, K16_NOISE, K16_PRECOND = 8192, 16384, 16, 1e-4, 30
K16_CAP = 100000


def rank16_leg(args, sptr, barrier):
    """Mixed precision at scale: n=8192, m=16384, k=16, FP32 M (512 MB, > L2,
    so no flush between timed sweeps), the FP32-class pass on the tensor
    cores (split-BF16 contractions, FP32 column and row solves, FP64 Grams
    and KKT terms).  Timed after K16_PRECOND
    sweeps from the U[0,1] start.  Reports sweeps/s, the M pass's HBM GB/s
    against the measured peak and its issued MMA TFLOP/s.  (The error of this
    pass against the FP64 oracle, on sampled columns and rows of the same
    workload, is checked by the test suite.)"""
    import torch
    import synth
    from paper_2101_08431_gb300 import NMF_PREC_MIXED, StreamingNMF
    n, m, k = K16_N, K16_M, K16_K
    M, _, _ = synth.pdf_like(n, m, k, noise=K16_NOISE, relative=True, seed=11)
    M32 = np.asfortranarray(M.astype(np.float32))
    del M
    X0, Y0 = synth.init_factors(n, m, k, seed=11)
    stream = torch.cuda.current_stream()
    h = StreamingNMF(n, k, m, prec=NMF_PREC_MIXED, kkt_target=0.0, stream=sptr)
    h.append_columns(M32)
    h.set_factors(X0, Y0)
    h.set_pass_mode(0)
    h.sweep(K16_PRECOND, want_stats=False)
    steps = max(10, args.steps // 10)
    for _ in range(3):
        h.sweep(1, want_stats=False)
    h.set_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier()
    for e0, e1 in ev:
        e0.record(stream)
        h.sweep(1, want_stats=False)
        e1.record(stream)
    barrier()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    tm = h.get_timing()
    h.set_timing(False)
    y_ms = tm["ypass_ms"] / max(tm["ypass_launches"], 1)
    x_ms = tm["xpass_ms"] / max(tm["xpass_launches"], 1)
    alg = n * m * 4 + 2 * m * k * 8 + n * k * 8
    mma_flops = n * m * 256.0      # issued: per element of M, 2 x 128x32x16 MMAs per 128x16 block in each GEMM
    peak, peak_kind = peaks()
    kk = h.objective_kkt()
    h.close()
    ttk = None if args.skip_k16_ttk else rank16_to_target(M32, X0, Y0, sptr, barrier)
    return {"workload": "PDF-like n=8192 m=16384 k=16 (1e-4 rel. noise), FP32 M (512 MB), tensor-core "
                        "FP32-class pass (split-BF16 tcgen05 contractions: B-GEMM and P-GEMM launches with the "
                        "column solves between them; FP32 column solves, FP64-checked row solves)",
            "time_to_kkt": ttk,
            "state": "timed sweeps follow %d sweeps from the U[0,1] start" % K16_PRECOND,
            "l2": "inputs larger than L2 (no flush)",
            "sweeps_per_s": steps / (ms / 1e3), "ms_per_sweep": ms / steps,
            "ypass_avg_ms": y_ms, "xpass_avg_ms": x_ms,
            "ypass_hbm_gbs": alg / (y_ms / 1e3) / 1e9, "ypass_hbm_frac": alg / (y_ms / 1e3) / 1e9 / peak,
            "peak_gbs": peak, "peak_kind": peak_kind, "alg_bytes_per_launch": alg,
            "ypass_mma_tflops_issued": mma_flops / (y_ms / 1e3) / 1e12,
            "columns_per_s": m * steps / (ms / 1e3),
            "kkt_rel_after": kk["kkt_rel"], "f_after": kk["f"]}


def rank16_to_target(M32, X0, Y0, sptr, barrier):
    """The mixed form at n=8192, m=16384, k=16 from the U[0,1] start to
    relative KKT 1e-8: tensor-core passes, then chunks of a compensated
    reference sweep and incremental sweeps; one run timed with CUDA events on
    the library's stream, the returned iterate certified by the oracle's KKT
    (FP64, the whole matrix)."""
    import torch
    import oracle
    from paper_2101_08431_gb300 import NMF_PREC_MIXED, StreamingNMF
    n, m, k = K16_N, K16_M, K16_K
    stream = torch.cuda.current_stream()
    h = StreamingNMF(n, k, m, prec=NMF_PREC_MIXED, kkt_target=1e-8, max_sweeps=K16_CAP, stream=sptr)
    h.append_columns(M32)
    h.set_factors(X0, Y0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    st = h.sweep(0, allow_notconv=True)
    e1.record(stream)
    barrier()
    secs = e0.elapsed_time(e1) / 1e3
    Xg, Yg, _, _ = h.get_factors()
    h.close()
    # the refinement's passes near convergence: 64 sweeps of pass mode 3
    # (chunks of a reference sweep and incremental sweeps) from the returned
    # iterate, with per-pass events, on a handle without a stopping target
    h = StreamingNMF(n, k, m, prec=NMF_PREC_MIXED, kkt_target=0.0, stream=sptr)
    h.append_columns(M32)
    h.set_factors(Xg, Yg)
    h.set_pass_mode(3)
    h.set_timing(True)
    h.sweep(64, want_stats=False)
    passes = {}
    for name in ("df", "inc"):
        t = h.get_pass_timing(name)
        if t["sweeps"]:
            passes[name] = {"sweeps": t["sweeps"], "ypass_avg_ms": t["ypass_ms"] / t["sweeps"],
                            "xpass_avg_ms": t["xpass_ms"] / t["sweeps"]}
    h.set_timing(False)
    h.close()
    kk = oracle.kkt(M32.astype(np.float64), Xg, Yg)
    return {"seconds": secs, "sweeps": st["sweeps"], "refinement_sweeps": st["fp64_sweeps"],
            "converged": bool(st["converged"]), "kkt_rel": st["kkt_rel"], "sweep_cap": K16_CAP,
            "oracle": {"kkt_rel": kk["rel"], "f": kk["f"], "note": "oracle_kkt of the returned iterate, FP64"},
            "refinement_passes_near_convergence": passes}


# The paper's synthetic experiments (Sec. 5.4: X, Y ~ U[0,1], M = XY + N(0, 0.1^2),
# negatives set to 0) and the AgMOR shape of Sec. 5.2 (PDF-like stand-in), with
# the paper's 2-STAGE MATLAB times (mean of 10 starts, one 2.7 GHz CPU core,
# stopping at E <= 1e-6) as context
PAPER_SHAPES = [("AgMOR shape, PDF-like stand-in", 3000, 36, 3, "pdf", 5.03, 30000)] + \
    [("Sec. 5.4 uniform", 2000, 50, k, "uniform", t, 300000) for k, t in ((3, 3.31), (4, 7.41), (5, 6.98), (6, 14.46))] + \
    [("Sec. 5.4 uniform", 2000, 100, k, "uniform", t, 300000) for k, t in ((3, 4.05), (4, 7.46), (5, 11.77), (6, 25.54))]


def paper_shapes_leg(args, sptr):
    """Time to the paper's stopping rule, absolute KKT error E <= 1e-6
    (Sec. 5.1), from the U[0,1] start (seed 0) on the paper's experiment
    shapes: the plain FP64 form and the mixed form on the GPU, and the oracle
    on one host core -- its time per sweep, measured on a short sample,
    times the sweeps the FP64 form needed (the same iteration in the same
    arithmetic).  Stage 1 only: the paper's times include its stage-2 interior
    point method."""
    import torch
    import synth
    import oracle
    from paper_2101_08431_gb300 import NMF_PREC_FP64, NMF_PREC_MIXED, StreamingNMF
    oracle.build()
    stream = torch.cuda.current_stream()
    rows = []
    for name, n, m, k, kind, paper_s, cap in PAPER_SHAPES:
        if kind == "uniform":
            M, _, _ = synth.paper_uniform(n, m, k, sigma=0.1, seed=0)
        else:
            M, _, _ = synth.pdf_like(n, m, k, noise=1e-3, relative=True, seed=0)
        X0, Y0 = synth.init_factors(n, m, k, seed=0)
        row = {"workload": name, "n": n, "m": m, "k": k, "paper_2stage_matlab_s": paper_s, "sweep_cap": cap}
        for prec, label in ((NMF_PREC_FP64, "fp64"), (NMF_PREC_MIXED, "mixed")):
            h = StreamingNMF(n, k, m, prec=prec, kkt_target=0.0, kkt_abs_target=1e-6, max_sweeps=cap,
                             stream=sptr)
            h.append_columns(np.asfortranarray(M if prec == NMF_PREC_FP64 else M.astype(np.float32)))
            h.set_factors(X0, Y0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = h.sweep(0, allow_notconv=True)
            e1.record(stream)
            torch.cuda.synchronize()
            row[label] = {"seconds": e0.elapsed_time(e1) / 1e3, "sweeps": st["sweeps"],
                          "converged": st["converged"] == 1, "E_abs": st["kkt_abs"], "f": st["f"]}
            h.close()
        X, Y = X0, Y0
        t0 = time.perf_counter()
        nsw = 0
        while nsw < 3 or time.perf_counter() - t0 < 0.3:
            X, Y, _, _, _ = oracle.sweep(M, X, Y)
            nsw += 1
        per = (time.perf_counter() - t0) / nsw
        row["oracle_1core"] = {"seconds_per_sweep": per, "seconds": per * row["fp64"]["sweeps"],
                               "sample": "%d oracle sweeps timed, times the FP64 form's sweep count" % nsw}
        rows.append(row)
    return {"rule": "absolute KKT error E <= 1e-6 (Sec. 5.1), stage 1 (ANLS) only, U[0,1] start of seed 0",
            "note": "E is absolute: the PDF-like stand-in is on another scale than the AgMOR data, and stage 1 "
                    "alone does not bring it to 1e-6 within its cap",
            "runs": rows}


def chain_leg(args, sptr):
    """Sec. 2's chain warm start (column j from column j - 1's new solution,
    one column after another) against the parallel warm start (every column
    from its own previous-sweep solution at once), FP64 form, PDF-like data
    (1e-3 relative noise) after 200 sweeps: device time per sweep and the
    column solves' entering steps per sweep, at a small and at the benchmark
    number of columns."""
    import torch
    import synth
    from paper_2101_08431_gb300 import NMF_PREC_FP64, NMF_WARM_CHAIN, NMF_WARM_PREV, StreamingNMF
    stream = torch.cuda.current_stream()
    res = []
    for n, m, k in ((3000, 64, 4), (3000, 2000, 4)):
        M, _, _ = synth.pdf_like(n, m, k, noise=NOISE, relative=True, seed=5)
        X0, Y0 = synth.init_factors(n, m, k, seed=5)
        row = {"n": n, "m": m, "k": k}
        for ws, name in ((NMF_WARM_PREV, "parallel"), (NMF_WARM_CHAIN, "chain")):
            h = StreamingNMF(n, k, m, prec=NMF_PREC_FP64, kkt_target=0.0, warm_start=ws, stream=sptr)
            h.append_columns(np.asfortranarray(M))
            h.set_factors(X0, Y0)
            h.sweep(200, want_stats=False)
            steps = [h.sweep(1)["entering_steps"] for _ in range(8)]
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.sweep(64, want_stats=False)
            e1.record(stream)
            torch.cuda.synchronize()
            row[name] = {"ms_per_sweep": e0.elapsed_time(e1) / 64, "entering_steps_per_sweep": float(np.mean(steps))}
            h.close()
        res.append(row)
    return res


BATCH_NPROB = 256


def batched_leg(args, rank, sptr, barrier, max_over_ranks, world):
    """256 independent PDF-like problems, n ~ U[500, 4000], m ~ U[100, 2000],
    k ~ U{2..8} (problem p seeded 1000 + p), FP32 M, swept by the batched
    persistent launches.  M totals ~2.5 GB (> L2), so no flush is needed
    between timed sweeps.  Reports batch sweeps/s and columns/s of the FP32
    and compensated passes with the autotuned schedule, and the M pass's
    HBM bytes against the measured peak; with --batch-ttk also the time for
    every problem to reach relative KKT 1e-8."""
    import torch
    import synth
    from paper_2101_08431_gb300 import StreamingNMFBatch
    shapes = synth.batch_problem_shapes(BATCH_NPROB, seed0=1000 + 100000 * rank)
    t0 = time.perf_counter()
    b = StreamingNMFBatch([(n, k, m) for n, m, k, _ in shapes], kkt_target=1e-8, max_sweeps=40000, stream=sptr)
    for j, (n, m, k, seed) in enumerate(shapes):
        M, _, _ = synth.pdf_like(n, m, k, noise=NOISE, relative=True, seed=seed)
        X, Y = synth.init_factors(n, m, k, seed=seed)
        b.append_columns(j, np.asfortranarray(M, dtype=np.float32))
        b.set_factors(j, X, Y)
    setup_s = time.perf_counter() - t0
    mbytes = sum(n * m * 4 for n, m, k, _ in shapes)
    fbytes = sum(2 * m * k * 8 + n * k * 4 for n, m, k, _ in shapes)
    cols = sum(m for n, m, k, _ in shapes)
    tune = b.autotune(trial_sweeps=2)
    res = {"workload": "%d PDF-like problems, n~U[500,4000], m~U[100,2000], k~U{2..8}, FP32 M (%.2f GB), "
                       "FP64 solve" % (BATCH_NPROB, mbytes / 1e9),
           "setup_s": setup_s, "autotune": tune, "l2": "inputs larger than L2 (no flush)"}
    peak, peak_kind = peaks()
    for mode, name in ((0, "fp32_pass"), (2, "compensated_pass")):
        b.set_pass_mode(mode)
        b.sweep(3)
        nb = 16
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = b.launches
        e0.record(torch.cuda.current_stream())
        stats, nrun = b.sweep(nb)
        e1.record(torch.cuda.current_stream())
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1))
        per = ms / nrun
        gbs = (mbytes + fbytes) / (per / 1e3) / 1e9
        res[name] = {"batch_sweeps_per_s": world * nrun / (ms / 1e3), "ms_per_batch_sweep": per,
                     "columns_per_s": world * cols * nrun / (ms / 1e3), "gpu_launches": b.launches - l0,
                     "hbm_gbs": gbs, "hbm_frac": gbs / peak, "peak_kind": peak_kind}
    if args.batch_ttk:
        b.set_pass_mode(-1)
        for j, (n, m, k, seed) in enumerate(shapes):
            X, Y = synth.init_factors(n, m, k, seed=seed)
            b.set_factors(j, X, Y)
        barrier()
        t1 = time.perf_counter()
        stats, nrun = b.sweep(0, allow_notconv=True)
        barrier()
        rels = [s["kkt_rel"] for s in stats]
        res["time_to_kkt"] = {"seconds": time.perf_counter() - t1, "batch_sweeps": nrun,
                              "converged": sum(1 for s in stats if s["converged"] == 1),
                              "max_kkt_rel": max(rels), "max_sweeps_of_a_problem": max(s["sweeps"] for s in stats)}
    b.close()
    return res


BTTK_N, BTTK_MAX = 8, 30000


def batched_ttk_leg(args, sptr):
    """Time to relative KKT 1e-8 from the U[0,1] start for the first BTTK_N
    problems of the batched workload: the mixed-precision batched form (one
    batch, device-driven FP32 -> compensated schedule) against the plain FP64
    GPU form (one FP64 handle per problem, each on its own stream, driven
    concurrently from host threads).  Wall time of each whole run."""
    import threading
    import torch
    import synth
    from paper_2101_08431_gb300 import NMF_PREC_FP64, StreamingNMF, StreamingNMFBatch
    shapes = synth.batch_problem_shapes(BATCH_NPROB)[:BTTK_N]
    data = []
    for n, m, k, seed in shapes:
        M, _, _ = synth.pdf_like(n, m, k, noise=NOISE, relative=True, seed=seed)
        X, Y = synth.init_factors(n, m, k, seed=seed)
        data.append((np.asfortranarray(M, dtype=np.float32), X, Y))
    b = StreamingNMFBatch([(n, k, m) for n, m, k, _ in shapes], kkt_target=1e-8, max_sweeps=BTTK_MAX, stream=sptr)
    for j, (M32, X, Y) in enumerate(data):
        b.append_columns(j, M32)
        b.set_factors(j, X, Y)
    b.set_pass_mode(-1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stats, nrun = b.sweep(0, allow_notconv=True)
    torch.cuda.synchronize()
    t_mixed = time.perf_counter() - t0
    b.close()
    streams = [torch.cuda.Stream() for _ in shapes]
    hs = []
    for (n, m, k, _), (M32, X, Y), s in zip(shapes, data, streams):
        h = StreamingNMF(n, k, m, prec=NMF_PREC_FP64, kkt_target=1e-8, max_sweeps=BTTK_MAX, stream=s.cuda_stream)
        h.append_columns(M32.astype(np.float64))
        h.set_factors(X, Y)
        hs.append(h)
    torch.cuda.synchronize()
    out = [None] * len(hs)

    def run(i):
        out[i] = hs[i].sweep(0, allow_notconv=True)

    th = [threading.Thread(target=run, args=(i,)) for i in range(len(hs))]
    t0 = time.perf_counter()
    for x in th:
        x.start()
    for x in th:
        x.join()
    torch.cuda.synchronize()
    t_fp64 = time.perf_counter() - t0
    for h in hs:
        h.close()
    fd = max(abs(s["f"] - o["f"]) / max(abs(o["f"]), 1e-300) for s, o in zip(stats, out))
    return {"problems": "the first %d problems of the batched workload, from the U[0,1] start" % BTTK_N,
            "mixed_batched": {"seconds": t_mixed, "converged": sum(1 for s in stats if s["converged"] == 1),
                              "sweeps": [s["sweeps"] for s in stats],
                              "max_kkt_rel": max(s["kkt_rel"] for s in stats)},
            "fp64_handles": {"seconds": t_fp64, "converged": sum(1 for o in out if o["converged"] == 1),
                             "sweeps": [o["sweeps"] for o in out],
                             "max_kkt_rel": max(o["kkt_rel"] for o in out)},
            "max_rel_f_difference": fd, "sweep_cap": BTTK_MAX}


SERVE_STREAMS, SERVE_N, SERVE_K, SERVE_CAP = 32, 2048, 6, 8192
SERVE_RATE, SERVE_INIT = 200.0, 256


def serving_leg(args, rank, sptr):
    """Streaming serving: 32 streams (n=2048, k=6, history capped at 8192
    resident columns), FP32 M.  Each stream first receives SERVE_INIT columns
    (solved to the target, untimed); then chunks of U{1..64} columns arrive
    with Poisson arrivals at 200 chunks/s in aggregate, each to a uniformly
    drawn stream, for serve_seconds.  Reports per-chunk latency (arrival to
    completion at relative KKT <= 1e-6), columns/s and the server's rounds."""
    import synth
    from paper_2101_08431_gb300 import StreamingServer
    g = np.random.default_rng(7 + rank)
    D = args.serve_seconds
    horizon = SERVE_INIT + int(SERVE_RATE * D * 33.0 / SERVE_STREAMS * 2.0) + 256
    data = []
    for sidx in range(SERVE_STREAMS):
        M, _, _ = synth.pdf_like(SERVE_N, horizon, SERVE_K, noise=NOISE, relative=True, seed=2000 + sidx)
        data.append(np.asfortranarray(M, dtype=np.float32))
    srv = StreamingServer(kkt_target=1e-6, max_sweeps_per_chunk=2000, sweeps_per_round=8, stream=sptr)
    ids = [srv.open_stream(SERVE_N, SERVE_K, SERVE_CAP, seed=2000 + i) for i in range(SERVE_STREAMS)]
    pos = [0] * SERVE_STREAMS
    t_init = time.perf_counter()
    pend = set()
    for i, sid in enumerate(ids):
        pend.add(srv.submit(sid, data[i][:, :SERVE_INIT]))
        pos[i] = SERVE_INIT
    while pend:
        for r in srv.poll(wait_ms=100):
            pend.discard(r["ticket"])
    init_s = time.perf_counter() - t_init
    st0 = srv.stats()
    # the timed phase: Poisson arrivals
    arrivals, t = [], 0.0
    while True:
        t += g.exponential(1.0 / SERVE_RATE)
        if t >= D:
            break
        arrivals.append((t, int(g.integers(0, SERVE_STREAMS)), int(g.integers(1, 65))))
    lat, csweeps, cols_done, pend = [], [], 0, set()
    t0 = time.perf_counter()
    k = 0
    while k < len(arrivals) or pend:
        now = time.perf_counter() - t0
        while k < len(arrivals) and arrivals[k][0] <= now:
            _, i, c = arrivals[k]
            if pos[i] + c > horizon:
                c = max(0, horizon - pos[i])
            if c:
                pend.add(srv.submit(ids[i], data[i][:, pos[i]:pos[i] + c]))
                pos[i] += c
            k += 1
        wait = 0 if k < len(arrivals) else 50
        nxt = arrivals[k][0] - (time.perf_counter() - t0) if k < len(arrivals) else 0.0
        for r in srv.poll(wait_ms=max(0, min(int(nxt * 1e3), 2)) if k < len(arrivals) else wait):
            if r["ticket"] in pend:
                pend.discard(r["ticket"])
                lat.append(r["t_done_s"] - r["t_submit_s"])
                csweeps.append(r["sweeps"])
                cols_done += r["ncols"]
        if k < len(arrivals):
            time.sleep(max(0.0, min(0.001, arrivals[k][0] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat = np.array(lat)
    rounds = st["rounds"] - st0["rounds"]
    return {"workload": "%d streams, n=%d, k=%d, history cap %d columns, FP32 M; chunks U{1..64} columns, "
                        "Poisson arrivals %.0f chunks/s for %.0f s" % (SERVE_STREAMS, SERVE_N, SERVE_K, SERVE_CAP,
                                                                      SERVE_RATE, D),
            "target": "relative KKT <= 1e-6 per chunk (2000 sweeps at most)",
            "chunks": int(len(lat)), "columns": int(cols_done), "columns_per_s": cols_done / wall,
            "latency_p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "latency_p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
            "latency_mean_ms": float(lat.mean() * 1e3) if len(lat) else None,
            "chunk_sweeps": {"p50": float(np.percentile(csweeps, 50)) if csweeps else None,
                             "p99": float(np.percentile(csweeps, 99)) if csweeps else None,
                             "max": int(max(csweeps)) if csweeps else None,
                             "at_cap": int(sum(1 for v in csweeps if v >= 2000)),
                             "note": "sweeps a stream ran between a chunk's first round and its completion"},
            "rounds": rounds, "batch_sweeps": st["batch_sweeps"] - st0["batch_sweeps"],
            "streams_per_round": (st["stream_rounds"] - st0["stream_rounds"]) / max(rounds, 1),
            "streams_admitted": st["streams_admitted"], "hbm_in_use_gb": st["hbm_in_use_bytes"] / 1e9,
            "init_s": init_s}


def run_ncu_case(args):
    """A short, fixed launch sequence for ncu captures: priming, PRECOND_NCU
    sweeps of the chosen pass, then 3 more (capture them with -s/-c).
    "batch": 16 problems of the batched workload, 3 FP32-pass sweeps in one
    plain persistent launch per class."""
    import torch
    from paper_2101_08431_gb300 import NMF_PREC_FP64, NMF_PREC_MIXED, StreamingNMF, StreamingNMFBatch, build
    build.build()
    if args.ncu_case == "batch":
        import synth
        shapes = synth.batch_problem_shapes(16)
        b = StreamingNMFBatch([(n, k, m) for n, m, k, _ in shapes], kkt_target=0.0)
        for j, (n, m, k, seed) in enumerate(shapes):
            M, _, _ = synth.pdf_like(n, m, k, noise=NOISE, relative=True, seed=seed)
            X, Y = synth.init_factors(n, m, k, seed=seed)
            b.append_columns(j, np.asfortranarray(M, dtype=np.float32))
            b.set_factors(j, X, Y)
        b.set_pass_mode(0)
        b.sweep(3)
        torch.cuda.synchronize()
        b.close()
        print("ncu case batch: 16 problems, 3 sweeps")
        return 0
    if args.ncu_case == "k16near":
        # the refinement's incremental sweeps near convergence: a mixed run to
        # relative KKT 1e-7, then a fresh handle from that iterate, pass mode 3
        import synth
        n, m, k = K16_N, 6144, K16_K
        M, _, _ = synth.pdf_like(n, m, k, noise=K16_NOISE, relative=True, seed=11)
        M32 = np.asfortranarray(M, dtype=np.float32)
        X, Y = synth.init_factors(n, m, k, seed=11)
        h = StreamingNMF(n, k, m, prec=NMF_PREC_MIXED, kkt_target=1e-7, max_sweeps=20000)
        h.append_columns(M32)
        h.set_factors(X, Y)
        h.sweep(0, want_stats=False, allow_notconv=True)
        X, Y, _, _ = h.get_factors()
        h.close()
        h = StreamingNMF(n, k, m, prec=NMF_PREC_MIXED, kkt_target=0.0)
        h.append_columns(M32)
        h.set_factors(X, Y)
        h.set_pass_mode(3)
        h.sweep(args.ncu_precond + 3, want_stats=False)
        torch.cuda.synchronize()
        h.close()
        print("ncu case k16near: n=%d m=%d, a run to rel-KKT 1e-7, then 1 priming pair + %d sweeps of mode 3" %
              (n, m, args.ncu_precond + 3))
        return 0
    if args.ncu_case in ("k16", "k16inc"):
        import synth
        n, m, k = K16_N, 6144, K16_K     # 192 MB of FP32 M: above L2, a small device footprint
        M, _, _ = synth.pdf_like(n, m, k, noise=K16_NOISE, relative=True, seed=11)
        X, Y = synth.init_factors(n, m, k, seed=11)
        h = StreamingNMF(n, k, m, prec=NMF_PREC_MIXED, kkt_target=0.0)
        h.append_columns(np.asfortranarray(M, dtype=np.float32))
        h.set_factors(X, Y)
        # k16: tensor-core FP32-class sweeps; k16inc: chunks of a compensated
        # reference sweep and incremental sweeps
        h.set_pass_mode(0 if args.ncu_case == "k16" else 3)
        h.sweep(args.ncu_precond + 3, want_stats=False)
        torch.cuda.synchronize()
        h.close()
        print("ncu case %s: n=%d m=%d, 1 priming pair + %d sweeps" % (args.ncu_case, n, m, args.ncu_precond + 3))
        return 0
    M32, M64, X0, Y0 = make_data(0)
    fp64 = args.ncu_case == "f64"
    h = StreamingNMF(N_ROWS, RANK_K, M_COLS, prec=NMF_PREC_FP64 if fp64 else NMF_PREC_MIXED, kkt_target=0.0)
    h.append_columns(M64 if fp64 else M32)
    h.set_factors(X0, Y0)
    if not fp64:
        h.set_pass_mode({"ref": 1, "df": 2, "inc": 3}.get(args.ncu_case, 0))
    h.sweep(args.ncu_precond + 3, want_stats=False)
    torch.cuda.synchronize()
    h.close()
    print("ncu case %s: 1 priming pair + %d sweeps" % (args.ncu_case, args.ncu_precond + 3))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-ttk", action="store_true")
    ap.add_argument("--skip-batch", action="store_true", help="skip the 256-problem batched leg")
    ap.add_argument("--skip-serve", action="store_true", help="skip the streaming-serving leg")
    ap.add_argument("--skip-k16", action="store_true", help="skip the rank-16 tensor-core leg")
    ap.add_argument("--skip-k16-ttk", action="store_true",
                    help="skip the rank-16 run to relative KKT 1e-8 (inside the rank-16 leg)")
    ap.add_argument("--skip-batch-ttk", action="store_true",
                    help="skip the batched-vs-FP64 time to relative KKT 1e-8 on a subset of the batch")
    ap.add_argument("--skip-paper", action="store_true", help="skip the paper-shape runs to E <= 1e-6")
    ap.add_argument("--serve-seconds", type=float, default=12.0)
    ap.add_argument("--batch-ttk", action="store_true",
                    help="also run every batched problem to relative KKT 1e-8")
    ap.add_argument("--ncu-case", choices=["f32", "ref", "f64", "df", "inc", "batch", "k16", "k16inc", "k16near"], default=None,
                    help="run only a short launch sequence for an ncu capture")
    ap.add_argument("--ncu-precond", type=int, default=200)
    args = ap.parse_args()
    if args.ncu_case:
        return run_ncu_case(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
