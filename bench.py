"""Benchmark: syndrome-based sum-product LDPC decoding with early termination.

One step = one ldpc_decode call over the workload's frames (inputs resident
in HBM): by default the n = 1,000,000, R = 0.02 QC code (49 x 50 base,
Z = 20000), 32 frames at beta = 0.93, max 500 iterations, the paper's rule
(PCE-ET + VNR-ET).  The same frames are also decoded with the fixed-iteration
baselines (PCE-ET only, and no early termination) for the comparison.

Prints ONE JSON line (rank 0).  `python bench.py --impl reference` times the
FP64 CPU oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2507_03509_gb300 import gen  # noqa: E402

METRIC = "decoded Mbit/s (PCE+VNR early termination), n=1e6 R=0.02"
UNIT = "Mbit/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--frames", type=int, default=None)
    ap.add_argument("--slots", type=int, default=0, help="max_active_frames (0 = automatic)")
    ap.add_argument("--grid", type=int, default=0, help="grid_ctas (0 = all that fit)")
    ap.add_argument("--groups", type=int, default=0, help="independent CTA groups (0 = automatic)")
    ap.add_argument("--schedule", default="auto", choices=["auto", "lockstep", "dataflow", "frame", "frame_pair"],
                    help="decode schedule (auto: frame per CTA for small CSR codes, lock-step otherwise)")
    ap.add_argument("--flow-lag", type=int, default=0, help="dataflow schedule lag (0 = default)")
    ap.add_argument("--compare-steps", type=int, default=2, help="timed steps of each fixed-iteration rule")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--max-iter", type=int, default=None, help="override D_max (profiling runs)")
    ap.add_argument("--lean", action="store_true",
                    help="only the timed decodes: no fixed-iteration runs, no host-buffer runs, no CPU baseline")
    ap.add_argument("--sweep", action="store_true",
                    help="beta sweep (paper Figs. 1-2): FER, mean iterations and throughput K for PCE-ET with "
                         "D_max in {100, 250, 500, 1000} against PCE+VNR-ET; prints one JSON line per beta")
    ap.add_argument("--betas", default="0.84,0.85,0.86,0.87,0.88,0.89,0.90,0.92")
    ap.add_argument("--et-frames", type=int, default=512,
                    help="frames per beta of the equal-FER early-termination comparison")
    return ap.parse_args()


def shard_first_frame(rank: int, frames_per_rank: int) -> int:
    """Replicas only: rank r decodes frames r*F .. r*F + F - 1 of the workload
    (weak scaling; frames are independent, so no data is exchanged)."""
    return rank * frames_per_rank


def job_time_ms(local_ms: float, dist=None, device=None) -> float:
    """Whole-job time: the slowest rank's time (a MAX all-reduce)."""
    if dist is None:
        return local_ms
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value_mbit_s(n: int, frames_per_rank: int, steps: int, world: int, job_ms: float) -> float:
    """Decoded Mbit/s of the whole job: every rank's frames over the slowest rank's time."""
    return n * frames_per_rank * steps * world / (job_ms * 1e-3) / 1e6


def algorithmic_bytes_per_frame_iter(code) -> int:
    """8E (c2v read + write) + 12n (Lch read, APP write, APP read once), plus
    for a CSR code its index reads: col_idx on the check side (4E) and the
    variable-major edge list on the variable side (4E).  A QC code needs no
    index bytes (positions come from the shift table)."""
    return 8 * int(code.edges) + 12 * int(code.n) + csr_index_bytes_per_frame_iter(code)


MUFU_PER_SM_CLK = 16  # special-function (exp2, log2, reciprocal) lanes per SM and clock


def check_degrees_of(code) -> np.ndarray:
    """Degree of every check of a CSR or QC code."""
    if hasattr(code, "shifts"):
        return np.repeat((np.asarray(code.shifts) >= 0).sum(axis=1).astype(np.int64), code.Z)
    return code.check_degrees()


def mufu_per_frame_iter(code) -> int:
    """Special-function operations of one check pass (the FP32 check rule): a
    check of degree d in 3..6 takes d exponentials (r = exp(-|v|)), 3(d - 2)
    reciprocals (the prefix, suffix and middle boxplus combinations) and d
    logarithms (the outputs), 5d - 6 in all; the general path for d > 6 takes
    one combination more (5d - 5); checks of degree 1 and 2 take none (a
    constant and a copy)."""
    d = check_degrees_of(code)
    small = (d >= 3) & (d <= 6)
    return int((5 * d[small] - 6).sum() + (5 * d[d > 6] - 5).sum())


def frame_schedule_applies(code) -> bool:
    """Whether the frame-per-CTA kernel takes a CSR code: 16-bit indices and its
    shared memory (frame, q partials and index lists, 16-byte aligned pieces)
    within 220 KB -- the library's own rule, restated for naming the kernel."""
    n, m, E = code.n, code.m, int(code.edges)
    if hasattr(code, "shifts") or max(n, m, E) > 65535:
        return False
    r16 = lambda b: (b + 15) // 16 * 16
    nqb, swords = (n + 1023) // 1024, (m + 31) // 32
    total = (2 * r16(nqb * 8 * 8) + r16(4 * E) + 2 * r16(4 * n) + r16(4 * swords) + 2 * r16(2 * E)
             + r16(2 * (m + 1)) + r16(2 * m) + r16(2 * (n + 1)))
    return total <= 220 * 1024


def decoder_kernel_name(code, schedule="auto", frames=None, sms=152) -> str:
    """The decode kernel a decode of this code runs (FP32).  Automatic
    selection takes a CTA pair per frame when every frame gets its own pair at
    once (taken here as 2 x frames <= SMs)."""
    qc = hasattr(code, "shifts")
    if qc and schedule == "dataflow":
        return "bp_flow_kernel<float>"
    if not qc and schedule in ("auto", "frame", "frame_pair") and frame_schedule_applies(code):
        pair = schedule == "frame_pair" or (schedule == "auto" and frames is not None and 2 * frames <= sms)
        return "csr_frame_kernel<false,%d>" % (2 if pair else 1)
    return "bp_decode_kernel<float,%s>" % ("QcDev" if qc else "CsrDev")


# the lock-step decoder's device code and its launcher (the dataflow and frame
# kernels live in files of their own and do not change it)
DECODER_SOURCES = ("bp_kernels.cuh", "cn_math.cuh", "device_types.h", "host_common.h", "ldpc_api.cu")


def kernel_source_hash() -> str:
    """Hash of the sources the lock-step persistent decoder kernel is built from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2507_03509_gb300", "csrc")
    for name in DECODER_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload_name: str):
    """DRAM bytes per frame-iteration from the committed ncu summary, if it was
    taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "bp_decode_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    for line in open(path):
        parts = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if parts.get("source") == want and parts.get("workload") == workload_name:
            return float(parts["dram_bytes_per_frame_iter"])
    return None


def sfu_roof(code, fi_per_launch, kernel_ms, clk, dev):
    """Secondary roof: special-function operations per launch over the kernel
    time, against MUFU_PER_SM_CLK x SMs x the SM clock sampled under load (the
    maximum clock when no sample was taken)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    per_fi = mufu_per_frame_iter(code)
    achieved = fi_per_launch * per_fi / (kernel_ms * 1e-3)
    peak = MUFU_PER_SM_CLK * sms * mhz * 1e6
    return {"bound": "sfu", "achieved": achieved, "peak": peak, "unit": "MUFU op/s", "frac": achieved / peak,
            "mufu_per_frame_iter": per_fi, "sms": sms, "sm_mhz": mhz}


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s, r in zip(sm, rows) if num(r[3]) > 200.0] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(num(r[2]) for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline object)
# ---------------------------------------------------------------------------
def oracle_iters_mean(wl_name: str, rule: str):
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{wl_name}_{rule}.txt")
    if not os.path.exists(path):
        return None
    its = [int(l.split()[1]) for l in open(path) if l.strip() and not l.startswith("#")]
    return float(np.mean(its)) if its else None


def time_oracle_sample(code_csr, frames, max_sample_iters: int, target_s: float):
    """Time the oracle on one frame per core for I iterations (rule NONE, so
    every frame runs all I); returns (seconds per frame-iteration of the whole
    machine, cores, frames, iterations)."""
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    F = min(cores, frames.llr.shape[0])
    llr, syn = frames.llr[:F], frames.syndrome[:F]
    t0 = time.perf_counter()
    oracle.decode(code_csr, llr, syn, 1, oracle.RULE_NONE)
    t1 = time.perf_counter() - t0
    iters = int(max(1, min(max_sample_iters, target_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    oracle.decode(code_csr, llr, syn, iters, oracle.RULE_NONE)
    dt = time.perf_counter() - t0
    return dt / (F * iters), cores, F, iters, dt


def oracle_single_thread(code, frames, target_s: float = 3.0):
    """Seconds per frame-iteration of the oracle on one host thread (one frame,
    rule NONE, so every iteration runs), the per-core figure reported beside
    the all-core rate; returns (seconds, iterations timed)."""
    import oracle
    oracle.build()
    code_csr = code.to_csr() if hasattr(code, "to_csr") else code
    llr, syn = frames.llr[:1], frames.syndrome[:1]
    t0 = time.perf_counter()
    oracle.decode(code_csr, llr, syn, 1, oracle.RULE_NONE, threads=1)
    t1 = time.perf_counter() - t0
    iters = int(max(1, min(50, target_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    oracle.decode(code_csr, llr, syn, iters, oracle.RULE_NONE, threads=1)
    return (time.perf_counter() - t0) / iters, iters


def cpu_rate(code, wl, frames, target_s, d_mean, d_src):
    csr = code.to_csr() if hasattr(code, "to_csr") else code
    s_fi, cores, F, iters, dt = time_oracle_sample(csr, frames, wl["max_iter"], target_s)
    mbps = code.n / (d_mean * s_fi) / 1e6
    sample = (f"{F} frames x {iters} iterations of the FP64 oracle ({dt:.1f} s, {cores} threads); "
              f"per-frame-iteration time scaled to mean D = {d_mean:.1f} ({d_src})")
    return mbps, cores, sample, s_fi


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = gen.WORKLOADS[args.workload]
    code = gen.workload_code(args.workload)
    frames = gen.workload_frames(args.workload, code, frames=args.frames)
    d_mean = oracle_iters_mean(wl["name"], "pce_vnr")
    d_src = "oracle's own decisions on these frames"
    if d_mean is None:
        d_mean, d_src = float(wl["max_iter"]), "max_iter (no stored oracle decisions)"
    target = max(1.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        mbps, cores, sample, _ = cpu_rate(code, wl, frames, target, d_mean, d_src)
        if i >= args.warmup:
            vals.append(mbps)
            secs.append(time.perf_counter() - t0)
    v = float(np.mean(vals))
    st_s, st_iters = oracle_single_thread(code, frames, min(3.0, target))
    # a step of this arm is one bounded sample of the workload, so ms_per_step
    # is the wall time of that sample (calibration pass included), not the
    # time the oracle would take for the whole workload
    ms = float(np.mean(secs)) * 1e3
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "frames": int(frames.llr.shape[0]), "n": code.n, "m": code.m,
                       "edges": int(code.edges), "beta": wl["beta"], "max_iter": wl["max_iter"],
                       "rule": "pce_vnr"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "single_thread_s_per_frame_iter": st_s,
                             "single_thread_sample": f"1 frame x {st_iters} iterations, 1 thread",
                             "whole_workload_ms": code.n * frames.llr.shape[0] / (v * 1e6) * 1e3},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    ctx = gpu_context()
    ldpc, dev, dist, world, rank, local = ctx

    wl = dict(gen.WORKLOADS[args.workload])
    if args.max_iter:
        wl["max_iter"] = args.max_iter
    code = gen.workload_code(args.workload)
    F = args.frames or wl["frames"]
    frames = gen.workload_frames(args.workload, code, frames=F, first=shard_first_frame(rank, F))

    # CPU baseline first (rank 0, N = 1), before any GPU work in this process.
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.lean:
        cpu_pending = True
    else:
        cpu_pending = False

    graph = ldpc.Graph.from_code(code)
    llr = torch.from_numpy(frames.llr).to(dev)
    syn = torch.from_numpy(frames.syndrome).to(dev)
    out = (torch.empty((F, code.n), dtype=torch.uint8, device=dev), torch.empty(F, dtype=torch.uint8, device=dev),
           torch.empty(F, dtype=torch.int32, device=dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)
    B = algorithmic_bytes_per_frame_iter(code)

    def one(rule, stats):
        return ldpc.decode(graph, llr, syn, wl["max_iter"], rule, out=out, stats=stats,
                           max_active_frames=args.slots, grid_ctas=args.grid, groups=args.groups,
                           schedule=args.schedule, flow_lag=args.flow_lag)

    def timed(rule, steps, warmup):
        for _ in range(warmup):
            one(rule, ldpc.ldpc_decode_stats())
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        recs = []
        for _ in range(steps):
            flush.fill_(1.0)  # evict the previous step's data from L2 (outside the timed events)
            st = ldpc.ldpc_decode_stats()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one(rule, st)
            e1.record(stream)
            e1.synchronize()
            recs.append(dict(ms=e0.elapsed_time(e1), kernel_ms=st.kernel_ms, fi=st.frame_iterations,
                             launches=st.kernel_launches, grid=st.grid_ctas, slots=st.active_frames))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        res = dict(ms=sum(r["ms"] for r in recs), kernel_ms=sum(r["kernel_ms"] for r in recs),
                   fi=sum(r["fi"] for r in recs), launches=sum(r["launches"] for r in recs),
                   grid=recs[-1]["grid"], slots=recs[-1]["slots"], steps=steps,
                   per_launch_kernel_ms=[r["kernel_ms"] for r in recs])
        flags = out[1].cpu().numpy()
        iters = out[2].cpu().numpy()
        bits = out[0]
        errs = (bits.cpu().numpy() != frames.x).any(1)
        res.update(fer=float(np.mean(errs | ((flags & 1) == 0))), d_mean=float(iters.mean()),
                   success=int(((flags & 1) > 0).sum()), aborted=int(((flags & 2) > 0).sum()),
                   ok_frames=int((~errs & ((flags & 1) > 0)).sum()))
        return res

    clocks = ClockSampler(local)
    clocks.start()
    main = timed("pce_vnr", args.steps, max(3, args.warmup))
    clk = clocks.stop()

    ms_total = job_time_ms(main["ms"], dist, dev)
    value = job_value_mbit_s(code.n, F, args.steps, world, ms_total)
    edge_msgs = main["fi"] * 2 * code.edges / (main["ms"] * 1e-3)
    goodput = main["ok_frames"] * code.n * code.rate * args.steps / (main["ms"] * 1e-3) / 1e6

    # fixed-iteration baselines on the same frames
    comp = {}
    for rule in (() if args.lean else ("pce", "none")):
        r = timed(rule, args.compare_steps, 1)
        comp[rule] = dict(mbit_s=code.n * F * r["steps"] / (r["ms"] * 1e-3) / 1e6, d_mean=r["d_mean"],
                          fer=r["fer"], ms_per_step=r["ms"] / r["steps"],
                          edge_msgs_per_s=r["fi"] * 2 * code.edges / (r["ms"] * 1e-3),
                          hbm_frac=(r["fi"] * B / (r["kernel_ms"] * 1e-3) / 1e9) / hbm_peak()[0])

    # roofline of the dominant kernel (the persistent decoder)
    peak, peak_src = hbm_peak()
    achieved = main["fi"] * B / (main["kernel_ms"] * 1e-3) / 1e9
    traffic_fi = measured_traffic(wl["name"])
    per_launch_fi = main["fi"] / max(1, main["steps"])

    # end to end through the host-buffer entry point (pinned memory)
    h_llr = torch.from_numpy(frames.llr).pin_memory()
    h_syn = torch.from_numpy(frames.syndrome).pin_memory()
    h_bits = torch.empty((F, code.n), dtype=torch.uint8).pin_memory()
    h_flags = torch.empty(F, dtype=torch.uint8).pin_memory()
    h_iters = torch.empty(F, dtype=torch.int32).pin_memory()
    e2e_steps = 0 if args.lean else max(1, min(args.steps, 5))
    for _ in range(1 if e2e_steps else 0):
        ldpc.decode_host(graph, h_llr.numpy(), h_syn.numpy(), wl["max_iter"], "pce_vnr",
                         out=(h_bits.numpy(), h_flags.numpy(), h_iters.numpy()), stream=stream.cuda_stream,
                         max_active_frames=args.slots, grid_ctas=args.grid, groups=args.groups,
                         schedule=args.schedule, flow_lag=args.flow_lag)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ldpc.decode_host(graph, h_llr.numpy(), h_syn.numpy(), wl["max_iter"], "pce_vnr",
                         out=(h_bits.numpy(), h_flags.numpy(), h_iters.numpy()), stream=stream.cuda_stream,
                         max_active_frames=args.slots, grid_ctas=args.grid, groups=args.groups,
                         schedule=args.schedule, flow_lag=args.flow_lag)
    e2e_s = time.perf_counter() - t0
    e2e = None if not e2e_steps else {"value": code.n * F * e2e_steps / e2e_s / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": int(frames.llr.nbytes + frames.syndrome.nbytes),
           "d2h_bytes_per_step": int(F * code.n + F + 4 * F)}

    et_regime = None
    if not args.lean and world == 1:
        et_regime = {"tbp_like_r0.02": et_equal_fer(ldpc, dev, 7, (0.83, 0.84), frames=args.et_frames),
                     "regular_3_6": et_equal_fer(ldpc, dev, 6, (0.8735, 0.875), frames=args.et_frames)}
    others = None
    if not args.lean and world == 1 and args.workload == 2:
        others = other_configurations(args, ctx)
    learned = None
    if wl.get("code_from") == 2 and not args.lean and world == 1:  # the streaming configuration
        learned = {"this_workload": learned_weights_comparison(ldpc, dev, args.workload, code, frames, wl["max_iter"]),
                   "tbp_like_beta_0.84": learned_weights_comparison(
                       ldpc, dev, 7, gen.workload_code(7), gen.workload_frames(7, gen.workload_code(7), frames=32,
                                                                               beta=0.84), 500)}

    if cpu_pending:
        d_mean_o = oracle_iters_mean(wl["name"], "pce_vnr")
        src = "oracle's own decisions on these frames"
        if d_mean_o is None:
            d_mean_o, src = main["d_mean"], "mean D of this run"
        mbps, cores, sample, _ = cpu_rate(code, wl, frames, args.cpu_seconds, d_mean_o, src)
        st_s, st_iters = oracle_single_thread(code, frames, min(3.0, args.cpu_seconds))
        cpu = {"value": mbps, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread_s_per_frame_iter": st_s,
               "single_thread_sample": f"1 frame x {st_iters} iterations, 1 thread"}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["name"], "frames_per_gpu": F, "n": code.n, "m": code.m, "edges": int(code.edges),
                   "rate": code.rate, "beta": wl["beta"], "max_iter": wl["max_iter"], "rule": "pce_vnr",
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs 159 MB + decoder state > L2 (129 MB); L2 also flushed between steps",
                   "slots": main["slots"], "grid_ctas": main["grid"], "groups": args.groups or "auto"},
        "d_mean": main["d_mean"], "fer": main["fer"], "success_frames": main["success"],
        "aborted_frames": main["aborted"], "edge_msgs_per_s": edge_msgs, "goodput_mbit_s": goodput,
        "fixed_iteration": comp,
        "et_speedup": None if not comp else {
            "vs_pce": comp["pce"]["ms_per_step"] / (main["ms"] / args.steps),
            "vs_none": comp["none"]["ms_per_step"] / (main["ms"] / args.steps)},
        "et_equal_fer": et_regime,
        "learned_weights": learned,
        "other_configurations": others,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_src,
                     "traffic": (traffic_fi * per_launch_fi) if traffic_fi else None,
                     "algorithmic_bytes_per_launch": per_launch_fi * B,
                     "kernel": decoder_kernel_name(code, args.schedule, int(frames.llr.shape[0]),
                                                   torch.cuda.get_device_properties(dev).multi_processor_count),
                     "kernel_ms_per_launch": main["kernel_ms"] / main["steps"]},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": main["launches"],
        "clocks": clk,
    }
    line["secondary_roofs"] = {"sfu": sfu_roof(code, per_launch_fi, main["kernel_ms"] / main["steps"], clk, dev)}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def learned_weights_comparison(ldpc, dev, number, code, frames, max_iter, T=20, train_frames=16, steps=30,
                               warm=True):
    """Plain flooding (D_max), PCE+VNR early termination, and early termination
    with learned weights (one per iteration and base block, trained by the
    weighted-BP adjoint on other frames of the same workload: T unrolled
    iterations, BCE loss, normalised gradient steps: each moves the largest
    weight by 0.01) on the same frames: decoded Mbit/s, mean iterations, FER."""
    import torch
    nblk = int((code.shifts >= 0).sum())
    cls = np.arange(nblk, dtype=np.int32)
    g = ldpc.Graph.from_code(code)
    wl = gen.WORKLOADS[number]
    beta = float(gen.biawgn_capacity(frames.sigma[0]))
    beta = code.rate / beta
    train = gen.workload_frames(number, code, frames=train_frames, first=100000, beta=beta)
    plan = ldpc.WeightedBP(g, train_frames, T, cls, nblk, checkpoint_every=5)
    tl, ts, tx = (torch.from_numpy(a).to(dev) for a in (train.llr, train.syndrome, train.x))
    w = torch.ones((T, nblk), dtype=torch.float32, device=dev)
    losses = []
    t0 = time.perf_counter()
    for _ in range(steps):
        app = plan.forward(tl, ts, w)
        loss, gapp = plan.loss(app, tx)
        gw, _ = plan.backward(tl, ts, w, gapp)
        plan.sgd_step(w, gw, 0.01 / max(float(gw.abs().max().item()), 1e-30))
        losses.append(float(loss.item()))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    llr = torch.from_numpy(frames.llr).to(dev)
    syn = torch.from_numpy(frames.syndrome).to(dev)
    F = frames.llr.shape[0]
    out = {"code": wl["name"], "beta": round(beta, 4), "frames": F, "max_iter": max_iter,
           "training": {"frames": train_frames, "iters": T, "steps": steps, "loss_first": losses[0],
                        "loss_last": losses[-1], "seconds": train_s,
                        "weights_min": float(w.min().item()), "weights_max": float(w.max().item())}}

    def stats(bits, flags, iters, ms):
        b, fl, it = bits.cpu().numpy(), flags.cpu().numpy(), iters.cpu().numpy()
        ok = ((fl & 1) > 0) & (b == frames.x).all(1)
        return {"mbit_s": code.n * F / (ms * 1e-3) / 1e6, "d_mean": float(it.mean()), "fer": float(1 - ok.mean()),
                "aborted": int(((fl & 2) > 0).sum()), "ms": ms}

    def timed(fn):
        if warm:
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        e1.synchronize()
        return r, e0.elapsed_time(e1)

    for name, fn in (("flooding", lambda: ldpc.decode(g, llr, syn, max_iter, "none")),
                     ("early_termination", lambda: ldpc.decode(g, llr, syn, max_iter, "pce_vnr")),
                     ("learned_weights_et", lambda: plan.decode(llr, syn, w, max_iter, "pce_vnr"))):
        r, ms = timed(fn)
        out[name] = stats(*r, ms)
    plan.close()
    g.close()
    return out


def csr_index_bytes_per_frame_iter(code) -> int:
    """A CSR code's index traffic per frame-iteration: the check side reads
    col_idx (4E) and the variable side the variable-major edge list (4E)."""
    return 0 if hasattr(code, "shifts") else 8 * int(code.edges)


def l2_copy_gbs(dev, mbytes=32, reps=200):
    """Measured on-chip (L2-resident) copy bandwidth: a mbytes buffer copied
    into another (both fit the 129 MB L2) reps times; read + write bytes over
    CUDA-event time, best of 5."""
    import torch
    a = torch.ones(mbytes * 2**20 // 4, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    for _ in range(10):
        b.copy_(a)
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.copy_(a)
        e1.record()
        e1.synchronize()
        best = max(best, 2 * a.numel() * 4 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


def l2_resident(ldpc, dev, steps=10):
    """The oracle-sized workload (n = 4096 random CSR code, 64 frames, D_max
    200): one frame's state is ~80 KB and all 64 frames plus the code's
    indices (~100 KB) stay in L2, so throughput is reported against the
    measured L2 copy bandwidth, with algorithmic bytes 8E + 12n plus the CSR
    index bytes 8E per frame-iteration (algorithmic_bytes_per_frame_iter)."""
    import torch
    wl = gen.WORKLOADS[1]
    code = gen.workload_code(1)
    fr = gen.workload_frames(1, code)
    g = ldpc.Graph.from_code(code)
    llr, syn = torch.from_numpy(fr.llr).to(dev), torch.from_numpy(fr.syndrome).to(dev)
    B = algorithmic_bytes_per_frame_iter(code)
    l2 = l2_copy_gbs(dev)
    out = {"workload": wl["name"], "frames": int(fr.llr.shape[0]), "n": code.n, "edges": int(code.edges),
           "max_iter": wl["max_iter"], "bytes_per_frame_iter": B, "l2_copy_gbs_measured": l2, "rules": {},
           "schedules": {}}
    for sched in ("auto", "lockstep", "frame", "frame_pair"):
        res = {}
        for rule in ("pce_vnr", "pce", "none"):
            for _ in range(3):
                ldpc.decode(g, llr, syn, wl["max_iter"], rule, schedule=sched)
            kms, tms, fi = [], [], 0
            for _ in range(steps):
                st = ldpc.ldpc_decode_stats()
                bits, flags, iters = ldpc.decode(g, llr, syn, wl["max_iter"], rule, stats=st, schedule=sched)
                kms.append(st.kernel_ms)
                tms.append(st.total_ms)
                fi = st.frame_iterations
            k = statistics.median(kms) * 1e-3
            t = statistics.median(tms) * 1e-3
            ok = ((flags.cpu().numpy() & 1) > 0) & (bits.cpu().numpy() == fr.x).all(1)
            gbs = fi * B / k / 1e9
            res[rule] = {"decoded_mbit_s": code.n * fr.llr.shape[0] / t / 1e6, "kernel_ms": k * 1e3,
                         "total_ms": t * 1e3, "d_mean": fi / fr.llr.shape[0], "fer": float(1 - ok.mean()),
                         "achieved_gbs": gbs, "frac_of_l2_copy": gbs / l2, "frac_of_hbm_peak": gbs / hbm_peak()[0]}
        if sched == "auto":
            out["rules"] = res
        else:
            out["schedules"][sched] = {r: {key: v[key] for key in ("kernel_ms", "decoded_mbit_s", "frac_of_l2_copy")}
                                       for r, v in res.items()}
    g.close()
    return out


def stream_measure(ldpc, dev):
    """The streaming workload (512 frames of the n = 10^6 code at beta = 0.95,
    D_max 1000), all frames in one call: PCE+VNR early termination with its
    roofline fraction, PCE-ET alone and fixed-iteration decoding on the same
    frames, and the learned-weight decoder next to both."""
    import torch
    number = 5
    wl = gen.WORKLOADS[number]
    code = gen.workload_code(number)
    fr = gen.workload_frames(number, code)
    F = fr.llr.shape[0]
    g = ldpc.Graph.from_code(code)
    llr, syn = torch.from_numpy(fr.llr).to(dev), torch.from_numpy(fr.syndrome).to(dev)
    B = algorithmic_bytes_per_frame_iter(code)
    ldpc.decode(g, llr, syn, 5, "pce")  # sizes the workspace for 512 slots
    out = {"workload": wl["name"], "frames": F, "n": code.n, "beta": wl["beta"], "max_iter": wl["max_iter"]}
    for rule in ("pce_vnr", "pce", "none"):
        st = ldpc.ldpc_decode_stats()
        bits, flags, iters = ldpc.decode(g, llr, syn, wl["max_iter"], rule, stats=st)
        ok = ((flags.cpu().numpy() & 1) > 0) & (bits.cpu().numpy() == fr.x).all(1)
        out[rule] = {"decoded_mbit_s": code.n * F / (st.total_ms * 1e-3) / 1e6, "ms": st.total_ms,
                     "d_mean": st.frame_iterations / F, "fer": float(1 - ok.mean()),
                     "hbm_frac": st.frame_iterations * B / (st.kernel_ms * 1e-3) / 1e9 / hbm_peak()[0]}
    out["et_speedup"] = {"vs_pce": out["pce"]["ms"] / out["pce_vnr"]["ms"],
                         "vs_none": out["none"]["ms"] / out["pce_vnr"]["ms"]}
    del llr, syn
    g.close()
    out["learned_weights"] = learned_weights_comparison(ldpc, dev, number, code, fr, wl["max_iter"], warm=False)
    torch.cuda.empty_cache()
    return out


def compact(line, keys):
    """The named keys of a workload's bench line (a sub-object of the headline line)."""
    return {k: line[k] for k in keys if k in line}


def other_configurations(args, ctx):
    """Short runs of the other configurations for the headline line: the
    L2-resident oracle-sized workload, the 256-frame mixed batch (autotuned,
    CUDA graph), one weighted-BP training step, and the 512-frame stream."""
    import torch
    ldpc, dev = ctx[0], ctx[1]
    res = {"l2_resident_n4096": l2_resident(ldpc, dev)}
    torch.cuda.empty_cache()
    sub = argparse.Namespace(**{**vars(args), "steps": 3, "warmup": 3, "frames": None, "groups": 0, "slots": 0,
                                "max_iter": None, "lean": False, "compare_steps": 1, "no_cpu_baseline": True})
    sub.workload = 3
    b = run_batch(sub, ctx, compact=True)
    res["batch_mixed_256"] = compact(b, ("metric", "value", "unit", "ms_per_step", "d_mean", "fer", "et_speedup",
                                         "fixed_iteration", "per_code", "roofline", "gpu_launches"))
    res["batch_mixed_256"]["schedule"] = b["config"]["schedule"]
    torch.cuda.empty_cache()
    sub.workload = 4
    sub.steps = 10
    w = run_wbp(sub, ctx, compact=True)
    res["wbp_training_step"] = compact(w, ("metric", "value", "unit", "ms_per_step", "loss_first_step",
                                           "loss_after_steps", "forward_only", "roofline", "gpu_launches"))
    torch.cuda.empty_cache()
    res["stream_512"] = stream_measure(ldpc, dev)
    return res


ET_DMAX = (100, 150, 200, 250, 300, 400, 500, 1000)


def wilson_interval(k: int, n: int, z: float = 1.959964):
    """95 % Wilson score interval of a proportion k/n."""
    if n == 0:
        return (0.0, 1.0)
    p = k / n
    den = 1.0 + z * z / n
    mid = (p + z * z / (2 * n)) / den
    half = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return (max(0.0, mid - half), min(1.0, mid + half))


def pce_decoded_at(ok, iters):
    """Iteration at which PCE-ET decoded each frame correctly (success with
    x^ = x), or a value above any D_max for a frame it did not."""
    return np.where(np.asarray(ok, dtype=bool), np.asarray(iters, dtype=np.int64), np.iinfo(np.int64).max)


def fer_at(k_ok, dmax: int) -> float:
    """FER of PCE-ET at D_max = dmax on the same frames: a frame that PCE-ET
    decodes at iteration k follows the same trajectory, and stops with the
    same bits, for every D_max >= k."""
    return 1.0 - float((np.asarray(k_ok) <= dmax).mean())


def matched_dmax(k_ok, fer_target: float, dmax_max: int) -> int:
    """Smallest D_max (1 .. dmax_max) at which PCE-ET's FER is not above
    fer_target (equal FER, up to a quarter frame of rounding)."""
    F = np.asarray(k_ok).size
    for D in range(1, dmax_max + 1):
        if fer_at(k_ok, D) <= fer_target + 0.25 / F:
            return D
    return dmax_max


def et_equal_fer(ldpc, dev, number, betas, frames=512, vnr_dmax=1000):
    """Early termination against the D_max baselines at equal FER (paper,
    section "Simulations" and Fig. 2 left), on the same frames at each beta:

    * PCE-ET at every D_max in ET_DMAX and PCE+VNR-ET at vnr_dmax: FER with
      its 95 % Wilson interval, mean iterations, CUDA-event time, decoded and
      goodput Mbit/s, and K = N R (1 - FER) / D (Eq. 2);
    * the matched baseline: under PCE-ET a frame decoded at iteration k is
      decoded for every D_max >= k, so the D_max = 1000 run gives FER(D) for
      every D exactly; D* is the smallest D_max with FER(D*) <= FER(VNR), and
      PCE-ET at D_max = D* is decoded and timed as well.  Its time over the
      time of PCE+VNR is the speed-up at equal FER;
    * FER(500) against FER(1000) (the paper finds the two curves identical)."""
    import torch
    code = gen.workload_code(number)
    graph = ldpc.Graph.from_code(code)
    wl = gen.WORKLOADS[number]
    t0 = time.perf_counter()
    frs = gen.workload_frames_betas(number, code, betas, frames=frames)
    gen_s = time.perf_counter() - t0
    out = {"workload": wl["name"], "n": code.n, "rate": code.rate, "frames": frames, "vnr_d_max": vnr_dmax,
           "frame_generation_s": gen_s, "points": []}
    for beta, fr in zip(betas, frs):
        llr = torch.from_numpy(fr.llr).to(dev)
        syn = torch.from_numpy(fr.syndrome).to(dev)
        x_dev = torch.from_numpy(fr.x).to(dev)
        bits = torch.empty((frames, code.n), dtype=torch.uint8, device=dev)
        flg = torch.empty(frames, dtype=torch.uint8, device=dev)
        its = torch.empty(frames, dtype=torch.int32, device=dev)

        def run(rule, dmax):
            st = ldpc.ldpc_decode_stats()
            ldpc.decode(graph, llr, syn, dmax, rule, out=(bits, flg, its), stats=st)
            ok = (((flg & 1) > 0) & (bits == x_dev).all(1)).cpu().numpy()
            it = its.cpu().numpy()
            k_ok = int(ok.sum())
            fer = 1.0 - k_ok / frames
            d = float(it.mean())
            t = st.total_ms * 1e-3
            return {"fer": fer, "fer_ci95": wilson_interval(frames - k_ok, frames), "d_mean": d,
                    "aborted": int(((flg.cpu().numpy() & 2) > 0).sum()), "ms": st.total_ms,
                    "decoded_mbit_s": code.n * frames / t / 1e6,
                    "goodput_mbit_s": k_ok * code.n * code.rate / t / 1e6,
                    "K": code.n * code.rate * (1.0 - fer) / d}, ok, it

        ldpc.decode(graph, llr, syn, 20, "pce", out=(bits, flg, its))  # workspace for these frames
        pce, k_ok = {}, None
        for dmax in ET_DMAX:
            r, ok, it = run("pce", dmax)
            pce[str(dmax)] = r
            if dmax == max(ET_DMAX):
                k_ok = pce_decoded_at(ok, it)
        vnr, _, _ = run("pce_vnr", vnr_dmax)
        # the curve must reproduce every measured D_max run (same frames, same trajectories)
        curve_ok = all(abs(fer_at(k_ok, int(d)) - r["fer"]) < 0.5 / frames for d, r in pce.items())
        d_star = matched_dmax(k_ok, vnr["fer"], max(ET_DMAX))
        star, _, _ = run("pce", d_star)
        pt = {"beta": beta, "pce": pce, "pce_vnr": vnr,
              "equal_fer": {"d_max": d_star, **star, "speedup_vs_pce_vnr": star["ms"] / vnr["ms"],
                            "goodput_ratio_vnr_over_pce": (vnr["goodput_mbit_s"] / star["goodput_mbit_s"]
                                                           if star["goodput_mbit_s"] > 0 else None)},
              "fer_curve_matches_runs": curve_ok,
              "fer_500_vs_1000": {"fer_500": pce["500"]["fer"], "fer_1000": pce["1000"]["fer"],
                                  "frames_decoded_after_500": int(round((pce["500"]["fer"] - pce["1000"]["fer"])
                                                                        * frames))},
              "K_ratio_vnr_over_pce": {d: (vnr["K"] / r["K"] if r["K"] > 0 else None) for d, r in pce.items()},
              "time_ratio_pce_over_vnr": {d: r["ms"] / vnr["ms"] for d, r in pce.items()}}
        out["points"].append(pt)
        del llr, syn, bits, flg, its
        torch.cuda.empty_cache()
    graph.close()
    return out


def run_sweep(args):
    """FER, mean iterations D and throughput against beta for the paper's
    D_max baselines (PCE-ET on) and for PCE+VNR-ET, on the same frames.

    K = N R (1 - FER) / D is the paper's Eq. 2 throughput in bits per iteration
    latency; goodput is the measured rate of correctly decoded information bits."""
    import torch
    from paper_2507_03509_gb300 import build
    build.build()
    from paper_2507_03509_gb300 import ldpc
    dev = torch.device("cuda", 0)
    number = args.workload if args.workload != 2 else 6
    wl = gen.WORKLOADS[number]
    code = gen.workload_code(number)
    graph = ldpc.Graph.from_code(code)
    F = args.frames or wl["frames"]
    runs = [("pce", 100), ("pce", 250), ("pce", 500), ("pce", 1000), ("pce_vnr", 1000)]
    betas = [float(b) for b in args.betas.split(",")]
    for beta, frames in zip(betas, gen.workload_frames_betas(number, code, betas, frames=F)):
        llr = torch.from_numpy(frames.llr).to(dev)
        syn = torch.from_numpy(frames.syndrome).to(dev)
        row = {"experiment": "beta_sweep", "workload": wl["name"], "n": code.n, "rate": code.rate, "frames": F,
               "beta": beta, "sigma": float(frames.sigma[0]), "runs": {}}
        for rule, dmax in runs:
            ldpc.decode(graph, llr, syn, dmax, rule)  # warm-up
            ms = []
            for _ in range(max(1, args.steps)):
                st = ldpc.ldpc_decode_stats()
                bits, flags, iters = ldpc.decode(graph, llr, syn, dmax, rule, stats=st)
                ms.append(st.total_ms)
            t = float(np.median(ms)) * 1e-3
            flags = flags.cpu().numpy()
            iters = iters.cpu().numpy()
            ok = ((flags & 1) > 0) & (bits.cpu().numpy() == frames.x).all(1)
            fer = float(1.0 - ok.mean())
            dmean = float(iters.mean())
            row["runs"][f"{rule}_{dmax}"] = {
                "fer": fer, "fer_ci95": wilson_interval(int(F - ok.sum()), F), "d_mean": dmean,
                "aborted": int(((flags & 2) > 0).sum()),
                "ms": t * 1e3, "decoded_mbit_s": code.n * F / t / 1e6,
                "goodput_mbit_s": float(ok.sum()) * code.n * code.rate / t / 1e6,
                "K_bits_per_iteration": code.n * code.rate * (1.0 - fer) / dmean}
        kv = row["runs"]["pce_vnr_1000"]["K_bits_per_iteration"]
        row["K_ratio_vnr_over"] = {k: (kv / v["K_bits_per_iteration"] if v["K_bits_per_iteration"] > 0 else None)
                                   for k, v in row["runs"].items() if k != "pce_vnr_1000"}
        print(json.dumps(row), flush=True)


# ---------------------------------------------------------------------------
# Batched frames of several codes (one persistent kernel in a CUDA graph)
# ---------------------------------------------------------------------------
BATCH_METRIC = "decoded Mbit/s (PCE+VNR early termination), 256 frames of 3 QC codes n=64k..1e6"


def batch_oracle_rate(codes, bf, d_per_frame, target_s, d_src):
    """CPU rate of the oracle on the batch: seconds per frame-iteration of each
    code from a bounded sample, times each frame's D."""
    s_fi = {}
    cores = 1
    parts = []
    for c, code in enumerate(codes):
        idx = np.nonzero(bf.frame_code == c)[0]
        if idx.size == 0:
            continue
        fr = gen.Frames(None, np.stack([bf.llr[bf.var_off[f]:bf.var_off[f + 1]] for f in idx[:16]]),
                        np.stack([bf.syndrome[bf.syn_off[f]:bf.syn_off[f + 1]] for f in idx[:16]]), None)
        t, cores, F, iters, dt = time_oracle_sample(code.to_csr(), fr, 500, target_s / len(codes))
        s_fi[c] = t
        parts.append(f"code {c}: {F} frames x {iters} iterations ({dt:.1f} s)")
    cpu_s = sum(d_per_frame[f] * s_fi[int(bf.frame_code[f])] for f in range(bf.frame_code.size))
    mbps = float(bf.var_off[-1]) / cpu_s / 1e6
    sample = ("FP64 oracle, " + "; ".join(parts) + f"; {cores} threads; per-frame-iteration times of each "
              f"code scaled to every frame's D ({d_src})")
    return mbps, cores, sample


def batch_oracle_iters(wl_name):
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{wl_name}_pce_vnr.txt")
    if not os.path.exists(path):
        return None
    its = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f, it = line.split()[:2]
            its[int(f)] = int(it)
    return its


def run_batch_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = gen.WORKLOADS[args.workload]
    codes = gen.batch_codes(args.workload)
    bf = gen.workload_batch(args.workload, codes, frames=args.frames)
    F = bf.frame_code.size
    its = batch_oracle_iters(wl["name"])
    if its is not None and all(f in its for f in range(F)):
        d, src = [its[f] for f in range(F)], "oracle's own decisions on these frames"
    else:
        d, src = [wl["max_iter"]] * F, "max_iter (no stored oracle decisions)"
    target = max(1.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        mbps, cores, sample = batch_oracle_rate(codes, bf, d, target, src)
        if i >= args.warmup:
            vals.append(mbps)
            secs.append(time.perf_counter() - t0)
    v = float(np.mean(vals))
    # one step of this arm is one bounded sample: ms_per_step is its wall time
    line = {"metric": BATCH_METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(secs)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "frames": F, "bits_per_step": int(bf.var_off[-1]),
                       "max_iter": wl["max_iter"], "rule": "pce_vnr"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "whole_workload_ms": float(bf.var_off[-1]) / (v * 1e6) * 1e3},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def gpu_context():
    """(ldpc binding, device, dist or None, world, rank, local rank) of this
    process: one rank per GPU under torchrun, NCCL only for timing."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2507_03509_gb300 import build
    build.build()
    from paper_2507_03509_gb300 import ldpc
    return ldpc, dev, dist, world, rank, local


def run_batch(args, ctx=None, compact=False):
    """One step = one replay of a CUDA graph holding a whole batch decode
    (control init, syndrome packing, the persistent decoder, status word) of
    the workload's frames, inputs resident in HBM; schedule from the autotuner.
    compact: no host-buffer (e2e) or CPU legs and only the PCE-ET baseline;
    the line is returned (a sub-object of the headline line), not printed."""
    import torch
    ldpc, dev, dist, world, rank, local = ctx or gpu_context()

    wl = gen.WORKLOADS[args.workload]
    max_iter = args.max_iter or wl["max_iter"]
    codes = gen.batch_codes(args.workload)
    F = args.frames or wl["frames"]
    bf = gen.workload_batch(args.workload, codes, frames=F, first=shard_first_frame(rank, F))
    bits_per_step = int(bf.var_off[-1])
    graphs = [ldpc.Graph.from_code(c) for c in codes]
    batch = ldpc.Batch(graphs, bf.frame_code)
    llr = torch.from_numpy(bf.llr).to(dev)
    syn = torch.from_numpy(bf.syndrome).to(dev)
    out = batch.outputs(dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    # schedule: the autotuner's pick unless given on the command line (untimed)
    t0 = time.perf_counter()
    if args.groups or args.slots:
        tuned = None
        opt = dict(groups=args.groups, max_active_frames=args.slots)
    else:
        tuned = batch.autotune(llr, syn, max_iter, "pce_vnr", out=out)
        opt = {}
    tune_s = time.perf_counter() - t0
    batch.decode(llr, syn, max_iter, "pce_vnr", out=out, **opt)  # sizes the workspace for this schedule

    # capture one decode in a CUDA graph (warmed up on a side stream first)
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        batch.decode_async(llr, syn, max_iter, "pce_vnr", out, status, **opt)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg):
        batch.decode_async(llr, syn, max_iter, "pce_vnr", out, status, **opt)
    for _ in range(max(3, args.warmup)):
        cg.replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)  # evict the previous step's data from L2 (outside the timed events)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cg.replay()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    if int(status.item()) != 0:
        raise RuntimeError(f"batch decode failed: {ldpc.ldpc_status_str(int(status.item()))}")
    ms_total = job_time_ms(sum(ms), dist, dev)
    value = bits_per_step * args.steps * world / (ms_total * 1e-3) / 1e6

    iters = out[2].cpu().numpy()
    flags = out[1].cpu().numpy()
    bits = out[0].cpu().numpy()
    errs = np.array([(bits[bf.var_off[f]:bf.var_off[f + 1]] != bf.x[bf.var_off[f]:bf.var_off[f + 1]]).any()
                     for f in range(F)])
    ok = ~errs & ((flags & 1) > 0)
    B = [algorithmic_bytes_per_frame_iter(c) for c in codes]
    bytes_per_step = float(sum(int(iters[f]) * B[int(bf.frame_code[f])] for f in range(F)))
    peak, peak_src = hbm_peak()
    achieved = bytes_per_step / (statistics.mean(ms) * 1e-3) / 1e9
    per_code = {}
    for c, code in enumerate(codes):
        idx = bf.frame_code == c
        per_code[gen.WORKLOADS[args.workload]["codes"][c]["name"]] = {
            "frames": int(idx.sum()), "d_mean": float(iters[idx].mean()) if idx.any() else None,
            "fer": float(1 - ok[idx].mean()) if idx.any() else None,
            "aborted": int(((flags[idx] & 2) > 0).sum())}

    # fixed-iteration baselines (synchronous decodes of the same batch)
    comp = {}
    for rule in (() if args.lean else (("pce",) if compact else ("pce", "none"))):
        batch.decode(llr, syn, max_iter, rule, out=out, **opt)
        t = []
        for _ in range(args.compare_steps):
            flush.fill_(1.0)
            st = ldpc.ldpc_decode_stats()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.decode(llr, syn, max_iter, rule, out=out, stats=st, **opt)
            e1.record(stream)
            e1.synchronize()
            t.append(e0.elapsed_time(e1))
        comp[rule] = {"mbit_s": bits_per_step / (statistics.mean(t) * 1e-3) / 1e6,
                      "ms_per_step": statistics.mean(t), "d_mean": float(out[2].float().mean().item())}

    # end to end: pinned host buffers copied in, graph replayed, results copied out, every step
    e2e = None
    if not args.lean and not compact:
        h_llr = torch.from_numpy(bf.llr).pin_memory()
        h_syn = torch.from_numpy(bf.syndrome).pin_memory()
        h_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in out]
        e2e_steps = max(1, min(args.steps, 5))
        def e2e_step():
            llr.copy_(h_llr, non_blocking=True)
            syn.copy_(h_syn, non_blocking=True)
            cg.replay()
            for h, d in zip(h_out, out):
                h.copy_(d, non_blocking=True)
            stream.synchronize()
        e2e_step()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": bits_per_step * e2e_steps / e2e_s / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(bf.llr.nbytes + bf.syndrome.nbytes),
               "d2h_bytes_per_step": int(sum(t.numel() * t.element_size() for t in out))}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.lean and not compact:
        mbps, cores, sample = batch_oracle_rate(codes, bf, [int(i) for i in iters], args.cpu_seconds,
                                                "D of this run")
        cpu = {"value": mbps, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    if rank != 0:
        return
    line = {
        "metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["name"], "frames_per_gpu": F, "bits_per_step": bits_per_step,
                   "codes": [{"n": c.n, "m": c.m, "edges": int(c.edges), "rate": c.rate} for c in codes],
                   "beta": [wl["beta_lo"], wl["beta_hi"]], "max_iter": max_iter, "rule": "pce_vnr",
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs > L2 (129 MB); L2 also flushed between steps",
                   "schedule": {"autotuned": tuned is not None, "groups": tuned[0] if tuned else args.groups,
                                "slots": tuned[1] if tuned else args.slots, "autotune_s": tune_s},
                   "cuda_graph": "init + pack + persistent decoder + status kernels, replayed once per step"},
        "d_mean": float(iters.mean()), "fer": float(1 - ok.mean()), "per_code": per_code,
        "fixed_iteration": comp,
        "et_speedup": None if not comp else {r: comp[r]["ms_per_step"] / (ms_total / args.steps) for r in comp},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_src, "traffic": None, "algorithmic_bytes_per_launch": bytes_per_step,
                     "kernel": "bp_decode_kernel<float,QcDev>",
                     "timed": "whole graph replay (the decoder plus three one-CTA kernels)"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": 4 * args.steps,
        "clocks": clk,
    }
    batch.close()
    for g in graphs:
        g.close()
    if compact:
        return line
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Weighted BP training (forward, loss, adjoint, gradient step in one CUDA graph)
# ---------------------------------------------------------------------------
WBP_METRIC = "trained Mbit/s (weighted BP, 20 unrolled iterations, forward + adjoint + step), QC n=65536"


def wbp_bytes_per_frame_iter(code) -> int:
    """Forward 8E + 12n (as the decoder) plus adjoint 12E + 12n: c2v^(k-1) and
    G read, G^(k-1) written, APP^(k-1) read, dloss/dLch read and written."""
    return 20 * int(code.edges) + 24 * int(code.n)


def wbp_setup(number):
    wl = gen.WORKLOADS[number]
    code = gen.workload_code(number)
    nblk = int((code.shifts >= 0).sum())
    cls_blk = np.arange(nblk, dtype=np.int32)
    return wl, code, nblk, cls_blk


def wbp_oracle_rate(code, cls_csr, C, fr, T, target_s):
    """Oracle training throughput (forward, loss and gradient, FP64) on a
    bounded sample: one frame per core, frames decoded together."""
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    csr = code.to_csr()
    w = np.ones((T, C))
    F = min(cores, fr.llr.shape[0])
    done, calls = 0, 0
    t0 = time.perf_counter()
    while True:  # groups of one frame per core until the target time is used
        lo = (calls * F) % fr.llr.shape[0]
        sel = slice(lo, min(lo + F, fr.llr.shape[0]))
        oracle.wbp(csr, fr.llr[sel], fr.syndrome[sel], fr.x[sel], T, cls_csr, w)
        done += sel.stop - sel.start
        calls += 1
        dt = time.perf_counter() - t0
        if dt >= target_s:
            break
    return code.n * done / dt / 1e6, cores, (f"{done} frames ({calls} calls of {F}) x {T} iterations, forward + "
                                             f"loss + gradient of the FP64 oracle ({dt:.1f} s, {cores} threads)")


def run_wbp_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl, code, nblk, cls_blk = wbp_setup(args.workload)
    cls_csr = cls_blk[gen.qc_csr_edge_blocks(code)]
    fr = gen.workload_frames(args.workload, code, frames=min(wl["frames"], 64))
    target = max(1.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        v, cores, sample = wbp_oracle_rate(code, cls_csr, nblk, fr, wl["iters"], target)
        if i >= args.warmup:
            vals.append(v)
            secs.append(time.perf_counter() - t0)
    v = float(np.mean(vals))
    F = wl["frames"]
    # one step of this arm is one bounded sample: ms_per_step is its wall time
    line = {"metric": WBP_METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(secs)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "frames": F, "n": code.n, "iters": wl["iters"], "classes": nblk},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "whole_workload_ms": code.n * F / (v * 1e6) * 1e3},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_wbp(args, ctx=None, compact=False):
    """One step = one replay of a CUDA graph holding a whole training step of
    the weighted decoder on the workload's frames (inputs resident in HBM):
    forward over T iterations with checkpoints, BCE loss, adjoint with
    recomputation, SGD update of the weights.  compact: as in run_batch."""
    import torch
    ldpc, dev, dist, world, rank, local = ctx or gpu_context()

    wl, code, nblk, cls_blk = wbp_setup(args.workload)
    F = args.frames or wl["frames"]
    T = wl["iters"]
    fr = gen.workload_frames(args.workload, code, frames=F, first=shard_first_frame(rank, F))
    graph = ldpc.Graph.from_code(code)
    plan = ldpc.WeightedBP(graph, F, T, cls_blk, nblk, checkpoint_every=wl["checkpoint"])
    llr = torch.from_numpy(fr.llr).to(dev)
    syn = torch.from_numpy(fr.syndrome).to(dev)
    x = torch.from_numpy(fr.x).to(dev)
    w = torch.ones((T, nblk), dtype=torch.float32, device=dev)
    app = torch.empty((F, code.n), dtype=torch.float32, device=dev)
    gw = torch.empty_like(w)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    lr = 20.0

    def step():
        plan.forward(llr, syn, w, app=app)
        loss, gapp = plan.loss(app, x)
        plan.backward(llr, syn, w, gapp, grad_w=gw)
        plan.sgd_step(w, gw, lr)
        return loss

    first_loss = float(step().item())
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg):
        loss_g = step()
    cgf = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cgf):
        plan.forward(llr, syn, w, app=app, save=False)
    for _ in range(max(3, args.warmup)):
        cg.replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cg.replay()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    last_loss = float(loss_g.item())
    fwd_ms = []
    for _ in range(max(3, args.steps)):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cgf.replay()
        e1.record(stream)
        e1.synchronize()
        fwd_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = job_time_ms(sum(ms), dist, dev)
    value = code.n * F * args.steps * world / (ms_total * 1e-3) / 1e6
    peak, peak_src = hbm_peak()
    B = wbp_bytes_per_frame_iter(code) * F * T
    achieved = B / (statistics.mean(ms) * 1e-3) / 1e9
    Bf = algorithmic_bytes_per_frame_iter(code) * F * T
    fwd_achieved = Bf / (statistics.mean(fwd_ms) * 1e-3) / 1e9
    every = wl["checkpoint"]
    # forward 2T (+1 interleaving Lch and the syndrome), loss 2, backward 1 + 3T + 2 per recomputed
    # iteration (+1 interleaving), SGD 1; FP32 QC plans interleave four frames per message
    x4 = 1
    n_launch = (2 * T + x4 + 2) + (1 + x4 + 3 * T + 2 * (T - (T + every - 1) // every)) + 1

    # context: the same step keeping every iteration (no recomputation; T x 117 MB more memory)
    keep_all = None
    if not args.lean and not compact:
        plan1 = ldpc.WeightedBP(graph, F, T, cls_blk, nblk, checkpoint_every=1)
        w1 = torch.ones_like(w)
        gw1 = torch.empty_like(w)

        def step1():
            plan1.forward(llr, syn, w1, app=app)
            l1, ga1 = plan1.loss(app, x)
            plan1.backward(llr, syn, w1, ga1, grad_w=gw1)
            plan1.sgd_step(w1, gw1, lr)

        step1()
        torch.cuda.synchronize()
        cg1 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg1):
            step1()
        for _ in range(3):
            cg1.replay()
        ms1 = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cg1.replay()
            e1.record(stream)
            e1.synchronize()
            ms1.append(e0.elapsed_time(e1))
        keep_all = {"checkpoint_every": 1, "ms_per_step": statistics.mean(ms1),
                    "mbit_s": code.n * F / (statistics.mean(ms1) * 1e-3) / 1e6,
                    "frac": B / (statistics.mean(ms1) * 1e-3) / 1e9 / peak}
        plan1.close()

    # end to end: inputs copied in from pinned host memory, the step replayed,
    # loss and weights read back, every step
    e2e = None
    if not args.lean and not compact:
        h_llr = torch.from_numpy(fr.llr).pin_memory()
        h_syn = torch.from_numpy(fr.syndrome).pin_memory()
        h_x = torch.from_numpy(fr.x).pin_memory()
        h_w = torch.empty_like(w, device="cpu").pin_memory()
        h_loss = torch.empty(1, dtype=torch.float32).pin_memory()
        e2e_steps = max(1, min(args.steps, 5))
        def e2e_step():
            llr.copy_(h_llr, non_blocking=True)
            syn.copy_(h_syn, non_blocking=True)
            x.copy_(h_x, non_blocking=True)
            cg.replay()
            h_loss.copy_(loss_g, non_blocking=True)
            h_w.copy_(w, non_blocking=True)
            stream.synchronize()
        e2e_step()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": code.n * F * e2e_steps / e2e_s / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(fr.llr.nbytes + fr.syndrome.nbytes + fr.x.nbytes),
               "d2h_bytes_per_step": int(4 + w.numel() * 4)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.lean and not compact:
        cls_csr = cls_blk[gen.qc_csr_edge_blocks(code)]
        v, cores, sample = wbp_oracle_rate(code, cls_csr, nblk, fr, T, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    if rank != 0:
        return
    line = {
        "metric": WBP_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["name"], "frames_per_gpu": F, "n": code.n, "m": code.m, "edges": int(code.edges),
                   "rate": code.rate, "beta": wl["beta"], "iters": T, "classes": nblk,
                   "checkpoint_every": every, "lr": lr,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "decoder state (~1 GB) > L2 (129 MB); L2 also flushed between steps",
                   "cuda_graph": "forward + loss + adjoint + SGD step, replayed once per step"},
        "loss_first_step": first_loss, "loss_after_steps": last_loss,
        "keep_every_iteration": keep_all,
        "forward_only": {"mbit_s": code.n * F / (statistics.mean(fwd_ms) * 1e-3) / 1e6,
                         "ms": statistics.mean(fwd_ms), "achieved_gbs": fwd_achieved,
                         "frac": fwd_achieved / peak},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_src, "traffic": None, "algorithmic_bytes_per_launch": B,
                     "kernel": "training step (wbp::cn_kernel / vn_*_kernel / wgrad_kernel)",
                     "timed": "whole graph replay"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": n_launch * args.steps,
        "clocks": clk,
    }
    plan.close()
    graph.close()
    if compact:
        return line
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    kind = gen.WORKLOADS.get(args.workload, {}).get("kind")
    if kind == "wbp":
        return run_wbp_reference(args) if args.impl == "reference" else run_wbp(args)
    batch = kind == "batch"
    if args.impl == "reference":
        run_batch_reference(args) if batch else run_reference(args)
    elif args.sweep:
        run_sweep(args)
    elif batch:
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
