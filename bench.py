"""Benchmark: batched syndrome decoding of the N=1054 lifted-product code on one GB300 (per rank).

One step = one decode launch over a batch of 65536 syndromes of the [[1054]] lifted-product code
(H_Z, 465 checks), i.i.d. X noise, plain normalized min-sum (alpha = 0.75), max 50 iterations,
early stop on.  Steps cycle through five pre-generated batches at p = 0.01 ... 0.05 (seeds
2001..2005), so consecutive steps read different inputs (5 x 30.5 MB of syndromes plus 69 MB of
outputs per step, more than the 129 MB L2).

Printed as one JSON line on rank 0:
  value        syndromes/s of the device-resident decode (inputs in HBM), whole job
  e2e          the same through qldpc_decode_host with pinned HOST buffers (copies timed)
  roofline     the decoder kernel against its binding on-chip roof (shared-memory message traffic),
               with the ALU-issue and HBM roofs beside it
  cpu_baseline the CPU oracle on a bounded sample of the same workload, all host cores
  clocks       SM clock and throttle reasons sampled during the timed region
  details      latency      single-shot (B = 1) end-to-end latency percentiles vs the 63 us
                            threshold: launch path and persistent server, flooding and layered
               paper_mode   the paper's timing conditions: BB-144 X+Z pair in one launch, FP32,
                            10 iterations, no early stop, B = 1, end to end (host buffers)
               bb_sweep     BB-144 / BB-288 pair, depolarizing p = 0.01..0.05, max 64, B = 1
               configs      HGP-400 1000-shot batch; LP-1054 at B = 64, 4096, 65536 (FP32/INT16/INT8)
               serving      the persistent server under a 40/40/20 mix of the N=400, 1054 and 288
                            codes, Poisson arrivals 20 us apart, per-code learned / plain weights
               precisions, layered, learned, soft_syndrome
  headline     the headline scalars, last on the line

``--impl reference`` times the CPU oracle (the reference arm) on the same workload instead.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

P_GRID = (0.01, 0.02, 0.03, 0.04, 0.05)
SEEDS = (2001, 2002, 2003, 2004, 2005)
BATCH = 65536
MAX_ITER = 50
CPU_SHOTS_PER_P = 8192       # oracle sample per error rate: about 20 core-seconds on the host
ALPHA = 0.75
LAT_P = 0.03
LAT_SHOTS = 10000
LAT_WARMUP = 200
THRESHOLD_US = 63.0
SERVE_REQUESTS = 1_000_000   # FP32 mixed stream (learned LP-1054, plain HGP-400 / BB-288)
SERVE_REQUESTS_FIXED = 100_000   # the INT16 / INT8 mixed streams and the saturated replays
SERVE_GAP_NS = 20000         # mean Poisson inter-arrival
SERVE_MIX = (0.4, 0.4, 0.2)  # N=400 HGP, N=1054 LP, N=288 BB (H_Z, i.i.d. X noise at p = 0.03)
LAT_SERVER_GAP_NS = 50000    # isolated single-shot requests through the server
LEARN_T = 20                 # unrolled learned iterations
LEARN_SHOTS = 2_000_000      # training shots
LEARN_BATCH = 4096
LEARN_LR = 1e-3
LEARN_P = (0.02, 0.06)       # per-shot rate range, training and evaluation
LEARN_EVAL = 1_000_000       # fresh evaluation shots
LEARN_SEEDS = (7, 99)        # training, evaluation
LEARN_INIT = 0.7             # initial weight of the configured run: the best constant scale untrained
# Algorithmic operations per edge per iteration: check step |q|, sign parity, three min/max, select,
# alpha multiply, sign apply; variable step add and extrinsic add.  Seven of them (all but the
# multiply and the two adds) are ALU-pipe work.
OPS_PER_EDGE_ITER = 10
ALU_OPS_PER_EDGE_ITER = 7
ALU_LANES_PER_SM = 128          # FP32/INT32 lanes per SM, one operation per lane per clock
ALU_PIPE_LANES_PER_SM = 64      # the ALU pipe (integer, logic, compare, min/max) is half rate
# Shared-memory message traffic per edge per iteration: the check step reads q and writes r, the
# variable step reads r and writes q (4 accesses of one message: 16 B FP32, 8 B INT16, 4 B INT8).
SMEM_ACCESSES_PER_EDGE_ITER = 4
MSG_BYTES = {"fp32": 4, "int16": 2, "int8": 1}
SMEM_BYTES_PER_CLK_PER_SM = 128  # 32 banks x 4 B

# DRAM bytes of one decoder launch on the benchmark batch (FP32), from ncu captures (the sum of
# dram__bytes_read.sum and dram__bytes_write.sum, mean over launches of the five rates), valid only for
# the kernel source they were taken on (sha256 prefix of that file); null once that source changes.
NCU_TRAFFIC = {"msa_batch_kernel": {"source": "msa_kernel.cuh", "source_sha16": "61e9fb1b9d8386fc",
                                    "bytes_per_launch": 39156923},
               "msa_packed_kernel": {"source": "msa_packed.cuh", "source_sha16": "7e5f890b9cc2f38f",
                                     "bytes_per_launch": 39615684}}

FALLBACK_HBM_GBS = 6800.0     # the profiling recipe's fallback when MEASURED_PEAKS.json is absent
WORKLOAD = "LP-1054 H_Z (465x1054, E=3720), iid X noise p=0.01..0.05, B=65536/step, max 50 it, alpha 0.75"


def measured_hbm():
    """(HBM copy GB/s, basis) from MEASURED_PEAKS.json beside this file, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM_GBS, "6.8 TB/s (of fallback)"


def bench_config(batch: int, world: int, precision: str) -> dict:
    """The workload description both arms print."""
    return {"workload": WORKLOAD, "global_batch": batch * world, "precision": precision,
            "l2": "inputs rotate over 5 batches (152 MB) + 69 MB outputs per step > 129 MB L2",
            "rates": "step i decodes the batch of p = 0.01, 0.02, ..., 0.05 at i mod 5; a step count "
                     "that is a multiple of 5 weights the five rates equally",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "int16", "int8"], default="fp32")
    ap.add_argument("--kernel", choices=["auto", "batch", "packed"], default="auto",
                    help="throughput kernel of the timed decode (packed: two fixed-point shots per word)")
    ap.add_argument("--profile", choices=["none", "server", "server-layered", "launch", "launch-layered"],
                    default="none",
                    help="only run single LP-1054 shots, each in a kernel launch of its own that ends by itself "
                         "(server: isolated requests to workers with a 50 us idle timeout; launch: "
                         "qldpc_decode_host with B = 1), for an ncu capture of that kernel, then exit")
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-latency", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--latency-shots", type=int, default=LAT_SHOTS)
    ap.add_argument("--serve-requests", type=int, default=SERVE_REQUESTS)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-layered", action="store_true")
    ap.add_argument("--no-precisions", action="store_true")
    ap.add_argument("--no-soft", action="store_true")
    ap.add_argument("--learned-train-shots", type=int, default=LEARN_SHOTS)
    ap.add_argument("--learned-eval-shots", type=int, default=LEARN_EVAL)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def kernel_traffic(kernel_name: str):
    """DRAM bytes of one launch of the named decoder kernel on the benchmark batch, from the ncu
    capture recorded for its current source, else None."""
    import hashlib
    rec = NCU_TRAFFIC.get(kernel_name)
    if rec is None:
        return None
    src = os.path.join(ROOT, "paper_2508_07879_gb300", "csrc", rec["source"])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return rec["bytes_per_launch"] if sha == rec["source_sha16"] else None


def shard(rank: int, world: int, batch: int):
    """Weak scaling over replicas: rank r decodes its own `batch` shots [r*batch, (r+1)*batch).

    Shots are independent and the sampler is counter-based, so the shards are disjoint and their
    union is the single-process sequence of world*batch shots; no data crosses ranks.
    """
    return rank * batch, batch


def reduce_max(x: float, device=None) -> float:
    """The slowest rank's value (the job's time); a no-op outside torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_batches(batch: int, first_shot: int):
    from paper_2508_07879_gb300 import workloads as w
    code = w.lp_code(1054)
    out = []
    for p, seed in zip(P_GRID, SEEDS):
        b = w.x_error_batch(code, p, batch, seed, first_shot=first_shot)
        out.append(b)
    return code, out


# ------------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout_s: float = 3.0):
        """Block until the sampler has produced a line (nvidia-smi takes a moment to start)."""
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout_s:
            time.sleep(0.01)

    def mark(self) -> int:
        return len(self.lines)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self, lo: int = 0, hi=None):
        """Median SM clock, max clock and throttle reasons of the samples lines[lo:hi] (the timed
        region when the caller marked it), or of every sample when that window is empty."""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        window = self.lines[lo:hi] if self.lines[lo:hi] else self.lines
        for line in window:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# CPU baseline / reference arm: the oracle as it stands, all host cores
# ------------------------------------------------------------------------------------------------
def oracle_rate(batches, shots_per_batch: int, precision: str, threads: int):
    import oracle
    oprec = {"fp32": "f32", "int16": "i16", "int8": "i8"}[precision]
    total = 0
    t0 = time.perf_counter()
    for b in batches:
        syn = b.syndromes[:shots_per_batch]
        oracle.msa(b.h.row_ptr, b.h.col_idx, b.h.m, b.h.n, syn, b.prior, MAX_ITER, ALPHA, oprec,
                   True, threads=threads)
        total += syn.shape[0]
    dt = time.perf_counter() - t0
    return total / dt, total, dt


def oracle_single_thread(batches, precision: str, shots: int = 2000):
    """The oracle on one core, one shot per call, on the p = 0.03 batch: shots/s and per-shot
    latency percentiles (host clock around each call, Python call overhead included)."""
    import oracle
    oprec = {"fp32": "f32", "int16": "i16", "int8": "i8"}[precision]
    b = batches[P_GRID.index(0.03)]
    shots = min(shots, b.syndromes.shape[0])
    lat = np.empty(shots)
    for i in range(shots):
        t0 = time.perf_counter_ns()
        oracle.msa(b.h.row_ptr, b.h.col_idx, b.h.m, b.h.n, b.syndromes[i:i + 1], b.prior, MAX_ITER, ALPHA,
                   oprec, True, threads=1)
        lat[i] = (time.perf_counter_ns() - t0) / 1e3
    return {"shots_per_s": shots / (lat.sum() / 1e6), "p50_us": float(np.percentile(lat, 50)),
            "p99_us": float(np.percentile(lat, 99)), "p999_us": float(np.percentile(lat, 99.9)),
            "shots": shots, "p": 0.03, "cores": 1}


def oracle_configs(threads: int) -> dict:
    """The oracle on each configuration's workload (the CPU baseline table): single-thread shots/s and
    per-shot latency percentiles (one shot per call), all-core shots/s, mean iterations.  HGP-400: 1000
    shots at p = 0.05, max 32; LP-1054: the p = 0.03 benchmark rate, max 50; BB-144 / BB-288: X+Z
    pairs (two decodes per shot) at p = 0.03 depolarizing, max 64.  FP32 and INT16."""
    import oracle
    from paper_2508_07879_gb300 import workloads as w
    out = {"cores": threads}
    cases = {"hgp400": (w.x_error_batch(w.hgp_code(400), 0.05, 1000, seed=1), None, 32, 300),
             "lp1054": (w.x_error_batch(w.lp_code(1054), 0.03, 4096, seed=2003), None, 50, 300)}
    for name in ("bb144", "bb288"):
        code = w.CONFIG_CODES[name]()
        ex, ez = w.depolarizing_errors(code.n, 0.03, 2000, seed=3003)
        prior = np.full(code.n, w.prior_llr(0.02), dtype=np.float32)
        cases[name] = ((code.hz_csr, w.syndromes(code.hz_csr, ex), prior),
                       (code.hx_csr, w.syndromes(code.hx_csr, ez), prior), 64, 300)
    for name, (a, b, max_iter, single) in cases.items():
        halves = [(a.h, a.syndromes, a.prior)] if b is None else [a, b]
        row = {}
        for prec, oprec in (("fp32", "f32"), ("int16", "i16")):
            shots = halves[0][1].shape[0]
            t0 = time.perf_counter()
            its = 0
            for h, syn, prior in halves:
                its += int(oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, syn, prior, max_iter, ALPHA, oprec, True,
                                      threads=threads)["iters"].sum())
            all_core = shots / (time.perf_counter() - t0)
            lat = np.empty(single)
            for i in range(single):
                t1 = time.perf_counter_ns()
                for h, syn, prior in halves:
                    oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, syn[i:i + 1], prior, max_iter, ALPHA, oprec, True,
                               threads=1)
                lat[i] = (time.perf_counter_ns() - t1) / 1e3
            row[prec] = {"all_core_shots_per_s": all_core, "single_thread_shots_per_s": single / (lat.sum() / 1e6),
                         "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                         "mean_iters": its / (shots * len(halves)), "shots": shots, "single_thread_shots": single}
        out[name] = row
    return out


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle, as it stands, on all host cores.  Each step decodes the
    same sample the cpu_baseline leg uses, 8192 shots of one rate's benchmark batch, cycling
    p = 0.01..0.05."""
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    per_step = CPU_SHOTS_PER_P
    code, batches = make_batches(per_step, 0)
    import oracle
    oracle.build()
    oprec = {"fp32": "f32", "int16": "i16", "int8": "i8"}[args.precision]

    def step(i):
        b = batches[i % len(batches)]
        oracle.msa(b.h.row_ptr, b.h.col_idx, b.h.m, b.h.n, b.syndromes, b.prior, MAX_ITER, ALPHA, oprec, True,
                   threads=threads)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i)
    dt = time.perf_counter() - t0
    value = args.steps * per_step / dt
    line = {
        "impl": "reference", "metric": "syndromes/sec", "value": value, "unit": "syndromes/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "int16": "i16", "int8": "i8"}[args.precision],
        "data": "synthetic",
        "config": bench_config(BATCH, world, args.precision),
        "cpu_baseline": {"value": value, "unit": "syndromes/s", "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} steps x {per_step} shots (the first {per_step} shots of the "
                                   f"benchmark batch of one rate per step, cycling p=0.01..0.05), the sample the "
                                   f"cpu_baseline leg of the GPU arm decodes",
                         "single_thread": oracle_single_thread(batches, args.precision, 500)},
        "e2e": {"value": value, "unit": "syndromes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist
    from paper_2508_07879_gb300 import build as libbuild
    libbuild.build()
    from paper_2508_07879_gb300 import qldpc

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.profile != "none":
        return profile_single(qldpc, args.profile, args.precision)
    B = args.batch
    first, _ = shard(rank, world, B)
    code, batches = make_batches(B, first_shot=first)       # each rank its own shots (weak scaling)
    h = batches[0].h
    graph = qldpc.Graph.from_csr(h)
    if args.kernel != "auto":
        graph.set_launch(args.kernel)
    dev = torch.device("cuda", local)
    syn_d = [torch.from_numpy(b.syndromes).to(dev) for b in batches]
    pri_d = [torch.from_numpy(b.prior).to(dev) for b in batches]
    out = (torch.empty((B, h.n), dtype=torch.uint8, device=dev),
           torch.empty(B, dtype=torch.int32, device=dev),
           torch.empty(B, dtype=torch.uint8, device=dev), None)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()

    # total iterations per batch (deterministic): the units of the algorithmic op count
    iters_per_batch = []
    with torch.cuda.stream(stream):
        for i in range(len(batches)):
            qldpc.decode(graph, syn_d[i], pri_d[i], MAX_ITER, ALPHA, args.precision, out=out, stream=stream)
            stream.synchronize()
            iters_per_batch.append(int(out[1].to(torch.int64).sum().item()))

    def step(i):
        j = i % len(batches)
        qldpc.decode(graph, syn_d[j], pri_d[j], MAX_ITER, ALPHA, args.precision, out=out, stream=stream)

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # clocks sampled every 20 ms from before the warm-up, so that the sampler is running when the
    # (short) timed region starts; the summary takes the samples of the timed region
    with ClockSampler(local) as clk:
        clk.wait_first()
        for i in range(args.warmup):
            step(i)
        stream.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        lo = clk.mark()
        e0.record(stream)
        for i in range(args.steps):
            step(i)
        e1.record(stream)
        stream.synchronize()
        time.sleep(0.03)                     # the sample that covers the region's end
        hi = clk.mark()
    torch.cuda.synchronize()
    ms = reduce_max(e0.elapsed_time(e1), dev)
    if world > 1:
        dist.barrier()
    ms_per_step = ms / args.steps
    value = world * B * args.steps / (ms / 1e3)
    launches = args.steps

    # roofline of the decoder kernel (one launch per step); the units of one launch are the
    # edge-iterations it runs: E x (iterations summed over its 65536 shots)
    props = torch.cuda.get_device_properties(dev)
    clocks = clk.summary(lo, hi)
    kernel_name = "msa_batch_kernel" if args.kernel == "batch" else "msa_packed_kernel"
    roofline = decoder_roofline(h, B, iters_per_batch, args.steps, ms_per_step, args.precision,
                                props.multi_processor_count, clocks["sm_max_mhz"] or 2070.0, kernel_name)

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(qldpc, graph, batches, args, B, world, dev)
    details = {}
    if rank == 0:
        if not args.no_latency:
            details["latency"] = measure_latency(qldpc, graph, code, args)
            details["paper_mode"] = measure_paper_mode(qldpc, args)
            details["bb_sweep"] = measure_bb_sweep(qldpc, args)
        if not args.no_precisions:
            details["precisions"] = measure_precisions(qldpc, graph, syn_d, pri_d, out, stream, B, args)
            details["configs"] = measure_configs(qldpc, graph, syn_d, pri_d, args)
        if not args.no_layered:
            details["layered"] = measure_layered(qldpc, graph, code, syn_d, pri_d, out, stream, B, args)
        learned_weights = None
        if not args.no_learned:
            details["learned"], learned_weights = measure_learned(qldpc, args)
        if not args.no_serving:
            details["serving"] = measure_serving(qldpc, args, learned_weights)
        if not args.no_soft:
            details["soft_syndrome"] = measure_soft_syndrome(qldpc, args)
    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        threads = os.cpu_count() or 1
        rate, n, dt = oracle_rate(batches, CPU_SHOTS_PER_P, args.precision, threads)
        cpu = {"value": rate, "unit": "syndromes/s", "cores": threads, "kind": "oracle",
               "sample": f"{n} shots ({CPU_SHOTS_PER_P} per p at p=0.01..0.05) of the same batches, "
                         f"{dt:.1f} s wall, about {dt * threads:.0f} core-s",
               "single_thread": oracle_single_thread(batches, args.precision),
               "per_config": oracle_configs(threads)}

    if rank == 0:
        line = {
            "metric": "syndromes/sec", "value": value, "unit": "syndromes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "int16": "i16", "int8": "i8"}[args.precision], "data": "synthetic",
            "config": bench_config(B, world, args.precision),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "mean_iters": sum(iters_per_batch) / (len(iters_per_batch) * B),
            "details": details,
        }
        line["headline"] = headline(line)      # last, so that the end of the line carries it
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def profile_single(qldpc, mode: str, precision: str, shots: int = 40):
    """Single LP-1054 shots (p = 0.03), each in a kernel launch of its own that ends by itself (the
    form an ncu capture of a persistent worker needs).  server / server-layered: isolated requests to
    workers that leave 50 us after their last request, each collected before the next is submitted;
    launch / launch-layered: qldpc_decode_host with B = 1."""
    from paper_2508_07879_gb300 import workloads as w
    b = w.x_error_batch(w.lp_code(1054), LAT_P, shots, seed=4003)
    g = qldpc.Graph.from_csr(b.h)
    layered = mode.endswith("layered")
    if mode.startswith("server"):
        with qldpc.Server([g], [b.prior], MAX_ITER, ALPHA, precision, blocks=[8], idle_timeout_s=5e-5,
                          layered=layered) as srv:
            for i in range(shots):
                t = srv.submit(0, b.syndromes[i])
                res = None
                deadline = time.time() + 10
                while res is None and time.time() < deadline:
                    res = srv.poll(0, t)
                if res is None:
                    raise RuntimeError("server request timed out")
                time.sleep(2e-4)                     # > idle timeout: the workers leave
    else:
        for i in range(shots):
            qldpc.decode_host(g, b.syndromes[i:i + 1], b.prior, MAX_ITER, ALPHA, precision, layered=layered)
    print(json.dumps({"profile": mode, "precision": precision, "shots": shots}), flush=True)
    return 0


def decoder_roofline(h, B, iters_per_batch, steps, ms_per_step, precision, sms, max_mhz, kernel_name):
    """Algorithmic work of one launch against the kernel's roofs.  The binding roof is the one with
    the longest time at peak: shared-memory message traffic (4 accesses of one message per edge and
    iteration, 32 banks x 4 B per clock per SM) or ALU issue (10 operations per edge and iteration,
    128 lanes per SM per clock); HBM (syndromes in, decisions, iterations and ok out) is far below
    either."""
    edge_iters = h.nnz * sum(iters_per_batch[i % len(iters_per_batch)] for i in range(steps)) / steps
    t = ms_per_step / 1e3
    smem_bytes = SMEM_ACCESSES_PER_EDGE_ITER * MSG_BYTES[precision] * edge_iters
    smem_peak = sms * SMEM_BYTES_PER_CLK_PER_SM * max_mhz * 1e6
    ops = OPS_PER_EDGE_ITER * edge_iters
    alu_peak = sms * ALU_LANES_PER_SM * max_mhz * 1e6
    hbm_bytes = (h.m + h.n + 5) * B
    hbm_gbs, hbm_basis = measured_hbm()
    hbm_peak = hbm_gbs * 1e9
    smem = {"achieved": round(smem_bytes / t / 1e9, 1), "peak": round(smem_peak / 1e9, 1), "unit": "GB/s",
            "frac": round(smem_bytes / t / smem_peak, 4), "time_at_peak_ms": round(smem_bytes / smem_peak * 1e3, 4),
            "bytes_per_launch": smem_bytes,
            "units": f"{SMEM_ACCESSES_PER_EDGE_ITER} x {MSG_BYTES[precision]} B per edge-iteration x E={h.nnz} x "
                     f"iterations run",
            "peak_basis": f"{sms} SMs x {SMEM_BYTES_PER_CLK_PER_SM} B/clk x {max_mhz:.0f} MHz (derived)"}
    alu = {"achieved": round(ops / t / 1e12, 3), "peak": round(alu_peak / 1e12, 3), "unit": "Tops/s",
           "frac": round(ops / t / alu_peak, 4), "time_at_peak_ms": round(ops / alu_peak * 1e3, 4),
           "ops_per_launch": ops,
           "units": f"{OPS_PER_EDGE_ITER} ALU ops per edge-iteration x E={h.nnz} x iterations run",
           "peak_basis": f"{sms} SMs x {ALU_LANES_PER_SM} lanes x {max_mhz:.0f} MHz (derived)",
           "op_mix_frac": round(ops / t / (alu_peak * (ALU_PIPE_LANES_PER_SM / ALU_LANES_PER_SM)
                                            * OPS_PER_EDGE_ITER / ALU_OPS_PER_EDGE_ITER), 4)}
    hbm = {"achieved": round(hbm_bytes / t / 1e9, 2), "peak": hbm_gbs, "unit": "GB/s",
           "frac": round(hbm_bytes / t / hbm_peak, 5), "bytes_per_launch": hbm_bytes, "peak_basis": hbm_basis}
    binding = "smem" if smem["time_at_peak_ms"] >= alu["time_at_peak_ms"] else "alu"
    top = smem if binding == "smem" else alu
    traffic = kernel_traffic(kernel_name) if (B == BATCH and precision == "fp32") else None
    return {"bound": binding, "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"],
            "frac": top["frac"], "traffic": traffic,
            "traffic_source": {"kind": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch",
                               "recorded": NCU_TRAFFIC.get(kernel_name), "current": traffic is not None},
            "kernel": kernel_name, "smem": smem, "alu": alu, "hbm": hbm}


def headline(line) -> dict:
    """The headline scalars (BASELINE metric: p99 single-shot latency vs 63 us, syndromes/s, learned
    vs plain LER), with the paper's own figures as context."""
    d = line.get("details", {})
    lat, pm, srv, lay, prec, lrn = (d.get(k) or {} for k in ("latency", "paper_mode", "serving", "layered",
                                                            "precisions", "learned"))
    g = lambda obj, *ks: _dig(obj, ks)
    out = {
        "syndromes_per_s": round(line["value"]),
        "e2e_syndromes_per_s": round(g(line, "e2e", "value") or 0) or None,
        "roofline": f"{line['roofline']['bound']} {line['roofline']['frac']}",
        "latency_p50_us": g(lat, "p50_us"), "latency_p99_us": g(lat, "p99_us"),
        "latency_p999_us": g(lat, "p999_us"), "latency_path": g(lat, "headline"),
        "layered_p99_us": g(lat, "layered_p99_us"),
        "launch_path_p99_us": g(lat, "launch_path", "fp32", "p99_us"),
        "paper_mode_bb144_pair_mean_us": g(pm, "launch_path", "mean_us"),
        "paper_mode_bb144_pair_p99_us": g(pm, "launch_path", "p99_us"),
        "serving_p99_us": g(srv, "fp32", "p99_us"), "serving_p999_us": g(srv, "fp32", "p999_us"),
        "serving_saturated_per_s": g(srv, "fp32", "saturated_shots_per_s"),
        "int16_syndromes_per_s": g(prec, "int16", "value"), "int8_syndromes_per_s": g(prec, "int8", "value"),
        "layered_syndromes_per_s": g(lay, "value"),
        "ler_plain_20": g(lrn, "ler", "plain_20"), "ler_learned_20": g(lrn, "ler", "learned_20"),
        "iters_plain_20": g(lrn, "mean_iters", "plain_20"), "iters_learned_20": g(lrn, "mean_iters", "learned_20"),
        "learned_minus_plain_ci95": g(lrn, "paired", "learned_20|plain_20", "ci95"),
        "paper_context": "avg 23.3-62.9 us end to end, FP32, 10 it., RTX 3090/4090 (Sec. 3); 63 us threshold",
    }
    return {k: (round(v, 3) if isinstance(v, float) else v) for k, v in out.items()}


def _dig(obj, keys):
    for k in keys:
        if not isinstance(obj, dict) or k not in obj:
            return None
        obj = obj[k]
    return obj


def measure_soft_syndrome(qldpc, args, q=0.01, shots=65536, evaluated=16384, steps=20):
    """Syndrome read errors: LP-1054 with data errors at p and every syndrome bit misread with
    probability q.  The hard decoder runs on H with the measured bits; the soft-syndrome decoder runs
    on the data-syndrome graph [H | I] with the read-error LLR ln((1-q)/q).  A shot succeeds when the
    residual data error has zero syndrome and commutes with every logical."""
    import torch
    from paper_2508_07879_gb300 import gf2
    from paper_2508_07879_gb300 import learned
    from paper_2508_07879_gb300 import workloads as w
    code = w.lp_code(1054)
    h = code.hz_csr
    gh, ga = qldpc.Graph.from_csr(h), qldpc.Graph.from_csr(w.data_syndrome_csr(h))
    lam = torch.full((h.m,), w.prior_llr(q), device="cuda")
    logicals = learned.z_logicals(code)
    out = {"workload": f"LP-1054 H_Z, data errors at p, syndrome read errors q={q}, {shots} shots per p",
           "success": "residual data error with zero syndrome, commuting with every logical",
           "evaluated_shots": evaluated}
    for p in (0.01, 0.03):
        e, es, s = w.noisy_syndrome_batch(h, p, q, shots, seed=5001)
        st = torch.from_numpy(s).cuda()
        gamma = torch.full((h.n,), w.prior_llr(p), device="cuda")
        row = {}
        for name in ("hard", "soft"):
            if name == "hard":
                run = lambda: qldpc.decode(gh, st, gamma, MAX_ITER, ALPHA)
            else:
                run = lambda: qldpc.decode_soft(ga, st, gamma, lam, MAX_ITER, ALPHA)
            res = run()
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            for _ in range(steps):
                run()
            ev[1].record()
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1]) / steps
            e_hat = res[0].cpu().numpy()
            iters, ok = (res[1], res[2]) if name == "hard" else (res[2], res[3])
            r = e[:evaluated] ^ e_hat[:evaluated]
            fail = w.syndromes(h, r).any(axis=1) | gf2.logical_failures(r, logicals).astype(bool)
            row[name] = {"success": float(1.0 - fail.mean()), "decoded_fraction": float(ok.float().mean().item()),
                         "mean_iters": float(iters.float().mean().item()), "syndromes_per_s": shots / (ms / 1e3)}
        out[f"p={p}"] = row
    return out


def measure_e2e(qldpc, graph, batches, args, B, world, dev):
    import torch
    import torch.distributed as dist
    h = batches[0].h
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    syn_h = [pin(b.syndromes) for b in batches]
    pri_h = [b.prior.copy() for b in batches]
    err = torch.empty((B, h.n), dtype=torch.uint8).pin_memory().numpy()
    it = torch.empty(B, dtype=torch.int32).pin_memory().numpy()
    ok = torch.empty(B, dtype=torch.uint8).pin_memory().numpy()
    graph.reserve(B)
    steps = max(3, min(args.steps, 40))
    for i in range(3):
        qldpc.decode_host(graph, syn_h[i % 5], pri_h[i % 5], MAX_ITER, ALPHA, args.precision, out=(err, it, ok))
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(steps):
        qldpc.decode_host(graph, syn_h[i % 5], pri_h[i % 5], MAX_ITER, ALPHA, args.precision, out=(err, it, ok))
    dt = reduce_max(time.perf_counter() - t0, dev)
    return {"value": world * B * steps / dt, "unit": "syndromes/s",
            "h2d_bytes_per_step": B * h.m + h.n * 4, "d2h_bytes_per_step": B * (h.n + 4 + 1),
            "steps": steps, "path": "qldpc_decode_host, pinned host buffers, synchronous per step"}


def measure_latency(qldpc, graph, code, args):
    """B = 1 end-to-end latency of LP-1054 shots at p = 0.03, host clock per shot.

    Launch path: page-locked syndrome -> one kernel launch that reads it and writes e_hat,
    iterations and ok into page-locked host memory -> stream synchronize.  Server path: the same
    shots as isolated requests to the persistent server (no launch, copy or synchronize).
    """
    import torch
    from paper_2508_07879_gb300 import workloads as w
    shots = args.latency_shots
    warm = min(LAT_WARMUP, max(shots // 10, 10))
    b = w.x_error_batch(code, LAT_P, shots + warm, seed=4003)
    h = b.h
    syn = torch.from_numpy(b.syndromes).pin_memory().numpy()
    err = torch.empty((1, h.n), dtype=torch.uint8).pin_memory().numpy()
    it = torch.empty(1, dtype=torch.int32).pin_memory().numpy()
    ok = torch.empty(1, dtype=torch.uint8).pin_memory().numpy()
    prior = b.prior.copy()
    lat = {}
    # the C entry point through ctypes with addresses computed once (the per-call cost of extracting
    # numpy pointers in Python is not the library's)
    syn0, pr0, e0, i0, o0 = (a.ctypes.data for a in (syn, prior, err, it, ok))
    for prec in ("fp32", "int16", "int8"):
        ts = np.empty(shots + warm)
        iters = np.empty(shots + warm, dtype=np.int32)
        pc = qldpc.PRECISIONS[prec]
        for i in range(shots + warm):
            t0 = time.perf_counter_ns()
            rc = qldpc.qldpc_decode_host(graph.handle, syn0 + i * h.m, 1, pr0, MAX_ITER, ALPHA, e0, i0, o0, pc, 0,
                                         None)
            ts[i] = (time.perf_counter_ns() - t0) / 1e3
            if rc:
                raise qldpc.QldpcError(rc, "qldpc_decode_host")
            iters[i] = it[0]
        x = ts[warm:]
        lat[prec] = {"p50_us": float(np.percentile(x, 50)), "p99_us": float(np.percentile(x, 99)),
                     "p999_us": float(np.percentile(x, 99.9)), "mean_us": float(x.mean()),
                     "max_iter_shots": int((iters[warm:] == MAX_ITER).sum())}
    out = {"metric": "p99 single-shot decode latency", "unit": "us", "threshold_us": THRESHOLD_US,
           "code": "LP-1054 H_Z", "p": LAT_P, "shots": shots, "max_iter": MAX_ITER,
           "launch_path": {"path": "qldpc_decode_host through ctypes, page-locked buffers read/written by the "
                                   "kernel, host clock, B=1", **lat}}
    # device-only time of the same single-shot launches: device-resident buffers, CUDA events
    # recorded on the launch stream around each launch (no host clock, copies or synchronize)
    import ctypes
    dev = torch.device("cuda")
    syn_d = torch.from_numpy(b.syndromes).to(dev)
    pri_d = torch.from_numpy(prior).to(dev)
    err_d = torch.empty((1, h.n), dtype=torch.uint8, device=dev)
    it_d = torch.empty(1, dtype=torch.int32, device=dev)
    ok_d = torch.empty(1, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    dev_lat = {}
    for prec in ("fp32", "int16", "int8"):
        pc = qldpc.PRECISIONS[prec]
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(shots + warm)]
        for i in range(shots + warm):
            ev[i][0].record(stream)
            rc = qldpc.qldpc_decode_ex(graph.handle, syn_d.data_ptr() + i * h.m, 1, pri_d.data_ptr(), MAX_ITER, ALPHA,
                                       err_d.data_ptr(), it_d.data_ptr(), ok_d.data_ptr(), None, pc, 0, sp)
            ev[i][1].record(stream)
            if rc:
                raise qldpc.QldpcError(rc, "qldpc_decode_ex")
        torch.cuda.synchronize()
        x = np.array([e0.elapsed_time(e1) * 1e3 for e0, e1 in ev[warm:]])
        dev_lat[prec] = {"p50_us": float(np.percentile(x, 50)), "p99_us": float(np.percentile(x, 99)),
                         "p999_us": float(np.percentile(x, 99.9)), "mean_us": float(x.mean())}
    out["device_path"] = {"path": "qldpc_decode_ex, device-resident buffers, CUDA events around each B=1 launch",
                          **dev_lat}
    # the same shots through the persistent server: requests 50 us apart, latency = result seen by
    # the host - scheduled arrival (host steady clock inside the C ABI)
    def served(layered):
        res = {}
        for prec in ("fp32", "int16", "int8"):
            with qldpc.Server([graph], [prior], MAX_ITER, ALPHA, prec, blocks=[8], ring_capacity=1024,
                              layered=layered) as srv:
                arrival = (np.arange(shots + warm) * LAT_SERVER_GAP_NS).astype(np.int64)
                _, iters, _, lat_ns = srv.replay(np.zeros(shots + warm, np.int32), list(syn), arrival)
            x = lat_ns[warm:] / 1e3
            res[prec] = {"p50_us": float(np.percentile(x, 50)), "p99_us": float(np.percentile(x, 99)),
                         "p999_us": float(np.percentile(x, 99.9)), "mean_us": float(x.mean()),
                         "mean_iters": float(iters[warm:].mean()),
                         "max_iter_shots": int((iters[warm:] == MAX_ITER).sum())}
        return res
    srv_lat = served(False)
    out["server_path"] = {"path": "qldpc_server_replay: persistent kernel, 8 LP workers, requests 50 us apart",
                          **srv_lat}
    out["server_layered_path"] = {"path": "the same requests to workers on the layered schedule (QLDPC_LAYERED): "
                                          "7 layers of at most 93 checks, one 96-thread block per request",
                                  **served(True)}
    out["p99_us"] = srv_lat["fp32"]["p99_us"]
    out["p50_us"] = srv_lat["fp32"]["p50_us"]
    out["p999_us"] = srv_lat["fp32"]["p999_us"]
    out["headline"] = "server_path fp32"
    out["layered_p99_us"] = out["server_layered_path"]["fp32"]["p99_us"]
    out["layered_per_code"] = measure_layered_codes(qldpc, args)
    return out


def layered_serving_code(name):
    """A serving code's H_Z in the row order the layered workers use: LP-1054 as built (7 layers);
    HGP-400 and BB-288 reordered by workloads.layer_order (15 -> 7 and 56 -> 3 layers).  Returns
    (H, row order) with the syndromes of H = the original syndromes[:, order]."""
    from paper_2508_07879_gb300 import workloads as w
    h = w.CONFIG_CODES[name]().hz_csr
    if name == "lp1054":
        return h, np.arange(h.m)
    order = w.layer_order(h)
    return w.csr_rows(h, order), order


def measure_layered_codes(qldpc, args, shots=None):
    """Isolated single-shot requests (50 us apart, p = 0.03) of each serving code to a layered-schedule
    server of that code alone, FP32, INT16 and INT8: latency percentiles and iterations."""
    from paper_2508_07879_gb300 import workloads as w
    shots = shots or max(1000, args.latency_shots // 2)
    warm = min(LAT_WARMUP, max(shots // 10, 10))
    res = {}
    for name in ("hgp400", "lp1054", "bb288"):
        h, order = layered_serving_code(name)
        b = w.x_error_batch(w.CONFIG_CODES[name](), LAT_P, shots + warm, seed=4103)
        syn = np.ascontiguousarray(b.syndromes[:, order])
        g = qldpc.Graph.from_csr(h)
        layers, widest = g.layers(widest=True)
        row = {"layers": layers, "widest_layer": widest, "row_order": "natural" if name == "lp1054" else "layer_order"}
        for prec in ("fp32", "int16", "int8"):
            with qldpc.Server([g], [b.prior], MAX_ITER, ALPHA, prec, blocks=[8], ring_capacity=1024,
                              layered=True) as srv:
                arrival = (np.arange(shots + warm) * LAT_SERVER_GAP_NS).astype(np.int64)
                _, iters, ok, lat_ns = srv.replay(np.zeros(shots + warm, np.int32), list(syn), arrival)
            x = lat_ns[warm:] / 1e3
            row[prec] = {"p50_us": float(np.percentile(x, 50)), "p99_us": float(np.percentile(x, 99)),
                         "p999_us": float(np.percentile(x, 99.9)), "mean_iters": float(iters[warm:].mean()),
                         "decoded_fraction": float(ok[warm:].mean()),
                         "max_iter_shots": int((iters[warm:] == MAX_ITER).sum())}
        res[name] = row
        g.close()
    return res


def pair_host_call(qldpc, gz, gx, sx, sz, prior, outs, max_iter, early_stop):
    """call(i): qldpc_decode_pair_host on shot i of the page-locked syndrome arrays sx / sz, through
    ctypes with every address computed once."""
    (ex, ix, ox), (ez, iz, oz) = outs
    a = [x.ctypes.data for x in (sx, sz, prior, ex, ez, ix, iz, ox, oz)]
    mz, mx = gz.m, gx.m
    flags = 0 if early_stop else qldpc.QLDPC_NO_EARLY_STOP
    hz, hx = gz.handle, gx.handle
    fn = qldpc.qldpc_decode_pair_host

    def call(i):
        rc = fn(hz, hx, a[0] + i * mz, a[1] + i * mx, 1, a[2], a[2], max_iter, ALPHA, a[3], a[4], a[5], a[6], a[7],
                a[8], qldpc.QLDPC_FP32, flags, None)
        if rc:
            raise qldpc.QldpcError(rc, "qldpc_decode_pair_host")
    return call


def measure_paper_mode(qldpc, args, shots=10000, warm=100):
    """The paper's timing conditions (Sec. 3): X and Z decoded in one kernel, FP32, 10 iterations,
    no early stop, B = 1, average end-to-end latency including the transfers.  BB-144 ([[144,12,12]],
    the one code of the paper's set that is reproducible here), depolarizing p = 0.03; host clock
    around qldpc_decode_pair_host with page-locked buffers (no copies: the kernel reads and writes
    host memory), and the same pairs as two concurrent requests to the persistent server."""
    import torch
    from paper_2508_07879_gb300 import workloads as w
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    out = {"conditions": "FP32, 10 iterations, no early stop, B = 1, X+Z, end to end (host buffers)",
           "paper": "[[144,12,12]] among the BB codes: about 28 us (RTX 4090) / 35 us (RTX 3090) average, Sec. 3"}
    for name in ("bb144", "bb288"):
        code = w.CONFIG_CODES[name]()
        gz, gx = qldpc.Graph.from_csr(code.hz_csr), qldpc.Graph.from_csr(code.hx_csr)
        ex, ez = w.depolarizing_errors(code.n, 0.03, shots + warm, seed=3203)
        sx, sz = pin(w.syndromes(code.hz_csr, ex)), pin(w.syndromes(code.hx_csr, ez))
        prior = np.full(code.n, w.prior_llr(2 * 0.03 / 3), dtype=np.float32)
        outs = tuple((pin(np.zeros((1, code.n), np.uint8)), pin(np.zeros(1, np.int32)), pin(np.zeros(1, np.uint8)))
                     for _ in range(2))
        call = pair_host_call(qldpc, gz, gx, sx, sz, prior, outs, 10, False)
        ts = np.empty(shots + warm)
        for i in range(shots + warm):
            t0 = time.perf_counter_ns()
            call(i)
            ts[i] = (time.perf_counter_ns() - t0) / 1e3
        x = ts[warm:]
        row = {"launch_path": {"path": "qldpc_decode_pair_host through ctypes, one launch for X and Z",
                               "mean_us": float(x.mean()), "p50_us": float(np.percentile(x, 50)),
                               "p99_us": float(np.percentile(x, 99)), "p999_us": float(np.percentile(x, 99.9))}}
        with qldpc.Server([gz, gx], [prior, prior], 10, ALPHA, "fp32", early_stop=False, blocks=[8, 8],
                          ring_capacity=1024) as srv:
            n = shots + warm
            codes = np.tile(np.array([0, 1], np.int32), n)
            syn = [r for pair in zip(sx, sz) for r in pair]
            arrival = np.repeat(np.arange(n) * LAT_SERVER_GAP_NS, 2).astype(np.int64)
            _, iters, _, lat_ns = srv.replay(codes, syn, arrival)
        pair_us = np.maximum(lat_ns[0::2], lat_ns[1::2])[warm:] / 1e3
        row["server_path"] = {"path": "the X and Z halves as two requests at the same instant to the persistent "
                                      "server; latency = the later of the two",
                              "mean_us": float(pair_us.mean()), "p50_us": float(np.percentile(pair_us, 50)),
                              "p99_us": float(np.percentile(pair_us, 99)),
                              "p999_us": float(np.percentile(pair_us, 99.9))}
        row["shots"] = shots
        out[name] = row
        if name == "bb144":
            out["launch_path"] = row["launch_path"]
        gz.close()
        gx.close()
    return out


def measure_bb_sweep(qldpc, args, shots=10000, warm=100):
    """BB-144 and BB-288 single-shot latency sweep: depolarizing noise at p = 0.01..0.05 split into
    its X and Z parts, both halves decoded in one launch (max 64 iterations, early stop), B = 1,
    host clock around qldpc_decode_pair_host with page-locked buffers."""
    import torch
    from paper_2508_07879_gb300 import workloads as w
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    shots = min(shots, max(1000, args.latency_shots))
    out = {"max_iter": 64, "shots_per_p": shots,
           "path": "qldpc_decode_pair_host through ctypes (X+Z in one launch), FP32, page-locked buffers; "
                   "server_path: the two halves as two requests at the same instant, latency = the later"}
    for ci, name in enumerate(("bb144", "bb288")):
        code = w.CONFIG_CODES[name]()
        gz, gx = qldpc.Graph.from_csr(code.hz_csr), qldpc.Graph.from_csr(code.hx_csr)
        outs = tuple((pin(np.zeros((1, code.n), np.uint8)), pin(np.zeros(1, np.int32)), pin(np.zeros(1, np.uint8)))
                     for _ in range(2))
        rows = {}
        for pi, p in enumerate(P_GRID):
            ex, ez = w.depolarizing_errors(code.n, p, shots + warm, seed=3001 + 100 * ci + pi)
            sx, sz = pin(w.syndromes(code.hz_csr, ex)), pin(w.syndromes(code.hx_csr, ez))
            prior = np.full(code.n, w.prior_llr(2 * p / 3), dtype=np.float32)
            ts = np.empty(shots + warm)
            both_ok = np.empty(shots + warm, dtype=bool)
            its = np.empty(shots + warm)
            call = pair_host_call(qldpc, gz, gx, sx, sz, prior, outs, 64, True)
            for i in range(shots + warm):
                t0 = time.perf_counter_ns()
                call(i)
                ts[i] = (time.perf_counter_ns() - t0) / 1e3
                both_ok[i] = outs[0][2][0] and outs[1][2][0]
                its[i] = max(outs[0][1][0], outs[1][1][0])
            x = ts[warm:]
            rows[f"p={p}"] = {"mean_us": float(x.mean()), "p50_us": float(np.percentile(x, 50)),
                              "p99_us": float(np.percentile(x, 99)), "p999_us": float(np.percentile(x, 99.9)),
                              "decoded_fraction": float(both_ok[warm:].mean()),
                              "mean_max_iters": float(its[warm:].mean())}
            # the same pairs as two requests at the same instant to the persistent server
            with qldpc.Server([gz, gx], [prior, prior], 64, ALPHA, "fp32", blocks=[8, 8], ring_capacity=1024) as srv:
                n = shots + warm
                codes = np.tile(np.array([0, 1], np.int32), n)
                arrival = np.repeat(np.arange(n) * LAT_SERVER_GAP_NS, 2).astype(np.int64)
                _, _, _, lat_ns = srv.replay(codes, [r for pair in zip(sx, sz) for r in pair], arrival)
            y = np.maximum(lat_ns[0::2], lat_ns[1::2])[warm:] / 1e3
            rows[f"p={p}"]["server_path"] = {"mean_us": float(y.mean()), "p50_us": float(np.percentile(y, 50)),
                                             "p99_us": float(np.percentile(y, 99)),
                                             "p999_us": float(np.percentile(y, 99.9))}
        out[name] = rows
        gz.close()
        gx.close()
    return out


def measure_configs(qldpc, graph, syn_d, pri_d, args, steps=50):
    """Config 1 (HGP-400, 1000 shots at p = 0.05, max 32, FP32 and INT16) and config 2 at B = 64
    and 4096 (LP-1054, the benchmark batches, max 50): device throughput (CUDA events over repeated
    launches), decoded fraction and mean iterations."""
    import torch
    from paper_2508_07879_gb300 import workloads as w

    def timed(g, s, p, max_iter, prec):
        res = qldpc.decode(g, s, p, max_iter, ALPHA, prec)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(steps):
            qldpc.decode(g, s, p, max_iter, ALPHA, prec)
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / steps
        return {"ms_per_launch": ms, "syndromes_per_s": s.shape[0] / (ms / 1e3),
                "decoded_fraction": float(res[2].float().mean().item()),
                "mean_iters": float(res[1].float().mean().item())}

    out = {}
    b = w.x_error_batch(w.hgp_code(400), 0.05, 1000, seed=1)
    g = qldpc.Graph.from_csr(b.h)
    s, p = torch.from_numpy(b.syndromes).cuda(), torch.from_numpy(b.prior).cuda()
    out["c1_hgp400_b1000"] = {prec: timed(g, s, p, 32, prec) for prec in ("fp32", "int16", "int8")}
    g.close()
    for B in (64, 4096):
        rows = {}
        for prec in ("fp32", "int16", "int8"):
            per_p = [timed(graph, syn_d[j][:B].contiguous(), pri_d[j], MAX_ITER, prec) for j in range(len(syn_d))]
            ms = sum(r["ms_per_launch"] for r in per_p) / len(per_p)
            rows[prec] = {"syndromes_per_s": B / (ms / 1e3), "ms_per_launch": ms,
                          "decoded_fraction": sum(r["decoded_fraction"] for r in per_p) / len(per_p),
                          "mean_iters": sum(r["mean_iters"] for r in per_p) / len(per_p)}
        out[f"c2_lp1054_b{B}"] = rows
    return out


def measure_serving(qldpc, args, learned_weights=None):
    """Config 5: Poisson arrivals (mean gap 20 us) of syndrome rounds mixed 40/40/20 from the N=400,
    1054 and 288 codes (H_Z, iid X noise at p = 0.03) through one persistent server whose workers
    serve every code.  FP32 with per-code weights (LP-1054 learned, when the learned section trained
    them, then the plain fallback; HGP-400 and BB-288 plain), 10^6 requests; FP32 plain, INT16 and
    INT8 over the first 10^5 requests of the same stream.  Requests cycle through 10^5 distinct
    syndromes per code.  Latency = completion seen by the host - scheduled arrival."""
    from paper_2508_07879_gb300 import workloads as w
    rng = np.random.default_rng(5005)
    n = args.serve_requests
    codes = rng.choice(3, size=n, p=list(SERVE_MIX)).astype(np.int32)
    arrival = np.cumsum(rng.exponential(SERVE_GAP_NS, size=n)).astype(np.int64)
    names = ("hgp400", "lp1054", "bb288")
    graphs, priors, rows = [], [], []
    for ci, name in enumerate(names):
        count = max(1, min(int((codes == ci).sum()), 100_000))
        b = w.x_error_batch(w.CONFIG_CODES[name](), 0.03, count, seed=5001 + ci)
        graphs.append(qldpc.Graph.from_csr(b.h))
        priors.append(b.prior)
        rows.append(b.syndromes)
    cursor = [0, 0, 0]
    syn = []
    for c in codes:
        syn.append(rows[c][cursor[c] % rows[c].shape[0]])
        cursor[c] += 1
    out = {"workload": "40/40/20 HGP-400 / LP-1054 / BB-288 (H_Z, iid X, p=0.03), Poisson mean gap 20 us",
           "requests": n, "max_iter": MAX_ITER}
    runs = [("fp32", "fp32", n, learned_weights is not None), ("fp32_plain", "fp32", SERVE_REQUESTS_FIXED, False),
            ("int16", "int16", SERVE_REQUESTS_FIXED, False), ("int8", "int8", SERVE_REQUESTS_FIXED, False)]
    for key, prec, count, use_learned in runs:
        count = min(count, n)
        if use_learned:
            graphs[1].set_weights(learned_weights)
        with qldpc.Server(graphs, priors, MAX_ITER, ALPHA, prec, ring_capacity=4096, learned=use_learned) as srv:
            info = srv.info()
            _, iters, _, lat_ns, workers = srv.replay(codes[:count], syn[:count], arrival[:count], timeout_s=60.0,
                                                     want_workers=True)
            sat = min(count, SERVE_REQUESTS_FIXED)
            t0 = time.perf_counter()
            srv.replay(codes[:sat], syn[:sat], np.zeros(sat, np.int64), timeout_s=60.0)
            dt = time.perf_counter() - t0
        if use_learned:
            graphs[1].set_weights(None)
        x = lat_ns / 1e3
        per = {}
        for ci, name in enumerate(names):
            sel = codes[:count] == ci
            xs = x[sel]
            per[name] = {"p50_us": float(np.percentile(xs, 50)), "p99_us": float(np.percentile(xs, 99)),
                         "mean_iters": float(iters[sel].mean()), "distinct_workers": int(len(set(workers[sel].tolist())))}
        out[key] = {"requests": count, "p50_us": float(np.percentile(x, 50)), "p99_us": float(np.percentile(x, 99)),
                    "p999_us": float(np.percentile(x, 99.9)), "mean_us": float(x.mean()), "per_code": per,
                    "saturated_shots_per_s": sat / dt, "saturated_requests": sat,
                    "offered_per_s": 1e9 / SERVE_GAP_NS, "workers": info["workers"],
                    "threads_per_block": info["threads_per_block"], "smem_per_block": info["smem_per_block"],
                    "weights": "LP-1054 learned (configured training run), others plain" if use_learned else "plain"}
    for g in graphs:
        g.close()
    return out


def measure_precisions(qldpc, graph, syn_d, pri_d, out, stream, B, args, steps=100):
    """Flooding decode of the benchmark's batches in each precision: throughput and decoded fraction."""
    import torch
    res = {}
    for name in ("fp32", "int16", "int8", "fp32_one_shot", "int16_one_shot", "int8_one_shot"):
        prec = name.split("_")[0]
        graph.set_launch("batch" if name.endswith("_one_shot") else "auto")
        ok = iters = 0
        with torch.cuda.stream(stream):
            for j in range(len(syn_d)):
                qldpc.decode(graph, syn_d[j], pri_d[j], MAX_ITER, ALPHA, prec, out=out, stream=stream)
                stream.synchronize()
                ok += int(out[2].to(torch.int64).sum().item())
                iters += int(out[1].to(torch.int64).sum().item())
            for i in range(5):
                qldpc.decode(graph, syn_d[i % len(syn_d)], pri_d[i % len(syn_d)], MAX_ITER, ALPHA, prec, out=out,
                             stream=stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            stream.synchronize()
            e0.record(stream)
            for i in range(steps):
                j = i % len(syn_d)
                qldpc.decode(graph, syn_d[j], pri_d[j], MAX_ITER, ALPHA, prec, out=out, stream=stream)
            e1.record(stream)
            stream.synchronize()
        res[name] = {"value": B * steps / (e0.elapsed_time(e1) / 1e3), "unit": "syndromes/s",
                     "decoded_fraction": ok / (len(syn_d) * B), "mean_iters": iters / (len(syn_d) * B),
                     "kernel": "msa_batch_kernel (one shot per block)" if name.endswith("_one_shot")
                     else "msa_packed_kernel (two shots per block)"}
    graph.set_launch("auto")
    return res


def measure_layered(qldpc, graph, code, syn_d, pri_d, out, stream, B, args, steps=100):
    """The layered schedule on the benchmark's own batches (device throughput, iterations) and on the
    single-shot workload of the latency measurement (launch path)."""
    import torch
    from paper_2508_07879_gb300 import workloads as w
    res = {"schedule": "row-serial in ascending check order, checks without shared variables in parallel"}
    iters = ok = 0
    with torch.cuda.stream(stream):
        for j in range(len(syn_d)):
            qldpc.decode(graph, syn_d[j], pri_d[j], MAX_ITER, ALPHA, args.precision, out=out, stream=stream,
                         layered=True)
            stream.synchronize()
            iters += int(out[1].to(torch.int64).sum().item())
            ok += int(out[2].to(torch.int64).sum().item())
        for i in range(5):
            qldpc.decode(graph, syn_d[i % len(syn_d)], pri_d[i % len(syn_d)], MAX_ITER, ALPHA, args.precision,
                         out=out, stream=stream, layered=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        for i in range(steps):
            j = i % len(syn_d)
            qldpc.decode(graph, syn_d[j], pri_d[j], MAX_ITER, ALPHA, args.precision, out=out, stream=stream,
                         layered=True)
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1) / steps
    res["value"] = B / (ms / 1e3)
    res["unit"] = "syndromes/s"
    res["ms_per_step"] = ms
    res["mean_iters"] = iters / (len(syn_d) * B)
    res["decoded_fraction"] = ok / (len(syn_d) * B)
    if args.no_latency:
        return res
    # single shot, launch path: the shots of the flooding latency measurement
    shots = args.latency_shots
    warm = min(LAT_WARMUP, max(shots // 10, 10))
    b = w.x_error_batch(code, LAT_P, shots + warm, seed=4003)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    syn = pin(b.syndromes)
    err, it, okk = pin(np.zeros((1, b.h.n), np.uint8)), pin(np.zeros(1, np.int32)), pin(np.zeros(1, np.uint8))
    ts = np.empty(shots + warm)
    its = np.empty(shots + warm, dtype=np.int32)
    prior = np.ascontiguousarray(b.prior, dtype=np.float32)
    syn0, pr0, e0, i0, o0 = (a.ctypes.data for a in (syn, prior, err, it, okk))
    for i in range(shots + warm):
        t0 = time.perf_counter_ns()
        rc = qldpc.qldpc_decode_host(graph.handle, syn0 + i * b.h.m, 1, pr0, MAX_ITER, ALPHA, e0, i0, o0,
                                     qldpc.QLDPC_FP32, qldpc.QLDPC_LAYERED, None)
        ts[i] = (time.perf_counter_ns() - t0) / 1e3
        if rc:
            raise qldpc.QldpcError(rc, "qldpc_decode_host")
        its[i] = it[0]
    x = ts[warm:]
    res["latency_launch_path_fp32"] = {"p50_us": float(np.percentile(x, 50)), "p99_us": float(np.percentile(x, 99)),
                                       "p999_us": float(np.percentile(x, 99.9)), "mean_us": float(x.mean()),
                                       "mean_iters": float(its[warm:].mean()), "shots": int(shots), "p": LAT_P}
    return res


def measure_learned(qldpc, args):
    """Config 4: learned normalized min-sum on LP-1054 (H_Z), trained and evaluated on the device,
    once with each training loss (BCE against the sampled error; BCE of the soft syndrome)."""
    import torch
    from paper_2508_07879_gb300 import learned
    from paper_2508_07879_gb300 import workloads as w
    code = w.lp_code(1054)
    h = code.hz_csr
    prior = np.full(h.n, w.prior_llr(0.04), dtype=np.float32)   # one prior at the centre of the range
    g = qldpc.Graph.from_csr(h)
    logicals = learned.z_logicals(code)
    steps = args.learned_train_shots // LEARN_BATCH
    edge_iters = LEARN_BATCH * LEARN_T * h.nnz
    out = {
        "workload": "LP-1054 H_Z, iid X noise, p uniform in [0.02, 0.06) per shot, prior ln(0.96/0.04)",
        "T": LEARN_T, "train_shots": steps * LEARN_BATCH, "batch": LEARN_BATCH, "lr": LEARN_LR,
        "eval_shots": args.learned_eval_shots,
        "decoders": "plain_K: alpha 0.75, max K iterations; learned_20: 20 learned iterations alone; "
                    "learned_20_fallback_K: then plain min-sum from the prior for up to K iterations",
        "losses": {"error": "mean over iterations and variables of BCE(sigma(-Q), e)",
                   "syndrome": "mean over iterations and checks of -log P(soft syndrome bit = s)"},
    }
    plain = {"plain_20": (20, False), "plain_50": (50, False)}
    res = learned.evaluate(g, prior, logicals, plain, shots=args.learned_eval_shots, p_lo=LEARN_P[0],
                           p_hi=LEARN_P[1], seed=LEARN_SEEDS[1])
    ler = {k: v["ler"] for k, v in res.items()}
    iters = {k: v["mean_iters"] for k, v in res.items()}
    # the plain decoder at the initial weight of the configured run, for context
    res = learned.evaluate(g, prior, logicals, {"plain_20": (20, False)}, shots=args.learned_eval_shots,
                           p_lo=LEARN_P[0], p_hi=LEARN_P[1], seed=LEARN_SEEDS[1], alpha=LEARN_INIT)
    ler[f"plain_20_alpha{LEARN_INIT}"] = res["plain_20"]["ler"]
    iters[f"plain_20_alpha{LEARN_INIT}"] = res["plain_20"]["mean_iters"]
    paired = {}
    configured = None
    # (key prefix, loss, Adam lr, initial weight): the configured run (syndrome loss, lr 1e-3, started
    # at the best constant scale of the untrained sweep), the same from 0.75, a larger step, the error loss
    runs = (("", "syndrome", LEARN_LR, LEARN_INIT), ("init0.75_", "syndrome", LEARN_LR, 0.75),
            ("lr1e-2_", "syndrome", 1e-2, 0.75), ("error_loss_", "error", LEARN_LR, 0.75))
    for prefix, loss, lr, init in runs:
        model = learned.NeuralMinSum(h, prior, T=LEARN_T, init=init, max_batch=LEARN_BATCH, graph=g, loss=loss)
        # kernel times of one training step, events on the launching (current) stream
        err, syn = qldpc.sample_errors(g, LEARN_SEEDS[0] + 1000, 0, LEARN_BATCH, *LEARN_P)
        gl = torch.full((LEARN_BATCH,), 1.0 / LEARN_BATCH, device=syn.device)
        w0 = model.weights.detach()
        for _ in range(3):
            qldpc.nms_forward(g, syn, err, model.prior, w0, model.workspace, loss=loss)
            qldpc.nms_backward(g, syn, err, model.prior, LEARN_T, gl, model.workspace, loss=loss)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        tf = tb = 0.0
        reps = 10
        for _ in range(reps):
            ev[0].record()
            qldpc.nms_forward(g, syn, err, model.prior, w0, model.workspace, loss=loss)
            ev[1].record()
            qldpc.nms_backward(g, syn, err, model.prior, LEARN_T, gl, model.workspace, loss=loss)
            ev[2].record()
            torch.cuda.synchronize()
            tf += ev[0].elapsed_time(ev[1])
            tb += ev[1].elapsed_time(ev[2])
        tf, tb = tf / reps, tb / reps
        # training: sampling, forward, backward and Adam per step, wall clock
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist = model.train(shots=args.learned_train_shots, batch=LEARN_BATCH, p_lo=LEARN_P[0], p_hi=LEARN_P[1],
                           seed=LEARN_SEEDS[0], lr=lr, record_every=50)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        model.publish()
        t0 = time.perf_counter()
        res = learned.evaluate(g, prior, logicals, {"learned_20": (0, True), "learned_20_fallback_30": (30, True),
                                                    "learned_20_fallback_50": (50, True), "plain_20": (20, False),
                                                    "plain_50": (50, False)},
                               shots=args.learned_eval_shots, p_lo=LEARN_P[0], p_hi=LEARN_P[1], seed=LEARN_SEEDS[1],
                               paired=(("learned_20", "plain_20"), ("learned_20_fallback_50", "plain_50")))
        eval_s = time.perf_counter() - t0
        for k, v in res.items():
            if k == "paired":
                paired.update({prefix + pk: pv for pk, pv in v.items()})
            elif not k.startswith("plain"):
                ler[prefix + k] = v["ler"]
                iters[prefix + k] = v["mean_iters"]
        if not prefix:
            configured = model.weights.detach().cpu().numpy().copy()
        wmean = model.weights.detach().mean(dim=1).cpu().numpy()
        out[(prefix or "syndrome_") + "training"] = {
            "loss": loss, "lr": lr, "init": init, "mean_weight_per_iteration": [round(float(x), 4) for x in wmean],
            "train_s": train_s, "train_shots_per_s": steps * LEARN_BATCH / train_s,
            "loss_first": float(hist[0]) if len(hist) else None, "loss_last": float(hist[-1]) if len(hist) else None,
            "step_kernel_ms": {"forward": tf, "backward_and_reduce": tb},
            "train_edge_iters_per_s": {"forward": edge_iters / (tf / 1e3), "backward": edge_iters / (tb / 1e3)},
            "eval_s": eval_s,
        }
        g.set_weights(None)
    out["ler"] = ler
    out["mean_iters"] = iters
    out["paired"] = paired
    out["learned_keys"] = (f"learned_*: syndrome loss, lr 1e-3, weights started at {LEARN_INIT} (the configured run); "
                           "init0.75_learned_*: the same started at 0.75; lr1e-2_learned_*: syndrome loss, lr 1e-2; "
                           "error_loss_learned_*: error loss, lr 1e-3; paired: learned minus plain LER on the same "
                           "shots with its 95 % CI (discordant-shot counts)")
    return out, configured


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
