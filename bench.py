"""Benchmark: batched syndrome decoding of the N=1054 lifted-product code on one GB300 (per rank).

One step = one decode launch over a batch of 65536 syndromes of the [[1054]] lifted-product code
(H_Z, 465 checks), i.i.d. X noise, plain normalized min-sum (alpha = 0.75), max 50 iterations,
early stop on.  Steps cycle through five pre-generated batches at p = 0.01 ... 0.05 (seeds
2001..2005), so consecutive steps read different inputs (5 x 30.5 MB of syndromes plus 69 MB of
outputs per step, more than the 129 MB L2).

Printed as one JSON line on rank 0:
  value        syndromes/s of the device-resident decode (inputs in HBM), whole job
  e2e          the same through qldpc_decode_host with pinned HOST buffers (copies timed)
  latency      single-shot (B = 1) end-to-end latency percentiles vs the 63 us threshold, through
               the launch path (qldpc_decode_host) and the persistent server (qldpc_server_*)
  serving      the persistent server under a 40/40/20 mix of the N=400, 1054 and 288 codes with
               Poisson arrivals 20 us apart: latency percentiles and the saturated request rate
  precisions   the same batches decoded in FP32, INT16 and INT8 (device throughput, decoded fraction)
  layered      the row-serial (layered) schedule on the same batches and shots: device throughput,
               mean iterations, decode success, and single-shot latency through qldpc_decode_host
  learned      the learned (neural) min-sum on the same code: training time and kernel times on
               2e6 device-sampled shots (T = 20, batch 4096, Adam lr 1e-3, p uniform in
               [0.02, 0.06]), then logical error rates of learned and plain decoding on 1e6 fresh
               shots
  roofline     the decoder kernel against the SM integer/FP32 issue roof ("alu")
  cpu_baseline the CPU oracle on a bounded sample of the same workload, all host cores
  clocks       SM clock and throttle reasons sampled during the timed region

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
SERVE_REQUESTS = 100000
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
# Algorithmic operations per edge per iteration: check step |q|, sign parity, three min/max, select,
# alpha multiply, sign apply; variable step add and extrinsic add.  Seven of them (all but the
# multiply and the two adds) are ALU-pipe work.
OPS_PER_EDGE_ITER = 10
ALU_OPS_PER_EDGE_ITER = 7
ALU_LANES_PER_SM = 128          # FP32/INT32 lanes per SM, one operation per lane per clock
ALU_PIPE_LANES_PER_SM = 64      # the ALU pipe (integer, logic, compare, min/max) is half rate

# DRAM traffic of one decoder launch from an ncu capture, valid only for the kernel source it was
# measured on (profiles/msa_batch_lp1054_b65536_fp32.md); reported as null once the source changes.
NCU_TRAFFIC = {"source_sha16": "1a1f4f5b43445955", "bytes_per_launch": 30665216 + 11027456,
               "profile": "profiles/msa_batch_lp1054_b65536_fp32.md"}

WORKLOAD = "LP-1054 H_Z (465x1054, E=3720), iid X noise p=0.01..0.05, B=65536/step, max 50 it, alpha 0.75"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "int16"], default="fp32")
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


def kernel_traffic():
    import hashlib
    src = os.path.join(ROOT, "paper_2508_07879_gb300", "csrc", "msa_kernel.cuh")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return NCU_TRAFFIC["bytes_per_launch"] if sha == NCU_TRAFFIC["source_sha16"] else None


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
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
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
    oprec = {"fp32": "f32", "int16": "i16"}[precision]
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
    oprec = {"fp32": "f32", "int16": "i16"}[precision]
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


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    per_step = 256
    code, batches = make_batches(max(per_step * 4, 4096), 0)
    import oracle
    oracle.build()
    oprec = {"fp32": "f32", "int16": "i16"}[args.precision]

    def step(i):
        b = batches[i % len(batches)]
        lo = (i // len(batches)) * per_step % (b.syndromes.shape[0] - per_step + 1)
        oracle.msa(b.h.row_ptr, b.h.col_idx, b.h.m, b.h.n, b.syndromes[lo:lo + per_step], b.prior,
                   MAX_ITER, ALPHA, oprec, True, threads=threads)

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
        "vs_baseline": None, "dtype": {"fp32": "f32", "int16": "i16"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference_step": f"{per_step} shots on the CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "syndromes/s", "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} steps x {per_step} shots cycling p=0.01..0.05",
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
    B = args.batch
    first, _ = shard(rank, world, B)
    code, batches = make_batches(B, first_shot=first)       # each rank its own shots (weak scaling)
    h = batches[0].h
    graph = qldpc.Graph.from_csr(h)
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

    for i in range(args.warmup):
        step(i)
    stream.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for i in range(args.steps):
            step(i)
        e1.record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    ms = reduce_max(e0.elapsed_time(e1), dev)
    if world > 1:
        dist.barrier()
    ms_per_step = ms / args.steps
    value = world * B * args.steps / (ms / 1e3)
    launches = args.steps

    # roofline of the decoder kernel (one launch per step)
    sum_iters = sum(iters_per_batch[i % len(batches)] for i in range(args.steps))
    ops = OPS_PER_EDGE_ITER * h.nnz * sum_iters / args.steps          # per launch
    achieved = ops / (ms_per_step / 1e3) / 1e12                        # Tops/s
    props = torch.cuda.get_device_properties(dev)
    clocks = clk.summary()
    max_mhz = clocks["sm_max_mhz"] or 2070.0
    peak = props.multi_processor_count * ALU_LANES_PER_SM * max_mhz * 1e6 / 1e12
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3),
                "unit": "Tops/s", "frac": round(achieved / peak, 4),
                "traffic": kernel_traffic() if B == BATCH and args.precision == "fp32" else None,
                "kernel": "msa_batch_kernel", "ops_per_launch": ops,
                "units": "10 ALU ops per edge per iteration x E=3720 x iterations run",
                "peak_basis": f"{props.multi_processor_count} SMs x {ALU_LANES_PER_SM} lanes x {max_mhz:.0f} MHz (max SM clock)",
                # the op mix on the half-rate ALU pipe: 7 ALU-pipe ops per 10 bound the rate
                "op_mix_peak": round(peak * (ALU_PIPE_LANES_PER_SM / ALU_LANES_PER_SM)
                                     * OPS_PER_EDGE_ITER / ALU_OPS_PER_EDGE_ITER, 3),
                "op_mix_frac": round(achieved / (peak * (ALU_PIPE_LANES_PER_SM / ALU_LANES_PER_SM)
                                                 * OPS_PER_EDGE_ITER / ALU_OPS_PER_EDGE_ITER), 4),
                "hbm_algorithmic_gbs": round((h.m + h.n + 5) * B / (ms_per_step / 1e3) / 1e9, 2),
                "hbm_peak_gbs_measured": 6758.9}

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(qldpc, graph, batches, args, B, world, dev)
    latency = None
    if not args.no_latency and rank == 0:
        latency = measure_latency(qldpc, graph, code, args)
    serving = None
    if not args.no_serving and rank == 0:
        serving = measure_serving(qldpc, args)
    precisions = None
    if not args.no_precisions and rank == 0:
        precisions = measure_precisions(qldpc, graph, syn_d, pri_d, out, stream, B, args)
    layered_res = None
    if not args.no_layered and rank == 0:
        layered_res = measure_layered(qldpc, graph, code, syn_d, pri_d, out, stream, B, args)
    learned_res = None
    if not args.no_learned and rank == 0:
        learned_res = measure_learned(qldpc, args)
    soft_res = None
    if not args.no_soft and rank == 0:
        soft_res = measure_soft_syndrome(qldpc, args)
    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        threads = os.cpu_count() or 1
        rate, n, dt = oracle_rate(batches, CPU_SHOTS_PER_P, args.precision, threads)
        cpu = {"value": rate, "unit": "syndromes/s", "cores": threads, "kind": "oracle",
               "sample": f"{n} shots ({CPU_SHOTS_PER_P} per p at p=0.01..0.05) of the same batches, "
                         f"{dt:.1f} s wall, about {dt * threads:.0f} core-s",
               "single_thread": oracle_single_thread(batches, args.precision)}

    if rank == 0:
        line = {
            "metric": "syndromes/sec", "value": value, "unit": "syndromes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "int16": "i16"}[args.precision], "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": B * world, "precision": args.precision,
                       "l2": "inputs rotate over 5 batches (152 MB) + 69 MB outputs per step > 129 MB L2",
                       "rates": "step i decodes the batch of p = 0.01, 0.02, ..., 0.05 at i mod 5; a step count "
                                "that is a multiple of 5 weights the five rates equally",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "latency": latency,
            "serving": serving,
            "precisions": precisions,
            "layered": layered_res,
            "learned": learned_res,
            "soft_syndrome": soft_res,
            "gpu_launches": launches,
            "clocks": clocks,
            "mean_iters": sum(iters_per_batch) / (len(iters_per_batch) * B),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


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
    for prec in ("fp32", "int16", "int8"):
        ts = np.empty(shots + warm)
        iters = np.empty(shots + warm, dtype=np.int32)
        for i in range(shots + warm):
            row = syn[i:i + 1]
            t0 = time.perf_counter_ns()
            qldpc.decode_host(graph, row, prior, MAX_ITER, ALPHA, prec, out=(err, it, ok))
            ts[i] = (time.perf_counter_ns() - t0) / 1e3
            iters[i] = it[0]
        x = ts[warm:]
        lat[prec] = {"p50_us": float(np.percentile(x, 50)), "p99_us": float(np.percentile(x, 99)),
                     "p999_us": float(np.percentile(x, 99.9)), "mean_us": float(x.mean()),
                     "max_iter_shots": int((iters[warm:] == MAX_ITER).sum())}
    out = {"metric": "p99 single-shot decode latency", "unit": "us", "threshold_us": THRESHOLD_US,
           "code": "LP-1054 H_Z", "p": LAT_P, "shots": shots, "max_iter": MAX_ITER,
           "launch_path": {"path": "qldpc_decode_host from Python, page-locked buffers read/written by the "
                                   "kernel, host clock, B=1", **lat}}
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
    return out


def measure_serving(qldpc, args):
    """Config 5: Poisson arrivals of syndrome rounds mixed 40/40/20 from three codes."""
    from paper_2508_07879_gb300 import workloads as w
    rng = np.random.default_rng(5005)
    n = args.serve_requests
    codes = rng.choice(3, size=n, p=list(SERVE_MIX)).astype(np.int32)
    arrival = np.cumsum(rng.exponential(SERVE_GAP_NS, size=n)).astype(np.int64)
    graphs, priors, rows = [], [], []
    for ci, name in enumerate(("hgp400", "lp1054", "bb288")):
        b = w.x_error_batch(w.CONFIG_CODES[name](), 0.03, int((codes == ci).sum()), seed=5001 + ci)
        graphs.append(qldpc.Graph.from_csr(b.h))
        priors.append(b.prior)
        rows.append(b.syndromes)
    cursor = [0, 0, 0]
    syn = []
    for c in codes:
        syn.append(rows[c][cursor[c]])
        cursor[c] += 1
    out = {"workload": "40/40/20 HGP-400 / LP-1054 / BB-288 (H_Z, iid X, p=0.03), Poisson mean gap 20 us",
           "requests": n, "max_iter": MAX_ITER}
    for prec in ("fp32", "int16", "int8"):
        with qldpc.Server(graphs, priors, MAX_ITER, ALPHA, prec, ring_capacity=4096) as srv:
            _, _, _, lat_ns = srv.replay(codes, syn, arrival, timeout_s=60.0)
            t0 = time.perf_counter()
            srv.replay(codes, syn, np.zeros(n, np.int64), timeout_s=60.0)
            dt = time.perf_counter() - t0
        x = lat_ns / 1e3
        per = {}
        for ci, name in enumerate(("hgp400", "lp1054", "bb288")):
            xs = x[codes == ci]
            per[name] = {"p50_us": float(np.percentile(xs, 50)), "p99_us": float(np.percentile(xs, 99))}
        out[prec] = {"p50_us": float(np.percentile(x, 50)), "p99_us": float(np.percentile(x, 99)),
                     "p999_us": float(np.percentile(x, 99.9)), "per_code": per,
                     "saturated_shots_per_s": n / dt}
    return out


def measure_precisions(qldpc, graph, syn_d, pri_d, out, stream, B, args, steps=100):
    """Flooding decode of the benchmark's batches in each precision: throughput and decoded fraction."""
    import torch
    res = {}
    for prec in ("fp32", "int16", "int8"):
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
        res[prec] = {"value": B * steps / (e0.elapsed_time(e1) / 1e3), "unit": "syndromes/s",
                     "decoded_fraction": ok / (len(syn_d) * B), "mean_iters": iters / (len(syn_d) * B)}
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
    for i in range(shots + warm):
        t0 = time.perf_counter_ns()
        qldpc.decode_host(graph, syn[i:i + 1], b.prior, MAX_ITER, ALPHA, "fp32", out=(err, it, okk), layered=True)
        ts[i] = (time.perf_counter_ns() - t0) / 1e3
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
    # (key prefix, loss, Adam lr): the configured lr, and the syndrome loss at a larger step
    runs = (("", "syndrome", LEARN_LR), ("lr1e-2_", "syndrome", 1e-2), ("error_loss_", "error", LEARN_LR))
    for prefix, loss, lr in runs:
        model = learned.NeuralMinSum(h, prior, T=LEARN_T, max_batch=LEARN_BATCH, graph=g, loss=loss)
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
                                                    "learned_20_fallback_50": (50, True)},
                               shots=args.learned_eval_shots, p_lo=LEARN_P[0], p_hi=LEARN_P[1], seed=LEARN_SEEDS[1])
        eval_s = time.perf_counter() - t0
        ler.update({prefix + k: v["ler"] for k, v in res.items()})
        iters.update({prefix + k: v["mean_iters"] for k, v in res.items()})
        wmean = model.weights.detach().mean(dim=1).cpu().numpy()
        out[(prefix or "syndrome_") + "training"] = {
            "loss": loss, "lr": lr, "mean_weight_per_iteration": [round(float(x), 4) for x in wmean],
            "train_s": train_s, "train_shots_per_s": steps * LEARN_BATCH / train_s,
            "loss_first": float(hist[0]) if len(hist) else None, "loss_last": float(hist[-1]) if len(hist) else None,
            "step_kernel_ms": {"forward": tf, "backward_and_reduce": tb},
            "train_edge_iters_per_s": {"forward": edge_iters / (tf / 1e3), "backward": edge_iters / (tb / 1e3)},
            "eval_s": eval_s,
        }
        g.set_weights(None)
    out["ler"] = ler
    out["mean_iters"] = iters
    out["learned_keys"] = ("learned_*: syndrome loss, lr 1e-3 (the configured run); lr1e-2_learned_*: syndrome "
                           "loss, lr 1e-2; error_loss_learned_*: error loss, lr 1e-3")
    return out


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
