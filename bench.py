"""Benchmark of the GB300 CP-ARLS-LEV hot path.

Workload (default): the 8,211,298 x 176,962 x 8,116,559 planted log(1 + count)
tensor with about 4.69e9 nonzeros (the shape and nonzero count of the paper's Reddit
tensor, Table 6.1; synthetic, planted rank 25, Zipf(1.2) popularity, generated on the
GPU), CP rank 25, s = 2^17 samples per least-squares problem, hybrid threshold
tau = 1/s, range-finder start and estimated fit as the paper runs this size.

One step = one epoch of Alg. 3: eta = 5 outer iterations, each updating all 3 modes
(sampling, sampled Gram and its factorisation, sampled MTTKRP with the solve folded
in, leverage refresh), then the estimated fit -- 15 mode updates through one
cp_arls_lev call that continues the decomposition (iter_offset advances).  value =
FP64 mode updates per second over the timed steps, inputs resident in HBM (the index,
145 GB, far larger than L2).  The mixed-precision series, the end-to-end series
through host buffers and the oracle on the host cores are reported beside it.

--workload amazon: the 1.74e9-nonzero Amazon-shaped tensor; --workload uber: the
183 x 24 x 1140 x 1717 Uber-shaped tensor (3.3M nonzeros, FP64, exact fit) with the
batched and equal-fit comparisons.  --impl reference times the FP64 CPU oracle and
prints the same JSON line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "CP-ARLS-LEV mode-updates/sec and sampled-MTTKRP HBM GB/s at equal fit vs FP64 GPU path"
UNIT = "mode-updates/s"
RANK, SAMPLES, TAU_EXP, ETA = 25, 2 ** 17, 17, 5
WORKLOAD = "uber-shaped 183x24x1140x1717 planted counts, ~3.31M nnz, r=25, s=2^17, tau=2^-17, FP64"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision series")
    p.add_argument("--no-equal-fit", action="store_true", help="skip the equal-fit comparison")
    p.add_argument("--equal-fit-restarts", type=int, default=32)
    p.add_argument("--equal-fit-epochs", type=int, default=30)
    p.add_argument("--no-batched", action="store_true", help="skip the 64-problem batched comparison")
    p.add_argument("--batched-problems", type=int, default=64)
    p.add_argument("--cpu-sample-updates", type=int, default=4,
                   help="mode updates the CPU baseline times (bounded sample)")
    p.add_argument("--workload", default="reddit", choices=["uber", "amazon", "reddit"],
                   help="reddit (default): the 8.2M x 177K x 8.1M, 4.7e9-nonzero tensor; amazon: the "
                        "4.8M x 1.8M x 1.8M, 1.7e9-nonzero tensor (both generated on the GPU); uber: the "
                        "183 x 24 x 1140 x 1717, 3.3M-nonzero tensor")
    p.add_argument("--fit-samples", type=int, default=1 << 27,
                   help="elements of the estimated fit's sample (billion-nonzero workloads)")
    p.add_argument("--fraction", "--amazon-fraction", dest="fraction", type=float, default=1.0,
                   help="fraction of the amazon- or reddit-shaped tensor's events (dims kept)")
    p.add_argument("--shrink", type=int, default=1,
                   help="amazon/reddit: every dimension divided by this and the events by its cube (the same "
                        "planted model at a few GB, for profiler captures); the estimated fit's sample shrinks "
                        "with the events")
    p.add_argument("--cpu-fraction", type=float, default=1.0 / 1024,
                   help="fraction of the events in the oracle's same-shape tensor (billion-nonzero workloads)")
    p.add_argument("--cpu-procs", type=int, default=0,
                   help="oracle processes of the CPU baseline (0: all host cores, as memory allows)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, world, device):
    """The largest value of x over the ranks (the job's time is the slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(updates_per_rank, world, max_ms):
    """Whole-job mode updates per second: the updates of all ranks over the slowest
    rank's time."""
    return updates_per_rank * world / (max_ms / 1000.0)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def make_workload():
    import synth
    coo = synth.uber_like_tensor(0)
    init = synth.gaussian_factors(coo.dims, RANK, seed=0)
    return coo, init


def mttkrp_bytes(stats, d, b_f, b_val=8):
    """Algorithmic bytes of the fused probe + sampled-KRP + sampled-MTTKRP kernel,
    summed over updates: per kept sample its key and weight (16 B), its fibre probe
    (key and offset, 16 B) and the gathers of its d factor rows (d r b_f B); per
    sampled nonzero its mode index and value (4 + b_val B).  M (n_k r b_f B per
    update) is added by the caller."""
    return stats["sbar_total"] * (32 + d * RANK * b_f) + stats["nnz_sampled_total"] * (4 + b_val)


def krp_gram_flops(stats, d):
    """Algorithmic floating-point operations of the sampled-KRP + sampled-Gram kernel
    summed over updates: per kept sample, the D-1 multiplications of each of the r
    entries of y_j = w_j * prod of D-1 factor rows, and the upper triangle of
    y_j y_j^T accumulated into G (r(r+1)/2 fused multiply-adds = r(r+1) flops)."""
    return stats["sbar_total"] * (RANK * (RANK + 1) + RANK * (d - 1))


# FP64 and FP32 peaks of one GB300 from unit counts and the maximum SM clock:
# 152 SMs x 2 FP64 FMA/clk (resp. 128 FP32 FMA/clk) x 2 flops x 2.07 GHz.
SMS, SM_MAX_GHZ = 152, 2.07
FP64_PEAK_TFLOPS = SMS * 2 * 2 * SM_MAX_GHZ / 1000.0
FP64_OPS_PEAK = SMS * 2 * SM_MAX_GHZ / 1000.0  # FP64 instructions (multiply or FMA) per second, x1e12
FP32_PEAK_TFLOPS = SMS * 128 * 2 * SM_MAX_GHZ / 1000.0
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense tensor rates of the part

STAGES = ["sample", "krp_gram", "mttkrp", "solve", "leverage", "fit"]


def captured_traffic(kernel, source):
    """DRAM bytes of `kernel` (per launch, or per mode update for a stage) from the
    committed ncu summary (profiles/traffic.json), or None when the kernel's source
    changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, source), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != rec["source_sha1"]:
                return None
        return rec.get("dram_bytes_per_launch", rec.get("dram_bytes_per_update"))
    except Exception:
        return None
WHOLE = 8


def run_reference(args, rank):
    import oracle
    if rank != 0:
        return 0
    coo, init = make_workload()
    idx = oracle.Index(coo)
    s, tau = SAMPLES, 2.0 ** -TAU_EXP
    fs = [a.copy() for a in init]
    per_step = max(1, args.cpu_sample_updates)
    times = []
    k_total = args.warmup + args.steps
    it = 0
    for step in range(k_total):
        t0 = time.perf_counter()
        for u in range(per_step):
            k = u % len(coo.dims)
            res = oracle.mode_update(idx, fs, k, rank=RANK, samples=s, tau=tau, seed=0, it=it)
            fs[k] = res["A"]
            if k == len(coo.dims) - 1:
                it += 1
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = per_step * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "step": f"{per_step} mode updates"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} mode updates per step of the same workload "
                                   "(leverage of every mode recomputed by Householder QR per update)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(coo, init, n_updates):
    """The oracle as it stands, timed on a bounded sample of the same workload."""
    import oracle
    idx = oracle.Index(coo)
    fs = [a.copy() for a in init]
    t0 = time.perf_counter()
    for u in range(n_updates):
        k = u % len(coo.dims)
        res = oracle.mode_update(idx, fs, k, rank=RANK, samples=SAMPLES, tau=2.0 ** -TAU_EXP, seed=0, it=0)
        fs[k] = res["A"]
    dt = time.perf_counter() - t0
    return {"value": n_updates / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n_updates} mode updates of the same workload (index built untimed)"}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if args.workload in LARGE:
            return run_reference_large(args, LARGE[args.workload], rank)
        return run_reference(args, rank)
    if args.workload in LARGE:
        return run_large(args, LARGE[args.workload], rank, world, local)
    import torch
    import paper_2006_16438_gb300 as cpa
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    coo, init = make_workload()
    index = cpa.cpa_index_build(coo)
    s, tau = SAMPLES, 2.0 ** -TAU_EXP
    seed = rank  # independent decompositions per rank (random restarts)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def series(precision, profile):
        """W untimed + K timed epochs from the same initial factors.  profile = 1 adds
        CUDA-event nodes around every stage (the Gram and MTTKRP branches then run one
        after the other); the headline series runs without them."""
        fs = [torch.from_numpy(a).cuda() for a in init]
        lam = torch.empty(RANK, dtype=torch.float64, device="cuda")
        fitd = torch.empty(1, dtype=torch.float64, device="cuda")
        state = {"it": 0}

        def step():
            res = cpa.cp_arls_lev(index, None, rank=RANK, samples=s, tau=tau, iters=ETA, seed=seed,
                                  iter_offset=state["it"], profile=profile, out=(fs, lam, fitd),
                                  precision=precision)
            state["it"] += ETA
            return res

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        times, stages, fits, last = [], np.zeros(12), [], {}
        acc = {"sbar_total": 0, "nnz_sampled_total": 0, "kernel_launches": 0}
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.add_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = step()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            st = res.stats
            stages += np.array(st["stage_ms"])
            acc["sbar_total"] += st["sbar_total"]
            acc["nnz_sampled_total"] += st["nnz_sampled_total"]
            if acc["kernel_launches"] is not None and st["kernel_launches"] >= 0:
                acc["kernel_launches"] += st["kernel_launches"]
            else:
                acc["kernel_launches"] = None
            fits.append(res.fit)
            last = st
        total_ms = max_over_ranks(sum(times), world, "cuda")
        return dict(total_ms=total_ms, stages=stages, acc=acc, fit=fits[-1], last=last,
                    step_ms={"min": min(times), "median": statistics.median(times), "max": max(times)})

    clocks = ClockSampler(local)
    clocks.start()
    f64 = series(cpa.binding.FP64, 0)
    clk = clocks.stop()
    f64p = series(cpa.binding.FP64, 1)  # per-stage CUDA-event times, same workload
    mixed = mixedp = None
    if not args.no_mixed:
        mixed = series(cpa.binding.MIXED, 0)
        mixedp = series(cpa.binding.MIXED, 1)
    updates = args.steps * ETA * len(coo.dims)
    value = job_throughput(updates, world, f64["total_ms"])
    peaks, peak_src = load_peaks()
    n_updates = updates
    stages, stat_acc, last_stats = f64p["stages"], f64p["acc"], f64["last"]
    d = len(coo.dims)

    def rooflines(stg, acc, b_f):
        nk_bytes = sum(n * RANK * b_f for n in coo.dims) * (n_updates // d)
        # fused probe + sampled KRP + sampled MTTKRP (stage 2)
        mk_ms = stg[2]
        mk_bytes = mttkrp_bytes(acc, d - 1, b_f) + nk_bytes
        mk_gbs = mk_bytes / (mk_ms / 1000.0) / 1e9 if mk_ms > 0 else None
        mk_kernel = ("k_det_prep + k_det_expand + radix sort + k_det_tiles + k_det_fixup (probe + sampled KRP; "
                     "the sampled nonzeros sorted by row and reduced in fixed tiles: reproducible FP64)"
                     if b_f == 8 and os.environ.get("CPA_DET_MTTKRP", "1") != "0"
                     else "k_tnsr_mttkrp + k_tnsr_heavy (probe + sampled KRP + sampled MTTKRP, atomics)")
        mk = {"bound": "hbm", "kernel": mk_kernel,
              "achieved": mk_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
              "frac": (mk_gbs / peaks["hbm_gbs"]) if mk_gbs else None,
              "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
              "bytes_per_update": mk_bytes / n_updates, "ms_per_update": mk_ms / n_updates}
        # sampled KRP rows + sampled Gram (stage 1)
        kg_ms = stg[1]
        kg_flops = krp_gram_flops(acc, d)
        kg_tf = kg_flops / (kg_ms / 1000.0) / 1e12 if kg_ms > 0 else None
        if b_f == 8:
            kg = {"bound": "alu", "kernel": "k_krp_gram (sampled KRP rows + sampled Gram, FP64)",
                  "achieved": kg_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                  "frac": (kg_tf / FP64_PEAK_TFLOPS) if kg_tf else None,
                  "traffic": captured_traffic("k_krp_gram<double,1>", "paper_2006_16438_gb300/csrc/mttkrp.cu"),
                  "traffic_unit": "DRAM bytes per launch (ncu, profiles/traffic.json)",
                  "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz",
                  "flops_per_update": kg_flops / n_updates, "ms_per_update": kg_ms / n_updates}
        elif os.environ.get("CPA_GRAM_TENSOR_CORES", "0") not in ("", "0"):
            # tensor cores, kind::tf32: the measured bf16 peak times the nominal tf32/bf16 ratio
            pk = peaks["bf16_tflops"] * TF32_PER_BF16
            issued = acc["sbar_total"] * 128 * (32 if RANK <= 32 else 64) * 2 * 3  # M=128 x N x 2 flops x 3 products
            kg = {"bound": "tensor", "kernel": "k_krp_gram_tc (sampled KRP rows + sampled Gram, tcgen05 kind::tf32, "
                                               "3-product split)",
                  "achieved": kg_tf, "peak": pk, "unit": "TFLOP/s", "frac": (kg_tf / pk) if kg_tf else None,
                  "traffic": None,
                  "peak_source": f"{peak_src} bf16_tflops x nominal tf32/bf16 ratio {TF32_PER_BF16:.3f}",
                  "tensor_flops_issued_per_update": issued / n_updates,
                  "flops_per_update": kg_flops / n_updates, "ms_per_update": kg_ms / n_updates}
        else:
            # FP32 pipe (the default): FP32 tile sums added across tiles in FP64
            kg = {"bound": "alu", "kernel": "k_krp_gram (sampled KRP rows + sampled Gram, FP32 tile sums, FP64 across tiles)",
                  "achieved": kg_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                  "frac": (kg_tf / FP32_PEAK_TFLOPS) if kg_tf else None, "traffic": None,
                  "peak_source": "derived: 152 SMs x 128 FP32 FMA/clk x 2 flops x 2.07 GHz",
                  "flops_per_update": kg_flops / n_updates, "ms_per_update": kg_ms / n_updates}
        return kg, mk

    kg64, mk64 = rooflines(stages, stat_acc, 8)
    stage_share = {nm: round(float(stages[i] / max(stages[WHOLE], 1e-9)), 4) for i, nm in enumerate(STAGES)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": f64["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": "1 epoch = 5 outer iterations x 4 mode updates + exact fit",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"{world} independent replicas" if world > 1 else "single GPU"},
        "roofline": kg64,
        "mttkrp_hbm": mk64,
        "timing_note": "value from the series without stage events; stage and kernel times from a "
                       "second series of the same workload with CUDA-event nodes around every stage",
        "stages_ms_per_update": {nm: float(stages[i] / n_updates) for i, nm in enumerate(STAGES)},
        "stage_share": stage_share,
        "nnz_sampled_per_update": stat_acc["nnz_sampled_total"] / n_updates,
        "last_update": {k: last_stats.get(k) for k in ("sdet_last", "pdet_last", "attempts_last", "sbar_last",
                                                       "nnz_sampled_last")},
        "sbar_per_update": stat_acc["sbar_total"] / n_updates,
        "fit": f64["fit"],
        "clocks": clk,
        "step_ms": f64["step_ms"],
        "gpu_launches": f64["acc"]["kernel_launches"],
    }
    if mixed is not None:
        mv = updates * world / (mixed["total_ms"] / 1000.0)
        kg32, mk32 = rooflines(mixedp["stages"], mixedp["acc"], 4)
        line["mixed_precision"] = {
            "value": mv, "unit": UNIT, "speedup_vs_fp64": mv / value, "fit": mixed["fit"],
            "fit_fp64": f64["fit"], "fit_diff": mixed["fit"] - f64["fit"],
            "stages_ms_per_update": {nm: float(mixedp["stages"][i] / n_updates) for i, nm in enumerate(STAGES)},
            "krp_gram": kg32, "mttkrp_hbm": mk32,
            "note": "same init and epochs; FP32 factors/Grams/products, FP64 factorisations"}
    if not args.no_batched and rank == 0:
        line["batched"] = batched(cpa, args, stream)
    if mixed is not None and not args.no_equal_fit:
        line["mixed_precision"]["equal_fit"] = equal_fit(cpa, coo, seed, stream, args.equal_fit_restarts,
                                                         args.equal_fit_epochs)
    if rank == 0 and not args.no_e2e:
        line["e2e"] = e2e(cpa, coo, init, args)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(coo, init, args.cpu_sample_updates)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


AMAZON_DIMS = (4_821_207, 1_774_269, 1_805_187)
AMAZON_NNZ = 1_740_000_000
AMAZON_EVENTS_PER_NNZ = 1.43  # Poisson events per distinct nonzero of this planted model
# The billion-nonzero workloads: shape, target nonzeros, Poisson events per distinct
# nonzero of the planted model at that size, Zipf exponent, values.
LARGE = {
    "amazon": {"name": "amazon-shaped", "dims": AMAZON_DIMS, "nnz": AMAZON_NNZ,
               "events_per_nnz": AMAZON_EVENTS_PER_NNZ, "zipf": 1.1, "log_counts": False,
               "values": "counts"},
    "reddit": {"name": "reddit-shaped", "dims": (8_211_298, 176_962, 8_116_559), "nnz": 4_690_000_000,
               "events_per_nnz": 2.9, "zipf": 1.2, "log_counts": True, "values": "log(1 + count)"},
}
# The oracle's time per mode update on the full shape (Householder QR of two factors
# of ~8M rows) is about a minute on one core, so the reference arm runs it on the
# Reddit-shaped model with every dimension divided by this and the events by its cube.
REF_SHRINK = 16


def large_workload_name(spec, nnz, frac, fit_samples=1 << 27, shrink=1):
    fs = int(fit_samples)
    fit = f"2^{fs.bit_length() - 1}" if fs & (fs - 1) == 0 else str(fs)
    scale = ""
    if shrink > 1:
        scale = f" (the model with dimensions / {shrink} and events / {shrink}^3)"
    elif frac != 1.0:
        scale = f" ({frac:g} of the events)"
    return (f"{spec['name']} {'x'.join(str(n) for n in spec['dims'])} planted {spec['values']}, {nnz} nnz{scale}, "
            f"r=25, s=2^17, tau=2^-17, range-finder start, estimated fit {fit}")


def large_mttkrp_bytes(st, dims, b_f):
    """Algorithmic bytes of the sampled MTTKRP over the updates of `st`: per kept
    sample its key, weight and probe (32 B) and its d = 2 factor rows (2 r b_f); per
    sampled nonzero i_k and its FP32 value (8 B); per update the n_k x r output rows."""
    n_up = st["mode_updates"]
    per_mode = sum(dims) * RANK * b_f * (n_up // len(dims))
    return st["sbar_total"] * (32 + 2 * RANK * b_f) + st["nnz_sampled_total"] * 8 + per_mode


def run_large(args, spec, rank, world, local):
    """A billion-nonzero planted tensor generated on the GPU (int32 COO, FP32 values):
    by default the 8,211,298 x 176,962 x 8,116,559 log(1 + count) tensor with Zipf(1.2)
    popularity (about 4.69e9 nonzeros), or the 4,821,207 x 1,774,269 x 1,805,187
    counts with Zipf(1.1) (about 1.74e9); r = 25, s = 2^17, tau = 2^-17, the paper's
    setting for these sizes: range-finder start (App. F, s_init = 1e5) and the
    estimated fit (Sec. 5.4, 2^27 stratified samples).  One step = one epoch: eta = 5
    outer iterations (15 mode updates) and the estimated fit, one cp_arls_lev call
    continuing the run.  The headline series is FP64; the mixed-precision series
    starts from the same factors.  One further epoch with stage events gives the stage
    times and the sampled MTTKRP's rates.  The COO is dropped once the index is built."""
    import torch
    import paper_2006_16438_gb300 as cpa
    from synth import gpu as sgpu
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    frac = args.fraction
    shrink = max(1, args.shrink)
    if shrink > 1:  # the same model at a profiler-sized scale
        spec = dict(spec, dims=tuple(max(RANK, n // shrink) for n in spec["dims"]))
        frac = frac / shrink ** 3
        args.fit_samples = max(1 << 16, args.fit_samples // shrink ** 3)
    dims = spec["dims"]
    t0 = time.perf_counter()
    idx, vals = sgpu.planted_cp_tensor_gpu(dims, RANK, events=int(spec["events_per_nnz"] * spec["nnz"] * frac),
                                           seed=rank, zipf_alpha=spec["zipf"], log_counts=spec["log_counts"])
    torch.cuda.synchronize()
    torch.cuda.empty_cache()  # the generator's cached blocks: the build needs the room
    gen_s = time.perf_counter() - t0
    nnz = int(vals.numel())
    coo_bytes = sum(int(i.numel()) * 4 for i in idx) + nnz * 4
    t0 = time.perf_counter()
    index = cpa.cpa_index_build(dims, device_tensors=(idx, vals))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    del idx, vals
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    g = torch.Generator(device="cuda")
    g.manual_seed(1000 + rank)
    init = [cpa.cpa_rrf_init(index, k, torch.randn(100000, RANK, dtype=torch.float64, device="cuda", generator=g),
                             seed=k) for k in range(3)]
    torch.cuda.synchronize()
    s, tau = SAMPLES, 2.0 ** -TAU_EXP
    n_up = ETA * 3

    def series(prec):
        fs = [a.clone() for a in init]
        lam = torch.empty(RANK, dtype=torch.float64, device="cuda")
        fitd = torch.empty(1, dtype=torch.float64, device="cuda")
        it = [0]

        def step(profile=0):
            res = cpa.cp_arls_lev(index, None, rank=RANK, samples=s, tau=tau, iters=ETA, seed=rank,
                                  iter_offset=it[0], out=(fs, lam, fitd), precision=prec,
                                  fit_mode=cpa.binding.FIT_ESTIMATED, fit_samples=args.fit_samples, profile=profile)
            it[0] += ETA
            return res

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        launches = 0
        evs[0].record(stream)
        est = []
        tag = "fp64_epoch" if prec == cpa.binding.FP64 else "mixed_epoch"
        for i in range(args.steps):
            torch.cuda.nvtx.range_push(tag)  # lets a profiler select the timed epochs
            res = step()
            torch.cuda.nvtx.range_pop()
            evs[i + 1].record(stream)
            est.append(res.fit)
            launches = launches + res.stats["kernel_launches"] if res.stats["kernel_launches"] >= 0 else launches
        torch.cuda.synchronize()
        clk = clocks.stop()
        step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
        total_ms = max_over_ranks(sum(step_ms), world, "cuda")
        prof = step(profile=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        exact = cpa.cpa_fit(index, fs, lam)
        exact_s = time.perf_counter() - t0
        out = dict(total_ms=total_ms, step_ms=step_ms, launches=launches, clocks=clk, stats=prof.stats,
                   est_fit=est[-1] if est else None, exact_fit=exact, exact_fit_s=exact_s,
                   epochs=args.warmup + args.steps + 1)
        del fs
        return out

    f64 = series(cpa.binding.FP64)
    mixed = None if args.no_mixed else series(cpa.binding.MIXED)
    updates = args.steps * n_up
    value = job_throughput(updates, world, f64["total_ms"])
    peaks, peak_src = load_peaks()

    def stage_table(st):
        return {nm: float(st["stage_ms"][i] / n_up) for i, nm in enumerate(STAGES)}

    def mttkrp_rates(st, b_f):
        ms = st["stage_ms"][2]
        byts = large_mttkrp_bytes(st, dims, b_f)
        gbs = byts / (ms / 1000.0) / 1e9 if ms > 0 else None
        return {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / peaks["hbm_gbs"] if gbs else None,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "bytes_per_update": byts / n_up, "ms_per_update": ms / n_up,
                "sampled_nonzeros_per_update": st["nnz_sampled_total"] / n_up,
                "row_additions_per_s": st["nnz_sampled_total"] / (ms / 1000.0) if ms > 0 else None}

    st64 = f64["stats"]
    mk64 = mttkrp_rates(st64, 8)
    # the headline roofline: the sampled MTTKRP's algorithmic bytes per second against
    # the measured HBM copy rate (the metric's GB/s).  Its on-chip limits are given
    # beside: the FP64 multiplies (r per sampled nonzero; 2 r + 1 Khatri-Rao multiplies
    # and r^2 multiply-adds of the folded solve per sample) against the FP64 pipe
    # (152 SMs x 2 FP64 instructions per clock per SM x 2.07 GHz), and the row additions
    # (one FP64 atomic row of r words per sampled nonzero).
    fp64_ops = st64["nnz_sampled_total"] * RANK + st64["sbar_total"] * (2 * RANK + 1 + RANK * RANK)
    ms2 = st64["stage_ms"][2]
    fp64_rate = fp64_ops / (ms2 / 1000.0) / 1e12 if ms2 > 0 else None
    roof = dict(mk64)
    roof.update({
        "kernel": "sampled MTTKRP, FP64 (k_slab_prep: probe + sampled Khatri-Rao rows times the inverse sampled "
                  "Gram; k_slab_light + k_slab_heavy: FP64 products added into row slabs of A_k)",
        "traffic": (captured_traffic(f"sampled_mttkrp_fp64_{args.workload}", "paper_2006_16438_gb300/csrc/mttkrp.cu")
                    if shrink == 1 and frac == 1.0 else None),
        "traffic_unit": "DRAM bytes per mode update, all launches of the stage (ncu, profiles/traffic.json)",
        "fp64_pipe": {"achieved": fp64_rate, "peak": FP64_OPS_PEAK, "unit": "T FP64 instructions/s",
                      "frac": fp64_rate / FP64_OPS_PEAK if fp64_rate else None,
                      "peak_source": "derived: 152 SMs x 2 FP64 lanes/clk x 2.07 GHz"}})
    nfib = [index.nfib(k) for k in range(3)]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": f64["total_ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": large_workload_name(spec, nnz, frac, args.fit_samples, shrink),
                   "step": "1 epoch = 5 outer iterations x 3 mode updates + estimated fit",
                   "l2": f"inputs far larger than L2 ({index.device_bytes() / 1e9:.0f} GB of index)",
                   "parallelism": f"{world} independent replicas" if world > 1 else "single GPU"},
        "roofline": roof,
        "mttkrp_hbm": mk64,
        "stages_ms_per_update": stage_table(st64),
        "fit": {"estimated": f64["est_fit"], "exact": f64["exact_fit"], "epochs": f64["epochs"]},
        "clocks": f64["clocks"],
        "step_ms": {"min": min(f64["step_ms"]), "median": statistics.median(f64["step_ms"]),
                    "max": max(f64["step_ms"])},
        "gpu_launches": f64["launches"],
        "memory": {"index_bytes": index.device_bytes(), "fibres_per_mode": nfib},
        "generate_s": gen_s, "index_build_s": build_s,
    }
    if mixed is not None:
        stm = mixed["stats"]
        mv = job_throughput(updates, world, mixed["total_ms"])
        line["mixed_precision"] = {
            "value": mv, "unit": UNIT, "speedup_vs_fp64": mv / value,
            "fit": {"estimated": mixed["est_fit"], "exact": mixed["exact_fit"]},
            "exact_fit_diff_vs_fp64": mixed["exact_fit"] - f64["exact_fit"],
            "stages_ms_per_update": stage_table(stm),
            "mttkrp_hbm": dict(mttkrp_rates(stm, 4),
                               traffic=(captured_traffic(f"sampled_mttkrp_mixed_{args.workload}",
                                                         "paper_2006_16438_gb300/csrc/mttkrp.cu")
                                        if shrink == 1 and frac == 1.0 else None),
                               traffic_unit="DRAM bytes per mode update, all launches of the stage (ncu, "
                                            "profiles/traffic.json)"),
            "clocks": mixed["clocks"], "gpu_launches": mixed["launches"],
            "note": "same range-finder start and epochs as the FP64 series; FP32 factors, Grams and sampled "
                    "products, FP64 factorisations and leverage; exact fits (Eq. 5.1) after the same epochs"}
    free_b, total_b = torch.cuda.mem_get_info()
    line["memory"]["device_bytes_in_use"] = total_b - free_b
    if rank == 0 and not args.no_e2e:
        line["e2e"] = e2e_large(cpa, index, init, args, coo_bytes, gen_s, build_s)
    del init
    index.free()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_large(spec, args)
    if rank == 0 and mixed is not None and not args.no_equal_fit:
        # equal fit needs many restarts with an exact fit per epoch: measured on the
        # Uber-shaped tensor, where an epoch takes milliseconds
        import synth
        line["mixed_precision"]["equal_fit"] = equal_fit(cpa, synth.uber_like_tensor(0), 0, stream,
                                                         args.equal_fit_restarts, args.equal_fit_epochs)
    if rank == 0 and not args.no_batched:
        line["batched"] = batched(cpa, args, stream)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def e2e_large(cpa, index, init, args, coo_bytes, gen_s, build_s):
    """The FP64 series through cp_arls_lev with HOST factor buffers in pinned memory:
    every step copies the factors in, runs one epoch on the resident index and copies
    the factors, lambda and the fit back (the library's own copies, inside the timed
    region).  The index is the resident form of the tensor, built once (its one-time
    cost is reported beside)."""
    import torch
    keep = [a.cpu().pin_memory() for a in init]
    fs = [t.numpy() for t in keep]
    fac_bytes = sum(a.nbytes for a in fs)
    s, tau = SAMPLES, 2.0 ** -TAU_EXP

    def step(i):
        return cpa.cp_arls_lev(index, fs, rank=RANK, samples=s, tau=tau, iters=ETA, seed=0, iter_offset=ETA * i,
                               on_device=False, inplace=True, precision=cpa.binding.FP64,
                               fit_mode=cpa.binding.FIT_ESTIMATED, fit_samples=args.fit_samples)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": ETA * 3 * args.steps / dt, "unit": UNIT, "h2d_bytes_per_step": int(fac_bytes),
            "d2h_bytes_per_step": int(fac_bytes + 8 * RANK + 8), "steps": args.steps,
            "note": "cp_arls_lev on host factor buffers (pinned), FP64, every step's copies in the timed region; "
                    "the tensor is resident as its index",
            "one_time": {"coo_bytes": coo_bytes, "generate_s": gen_s, "index_build_s": build_s}}


def _oracle_update_worker(task):
    """One mode update of the oracle (in a spawned process): loads the COO saved by the
    parent, builds the oracle's index and times oracle.mode_update."""
    path, dims, k, seed = task
    import oracle
    import synth
    z = np.load(path)
    coo = synth.Coo(tuple(dims), [z[f"i{m}"] for m in range(len(dims))], z["v"])
    idx = oracle.Index(coo)
    fs = synth.gaussian_factors(dims, RANK, seed=seed)
    t0 = time.perf_counter()
    oracle.mode_update(idx, fs, k, rank=RANK, samples=SAMPLES, tau=2.0 ** -TAU_EXP, seed=seed, it=0)
    return time.perf_counter() - t0


def _mem_available_bytes():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except Exception:
        pass
    return 0


def cpu_baseline_large(spec, args):
    """The oracle as it stands on the host cores: one mode update per process, all
    processes at once, on a tensor of the same shape (so the factor matrices and
    their leverage QRs are the full size) with 1/1024 of the planted model's events
    (generated on the GPU by the same generator, seed 7)."""
    import multiprocessing
    import tempfile
    import torch
    from synth import gpu as sgpu
    dims = spec["dims"]
    frac = args.cpu_fraction
    idx, vals = sgpu.planted_cp_tensor_gpu(dims, RANK, events=int(spec["events_per_nnz"] * spec["nnz"] * frac),
                                           seed=7, zipf_alpha=spec["zipf"], log_counts=spec["log_counts"])
    arrs = {f"i{m}": idx[m].cpu().numpy() for m in range(len(dims))}
    arrs["v"] = vals.cpu().numpy().astype(np.float64)
    nnz = int(vals.numel())
    del idx, vals
    torch.cuda.empty_cache()
    tmp = tempfile.mkdtemp(prefix="cpa_oracle_")
    path = os.path.join(tmp, "coo.npz")
    np.savez(path, **arrs)
    del arrs
    # per process: the factors (and the oracle's copies of them) and its index
    per_proc = 4 * sum(dims) * RANK * 8 + nnz * 64 + (1 << 30)
    cores = os.cpu_count() or 1
    procs = max(1, min(cores, args.cpu_procs or cores, int(0.6 * _mem_available_bytes() // per_proc)))
    ctx = multiprocessing.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(procs) as pool:
        times = pool.map(_oracle_update_worker, [(path, list(dims), p % 3, p) for p in range(procs)])
    wall = time.perf_counter() - t0
    try:
        os.remove(path)
        os.rmdir(tmp)
    except OSError:
        pass
    return {"value": procs / max(times), "unit": UNIT, "cores": procs, "kind": "oracle",
            "nproc": cores, "single_process_value": 1.0 / statistics.median(times),
            "seconds_per_update": {"min": min(times), "median": statistics.median(times), "max": max(times)},
            "wall_s": wall,
            "sample": f"{procs} processes at once, one mode update each (modes cycled), FP64 oracle on a "
                      f"{'x'.join(str(n) for n in dims)} tensor with {nnz} nnz ({frac:g} of the planted model's "
                      "events), r=25, s=2^17, tau=2^-17; value = updates / slowest process's time"}


def run_reference_large(args, spec, rank):
    """--impl reference for the billion-nonzero workloads: the FP64 oracle on the host,
    one mode update per step (modes cycled, the decomposition continuing), on the same
    planted model with every dimension divided by REF_SHRINK and the events by its cube
    (generated on the host) -- the full shape takes about a minute per update on one
    core."""
    import oracle
    import synth
    if rank != 0:
        return 0
    dims = tuple(max(RANK, n // REF_SHRINK) for n in spec["dims"])
    events = int(spec["events_per_nnz"] * spec["nnz"] / REF_SHRINK ** 3)
    coo = synth.planted_cp_tensor(dims, RANK, events=events, seed=0, zipf_alpha=spec["zipf"],
                                  log_counts=spec["log_counts"])
    idx = oracle.Index(coo)
    fs = synth.gaussian_factors(dims, RANK, seed=0)
    times = []
    it = 0
    for step in range(args.warmup + args.steps):
        k = step % 3
        t0 = time.perf_counter()
        res = oracle.mode_update(idx, fs, k, rank=RANK, samples=SAMPLES, tau=2.0 ** -TAU_EXP, seed=0, it=it)
        dt = time.perf_counter() - t0
        fs[k] = res["A"]
        if k == 2:
            it += 1
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = len(times) / total
    wl = (f"{spec['name']} model with dimensions / {REF_SHRINK} ({'x'.join(str(n) for n in dims)}), "
          f"{coo.nnz} nnz, r=25, s=2^17, tau=2^-17, FP64")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl, "step": "1 mode update"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "nproc": os.cpu_count(),
                         "sample": f"1 mode update per step of the {wl} tensor (the oracle recomputes the "
                                   "leverage of the other modes by Householder QR in every update)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batched(cpa, args, stream, max_nnz=10 ** 7):
    """Many independent decompositions: the same epoch (5 outer iterations + fit) of
    every problem, run as sequential cp_arls_lev calls and as one batch graph
    (cpa_batch_*, autotuned), from the same initial factors and offsets, in FP64 and
    in mixed precision.  The 64 problems (synth.batch_specs: 3- and 4-way, dims
    log-uniform 1e2-1e5, nnz log-uniform 1e4-max_nnz, ranks 5-50) are generated on the
    GPU."""
    import torch
    import synth
    from synth import gpu as sgpu
    t0 = time.perf_counter()
    probs = []
    for sp, idx, vals in sgpu.batch_problems_gpu(args.batched_problems, 0, max_nnz):
        index = cpa.cpa_index_build(sp["dims"], device_tensors=(idx, vals))
        nnz = int(vals.numel())
        del idx, vals
        probs.append(dict(index=index, dims=sp["dims"], nnz=nnz, rank=sp["rank"], samples=sp["samples"],
                          tau=sp["tau"], seed=sp["seed"],
                          init=synth.gaussian_factors(sp["dims"], sp["rank"], seed=sp["seed"])))
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    gen_s = time.perf_counter() - t0
    updates = sum(ETA * len(p["dims"]) for p in probs)
    reps = max(3, min(args.steps, 7))

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    def compare(precision):
        state = [[torch.from_numpy(a).cuda() for a in p["init"]] for p in probs]
        outs = [(torch.empty(p["rank"], dtype=torch.float64, device="cuda"),
                 torch.empty(1, dtype=torch.float64, device="cuda")) for p in probs]

        def sequential(offset):
            return [cpa.cp_arls_lev(p["index"], None, rank=p["rank"], samples=p["samples"], tau=p["tau"],
                                    iters=ETA, seed=p["seed"], iter_offset=offset, precision=precision,
                                    out=(state[i], outs[i][0], outs[i][1])).fit for i, p in enumerate(probs)]

        sequential(0)  # warm-up: plans and graphs
        sequential(ETA)
        seq_ms, seq_fits = [], None
        for r in range(reps):
            ms, seq_fits = timed(lambda: sequential(ETA * (r + 2)))
            seq_ms.append(ms)
        bprobs = [dict(index=p["index"], factors=[torch.from_numpy(a).cuda() for a in p["init"]], rank=p["rank"],
                       samples=p["samples"], tau=p["tau"], iters=ETA, seed=p["seed"], precision=precision)
                  for p in probs]
        t1 = time.perf_counter()
        batch = cpa.Batch(bprobs, autotune=1)
        tune_s = time.perf_counter() - t1
        batch.run()  # warm-up (the same first two epochs as the sequential warm-up)
        batch.run()
        b_ms, b_att, b_pdet = [], [], []
        for r in range(reps):
            ms, st = timed(batch.run)
            b_ms.append(ms)
            worst = max(range(len(st)), key=lambda i: st[i]["attempts_last"])
            b_att.append([worst, st[worst]["attempts_last"], probs[worst]["samples"]])
            b_pdet.append(max(x["pdet_last"] for x in st))
        diffs = sorted(abs(a - b) for a, b in zip(seq_fits, batch.fits()))
        seq_v = updates / (statistics.median(seq_ms) / 1000.0)
        b_v = updates / (statistics.median(b_ms) / 1000.0)
        res = {"sequential": {"value": seq_v, "unit": UNIT, "ms_per_pass": seq_ms,
                              "value_mean": updates * reps / (sum(seq_ms) / 1000.0)},
               "batched": {"value": b_v, "unit": UNIT, "ms_per_pass": b_ms,
                           "value_mean": updates * reps / (sum(b_ms) / 1000.0),
                           "most_attempts_per_pass": b_att, "max_pdet_per_pass": b_pdet},
               "speedup": b_v / seq_v,
               "timing": "value = updates per pass / median pass time; value_mean = over the sum",
               "fit_diff_median": diffs[len(diffs) // 2], "fit_diff_max": diffs[-1],
               "autotune": batch.info(), "tune_s": tune_s}
        batch.free()
        return res

    out = {"problems": len(probs), "total_nnz": int(sum(p["nnz"] for p in probs)),
           "largest_nnz": int(max(p["nnz"] for p in probs)),
           "mode_updates_per_pass": updates, "passes": reps, "generate_s": gen_s,
           "fp64": compare(cpa.binding.FP64), "mixed": compare(cpa.binding.MIXED),
           "note": "fits after the same epochs with the same seeds (FP64: reproducible sums, so batched and "
                   "sequential runs agree bit for bit; mixed: FP32 atomics, so a few unstable problems drift)",
           "workload": f"{len(probs)} planted count tensors, 3-/4-way, dims log-uniform 1e2-1e5, nnz log-uniform "
                       f"1e4-{max_nnz:.0e} (<= 10% of cells, >= 50 N_k/s), Zipf alpha U[1.0,1.3], rank 5-50, "
                       "s = 2^14..2^17 capped at 1/128 of the fewest Khatri-Rao rows and >= 16 r, tau = 1/s; "
                       "one pass = one epoch (5 outer iterations + exact fit) of every problem"}
    for p in probs:
        p["index"].free()
    return out


def equal_fit(cpa, coo, seed, stream, restarts, epochs):
    """Mixed precision against FP64 at equal fit on `coo` (r = 25, s = 2^17,
    tau = 2^-17), over `restarts` random initial factors (Gaussian, Section 6), paired
    by restart.  Per restart both precisions run `epochs` epochs (eta = 5 outer
    iterations each), one cp_arls_lev call per epoch with the exact fit (Eq. 5.1)
    after it, timed with CUDA events (fits included).  The restart's target is the
    lower of the two best fits minus 1e-4, a fit both precisions reach; the time each
    needs to first reach it gives the restart's speedup at equal fit (FP64 time /
    mixed time).  A change of precision moves a randomized trajectory as a change of
    seed does, so the speedup is a distribution over restarts: its median with a
    bootstrap 95 % interval (4000 resamples of the restarts), its geometric mean, and
    the per-epoch speedup are reported, with the paired differences of the best and
    final fits."""
    import torch
    import synth
    s, tau = SAMPLES, 2.0 ** -TAU_EXP
    dims = coo.dims
    indices = {cpa.binding.FP64: cpa.cpa_index_build(coo), cpa.binding.MIXED: cpa.cpa_index_build(coo)}

    def trace(init, precision):
        fs = [torch.from_numpy(a).cuda() for a in init]
        lam = torch.empty(RANK, dtype=torch.float64, device="cuda")
        fitd = torch.empty(1, dtype=torch.float64, device="cuda")
        fits, ms = [], []
        for ep in range(epochs):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = cpa.cp_arls_lev(indices[precision], None, rank=RANK, samples=s, tau=tau, iters=ETA, seed=seed,
                                  iter_offset=ETA * ep, out=(fs, lam, fitd), precision=precision)
            e1.record(stream)
            torch.cuda.synchronize()
            fits.append(res.fit)
            ms.append(e0.elapsed_time(e1))
        return fits, ms

    warm = synth.gaussian_factors(dims, RANK, seed=999)
    for prec in indices:  # workspaces and graphs
        trace(warm, prec)
    tr = []
    for rs in range(restarts):
        init = synth.gaussian_factors(dims, RANK, seed=1000 + rs)
        f64, m64 = trace(init, cpa.binding.FP64)
        fmx, mmx = trace(init, cpa.binding.MIXED)
        target = min(max(f64), max(fmx)) - 1e-4

        def reach(fits, ms):
            for i, f in enumerate(fits):
                if f >= target:
                    return i + 1, sum(ms[:i + 1])
            return None, None

        e64, t64 = reach(f64, m64)
        emx, tmx = reach(fmx, mmx)
        tr.append({"target": target, "best_fp64": max(f64), "best_mixed": max(fmx), "final_fp64": f64[-1],
                   "final_mixed": fmx[-1], "epochs_fp64": e64, "epochs_mixed": emx, "ms_fp64": t64,
                   "ms_mixed": tmx, "ms_per_epoch_fp64": sum(m64) / len(m64),
                   "ms_per_epoch_mixed": sum(mmx) / len(mmx)})
    for ix in indices.values():
        ix.free()
    ratios = np.array([t["ms_fp64"] / t["ms_mixed"] for t in tr])
    g = np.random.default_rng(0)
    boot = np.median(ratios[g.integers(0, ratios.size, size=(4000, ratios.size))], axis=1)

    def paired(xs, ys):
        d = np.array([x - y for x, y in zip(xs, ys)])
        se = float(d.std(ddof=1) / math.sqrt(d.size)) if d.size > 1 else 0.0
        return {"mean": float(d.mean()), "se": se, "abs_median": float(np.median(np.abs(d)))}

    return {
        "workload": f"{'x'.join(str(n) for n in dims)} planted counts, {coo.nnz} nnz, r=25, s=2^17, tau=2^-17",
        "restarts": restarts, "epochs": epochs,
        "speedup_at_equal_fit": {"median": float(np.median(ratios)),
                                 "ci95": [float(np.percentile(boot, 2.5)), float(np.percentile(boot, 97.5))],
                                 "geomean": float(np.exp(np.mean(np.log(ratios)))),
                                 "per_restart": [round(float(x), 3) for x in ratios]},
        "per_epoch_speedup": float(np.mean([t["ms_per_epoch_fp64"] for t in tr]) /
                                   np.mean([t["ms_per_epoch_mixed"] for t in tr])),
        "fit_diff_best": paired([t["best_mixed"] for t in tr], [t["best_fp64"] for t in tr]),
        "fit_diff_final": paired([t["final_mixed"] for t in tr], [t["final_fp64"] for t in tr]),
        "mixed_reaches_fp64_best": int(sum(t["best_mixed"] >= t["best_fp64"] - 1e-4 for t in tr)),
        "note": "fit_diff_* = mixed - FP64 per restart (mean, standard error, median |diff|); the target of a "
                "restart is a fit both precisions reach (the lower best fit minus 1e-4)"}


def e2e(cpa, coo, init, args):
    """Same metric through cp_arls_lev_coo with HOST buffers in pinned memory (filled
    once, outside the timed region): each step copies the COO tensor and the factors
    in, builds the index, runs one epoch and copies the factors, lambda and fit back
    (the factors into the same pinned arrays)."""
    import torch
    import synth
    keep = []

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        keep.append(t)
        return t.numpy()

    pcoo = synth.Coo(coo.dims, [pinned(np.asarray(i, dtype=np.int32)) for i in coo.idx],
                     pinned(np.asarray(coo.vals, dtype=np.float64)))
    fs = [pinned(np.asarray(a, dtype=np.float64)) for a in init]
    idx_bytes = sum(i.nbytes for i in pcoo.idx) + pcoo.vals.nbytes
    fac_bytes = sum(a.nbytes for a in fs)
    times = []
    for i in range(max(1, min(3, args.steps)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cpa.cp_arls_lev_coo(pcoo, fs, rank=RANK, samples=SAMPLES, tau=2.0 ** -TAU_EXP, iters=ETA,
                            seed=0, iter_offset=ETA * i, inplace=True)
        t1 = time.perf_counter()
        if i > 0:
            times.append(t1 - t0)
    per = sum(times) / len(times)
    return {"value": ETA * len(coo.dims) / per, "unit": UNIT,
            "h2d_bytes_per_step": int(idx_bytes + fac_bytes),
            "d2h_bytes_per_step": int(fac_bytes + 8 * RANK + 8),
            "note": "index build included in every step; inputs and factors in pinned host memory"}


if __name__ == "__main__":
    sys.exit(main())
