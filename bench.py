"""Benchmark: all-mode sparse MTTKRP sweep on a GB300 (one JSON line on stdout).

A step is one all-mode sweep (Algorithm 5): for every mode n, the fused
spMTTKRP + dynamic-remap kernel and, when the mode has split rows, the fix-up.
Default workload: 3-mode 120000 x 90000 x 2000000 tensor, 100M distinct
nonzeros with Zipf(1.1) index skew on every mode, FP32 values, rank 32, FP32
factors (synthetic stand-in for the paper's FROSTT / recommender tensors).

Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2] [--rank R]
                  [--dtype f32|bf16] [--impl mine|reference]
Multi-GPU (one process per GPU via torchrun): independent replicas, one per
rank (the sweep has no cross-GPU exchange in this build), weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD_INDEX = {"c1": 0, "c2": 1, "c3": 2, "c4a": 3, "c4b": 3, "c5": 4}
PROFILES = os.path.join(ROOT, "profiles")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--rank", type=int, default=0)
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--nnz", type=int, default=0, help="override nonzero count (small runs)")
    ap.add_argument("--nblk", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--variant", type=int, default=0,
                    help="0 warp blocks with staged tiles, 1 CTA blocks with direct runs, "
                         "2 tile form, 3 warp blocks with a remap warp per CTA")
    ap.add_argument("--unroll", type=int, default=0)
    ap.add_argument("--stages", type=int, default=0)
    ap.add_argument("--element-bytes", type=int, default=0)
    ap.add_argument("--hints", type=int, default=0, help="-1 none, 0 default, 1..3 bits")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip the plan's autotuner (by default it runs, untimed, before "
                         "the warm-up and picks blocks per SM, tile, ring depth and form)")
    ap.add_argument("--partition", type=int, default=0, choices=[0, 1],
                    help="0: contiguous split with heavy-row splitting; 1: Algorithm 1 (LPT)")
    ap.add_argument("--keep-base", action="store_true",
                    help="keep the mode-0 copy resident: the last mode's pass writes no remap")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the BF16 sweep, CP-loss and CP-ALS measurements")
    ap.add_argument("--no-workload-extras", action="store_true",
                    help="skip the lines on the other workloads (4-mode FP32/BF16, CP loss "
                         "on the completion tensor, CP-ALS on the 5- and 6-mode tensors) "
                         "and the memory-ceiling probe")
    return ap.parse_args()


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world <= 1:
        return x
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload_tensors(name, nnz_override, device):
    spec = synth.workload(name)
    nnz = nnz_override or spec.nnz
    coo, vals = synth.make_coo(spec.dims, nnz, spec.skew, spec.seed, device=device)
    return spec, coo, vals


def compulsory_bytes(dims, nnz, R, s, touched, N, keep_base=False):
    """Algorithmic bytes of mode n's fused pass (elements read + next_pos + remapped write,
    each touched factor row once, output written once).  With the mode-0 copy kept
    resident the last mode's pass reads no next_pos and writes no remapped copy."""
    E = 4 * N + 4
    out = []
    for n in range(N):
        b = nnz * (E + 4 + E) if not (keep_base and n == N - 1) else nnz * E
        b += sum(touched[k] * R * s for k in range(N) if k != n)
        b += dims[n] * R * 4
        out.append(b)
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
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
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# sources that define and launch the fused spMTTKRP + remap kernel
KERNEL_SOURCES = ("mttkrp_common.cuh", "mttkrp_kernel.cuh", "mttkrp_direct.cuh", "mttkrp_tile.cuh",
                  "kernels_f32.cu", "kernels_bf16.cu", "kernels_tile.cu", "kernels_misc.cu")


def kernel_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2405_08470_gb300", "csrc")
    for f in sorted(KERNEL_SOURCES):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, R, dtype, nnz, info):
    """DRAM bytes per launch of the fused kernel from a committed ncu summary: bytes
    measured on a smaller tensor of the same shape (one kernel, its three mode
    launches), scaled to this run's nonzero count (per-nonzero traffic: the stream,
    the scattered copy and the factor-row misses all grow with the nonzeros).
    Used only while the kernel sources hash to the captured digest and the run has
    the captured configuration (blocks per SM, kernel form, stride, plan options);
    else null."""
    path = os.path.join(PROFILES, "mttkrp_remap_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("kernel_digest") != kernel_digest():
        return None
    e = d.get("entries", {}).get(f"{workload}_R{R}_{dtype}")
    if not e:
        return None
    cfg = e.get("config", {})
    if any(info.get(k) != v for k, v in cfg.items()):
        return None
    return e["dram_bytes_per_nonzero_per_launch"] * nnz


def cpu_oracle_full(coo_h, vals_h, dims, R, seed, one_thread_seconds=4.0):
    """The multi-threaded C FP64 oracle on ALL nonzeros of the workload, every mode,
    on all host threads (median of 3 sweeps).  A one-thread figure is timed on the
    first S nonzeros only (S sized to about `one_thread_seconds` per sweep) and
    scaled by nnz / S; it is labelled as such."""
    from oracle import ref_c
    F = [f.numpy().astype(np.float64) for f in synth.make_factors(dims, R, seed=seed)]
    nnz = coo_h.shape[0]
    N = len(dims)
    vals64 = vals_h.astype(np.float64)

    def sweep(S, threads):
        per = []
        for n in range(N):
            t0 = time.perf_counter()
            ref_c.mttkrp(coo_h[:S], vals64[:S], dims, F, n, nthreads=threads)
            per.append(time.perf_counter() - t0)
        return per

    med = lambda runs: [float(np.median([r[n] for r in runs])) for n in range(N)]  # noqa: E731
    allt = med([sweep(nnz, 0) for _ in range(3)])
    S = min(nnz, 1_000_000)
    dt = sum(sweep(S, 1))
    S = min(nnz, max(S, int(S * one_thread_seconds / max(dt, 1e-3))))
    one = med([sweep(S, 1)])
    return {"value": sum(allt) * 1e3, "unit": "ms", "cores": ref_c.threads(), "kind": "oracle",
            "sample": f"all {nnz} nonzeros of the workload, all {N} modes, C FP64 oracle "
                      f"(OpenMP over output rows), median of 3 sweeps",
            "per_mode_ms": [t * 1e3 for t in allt],
            "one_thread": {"value": sum(one) * 1e3 * nnz / S,
                           "per_mode_ms": [t * 1e3 * nnz / S for t in one],
                           "sample": f"first {S} nonzeros (draw order), one sweep, time "
                                     f"scaled by nnz/{S}"}}


def run_reference(args, rank, world):
    """The oracle as it stands (the C FP64 spMTTKRP, OpenMP over rows), timed on the
    host cores on the whole workload: every step is a full all-mode sweep over all
    nonzeros.  A sweep takes seconds, so the run keeps at most 2 timed steps and 1
    warm-up step (the line states the numbers it ran and the ones requested)."""
    if rank != 0:
        return
    spec = synth.workload(args.workload)
    R = args.rank or spec.ranks[0]
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    nnz_full = args.nnz or spec.nnz
    coo, vals = synth.make_coo(spec.dims, nnz_full, spec.skew, spec.seed, device=dev)
    coo_h = coo.cpu().numpy()
    vals_h = vals.cpu().numpy()
    del coo, vals
    from oracle import ref_c
    F = [f.numpy().astype(np.float64) for f in synth.make_factors(spec.dims, R, seed=synth.factor_seed(
        WORKLOAD_INDEX[args.workload]))]
    N = len(spec.dims)
    vals64 = vals_h.astype(np.float64)

    def step():
        for n in range(N):
            ref_c.mttkrp(coo_h, vals64, spec.dims, F, n)

    steps, warm = max(1, min(args.steps, 2)), min(args.warmup, 1)
    for _ in range(warm):
        step()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    ms = (time.perf_counter() - t0) / steps * 1e3
    line = {
        "impl": "reference", "metric": "all-mode spMTTKRP ms per sweep", "value": ms,
        "unit": "ms", "n_gpus": args.gpus, "steps": steps, "warmup": warm,
        "steps_requested": args.steps, "warmup_requested": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": spec.name if nnz_full == spec.nnz else
                   f"{spec.name}; reduced to {nnz_full} nonzeros",
                   "dims": list(spec.dims), "nnz": nnz_full, "rank": R},
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": ref_c.threads(), "kind": "oracle",
                         "sample": f"all {coo_h.shape[0]} nonzeros of the workload, all {N} "
                                   f"modes per step, C FP64 oracle (OpenMP over output rows); "
                                   f"{steps} timed step(s) after {warm} warm-up"},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def e2e_pipelined(plan, Fh, Oh, dims, R, dev, stream, K):
    """Mean ms per step of K sweeps whose factors come from pinned host memory and whose
    outputs go back to it, the copies on a second stream overlapping the neighbouring
    steps' sweeps (double-buffered device factors and outputs)."""
    cs = torch.cuda.Stream()
    Fd = [[torch.empty_like(f, device=dev) for f in Fh] for _ in range(2)]
    Od = [[torch.empty(d, R, device=dev) for d in dims] for _ in range(2)]
    h2d_done = [torch.cuda.Event(), torch.cuda.Event()]
    comp_done = [torch.cuda.Event(), torch.cuda.Event()]
    d2h_done = [torch.cuda.Event(), torch.cuda.Event()]

    def run(steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cs.wait_event(e0)
        with torch.cuda.stream(cs):
            for a, b in zip(Fd[0], Fh):
                a.copy_(b, non_blocking=True)
            h2d_done[0].record(cs)
        for k in range(steps):
            b = k % 2
            stream.wait_event(h2d_done[b])
            if k >= 2:
                stream.wait_event(d2h_done[b])  # the outputs of step k-2 have left
            plan.sweep(Fd[b], Od[b], graph=True)
            comp_done[b].record(stream)
            with torch.cuda.stream(cs):
                if k + 1 < steps:
                    nb = (k + 1) % 2
                    if k >= 1:
                        cs.wait_event(comp_done[nb])  # step k-1 has read these factors
                    for a, bb in zip(Fd[nb], Fh):
                        a.copy_(bb, non_blocking=True)
                    h2d_done[nb].record(cs)
                cs.wait_event(comp_done[b])
                for a, bb in zip(Oh, Od[b]):
                    a.copy_(bb, non_blocking=True)
                d2h_done[b].record(cs)
        stream.wait_stream(cs)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    run(2)  # warm-up: graphs for both buffer sets
    return run(K)


def time_events(fn, reps, stream):
    """Mean ms of fn() over reps calls, CUDA events on `stream`, after one warm call."""
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def extra_measurements(args, plan, spec, coo_h, vals_h, F, outs, R, fseed, stream, world):
    """BF16 factor sweep, CP-loss forward+backward throughput (FP32 and BF16) and one
    graph-replayed CP-ALS iteration, on the same tensor."""
    from paper_2405_08470_gb300 import Plan
    from paper_2405_08470_gb300.cp import CPLoss
    dev = F[0].device
    nnz = int(vals_h.shape[0])
    reps = max(2, min(args.steps, 5))
    res = {}
    # CP loss fwd+bwd on the FP32 plan (observed entries = the tensor's values)
    Fg = [(f.float() * 0.1).requires_grad_(True) for f in F]

    def loss_step(pl, fs):
        for f in fs:
            f.grad = None
        CPLoss.apply(pl, *fs).backward()

    ms32 = time_events(lambda: loss_step(plan, Fg), reps, stream)
    res["cp_loss_fwd_bwd"] = {"f32": {"nnz_per_s": nnz / (ms32 * 1e-3), "ms": ms32}}
    # BF16 factors: sweep time and CP loss on a BF16 plan of the same tensor
    pb = Plan(coo_h, vals_h, spec.dims, R, dtype="bf16", nblk=args.nblk, tile=args.tile,
              element_bytes=args.element_bytes)
    Fb = [f.to(torch.bfloat16) for f in F]
    ob = [torch.empty_like(o) for o in outs]
    if args.autotune:
        pb.autotune(Fb, ob)
    msb = time_events(lambda: pb.sweep(Fb, ob, graph=True), reps, stream)
    plan.sweep(F, outs, graph=True)
    torch.cuda.synchronize()
    num = sum(float(torch.linalg.vector_norm((a - b).double())) ** 2 for a, b in zip(ob, outs))
    den = sum(float(torch.linalg.vector_norm(b.double())) ** 2 for b in outs)
    res["bf16_sweep"] = {"ms_per_sweep": msb,
                         "normwise_diff_vs_f32_sweep": (num / den) ** 0.5 if den else None}
    Fbg = [(f * 0.1).to(torch.bfloat16).requires_grad_(True) for f in F]
    msl = time_events(lambda: loss_step(pb, Fbg), reps, stream)
    res["cp_loss_fwd_bwd"]["bf16"] = {"nnz_per_s": nnz / (msl * 1e-3), "ms": msl}
    pb.close()
    del ob, Fb, Fbg
    # the same sweep with the mode-0 copy kept resident (N-1 remap scatters per
    # sweep), and with 3-mode nonzeros unpadded (16 bytes, half-sector remap stores)
    variants = {} if args.keep_base else {"keep_base_sweep": dict(keep_base=True)}
    if len(spec.dims) == 3 and args.element_bytes != 16:
        variants["element_bytes_16_sweep"] = dict(element_bytes=16, keep_base=args.keep_base)
    for name, kw in variants.items():
        pk = Plan(coo_h, vals_h, spec.dims, R, dtype=args.dtype, nblk=args.nblk, tile=args.tile,
                  **kw)
        ok = [torch.empty_like(o) for o in outs]
        if args.autotune:
            pk.autotune(F, ok)
        msk = time_events(lambda: pk.sweep(F, ok, graph=True), reps, stream)
        # tuned plans may cut blocks differently (FP32 sums in another order)
        num = sum(float(torch.linalg.vector_norm((a - b).double())) ** 2 for a, b in zip(ok, outs))
        den = sum(float(torch.linalg.vector_norm(b.double())) ** 2 for b in outs)
        res[name] = {"ms_per_sweep": msk, "config": {k: pk.info()[k] for k in
                                                     ("nblk", "tile", "stages", "variant",
                                                      "elem_bytes", "keep_base")},
                     "normwise_diff_vs_bench_plan": (num / den) ** 0.5 if den else None}
        pk.close()
        del ok
    # the remap scatter on its own: a cycle of N remap-only passes (nonzero stream and
    # next_pos read in order, each nonzero stored at its place in the next mode's
    # order) against a plain device copy of the same bytes
    N = len(spec.dims)
    info = plan.info()
    start = info["cur_mode"]

    def remap_cycle():
        for j in range(1, N + 1):
            plan.remap((start + j) % N)

    ms_remap = time_events(remap_cycle, reps, stream) / N
    nbytes = nnz * info["elem_bytes"]
    src = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    dst = torch.empty_like(src)
    ms_copy = time_events(lambda: dst.copy_(src), reps, stream)
    del src, dst
    res["remap_only_pass"] = {"ms_per_mode": ms_remap, "plain_copy_same_bytes_ms": ms_copy,
                              "elem_bytes": info["elem_bytes"],
                              "note": "a remap pass reads and writes the same bytes as the "
                                      "copy; the gap is the cost of scattered stores"}
    # remap share (the split of the paper's Section 5.2): every mode once more from a
    # copy already in its order, writing no remap, against the same modes in the sweep
    N = len(spec.dims)
    start = plan.info()["cur_mode"]
    no_remap = [0.0] * N
    for j in range(N):
        n = (start + j) % N
        plan.remap(n)  # untimed remap-only passes bring the copy into mode-n order
        no_remap[n] = time_events(lambda: plan.compute(n, F, outs[n], keep_order=True), reps,
                                  stream)
    plan.remap(start)
    t_sweep = time_events(lambda: plan.sweep(F, outs, graph=True), reps, stream)
    res["remap_share"] = {"sweep_ms": t_sweep, "no_remap_per_mode_ms": no_remap,
                          "share": 1.0 - sum(no_remap) / t_sweep}
    # preprocessing (plan build: sorts, remap ids, partition, upload), on the device
    # (the bench plan) and on the host cores
    t0 = time.perf_counter()
    ph = Plan(coo_h, vals_h, spec.dims, R, dtype=args.dtype, plan_on_host=True)
    res["plan_build_s"] = {"device_orders": args.plan_seconds,
                           "host_orders": time.perf_counter() - t0,
                           "host_threads": os.cpu_count()}
    ph.close()
    # one CP-ALS iteration (FP64 Gram/Cholesky on the GPU), replayed as a CUDA graph
    Fa = [f.clone() for f in F]
    lam = torch.empty(R, device=dev)
    fits = [plan.als_iter(Fa, lam)]  # eager run + capture
    t0 = time.perf_counter()
    for _ in range(3):
        fits.append(plan.als_iter(Fa, lam))
    t_als = (time.perf_counter() - t0) / 3 * 1e3
    # the ALS loop as one graph launch (tol 0: every iteration runs); the first
    # call captures it, the second is timed
    loop = 10
    plan.als_run(Fa, lam, loop, 0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run_fits = plan.als_run(Fa, lam, loop, 0.0)
    t_run = (time.perf_counter() - t0) / len(run_fits) * 1e3
    res["cp_als"] = {"ms_per_iter_host_timed_incl_fit_sync": t_als, "fits": fits,
                     "loop_graph": {"iterations": len(run_fits),
                                    "ms_per_iter_host_timed": t_run,
                                    "last_fit": run_fits[-1]}}
    return res


def _sample_rows(dim, k, seed):
    g = np.random.default_rng(seed)
    return np.unique(np.concatenate([g.integers(0, dim, k), [0, dim - 1]]))


def _rows_err(got_rows, want_rows):
    den = float(np.linalg.norm(want_rows))
    return float(np.linalg.norm(got_rows - want_rows)) / den if den else 0.0


def _guard(name, fn, res):
    """Runs one extra measurement; a failure is recorded in the line, not raised."""
    try:
        res[name] = fn()
    except Exception as ex:  # noqa: BLE001 - report and keep the rest of the line
        res[name] = {"error": f"{type(ex).__name__}: {ex}"}
    torch.cuda.empty_cache()


def memory_ceiling(nnz, stream, reps):
    """Memory-system ceilings for the remap's access pattern on this GPU: a copy,
    scattered writes and gathered reads of nnz 32-byte records (random permutation
    of runs of 1, 2 or 4 consecutive records; 4 records = one 128-byte line)."""
    from paper_2405_08470_gb300.binding import memprobe
    a = torch.empty(nnz * 8, dtype=torch.int32, device="cuda")
    b = torch.empty_like(a)
    a.fill_(1)
    out = {"records": nnz, "record_bytes": 32, "buffer_gb": nnz * 32 / 1e9}
    for name, kind, run in (("copy", 0, 1), ("scatter_run1", 1, 1), ("scatter_run2", 1, 2),
                            ("scatter_run4", 1, 4), ("gather_run1", 2, 1)):
        if nnz % run:
            continue
        ms = time_events(lambda: memprobe(kind, a, b, nnz, run, stream), reps, stream)
        out[name] = {"ms": ms, "gbs_read_plus_write": 2 * nnz * 32 / (ms * 1e-3) / 1e9,
                     "g_records_per_s": nnz / (ms * 1e-3) / 1e9}
    del a, b
    return out


def c3_precision(args, stream, reps):
    """Configuration 3: 4-mode 1000000x20000x2000x500, 150M nonzeros, R=32 and 64:
    one all-mode sweep with FP32 and with BF16 factors (autotuned), each with its
    per-mode normwise error against the FP64 oracle on sampled output rows (BF16:
    against the oracle on the BF16-rounded factors, the accumulation error, and
    on the FP32 factors, the quantisation error).  R=32 at the top level, R=64
    under "R64"."""
    import oracle as O
    from paper_2405_08470_gb300 import Plan
    spec = synth.workload("c3")
    coo, vals = synth.make_coo(spec.dims, spec.nnz, spec.skew, spec.seed, device="cuda")
    coo_h, vals_h = coo.cpu().numpy(), vals.cpu().numpy()
    del coo, vals
    torch.cuda.empty_cache()
    rows = [_sample_rows(d, 24, 30 + n) for n, d in enumerate(spec.dims)]

    def one_rank(R):
        F = synth.make_factors(spec.dims, R, seed=synth.factor_seed(2), device="cuda")
        F64 = [f.double().cpu().numpy() for f in F]
        Fq64 = [f.to(torch.bfloat16).double().cpu().numpy() for f in F]
        want = [O.mttkrp_rows(coo_h, vals_h, F64, n, rows[n]) for n in range(4)]
        wantq = [O.mttkrp_rows(coo_h, vals_h, Fq64, n, rows[n]) for n in range(4)]
        res = {}
        for dt in ("f32", "bf16"):
            Fd = [f.to(torch.bfloat16) for f in F] if dt == "bf16" else F
            p = Plan(coo_h, vals_h, spec.dims, R, dtype=dt)
            outs = [torch.empty(d, R, device="cuda") for d in spec.dims]
            p.autotune(Fd, outs)
            ms = time_events(lambda: p.sweep(Fd, outs, graph=True), reps, stream)
            got = [outs[n].cpu().numpy()[rows[n]].astype(np.float64) for n in range(4)]
            e = {"ms_per_sweep": ms, "nblk": p.info()["nblk"], "kernel_form": p.info()["variant"]}
            if dt == "f32":
                e["err_vs_fp64_per_mode"] = [_rows_err(got[n], want[n]) for n in range(4)]
            else:
                e["err_vs_fp64_bf16_factors_per_mode"] = [_rows_err(got[n], wantq[n])
                                                          for n in range(4)]
                e["err_vs_fp64_fp32_factors_per_mode"] = [_rows_err(got[n], want[n])
                                                          for n in range(4)]
            res[dt] = e
            p.close()
            del outs
            torch.cuda.empty_cache()
        del F
        torch.cuda.empty_cache()
        return res

    out = {"workload": spec.name, "rank": 32, "nnz": spec.nnz,
           "rows_checked_per_mode": [len(r) for r in rows]}
    out.update(one_rank(32))
    out["R64"] = one_rank(64)
    return out


def c5_cp_loss(args, stream, reps):
    """Configuration 5: CP completion, 2000000x2000000x100000 with 200M observed
    entries (Zipf 1.1), targets from a planted rank-8 model plus N(0, 0.01) noise,
    fitted factors N(0,1)*0.1 at R=64: CP-loss forward + backward (the autograd
    function) in nonzeros per second with FP32 and BF16 factors, each with its
    gradient error against the FP64 oracle on sampled rows of every mode."""
    import oracle as O
    from paper_2405_08470_gb300 import Plan
    from paper_2405_08470_gb300.cp import CPLoss
    spec = synth.workload("c5")
    R = 64
    coo, _ = synth.make_coo(spec.dims, spec.nnz, spec.skew, spec.seed, device="cuda")
    x = synth.make_planted_targets(coo, spec.dims, 8, 0.1, spec.seed + 1)
    coo_h, x_h = coo.cpu().numpy(), x.cpu().numpy()
    del coo, x
    torch.cuda.empty_cache()
    F = synth.make_factors(spec.dims, R, seed=synth.factor_seed(4), device="cuda", scale=0.1)
    rows = [_sample_rows(d, 16, 50 + n) for n, d in enumerate(spec.dims)]
    out = {"workload": spec.name + ", planted rank-8 targets + N(0,0.01) noise", "rank": R,
           "nnz": spec.nnz, "rows_checked_per_mode": [len(r) for r in rows]}
    G64 = [O.cp_loss_grad_rows(coo_h, x_h, [f.double().cpu().numpy() for f in F], n, rows[n])
           for n in range(3)]
    for dt in ("f32", "bf16"):
        tdt = torch.bfloat16 if dt == "bf16" else torch.float32
        p = Plan(coo_h, x_h, spec.dims, R, dtype=dt)
        Fg = [f.detach().clone().to(tdt).requires_grad_(True) for f in F]
        scratch = [torch.empty(d, R, device="cuda") for d in spec.dims]
        p.autotune([f.detach() for f in Fg], scratch)
        del scratch

        def step():
            for f in Fg:
                f.grad = None
            CPLoss.apply(p, *Fg).backward()

        ms = time_events(step, reps, stream)
        # FP32 gradients straight from the engine (autograd casts BF16 ones to BF16)
        g32 = [torch.empty(d, R, device="cuda") for d in spec.dims]
        lossv = torch.empty((), device="cuda")
        fs = [f.detach() for f in Fg]
        p.loss_fwd(fs, lossv)
        p.loss_bwd(fs, torch.ones((), device="cuda"), g32)
        got = [g32[n].cpu().numpy()[rows[n]].astype(np.float64) for n in range(3)]
        e = {"ms_fwd_bwd": ms, "nnz_per_s": spec.nnz / (ms * 1e-3), "loss": float(lossv)}
        if dt == "f32":
            e["grad_err_vs_fp64_per_mode"] = [_rows_err(got[n], G64[n]) for n in range(3)]
        else:
            Fq = [f.to(torch.bfloat16).double().cpu().numpy() for f in F]
            Gq = [O.cp_loss_grad_rows(coo_h, x_h, Fq, n, rows[n]) for n in range(3)]
            e["grad_err_vs_fp64_bf16_factors_per_mode"] = [_rows_err(got[n], Gq[n])
                                                           for n in range(3)]
            e["grad_err_vs_fp64_fp32_factors_per_mode"] = [_rows_err(got[n], G64[n])
                                                           for n in range(3)]
        out[dt] = e
        p.close()
        del Fg, g32, fs
        torch.cuda.empty_cache()
    return out


def c4_als(args, stream, reps):
    """Configuration 4: one CPD-ALS iteration (every mode's fused pass, the FP64
    Gram Hadamard and Cholesky on the GPU, the solve and the column scaling,
    replayed as one CUDA graph) on the 5-mode 60M and 6-mode 40M tensors at
    R = 16, 32, 64, each plan autotuned; host-timed per iteration including the
    read-back of the fit (median of 5 after the capture); and the ALS loop as one
    graph launch (cp_als_run, five iterations), host-timed per iteration."""
    from paper_2405_08470_gb300 import Plan
    out = {}
    for name, ci in (("c4a", 3), ("c4b", 3)):
        spec = synth.workload(name)
        coo, vals = synth.make_coo(spec.dims, spec.nnz, spec.skew, spec.seed, device="cuda")
        coo_h, vals_h = coo.cpu().numpy(), vals.cpu().numpy()
        del coo, vals
        torch.cuda.empty_cache()
        ent = {"workload": spec.name}
        for R in spec.ranks:
            p = Plan(coo_h, vals_h, spec.dims, R)
            F = synth.make_factors(spec.dims, R, seed=synth.factor_seed(ci), device="cuda")
            scratch = [torch.empty(d, R, device="cuda") for d in spec.dims]
            p.autotune(F, scratch)
            t0 = time.perf_counter()
            p.sweep(F, scratch, graph=True)
            torch.cuda.synchronize()
            sweep_ms = time_events(lambda: p.sweep(F, scratch, graph=True), reps, stream)
            del scratch
            lam = torch.empty(R, device="cuda")
            fits = [p.als_iter(F, lam)]  # eager + capture
            ts = []
            for _ in range(5):
                t0 = time.perf_counter()
                fits.append(p.als_iter(F, lam))
                ts.append((time.perf_counter() - t0) * 1e3)
            # the ALS loop as one graph launch (column scales folded; 5 iterations,
            # tol 0): the first call captures it, the second is timed
            p.als_run(F, lam, 5, 0.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            run_fits = p.als_run(F, lam, 5, 0.0)
            t_run = (time.perf_counter() - t0) / len(run_fits) * 1e3
            ent[f"R{R}"] = {"als_iter_ms": float(np.median(ts)), "sweep_ms": sweep_ms,
                            "fits": fits, "nblk": p.info()["nblk"],
                            "kernel_form": p.info()["variant"],
                            "loop_graph_ms_per_iter": t_run, "loop_last_fit": run_fits[-1]}
            p.close()
            del F
            torch.cuda.empty_cache()
        out[name] = ent
    return out


def main():
    args = parse()
    rank, world = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    from paper_2405_08470_gb300 import Plan, _build
    _build.build()
    dev = torch.device("cuda")
    spec, coo, vals = workload_tensors(args.workload, args.nnz, dev)
    N = len(spec.dims)
    R = args.rank or spec.ranks[0]
    nnz = int(coo.shape[0])
    s = 2 if args.dtype == "bf16" else 4
    tdt = torch.bfloat16 if args.dtype == "bf16" else torch.float32
    fseed = synth.factor_seed(WORKLOAD_INDEX[args.workload])
    F = [f.to(tdt) for f in synth.make_factors(spec.dims, R, seed=fseed, device=dev)]
    touched = [int(torch.unique(coo[:, k]).numel()) for k in range(N)]
    coo_h = coo.cpu().numpy()
    vals_h = vals.cpu().numpy()
    del coo, vals
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    plan = Plan(coo_h, vals_h, spec.dims, R, dtype=args.dtype, nblk=args.nblk, tile=args.tile,
                variant=args.variant, unroll=args.unroll, cache_hints=args.hints,
                stages=args.stages, element_bytes=args.element_bytes,
                keep_base=args.keep_base, partition=args.partition)
    plan_s = time.perf_counter() - t0
    args.plan_seconds = plan_s
    outs = [torch.empty(d, R, device=dev) for d in spec.dims]
    tune_s = None
    # an explicitly requested launch configuration is measured as given
    args.autotune = args.autotune and not (args.nblk or args.tile or args.stages or args.variant
                                           or args.unroll)
    if args.autotune:
        t0 = time.perf_counter()
        plan.autotune(F, outs)
        tune_s = time.perf_counter() - t0
    info = plan.info()
    stream = torch.cuda.current_stream()

    # warm-up (untimed)
    for _ in range(args.warmup):
        plan.sweep(F, outs)
    torch.cuda.synchronize()

    # timed region: K sweeps, CUDA events around every mode's launches
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(N + 1)] for _ in range(K)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.4)
    barrier(world)
    torch.cuda.synchronize()
    start_mode = info["cur_mode"]
    for i in range(K):
        ev[i][0].record(stream)
        for j in range(N):
            n = (start_mode + j) % N
            plan.compute(n, F, outs[n])
            ev[i][j + 1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    per_mode = np.zeros(N)
    total = 0.0
    for i in range(K):
        total += ev[i][0].elapsed_time(ev[i][N])
        for j in range(N):
            per_mode[(start_mode + j) % N] += ev[i][j].elapsed_time(ev[i][j + 1])
    ms = total / K
    per_mode /= K
    ms = max_over_ranks(ms, world)

    peak, peak_kind = load_peaks()
    byts = compulsory_bytes(spec.dims, nnz, R, s, touched, N, args.keep_base)
    t_roof_ms = sum(byts) / (peak * 1e9) * 1e3
    achieved = sum(byts) / (per_mode.sum() * 1e-3) / 1e9
    traffic = ncu_traffic(args.workload, R, args.dtype, nnz,
                          dict(info, unroll=args.unroll or 8, cache_hints=args.hints,
                               blocks_per_sm=info["nblk"] / info["num_sms"]))
    # per-nonzero gathers counted every time (no reuse in L1/L2), for comparison
    E = 4 * N + 4
    no_reuse = sum(nnz * (E + 4 + E) + nnz * (N - 1) * R * s + spec.dims[n] * R * 4
                   for n in range(N))

    # end to end through the public API with host buffers: H2D factors, sweep, D2H outputs
    e2e = None
    if not args.no_e2e:
        Fh = [f.cpu().pin_memory() for f in F]
        Oh = [torch.empty(d, R, pin_memory=True) for d in spec.dims]
        Fd = [torch.empty_like(f, device=dev) for f in Fh]
        h2d = sum(f.numel() * f.element_size() for f in Fh)
        d2h = sum(o.numel() * o.element_size() for o in Oh)
        for _ in range(2):
            for a, b in zip(Fd, Fh):
                a.copy_(b, non_blocking=True)
            plan.sweep(Fd, outs, graph=True)
            for a, b in zip(Oh, outs):
                a.copy_(b, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        e0.record(stream)
        for _ in range(K):
            for a, b in zip(Fd, Fh):
                a.copy_(b, non_blocking=True)
            plan.sweep(Fd, outs, graph=True)
            for a, b in zip(Oh, outs):
                a.copy_(b, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        serial_ms = max_over_ranks(e0.elapsed_time(e1) / K, world)
        del Fd
        barrier(world)
        piped_ms = max_over_ranks(e2e_pipelined(plan, Fh, Oh, spec.dims, R, dev, stream, K), world)
        same = all(torch.equal(a, b.cpu()) for a, b in zip(Oh, outs))
        e2e = {"value": piped_ms, "unit": "ms", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "how": "every step copies its factors from pinned host memory and its outputs "
                      "back; copies run on a second stream, two steps deep (double-buffered "
                      "device factors and outputs), all inside the timed region",
               "serial_value": serial_ms, "outputs_equal_serial_run": same}

    extra = {}
    if not args.no_extras:
        extra = extra_measurements(args, plan, spec, coo_h, vals_h, F, outs, R, fseed, stream, world)
    if e2e is not None:
        # one shot from host data: plan build from the host COO (sorts, remap ids,
        # partition, uploads), factors uploaded, one sweep, outputs read back
        Fh1 = [f.cpu() for f in F]
        plan.close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p1 = Plan(coo_h, vals_h, spec.dims, R, dtype=args.dtype, nblk=args.nblk,
                  tile=args.tile, variant=info["variant"], element_bytes=args.element_bytes,
                  keep_base=args.keep_base, partition=args.partition)
        Fd1 = [f.to(dev) for f in Fh1]
        p1.sweep(Fd1, outs)
        Oh1 = [o.cpu() for o in outs]
        torch.cuda.synchronize()
        e2e["one_shot_ms"] = (time.perf_counter() - t0) * 1e3
        e2e["one_shot_how"] = ("host COO (int64) and values to outputs on the host: plan build "
                               "(device sorts, remap ids, write orders, partition, uploads), "
                               "factor upload, one all-mode sweep, output download; host-timed")
        del Oh1, Fd1, Fh1
        plan = p1
    plan.close()
    del F, outs
    torch.cuda.empty_cache()
    if not (args.no_extras or args.no_workload_extras) and world == 1 and nnz == spec.nnz \
            and args.workload == "c2":
        reps = max(2, min(args.steps, 5))
        _guard("memory_ceiling", lambda: memory_ceiling(nnz, stream, reps), extra)
        _guard("c3_fp32_vs_bf16", lambda: c3_precision(args, stream, reps), extra)
        _guard("cp_loss_c5", lambda: c5_cp_loss(args, stream, reps), extra)
        _guard("cp_als_c4", lambda: c4_als(args, stream, reps), extra)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_full(coo_h, vals_h, spec.dims, R, fseed)

    launches = info["launches_per_sweep"] * K
    if rank == 0:
        line = {
            "metric": "all-mode spMTTKRP ms per sweep", "value": ms, "unit": "ms",
            "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": spec.name if nnz == spec.nnz else
                       f"{spec.name}; reduced to {nnz} nonzeros",
                       "dims": list(spec.dims), "nnz": nnz, "rank": R,
                       "factor_dtype": args.dtype, "nblk": info["nblk"], "tile": info["tile"],
                       "kernel_form": ["warp blocks, bulk-async staged tiles",
                                       "CTA blocks, direct runs",
                                       "persistent CTAs, 960-nonzero tiles, remap stores in "
                                       "destination order",
                                       "warp blocks, bulk-async staged tiles, one remap warp "
                                       "per CTA storing in destination order"][info["variant"]],
                       "autotuned": bool(args.autotune),
                       "unroll": args.unroll or 8, "cache_hints": args.hints,
                       "stages": info["stages"],
                       "element_bytes": info["elem_bytes"],
                       "keep_base": bool(args.keep_base),
                       "partition": ["contiguous split, heavy rows split",
                                     "Algorithm 1 (LPT), rows never split"][args.partition],
                       "l2": "inputs larger than L2 (element stream "
                             f"{nnz * info['elem_bytes'] / 1e9:.2f} GB per mode)",
                       "parallelism": f"replicas x{world}"},
            "pct_hbm_roofline": t_roof_ms / ms,
            "t_roof_ms": t_roof_ms,
            "per_mode_ms": per_mode.tolist(),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "kernel": ["mttkrp_warp_kernel", "mttkrp_direct_kernel",
                                    "mttkrp_tile_kernel", "mttkrp_warp_kernel"][info["variant"]] +
                                   " (+ split-row fix-up; CUDA events around each mode)",
                         "algorithmic_bytes_per_sweep": int(sum(byts)),
                         "no_reuse_bytes_per_sweep": int(no_reuse),
                         "dram_gbs_ncu_bytes_over_event_time": (traffic * N / (per_mode.sum() * 1e-3) / 1e9
                                          if traffic else None),
                         "nominal_hbm_gbs": 7900.0},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
            "plan_seconds": plan_s,
            "autotune_seconds": tune_s,
            "touched_rows": touched,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
