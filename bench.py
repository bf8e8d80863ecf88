#!/usr/bin/env python
"""Effective GFLOPS (2MNK / time) of the recursive Strassen-Winograd SGEMM
against the library's own classical tensor-core GEMM on one GB300.

One step = one C = A*B call of the whole hot path (pre-additions, all leaf
products in one tcgen05 launch, post-additions) on square n x n fp32 operands
(default n = 16384, A, B ~ U[-1, 1] from a fixed seed; each operand 1.07 GB,
larger than the 129 MB L2, so no flush is needed between steps).

  value   device-resident operands, CUDA events around K steps on the
          launching stream, max over ranks, GFLOPS summed over ranks
  e2e     the same call with operands in pinned host memory: every step
          copies A and B in and C out inside the timed region
Multi-GPU runs are independent replicas (weak scaling): the method has no
exchange step on one problem, so no collective touches the data path.

``--impl reference`` times the CPU oracle (``oracle/``) as it stands on the
host cores, each step a bounded sample of the same workload (one of the seven
root products of the n = 16384 depth-3 call: n = 8192 at depth 2).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TF32_OVER_BF16 = 1.1 / 2.25   # nominal dense tensor-rate ratio, GB300


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fmm", choices=["fmm", "reference"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--depth", type=int, default=-1, help="-1: planner default")
    ap.add_argument("--leaf-tile", type=int, default=0)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--no-classical", action="store_true")
    ap.add_argument("--no-residual", action="store_true", help="skip timing the Freivalds residual check")
    ap.add_argument("--no-split", action="store_true",
                    help="skip the split-precision (FP16x3, BF16x3) runs reported beside plain FP32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="square",
                    choices=["square", "single1024", "sweep", "fine_sweep", "large", "rmul", "split", "batched",
                             "planner", "residual", "profile_case"],
                    help="square: the headline line; the others measure the other configurations")
    ap.add_argument("--out", default=None, help="also append the JSON lines to this file")
    ap.add_argument("--model-out", default=None,
                    help="planner workload: write the trained cost model to this file")
    ap.add_argument("--sizes", default=None, help="fine_sweep: comma-separated sizes instead of 4096..20480 step 256")
    ap.add_argument("--odd", default="auto", choices=["pad", "peel", "tile", "auto"],
                    help="fine_sweep: odd-size mode of the Winograd plans")
    ap.add_argument("--fuse-last", type=int, default=0, choices=[-1, 0, 1],
                    help="profile_case: last Winograd level in the leaf launch (1), separate (-1), library default (0)")
    ap.add_argument("--calls", type=int, default=3, help="profile_case: calls of the plan")
    ap.add_argument("--host-copy", default="default", choices=["default", "engine", "sm"],
                    help="e2e leg: how host operands cross the link (library default, copy engines, SM copies)")
    ap.add_argument("--model-in", default=None,
                    help="batched workload: a trained cost model (planner workload's --model-out) for the learned planner")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []          # (host time, csv line) per sample
        self.window = None       # host-time bounds of the timed region

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line))

    def start(self):
        """Start sampling and wait (up to 5 s) for the first sample, so that the
        sampler is running before the timed region begins."""
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 5.0:
            time.sleep(0.02)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.reader.join(timeout=5)
        return summarize_clock_samples(self.lines, self.window)


def summarize_clock_samples(lines, window):
    """Median SM clock, maximum SM clock and the throttle reasons seen, from
    (host time, nvidia-smi csv line) samples (the query of Clocks.Q); only the
    samples inside `window` (host-time bounds of the timed region) when there
    are any.  None without a usable sample."""
    where = "whole run"
    if window:
        inside = [x for x in lines if window[0] <= x[0] <= window[1]]
        if inside:
            lines, where = inside, "timed region"
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for _, line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
            "samples_in": where,
            "reasons": sorted(reasons)}


def source_sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def ncu_traffic(kernel_file, workload_key, path=None):
    """Per-launch DRAM bytes of the leaf kernel from the committed ncu summary,
    valid only while the kernel source is the one that was profiled."""
    path = path or os.path.join(ROOT, "profiles", "leaf_gemm_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("source_sha") != source_sha(kernel_file):
        return None
    v = rec.get("per_launch_bytes", {}).get(workload_key)
    return float(v) if v is not None else None


# ---------------------------------------------------------------------------------- oracle legs

def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def cpu_threads():
    """Threads the oracle's BLAS calls use: the cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def cpu_oracle_headline(A, B, depth, rows=64):
    """The oracle at the headline configuration: one fp32 Winograd call (O2, numpy,
    the bench's depth) on the full n x n operands, and the float64 classical
    definition (O1) on `rows` sampled rows, both timed on the host cores."""
    import numpy as np
    from oracle import fmm_oracle as O
    n = A.shape[0]
    t0 = time.perf_counter()
    O.winograd(A, B, depth, "pad")
    t_w = time.perf_counter() - t0
    r = np.random.default_rng(7).choice(n, size=rows, replace=False)
    t0 = time.perf_counter()
    O.classical_rows(A, B, r)
    t_c = time.perf_counter() - t0
    return {"value": round(2.0 * n ** 3 / t_w / 1e9, 2), "unit": "GFLOPS", "cores": cpu_threads(),
            "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"one fp32 Winograd oracle call (numpy, depth {depth}) on the full n={n} operands "
                      f"in {t_w:.1f} s; float64 classical definition on {rows} sampled rows in {t_c:.2f} s "
                      f"({2.0 * rows * n * n / t_c / 1e9:.1f} GFLOPS)"}


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores.  Each step is a bounded sample
    of the headline workload: one of the seven root products of the n x n,
    depth-3 call, i.e. an (n/2)^3 fp32 Winograd product at depth 2; throughput is
    its effective 2 (n/2)^3 / t."""
    if rank != 0:
        return
    n = max(args.n // 2, 2)
    depth = 2
    from oracle import fmm_oracle as O
    from paper_1205_2927_gb300 import inputs as I
    A, B = I.operands(n, n, n, I.seed_for(2, 0))
    for _ in range(args.warmup):
        O.winograd(A, B, depth, "pad")
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.winograd(A, B, depth, "pad")
    el = time.perf_counter() - t0
    val = 2.0 * n ** 3 * args.steps / el / 1e9
    sample = (f"fp32 Winograd oracle (numpy) on one root product of the n={args.n} depth-3 call per step: "
              f"n={n}, depth {depth}")
    line = {"impl": "reference", "metric": "effective GFLOPS (2MNK/s) Winograd vs classical GEMM on 1 GB300 at stated error",
            "value": round(val, 2), "unit": "GFLOPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"winograd_fp32_square_n{args.n}", "n": args.n, "sample_n": n, "depth": 3},
            "cpu_baseline": {"value": round(val, 2), "unit": "GFLOPS", "cores": cpu_threads(), "cpu_model": cpu_model(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(val, 2), "unit": "GFLOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------- GPU legs

def sampled_error(np, torch, dC, A_h, B_h, nrows=16, seed=1):
    """max|C - C64| / (max|A| max|B| K) over `nrows` random rows; C64 rows by a
    float64 matrix product on the host."""
    m, k = A_h.shape
    rows = np.sort(np.random.default_rng(seed).choice(m, size=min(nrows, m), replace=False))
    C_rows = dC[torch.from_numpy(rows).to(dC.device)].cpu().numpy().astype(np.float64)
    ref = A_h[rows].astype(np.float64) @ B_h.astype(np.float64)
    return float(np.max(np.abs(C_rows - ref))) / (float(np.abs(A_h).max()) * float(np.abs(B_h).max()) * k)


def emit(args, rec):
    line = json.dumps(rec)
    print(line, flush=True)
    if args.out:
        with open(args.out, "a") as f:
            f.write(line + "\n")


def event_ms(torch, fn, steps, warmup):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(steps):
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        ts.append(s.elapsed_time(e))
    ts.sort()
    return ts[len(ts) // 2]


def wl_single1024(args):
    """n = 1024, depth 2 (leaf 256), device-resident single call: median of 20 after 5 warm-ups."""
    import numpy as np
    import torch
    from paper_1205_2927_gb300 import fmm, inputs
    n = 1024
    A_h, B_h = inputs.operands(n, n, n, inputs.seed_for(1, 0))
    dA, dB = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
    dC = torch.empty((n, n), device="cuda")
    for d in (0, 2):
        p = fmm.Plan(n, n, n, depth=d)
        ms = event_ms(torch, lambda: p(dA, dB, dC), 20, 5)
        emit(args, {"workload": "single_n1024", "depth": d, "leaf_tile": p.info["leaf_tile"], "ms": round(ms, 4),
                    "gflops": round(2 * n ** 3 / ms / 1e6, 1), "error": sampled_error(np, torch, dC, A_h, B_h, 64)})
        p.close()


def wl_sweep(args):
    """n in {4096, 8192, 16384, 19000} x depth 0..4, U[-1,1] and N(0,1): device-resident
    time and host-resident wall-clock (pinned operands, transfers inside), error on sampled rows."""
    import numpy as np
    import torch
    from paper_1205_2927_gb300 import fmm, inputs
    for n in (4096, 8192, 16384, 19000):
        for dist in ("uniform", "normal"):
            A_h, B_h = inputs.operands(n, n, n, inputs.seed_for(2, n % 97), dist)
            dA, dB = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
            dC = torch.empty((n, n), device="cuda")
            pA, pB = torch.from_numpy(A_h).pin_memory(), torch.from_numpy(B_h).pin_memory()
            pC = torch.empty((n, n)).pin_memory()
            for d in range(0, 5):
                for odd in (("pad", "peel", "auto") if n == 19000 and d > 0 else ("pad",)):
                    p = fmm.Plan(n, n, n, depth=d, odd=odd)
                    ms = event_ms(torch, lambda: p(dA, dB, dC), 3, 2)
                    err = sampled_error(np, torch, dC, A_h, B_h)
                    tile = p.info["leaf_tile"]
                    p.close()
                    wall = None
                    if odd == "pad" and dist == "uniform":
                        hp = fmm.Plan(n, n, n, depth=d, host_operands=1)
                        for _ in range(2):
                            hp(pA, pB, pC)
                        torch.cuda.synchronize()
                        ws = []
                        for _ in range(3):
                            t0 = time.perf_counter()
                            hp(pA, pB, pC)
                            torch.cuda.current_stream().synchronize()
                            ws.append((time.perf_counter() - t0) * 1e3)
                        wall = sorted(ws)[1]
                        hp.close()
                    emit(args, {"workload": "sweep", "n": n, "depth": d, "leaf_tile": tile, "odd": odd, "dist": dist,
                                "device_ms": round(ms, 3), "device_gflops": round(2 * n ** 3 / ms / 1e6, 1),
                                "host_wallclock_ms": round(wall, 3) if wall else None,
                                "host_gflops": round(2 * n ** 3 / wall / 1e6, 1) if wall else None,
                                "error": err})
            del dA, dB, dC, pA, pB, pC
            torch.cuda.empty_cache()


def wl_fine_sweep(args):
    """Square n from 4096 to 20480 in steps of 256, U[-1,1], device-resident FP32:
    the classical GEMM (depth 0) and Winograd at depths 1-3 where every leaf
    dimension stays >= 1024, CUDA-event median of 3 calls after 1 warm-up.  The
    rows show how much of a saw-tooth over n remains (leaf-tile quantisation,
    padding to the level granule, the choice of depth)."""
    import torch
    from paper_1205_2927_gb300 import fmm, inputs
    sizes = [int(x) for x in args.sizes.split(",")] if args.sizes else list(range(4096, 20480 + 1, 256))
    for n in sizes:
        A_h, B_h = inputs.operands(n, n, n, inputs.seed_for(2, 40 + n // 256))
        dA, dB = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
        dC = torch.empty((n, n), device="cuda")
        rec = {"workload": "fine_sweep", "n": n, "odd": args.odd}
        for d in range(0, 4):
            if d > 0 and (n >> d) < 1024:
                break
            p = fmm.Plan(n, n, n, depth=d, odd=args.odd if d > 0 else "pad")
            ms = event_ms(torch, lambda: p(dA, dB, dC), 3, 1)
            assert p.device_status() == 0
            taken = p.info["odd"]
            p.close()
            rec[f"d{d}_ms"] = round(ms, 3)
            rec[f"d{d}_tflops"] = round(2.0 * n ** 3 / ms / 1e9, 1)
            if taken != 0:
                # the mode taken is not padding: time the padded plan beside it on the same GPU
                rec[f"d{d}_odd"] = {1: "peel", 2: "tile"}.get(taken, taken)
                q = fmm.Plan(n, n, n, depth=d, odd="pad")
                pms = event_ms(torch, lambda: q(dA, dB, dC), 3, 1)
                q.close()
                rec[f"d{d}_pad_ms"] = round(pms, 3)
        best = min((rec[f"d{d}_ms"], d) for d in range(4) if f"d{d}_ms" in rec)
        rec["best_depth"] = best[1]
        rec["speedup_vs_d0"] = round(rec["d0_ms"] / best[0], 3)
        emit(args, rec)
        del dA, dB, dC
        torch.cuda.empty_cache()


def wl_large(args):
    """n = 32768 (4.3 GB per matrix), U[-1,1], device-resident, depth 0 (classical) and the
    deep plans where the additions' n^2 cost falls behind the leaves' n^3 work; CUDA-event
    median of 3 calls after 2 warm-ups, error on sampled rows."""
    import numpy as np
    import torch
    from paper_1205_2927_gb300 import fmm, inputs
    n = 32768
    A_h, B_h = inputs.operands(n, n, n, inputs.seed_for(2, 5))
    dA, dB = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
    dC = torch.empty((n, n), device="cuda")
    base = None
    for d in (0, 3, 4):
        p = fmm.Plan(n, n, n, depth=d)
        p.profile(True)
        ms = event_ms(torch, lambda: p(dA, dB, dC), 3, 2)
        prof = p.profile_read()
        calls = max(prof["calls"], 1)
        err = sampled_error(np, torch, dC, A_h, B_h, 8)
        tile = p.info["leaf_tile"]
        ws_gb = p.workspace.numel() / 1e9
        p.close()
        del p
        torch.cuda.empty_cache()
        base = ms if d == 0 else base
        emit(args, {"workload": "large_n32768", "depth": d, "leaf_tile": tile, "ms": round(ms, 2),
                    "gflops": round(2 * n ** 3 / ms / 1e6, 1), "speedup_vs_depth0": round(base / ms, 3),
                    "pre_ms": round(prof["pre_ms"] / calls, 2), "leaf_ms": round(prof["leaf_ms"] / calls, 2),
                    "post_ms": round(prof["post_ms"] / calls, 2), "workspace_gb": round(ws_gb, 1), "error": err})


def wl_rmul(args):
    """The classical quadrant recursion of Table 1 (RMUL, k-blocks accumulated in C)
    against Winograd at the same depth, n = 16384, U[-1,1], device-resident, CUDA-event
    median of 3 calls after 2 warm-ups; error on sampled rows."""
    import numpy as np
    import torch
    from paper_1205_2927_gb300 import fmm, inputs
    n = 16384
    A_h, B_h = inputs.operands(n, n, n, inputs.seed_for(2, 0))
    dA, dB = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
    dC = torch.empty((n, n), device="cuda")
    for algo in ("classical", "winograd"):
        for d in (0, 1, 2, 3):
            if algo == "winograd" and d == 0:
                continue
            p = fmm.Plan(n, n, n, depth=d, algo=algo)
            ms = event_ms(torch, lambda: p(dA, dB, dC), 3, 2)
            err = sampled_error(np, torch, dC, A_h, B_h)
            p.close()
            emit(args, {"workload": "rmul_vs_winograd_n16384", "algo": algo, "depth": d, "ms": round(ms, 3),
                        "gflops": round(2 * n ** 3 / ms / 1e6, 1), "error": err})


def wl_split(args):
    """Split-precision leaves: {fp32 (3xTF32), tf32, bf16x3, fp16x3} x depth 0..4 on
    19000x12000x15000 and 16384^3, entries N(0,1) and log-uniform [1e-3, 1e3]; error
    against a float64 product on sampled rows, and throughput."""
    import numpy as np
    import torch
    from paper_1205_2927_gb300 import fmm, inputs
    for (m, k, n) in ((19000, 12000, 15000), (16384, 16384, 16384)):
        for dist in ("normal", "loguniform"):
            A_h, B_h = inputs.operands(m, k, n, inputs.seed_for(3, m % 89), dist)
            dA, dB = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
            dC = torch.empty((m, n), device="cuda")
            for prec in ("fp32", "tf32", "bf16x3", "fp16x3"):
                for d in range(0, 5):
                    p = fmm.Plan(m, n, k, depth=d, precision=prec)
                    ms = event_ms(torch, lambda: p(dA, dB, dC), 2, 1)
                    err = sampled_error(np, torch, dC, A_h, B_h)
                    tile = p.info["leaf_tile"]
                    p.close()
                    emit(args, {"workload": "split", "M": m, "K": k, "N": n, "dist": dist, "precision": prec,
                                "depth": d, "leaf_tile": tile, "ms": round(ms, 3), "gflops": round(2 * m * n * k / ms / 1e6, 1),
                                "error": err, "finite": bool(torch.isfinite(dC).all().item())})
            del dA, dB, dC
            torch.cuda.empty_cache()


def wl_batched(args):
    """512 independent products, M, K, N log-uniform in [128, 4096] (multiples of 4),
    U[-1,1]; one persistent leaf launch per replay of a CUDA graph.  The plan
    comes from the library: the fixed rule, the exhaustive per-size-class tuner
    (fmm_batched_plan with planner="exhaustive": whole-batch timings, one depth
    per class, one leaf tile per launch) and, with --model-in, the learned
    planner (`--precision` selects the leaves: fp32 = 3xTF32, tf32, bf16x3,
    fp16x3)."""
    import numpy as np
    import torch
    from paper_1205_2927_gb300 import fmm, inputs
    from paper_1205_2927_gb300 import planner as PL
    shapes = inputs.batched_shapes(512, inputs.seed_for(4, 0))
    flops = sum(2.0 * m * k * n for m, k, n in shapes)
    As = [torch.from_numpy(inputs.uniform((m, k), inputs.seed_for(4, 1) + 3 * i)).cuda() for i, (m, k, n) in enumerate(shapes)]
    Bs = [torch.from_numpy(inputs.uniform((k, n), inputs.seed_for(4, 2) + 3 * i)).cuda() for i, (m, k, n) in enumerate(shapes)]
    Cs = [torch.empty((m, n), device="cuda") for m, k, n in shapes]
    probe = tensor_peak(fmm, 0, "tf32" if args.precision in ("fp32", "tf32") else "bf16")
    pk = peaks()[0]
    tc_products = 1 if args.precision == "tf32" else 3
    es = 4 if args.precision in ("fp32", "tf32") else 2
    planners = ["fixed", "exhaustive"]
    if args.model_in:
        PL.register(*PL.load(args.model_in))
        planners.append("mlp")
    for planner in planners:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bp = fmm.BatchedPlan(As, Bs, Cs, planner=planner, precision=args.precision)
        torch.cuda.synchronize()
        plan_s = time.perf_counter() - t0
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            bp.run(s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            bp.run(torch.cuda.current_stream())
        ms = event_ms(torch, g.replay, 20, 3)
        info = bp.info()
        errs = []
        for i in range(0, 512, 37):
            A_h, B_h = As[i].cpu().numpy(), Bs[i].cpu().numpy()
            ref = A_h.astype(np.float64) @ B_h.astype(np.float64)
            errs.append(float(np.max(np.abs(Cs[i].cpu().numpy() - ref))) /
                        (float(np.abs(A_h).max()) * float(np.abs(B_h).max()) * A_h.shape[1]))
        depth_hist = {d: int(sum(1 for x in info["depths"] if x == d)) for d in sorted(set(info["depths"]))}
        # roofline of the replay: tensor work of every leaf (padded to the level
        # granule, 7^d leaves per recursing problem) against the probe's rate, plus
        # the split pass of the depth-0 operands and the C writes against HBM
        leaf_flops, hbm_bytes = 0.0, 0.0
        for (m, k, n), d in zip(shapes, info["depths"]):
            g = 4 << d if d > 0 else 1
            m0, k0, n0 = -(-m // g) * g, -(-k // g) * g, -(-n // g) * g
            leaf_flops += tc_products * 2.0 * (7 ** d) * (m0 >> d) * (k0 >> d) * (n0 >> d)
            hbm_bytes += 4.0 * m * n + ((m * k + k * n) * (4 + 2 * es) if d == 0 and args.precision != "tf32"
                                        else 0.0)
        t_star = (leaf_flops / (probe["tflops"] * 1e12) + hbm_bytes / (pk["hbm_gbs"] * 1e9)) * 1e3
        emit(args, {"workload": "batched512", "precision": args.precision, "planner": planner,
                    "leaf_tile": info["leaf_tile"], "size_classes": info["nclasses"], "depths": depth_hist,
                    "graph_replay_ms": round(ms, 3), "gflops": round(flops / ms / 1e6, 1), "total_flops": flops,
                    "plan_s": round(plan_s, 2), "leaf_tiles": info["total_tiles"],
                    "max_error_sampled": max(errs),
                    "roofline": {"bound": "tensor", "tensor_tflops_over_replay": round(leaf_flops / ms / 1e9, 1),
                                 "peak": round(probe["tflops"], 1), "unit": "TFLOP/s",
                                 "frac": round(leaf_flops / ms / 1e9 / probe["tflops"], 3),
                                 "leaf_tensor_flops": leaf_flops, "split_and_c_bytes": hbm_bytes,
                                 "t_star_ms": round(t_star, 3), "t_star_over_measured": round(t_star / ms, 3),
                                 "model": "leaf flops / probe rate + split and C bytes / HBM copy bandwidth"}})
        del g
        bp.close()
    if args.model_in:
        fmm.fmm_set_cost_model(None)


def wl_residual(args):
    """The Freivalds residual check alone at n x n (A, B, C U[-1,1], a +-1 probe):
    one pass over A, B and C per call, fp32 and fp64 accumulation; CUDA events
    over 10 calls after 2 warm-ups."""
    import torch
    from paper_1205_2927_gb300 import fmm, inputs
    n = args.n
    A, B, C = (torch.from_numpy(inputs.uniform((n, n), inputs.seed_for(5, i))).cuda() for i in range(3))
    x = torch.from_numpy(inputs.rademacher(n, inputs.seed_for(5, 3))).cuda()
    nbytes = 4.0 * 3 * n * n
    peak = peaks()[0]["hbm_gbs"]
    for name, fp64 in (("fp32", False), ("fp64", True)):
        ms = event_ms(torch, lambda: fmm.fmm_residual(A, B, C, x, fp64=fp64), 10, 2)
        emit(args, {"workload": "residual", "n": n, "accumulation": name, "ms": round(ms, 4),
                    "achieved_gbs": round(nbytes / ms / 1e6, 1), "frac": round(nbytes / ms / 1e6 / peak, 3)})


def wl_planner(args):
    """Learned planner: ~20k candidate timings on shapes of the other configurations,
    network trained on the GPU, plans picked for 1000 unseen shapes; compared with
    the exhaustive autotuner (planning time, chosen-plan GFLOPS) and the fixed rule."""
    import numpy as np
    import torch
    from paper_1205_2927_gb300 import fmm, inputs
    from paper_1205_2927_gb300 import planner as PL
    rng = np.random.default_rng(inputs.seed_for(5, 0))
    big = [(int(a), int(b), int(c)) for a, b, c in (rng.integers(1024, 4864, size=(160, 3)) * 4)]
    squares = [(n, n, n) for n in (4096, 8192, 16384, 19000)]
    train_shapes = (inputs.batched_shapes(5200, inputs.seed_for(5, 1)) + big + squares
                    + [(19000, 12000, 15000), (16384, 16384, 16384)])
    test_shapes = inputs.batched_shapes(1000, inputs.seed_for(5, 2))
    t0 = time.perf_counter()
    recs = PL.collect(train_shapes, reps=1, seed=5)
    t_collect = time.perf_counter() - t0
    X, y = PL.features(recs)
    t0 = time.perf_counter()
    params, mean, std, losses = PL.train(X, y, steps=3000, lr=3e-3)
    t_train = time.perf_counter() - t0
    if args.model_out:
        PL.save(args.model_out, params, mean, std)
    PL.register(params, mean, std)
    t0 = time.perf_counter()
    test = PL.collect(test_shapes, reps=1, seed=6)
    t_exhaustive = time.perf_counter() - t0
    ev = PL.evaluate(test)
    t0 = time.perf_counter()
    for (M, K, N) in test_shapes[:200]:
        PL.choice(M, N, K, "mlp")
    t_mlp_plan = (time.perf_counter() - t0) / 200
    fmm.fmm_set_cost_model(None)
    s = PL.summary(ev)
    emit(args, {"workload": "planner", "train_records": len(recs), "train_shapes": len(train_shapes),
                "test_shapes": len(test_shapes), "final_train_loss": losses[-1][1],
                "collect_s": round(t_collect, 1), "train_s": round(t_train, 2),
                "exhaustive_plan_ms_per_shape": round(t_exhaustive / len(test_shapes) * 1e3, 2),
                "mlp_plan_ms_per_shape": round(t_mlp_plan * 1e3, 3), **{k: (round(v, 4) if isinstance(v, float) else v)
                                                                           for k, v in s.items()}})


def wl_profile_case(args):
    """One plan (n, depth, leaf tile, fuse_last from the flags; U[-1,1] operands
    of the headline seed) called `--calls` times, untimed, its device status
    checked: the launches an ncu capture selects with -k / -s / -c."""
    import torch
    from paper_1205_2927_gb300 import fmm, inputs
    n = args.n
    A_h, B_h = inputs.operands(n, n, n, inputs.seed_for(2, 0))
    dA, dB = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
    dC = torch.empty((n, n), device="cuda")
    kw = {"fuse_last": args.fuse_last}
    if args.depth >= 0:
        kw["depth"] = args.depth
    if args.leaf_tile:
        kw["leaf_tile"] = args.leaf_tile
    p = fmm.Plan(n, n, n, precision=args.precision, **kw)
    for _ in range(args.calls):
        p(dA, dB, dC)
    torch.cuda.synchronize()
    status = p.device_status()
    info = p.info
    p.close()
    if status != 0:
        raise SystemExit(f"device status {status:#x}")
    emit(args, {"workload": "profile_case", "n": n, "depth": info["depth"], "leaf_tile": info["leaf_tile"],
                "fuse_last": info["fuse_last"], "calls": args.calls})


WORKLOADS = {"single1024": wl_single1024, "profile_case": wl_profile_case, "sweep": wl_sweep, "fine_sweep": wl_fine_sweep, "large": wl_large, "rmul": wl_rmul, "split": wl_split,
             "batched": wl_batched,
             "planner": wl_planner, "residual": wl_residual}

def cublas_tf32_tflops(torch, n=8192, reps=10):
    """TF32 tensor-core rate of the vendor library on this GPU (a live
    microbenchmark: torch.matmul with TF32 allowed, n^3, median of reps)."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        a = torch.rand(n, n, device="cuda")
        b = torch.rand(n, n, device="cuda")
        c = torch.empty(n, n, device="cuda")
        for _ in range(3):
            torch.matmul(a, b, out=c)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            torch.matmul(a, b, out=c)
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        del a, b, c
        return 2.0 * n ** 3 / (statistics.median(ts) * 1e-3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def tensor_peak(fmm, gpu_index, kind="tf32", runs=3, batches=30000):
    """The project's tensor-pipe probe (fmm_tensor_peak), best of `runs`, with
    the SM clock sampled while the probe ran."""
    clk = Clocks(gpu_index)
    clk.start()
    t0 = time.perf_counter()
    best = max(fmm.fmm_tensor_peak(kind, batches, seed=r + 1)[0] for r in range(runs))
    clk.window = (t0, time.perf_counter())
    c = clk.stop() or {}
    return {"tflops": best, "kind": f"kind::{kind}" if kind == "tf32" else "kind::f16 (bf16)",
            "sm_mhz": c.get("sm_mhz"), "reasons": c.get("reasons")}


def max_over_ranks(torch, dist, world, value, device):
    """The largest of every rank's `value` (the step time of the slowest
    replica); the value itself with one rank."""
    if world <= 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def timed(torch, dist, world, fn, steps, warmup, clocks=None):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    s.record()
    for _ in range(steps):
        fn()
    e.record()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.window = (t0, time.perf_counter())
    if world > 1:
        dist.barrier()
    return max_over_ranks(torch, dist, world, s.elapsed_time(e) / steps, "cuda")


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload != "square":
        WORKLOADS[args.workload](args)
        return
    import numpy as np
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1205_2927_gb300 import build as B_
    from paper_1205_2927_gb300 import fmm, inputs

    n = args.n
    flops = 2.0 * n ** 3
    A_h, B_h = inputs.operands(n, n, n, inputs.seed_for(2, rank))
    dA = torch.from_numpy(A_h).cuda()
    dB = torch.from_numpy(B_h).cuda()
    dC = torch.empty((n, n), device="cuda")

    wplan = fmm.Plan(n, n, n, depth=args.depth, precision=args.precision, leaf_tile=args.leaf_tile)
    depth = wplan.info["depth"]
    bn = wplan.info["leaf_tile"]
    fused_last = wplan.info["fuse_last"]
    step = lambda: wplan(dA, dB, dC)

    clocks = Clocks(local)
    clocks.start()
    wplan.profile(True)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    wplan.profile(True)  # reset: count only the timed steps
    ms = timed(torch, dist, world, step, args.steps, 0, clocks)
    clk = clocks.stop()
    phase_bytes = wplan.phase_bytes()
    prof = wplan.profile_read()
    wplan.profile(False)
    assert wplan.device_status() == 0, "device status word set"

    # accuracy of the benchmarked result on sampled rows against a float64 product
    err = sampled_error(np, torch, dC, A_h, B_h)

    # the residual check on the benchmarked product: r = C x - A (B x) for a
    # +-1 probe, one pass over A, B and C (HBM-bound), fp32 and fp64 accumulation
    residual = None
    if not args.no_residual:
        x = torch.from_numpy(inputs.rademacher(n, inputs.seed_for(2, 95))).cuda()
        rbytes = 4.0 * 3 * n * n
        peak_gbs = peaks()[0]["hbm_gbs"]
        scale = float(np.abs(A_h).max()) * float(np.abs(B_h).max()) * n * n
        residual = {"bytes": rbytes, "peak_gbs": peak_gbs}
        for name, fp64 in (("fp32", False), ("fp64", True)):
            rms = timed(torch, dist, world, lambda: fmm.fmm_residual(dA, dB, dC, x, fp64=fp64), min(args.steps, 20), 3)
            r = fmm.fmm_residual(dA, dB, dC, x, fp64=fp64)
            residual[name] = {"ms": round(rms, 4), "achieved_gbs": round(rbytes / rms / 1e6, 1),
                              "frac": round(rbytes / rms / 1e6 / peak_gbs, 3),
                              "max_abs_r_over_maxA_maxB_n2": float(r.abs().max().item()) / scale}

    classical = None
    if not args.no_classical:
        cplan = fmm.Plan(n, n, n, depth=0, precision=args.precision, leaf_tile=args.leaf_tile)
        cms = timed(torch, dist, world, lambda: cplan(dA, dB, dC), args.steps, args.warmup)
        classical = {"gflops": round(flops * world / cms / 1e6, 1), "ms_per_step": round(cms, 3)}
        cplan.close()

    # the split-precision forms beside plain FP32: same operands, same depth,
    # each with its own classical (depth-0) GEMM and its error on the same
    # float64 rows; outside the timed region of `value`
    split = None
    if args.precision == "fp32" and not args.no_split:
        split = {"depth": depth, "bound": 2e-6}
        # the 16-bit leaves' roofline: kind::f16 work of the leaf launch against the
        # project's tcgen05 probe in the same instruction shape (bf16 operands)
        probe16 = tensor_peak(fmm, local, "bf16")
        split["peak_bf16_probe_tflops"] = round(probe16["tflops"], 1)
        leaf_side = ((n + (4 << depth) - 1) // (4 << depth) * (4 << depth)) >> depth if depth > 0 else n
        leaf_work16 = 3 * 2.0 * 7 ** depth * float(leaf_side) ** 3
        dC2 = torch.empty((n, n), device="cuda")
        for prec in ("fp16x3", "bf16x3"):
            sp = fmm.Plan(n, n, n, depth=depth, precision=prec, leaf_tile=args.leaf_tile)
            sms = timed(torch, dist, world, lambda: sp(dA, dB, dC2), min(args.steps, 10), 3)
            assert sp.device_status() == 0, "device status word set"
            # phase split from a few more calls with the plan's CUDA-event marks
            sp.profile(True)
            for _ in range(3):
                sp(dA, dB, dC2)
            torch.cuda.synchronize()
            pr = sp.profile_read()
            sp.close()
            calls = max(pr["calls"], 1)
            leaf16_ms = pr["leaf_ms"] / calls
            entry = {"gflops": round(flops * world / sms / 1e6, 1), "ms_per_step": round(sms, 3),
                     "error": sampled_error(np, torch, dC2, A_h, B_h),
                     "phases": {"pre_add_ms": round(pr["pre_ms"] / calls, 3), "leaf_ms": round(leaf16_ms, 3),
                                "post_add_ms": round(pr["post_ms"] / calls, 3)},
                     "leaf_tflops": round(leaf_work16 / (leaf16_ms * 1e-3) / 1e12, 1),
                     "leaf_frac_of_bf16_probe": round(leaf_work16 / (leaf16_ms * 1e-3) / 1e12 / probe16["tflops"], 3)}
            if classical:
                sc = fmm.Plan(n, n, n, depth=0, precision=prec, leaf_tile=args.leaf_tile)
                scms = timed(torch, dist, world, lambda: sc(dA, dB, dC2), min(args.steps, 10), 3)
                sc.close()
                entry["classical_gflops"] = round(flops * world / scms / 1e6, 1)
                entry["speedup_vs_classical"] = round(scms / sms, 3)
            split[prec] = entry
        del dC2

    e2e = None
    if not args.no_e2e:
        # host-resident operands through the C ABI (host_operands = 1): the call
        # streams the quadrants of A and B in and C out, overlapped with compute
        pA = torch.from_numpy(A_h).pin_memory()
        pB = torch.from_numpy(B_h).pin_memory()
        pC = torch.empty((n, n), dtype=torch.float32).pin_memory()
        del dC
        wplan.close()
        hplan = fmm.Plan(n, n, n, depth=depth, precision=args.precision, leaf_tile=bn, host_operands=1,
                         host_copy=args.host_copy)
        # at least 16 warm-up calls (about 450 ms, longer than the period of the
        # copy-engine stalls some hosts show): the library's default host copies
        # settle on their path (copy engines, or SM copies once a call's
        # transfers stalled) before the timed calls, which run ahead of the GPU
        e2e_warmup = max(args.warmup, 16)
        ems = timed(torch, dist, world, lambda: hplan(pA, pB, pC), args.steps, e2e_warmup)
        e2e = {"value": round(flops * world / ems / 1e6, 1), "unit": "GFLOPS",
               "h2d_bytes_per_step": int(pA.numel() * 4 + pB.numel() * 4),
               "d2h_bytes_per_step": int(pC.numel() * 4), "ms_per_step": round(ems, 3),
               "path": f"fmm_gemm with pinned host operands (host_operands=1, host_copy={args.host_copy})",
               "warmup": e2e_warmup, "host_copy_after": hplan.host_copy()}
        hplan.close()

    # roofline of the dominant kernel (the leaf launch): tensor-pipe TF32 work per launch / time per launch
    pk, pk_kind = peaks()
    leaf_dim = (n + (4 << depth) - 1) // (4 << depth) * (4 << depth) >> depth if depth > 0 else n
    leaf_count = 7 ** depth
    tc_products = 3 if args.precision == "fp32" else 1
    leaf_flops = tc_products * 2.0 * leaf_count * float(leaf_dim) ** 3
    leaf_ms = prof["leaf_ms"] / max(prof["calls"], 1)
    achieved = leaf_flops / (leaf_ms * 1e-3) / 1e12
    # peak: the project's own tensor-pipe probe (fmm_tensor_peak: back-to-back
    # tcgen05.mma of the leaf kernel's shape on shared-memory tiles), best of 3
    # runs with the SM clock sampled while it ran; the leaf launch is timed alone
    # (events around that launch only), so the burst figure is its ceiling
    probe = tensor_peak(fmm, local, "tf32" if args.precision in ("fp32", "tf32") else "bf16")
    peak_tc = probe["tflops"]
    peak_nominal = pk["bf16_tflops"] * (TF32_OVER_BF16 if args.precision in ("fp32", "tf32") else 1.0)
    traffic = ncu_traffic(os.path.join(ROOT, "paper_1205_2927_gb300", "csrc", "leaf_gemm.cu"),
                          f"n{n}_d{depth}_bn{bn}_{args.precision}")
    kname = "leaf_gemm_pair_kernel (cta_group::2, 256x256 tiles)" if bn == 512 else f"leaf_gemm_kernel (128x{bn} tiles)"
    if fused_last:
        kname += ", last Winograd level fused (node outputs, not products)"
    roofline = {"bound": "tensor", "kernel": kname + (" tcgen05 kind::tf32, pre-split raw/lo planes" if args.precision == "fp32"
                                                      else f" {args.precision}"),
                "achieved": round(achieved, 1), "peak": round(peak_tc, 1), "unit": "TFLOP/s",
                "frac": round(achieved / peak_tc, 3), "traffic": traffic,
                "peak_source": "measured: tcgen05 issue-rate probe (fmm_tensor_peak), "
                               f"{probe['kind']} M=256 N=256 CTA pairs, best of 3 runs",
                "peak_probe_sm_mhz": probe.get("sm_mhz"),
                "peak_nominal_ratio": round(peak_nominal, 1),
                "peak_nominal_ratio_source": f"{pk_kind} bf16 burst {pk['bf16_tflops']} x nominal tf32/bf16 1.1/2.25",
                "work": f"{tc_products} TF32 products x 2*{leaf_count}*{leaf_dim}^3 flops per launch",
                "leaf_ms_per_launch": round(leaf_ms, 3)}
    if args.precision in ("fp32", "tf32"):
        tf32 = cublas_tf32_tflops(torch)
        roofline["cublas_tf32_tflops"] = round(tf32, 1)
        roofline["frac_of_cublas_tf32"] = round(achieved / tf32, 3)
    phases = {"pre_add_ms": round(prof["pre_ms"] / max(prof["calls"], 1), 3), "leaf_ms": round(leaf_ms, 3),
              "post_add_ms": round(prof["post_ms"] / max(prof["calls"], 1), 3)}
    # the addition passes are HBM-bound: algorithmic bytes per call / phase time
    # against the measured copy bandwidth
    additions = {}
    for key, bkey, tkey in (("pre", "pre_bytes", "pre_add_ms"), ("post", "post_bytes", "post_add_ms")):
        b, t = phase_bytes[bkey], phases[tkey]
        if b > 0 and t > 0:
            gbs = b / (t * 1e-3) / 1e9
            additions[key] = {"bytes": int(b), "ms": t, "achieved_gbs": round(gbs, 1), "peak_gbs": pk["hbm_gbs"],
                              "frac": round(gbs / pk["hbm_gbs"], 3)}
    additions["peak_source"] = f"{pk_kind} HBM copy bandwidth"
    # end-to-end bound of the schedule: leaf work at the measured TF32 rate plus
    # the addition bytes at the measured HBM bandwidth, against the measured step
    if roofline.get("cublas_tf32_tflops"):
        add_s = (phase_bytes["pre_bytes"] + phase_bytes["post_bytes"]) / (pk["hbm_gbs"] * 1e9)
        t_star = (leaf_flops / (peak_tc * 1e12) + add_s) * 1e3
        t_star_cublas = (leaf_flops / (roofline["cublas_tf32_tflops"] * 1e12) + add_s) * 1e3
        additions["bound_ms"] = {"t_star": round(t_star, 3), "measured": round(ms, 3),
                                 "t_star_over_measured": round(t_star / ms, 3),
                                 "t_star_cublas_tf32": round(t_star_cublas, 3),
                                 "model": "leaf flops / probe TF32 rate + addition bytes / HBM copy bandwidth"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_headline(A_h, B_h, depth)

    value = flops * world / ms / 1e6
    line = {
        "metric": "effective GFLOPS (2MNK/s) Winograd vs classical GEMM on 1 GB300 at stated error",
        "value": round(value, 1), "unit": "GFLOPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"winograd_{args.precision}_square_n{n}", "n": n, "depth": depth, "leaf_tile": bn,
                   "fuse_last": int(fused_last),
                   "precision": "fp32 via 3xTF32 tensor-core leaves" if args.precision == "fp32" else args.precision,
                   "dist": "A,B ~ U[-1,1] seeded", "l2": "inputs larger than L2 (no flush needed)",
                   "parallelism": f"replicas{world}"},
        "error": {"metric": "max|C-C64|/(max|A| max|B| n) on 16 sampled rows", "value": err, "bound": 2e-6},
        "classical": classical,
        "speedup_vs_classical": round(value / classical["gflops"], 3) if classical else None,
        "split_precision": split,
        "residual": residual,
        "phases": phases,
        "additions": additions,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(prof["launches"]),
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    wplan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
