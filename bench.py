#!/usr/bin/env python
"""Benchmark of randomized-pivoting skeletonization (Algorithm 2) on GB300.

Headline workload (the largest single-GPU configuration; one "step" = the whole hot path on
one synthetic matrix resident in HBM):
  A: 65536 x 32768 FP32 (8.6 GB), A = U diag(sigma) V^T + 1e-7 floor, sigma_j = exp(-j/200),
     Haar U, V; k = 1024, oversampling p = 76 (l = 1100), Gaussian embedding.
  step = tensor-core sketch X = Gamma A (--prec, FP8 by default: e4m3 operands with one power-
         of-two scale per column of A, FP32 accumulation)  ->  LUPP on X (J_s, R^LU)
         [time-to-skeleton, the metric]  ->  column ID Z = C^+ A (Householder QR of C = A(:, J_s),
         W = Q_C^T A, FP64 solve)  [time to ID]  ->  Theorem 1's eta from R^LU.
Reported beside it: time-to-skeleton in every sketch precision (TF32, BF16, FP8) and in the
plain FP64 GPU form on the same A, each with its relative ID error ||A - C Z||_F / ||A||_F formed
directly on the device (the FP64 skeleton's error is the reference: the equal-error gate is
1.05x), the sketch's tensor-core roofline, per-kernel times from a serialised pass, the oracle
timed on the host cores on a bounded sample, an end-to-end number through host buffers, and
the 8192 x 8192 (k = 256) step with the row skeletons and the CUR as extra keys.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--prec bf16]
                  [--workload dense_65536x32768|dense_8192x8192] [--only ...]

Multi-GPU: N ranks run N independent replicas (one matrix each, weak scaling) with no
collective on the data path (the row-partitioned sketch with its one all-reduce is the
library's `dist` module, exercised by the multi-process tests).  --impl reference times the
FP64 CPU oracle (the only reference this paper has) on rank 0.
"""

import argparse
import json
import os
import resource
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-skeleton (ms) and A-streaming GB/s at rank k, mixed vs FP64 GPU, equal ID error"

# workloads: (m, n, k, p, floor, description)
WORKLOADS = {
    "dense_65536x32768": dict(m=65536, n=32768, k=1024, p=76,
               text="dense 65536x32768 fp32 (8.6 GB), sigma_j=exp(-j/200) (j<=3300) + 1e-7 floor, Haar U/V"),
    "dense_8192x8192": dict(m=8192, n=8192, k=256, p=16,
               text="dense 8192x8192 fp32, sigma_j=1/j + 1e-6 floor, Haar U/V"),
}
ORACLE_SAMPLE_COLS = 1024       # bounded oracle sample: this many columns of A


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dense_65536x32768", choices=sorted(WORKLOADS))
    ap.add_argument("--k", type=int, default=None, help="rank (default: the workload's)")
    ap.add_argument("--p", type=int, default=None, help="oversampling (default: the workload's)")
    ap.add_argument("--prec", default="fp8", choices=["tf32", "bf16", "fp8", "f32"])
    ap.add_argument("--blocks", type=int, default=4096, help="blocks of the batched run (--only batch)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 plain-GPU comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--no-extra", action="store_true", help="skip the 8192^2 extra keys")
    ap.add_argument("--xonly", action="store_true",
                    help="with --only lupp: pivot on a seeded Gaussian l x n sketch instead of building A (the "
                         "same shapes with a few hundred MB on the device, for profilers)")
    ap.add_argument("--cols", type=int, default=None,
                    help="with --only: this many columns of the workload's A instead of all of them (a smaller "
                         "case of the same kernels for profilers)")
    ap.add_argument("--only", default=None, choices=["sketch", "lupp", "rows", "pivots", "id", "cur", "id_cur", "eta", "batch", "next",
                                                     "srtt", "power", "cols"],
                    help="run only this call (warm-up + steps, no extras): a small command for profilers; "
                         "'batch' runs the batched configuration (4096 Gaussian-kernel blocks, k_max 128, "
                         "tol 1e-6) instead of the dense workload; 'next' times the rows beyond the hot "
                         "path (SRTT sketch, power sketch, column sketch, streaming selection, ID and CUR "
                         "from the sketch) on the same workload, one JSON line")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    args.k = w["k"] if args.k is None else args.k
    args.p = w["p"] if args.p is None else args.p
    return args


def workload_config(workload, k, p, prec):
    w = WORKLOADS[workload]
    steps = ("LUPP on X, column ID" if workload == "dense_65536x32768"
             else "LUPP on X, row LUPP on C, column ID + stable CUR")
    return {"workload": f"{w['text']}; rank k={k}, oversampling p={p} (l={k + p}); Gaussian sketch ({prec}), {steps}",
            "m": w["m"], "n": w["n"], "k": k, "l": k + p, "sketch_prec": prec,
            "l2": f"inputs larger than L2 (A is {4 * w['m'] * w['n'] / 1e6:.0f} MB; L2 129 MB)"}


def make_A(workload, device, seed, cols=None):
    import numpy as np
    import torch
    import workloads
    w = WORKLOADS[workload]
    n = min(cols, w["n"]) if cols else w["n"]
    if workload == "dense_65536x32768":
        return workloads.torch_dense_exp200(device, w["m"], n, seed=seed)
    sig = workloads.sigma_harmonic(min(w["m"], n))
    return workloads.torch_dense_spectrum(w["m"], n, sig, 1e-6 / np.sqrt(w["m"]), seed, device, torch.float32)


def seeds(workload, rank=0):
    import workloads
    return workloads.seed_for(workload) + rank, workloads.seed_for(workload, "gamma")


# ------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 50 ms while running (entering waits,
    up to 3 s, for the first sample so that the sampler is live when the timed region starts)."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# kernels timed with CUDA events in the serialised pass
TIMED_KERNELS = ("sketch_tc", "sketch_fp8", "fp8_quantize", "gemm_tc", "lupp_panel", "lupp_trail", "qr_panel", "qr_wy", "gemm_refine",
                 "trsm", "gemm_qr", "gemm_cur", "gemm_eta_h", "gemm_eta_sq", "gemm_simt", "transpose", "lupp_mult",
                 "trsm_ff")
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of
# the current kernel at this workload; None where no capture of the current code exists.
# 65536 x 32768 is too large to capture whole: the TF32 sketch was captured on the 65536 x 8192
# slice (2.164 GB read, 3.5 MB written) and scaled by the columns to the full 32768-column
# launch (the kernel reads each column of A once); the FP8 GEMM on the same slice (612.5 MB
# read: the 536.9 MB of A8 and Gamma's 75.5 MB of e4m3 normals; 0.15 MB written), its A8 part
# scaled by the columns.
TRAFFIC_PER_LAUNCH = {"dense_65536x32768": {"sketch_tc_tf32": 4 * (2.164166912e9 + 3.450624e6),
                             "sketch_fp8_fp8": 4 * (612513024 - 75497472 + 145408) + 75497472},
                      "dense_8192x8192": {"sketch_tc": 271.9e6, "gemm_tc": 332.4e6, "lupp_panel": 3.09e6,
                                          "qr_panel": 2.15e6}}
FP64_NOMINAL_TFLOPS = 1.25
TENSOR_RATIO = {"bf16": 1.0, "tf32": 1.1 / 2.25, "fp8": 2.0}     # nominal dense ratios to BF16


def load_peaks():
    """(hbm GB/s, bf16 TFLOP/s burst, source); the full record via load_peaks_full()."""
    d = load_peaks_full()
    return d["hbm_gbs"], d["bf16_tflops"], d["source"]


def load_peaks_full():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def tensor_peak(prec, peaks, sustained):
    base = peaks["bf16_tflops_sustained"] if sustained else peaks["bf16_tflops"]
    return base * TENSOR_RATIO[prec]


# ------------------------------------------------------------------------------------------
def cpu_sample_baseline(A_host_cols, m, n, k, p, seed_G):
    """The FP64 oracle's time-to-skeleton (sketch + LUPP on X) on a bounded sample: the first
    n' columns of A.  Gamma's generation does not depend on n and is timed on its own; the
    oracle's product and its LUPP (which updates every column at every step) scale linearly
    with n, so the full-size estimate is t_Gamma + (t_sketch - t_Gamma + t_lupp) n / n'.
    Threads: CPU time over wall time of the timed calls (numpy's BLAS threads the product)."""
    from oracle import embedding, pivoting, sketch
    ncols = A_host_cols.shape[1]
    l = k + p
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    w0 = time.perf_counter()
    t = time.perf_counter()
    embedding.gaussian_normals(l, m, seed_G)
    t_g = time.perf_counter() - t
    t = time.perf_counter()
    X = sketch.gaussian_sketch(A_host_cols, l, seed_G)
    t_sk = time.perf_counter() - t
    t = time.perf_counter()
    pivoting.lupp_columns(X, min(k, ncols))
    t_lu = time.perf_counter() - t
    wall = time.perf_counter() - w0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    est = t_g + (max(t_sk - t_g, 0.0) + t_lu) * n / ncols
    return {"value": est * 1e3, "unit": "ms", "cores": round(cpu / wall, 1), "kind": "oracle",
            "sample": (f"FP64 oracle sketch + LUPP on the first {ncols} of {n} columns of the same A "
                       f"(Gamma generation {t_g:.2f} s, sketch {t_sk:.2f} s, LUPP {t_lu:.2f} s measured; value = "
                       f"Gamma + (sketch - Gamma + LUPP) x {n}/{ncols}); cores = CPU time / wall time"),
            "host_cpus": os.cpu_count(), "measured_s": wall}


def run_reference(args, rank):
    if rank != 0:
        return
    import numpy as np
    import torch
    w = WORKLOADS[args.workload]
    seed_A, seed_G = seeds(args.workload)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A = make_A(args.workload, dev, seed_A)
    ncols = min(ORACLE_SAMPLE_COLS, w["n"])
    A_np = np.asfortranarray(A[:, :ncols].double().cpu().numpy())
    del A
    if dev == "cuda":
        torch.cuda.empty_cache()
    vals, last = [], None
    for i in range(args.warmup + args.steps):
        last = cpu_sample_baseline(A_np, w["m"], w["n"], args.k, args.p, seed_G)
        if i >= args.warmup:
            vals.append(last["value"])
    v = statistics.mean(vals)
    cb = dict(last, value=v)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, args.k, args.p, "f64 oracle"),
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------------------------------
def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def wall_steps(fn, steps):
    """Host wall-clock ms per call of fn (which ends by reading its result on the host), and
    each call's time: the end-to-end clock a user sees, launch and synchronization included."""
    import torch
    torch.cuda.synchronize()
    per = []
    t_all = time.perf_counter()
    for _ in range(steps):
        t0 = time.perf_counter()
        fn()
        per.append(round((time.perf_counter() - t0) * 1e3, 2))
    return (time.perf_counter() - t_all) * 1e3 / steps, per


def direct_rel_error(skel, A, Js, st):
    """||A - C Z||_F / ||A||_F with Z = C^+ A from skel_id, the residual formed on the device."""
    Z, sq, _ = skel.column_id(A, Js, status=st)
    e, _ = skel.error(A, Js, Z=Z, status=st)
    e, sq = e.cpu().numpy(), sq.cpu().numpy()
    gram = float(max(sq[0] - sq[1], 0.0) / sq[0]) ** 0.5
    del Z
    return float(e[1] / e[0]), gram


def time_skeleton(skel, A, l, k, prec, seed_G, st, reps=3):
    """Sketch + LUPP on X, timed alone with CUDA events (mean over reps after one warm-up)."""
    import torch
    X = torch.empty(l, A.shape[1], dtype=torch.float64 if prec == "f64" else torch.float32, device=A.device)

    def once():
        skel.sketch(A, l, prec=prec, seed=seed_G, X=X, status=st)
        return skel.pivot_lupp(X, k, factors=False, status=st)[0]

    Js = once()
    torch.cuda.synchronize()
    ev = _events(3 * reps)
    for r in range(reps):
        ev[3 * r].record()
        skel.sketch(A, l, prec=prec, seed=seed_G, X=X, status=st)
        ev[3 * r + 1].record()
        Js = skel.pivot_lupp(X, k, factors=False, status=st)[0]
        ev[3 * r + 2].record()
    torch.cuda.synchronize()
    skel.check_status(st, f"skeleton {prec}")
    sk = statistics.mean(ev[3 * r].elapsed_time(ev[3 * r + 1]) for r in range(reps))
    lu = statistics.mean(ev[3 * r + 1].elapsed_time(ev[3 * r + 2]) for r in range(reps))
    del X
    return Js, {"time_to_skeleton_ms": sk + lu, "sketch_ms": sk, "lupp_ms": lu, "reps": reps}


def measure_floors(skel, dev, col_words):
    """Measured floors for the latency- and ALU-bound kernels: FMA rates of the FP64 and FP32
    pipes, one grid-wide barrier round over every SM, one cluster candidate exchange (16 CTAs
    where the device offers them, else 8) with and without a pivot column of `col_words`."""
    import torch
    out = {"fp64_tflops": skel.debug_fma_rate(True, iters=1 << 12),
           "fp32_tflops": skel.debug_fma_rate(False, iters=1 << 14),
           "grid_barrier_ns": skel.debug_exchange_latency(0, torch.cuda.get_device_properties(dev).multi_processor_count,
                                                          steps=2000)}
    for cl in (16, 8):
        try:
            out["cluster_exchange_ns"] = skel.debug_exchange_latency(1, cl, steps=4000)
            out["cluster_exchange_col_ns"] = skel.debug_exchange_latency(1, cl, steps=4000, col_words=col_words)
            out["cluster_ctas"] = cl
            out["col_words"] = col_words
            break
        except skel.SkelError:
            continue
    return out


def latency_roofline(kernels, name, steps, floors):
    """A latency-bound chain of `steps` dependent exchanges: floor = steps x one exchange round
    (with the pivot column); frac = floor / measured time per step of the whole run."""
    kd = kernels.get(name)
    if not kd or "cluster_exchange_col_ns" not in floors:
        return None
    floor_ms = steps * floors["cluster_exchange_col_ns"] * 1e-6
    kd.update({"bound": "latency", "floor_ms": floor_ms, "frac": floor_ms / kd["ms_per_step"],
               "us_per_step": 1e3 * kd["ms_per_step"] / steps,
               "floor_what": f"{steps} steps x one {floors['cluster_ctas']}-CTA cluster exchange round "
                             f"({floors['cluster_exchange_col_ns']:.0f} ns, measured)"})
    return kd


def kernel_models(workload, m, n, k, l, prec, peaks, sustained, floors=None):
    """Algorithmic work of each timed kernel over one step: (bound, work, peak, unit)."""
    hbm = peaks["hbm_gbs"]
    a_bytes = 4.0 * m * n
    fp32_alu = (floors or {}).get("fp32_tflops") or 152 * 128 * 2 * 2.07e9 / 1e12     # TFLOP/s, FFMA
    fp64 = (floors or {}).get("fp64_tflops") or FP64_NOMINAL_TFLOPS
    b_pan = 24 if workload == "dense_65536x32768" else 64
    # LUPP trailing updates: every panel reads and writes the rows below it once (4 B each way)
    trail_bytes = sum(8.0 * max(k - t0 - b_pan, 0) * n for t0 in range(0, k, b_pan))
    mod = {
        "sketch_fp8": ("tensor", 2.0 * l * m * n / 1e12, tensor_peak("fp8", peaks, sustained), "TFLOP/s"),
        "fp8_quantize": ("hbm", 5.0 * m * n / 1e9, hbm, "GB/s"),   # A read (4 B), A8 written (1 B)
        "gemm_tc": ("tensor", 3 * 2.0 * k * m * n / 1e12, tensor_peak("tf32", peaks, sustained), "TFLOP/s"),
        "lupp_trail": ("hbm", trail_bytes / 1e9, hbm, "GB/s"),
        # Z = R^{-1} W in float-float on the FP32 pipes: k^2 n / 2 multiply-add terms, each at
        # least 12 FP32 instructions (exact product split, two-sum, carries)
        "trsm_ff": ("alu", (0.5 * k * k * n) / 1e12, fp32_alu / 2.0 / 12.0, "T terms/s"),
    }
    if prec in ("tf32", "bf16"):
        mod["sketch_tc"] = ("tensor", 2.0 * l * m * n / 1e12, tensor_peak(prec, peaks, sustained), "TFLOP/s")
    if workload == "dense_8192x8192":
        mod["trsm"] = ("alu", (4.0 * k ** 3) / 1e12, fp64, "TFLOP/s")      # U's and eta's k x k solves
    return mod


def kernel_table(skel, nsteps, total_ms, models):
    out = {}
    for nm in TIMED_KERNELS:
        tot, cnt = skel.kernel_time(nm)
        if cnt == 0:
            continue
        ent = {"ms_per_step": tot / nsteps, "launches_per_step": cnt / nsteps, "avg_us": 1e3 * tot / cnt,
               "share_of_step": tot / total_ms}
        if nm in models:
            b, w, pk, u = models[nm]
            a = w / (tot / nsteps * 1e-3)
            ent.update({"bound": b, "achieved": a, "peak": pk, "unit": u, "frac": a / pk})
        out[nm] = ent
    return out


def run_ours(args, rank, world):
    import numpy as np
    import torch
    import paper_2104_05877_gb300 as skel

    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    if not os.path.exists(skel.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    if args.only == "batch":
        import workloads
        run_batch(args, rank, dev, skel, workloads)
        return
    k, p = args.k, args.p
    l = k + p
    seed_A, seed_G = seeds(args.workload, rank)
    if args.cols and not args.only:
        raise SystemExit("--cols is a profiling aid for --only runs")
    if args.xonly:
        if args.only != "lupp":
            raise SystemExit("--xonly is a profiling aid for --only lupp")
        w = WORKLOADS[args.workload]
        g = torch.Generator(device=dev)
        g.manual_seed(seed_G)
        X = torch.randn(l, args.cols or w["n"], generator=g, device=dev)
        st = skel.new_status(dev)
        run_timed(args, rank, lambda: skel.pivot_lupp(X, k, status=st), st, workload_config(args.workload, k, p, "x only"))
        return
    A = make_A(args.workload, dev, seed_A, cols=args.cols)
    torch.cuda.synchronize()
    st = skel.new_status(dev)
    if args.only == "next":
        run_next(args, rank, A, skel, st, seed_G)
        return
    if args.only:
        run_only(args, rank, A, skel, st, seed_G)
        return
    if args.workload == "dense_8192x8192":
        res = run_dense_8192_step(args, rank, world, dev, A, skel, st, seed_G, headline=True)
        if rank == 0:
            print(json.dumps(res), flush=True)
        return
    run_dense_large(args, rank, world, dev, A, skel, st, seed_G, local)


def run_dense_large(args, rank, world, dev, A, skel, st, seed_G, local):
    import numpy as np
    import torch
    k, p = args.k, args.p
    l = k + p
    m, n = A.shape
    prec = args.prec
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    X = torch.empty(l, n, device=dev)
    names = ["sketch", "lupp", "id", "eta_after_id"]

    def step(evs, serial=False):
        evs[0].record()
        skel.sketch(A, l, prec=prec, seed=seed_G, X=X, status=st)
        evs[1].record()
        Js, _, Rf, _ = skel.pivot_lupp(X, k, status=st)
        evs[2].record()
        # eta needs only the pivot factor: it runs on a second stream while the column ID runs
        # on this one (on this stream too in the serialised per-kernel pass)
        if serial:
            e, _ = skel.error(A, Js, Rf=Rf, status=st)
        else:
            side.wait_stream(main)
            with torch.cuda.stream(side):
                e, _ = skel.error(A, Js, Rf=Rf, status=st)
        Z, sq, _ = skel.column_id(A, Js, status=st)
        evs[3].record()
        if not serial:
            main.wait_stream(side)
        evs[4].record()
        return Js, Z, sq, e

    mk = lambda: _events(len(names) + 1)
    for _ in range(args.warmup):
        step(mk())
    torch.cuda.synchronize()
    skel.check_status(st, "warmup")
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = skel.launch_count()
    all_evs = [mk() for _ in range(args.steps)]
    t_begin, t_end = _events(2)
    with ClockSampler(local) as clk:
        t_begin.record()
        for i in range(args.steps):
            out = step(all_evs[i])
        t_end.record()
        torch.cuda.synchronize()
    launches = skel.launch_count() - launches0
    if world > 1:
        torch.distributed.barrier()
    skel.check_status(st, "timed steps")
    total_ms = t_begin.elapsed_time(t_end)
    per = {nm: statistics.mean(ev[i].elapsed_time(ev[i + 1]) for ev in all_evs) for i, nm in enumerate(names)}
    tts = statistics.mean(ev[0].elapsed_time(ev[2]) for ev in all_evs)
    tts_median = statistics.median([ev[0].elapsed_time(ev[2]) for ev in all_evs])
    tid = statistics.mean(ev[0].elapsed_time(ev[3]) for ev in all_evs)
    if world > 1:
        t = torch.tensor([tts, total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        tts, total_ms = float(t[0]), float(t[1])
    Js, Z, sq, e = out
    del Z
    if rank != 0:
        return

    # serialised pass: the same steps on one stream, CUDA events around every hot launch
    peaks = load_peaks_full()
    floors = measure_floors(skel, dev, col_words=24)
    nser = max(2, min(args.steps, 5))
    skel.kernel_timing(True)
    s0, s1 = _events(2)
    s0.record()
    for _ in range(nser):
        step(mk(), serial=True)
    s1.record()
    torch.cuda.synchronize()
    ser_ms = s0.elapsed_time(s1)
    models = kernel_models("dense_65536x32768", m, n, k, l, prec, peaks, sustained=True, floors=floors)
    kernels = kernel_table(skel, nser, ser_ms, models)
    latency_roofline(kernels, "lupp_panel", k, floors)
    skel.kernel_timing(False)
    skel.check_status(st, "serialised pass")

    # the sketch kernel's roofline (the dominant kernel of time-to-skeleton)
    sk_name = "sketch_fp8" if prec == "fp8" else "sketch_tc"
    kd = kernels.get(sk_name, {})
    roofline = None
    if "bound" in kd:
        work = 2.0 * l * m * n
        achieved = work / (kd["avg_us"] * 1e-6) / 1e12
        pk = tensor_peak(prec, peaks, sustained=True)
        roofline = {"kernel": sk_name, "bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                    "frac": achieved / pk, "traffic": TRAFFIC_PER_LAUNCH["dense_65536x32768"].get(f"{sk_name}_{prec}"),
                    "peak_source": (f"{peaks['source']} MEASURED_PEAKS.json bf16_tflops_sustained x {TENSOR_RATIO[prec]:.3f} "
                                    f"(nominal {prec}:bf16 dense ratio)"),
                    "frac_of_burst_peak": achieved / tensor_peak(prec, peaks, sustained=False),
                    "work_per_launch": f"2 l m n = {work:.3e} flop", "avg_launch_us": kd["avg_us"],
                    "timing": "CUDA events on the launching stream around every launch, serialised pass of the same steps"}

    # every sketch precision: time-to-skeleton alone, and the ID error of its skeleton formed directly
    per_prec = {}
    for pr in ("tf32", "bf16", "fp8"):
        J, tm = time_skeleton(skel, A, l, k, pr, seed_G, st)
        rel, gram = direct_rel_error(skel, A, J, st)
        tm.update({"rel_id_error": rel, "rel_id_error_gram": gram, "a_streaming_gbs": 4.0 * m * n / (tm["sketch_ms"] * 1e-3) / 1e9,
                   "sketch_tflops": 2.0 * l * m * n / (tm["sketch_ms"] * 1e-3) / 1e12})
        per_prec[pr] = tm
    torch.cuda.synchronize()
    skel.check_status(st, "per precision")

    # the plain FP64 GPU form of the skeleton stage on the same A
    fp64 = None
    if not args.no_fp64:
        A64 = A.double().t().contiguous().t()
        J64, tm = time_skeleton(skel, A64, l, k, "f64", seed_G, st, reps=1)
        del A64
        torch.cuda.empty_cache()
        rel, gram = direct_rel_error(skel, A, J64, st)
        tm.update({"rel_id_error": rel, "rel_id_error_gram": gram,
                   "a_streaming_gbs": 8.0 * m * n / (tm["sketch_ms"] * 1e-3) / 1e9,
                   "id_error_note": "ID of the FP64 skeleton formed by skel_id on the FP32 A, residual on the device"})
        fp64 = tm
        for pr, ent in per_prec.items():
            ent["id_error_ratio_vs_fp64"] = ent["rel_id_error"] / rel
            ent["speedup_vs_fp64"] = tm["time_to_skeleton_ms"] / ent["time_to_skeleton_ms"]
    rel_id, rel_gram = direct_rel_error(skel, A, Js, st)

    # end to end through host buffers: the pinned host A streamed through the library in column
    # panels (copies overlapped with the sketch), LUPP, J_s back
    A_host = torch.empty(n, m, dtype=torch.float32, pin_memory=True)
    A_host.copy_(A.t())
    Js_h = torch.empty(k, dtype=torch.int32, pin_memory=True)

    def e2e_step():
        skel.sketch_host(A_host.t(), l, prec=prec, seed=seed_G, X=X, status=st)
        J, _, _, _ = skel.pivot_lupp(X, k, factors=False, status=st)
        Js_h.copy_(J, non_blocking=True)
        main.synchronize()          # the host reads the skeleton every step
        return int(Js_h[0])

    e2e_step()
    e_steps = max(3, min(args.steps, 10))
    e2e_ms, e2e_steps_ms = wall_steps(e2e_step, e_steps)
    skel.check_status(st, "e2e")
    e0, e1 = _events(2)
    # the panels' K-split sums in another order than the whole-matrix sketch, so near-tied pivots
    # may differ: report the shared fraction of the skeleton
    e2e_overlap = len(set(Js_h.tolist()) & set(Js.cpu().tolist())) / k
    # the link's floor: the same bytes as one host-to-device copy, nothing else
    A_dev = A.t()           # A's storage: the copy rewrites it with the same values
    A_dev.copy_(A_host, non_blocking=True)
    e0.record()
    for _ in range(3):
        A_dev.copy_(A_host, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    h2d_ms = e0.elapsed_time(e1) / 3

    # Algorithm 3 on the host A in one pass: both sketches from the same streamed panels, the
    # two LUPPs, both skeletons read on the host every step (the one-pass sketches have no FP8 form)
    Is_h = torch.empty(k, dtype=torch.int32, pin_memory=True)
    stream_prec = prec if prec in ("tf32", "bf16", "f32") else "tf32"

    def stream_step():
        Jx, Iy, _ = skel.skeletonize_streaming_host(A_host.t(), k, p, seed=seed_G, seed_omega=seed_G + 1,
                                                    prec=stream_prec, status=st)
        Js_h.copy_(Jx, non_blocking=True)
        Is_h.copy_(Iy, non_blocking=True)
        main.synchronize()
        return int(Js_h[0]) + int(Is_h[0])

    stream_step()
    stream_ms, stream_steps_ms = wall_steps(stream_step, 3)
    skel.check_status(st, "streaming selection")
    streaming = {"ms": stream_ms, "step_ms": stream_steps_ms, "median_ms": statistics.median(stream_steps_ms),
                 "clock": "host wall", "prec": stream_prec,
                 "h2d_bytes_per_step": int(4 * m * n), "passes_over_A": 1,
                 "what": "Algorithm 3 on the pinned host A: X = Gamma A and Y^T = Omega A^T from one streamed "
                         "pass (skel_sketch_host_two_sided), LUPP on X and on Y^T, J_s and I_s read back",
                 "link_floor_ms": h2d_ms}
    del A_host

    cpu = None
    if not args.no_cpu:
        ncols = min(ORACLE_SAMPLE_COLS, n)
        A_np = np.asfortranarray(A[:, :ncols].double().cpu().numpy())
        cpu = cpu_sample_baseline(A_np, m, n, k, p, seed_G)

    extra = extra3 = extra4 = None
    if not args.no_extra:
        del X
        torch.cuda.empty_cache()
        extra3 = run_c3(skel, dev)
        extra4 = batch_measure(skel, dev)
        A2 = make_A("dense_8192x8192", dev, seeds("dense_8192x8192", rank)[0])
        a2 = argparse.Namespace(**vars(args))
        a2.workload, a2.k, a2.p, a2.prec, a2.no_cpu = "dense_8192x8192", 256, 16, "tf32", True
        extra = run_dense_8192_step(a2, rank, world, dev, A2, skel, skel.new_status(dev), seeds("dense_8192x8192")[1],
                                    headline=False)
        del A2

    res = {
        "metric": METRIC, "value": tts, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": workload_config("dense_65536x32768", k, p, prec),
        "time_to_skeleton_median_ms": tts_median,     # rank 0's steps; `value` is the mean (max over ranks)
        "time_to_id_ms": tid, "calls_ms": per,
        "a_streaming_gbs": 4.0 * m * n / (per["sketch"] * 1e-3) / 1e9,
        "sketch_tflops": 2.0 * l * m * n / (per["sketch"] * 1e-3) / 1e12,
        "rel_id_error": rel_id, "rel_id_error_gram": rel_gram, "eta": float(e[3]),
        "id_error_ratio_vs_fp64": (rel_id / fp64["rel_id_error"]) if fp64 else None,
        "precisions": per_prec, "fp64_gpu": fp64,
        "roofline": roofline, "kernels": kernels, "serialised_ms_per_step": ser_ms / nser,
        "measured_floors": floors,
        "cpu_baseline": cpu,
        # the host link is shared with other tenants of the machine: single steps were seen at
        # 6x the rest, so the value is the median step, with the mean and every step beside it
        "e2e": {"value": statistics.median(e2e_steps_ms), "unit": "ms", "h2d_bytes_per_step": int(4 * m * n),
                "d2h_bytes_per_step": int(4 * k), "steps": e_steps, "statistic": "median of the steps",
                "mean_ms": e2e_ms, "skeleton_overlap_vs_device_sketch": e2e_overlap, "step_ms": e2e_steps_ms,
                "clock": "host wall", "h2d_copy_alone_ms": h2d_ms,
                "h2d_gbs": 4.0 * m * n / (h2d_ms * 1e-3) / 1e9,
                "what": "pinned host A streamed in column panels through skel_sketch_host (copies overlapped "
                        "with the sketch), LUPP, J_s copied back"},
        "streaming_selection_host_one_pass": streaming,
        "gpu_launches": launches, "clocks": clk.summary(),
        "extra_8192": extra,
        "extra_sparse_262144x4096": extra3,
        "extra_batched_4096_blocks": extra4,
    }
    print(json.dumps(res), flush=True)


def run_dense_8192_step(args, rank, world, dev, A, skel, st, seed_G, headline):
    """The 8192 x 8192 step: TF32 sketch -> both LUPPs pipelined (time-to-skeleton) -> column ID
    and stable CUR from one QR of C -> eta on a second stream."""
    import numpy as np
    import torch
    k, p = args.k, args.p
    l = k + p
    m, n = A.shape
    names = ["sketch", "pivots", "id_cur", "eta_after_id_cur"]
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()

    def step(evs, serial=False):
        evs[0].record()
        X, _ = skel.sketch(A, l, prec=args.prec, seed=seed_G, status=st)
        evs[1].record()
        Js, Is, _, Rf, _ = skel.pivot_skeleton(X, A, k, status=st)
        evs[2].record()
        if serial:
            e, _ = skel.error(A, Js, Rf=Rf, status=st)
        else:
            side.wait_stream(main)
            with torch.cuda.stream(side):
                e, _ = skel.error(A, Js, Rf=Rf, status=st)
        Z, U, sq_id, sq_cur, _ = skel.id_cur(A, Js, Is, status=st)
        evs[3].record()
        if not serial:
            main.wait_stream(side)
        evs[4].record()
        return Js, Is, Z, U, sq_id, sq_cur, e

    mk = lambda: _events(len(names) + 1)
    for _ in range(args.warmup):
        step(mk())
    torch.cuda.synchronize()
    skel.check_status(st, "warmup")
    if world > 1 and headline:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = skel.launch_count()
    all_evs = [mk() for _ in range(args.steps)]
    t_begin, t_end = _events(2)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    with ClockSampler(local) as clk:
        t_begin.record()
        for i in range(args.steps):
            out = step(all_evs[i])
        t_end.record()
        torch.cuda.synchronize()
    launches = skel.launch_count() - launches0
    skel.check_status(st, "timed steps")
    total_ms = t_begin.elapsed_time(t_end)
    per = {nm: statistics.mean(ev[i].elapsed_time(ev[i + 1]) for ev in all_evs) for i, nm in enumerate(names)}
    tts = statistics.mean(ev[0].elapsed_time(ev[2]) for ev in all_evs)
    tcur = statistics.mean(ev[0].elapsed_time(ev[3]) for ev in all_evs)
    if world > 1 and headline:
        t = torch.tensor([tts, total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        tts, total_ms = float(t[0]), float(t[1])
    Js, Is, Z, U, sq_id, sq_cur, e = out
    # errors formed directly from the residuals on the device
    er, _ = skel.error(A, Js, Z=Z, Is=Is, U=U, status=st)
    er = er.cpu().numpy()
    sq_id, sq_cur = sq_id.cpu().numpy(), sq_cur.cpu().numpy()
    rel_id, rel_cur = float(er[1] / er[0]), float(er[2] / er[0])
    rel_id_gram = float(np.sqrt(max(sq_id[0] - sq_id[1], 0.0) / sq_id[0]))
    rel_cur_gram = float(np.sqrt(max(sq_cur[0] - sq_cur[1], 0.0) / sq_cur[0]))
    if rank != 0:
        return None

    peaks = load_peaks_full()
    floors = measure_floors(skel, dev, col_words=64)
    nser = max(2, min(args.steps, 10))
    skel.kernel_timing(True)
    s0, s1 = _events(2)
    s0.record()
    for _ in range(nser):
        step(mk(), serial=True)
    s1.record()
    torch.cuda.synchronize()
    ser_ms = s0.elapsed_time(s1)
    models = kernel_models("dense_8192x8192", m, n, k, l, args.prec, peaks, sustained=False, floors=floors)
    kernels = kernel_table(skel, nser, ser_ms, models)
    skel.kernel_timing(False)
    latency_roofline(kernels, "lupp_panel", 2 * k, floors)      # column LUPP on X and row LUPP on C
    modeled = [nm for nm in kernels if kernels[nm].get("bound") in ("hbm", "tensor", "alu")]
    roofline = None
    if modeled:
        dom = max(modeled, key=lambda nm: kernels[nm]["ms_per_step"])
        kd = kernels[dom]
        roofline = {"kernel": dom, "bound": kd["bound"], "achieved": kd["achieved"], "peak": kd["peak"],
                    "unit": kd["unit"], "frac": kd["frac"], "traffic": TRAFFIC_PER_LAUNCH["dense_8192x8192"].get(dom),
                    "peak_source": (f"{peaks['source']} MEASURED_PEAKS.json (burst)" if kd["bound"] != "alu" else
                                    "FMA rate measured in this run (skel_debug_fma_rate)"),
                    "avg_launch_us": kd["avg_us"],
                    "timing": "CUDA events around every launch, serialised pass of the same steps"}

    # the FP64 refinement steps of Z and U (skel_id_refine, skel_cur_refine) against the unrefined calls
    def t_call(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = _events(2)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    refine = {"id_ms": t_call(lambda: skel.column_id(A, Js, status=st)),
              "id_refined_ms": t_call(lambda: skel.column_id_refined(A, Js, status=st)),
              "cur_ms": t_call(lambda: skel.cur(A, Js, Is, status=st)),
              "cur_refined_ms": t_call(lambda: skel.cur(A, Js, Is, status=st, refine=True))}
    skel.check_status(st, "refinement")

    # FP64 plain-GPU form of the skeleton stage on the same matrix
    fp64 = None
    if not args.no_fp64:
        A64 = A.double().t().contiguous().t()
        evs = _events(3)
        for rep in range(2):
            evs[0].record()
            X64, _ = skel.sketch(A64, l, prec="f64", seed=seed_G, status=st)
            evs[1].record()
            J64, I64, _, _, _ = skel.pivot_skeleton(X64, A64, k, factors=False, status=st)
            evs[2].record()
        torch.cuda.synchronize()
        skel.check_status(st, "fp64")
        rel64, _ = direct_rel_error(skel, A, J64, st)
        fp64 = {"time_to_skeleton_ms": evs[0].elapsed_time(evs[2]), "sketch_ms": evs[0].elapsed_time(evs[1]),
                "pivots_ms": evs[1].elapsed_time(evs[2]), "rel_id_error": rel64,
                "same_skeleton": bool(torch.equal(J64.cpu(), Js.cpu()))}
        del A64, X64

    # end to end through host buffers: pinned A -> device, skeleton, indices back
    A_host = torch.empty(n, m, dtype=torch.float32, pin_memory=True)
    A_host.copy_(A.t())
    A_dev = torch.empty(n, m, dtype=torch.float32, device=dev)
    Js_h = torch.empty(k, dtype=torch.int32, pin_memory=True)
    Is_h = torch.empty(k, dtype=torch.int32, pin_memory=True)

    def e2e_step():
        A_dev.copy_(A_host, non_blocking=True)
        Ad = A_dev.t()
        X, _ = skel.sketch(Ad, l, prec=args.prec, seed=seed_G, status=st)
        J, I, _, _, _ = skel.pivot_skeleton(X, Ad, k, factors=False, status=st)
        Js_h.copy_(J, non_blocking=True)
        Is_h.copy_(I, non_blocking=True)
        torch.cuda.current_stream().synchronize()     # the host reads the skeletons every step
        return int(Js_h[0]) + int(Is_h[0])

    for _ in range(2):
        e2e_step()
    e2e_ms, e2e_steps_ms = wall_steps(e2e_step, args.steps)
    skel.check_status(st, "e2e")

    cpu = None
    if not args.no_cpu:
        A_np = np.asfortranarray(A[:, :min(ORACLE_SAMPLE_COLS, n)].double().cpu().numpy())
        cpu = cpu_sample_baseline(A_np, m, n, k, p, seed_G)
    res = {
        "metric": METRIC, "value": tts, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
        "config": workload_config("dense_8192x8192", k, p, args.prec),
        "time_to_id_and_cur_ms": tcur, "a_streaming_gbs": 4.0 * m * n / (per["sketch"] * 1e-3) / 1e9,
        "sketch_tflops": 2.0 * l * m * n / (per["sketch"] * 1e-3) / 1e12, "calls_ms": per,
        "rel_id_error": rel_id, "rel_cur_error": rel_cur, "rel_id_error_gram": rel_id_gram,
        "rel_cur_error_gram": rel_cur_gram, "eta": float(e[3]),
        "fp64_gpu": fp64, "id_error_ratio_vs_fp64": (rel_id / fp64["rel_id_error"]) if fp64 else None,
        "fp64_refinement": refine,
        "roofline": roofline, "kernels": kernels, "serialised_ms_per_step": ser_ms / nser, "cpu_baseline": cpu,
        "measured_floors": floors,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(4 * m * n),
                "d2h_bytes_per_step": int(8 * k), "step_ms": e2e_steps_ms, "clock": "host wall"},
        "gpu_launches": launches, "clocks": clk.summary(),
    }
    return res


def run_c3(skel, dev, steps=10, warmup=3):
    """The tall sparse configuration: 262144 x 4096 SNN-style CSC (~1% dense), k = 256, sparse
    sign embedding with zeta = 8 and l = 2k.  Times the CSC sketch (algorithmic bytes: the CSC
    arrays read once and X written once), the skeletons (sketch + LUPP on X + row LUPP on
    C = A(:, J_s)) and the stable CUR with rows given; C, R and the CUR use the densified A
    (4.3 GB, column-major FP32)."""
    import numpy as np
    import torch
    import workloads
    m, n, r, k, zeta = 262144, 4096, 300, 256, 8
    l = 2 * k
    seed_G = workloads.seed_for("snn_262144x4096", "gamma")
    A = workloads.snn_csc(m, n, r, seed=workloads.seed_for("snn_262144x4096"))
    nnz = int(A.nnz)
    col_ptr = torch.from_numpy(A.indptr.astype(np.int64)).to(dev)
    row_idx = torch.from_numpy(A.indices.astype(np.int32)).to(dev)
    val = torch.from_numpy(A.data.astype(np.float32)).to(dev)
    cols = torch.repeat_interleave(torch.arange(n, device=dev), col_ptr[1:] - col_ptr[:-1])
    At = torch.zeros(n, m, dtype=torch.float32, device=dev)
    At[cols, row_idx.long()] = val
    Ad = At.t()
    del cols
    st = skel.new_status(dev)
    X = torch.empty(l, n, dtype=torch.float32, device=dev)
    Js = torch.empty(k, dtype=torch.int32, device=dev)

    def sk():
        skel.sketch_csc(col_ptr, row_idx, val, m, n, l, seed=seed_G, zeta=zeta, status=st, X=X)

    def timed(fn, reps):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = _events(2)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    sketch_ms = timed(sk, steps)
    skel.kernel_timing(True)
    sk()
    torch.cuda.synchronize()
    kern_ms = skel.kernel_time("sparse_csc")[0]
    skel.kernel_timing(False)

    out = {}

    def skeleton():
        sk()
        J, _, _, _ = skel.pivot_lupp(X, k, factors=False, status=st)
        I, _ = skel.pivot_rows(Ad, J, status=st)
        out["J"], out["I"] = J, I

    tts = timed(skeleton, steps)
    J, I = out["J"], out["I"]
    cur_ms = timed(lambda: skel.cur(Ad, J, I, status=st), max(2, steps // 2))
    skel.kernel_timing(True)
    _, U, _, _ = skel.cur(Ad, J, I, status=st)
    torch.cuda.synchronize()
    cur_kernels = kernel_table(skel, 1, cur_ms, {})
    skel.kernel_timing(False)
    e, _ = skel.error(Ad, J, Is=I, U=U, status=st)
    skel.check_status(st, "tall sparse configuration")
    e = e.cpu().numpy()
    hbm = load_peaks_full()["hbm_gbs"]
    a_bytes = 8.0 * nnz + 8.0 * (n + 1) + 4.0 * l * n
    k_ms = kern_ms if kern_ms > 0 else sketch_ms
    res = {"workload": f"262144x4096 SNN-style CSC (nnz {nnz}, {nnz / (m * n):.4f} dense), sparse sign zeta={zeta}, "
                       f"l={l}, k={k}; CUR with rows by LUPP on C",
           "sketch_ms": sketch_ms, "sketch_kernel_ms": kern_ms, "sketch_bytes": a_bytes,
           "sketch_gbs": a_bytes / (k_ms * 1e-3) / 1e9, "sketch_frac_of_hbm": a_bytes / (k_ms * 1e-3) / 1e9 / hbm,
           "time_to_skeleton_ms": tts, "cur_ms": cur_ms, "cur_kernels_serialised": cur_kernels,
           "rel_cur_error": float(e[2] / e[0])}
    del At, Ad, X
    torch.cuda.empty_cache()
    return res


def run_timed(args, rank, call, st, config):
    """--warmup + --steps calls of `call`, timed with CUDA events; one JSON line."""
    import torch
    import paper_2104_05877_gb300 as skel
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    skel.check_status(st, args.only)
    if rank == 0:
        print(json.dumps({"only": args.only, "ms": e0.elapsed_time(e1) / args.steps, "config": config}), flush=True)


def run_only(args, rank, A, skel, st, seed_G):
    """One call, --warmup + --steps times, timed with CUDA events: a small command for profilers."""
    import torch
    k, p = args.k, args.p
    l = k + p
    X, _ = skel.sketch(A, l, prec=args.prec, seed=seed_G, status=st)
    Js, _, Rf, _ = skel.pivot_lupp(X, k, status=st)
    Is = None
    if args.only in ("rows", "cur", "id_cur"):
        Is, _ = skel.pivot_rows(A, Js, status=st)
    call = {"sketch": lambda: skel.sketch(A, l, prec=args.prec, seed=seed_G, X=X, status=st),
            "lupp": lambda: skel.pivot_lupp(X, k, status=st),
            "rows": lambda: skel.pivot_rows(A, Js, status=st),
            "pivots": lambda: skel.pivot_skeleton(X, A, k, status=st),
            "id": lambda: skel.column_id(A, Js, status=st),
            "cur": lambda: skel.cur(A, Js, Is, status=st),
            "id_cur": lambda: skel.id_cur(A, Js, Is, status=st),
            "eta": lambda: skel.error(A, Js, Rf=Rf, status=st),
            "srtt": lambda: skel.sketch(A, l, kind="srtt", prec=args.prec, seed=seed_G, X=X, status=st),
            "power": lambda: skel.sketch_power(A, l, q=1, prec=args.prec, seed=seed_G, status=st),
            "cols": lambda: skel.sketch_cols(A, l, prec=args.prec, seed=seed_G + 1, status=st)}[args.only]
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    skel.check_status(st, args.only)
    if rank == 0:
        print(json.dumps({"only": args.only, "ms": e0.elapsed_time(e1) / args.steps,
                          "config": workload_config(args.workload, k, p, args.prec)}), flush=True)


def run_next(args, rank, A, skel, st, seed_G):
    """The rows beyond the hot path on the dense workload, each timed alone (CUDA events over
    --steps calls after --warmup): the SRTT sketch (tensor cores), the power-iterated sketch
    X = Omega (A^T A) (a transposed copy of A, then one pass over each), the column sketch
    Y^T = Omega A^T (tensor cores on the transposed copy),
    streaming selection (row and column sketches + two LUPPs), the column ID from the sketch
    (Z = X(:, J)^+ X) and the CUR core from the skeletons (U = A(Is, Js)^{-1})."""
    import torch
    k, p = args.k, args.p
    l = k + p
    m, n = A.shape
    prec = "tf32" if args.prec not in ("tf32", "bf16") else args.prec
    X, _ = skel.sketch(A, l, prec=prec, seed=seed_G, status=st)
    Js, _, Rf, _ = skel.pivot_lupp(X, k, status=st)
    Is, _ = skel.pivot_rows(A, Js, status=st)
    calls = {
        "srtt_sketch": (lambda: skel.sketch(A, l, kind="srtt", prec=prec, seed=seed_G, X=X, status=st), 1),
        "power_sketch_q1": (lambda: skel.sketch_power(A, l, q=1, prec=prec, seed=seed_G, status=st), 2),
        "col_sketch": (lambda: skel.sketch_cols(A, l, prec=prec, seed=seed_G + 1, status=st), 1),
        "streaming_selection": (lambda: skel.skeletonize_streaming(A, k, p, seed=seed_G, seed_omega=seed_G + 1,
                                                                   prec=prec, status=st), 2),
        "id_from_sketch": (lambda: skel.column_id_sketch(X, Js, status=st), 0),
        "cur_core_from_skeletons": (lambda: skel.cur_sketch(A, Js, Is, status=st), 0),
    }
    out = {}
    for nm, (fn, passes) in calls.items():
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = _events(2)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        skel.check_status(st, nm)
        ms = e0.elapsed_time(e1) / args.steps
        ent = {"ms": ms}
        if passes:
            ent["a_passes"] = passes
            ent["a_gbs"] = passes * 4.0 * m * n / (ms * 1e-3) / 1e9
        out[nm] = ent
    hbm, _, src = load_peaks()
    for ent in out.values():
        if "a_gbs" in ent:
            ent["frac_of_hbm"] = ent["a_gbs"] / hbm
    if rank == 0:
        print(json.dumps({"only": "next", "rows": out, "hbm_peak_gbs": hbm, "peak_source": src,
                          "config": workload_config(args.workload, k, p, prec)}), flush=True)


def batch_measure(skel, dev, nblocks=4096, steps=10, warmup=3, seed_offset=0):
    """Batched configuration: uneven Gaussian-kernel blocks (m_b ~ U[64, 1024], n_b ~ U[64, 512],
    FP32, ~2.5 GB for 4096 blocks), k_max = 128, p = 16, tol = 1e-6: one skel_batch_run per
    step (an autotuned plan replaying its captured CUDA graph), A read once per run."""
    import torch
    import workloads
    kmax, p, tol = 128, 16, 1e-6
    blocks = workloads.torch_kernel_blocks(nblocks, workloads.seed_for("kernel_blocks_4096") + seed_offset, dev)
    a_bytes = sum(4 * B.shape[0] * B.shape[1] for B in blocks)
    plan = skel.BatchPlan(blocks, kmax, p=p, tol=tol, seed=workloads.seed_for("kernel_blocks_4096", "gamma"),
                          graph=True, autotune=True)
    torch.cuda.synchronize()
    for _ in range(warmup):
        Js, ranks, Z, st = plan.run()
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    e0.record()
    for _ in range(steps):
        Js, ranks, Z, st = plan.run()
    e1.record()
    torch.cuda.synchronize()
    skel.check_status(st, "batch")
    ms = e0.elapsed_time(e1) / steps
    skel.kernel_timing(True)
    plan.run()
    torch.cuda.synchronize()
    kern = {nm: skel.kernel_time(nm)[0] for nm in ("batch_sketch", "batch_lupp", "batch_z")}
    skel.kernel_timing(False)
    r = ranks.float()
    hbm = load_peaks_full()["hbm_gbs"]
    out = {"ms": ms, "a_bytes": a_bytes, "a_streaming_gbs": a_bytes / (ms * 1e-3) / 1e9,
           "frac_of_hbm": a_bytes / (ms * 1e-3) / 1e9 / hbm, "kernel_ms": kern,
           "rank_mean": float(r.mean()), "rank_max": int(r.max()), "plan": plan.info,
           "workload": f"{nblocks} Gaussian-kernel blocks m_b~U[64,1024] n_b~U[64,512] fp32, k_max={kmax}, p={p}, "
                       f"tol={tol}; Z = X_b(:, J)^+ X_b", "steps": steps}
    del plan, blocks
    torch.cuda.empty_cache()
    out["points"] = batch_points_measure(skel, dev, nblocks, steps, warmup, seed_offset, a_bytes)
    return out


def batch_points_measure(skel, dev, nblocks, steps, warmup, seed_offset, a_bytes):
    """The same batched workload given implicitly by its point sets (kernel_points: the draws of
    the stored blocks, FP32): skel_batch_plan_create_points evaluates every kernel entry inside
    the sketch kernel (a two-float exponent and expf per entry), so the blocks are never
    stored; 32 bytes per point are read instead of 4 bytes per entry."""
    import numpy as np
    import torch
    import workloads
    kmax, p, tol = 128, 16, 1e-6
    pts = workloads.kernel_points(nblocks, workloads.seed_for("kernel_blocks_4096") + seed_offset)
    xs = [torch.from_numpy(x).to(dev) for x, _ in pts]
    ys = [torch.from_numpy(y).to(dev) for _, y in pts]
    entries = sum(x.shape[0] * y.shape[0] for x, y in pts)
    plan = skel.BatchPlan.from_points(xs, ys, 0.5, kmax, p=p, tol=tol,
                                      seed=workloads.seed_for("kernel_blocks_4096", "gamma"), graph=True, autotune=True)
    torch.cuda.synchronize()
    for _ in range(warmup):
        Js, ranks, Z, st = plan.run()
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    e0.record()
    for _ in range(steps):
        Js, ranks, Z, st = plan.run()
    e1.record()
    torch.cuda.synchronize()
    skel.check_status(st, "batch points")
    ms = e0.elapsed_time(e1) / steps
    skel.kernel_timing(True)
    plan.run()
    torch.cuda.synchronize()
    kern = {nm: skel.kernel_time(nm)[0] for nm in ("batch_sketch", "batch_lupp", "batch_z")}
    skel.kernel_timing(False)
    r = ranks.float()
    out = {"ms": ms, "kernel_ms": kern, "kernel_entries": entries,
           "entries_per_s": entries / (kern["batch_sketch"] * 1e-3) if kern["batch_sketch"] > 0 else None,
           "point_bytes": 32 * sum(x.shape[0] + y.shape[0] for x, y in pts), "stored_block_bytes": a_bytes,
           "rank_mean": float(r.mean()), "rank_max": int(r.max()), "plan": plan.info,
           "workload": f"the same {nblocks} blocks given by their FP32 point sets (3-D, h = 0.5), entries evaluated "
                       "inside the sketch kernel"}
    del plan, xs, ys
    torch.cuda.empty_cache()
    return out


def run_batch(args, rank, dev, skel, workloads):
    """--only batch: the batched configuration alone, one JSON line."""
    out = batch_measure(skel, dev, args.blocks, args.steps, args.warmup, seed_offset=rank)
    if rank == 0:
        out["only"] = "batch"
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank)
        else:
            run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
