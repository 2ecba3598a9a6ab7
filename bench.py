#!/usr/bin/env python
"""Benchmark of randomized-pivoting skeletonization (Algorithm 2) on GB300.

Workload (one "step" = the whole hot path on one synthetic matrix resident in HBM):
  A: 8192 x 8192 FP32, A = U diag(sigma) V^T + 1e-6 floor, sigma_j = 1/j, Haar U, V;
  k = 256, oversampling p = 16 (l = 272), Gaussian embedding.
  step = TF32 tensor-core sketch X = Gamma A  ->  LUPP on X (J_s, R^LU) with the row LUPP on
         C = A(:, J_s) (I_s) pipelined behind it  [time-to-skeleton]  ->  column ID Z and stable
         CUR U from one QR of C  [time to ID and CUR]  ->  Theorem 1's eta from R^LU (on a
         second stream, concurrent with the ID and CUR); errors from the Gram identities.
Reported: time-to-skeleton (ms, the metric), time to ID and CUR, A-streaming GB/s of the sketch,
per-call times, the FP64 plain-GPU form of the skeleton stage on the same A, relative ID
error against the FP64 oracle, a roofline entry for the dominant call, the oracle timed on
the host cores, and an end-to-end number through host buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--k 256]

Multi-GPU: N ranks run N independent replicas (one matrix each, weak scaling) with no
collective on the data path (the row-partitioned sketch with its one all-reduce is the
library's `dist` module, exercised by the multi-process tests).  --impl reference times the
FP64 CPU oracle (the only reference this paper has) on rank 0.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-skeleton (ms) and A-streaming GB/s at rank k, mixed vs FP64 GPU, equal ID error"
M_DIM = N_DIM = 8192


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=256)
    ap.add_argument("--p", type=int, default=16)
    ap.add_argument("--prec", default="tf32", choices=["tf32", "bf16", "fp8", "f32"])
    ap.add_argument("--blocks", type=int, default=4096, help="blocks of the batched run (--only batch)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 plain-GPU comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--only", default=None, choices=["sketch", "lupp", "rows", "pivots", "id", "cur", "id_cur", "eta", "batch", "next",
                                                     "srtt", "power", "cols"],
                    help="run only this call (warm-up + steps, no extras): a small command for profilers; "
                         "'batch' runs the batched configuration (4096 Gaussian-kernel blocks, k_max 128, "
                         "tol 1e-6) instead of the dense workload; 'next' times the rows beyond the hot "
                         "path (SRTT sketch, power sketch, column sketch, streaming selection, ID and CUR "
                         "from the sketch) on the same workload, one JSON line")
    return ap.parse_args()


def workload_config(k, p, prec):
    return {"workload": f"dense {M_DIM}x{N_DIM} fp32, sigma_j=1/j + 1e-6 floor, Haar U/V; "
                        f"rank k={k}, oversampling p={p} (l={k + p}); Gaussian sketch ({prec}), "
                        "LUPP on X, row LUPP on C, column ID + stable CUR",
            "m": M_DIM, "n": N_DIM, "k": k, "l": k + p, "sketch_prec": prec,
            "l2": "inputs larger than L2 (A is 268 MB; L2 129 MB)"}


def make_A(device, seed):
    import numpy as np
    import torch
    import workloads
    sig = workloads.sigma_config2(min(M_DIM, N_DIM))
    return workloads.torch_dense_spectrum(M_DIM, N_DIM, sig, 1e-6 / np.sqrt(M_DIM), seed, device,
                                          torch.float32)


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


# kernels timed with CUDA events during the timed region
TIMED_KERNELS = ("sketch_tc", "sketch_fp8", "fp8_quantize", "gemm_tc", "lupp_panel", "lupp_trail", "qr_panel", "qr_wy", "trsm", "gemm_qr",
                 "gemm_cur", "gemm_eta_h", "gemm_eta_sq", "gemm_simt")
# DRAM bytes (read + write) per launch from one ncu capture of the current kernel at this
# workload (None where no capture of the current code exists)
TRAFFIC_PER_LAUNCH = {"sketch_tc": 271.9e6, "gemm_tc": 332.4e6, "lupp_panel": 3.09e6, "qr_panel": 2.15e6}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d["hbm_gbs"], d["bf16_tflops"], "measured"
    return 6800.0, 1900.0, "fallback"


# ------------------------------------------------------------------------------------------
def oracle_skeleton(A_np, k, p, seed):
    """The FP64 CPU oracle's time-to-skeleton: sketch, LUPP on X, row LUPP on C."""
    from oracle import sketch, pivoting
    t0 = time.perf_counter()
    X = sketch.gaussian_sketch(A_np, k + p, seed)
    Js = pivoting.lupp_columns(X, k)["Js"]
    Is = pivoting.lupp_rows(A_np[:, Js], k)["Js"]
    return time.perf_counter() - t0, Js, Is


def run_reference(args, rank):
    if rank != 0:
        return
    import numpy as np
    import workloads
    seed_A, seed_G = workloads.seed_for(2), workloads.seed_for(2, "gamma")
    try:
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        A_np = np.asfortranarray(make_A(dev, seed_A).double().cpu().numpy())
    except Exception:
        A_np = workloads.dense_config2(M_DIM, N_DIM, seed=seed_A, dtype=np.float32).astype(np.float64)
    times = []
    for i in range(args.warmup + args.steps):
        dt, _, _ = oracle_skeleton(A_np, args.k, args.p, seed_G)
        if i >= args.warmup:
            times.append(dt * 1e3)
    v = statistics.mean(times)
    cores = os.cpu_count()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.k, args.p, "f64 oracle"),
        "cpu_baseline": {"value": v, "unit": "ms", "cores": cores, "kind": "oracle",
                         "sample": "full workload per step (sketch + LUPP on X + row LUPP on C)"},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------------------------------
def run_ours(args, rank, world):
    import numpy as np
    import torch
    import paper_2104_05877_gb300 as skel
    import workloads

    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    if not os.path.exists(skel.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    k, p = args.k, args.p
    l = k + p
    if args.only == "batch":
        run_batch(args, rank, dev, skel, workloads)
        return
    seed_A, seed_G = workloads.seed_for(2) + rank, workloads.seed_for(2, "gamma")
    A = make_A(dev, seed_A)
    torch.cuda.synchronize()
    st = skel.new_status(dev)

    names = ["sketch", "pivots", "id_cur", "eta_after_id_cur"]
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()

    def step(evs):
        evs[0].record()
        X, _ = skel.sketch(A, l, prec=args.prec, seed=seed_G, status=st)
        evs[1].record()
        # column LUPP on X and row LUPP on C = A(:, Js), the latter pipelined behind the former
        Js, Is, _, Rf, _ = skel.pivot_skeleton(X, A, k, status=st)
        evs[2].record()
        # eta needs only the pivot factor: it runs on a second stream while the column ID and
        # the stable CUR (one QR of C for both) run on this one
        side.wait_stream(main)
        with torch.cuda.stream(side):
            e, _ = skel.error(A, Js, Rf=Rf, status=st)
        Z, U, sq_id, sq_cur, _ = skel.id_cur(A, Js, Is, status=st)
        evs[3].record()
        main.wait_stream(side)
        evs[4].record()
        return Js, Is, sq_id, sq_cur, e

    if args.only == "next":
        run_next(args, rank, A, skel, st, seed_G)
        return
    if args.only:
        X, _ = skel.sketch(A, l, prec=args.prec, seed=seed_G, status=st)
        Js, _, Rf, _ = skel.pivot_lupp(X, k, status=st)
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
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            call()
        e1.record()
        torch.cuda.synchronize()
        skel.check_status(st, args.only)
        if rank == 0:
            print(json.dumps({"only": args.only, "ms": e0.elapsed_time(e1) / args.steps,
                              "config": workload_config(k, p, args.prec)}), flush=True)
        return

    mk = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
    for _ in range(args.warmup):
        step(mk())
    torch.cuda.synchronize()
    skel.check_status(st, "warmup")
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = skel.launch_count()
    all_evs = [mk() for _ in range(args.steps)]
    t_begin = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t_begin.record()
        for i in range(args.steps):
            out = step(all_evs[i])
        t_end.record()
        torch.cuda.synchronize()
    # second timed region, same steps, with CUDA events around the hot kernels' launches (kept
    # apart so that the recorded events do not touch the headline numbers)
    skel.kernel_timing(True)
    kev = [mk() for _ in range(args.steps)]
    k_begin, k_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k_begin.record()
    for i in range(args.steps):
        step(kev[i])
    k_end.record()
    torch.cuda.synchronize()
    ktimes = {nm: skel.kernel_time(nm) for nm in TIMED_KERNELS}
    skel.kernel_timing(False)
    k_total_ms = k_begin.elapsed_time(k_end)
    if world > 1:
        torch.distributed.barrier()
    launches = skel.launch_count() - launches0
    skel.check_status(st, "timed steps")
    total_ms = t_begin.elapsed_time(t_end)
    per = {nm: statistics.mean(ev[i].elapsed_time(ev[i + 1]) for ev in all_evs) for i, nm in enumerate(names)}
    tts = statistics.mean(ev[0].elapsed_time(ev[2]) for ev in all_evs)
    tcur = statistics.mean(ev[0].elapsed_time(ev[3]) for ev in all_evs)
    if world > 1:
        t = torch.tensor([tts, total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        tts, total_ms = float(t[0]), float(t[1])
    Js, Is, sq_id, sq_cur, e = out
    sq_id, sq_cur, e = sq_id.cpu().numpy(), sq_cur.cpu().numpy(), e.cpu().numpy()
    rel_id = float(np.sqrt(max(sq_id[0] - sq_id[1], 0.0) / sq_id[0]))
    rel_cur = float(np.sqrt(max(sq_cur[0] - sq_cur[1], 0.0) / sq_cur[0]))
    if rank != 0:
        return

    hbm, bf16, peak_src = load_peaks()
    tf32_peak = bf16 * (1.1 / 2.25)          # nominal TF32 : BF16 dense ratio
    m, n = M_DIM, N_DIM
    a_bytes = 4.0 * m * n
    sketch_gbs = a_bytes / (per["sketch"] * 1e-3) / 1e9
    sketch_tflops = 2.0 * l * m * n / (per["sketch"] * 1e-3) / 1e12
    fp32_alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12        # TFLOP/s, FFMA
    fp64_alu_peak = 1.25                                  # TFLOP/s, nominal FP64
    # Algorithmic work of each timed kernel over one step (bound, work, peak, unit):
    #   sketch_tc   X = Gamma A: 2 l m n TF32 flop (or 4 m n bytes of A if HBM-bound)
    #   sketch_fp8  X = Gamma8 A8 from the e4m3 copy of A: m n bytes; fp8_quantize reads A and
    #               writes A8: 5 m n bytes
    #   gemm_tc     W = Q^T A, shared by the ID and the CUR: 3 (2 k m n) TF32 flop (3 products)
    #   lupp_panel  s greedy steps over n (LUPP on X) and over m (row LUPP on C): the panel
    #               rank-1 updates, sum over panels of b^2 cols (mul + sub)
    #   qr_panel    the column steps of the two Householder QRs (C and R^T): 2 rows k^2
    #               flop each (the panels' WY factors are formed by other kernels)
    #   trsm        Z = R_C^{-1} W (k^2 n) and four k x k solves (CUR, eta): FP64
    #   gemm_eta_h  upper triangle of R R^T in float-float: k(k+1)/2 n products, each
    #               9 FP32 pipe instructions (exact product + two-sum); peak = one FP32
    #               instruction per lane per clock
    b_pan = 64
    lupp_flops = sum(min(b_pan, k - t0) ** 2 for t0 in range(0, k, b_pan)) * (n + m)
    models = {
        "sketch_tc": ("tensor", 2.0 * l * m * n / 1e12, tf32_peak, "TFLOP/s")
        if 2.0 * l * m * n / (tf32_peak * 1e12) > a_bytes / (hbm * 1e9) else ("hbm", a_bytes / 1e9, hbm, "GB/s"),
        "sketch_fp8": ("hbm", m * n / 1e9, hbm, "GB/s"),           # A8: one byte per element
        "fp8_quantize": ("hbm", 5.0 * m * n / 1e9, hbm, "GB/s"),   # A read (4 B), A8 written (1 B)
        "gemm_tc": ("tensor", 3 * 2.0 * k * m * n / 1e12, tf32_peak, "TFLOP/s"),
        "lupp_panel": ("alu", lupp_flops / 1e12, fp32_alu_peak, "TFLOP/s"),
        "qr_panel": ("alu", 2.0 * (m + n) * k * k / 1e12, fp32_alu_peak, "TFLOP/s"),
        "trsm": ("alu", (1.0 * k * k * n + 4.0 * k ** 3) / 1e12, fp64_alu_peak, "TFLOP/s"),
        "gemm_eta_h": ("alu", 9.0 * k * (k + 1) / 2 * n / 1e12, fp32_alu_peak / 2, "TOP/s"),
    }
    kernels = {}
    for nm, (tot, cnt) in ktimes.items():
        if cnt == 0:
            continue
        ent = {"ms_per_step": tot / args.steps, "launches_per_step": cnt / args.steps,
               "avg_us": 1e3 * tot / cnt, "share_of_step": tot / k_total_ms}
        if nm in models:
            b, w, pk, u = models[nm]
            a = w / (tot / args.steps * 1e-3)          # work per step / device time per step
            ent.update({"bound": b, "achieved": a, "peak": pk, "unit": u, "frac": a / pk})
        kernels[nm] = ent
    modeled = [nm for nm in kernels if "bound" in kernels[nm]]
    dom = max(modeled, key=lambda nm: kernels[nm]["ms_per_step"])
    kd = kernels[dom]
    roofline = {"kernel": dom, "bound": kd["bound"], "achieved": kd["achieved"], "peak": kd["peak"],
                "unit": kd["unit"], "frac": kd["frac"], "traffic": TRAFFIC_PER_LAUNCH.get(dom),
                "peak_source": f"{peak_src} MEASURED_PEAKS.json" if peak_src == "measured" else "fallback",
                "launches_per_step": kd["launches_per_step"], "avg_launch_us": kd["avg_us"],
                "timing": "CUDA events on the launching stream around every launch, in a second timed "
                          "region of the same steps"}
    calls = {nm: {"ms": per[nm], "share": per[nm] / sum(per.values())} for nm in names}

    # FP64 plain-GPU form of the skeleton stage on the same matrix
    fp64 = None
    if not args.no_fp64:
        A64 = A.double().t().contiguous().t()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        for rep in range(2):
            evs[0].record()
            X64, _ = skel.sketch(A64, l, prec="f64", seed=seed_G, status=st)
            evs[1].record()
            J64, I64, _, _, _ = skel.pivot_skeleton(X64, A64, k, factors=False, status=st)
            evs[2].record()
        torch.cuda.synchronize()
        _, sq64, _ = skel.column_id(A64, J64, status=st)
        torch.cuda.synchronize()
        skel.check_status(st, "fp64")
        sq64 = sq64.cpu().numpy()
        fp64 = {"time_to_skeleton_ms": evs[0].elapsed_time(evs[2]), "sketch_ms": evs[0].elapsed_time(evs[1]),
                "pivots_ms": evs[1].elapsed_time(evs[2]),
                "rel_id_error": float(np.sqrt(max(sq64[0] - sq64[1], 0.0) / sq64[0])),
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

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        e2e_step()
    e1.record()
    torch.cuda.synchronize()
    skel.check_status(st, "e2e")
    e2e_ms = e0.elapsed_time(e1) / args.steps

    # the FP64 CPU oracle on the host: one bounded sample of the same workload + its ID error
    cpu = None
    oracle_err = None
    if not args.no_cpu:
        from oracle import decomp, errors
        A_np = np.asfortranarray(A.double().cpu().numpy())
        dt, Jo, Io = oracle_skeleton(A_np, k, p, seed_G)
        cpu = {"value": dt * 1e3, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "one full time-to-skeleton run (FP64 sketch + LUPP on X + row LUPP on C) on the same A"}
        Zo = decomp.column_id(A_np, Jo)
        oracle_err = errors.rel_id_error(A_np, Jo, Zo)

    res = {
        "metric": METRIC, "value": tts, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
        "config": workload_config(k, p, args.prec),
        "time_to_id_and_cur_ms": tcur, "a_streaming_gbs": sketch_gbs,
        "sketch_tflops": sketch_tflops, "calls_ms": per,
        "rel_id_error": rel_id, "rel_cur_error": rel_cur, "eta": float(e[3]),
        "oracle_rel_id_error": oracle_err,
        "id_error_ratio_vs_oracle": (rel_id / oracle_err) if oracle_err else None,
        "fp64_gpu": fp64,
        "roofline": roofline, "kernels": kernels, "calls": calls, "cpu_baseline": cpu,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(4 * m * n),
                "d2h_bytes_per_step": int(8 * k)},
        "gpu_launches": launches, "clocks": clk.summary(),
    }
    print(json.dumps(res), flush=True)


def run_next(args, rank, A, skel, st, seed_G):
    """The rows beyond the hot path on the dense workload, each timed alone (CUDA events over
    --steps calls after --warmup): the SRTT sketch (tensor cores), the power-iterated sketch
    X = Omega (A^T A) (a transposed copy of A, then one pass over each), the column sketch
    Y^T = Omega A^T (tensor cores on the transposed copy),
    streaming selection (row and column sketches + two LUPPs), the column ID from the sketch
    (Z = R_1^{-1} R) and the CUR core from the skeletons (U = A(Is, Js)^{-1})."""
    import torch
    k, p = args.k, args.p
    l = k + p
    m, n = A.shape
    X, _ = skel.sketch(A, l, prec=args.prec, seed=seed_G, status=st)
    Js, _, Rf, _ = skel.pivot_lupp(X, k, status=st)
    Is, _ = skel.pivot_rows(A, Js, status=st)
    calls = {
        "srtt_sketch": (lambda: skel.sketch(A, l, kind="srtt", prec=args.prec, seed=seed_G, X=X, status=st), 1),
        "power_sketch_q1": (lambda: skel.sketch_power(A, l, q=1, prec=args.prec, seed=seed_G, status=st), 2),
        "col_sketch": (lambda: skel.sketch_cols(A, l, prec=args.prec, seed=seed_G + 1, status=st), 1),
        "streaming_selection": (lambda: skel.skeletonize_streaming(A, k, p, seed=seed_G, seed_omega=seed_G + 1,
                                                                   prec=args.prec, status=st), 2),
        "id_from_sketch": (lambda: skel.column_id_sketch(Rf, Js, status=st), 0),
        "cur_core_from_skeletons": (lambda: skel.cur_sketch(A, Js, Is, status=st), 0),
    }
    out = {}
    for nm, (fn, passes) in calls.items():
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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
                          "config": workload_config(k, p, args.prec)}), flush=True)


def run_batch(args, rank, dev, skel, workloads):
    """Batched configuration: uneven Gaussian-kernel blocks (4096 by default: m_b ~ U[64, 1024],
    n_b ~ U[64, 512], FP32, ~2.6 GB), k_max = 128, p = 16, tol = 1e-6: one skel_batch_run per
    step (an autotuned plan replaying its captured CUDA graph)."""
    import torch
    nblocks, kmax, p, tol = args.blocks, 128, 16, 1e-6
    blocks = workloads.torch_kernel_blocks(nblocks, workloads.seed_for(4) + rank, dev)
    a_bytes = sum(4 * B.shape[0] * B.shape[1] for B in blocks)
    plan = skel.BatchPlan(blocks, kmax, p=p, tol=tol, seed=workloads.seed_for(4, "gamma"), graph=True, autotune=True)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        Js, ranks, Z, st = plan.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        Js, ranks, Z, st = plan.run()
    e1.record()
    torch.cuda.synchronize()
    skel.check_status(st, "batch")
    ms = e0.elapsed_time(e1) / args.steps
    skel.kernel_timing(True)
    plan.run()
    torch.cuda.synchronize()
    kern = {nm: skel.kernel_time(nm)[0] for nm in ("batch_sketch", "batch_lupp")}
    skel.kernel_timing(False)
    r = ranks.float()
    if rank == 0:
        print(json.dumps({"only": "batch", "ms": ms, "a_bytes": a_bytes, "a_streaming_gbs": a_bytes / (ms * 1e-3) / 1e9,
                          "kernel_ms": kern, "rank_mean": float(r.mean()), "rank_max": int(r.max()),
                          "plan": plan.info,
                          "config": {"workload": f"{nblocks} Gaussian-kernel blocks m_b~U[64,1024] n_b~U[64,512] fp32, "
                                                 f"k_max={kmax}, p={p}, tol={tol}", "steps": args.steps}}), flush=True)


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
