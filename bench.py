#!/usr/bin/env python3
"""Benchmark of the decode-fused CSR-dtANS SpMV on GB300.

Workload (default): the 27-point 3-D Poisson stencil on a periodic 128^3 grid
(2,097,152 rows, 56,623,104 entries, FP64 values 26 / -1), x ~ U[-1, 1].
One step = one y = A x over the whole matrix with the entropy decode fused in
(one launch of the library's kernel through the C ABI).  The working set
(about 126 MB) is below the 129 MB L2, so L2 is flushed (a 2 x L2 buffer is
written) between timed steps; the flush is outside the timed events.

Output: one JSON line (rank 0) with the metric GFLOP/s = 2 nnz / t, the
HBM-roofline object of the kernel, the CPU-oracle baseline, the end-to-end
figure through the C ABI with host buffers (dtans_spmv_host), clocks and
launch count, and ``other_configs``: the other workloads measured in the
same run (PR1 n = 4096, the 4 M-row power-law matrix, the 64-matrix batch in
one graph launch, k = 1/4/8/16 right-hand sides on a 2^20-row matrix, and the
pruned 8192^2 layer's forward and backward), each with its kernel time,
GFLOP/s and HBM fraction or its speedups.

--impl reference times the CPU oracle (decode + compensated SpMV from the
compressed format) on the host cores on a bounded sample of the same workload.
Under torchrun with N > 1 each rank runs an independent replica (the multiply
has no exchange step on one matrix: "replicas only"); value = total flops of
all ranks / max time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
# GB300 FP64 pipe: 152 SMs x 2 DFMA per clock per SM x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = round(152 * 2 * 2 * 2.07e9 / 1e12, 4)
# encoder options per workload (unit_max_nnz, row_order, order_window,
# first_delta); empty = the paper's canonical format (one unit per row,
# absolute first deltas).  The stencil is timed with row-relative first deltas
# (smaller and faster on GB300); the power-law matrix with rows split into
# units of at most 32 entries, ordered by unit length within blocks of 2048
# rows (balanced slices whose near-diagonal x gathers share L1 lines).  The
# canonical-format time is reported beside either.
LAYOUT = {"stencil": {"first_delta": 1}, "pr1": {},
          "powerlaw": {"unit_max_nnz": 32, "row_order": 1, "order_window": 2048}}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return PEAKS_FALLBACK["hbm_gbs"], "fallback"


def make_workload(name: str, grid: int = 128):
    import workloads as WL
    if name == "stencil":
        A = WL.stencil27(grid, seed=1)
        A["label"] = f"stencil27_periodic_{grid}^3_fp64"
    elif name == "powerlaw":
        rows = int(os.environ.get("DTANS_BENCH_PL_ROWS", 4_194_304))
        A = WL.power_law(rows=rows, seed=2)
        A["label"] = f"power_law_{rows}_fp32"
    elif name == "pr1":
        A = WL.pr1(seed=0)
        A["label"] = "pr1_n4096_fp64"
    else:
        raise SystemExit(f"unknown workload {name}")
    return A


# host sources that do not change what a launch reads or writes (handle
# services: upload, save/load, info; the autotuner's driver loop)
_HASH_EXCLUDE = ("handle.cpp", "tune.cpp")


def kernel_hash():
    """Hash of the sources that decide a launch's memory traffic: the
    kernels, their headers and the encoder (the stream layout)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2603_01915_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")) and f not in _HASH_EXCLUDE:
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str):
    """DRAM bytes per launch from a committed ncu capture, if it was taken on
    the current kernel sources (profiles/traffic.json keyed by source hash)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload)
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    return e.get("dram_bytes_per_launch")


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None
        # DTANS_CLOCKS_CSV keeps the raw samples where the caller wants them
        self.path = os.environ.get("DTANS_CLOCKS_CSV") or f"/tmp/dtans_clocks_{os.getpid()}_{gpu_index}.csv"

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [t.strip() for t in line.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_ranks(ms_local: float, flops_local: float, world: int, device=None):
    """Whole-job figure of N replicas: the slowest rank's time and the flops of
    all ranks over it (GFLOP/s).  With world == 1 no collective is used."""
    if world <= 1:
        return ms_local, flops_local / (ms_local * 1e-3) / 1e9
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    f = torch.tensor([flops_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(f, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return ms, float(f.item()) / (ms * 1e-3) / 1e9


def cusparse_baselines(A, reps: int, our_ms: float, our_bytes: int, warm: bool = False):
    """Fastest and smallest of cuSPARSE CSR / COO / SELL on the same matrix
    (L2 flushed before each run, or back to back with warm=True)."""
    import ctypes as C

    import paper_2603_01915_gb300 as D
    try:
        L = C.CDLL(D.build_baseline())
        L.csb_benchmark_mode.restype = C.c_int
        L.csb_last_error.restype = C.c_char_p
        rp = np.ascontiguousarray(A["row_ptr"], np.int32)
        ci = np.ascontiguousarray(A["cols"], np.int32)
        v = np.ascontiguousarray(A["vals"])
        x = np.ascontiguousarray(A["x"].astype(v.dtype))
        ms = (C.c_double * 6)()
        by = (C.c_int64 * 6)()
        rc = L.csb_benchmark_mode(C.c_int64(A["m"]), C.c_int64(A["n"]), C.c_int64(len(ci)),
                                  rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                                  v.ctypes.data_as(C.c_void_p), C.c_int32(1 if v.dtype == np.float64 else 0),
                                  x.ctypes.data_as(C.c_void_p), C.c_int32(reps), C.c_int32(0 if warm else 1), ms, by)
        if rc != 0:
            return {"error": L.csb_last_error().decode()}
        names = ["csr_alg1", "csr_alg2", "coo_alg1", "coo_alg2", "sell32"]
        res = {f"{nm}_ms": (round(ms[i], 5) if ms[i] > 0 else None) for i, nm in enumerate(names)}
        fastest = min((ms[i], nm) for i, nm in enumerate(names) if ms[i] > 0)
        smallest = min(by[i] for i in (0, 2, 4))
        res.update(best=fastest[1], best_ms=round(fastest[0], 5), speedup_vs_best=round(fastest[0] / our_ms, 3),
                   bytes_csr=int(by[0]), bytes_coo=int(by[2]), bytes_sell=int(by[4]),
                   compression_vs_smallest=round(smallest / our_bytes, 3))
        return res
    except Exception as e:  # noqa: BLE001
        return {"error": str(e)[:300]}


def measure_ceilings(reps: int = 3):
    """Secondary ceilings of this GPU from the microbenchmarks beside the
    cuSPARSE baselines: DFMA rate (the FP64 products), IMAD rate (the decoder
    state update) and random / conflict-free shared-memory loads (the table
    lookups), per clock per SM at the device's maximum clock."""
    import ctypes as C

    import paper_2603_01915_gb300 as D
    try:
        L = C.CDLL(D.build_baseline())
        L.dtc_last_error.restype = C.c_char_p
        out = (C.c_double * 10)()
        if L.dtc_ceilings(out, C.c_int(reps)) != 0:
            return {"error": L.dtc_last_error().decode()}
        return {"dfma_tflops": round(out[0], 4), "dfma_per_clk_sm": round(out[1], 3),
                "imad_per_clk_sm": round(out[2], 2), "lds_random_lanes_per_clk_sm": round(out[3], 2),
                "lds_linear_lanes_per_clk_sm": round(out[4], 2), "clock_mhz": round(out[5], 1), "sms": int(out[6]),
                "imad_wide_s32_per_clk_sm": round(out[7], 2), "imad_wide_u32_per_clk_sm": round(out[8], 2),
                "imad_hi_per_clk_sm": round(out[9], 2)}
    except Exception as e:  # noqa: BLE001
        return {"error": str(e)}


def cpu_oracle_baseline(A, steps: int = 1, budget_s: float = 12.0, first_delta: int = 0, chain: int = 1):
    """CPU oracle: decode + compensated SpMV from the compressed format (the
    same first-delta convention as the GPU run), single-threaded, on the first
    2^17 rows (4096 slices) of the workload, repeated until `budget_s` seconds
    of work (at least `steps`)."""
    import oracle as O
    rows = min(A["m"], 1 << 17)
    rp = A["row_ptr"][: rows + 1]
    nnz = int(rp[-1])
    cols, vals = A["cols"][:nnz], A["vals"][:nnz]
    E = O.encode_matrix(rp, cols, vals, A["n"], first_delta=first_delta, chain=chain)
    x = A["x"].astype(np.float64)
    reps, t0 = 0, time.perf_counter()
    times = []
    while reps < steps or (time.perf_counter() - t0 < budget_s and reps < 1000):
        t = time.perf_counter()
        rp2, c2, v2 = O.decode_matrix(E)
        y, _ = O.spmm_ref(rp2, c2, v2.astype(np.float64), x)
        times.append(time.perf_counter() - t)
        reps += 1
    tot = sum(times)
    return {"value": 2.0 * nnz * reps / tot / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"first {rows} rows ({nnz} nnz) of the same matrix, decode + SpMV x{reps}",
            "seconds": round(tot, 3)}, times


def _oracle_block(job):
    """One worker of the all-core CPU baseline: encodes its row block with
    the oracle (untimed), then decodes and multiplies it for `budget_s`
    seconds.  Returns (entries processed, seconds)."""
    rp, cols, vals, n, x, first_delta, chain, budget_s = job
    import oracle as O
    E = O.encode_matrix(rp, cols, vals, n, first_delta=first_delta, chain=chain)
    nnz = int(rp[-1])
    reps, t0 = 0, time.perf_counter()
    while reps < 1 or time.perf_counter() - t0 < budget_s:
        rp2, c2, v2 = O.decode_matrix(E)
        O.spmm_ref(rp2, c2, v2.astype(np.float64), x)
        reps += 1
    return nnz * reps, time.perf_counter() - t0


def cpu_oracle_all_cores(A, budget_s: float = 8.0, first_delta: int = 0, chain: int = 1, workers: int = 0):
    """The oracle as it stands on every host core: the first 2^17 rows cut
    into one block per worker process (spawned, so no process forks after
    CUDA is up), each worker decoding and multiplying its block for
    `budget_s` seconds; the figure is the sum of the workers' rates."""
    import multiprocessing as mp
    P = workers or min(os.cpu_count() or 1, 64)
    rows = min(A["m"], 1 << 17)
    P = max(1, min(P, rows))
    x = A["x"].astype(np.float64)
    jobs = []
    for w in range(P):
        r0, r1 = rows * w // P, rows * (w + 1) // P
        a, b = int(A["row_ptr"][r0]), int(A["row_ptr"][r1])
        rp = (A["row_ptr"][r0:r1 + 1] - a).astype(np.int64)
        jobs.append((rp, A["cols"][a:b], A["vals"][a:b], A["n"], x, first_delta, chain, budget_s))
    with mp.get_context("spawn").Pool(P) as pool:
        res = pool.map(_oracle_block, jobs)
    rate = sum(e / t for e, t in res if t > 0)
    nnz = int(A["row_ptr"][rows])
    return {"value": 2.0 * rate / 1e9, "unit": "GFLOP/s", "cores": P, "kind": "oracle",
            "sample": f"first {rows} rows ({nnz} nnz) of the same matrix in {P} row blocks, one process each, "
                      f"decode + SpMV for {budget_s:g} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    A = make_workload(args.workload, args.grid)
    lay = LAYOUT.get(args.workload, {})
    fd = args.first_delta if args.first_delta is not None else lay.get("first_delta", 0)
    ch = args.chain if args.chain is not None else lay.get("chain", 1)
    res, times = cpu_oracle_baseline(A, steps=args.steps + args.warmup, budget_s=0.0, first_delta=fd, chain=ch)
    times = times[args.warmup:]
    ms = 1e3 * statistics.mean(times) if times else None
    out = {"metric": "fused decode+SpMV GFLOP/s", "value": res["value"], "unit": "GFLOP/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if A["vals"].dtype == np.float64 else "f32",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": A["label"], "sample": res["sample"]},
           "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": res["sample"], "value": res["value"],
                            "unit": "GFLOP/s"},
           "e2e": {"value": res["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def _timed_warm(fn, steps, batch: int = 10):
    """Warm cache: median over `steps` of the CUDA-event time of `batch`
    back-to-back fn() calls divided by `batch` (host launch time stays out of
    the figure, as in the cuSPARSE baseline's warm timing)."""
    import torch
    st = torch.cuda.current_stream()
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(batch):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) / batch)
    return statistics.median(ts)


def _timed(fn, steps, flush, warm):
    """Median of CUDA-event times of fn() on the current stream, L2 flushed before each."""
    import torch
    st = torch.cuda.current_stream()
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        if not warm:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn()
        b.record(st)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def _extra_layout(args):
    # random-column matrices with Poisson row lengths: rows sorted by length
    # (no split) balance the lanes of a slice (measured faster on GB300)
    lay = {"row_order": 1}
    lay.update({k: v for k, v in (("unit_max_nnz", args.unit_max_nnz), ("row_order", args.row_order),
                                  ("order_window", args.order_window), ("first_delta", args.first_delta))
                if v is not None})
    return lay


def measure_batch(args, flush, dev):
    """64 matrices of uneven size in one graph-captured persistent launch
    (configs: batched), against one launch per matrix."""
    import torch

    import paper_2603_01915_gb300 as D
    import workloads as WL
    lay = _extra_layout(args)
    mats = WL.batched(seed=3)
    Ms = [D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), **lay).cuda() for A in mats]
    xs = [torch.from_numpy(A["x"]).to(dev) for A in mats]
    ys = [torch.empty(A["m"], dtype=torch.float64, device=dev) for A in mats]
    nnz = sum(int(A["row_ptr"][-1]) for A in mats)
    B = D.Batch(Ms)
    B.bind(xs, ys)
    B.spmv()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        B.spmv()
    t_graph = _timed(g.replay, args.steps, flush, args.warm)
    t_loop = _timed(lambda: [M.spmv(x, y) for M, x, y in zip(Ms, xs, ys)], args.steps, flush, args.warm)
    for M in Ms:
        M.check()
    comp = sum(M.info.bytes_compressed for M in Ms)
    alg = comp + sum(8 * (A["m"] + A["n"]) for A in mats)
    peak = load_peaks()[0]
    res = {"workload": "batched_64_matrices_fp64", "matrices": len(mats), "nnz": nnz, "layout": lay,
           "one_launch_graph_ms": round(t_graph, 5), "per_matrix_launches_ms": round(t_loop, 5),
           "speedup_vs_launch_loop": round(t_loop / t_graph, 3),
           "gflops": round(2.0 * nnz / (t_graph * 1e-3) / 1e9, 2),
           "hbm": {"achieved": round(alg / (t_graph * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                   "frac": round(alg / (t_graph * 1e-3) / 1e9 / peak, 4), "algorithmic_bytes": int(alg)}}
    B.close()
    for M in Ms:
        M.close()
    return res, mats


def measure_multirhs(args, flush, dev):
    """One 2^20-row matrix of the batched kind with k = 1, 4, 8, 16
    right-hand sides, against the single-vector kernel (dtans_spmv) on the
    same matrix."""
    import torch

    import paper_2603_01915_gb300 as D
    import workloads as WL
    lay = _extra_layout(args)
    res = {}
    A = WL.multi_rhs(seed=3, k=16)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), **lay).cuda()
    nnz = int(A["row_ptr"][-1])
    x1 = torch.from_numpy(np.ascontiguousarray(A["X"][:, 0])).to(dev)
    y1 = torch.empty(A["m"], dtype=torch.float64, device=dev)
    t1 = _timed(lambda: M.spmv(x1, y1), args.steps, flush, args.warm)
    res["k1_spmv_ms"] = round(t1, 5)
    for k in (1, 4, 8, 16):
        X = torch.from_numpy(np.ascontiguousarray(A["X"][:, :k])).to(dev)
        Y = torch.empty((A["m"], k), dtype=torch.float64, device=dev)
        tk = _timed(lambda: M.spmm(X, Y), args.steps, flush, args.warm)
        if k >= 16:  # column-tile policy by measurement: 8-column passes or one 16-column pass
            M.set_tile_policy(1)
            tk1 = _timed(lambda: M.spmm(X, Y), args.steps, flush, args.warm)
            res[f"k{k}_ms_tiles8"], res[f"k{k}_ms_tiles16"] = round(tk, 5), round(tk1, 5)
            if tk1 < tk:
                tk = tk1
            else:
                M.set_tile_policy(0)
        res[f"k{k}_ms"] = round(tk, 5)
        res[f"k{k}_per_vector_speedup_vs_spmv"] = round(k * t1 / tk, 3)
    M.check()
    M.close()
    res.update(workload="multi_rhs_2^20_fp64", nnz=nnz, layout=lay,
               gflops_k8=round(2.0 * nnz * 8 / (res["k8_ms"] * 1e-3) / 1e9, 2))
    return res


def measure_pruned(args, flush, dev):
    """The pruned 8192 x 8192 FP32 layer with a batch of 32: forward,
    x_grad by atomics and by the transposed stream, value and codebook
    gradients."""
    import torch

    import paper_2603_01915_gb300 as D
    import workloads as WL
    A = WL.pruned_linear(seed=4)
    M, tuned, _ = D.tune(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), k=A["X"].shape[1], reps=3)
    lay = dict(unit_max_nnz=M.info.unit_max_nnz, row_order=M.info.row_order, order_window=M.info.order_window)
    rpt, ct, vt_ = D.transpose_csr(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]))
    MT = D.Matrix(rpt, ct, vt_, (A["n"], A["m"]), **lay).cuda()
    nnz = int(A["row_ptr"][-1])
    X = torch.from_numpy(A["X"]).to(dev)
    G = torch.from_numpy(A["G"]).to(dev)
    Y = torch.empty((A["m"], X.shape[1]), dtype=torch.float32, device=dev)
    XG = torch.empty((A["n"], X.shape[1]), dtype=torch.float32, device=dev)
    VG = torch.empty(nnz, dtype=torch.float32, device=dev)
    tf = _timed(lambda: M.spmm(X, Y), args.steps, flush, args.warm)
    tb_atomic = _timed(lambda: M.spmv_T(G, XG), args.steps, flush, args.warm)
    M.set_scatter(1)
    tb_agg = _timed(lambda: M.spmv_T(G, XG), args.steps, flush, args.warm)
    M.set_scatter(0)
    tb_stream = _timed(lambda: MT.spmm(G, XG), args.steps, flush, args.warm)
    tv = _timed(lambda: M.vals_grad(G, X, VG), args.steps, flush, args.warm)
    CB = torch.empty(int(M.info.kept_value) + 1, dtype=torch.float32, device=dev)
    tc = _timed(lambda: M.codebook_grad(G, X, CB), args.steps, flush, args.warm)
    M.check()
    MT.check()
    k = X.shape[1]
    res = {"workload": "pruned_linear_8192_fp32_batch32", "nnz": nnz, "forward_ms": round(tf, 5),
           "forward_gflops": round(2.0 * nnz * k / (tf * 1e-3) / 1e9, 2),
           "backward_xgrad_atomic_ms": round(tb_atomic, 5),
           "backward_xgrad_warp_aggregated_ms": round(tb_agg, 5),
           "backward_xgrad_transposed_stream_ms": round(tb_stream, 5),
           "vals_grad_ms": round(tv, 5), "codebook_grad_ms": round(tc, 5),
           "codebook_size": int(M.info.kept_value),
           "xgrad_choice": min((("atomics", tb_atomic), ("warp-aggregated atomics", tb_agg),
                                ("transposed stream", tb_stream)), key=lambda t: t[1])[0],
           "layout": lay, "tuned": tuned}
    M.close()
    MT.close()
    return res


def measure_single(name, args, flush, dev):
    """One decode-fused SpMV of the PR1 or power-law workload (cold L2,
    median of the steps) with its HBM roofline fraction and the fastest
    cuSPARSE format on the same matrix."""
    import torch

    import paper_2603_01915_gb300 as D
    A = make_workload(name)
    m, n, nnz = A["m"], A["n"], int(A["row_ptr"][-1])
    vt = A["vals"].dtype
    V = 8 if vt == np.float64 else 4
    lay = dict(LAYOUT.get(name, {}))
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (m, n), **lay).cuda()
    x = torch.from_numpy(A["x"].astype(vt)).to(dev)
    y = torch.empty(m, dtype=torch.float64 if vt == np.float64 else torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    t = _timed(lambda: D.dtans_spmv(M.h, x, y, 0.0, stream), max(args.steps, 7), flush, args.warm)
    M.check()
    inf = M.info
    alg = inf.bytes_words + inf.bytes_slice_off + inf.bytes_tables + inf.bytes_unit_meta + n * V + m * V
    peak = load_peaks()[0]
    res = {"workload": A["label"], "nnz": nnz, "layout": lay, "warps_per_cta": inf.warps or 24,
           "kernel_ms_median": round(t, 5), "gflops": round(2.0 * nnz / (t * 1e-3) / 1e9, 2),
           "bits_per_nnz": round(32.0 * inf.nwords / max(nnz, 1), 3),
           "hbm": {"achieved": round(alg / (t * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                   "frac": round(alg / (t * 1e-3) / 1e9 / peak, 4), "algorithmic_bytes": int(alg)}}
    if name == "powerlaw":  # x_grad = A^T g over the same stream: one atomic per entry, or warp-aggregated
        g = torch.from_numpy(A["x"][:m].astype(vt)).to(dev)
        xg = torch.empty(n, dtype=y.dtype, device=dev)
        res["spmv_T_atomic_ms"] = round(_timed(lambda: M.spmv_T(g, xg), max(args.steps // 2, 5), flush, args.warm), 5)
        M.set_scatter(1)
        res["spmv_T_warp_aggregated_ms"] = round(_timed(lambda: M.spmv_T(g, xg), max(args.steps // 2, 5), flush,
                                                        args.warm), 5)
        M.set_scatter(0)
        M.check()
    if not args.no_cusparse:
        cus = cusparse_baselines(A, max(5, args.steps // 2), t, inf.bytes_compressed)
        res["cusparse"] = {k: cus.get(k) for k in ("best", "best_ms", "speedup_vs_best", "compression_vs_smallest",
                                                    "csr_alg1_ms", "sell32_ms", "error") if k in cus}
    M.close()
    del A
    return res


def run_extra(args):
    """Reporting modes for the batched, multi-RHS and pruned-linear workloads
    (one JSON line each; the default stencil line is the headline)."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda")
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(2 * l2 // 4 + 1024, dtype=torch.int32, device=dev)
    out = {"metric": "fused decode+SpMV GFLOP/s", "unit": "GFLOP/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "data": "synthetic"}
    if args.workload == "batch":
        res, _ = measure_batch(args, flush, dev)
        out.update(value=res["gflops"], ms_per_step=res["one_launch_graph_ms"], dtype="f64", config=res,
                   roofline=dict(bound="hbm", **res["hbm"]), gpu_launches=1)
    elif args.workload == "multirhs":
        res = measure_multirhs(args, flush, dev)
        out.update(value=res["gflops_k8"], ms_per_step=res["k8_ms"], dtype="f64", config=res, gpu_launches=1)
    else:
        res = measure_pruned(args, flush, dev)
        out.update(value=res["forward_gflops"], ms_per_step=res["forward_ms"], dtype="f32", config=res,
                   gpu_launches=1)
    print(json.dumps(out), flush=True)
    return 0


def other_configs(args, flush, dev):
    """The other workloads beside the headline stencil: PR1 (n = 4096), the
    power-law matrix, the 64-matrix batch, k right-hand sides and the pruned
    layer; each failure is reported in place of its figures."""
    out = {}
    for key, fn in (("pr1_n4096_fp64", lambda: measure_single("pr1", args, flush, dev)),
                    ("power_law_4M_fp32", lambda: measure_single("powerlaw", args, flush, dev)),
                    ("batched_64_fp64", lambda: measure_batch(args, flush, dev)[0]),
                    ("multi_rhs_2^20_fp64", lambda: measure_multirhs(args, flush, dev)),
                    ("pruned_linear_8192_fp32", lambda: measure_pruned(args, flush, dev))):
        t0 = time.perf_counter()
        try:
            out[key] = fn()
        except Exception as e:  # noqa: BLE001
            out[key] = {"error": str(e)[:300]}
        out[key]["wall_s"] = round(time.perf_counter() - t0, 1)
        log(f"other config {key}: {out[key].get('wall_s')} s")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="stencil",
                    choices=["stencil", "powerlaw", "pr1", "batch", "multirhs", "pruned"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cusparse", action="store_true")
    ap.add_argument("--warm", action="store_true", help="do not flush L2 between steps")
    ap.add_argument("--grid", type=int, default=128, help="stencil grid edge (128 = the benchmark workload)")
    ap.add_argument("--unit-max-nnz", type=int, default=None, help="split rows longer than U into units (0 = off)")
    ap.add_argument("--row-order", type=int, default=None, help="1 = order rows by unit length")
    ap.add_argument("--order-window", type=int, default=None,
                    help="with --row-order 1: order within blocks of this many rows (0 = all rows)")
    ap.add_argument("--warps", type=int, default=0,
                    help="warps per CTA of the single-vector kernel (20/24/28/32; 0 = measure and pick)")
    ap.add_argument("--chain", type=int, default=None,
                    help="slices per chain of units (1 = the paper's one sequence per unit)")
    ap.add_argument("--first-delta", type=int, default=None,
                    help="0 = absolute first deltas (the paper's format), 1 = relative to the row")
    ap.add_argument("--tune", action="store_true", help="choose the layout with the autotuner (dtans_tune)")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="time only the headline workload (skip PR1, power-law, batch, k-RHS, pruned)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batch", "multirhs", "pruned"):
        return run_extra(args)

    import torch
    import torch.distributed as dist

    import paper_2603_01915_gb300 as D

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    A = make_workload(args.workload, args.grid)
    m, n, nnz = A["m"], A["n"], int(A["row_ptr"][-1])
    vt = A["vals"].dtype
    tdt = torch.float64 if vt == np.float64 else torch.float32
    V = 8 if vt == np.float64 else 4
    layout = dict(LAYOUT.get(args.workload, {}))
    if args.unit_max_nnz is not None:
        layout["unit_max_nnz"] = args.unit_max_nnz
    if args.row_order is not None:
        layout["row_order"] = args.row_order
    if args.order_window is not None:
        layout["order_window"] = args.order_window
    if args.first_delta is not None:
        layout["first_delta"] = args.first_delta
    if args.chain is not None:
        layout["chain"] = args.chain
    t0 = time.perf_counter()
    tune_report = None
    if args.tune:
        M, tune_report, _ = D.tune(A["row_ptr"], A["cols"], A["vals"], (m, n), reps=3, first_delta=2)
    else:
        M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (m, n), **layout)
    enc_s = time.perf_counter() - t0
    M.cuda()
    # launch shape by measurement: warps per CTA of the single-vector kernel
    warps_ms = None
    if args.warps:
        M.set_warps(args.warps)
    elif not args.tune:
        _, warps_ms = M.tune_warps(reps=5)
    inf = M.info
    x_host = torch.from_numpy(A["x"].astype(vt)).pin_memory()
    x = x_host.to(dev)
    y = torch.empty(m, dtype=tdt, device=dev)
    stream = torch.cuda.current_stream()
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(2 * l2 // 4 + 1024, dtype=torch.int32, device=dev)

    def step():
        D.dtans_spmv(M.h, x, y, 0.0, stream)

    # warm-up (correctness of the first result is covered by the tests)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    M.check()

    clocks = Clocks(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        if not args.warm:
            flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    times = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(times)
    ms_med = statistics.median(times)
    ms, value = aggregate_ranks(ms, 2.0 * nnz, world, dev)

    # roofline of the kernel: algorithmic bytes = compressed stream + slice
    # offsets + tables (once) + unit-to-row map (layouts with split or
    # reordered rows) + x (read once) + y (written once)
    alg_bytes = inf.bytes_words + inf.bytes_slice_off + inf.bytes_tables + inf.bytes_unit_meta + n * V + m * V
    # DRAM traffic records are per matrix and encoding
    traffic_key = f'{A["label"]}/U{inf.unit_max_nnz}_order{inf.row_order}_first{inf.first_delta}' + \
        (f"_chain{inf.chain_slices}" if inf.chain_slices > 1 else "") + \
        (f"_window{inf.order_window}" if inf.row_order == 1 and inf.order_window > 0 else "")
    peak, peak_src = load_peaks()
    gbs = alg_bytes / (ms_med * 1e-3) / 1e9
    hbm = {"achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
           "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
           "algorithmic_bytes": int(alg_bytes)}
    if vt == np.float64 and not inf.int_products:
        # One DFMA per nonzero: GB300's FP64 pipe, not HBM, bounds the FP64 path.
        tflops = 2.0 * nnz / (ms_med * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": round(tflops, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": round(tflops / FP64_PEAK_TFLOPS, 4), "traffic": recorded_traffic(traffic_key),
                "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived)",
                "kernel_ms_median": round(ms_med, 5), "hbm": hbm}
    else:
        # FP32, or FP64 on the integer-coefficient kernels (no FP64 operation
        # per entry): the HBM roofline
        roof = dict(bound="hbm", traffic=recorded_traffic(traffic_key), kernel_ms_median=round(ms_med, 5), **hbm)
        if vt == np.float64:
            roof["fp64_pipe_note"] = ("integer-coefficient products: three integer multiply-adds per entry, "
                                      "FP64 operations only per row; the FMA form is bound by the FP64 pipe at "
                                      f"{FP64_PEAK_TFLOPS} TFLOP/s")
    fp64 = None

    # end-to-end through the C ABI with host buffers: every step is one
    # dtans_spmv_host call, which copies its x in from pinned host memory,
    # multiplies and copies y back out (one cudaMemcpyAsync each way, on the
    # handle's own streams, three device buffer sets used in turn, so the
    # neighbouring steps' copies overlap a step's product).  No L2 flush: a step
    # streams the compressed matrix plus x in and y out.
    # at least 50 pipelined steps: the first copy in and the last copy out are
    # not overlapped, and over 20 steps they add about 9 us to each
    ne = max(50, args.steps)
    xs_host = [torch.from_numpy(A["x"].astype(vt) * (1.0 + 0.25 * (i % 4))).pin_memory() for i in range(4)]
    ys_host = [torch.empty(m, dtype=tdt).pin_memory() for _ in range(2)]
    for i in range(4):  # warm-up (creates the handle's host-I/O buffers and streams)
        D.dtans_spmv_host(M.h, D._host_ptr(xs_host[i % 4]), D._host_ptr(ys_host[i % 2]), 0.0, stream)
    torch.cuda.synchronize()
    # host wall clock from an idle device to the last y in host memory (the
    # call's copies do not wait for the stream, so a start event on it could
    # miss the first copy in)
    t_e0 = time.perf_counter()
    for i in range(ne):
        D.dtans_spmv_host(M.h, D._host_ptr(xs_host[i % 4]), D._host_ptr(ys_host[i % 2]), 0.0, stream)
    stream.synchronize()
    e2e_ms = (time.perf_counter() - t_e0) * 1e3 / ne
    M.check()
    # the same steps one at a time (each call synchronized before the next)
    seq = []
    for i in range(4):
        t_a = time.perf_counter()
        D.dtans_spmv_host(M.h, D._host_ptr(xs_host[i % 4]), D._host_ptr(ys_host[0]), 0.0, stream)
        stream.synchronize()
        seq.append(time.perf_counter() - t_a)
    seq_ms = 1e3 * statistics.mean(seq)
    # the link alone: one copy of x in and one of y out (pinned, CUDA events),
    # the other two bounds of a pipelined step
    xd_tmp = torch.empty(n, dtype=tdt, device=dev)
    link = {}
    for name, cp in (("copy_in_ms", lambda: xd_tmp.copy_(xs_host[0], non_blocking=True)),
                     ("copy_out_ms", lambda: ys_host[0].copy_(y, non_blocking=True))):
        ts = []
        with torch.cuda.stream(stream):
            for _ in range(5):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                cp()
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
        link[name] = round(statistics.median(ts[1:]), 4)
    del xd_tmp
    e2e = {"value": round(world * 2.0 * nnz / (e2e_ms * 1e-3) / 1e9, 2), "unit": "GFLOP/s",
           "h2d_bytes_per_step": n * V, "d2h_bytes_per_step": m * V, "ms_per_step": round(e2e_ms, 4),
           "steps": ne, "api": "dtans_spmv_host (C ABI; pinned host x and y; copies overlap neighbouring products)",
           "timer": "host wall clock, idle device to the last y in host memory",
           "l2": "not flushed; each step streams the compressed matrix, x in and y out",
           "one_call_at_a_time_ms": round(seq_ms, 4), **link}

    # cuSPARSE baselines on the same GPU: CSR (alg 1, 2), COO (alg 1, 2) and
    # SELL-32, each after an L2 flush (median of the steps)
    cus = None
    if not args.no_cusparse:
        cus = cusparse_baselines(A, max(5, args.steps // 2), ms_med, inf.bytes_compressed)
        # warm cache (no flush between runs; batches of back-to-back calls), both sides
        ms_warm = _timed_warm(step, max(5, args.steps // 2))
        cw = cusparse_baselines(A, max(5, args.steps // 2), ms_warm, inf.bytes_compressed, warm=True)
        cus["warm"] = {"ours_ms": round(ms_warm, 5), "best": cw.get("best"), "best_ms": cw.get("best_ms"),
                       "speedup_vs_best": cw.get("speedup_vs_best")}

    # the paper's canonical format (absolute first deltas, one unit per row)
    # on the same matrix, when the timed layout differs from it
    canonical = None
    if not args.tune and any(layout.get(k, 0) for k in ("unit_max_nnz", "row_order", "first_delta")) or \
            layout.get("chain", 1) > 1:
        Mc = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (m, n)).cuda()
        ms_c = _timed(lambda: D.dtans_spmv(Mc.h, x, y, 0.0, stream), max(args.steps, 5), flush, args.warm)
        Mc.check()
        canonical = {"kernel_ms_median": round(ms_c, 5), "gflops": round(2.0 * nnz / (ms_c * 1e-3) / 1e9, 2),
                     "bits_per_nnz": round(32.0 * Mc.info.nwords / max(nnz, 1), 3),
                     "compressed_bytes": Mc.info.bytes_compressed}
        Mc.close()

    # the same product with exact integer-coefficient sums (dtans_set_accumulate
    # mode 1), when the value table has integer coefficients: reported beside
    # the FMA kernel, not timed as the headline
    int_form = None
    if vt == np.float64 and inf.int_coefficients and not inf.int_products:
        M.set_accumulate(1)
        ms_i = _timed(step, max(args.steps, 5), flush, args.warm)
        M.check()
        M.set_accumulate(0)
        int_form = {"kernel_ms_median": round(ms_i, 5), "gflops": round(2.0 * nnz / (ms_i * 1e-3) / 1e9, 2),
                    "includes": "fixed-point conversion of x (two small kernels) and the decode-fused product"}

    # secondary ceilings (FP64 pipe, integer issue, shared-memory lookups) of this GPU
    ceil = measure_ceilings() if (rank == 0 and not args.no_cusparse) else None

    others = None
    if rank == 0 and world == 1 and not args.no_other_configs and args.workload == "stencil":
        others = other_configs(args, flush, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # all host cores (the baseline figure) and one core beside it
        one, _ = cpu_oracle_baseline(A, budget_s=6.0, first_delta=inf.first_delta, chain=inf.chain_slices)
        try:
            cpu = cpu_oracle_all_cores(A, budget_s=6.0, first_delta=inf.first_delta, chain=inf.chain_slices)
            cpu["single_core"] = one
        except Exception as e:  # noqa: BLE001
            cpu = dict(one, all_cores_error=str(e))

    if rank == 0:
        out = {"metric": "fused decode+SpMV GFLOP/s", "value": round(value, 2), "unit": "GFLOP/s",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 5),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64" if vt == np.float64 else "f32", "data": "synthetic",
               "config": {"workload": A["label"], "m": m, "n": n, "nnz": nnz,
                          "l2": "warm" if args.warm else "flushed between steps (2 x L2 buffer written)",
                          "compressed_bytes": inf.bytes_compressed, "words": inf.nwords,
                          "bits_per_nnz": round(32.0 * inf.nwords / max(nnz, 1), 3),
                          "encode_s": round(enc_s, 2), "parallelism": f"replicas x{world}",
                          "layout": {"unit_max_nnz": inf.unit_max_nnz, "row_order": inf.row_order,
                                     "order_window": inf.order_window,
                                     "first_delta": inf.first_delta, "chain_slices": inf.chain_slices,
                                     "units": inf.nunits, "tuned": tune_report},
                          "warps_per_cta": inf.warps,
                          "accumulate": ("integer coefficients (exact fixed-point sums, one rounding per row)"
                                         if inf.int_products else "FP64 fused multiply-adds" if vt == np.float64
                                         else "FP32 fused multiply-adds"),
                          "warps_ms": {str(k): round(v, 5) for k, v in warps_ms.items()} if warps_ms else None,
                          "canonical_format": canonical, "integer_coefficient_form": int_form},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "cusparse": cus, "ceilings": ceil,
               "clocks": ck, "gpu_launches": args.steps, "wall_s_timed_region": round(wall, 4),
               "other_configs": others}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
