#!/usr/bin/env python
"""RgCSR SpMV benchmark on GB300.

One step = one RgCSR SpMV of each of the three large synthetic matrices in
FP32 and in FP64 (six SpMVs), each in the configuration (group size,
kernel, row order, long-row segment schedule) the autotuner picked on
this GPU:
  (a) 3D 7-point Laplacian 128^3        n = 2,097,152  nnz = 14,581,760
  (b) power-law rows, n = 10^6          nnz ~ 15.6M, longest row 10,000
  (c) 27-point stencil 96^3, U[-1,1]    n = 884,736    nnz = 23,393,656
value = algorithmic bytes of the six SpMVs (values + columns of the
non-zeros, row lengths, group pointers at G = 32, x once, y once; padding
and the segment lists excluded, so the count does not depend on the
configuration) per second, whole job.  Inputs stay resident in HBM; each step streams
~1.3 GB of algorithmic data (more with padding), far more than the 129 MB
L2, so no SpMV finds its matrix in L2.

Also reported: per-case GB/s and GFLOP/s (2 nnz / t), the HYB comparator
on the same cases, the roofline of the dominant kernel against the
measured HBM copy bandwidth, an end-to-end figure through the host entry
point (x copied in, y copied out each step), and the CPU oracle as a
baseline on a bounded sample.

--impl reference runs the CPU oracle (plain FP64 CSR SpMV) on the same six
cases per step, on all host cores (row blocks in a thread pool).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1012_2270_gb300 import synth  # noqa: E402
from paper_1012_2270_gb300 import roofline  # noqa: E402

METRIC = "RgCSR SpMV GB/s (% of 8 TB/s HBM), GFLOP/s; batched/BF16/bwd vs plain"
UNIT = "GB/s"
GROUP = 32
CASES = [("a", synth.workload_a), ("b", synth.workload_b), ("c", synth.workload_c)]
DTYPES = ["f32", "f64"]
VB = {"f32": 4, "f64": 8}
NP = {"f32": np.float32, "f64": np.float64}
WORKLOAD_SHORT = ("RgCSR SpMV, FP32+FP64, tuned config: (a) 7-point 128^3, (b) power-law rows n=1e6 "
                  "(Zipf(2) lengths <= 10,000), (c) 27-point 96^3")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--cpu-seconds", type=float, default=10.0,
                   help="CPU work of the oracle baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip HYB and the other forms")
    p.add_argument("--forms", default="", help="comma-separated subset of the forms to run (default: all)")
    p.add_argument("--no-ir-sweep", action="store_true",
                   help="skip the inner-tolerance sweep of the IR-CG form (shorter profiling runs)")
    p.add_argument("--cases", default="",
                   help="comma-separated subset of the six cases (a_f32, ..., c_f64) for profiling runs; "
                        "the default runs all six (the step the metric is defined on)")
    p.add_argument("--detail-out", default=None,
                   help="write the full record (per-case detail, forms) to this JSON file; "
                        "default: print it on one line starting with 'detail: ' before the headline")
    p.add_argument("--tune-cache", default=None,
                   help="JSON file for the tuned configurations: read if present, else written "
                        "(lets a profiled run use the configurations of an unprofiled one)")
    return p.parse_args()


def rank_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of per-rank timings over the process group (the
    job takes as long as its slowest replica); the values themselves when
    there is no group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_gbs(world, steps, step_bytes, ms):
    """Every replica streams step_bytes per step: GB/s of the whole job."""
    return world * steps * step_bytes / (ms * 1e-3) / 1e9


def load_cases():
    mats = []
    for name, fn in CASES:
        A = fn()
        x = synth.uniform_vector(A.n_cols, seed=0)
        mats.append((name, A, x))
    return mats


def case_bytes(A, n_groups, dtype):
    return roofline.rgcsr_spmv_bytes(A.n_rows, A.n_cols, A.nnz, n_groups, VB[dtype])


def kernel_name(cfg, M, A, dt):
    """The kernel that a configuration runs (the library's dispatch rules)."""
    t = "float" if dt == "f32" else "double"
    if "tiles" in cfg:
        pipe = len(cfg["tiles"]) > 1 and cfg["tiles"][1] in (3, 4, 5)
        return f"rgcsr_spmv_tiles{'_pipe' if pipe else ''}_kernel<{t}>"
    if "long_rows" in cfg:
        return f"rgcsr_spmv_split+segments<{t}>"
    k, v = cfg.get("kernel", 0), cfg.get("variant", 0)
    if k == 0:
        k, v = M.auto_kernel()                  # the library's own rule
    if k == 4 and v in (1, 2, 4, 8, 9):
        return f"rgcsr_spmv_vec<{t}>"
    if k == 4 and v in (5, 6, 7):
        return f"rgcsr_spmv_vecp<{t}>"
    if k == 3 and v >= 4:
        return f"rgcsr_spmv_tma_multi<{t}>"
    return {1: "rgcsr_spmv_paper", 2: "rgcsr_spmv_split", 3: "rgcsr_spmv_tma", 4: "rgcsr_spmv_lean"}[k] + f"<{t}>"


def measured_traffic(kernel, cases):
    """DRAM bytes per launch of `kernel` (mean over the cases that ran it)
    from the committed ncu summary (case -> kernel -> bytes), or None if a
    case has no entry for that kernel or the kernel's source changed since
    the capture."""
    import hashlib
    try:
        table = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        return None
    vals = []
    for c in cases:
        if c["kernel"] != kernel:
            continue
        e = (table.get(c["key"]) or {}).get(kernel)
        if not e:
            return None
        try:
            sha = hashlib.sha1(open(os.path.join(ROOT, e["source"]), "rb").read()).hexdigest()
        except OSError:
            return None
        if sha != e.get("source_sha1"):
            return None
        vals.append(float(e["dram_bytes_per_launch"]))
    return sum(vals) / len(vals) if vals else None


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def oracle_case_inputs(mats):
    out = []
    for name, A, x in mats:
        for dt in DTYPES:
            val = A.val.astype(NP[dt]).astype(np.float64)
            xv = x.astype(NP[dt]).astype(np.float64)
            ng = (A.n_rows + GROUP - 1) // GROUP
            out.append((f"{name}_{dt}", A, val, xv, case_bytes(A, ng, dt)))
    return out


def row_slice(A, val, lo, hi):
    p0, p1 = A.rowptr[lo], A.rowptr[hi]
    return A.rowptr[lo:hi + 1] - p0, A.col[p0:p1], val[p0:p1]


def oracle_threads():
    return max(1, os.cpu_count() or 1)


def oracle_blocks(cases, parts):
    """Each case's rows cut into `parts` contiguous CSR blocks, so that the
    oracle (unchanged, one row at a time) runs on all host cores: the C loop
    is called through ctypes, which releases the interpreter lock."""
    out = []
    for key, A, val, xv, b in cases:
        edges = np.linspace(0, A.n_rows, parts + 1).astype(np.int64)
        out.append((key, [row_slice(A, val, int(edges[i]), int(edges[i + 1])) for i in range(parts)], xv, b))
    return out


def oracle_pass(pool, blocks):
    """One pass of the six SpMVs over all blocks; returns the bytes moved."""
    import oracle
    futs, nb = [], 0
    for _, parts, xv, b in blocks:
        futs += [pool.submit(oracle.csr_spmv, rp, col, v, xv) for rp, col, v in parts]
        nb += b
    for f in futs:
        f.result()
    return nb


def cpu_baseline(mats, seconds):
    """The oracle as it stands on all host cores (row blocks in a thread
    pool), repeated over the six cases for about `seconds`; GB/s of
    algorithmic bytes."""
    from concurrent.futures import ThreadPoolExecutor
    threads = oracle_threads()
    blocks = oracle_blocks(oracle_case_inputs(mats), 4 * threads)
    with ThreadPoolExecutor(threads) as pool:
        oracle_pass(pool, blocks)
        t0 = time.perf_counter()
        nbytes, passes = 0, 0
        while time.perf_counter() - t0 < seconds or passes == 0:
            nbytes += oracle_pass(pool, blocks)
            passes += 1
        t = time.perf_counter() - t0
    # the same loop on one thread, one pass
    with ThreadPoolExecutor(1) as pool1:
        t1 = time.perf_counter()
        nb1 = oracle_pass(pool1, blocks)
        t1 = time.perf_counter() - t1
    return {"value": nbytes / t / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{passes} pass(es) of the six SpMVs (FP64 CSR loop), {t:.1f} s on {threads} threads",
            "single_thread_gbs": nb1 / t1 / 1e9}


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return 0
    from concurrent.futures import ThreadPoolExecutor
    mats = load_cases()
    threads = oracle_threads()
    blocks = oracle_blocks(oracle_case_inputs(mats), 4 * threads)
    with ThreadPoolExecutor(threads) as pool:
        for _ in range(args.warmup):
            oracle_pass(pool, blocks)
        t0 = time.perf_counter()
        nb = 0.0
        for _ in range(args.steps):
            nb += oracle_pass(pool, blocks)
        t = time.perf_counter() - t0
    value = nb / t / 1e9
    sample = f"every step: the six full SpMVs, FP64 CSR oracle on {threads} host threads (row blocks)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_SHORT, "l2": "inputs larger than L2 (~1.3 GB per step)",
                   "timing": "host wall clock of K steps of the CPU oracle",
                   "parallelism": f"replicas x{world}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        ident = vis.split(",")[local_rank] if vis else str(local_rank)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", ident, "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [s.strip() for s in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CUDA-graph timing
# ---------------------------------------------------------------------------
COPIES = 3        # rotating copies of each case's matrix, x and y for the per-case graphs
ROUNDS = 8        # passes over the copies in one per-case graph (COPIES * ROUNDS launches)
REPLAYS = 15      # timed replays of each per-case graph (median taken)


def capture_graph(fns):
    """A CUDA graph of fns called in order (each enqueues its kernels on the
    current stream).  The calls run once eagerly on the capture stream
    first, so one-off set-up (kernel attributes) happens outside capture."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for f in fns:
            f()
    side.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        for f in fns:
            f()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    return g


def capture_graph_branches(fns):
    """A CUDA graph in which each of fns is its own branch (forked from one
    node, joined into one), so independent calls may run concurrently.  Each
    call runs on its own stream, once eagerly first, as in capture_graph."""
    import torch
    main = torch.cuda.Stream()
    main.wait_stream(torch.cuda.current_stream())
    sides = [torch.cuda.Stream() for _ in fns]
    for st, f in zip(sides, fns):
        st.wait_stream(main)
        with torch.cuda.stream(st):
            f()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=main):
        fork = torch.cuda.Event()
        fork.record(main)
        for st, f in zip(sides, fns):
            st.wait_event(fork)
            with torch.cuda.stream(st):
                f()
            join = torch.cuda.Event()
            join.record(st)
            main.wait_event(join)
    torch.cuda.current_stream().wait_stream(main)
    torch.cuda.synchronize()
    return g


def replay_us(g, replays, stream):
    """Microseconds of each of `replays` back-to-back replays of graph g,
    one event pair per replay on the launching stream."""
    import torch
    g.replay()
    torch.cuda.synchronize()
    ev = [_ev() for _ in range(replays)]
    for e0, e1 in ev:
        e0.record(stream)
        g.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    return [1e3 * e0.elapsed_time(e1) for e0, e1 in ev]


def rotating_us(fns, stream, rounds=ROUNDS, replays=REPLAYS):
    """Microseconds per call of one operation whose copies (fns: one call
    per copy, each on its own data) are called in turn, `rounds` times, in
    one CUDA graph: consecutive calls touch different data, so with three
    copies of >= 100 MB L2 holds none of a call's inputs when it starts;
    the graph removes host launch gaps.  Median over replays."""
    g = capture_graph([f for _ in range(rounds) for f in fns])
    t = statistics.median(replay_us(g, replays, stream))
    del g
    return t / (rounds * len(fns))


# ---------------------------------------------------------------------------
# the JSON line
# ---------------------------------------------------------------------------
def _r(v, digits=4):
    """Floats rounded to `digits` significant digits, recursively (keeps
    the headline line short)."""
    if isinstance(v, float):
        return float(f"{v:.{digits}g}") if v == v and v not in (float("inf"), float("-inf")) else None
    if isinstance(v, dict):
        return {k: _r(x, digits) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [_r(x, digits) for x in v]
    return v


HEADLINE_MAX_BYTES = 2048


def headline(*, value, world, steps, warmup, ms_per_step, gflops, launches, clocks, roof, e2e, cpu,
             cases, forms_summary, detail_file):
    """The one JSON line that ends the run: the metric, the roofline of the
    dominant kernel, the end-to-end and CPU figures, per-case times and a
    few numbers of the other forms.  Everything else goes to the detail
    record, so that this line stays under HEADLINE_MAX_BYTES."""
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32,f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_SHORT, "l2": "inputs larger than L2 (~1.3 GB per step)",
                   "timing": "graphs: the step (six branches) x K; per case 3 rotating copies",
                   "parallelism": f"replicas x{world}"},
        "gflops": gflops, "pct_of_8tbs": 100 * value / world / roofline.NOMINAL_HBM_GBS,
        "gpu_launches": launches, "clocks": clocks, "roofline": roof, "e2e": e2e,
        "cpu_baseline": cpu, "cases": cases, "forms": forms_summary, "detail": detail_file,
    }
    return _r(line)


def forms_summary(forms):
    """A few numbers of the other forms for the headline (the full tables
    are in the detail record)."""
    s = {}
    q = forms.get("quantized") or {}
    if "a_bf16" in q:
        s["bf16_a_vs_f32"] = q["a_bf16"]["speedup_vs_f32"]
        s["bf16_a_err"] = q["a_bf16"]["max_err_over_absAx_vs_f64"]
    bt = forms.get("batched_512_f32")
    if bt:
        s["batched_gbs"] = bt["gbs"]
        s["batched_vs_512_launches"] = bt["speedup_vs_plain"]
    bw = forms.get("backward_b_k8_f32")
    if bw:
        s["bwd_over_fwd"] = bw["backward_over_forward"]
    h = forms.get("hyb")
    if h:
        s["rgcsr_over_hyb"] = {k: v["rgcsr_speedup"] for k, v in h.items() if k.startswith("b")}
    ic = forms.get("ir_cg_poisson128")
    if ic:
        s["ir_cg_vs_fp64_cg"] = ic["fp64_cg_ms"] / ic["ms"]
        ok = [v for v in (ic.get("inner_tol_sweep") or {}).values() if v["final_rel_residual"] <= 1e-10]
        if ok:
            s["ir_cg_best_vs_fp64_cg"] = max(v["speedup_vs_fp64_cg"] for v in ok)
    sp = forms.get("spmm_b_f32")
    if sp and "k8" in sp:
        s["spmm_b_k8_gflops"] = sp["k8"]["gflops"]
    return s


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    mats = load_cases()

    # ---- convert (one-off): each case in its tuned configuration, in
    # COPIES copies (own matrix, x and y) for the per-case graphs ----
    from paper_1012_2270_gb300 import autotune
    if args.tune_cache:
        autotune.CACHE_PATH = os.path.abspath(args.tune_cache)
    cases = []
    only = set(args.cases.split(",")) if args.cases else None
    for name, A, x in mats:
        for dt in DTYPES:
            if only is not None and f"{name}_{dt}" not in only:
                continue
            tdt = torch.float32 if dt == "f32" else torch.float64
            vals = A.val.astype(NP[dt])
            # group size, kernel and long-row schedule chosen by timing on this GPU
            cfg = autotune.tune(A.rowptr, A.col, vals, A.n_cols, dtype=tdt, reps=12,
                                 use_cache=bool(args.tune_cache))
            copies = []
            for _ in range(COPIES):
                M, kw = autotune.build(A.rowptr, A.col, vals, A.n_cols, cfg, tdt)
                xd = torch.from_numpy(x.astype(NP[dt])).to(dev)
                copies.append((M, xd, torch.empty(A.n_rows, dtype=xd.dtype, device=dev)))
            M = copies[0][0]
            nb = case_bytes(A, (A.n_rows + GROUP - 1) // GROUP, dt)
            cases.append(dict(key=f"{name}_{dt}", name=name, dt=dt, A=A, M=M, kw=kw, x=copies[0][1],
                              y=copies[0][2], copies=copies, bytes=nb, nnz=A.nnz,
                              kernel=kernel_name(cfg, M, A, dt), config=cfg,
                              pad_pct=M.artificial_zero_percent(),
                              launches=2 if M._long is not None and M._long[0].n_segments > 0 else 1))
    torch.cuda.synchronize()
    step_bytes = sum(c["bytes"] for c in cases)

    def launcher(c, j):
        M, xd, yd = c["copies"][j]
        return lambda: M.spmv(xd, out=yd, **c["kw"])

    # ---- the step as one CUDA graph: the six SpMVs are independent, so each
    # is a branch of the graph and the GPU may overlap them (the gather-bound
    # (b) cases with the HBM-bound stencils); the same six back to back are
    # timed beside it ----
    step_graph = capture_graph_branches([launcher(c, 0) for c in cases])
    serial_graph = capture_graph([launcher(c, 0) for c in cases])
    for _ in range(args.warmup):
        step_graph.replay()
        serial_graph.replay()
    torch.cuda.synchronize()

    # ---- timed region: K replays of the step graph ----
    K = args.steps
    t_start, t_end = _ev()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if rank == 0 else None
    time.sleep(0.2 if clocks else 0)
    torch.cuda.nvtx.range_push("timed_region")    # lets a profiler capture just these launches
    t_start.record(stream)
    for _ in range(K):
        step_graph.replay()
    t_end.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    ms_total, = max_over_ranks([t_start.elapsed_time(t_end)], dev)
    value = whole_job_gbs(world, K, step_bytes, ms_total)
    s0, s1 = _ev()
    s0.record(stream)
    for _ in range(K):
        serial_graph.replay()
    s1.record(stream)
    torch.cuda.synchronize()
    ms_serial = s0.elapsed_time(s1) / K

    # ---- per case: a graph of its COPIES copies in turn, ROUNDS times ----
    per_case_us = [rotating_us([launcher(c, j) for j in range(COPIES)], stream) for c in cases]
    # and hot: the same copy every time (what of the case L2 can keep, it keeps)
    hot_us = [rotating_us([launcher(c, 0)] * COPIES, stream) for c in cases]
    clk = clocks.stop() if clocks else None

    detail = {}
    for c, us, hot in zip(cases, per_case_us, hot_us):
        detail[c["key"]] = {"gbs": c["bytes"] / us / 1e3, "gflops": 2 * c["nnz"] / us / 1e3,
                            "us": us, "hot_us": hot,
                            "pct_of_8tbs": 100 * c["bytes"] / us / 1e3 / roofline.NOMINAL_HBM_GBS,
                            "artificial_zero_pct": c["pad_pct"], "kernel": c["kernel"],
                            "launches": c["launches"],
                            "config": {k: v for k, v in c["config"].items() if k != "us"}}

    # ---- the same bytes as one plain device read (the library's streaming
    # read of a buffer of the case's algorithmic bytes, three rotating
    # buffers in a graph like the SpMVs): what a streaming kernel of this
    # size reaches, launch ramp and tail included ----
    from paper_1012_2270_gb300.rgcsr import stream_read
    for c in cases:
        bufs = [torch.ones(c["bytes"] // 16 * 4, dtype=torch.float32, device=dev) for _ in range(COPIES)]
        r_us = rotating_us([lambda b=b: stream_read(b) for b in bufs], stream)
        d = detail[c["key"]]
        d["same_size_read_us"] = r_us
        d["frac_of_same_size_read"] = r_us / d["us"]
        del bufs
    torch.cuda.empty_cache()
    # ---- FP64 FMA rate (the library's probe): an FP64 SpMV does one FMA per
    # non-zero, and on this GPU that rate is low enough to be a second floor ----
    from paper_1012_2270_gb300.rgcsr import fp64_fma_probe
    fp64_fma_probe(64, stream)
    fma_t = []
    for _ in range(3):
        e0, e1 = _ev()
        e0.record(stream)
        n_fma = fp64_fma_probe(1024, stream)
        e1.record(stream)
        e1.synchronize()
        fma_t.append(e0.elapsed_time(e1) * 1e-3)
    fma_rate = n_fma / statistics.median(fma_t)                      # FMA/s
    for c in cases:
        if c["dt"] == "f64":
            detail[c["key"]]["fp64_fma_floor_us"] = 1e6 * c["nnz"] / fma_rate
    # ---- random-gather rate (the library's probe: scattered 8-byte loads of
    # an 8 MB vector resident in L2), the ceiling of the power-law matrix's
    # x gathers ----
    from paper_1012_2270_gb300.rgcsr import gather_probe
    gx = torch.ones(1 << 20, dtype=torch.float64, device=dev)
    gather_probe(gx, 16, stream)
    g_t = []
    for _ in range(3):
        e0, e1 = _ev()
        e0.record(stream)
        n_loads = gather_probe(gx, 256, stream)
        e1.record(stream)
        e1.synchronize()
        g_t.append(e0.elapsed_time(e1) * 1e-3)
    gather_rate = n_loads / statistics.median(g_t)                 # loads/s
    del gx

    roof = roofline_of(cases, per_case_us, detail, fma_rate, clk, dev, gather_rate)

    # ---- end to end: host x in, host y out, through rgcsr_spmv_host ----
    e2e = measure_e2e(cases, world, step_bytes, K, stream, barrier, dev)

    # ---- forms beside plain ----
    forms = {}
    # with a subset of the cases (profiling runs) only explicitly requested
    # forms run, each on the cases it needs that are present
    if not args.no_forms and rank == 0 and (only is None or args.forms):
        forms = measure_forms(mats, cases, detail, dev, stream, tune_cache=bool(args.tune_cache),
                              only=set(args.forms.split(",")) if args.forms else None,
                              ir_sweep=not args.no_ir_sweep)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(mats, args.cpu_seconds)

    if rank == 0:
        record = {"cases": detail, "roofline": roof, "e2e": e2e, "cpu_baseline": cpu, "forms": forms,
                  "clocks": clk, "ms_per_step": ms_total / K,
                  "ms_per_step_back_to_back": ms_serial,
                  "sum_of_case_us": sum(per_case_us),
                  "tuned": {c["key"]: {k: v for k, v in c["config"].items() if k != "us"} for c in cases}}
        if args.detail_out:
            with open(args.detail_out, "w") as f:
                json.dump(record, f, indent=1)
        else:
            print("detail: " + json.dumps(record), flush=True)
        line = headline(
            value=value, world=world, steps=K, warmup=args.warmup, ms_per_step=ms_total / K,
            gflops=world * K * sum(2 * c["nnz"] for c in cases) / (ms_total * 1e-3) / 1e9,
            launches=K * sum(c["launches"] for c in cases),
            clocks={k: v for k, v in clk.items() if k != "samples"} if clk else None,
            roof={k: v for k, v in roof.items() if k not in ("fp64_fma", "cases")},
            e2e={k: v for k, v in e2e.items() if k not in ("note", "one_stream_value")},
            cpu={k: v for k, v in cpu.items() if k != "single_thread_gbs"} if cpu else None,
            cases={c["key"]: [d["us"], d["gbs"]]
                   for c, d in ((c, detail[c["key"]]) for c in cases)},
            forms_summary=forms_summary(forms), detail_file=args.detail_out)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def roofline_of(cases, per_case_us, detail, fma_rate, clk, dev, gather_rate):
    """Roofline of the dominant kernel (the one with the largest share of
    the step): algorithmic bytes per launch / its mean time per launch from
    the per-case graphs, against the measured HBM copy bandwidth."""
    import torch
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        peak_hbm = json.load(open(peaks_path))["hbm_gbs"]
        peak_src = "measured"
    else:
        peak_hbm, peak_src = 6800.0, "fallback"
    by_kernel = {}
    for c, us in zip(cases, per_case_us):
        d = by_kernel.setdefault(c["kernel"], {"us": 0.0, "bytes": 0, "launches": 0})
        d["us"] += us
        d["bytes"] += c["bytes"]
        d["launches"] += 1
    dom = max(by_kernel, key=lambda k: by_kernel[k]["us"])
    d = by_kernel[dom]
    achieved = d["bytes"] / d["us"] / 1e3
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
            "frac": achieved / peak_hbm, "traffic": measured_traffic(dom, cases), "kernel": dom,
            "cases": [c["key"] for c in cases if c["kernel"] == dom], "peak_source": peak_src,
            "share_of_step": d["us"] / sum(per_case_us),
            "bytes_per_launch": d["bytes"] / d["launches"], "avg_launch_us": d["us"] / d["launches"]}
    dom_cases = [(c, us) for c, us in zip(cases, per_case_us) if c["kernel"] == dom]
    # the same bytes as plain reads (launch ramp and tail included): the
    # ceiling a memory-bound kernel of this size can reach on this GPU
    read_us = sum(detail[c["key"]]["same_size_read_us"] for c, _ in dom_cases)
    read_gbs = sum(c["bytes"] for c, _ in dom_cases) / read_us / 1e3
    roof["same_size_read"] = {"gbs": read_gbs, "frac": achieved / read_gbs}
    if all(c["dt"] == "f64" for c, _ in dom_cases):
        # one FP64 FMA per non-zero: its floor next to the HBM floor
        nnz = sum(c["nnz"] for c, _ in dom_cases)
        t_us = sum(us for _, us in dom_cases)
        roof["fp64_fma"] = {
            "probe_tflops": 2 * fma_rate / 1e12, "nominal_tflops": roofline.NOMINAL_FP64_TFLOPS,
            "achieved_tflops": 2 * nnz / (t_us * 1e-6) / 1e12,
            "floor_us": 1e6 * nnz / fma_rate,
            "hbm_floor_us": 1e6 * sum(c["bytes"] for c, _ in dom_cases) / (peak_hbm * 1e9),
            "kernel_us": t_us, "frac_of_probe": (1e6 * nnz / fma_rate) / t_us}
    if all(c["name"] == "b" for c, _ in dom_cases):
        # random columns: every x gather is its own L2 request.  The
        # library's gather probe measures how many scattered loads per second
        # the SMs issue (about one per SM clock); the kernel's requests -- one
        # per non-zero plus one per 128-byte line of the algorithmic bytes --
        # at that rate are a second ceiling, below HBM
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clk or {}).get("sm_mhz") or 1920.0
        reqs = [c["nnz"] + c["bytes"] / 128 for c, _ in dom_cases]
        ceil_us = statistics.fmean(1e6 * r / gather_rate for r in reqs)
        t_us = statistics.fmean(us for _, us in dom_cases)
        roof["gather_request_ceiling"] = {"us": ceil_us, "frac": ceil_us / t_us,
                                          "probe_loads_per_sm_clk": gather_rate / (sms * mhz * 1e6)}
    return roof


def measure_e2e(cases, world, step_bytes, K, stream, barrier, dev):
    """The same six SpMVs end to end through rgcsr_spmv_host: per step and
    case x host->device, SpMV, y device->host (pinned buffers, matrix
    resident, as in a Krylov solver); one stream per case, so that one
    case's copies overlap another's SpMV."""
    import torch
    host = []
    for c in cases:
        xh = c["x"].cpu().pin_memory()
        yh = torch.empty(c["y"].numel(), dtype=c["y"].dtype).pin_memory()
        host.append((xh, yh, torch.empty_like(c["x"]), torch.empty_like(c["y"])))
    h2d = sum(h[0].numel() * h[0].element_size() for h in host)
    d2h = sum(h[1].numel() * h[1].element_size() for h in host)
    Ke = max(3, K // 4)
    # one stream per case: a schedule's scratch allows one product in flight,
    # and each case's chain (x in, SpMV, y out) then overlaps the other cases'
    streams = [torch.cuda.Stream() for _ in range(len(cases))]
    def e2e_run(n_steps, overlap):
        e0, e1 = _ev()
        e0.record(stream)
        for st in streams:
            st.wait_event(e0)
        for _ in range(n_steps):
            for i, (c, h) in enumerate(zip(cases, host)):
                c["M"].spmv_host(*h, stream=streams[i] if overlap else stream, **c["kw"])
        for st in streams:
            ev = torch.cuda.Event()
            ev.record(st)
            stream.wait_event(ev)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    e2e_run(1, True)
    e2e_run(1, False)
    barrier()
    ms_e2e = e2e_run(Ke, True)
    ms_e2e_serial = e2e_run(Ke, False)
    barrier()
    ms_e2e, ms_e2e_serial = max_over_ranks([ms_e2e, ms_e2e_serial], dev)
    return {"value": whole_job_gbs(world, Ke, step_bytes, ms_e2e), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "one_stream_value": whole_job_gbs(world, Ke, step_bytes, ms_e2e_serial),
            "note": "per step and case: x host->device, SpMV, y device->host through rgcsr_spmv_host (pinned "
                    "buffers, matrix resident); one stream per case so copies overlap SpMVs"}


# ---------------------------------------------------------------------------
# the other forms, each beside its plain counterpart
# ---------------------------------------------------------------------------
def _ev():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def time_flushed(fn, reps, flush, stream):
    """Microseconds of fn with L2 flushed (a 256 MB read, which leaves no
    dirty lines behind) before each call: the mean of the middle half of
    the samples.  Event times of short launches come in steps of about
    2 us on GB300, so a median of a few samples of a 10-30 us launch lands
    on a step; the interquartile mean resolves finer differences when the
    samples straddle steps."""
    import torch
    from paper_1012_2270_gb300 import autotune
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        autotune.flush_l2(flush)
        e0, e1 = _ev()
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(1e3 * e0.elapsed_time(e1))
    ts.sort()
    q = len(ts) // 4
    return statistics.fmean(ts[q:len(ts) - q])


def max_scaled_error(y, y_ref, absy):
    import torch
    err = (y.double() - y_ref.double()).abs()
    den = absy.double()
    ok = den > 0
    return float((err[ok] / den[ok]).max()) if bool(ok.any()) else 0.0


def measure_forms(mats, cases, detail, dev, stream, tune_cache=False, only=None, ir_sweep=True):
    """The forms beside the plain SpMV; `only` (a set of names: hyb,
    quantized, x_read_path, spmm, backward, ir_cg, jacobi, small, conversion,
    group_size_sweep, table6, batched) limits them, None runs all."""
    import torch
    from paper_1012_2270_gb300 import solvers
    from paper_1012_2270_gb300.autograd import SparseOperator, spmm
    from paper_1012_2270_gb300 import _lib as L
    from paper_1012_2270_gb300 import autotune
    from paper_1012_2270_gb300.autotune import model_group_size
    from paper_1012_2270_gb300.batched import BatchedRgCSR, BlockDiagonalBatch
    from paper_1012_2270_gb300.rgcsr import HybMatrix, RgCSRMatrix

    forms = {}
    flush = torch.ones(64 << 20, dtype=torch.float32, device=dev)
    by = {c["key"]: c for c in cases}
    b = [m for m in mats if m[0] == "b"][0][1]

    def want(name):
        return only is None or name in only

    TT = {"f32": torch.float32, "f64": torch.float64}

    if want("hyb"):
        # -- HYB (ELL + COO), the paper's comparison format, timed like the
        # RgCSR cases (three rotating copies in a graph) ---------------------
        forms["hyb"] = {}
        for name, A, x in mats:
            for dt in DTYPES:
                if f"{name}_{dt}" not in by:
                    continue
                c = by[f"{name}_{dt}"]
                Hs = [HybMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dt]), A.n_cols, dtype=TT[dt])
                      for _ in range(COPIES)]
                ys = [torch.empty_like(c["y"]) for _ in range(COPIES)]
                t = rotating_us([lambda H=H, xj=cp[1], y=y: H.spmv(xj, out=y)
                                 for H, cp, y in zip(Hs, c["copies"], ys)], stream)
                H = Hs[0]
                nb = roofline.hyb_spmv_bytes(A.n_rows, A.n_cols, A.nnz, H.nnz_coo, VB[dt])
                forms["hyb"][c["key"]] = {"gbs": nb / t / 1e3, "gflops": 2 * A.nnz / t / 1e3, "us": t,
                                          "ell_width": H.ell_width, "nnz_coo": H.nnz_coo,
                                          "rgcsr_speedup": t / detail[c["key"]]["us"]}
                del Hs, ys
        torch.cuda.empty_cache()

    if want("quantized"):
        # -- reduced-precision values (bf16 / fp16 + per-row scale), timed like
        # the FP32 cases: three rotating copies (quantised from the three FP64
        # copies) in a graph, x and y in float ------------------------------
        # The error is taken against the library's FP64 product (itself within
        # 1e-12 |A||x| of the CPU oracle in the parity tests), scaled by |A||x|.
        forms["quantized"] = {}
        for name in ("a", "b", "c"):
            if f"{name}_f64" not in by or f"{name}_f32" not in by:
                continue
            c64, c32 = by[f"{name}_f64"], by[f"{name}_f32"]
            A = c32["A"]
            absA = RgCSRMatrix.from_csr(A.rowptr, A.col, np.abs(A.val), A.n_cols, dtype=torch.float64)
            y64, absy = c64["M"].spmv(c64["x"]), absA.spmv(c64["x"].abs())
            del absA
            # Q has c64's layout; take the FP32 case's schedule when the two
            # layouts agree (Q computes in float), else c64's
            same = all(c32["config"].get(k) == c64["config"].get(k) for k in ("group_size", "row_order"))
            for fmt in ("bf16", "f16"):
                Qs = []
                for j in range(COPIES):
                    Q = c64["copies"][j][0].quantized(fmt)
                    Q.copy_schedule(c32["copies"][j][0] if same else c64["copies"][j][0])
                    Qs.append(Q)
                ys = [torch.empty(A.n_rows, dtype=torch.float32, device=dev) for _ in range(COPIES)]
                xs = [cp[1] for cp in c32["copies"]]
                # kernel: the default, or (G = 32, no schedule) 16-byte loads, whichever is faster here
                kws = [{}]
                if Qs[0].group_size == 32 and Qs[0]._tiles is None and Qs[0]._long is None:
                    kws += [dict(kernel=L.KERNEL_LEAN, variant=v) for v in (1, 2, 4, 5, 6, 7, 8, 9)]
                    kws += [dict(kernel=L.KERNEL_TMA, variant=v) for v in (4, 5, 6)]
                ts = {i: rotating_us([lambda Q=Q, xj=xj, y=y, k=k: Q.spmv(xj, out=y, **k)
                                      for Q, xj, y in zip(Qs, xs, ys)], stream)
                      for i, k in enumerate(kws)}
                best = min(ts, key=ts.get)
                t, kw = ts[best], kws[best]
                Qs[0].spmv(xs[0], out=ys[0], **kw)
                nb = roofline.rgcsr_spmv_bytes(A.n_rows, A.n_cols, A.nnz, Qs[0].s.n_groups, 2, x_bytes=4,
                                               row_scale=True)
                forms["quantized"][f"{name}_{fmt}"] = {
                    "gbs": nb / t / 1e3, "gflops": 2 * A.nnz / t / 1e3, "us": t,
                    "speedup_vs_f32": detail[f"{name}_f32"]["us"] / t, "kernel": kw or "default",
                    "us_by_kernel": {("default" if not k else f"k{k['kernel']}v{k['variant']}"): ts[i]
                                     for i, k in enumerate(kws)},
                    "max_err_over_absAx_vs_f64": max_scaled_error(ys[0], y64, absy)}
                del Qs, ys
            del y64, absy
        torch.cuda.empty_cache()

    if want("x_read_path"):
        # -- the x read-path study (Sec. 4.3: texture cache on/off), redone on
        # the same thread-per-row mapping (G = 32, the cases' own layouts) with
        # the four read paths: read-only loads, plain loads, texture fetches,
        # and x ranges staged in shared memory per block of 256 rows ---------
        # (the power-law matrix, whose rows reach 10,000 entries, takes the
        # warp-split kernel, and its blocks touch too many scattered columns
        # for any window: every one of them would gather from global memory)
        xr = {}
        for c in cases:
            stencil = c["name"] != "b"
            k_ = L.KERNEL_LEAN if stencil else L.KERNEL_SPLIT
            row = {"kernel": "thread per row" if stencil else "warp split"}
            for key, kw in (("nc", dict(kernel=k_, x_load=L.XLOAD_NC)),
                            ("plain", dict(kernel=k_, x_load=L.XLOAD_PLAIN)),
                            ("tex", dict(kernel=k_, x_load=L.XLOAD_TEX))):
                row[key + "_us"] = rotating_us([lambda M=M, xj=xj, y=y, kw=kw: M.spmv(xj, out=y, **kw)
                                                for M, xj, y in c["copies"]], stream)
            if stencil:
                for cp in c["copies"]:
                    cp[0].plan_x_window()
                recs = c["copies"][0][0].x_window_records()
                row["staged_blocks_pct"] = 100.0 * sum(1 for r in recs if r[0] > 0) / max(len(recs), 1)
                row["mean_staged_elems"] = statistics.fmean([r[1] for r in recs if r[0] > 0] or [0])
                row["smem_window_us"] = rotating_us([lambda M=M, xj=xj, y=y: M.spmv_xwindow(xj, out=y)
                                                     for M, xj, y in c["copies"]], stream)
                for cp in c["copies"]:
                    cp[0]._xwin = None
            for k in ("nc", "plain", "tex", "smem_window"):
                if k + "_us" in row:
                    row[k + "_gbs"] = c["bytes"] / row[k + "_us"] / 1e3
            xr[c["key"]] = row
        forms["x_read_path_g32"] = xr

    if want("spmm"):
        # -- multi-RHS SpMM on (b) ------------------------------------------------
        # natural row order, G = 1 with the long-row schedule (T = 16, 64-slot
        # segments): the lanes-per-row kernels; the thread-per-row kernel at the
        # byte model's group size beside it
        b = [m for m in mats if m[0] == "b"][0][1]
        Mb = RgCSRMatrix.from_csr(b.rowptr, b.col, b.val.astype(np.float32), b.n_cols, dtype=torch.float32,
                                  group_size=1).split_long_rows(16, 64)
        Gm = model_group_size(b.rowptr, 4)
        Mt = RgCSRMatrix.from_csr(b.rowptr, b.col, b.val.astype(np.float32), b.n_cols, dtype=torch.float32,
                                  group_size=Gm)
        # and G = 32 in descending row order with group tiles (the tiled kernels)
        Md = RgCSRMatrix.from_csr(b.rowptr, b.col, b.val.astype(np.float32), b.n_cols, dtype=torch.float32,
                                  group_size=32, row_order="descending").tile_groups(64)
        Hb = HybMatrix.from_csr(b.rowptr, b.col, b.val.astype(np.float32), b.n_cols, dtype=torch.float32)
        forms["spmm_b_f32"] = {"configs": {"lanes_per_row": "G=1, long-row schedule T=16 S=64",
                                           "tiles": "G=32, descending row order, group tiles C=64",
                                           "thread_per_row": f"G={Gm}"}}
        for k in (1, 4, 8, 16, 32):
            X = torch.rand(b.n_cols, k, device=dev)
            Y = torch.empty(b.n_rows, k, device=dev)
            ts = {}
            for cfg_name, Mx, reps in (("lanes_per_row", Mb, 10), ("tiles", Md, 10), ("thread_per_row", Mt, 5)):
                torch.cuda.nvtx.range_push(f"spmm_k{k}_{cfg_name}")         # a profiler can pick one out
                ts[cfg_name] = time_flushed(lambda: Mx.spmm(X, out=Y), reps, flush, stream)
                torch.cuda.nvtx.range_pop()
            best = min(ts, key=ts.get)
            t = ts[best]
            nb = roofline.spmm_bytes(b.n_rows, b.n_cols, b.nnz, (b.n_rows + GROUP - 1) // GROUP, 4, k)
            forms["spmm_b_f32"][f"k{k}"] = {"gbs": nb / t / 1e3, "gflops": 2 * b.nnz * k / t / 1e3, "us": t,
                                            "best": best, "us_by_config": ts,
                                            "hyb_us": time_flushed(lambda: Hb.spmm(X, out=Y), 5, flush, stream)}
            del X, Y
        del Mb, Mt, Md, Hb

    if want("backward"):
        # -- backward of Y = A X on (b), batch of 8 right-hand sides: three
        # operators (own matrices, values and X) called in turn, ten rounds
        # back to back, one event pair: the device time per call, with the
        # host's autograd overhead hidden behind the queued kernels and no
        # call finding its matrix in L2 ---------------------------------------
        G = 32
        ops = []
        for _ in range(COPIES):
            op = SparseOperator(b.rowptr, b.col, b.n_cols, dtype=torch.float32, group_size=G,
                                row_order="descending", tiles=64)
            vals = torch.from_numpy(b.val.astype(np.float32)).to(dev).requires_grad_(True)
            X = torch.rand(b.n_cols, 8, device=dev, requires_grad=True)
            ops.append((op, vals, X))

        def per_call_us(fn, rounds=10):
            for o in ops:
                fn(*o)
            torch.cuda.synchronize()
            e0, e1 = _ev()
            e0.record(stream)
            for _ in range(rounds):
                for o in ops:
                    fn(*o)
            e1.record(stream)
            torch.cuda.synchronize()
            return 1e3 * e0.elapsed_time(e1) / (rounds * len(ops))

        def fwd(op, vals, X):
            with torch.no_grad():
                return spmm(op, vals, X)

        def fwd_bwd(op, vals, X):
            # a fixed upstream gradient dY, so no loss kernel is timed
            vals.grad = None
            X.grad = None
            spmm(op, vals, X).backward(op._bench_dy)

        def spmm_only(op, vals, X):
            op.A.spmm(X.detach(), out=op._bench_y)

        # a training step changes the values before every forward: each
        # operator alternates between two value tensors (the second negated),
        # so every call finds values that differ from the ones it last loaded
        def changed(o):
            op, vals, X = o
            v = op._bench_vals[op._bench_flip]
            op._bench_flip ^= 1
            return op, v, X

        def fwd_changed(op, vals, X):
            return fwd(*changed((op, vals, X)))

        def fwd_bwd_changed(op, vals, X):
            return fwd_bwd(*changed((op, vals, X)))

        for o in ops:
            o[0]._bench_y = torch.empty(b.n_rows, 8, device=dev)
            o[0]._bench_dy = torch.rand(b.n_rows, 8, device=dev)
            o[0]._bench_vals = [o[1], (-o[1].detach()).requires_grad_(True)]
            o[0]._bench_flip = 0
        t_mm = per_call_us(spmm_only)
        torch.cuda.nvtx.range_push("autograd_forward")            # a profiler can pick it out
        t_f = per_call_us(fwd)
        torch.cuda.nvtx.range_pop()
        t_fb = per_call_us(fwd_bwd)
        t_fc = per_call_us(fwd_changed)
        t_fbc = per_call_us(fwd_bwd_changed)
        forms["backward_b_k8_f32"] = {"group_size": G, "schedule": "descending row order, group tiles C=64",
                                      "spmm_us": t_mm, "forward_us": t_f, "forward_backward_us": t_fb,
                                      "forward_over_spmm": t_f / t_mm, "backward_over_forward": (t_fb - t_f) / t_f,
                                      "values_changed": {"forward_us": t_fc, "forward_backward_us": t_fbc,
                                                         "forward_over_spmm": t_fc / t_mm,
                                                         "step_over_spmm": t_fbc / t_mm}}
        del ops

    if want("ir_cg") and "a_f64" in by:
        # -- mixed-precision iterative refinement CG, Poisson 128^3 ---------------
        a = [m for m in mats if m[0] == "a"][0][1]
        M64 = by["a_f64"]["M"]
        rhs = torch.from_numpy(synth.uniform_vector(a.n_rows, seed=0)).to(dev)
        lo = M64.quantized("bf16")
        e0, e1 = _ev()
        torch.cuda.nvtx.range_push("ir_cg")                # a profiler can pick it out
        e0.record(stream)
        x_ir, outer, inner, rel = solvers.ir_cg(M64, lo, rhs, outer_tol=1e-10, max_outer=50, inner_tol=1e-6,
                                                 max_inner=2000)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        t_ir = e0.elapsed_time(e1)
        e0, e1 = _ev()
        e0.record(stream)
        x64, its64, rel64 = solvers.cg(M64, rhs, rel_tol=1e-10, max_iter=5000)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1)
        # the inner tolerance sets how the iterations split into corrections:
        # each correction restarts the inner CG, so fewer, deeper inner solves
        # need fewer iterations in all (float CG reaches about 1e-6)
        sweep = {}
        for tol in (1e-3, 1e-4, 1e-5, 1e-6) if ir_sweep else ():
            e0, e1 = _ev()
            e0.record(stream)
            xs, o_, i_, r_ = solvers.ir_cg(M64, lo, rhs, outer_tol=1e-10, max_outer=50, inner_tol=tol, max_inner=2000)
            e1.record(stream)
            torch.cuda.synchronize()
            sweep[f"{tol:g}"] = {"ms": e0.elapsed_time(e1), "corrections": o_, "inner_iterations": i_,
                                 "final_rel_residual": r_, "speedup_vs_fp64_cg": t64 / e0.elapsed_time(e1)}
            del xs
        forms["ir_cg_poisson128"] = {
            "ms": t_ir, "corrections": outer, "inner_iterations": inner, "final_rel_residual": rel,
            "fp64_cg_ms": t64, "fp64_cg_iterations": its64,
            "rel_diff_vs_fp64_cg": float((x_ir - x64).norm() / x64.norm()),
            "inner_tol_sweep": sweep}
        del lo, x_ir, x64

    if want("jacobi"):
        # -- gradient through 100 damped-Jacobi steps, 96^3, checkpoint every 10 --
        J = synth.laplacian_3d(96)
        opj = SparseOperator(J.rowptr, J.col, J.n_cols, dtype=torch.float32)
        vj = torch.from_numpy(J.val.astype(np.float32)).to(dev).requires_grad_(True)
        bj = torch.from_numpy(synth.uniform_vector(J.n_rows, seed=0).astype(np.float32)).to(dev).requires_grad_(True)
        dinv = torch.full((J.n_rows,), 1.0 / 6.0, device=dev)
        res = {}
        for ck in (0, 10):
            def run():
                vj.grad = None
                bj.grad = None
                xj = solvers.jacobi(opj, vj, bj, dinv, 2.0 / 3.0, 100, checkpoint_every=ck)
                (xj * xj).sum().backward()
            run()                                   # warm-up
            torch.cuda.synchronize()
            torch.cuda.reset_peak_memory_stats()
            base = torch.cuda.memory_allocated()
            e0, e1 = _ev()
            e0.record(stream)
            run()
            e1.record(stream)
            torch.cuda.synchronize()
            res["checkpoint_every_10" if ck else "no_checkpoint"] = {
                "ms": e0.elapsed_time(e1),
                "peak_extra_mem_mb": (torch.cuda.max_memory_allocated() - base) / 2**20}
        forms["jacobi_grad_96_f32"] = res
        del opj

    if want("small"):
        # -- the small case (2D 5-point Laplacian 64 x 64, n = 4,096): it fits
        # in L2, so no roofline claim -- the device time per SpMV (a graph of
        # 20 back-to-back calls, median of 30 replays) and the latency of one
        # call through the Python binding, launch to synchronised result ----
        A = synth.workload_small_laplacian()
        small = {"n": A.n_rows, "nnz": A.nnz}
        for dt in DTYPES:
            M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dt]), A.n_cols, group_size=32,
                                     dtype=TT[dt])
            x = torch.from_numpy(synth.uniform_vector(A.n_cols, seed=0).astype(NP[dt])).to(dev)
            y = torch.empty(A.n_rows, dtype=TT[dt], device=dev)
            g = capture_graph([lambda: M.spmv(x, out=y)] * 20)
            dev_us = statistics.median(replay_us(g, 30, stream)) / 20
            del g
            ts = []
            for rep in range(210):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                M.spmv(x, out=y)
                torch.cuda.synchronize()
                if rep >= 10:
                    ts.append(1e6 * (time.perf_counter() - t0))
            small[dt] = {"device_us": dev_us, "call_us": statistics.median(ts), "kernel": kernel_name({}, M, A, dt)}
            del M, x, y
        forms["small_laplacian_64"] = small

    if want("conversion"):
        # -- conversion CSR -> RgCSR on the device (plan + convert; FP32 values,
        # CSR already in HBM): bytes = CSR read + RgCSR written ----------------
        conv = {}
        for name, A, x in mats:
            rp = torch.from_numpy(A.rowptr).to(dev)
            cl = torch.from_numpy(A.col).to(dev)
            vl = torch.from_numpy(A.val.astype(np.float32)).to(dev)
            order = "descending" if name == "b" else None
            ts = []
            for rep in range(6):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                M = RgCSRMatrix.from_csr(rp, cl, vl, A.n_cols, group_size=32, dtype=torch.float32, row_order=order)
                torch.cuda.synchronize()
                if rep:
                    ts.append(1e6 * (time.perf_counter() - t0))
            t = statistics.median(ts)
            nb = A.nnz * 8 + (A.n_rows + 1) * 8 + M.n_stored * 8 + A.n_rows * 4 + (M.s.n_groups + 1) * 8
            conv[name] = {"us": t, "gbs": nb / t / 1e3, "row_order": order or "natural",
                          "n_stored": M.n_stored, "note": "host wall time incl. the plan's one stream sync"}
            del M, rp, cl, vl
        forms["conversion_f32"] = conv

    if want("group_size_sweep"):
        # -- group-size sweep (the paper's Table 4 on these matrices), x read path
        # on/off (the texture study of Sec. 4.3) and sliced ELLPACK (Sec. 3.4) --
        forms.update(measure_tables(mats, flush, stream))

    if want("table6"):
        # -- the four matrix shapes of Sec. 4.4.2 (Table 6), FP64 ----------------
        forms["table6_fp64"] = measure_table6(flush, stream, tune_cache)

    if want("batched"):
        # -- batched: the 512-member uneven batch in one launch vs 512 launches ---
        members = synth.workload_batch(512)
        Bt = BatchedRgCSR.from_csr_list(members, dtype=torch.float32, group_sizes="model")
        xb = torch.rand(Bt.n_cols_total, device=dev)
        yb = torch.empty(Bt.n_rows_total, device=dev)
        g = Bt.capture(xb, yb, repeats=1)
        nb_batch = sum(roofline.rgcsr_spmv_bytes(m.n_rows, m.n_cols, m.nnz, (m.n_rows + GROUP - 1) // GROUP, 4)
                       for m in members)
        t_b = time_flushed(lambda: g.replay(), 10, flush, stream)
        plain = [RgCSRMatrix.from_csr(m.rowptr, m.col, m.val, m.n_cols, group_size=Gm, dtype=torch.float32)
                 for m, Gm in zip(members, Bt.group_sizes)]
        xs = [xb[Bt.member_slices(i)[0]] for i in range(len(members))]
        ys = [yb[Bt.member_slices(i)[1]] for i in range(len(members))]
        gp = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for M, xi, yi in zip(plain, xs, ys):
                M.spmv(xi, out=yi)
            side.synchronize()
            with torch.cuda.graph(gp, stream=side):
                for M, xi, yi in zip(plain, xs, ys):
                    M.spmv(xi, out=yi, stream=side)
        torch.cuda.current_stream().wait_stream(side)
        t_p = time_flushed(lambda: gp.replay(), 10, flush, stream)
        del plain, gp
        # the same batch as one block-diagonal matrix, rows in descending length
        # order over the whole batch, group tiles
        bd = {}
        for tile, var in ((64, 1), (64, 7), (128, 7), (256, 7)):
            Bd = BlockDiagonalBatch.from_csr_list(members, dtype=torch.float32, tile=tile, variant=var)
            gd = Bd.capture(xb, yb, repeats=1)
            bd[f"tiles_{tile}_v{var}"] = time_flushed(lambda: gd.replay(), 10, flush, stream)
            del Bd, gd
            torch.cuda.empty_cache()
        best = min(bd, key=bd.get)
        t_d = bd[best]
        forms["batched_512_f32"] = {
            "members": len(members), "rows": Bt.n_rows_total, "nnz": Bt.nnz,
            "gbs": nb_batch / min(t_b, t_d) / 1e3, "gflops": 2 * Bt.nnz / min(t_b, t_d) / 1e3, "us": min(t_b, t_d),
            "per_member_kernel_us": t_b, "block_diagonal_us": bd, "block_diagonal_best": best,
            "plain_512_launches_us": t_p, "plain_gbs": nb_batch / t_p / 1e3, "speedup_vs_plain": t_p / min(t_b, t_d)}
        del Bt, members

    return forms


def measure_table6(flush, stream, tune_cache):
    """Stand-ins for Hohn/fd18, AMD/G2_circuit, IBM_EDA/trans4 and Rajat/Raj1
    (their rows and longest / mean / shortest row length), FP64 like the
    paper's Table 6: GFLOP/s of the paper's kernel at G = 128 (read-only x,
    the paper's setting), of HYB, and of the autotuned RgCSR configuration,
    with the artificial-zero share of each RgCSR layout."""
    import torch
    from paper_1012_2270_gb300 import _lib as L
    from paper_1012_2270_gb300 import autotune
    from paper_1012_2270_gb300.rgcsr import HybMatrix, RgCSRMatrix
    out = {}
    for name in synth.TABLE6_ROWS:
        A = synth.table6_standin(name)
        x = torch.from_numpy(synth.uniform_vector(A.n_cols, seed=0)).cuda()
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        gf = lambda us: 2 * A.nnz / us / 1e3
        M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=128, dtype=torch.float64)
        t_paper = time_flushed(lambda: M.spmv(x, out=y, kernel=L.KERNEL_PAPER), 3, flush, stream)
        pad_paper = M.artificial_zero_percent()
        del M
        H = HybMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, dtype=torch.float64)
        torch.cuda.nvtx.range_push(f"table6_{name}_hyb")                 # a profiler can pick one out
        t_hyb = time_flushed(lambda: H.spmv(x, out=y), 20, flush, stream)
        torch.cuda.nvtx.range_pop()
        del H
        cfg = autotune.tune(A.rowptr, A.col, A.val, A.n_cols, dtype=torch.float64, reps=8,
                            use_cache=tune_cache)
        T, kw = autotune.build(A.rowptr, A.col, A.val, A.n_cols, cfg, torch.float64)
        torch.cuda.nvtx.range_push(f"table6_{name}_tuned")
        t_tuned = time_flushed(lambda: T.spmv(x, out=y, **kw), 20, flush, stream)
        torch.cuda.nvtx.range_pop()
        L_ = A.row_lengths()
        out[name] = {"rows": A.n_rows, "max": int(L_.max()), "mean": float(L_.mean()), "min": int(L_.min()),
                     "nnz": A.nnz,
                     "paper_kernel_G128": {"us": t_paper, "gflops": gf(t_paper), "artificial_zero_pct": pad_paper},
                     "hyb": {"us": t_hyb, "gflops": gf(t_hyb)},
                     "tuned": {"us": t_tuned, "gflops": gf(t_tuned), "artificial_zero_pct": T.artificial_zero_percent(),
                               "config": {k: v for k, v in cfg.items() if k != "us"}},
                     "paper_over_hyb": t_hyb / t_paper, "tuned_over_hyb": t_hyb / t_tuned}
        del T
        torch.cuda.empty_cache()
    return out


def measure_tables(mats, flush, stream):
    """Natural row order, G in {32, 64, 128, 256}, FP32 and FP64:
    artificial zeros and GB/s of the paper's kernel (one block per group)
    with x through the read-only path and with plain loads, of the
    warp-split kernel, and of sliced ELLPACK on the same slabs."""
    import torch
    from paper_1012_2270_gb300 import _lib as L
    from paper_1012_2270_gb300.rgcsr import RgCSRMatrix
    sweep = {}
    for name, A, x in mats:
        for dt in DTYPES:
            tdt = torch.float32 if dt == "f32" else torch.float64
            xd = torch.from_numpy(x.astype(NP[dt])).cuda()
            nb = case_bytes(A, (A.n_rows + GROUP - 1) // GROUP, dt)
            for G in (32, 64, 128, 256):
                M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dt]), A.n_cols, group_size=G, dtype=tdt)
                y = torch.empty(A.n_rows, dtype=tdt, device="cuda")
                row = {"artificial_zero_pct": M.artificial_zero_percent()}
                for key, kw in (("paper_readonly_x", dict(kernel=L.KERNEL_PAPER)),
                                ("paper_plain_x", dict(kernel=L.KERNEL_PAPER, x_load=L.XLOAD_PLAIN)),
                                ("paper_texture_x", dict(kernel=L.KERNEL_PAPER, x_load=L.XLOAD_TEX)),
                                ("split", dict(kernel=L.KERNEL_SPLIT)),
                                ("sliced_ellpack", dict(kernel=L.KERNEL_SELL))):
                    t = time_flushed(lambda: M.spmv(xd, out=y, **kw), 5, flush, stream)
                    row[key] = {"us": t, "gbs": nb / t / 1e3, "gflops": 2 * A.nnz / t / 1e3}
                sweep[f"{name}_{dt}_G{G}"] = row
                del M, y
                torch.cuda.empty_cache()
    return {"group_size_sweep": sweep}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
