"""Autotuning of the RgCSR launch parameters on the current GPU.

* ``model_group_size``: the group size G from a byte model -- the slots one
  SpMV streams, n_stored(G) * (value + index bytes), plus 8 bytes of group
  pointer per group -- preferring G = 32 (full 128-byte slot-rows, the
  vector-load and TMA-staged kernels) when it is within 5% of the best.  The paper fixed G
  per GPU by experiment (Sec. 4.3: 128 was best on a GTX 280); here the
  choice follows the matrix.
* ``tune``: times candidate (group size, kernel, variant) configurations
  in CUDA graphs, flushing L2 (by a read) before each launch, and caches
  the fastest per (matrix pattern, value type, GPU name) in a JSON file;
  the default configuration stays unless another is more than 2% faster.
* ``tune_hyb_width``: the same for the ELL width of the HYB format around
  the library's byte-cost rule.
* ``heuristic``: a configuration from the row lengths alone, without timing.
"""
from __future__ import annotations

import json
import os
import statistics
import zlib

import numpy as np
import torch

from . import _lib as L

CACHE_PATH = os.environ.get("RGCSR_TUNE_CACHE",
                            os.path.join(os.path.expanduser("~"), ".cache", "rgcsr", "autotune.json"))


def stored_slots(lengths: np.ndarray, G: int) -> int:
    """sum over groups of R_g * K_g (stored slots, padding included)."""
    n = lengths.size
    if n == 0:
        return 0
    pad = (-n) % G
    Lp = np.concatenate([lengths, np.zeros(pad, lengths.dtype)]).reshape(-1, G)
    K = Lp.max(axis=1).astype(np.int64)
    R = np.full(K.size, G, np.int64)
    R[-1] = n - G * (K.size - 1)
    return int((R * K).sum())


def model_group_size(rowptr, value_bytes: int, candidates=(8, 16, 32, 64, 128)) -> int:
    lengths = np.diff(np.asarray(rowptr, dtype=np.int64))
    n = lengths.size
    cost = {G: stored_slots(lengths, G) * (value_bytes + 4) + ((n + G - 1) // G) * 8 for G in candidates}
    best = min(cost.values())
    if 32 in cost and cost[32] <= 1.05 * best:
        return 32
    return min(candidates, key=lambda G: (cost[G], -G))


def signature(rowptr, col, n_cols: int, dtype: torch.dtype) -> str:
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    c = np.ascontiguousarray(col, dtype=np.int32)
    h = zlib.crc32(rp.tobytes())
    h = zlib.crc32(c[: 1 << 20].tobytes(), h)
    gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return f"{rp.size - 1}x{n_cols}:{int(rp[-1])}:{h:08x}:{str(dtype)}:{gpu}"


def _load_cache() -> dict:
    try:
        with open(CACHE_PATH) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(cache: dict) -> None:
    try:
        os.makedirs(os.path.dirname(CACHE_PATH), exist_ok=True)
        tmp = CACHE_PATH + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE_PATH)
    except OSError:
        pass


def flush_l2(flush: torch.Tensor) -> None:
    """Evicts L2 by READING a buffer larger than it.  A write would leave the
    L2 full of dirty lines, and their write-back would land in the next
    timed launch (a 142 MB read takes 30 us after a 256 MB memset, 26 us
    after a 256 MB read)."""
    flush.sum()


def _graph(fns):
    """A CUDA graph of fns called in order on a capture stream (each call
    enqueues its kernels on the current stream)."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        for f in fns:
            f()
    torch.cuda.current_stream().wait_stream(side)
    return g


def _replay_median(g, replays: int) -> float:
    g.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(replays)]
    for e0, e1 in ev:
        e0.record()
        g.replay()
        e1.record()
    torch.cuda.synchronize()
    return statistics.median(e0.elapsed_time(e1) for e0, e1 in ev)


def _time(fn, reps: int, flush: torch.Tensor) -> float:
    """Time in microseconds of fn() with L2 flushed before each call, from
    CUDA graphs: one of `reps` (flush, fn) pairs and one of the `reps`
    flushes alone, the difference of their median replay times divided by
    reps.  The graph leaves out host launch gaps, as the benchmark's own
    timing does, so the tuner ranks configurations the way they are
    measured."""
    fn()
    flush_l2(flush)
    torch.cuda.synchronize()
    r = max(reps, 4)
    g1 = _graph([f for _ in range(r) for f in (lambda: flush_l2(flush), fn)])
    g0 = _graph([lambda: flush_l2(flush) for _ in range(r)])
    t = (_replay_median(g1, 5) - _replay_median(g0, 5)) * 1e3 / r
    del g1, g0
    return max(t, 0.0)


def candidates(rowptr, dtype: torch.dtype):
    """Configurations worth timing: for dense groups the G = 32 kernels; for
    uneven rows small group sizes, with and without the long-row segment
    schedule (threshold T, 256 slots per segment), and the rows in
    descending length order (Sec. 4.4.2, Table 7), which makes the groups
    dense again, with the segment schedule or group tiles of C slot-rows
    (a one-warp-per-row-group kernel on a very long group would serialise,
    so those are not timed)."""
    lengths = np.diff(np.asarray(rowptr, dtype=np.int64))
    nnz = int(lengths.sum())
    irregular = stored_slots(lengths, 32) * 4 > nnz * 5
    cands = [dict(group_size=32, kernel=L.KERNEL_AUTO)]
    if not irregular:
        cands += [dict(group_size=32, kernel=L.KERNEL_TMA, variant=v) for v in range(7)]
        cands += [dict(group_size=G, kernel=k) for G in (32, 64) for k in (L.KERNEL_LEAN, L.KERNEL_SPLIT)]
        if dtype in (torch.float32, torch.float64):
            cands += [dict(group_size=32, kernel=L.KERNEL_LEAN, variant=v) for v in (1, 2, 4, 5, 6, 7, 8)]
    else:
        Gm = model_group_size(rowptr, dtype.itemsize)
        cands += [dict(group_size=G, kernel=L.KERNEL_SPLIT) for G in sorted({1, 2, 4, 8, Gm})]
        cands += [dict(group_size=G, long_rows=[T, 256]) for G in (1, 2, 4) for T in (16, 32, 64)]
        desc = dict(group_size=32, row_order="descending")
        cands += [dict(desc, long_rows=[T, 256]) for T in (32, 64, 128, 256)]
        cands += [dict(desc, tiles=[C, v]) for C in (32, 64, 128) for v in range(8)]
    if not irregular:
        cands += [dict(group_size=32, tiles=[64, v]) for v in (0, 1, 2)]
    return cands


def heuristic(rowptr, dtype: torch.dtype = torch.float32) -> dict:
    """A configuration without timing, from the row lengths alone: G = 32 in
    the CSR's row order when its groups are dense (padding <= 25% of the
    stored slots, the library then picks the kernel), else the rows in
    descending length order with group tiles of 64 slot-rows (pipelined
    for 4-byte arithmetic), the best shapes measured on the power-law
    matrix."""
    lengths = np.diff(np.asarray(rowptr, dtype=np.int64))
    nnz = int(lengths.sum())
    if stored_slots(lengths, 32) * 4 <= nnz * 5:
        return dict(group_size=32, kernel=L.KERNEL_AUTO)
    return dict(group_size=32, row_order="descending", tiles=[64, 2 if dtype == torch.float64 else 3])


def build(rowptr, col, val, n_cols: int, config: dict, dtype: torch.dtype):
    """The RgCSR matrix and spmv keyword arguments of a configuration."""
    from .rgcsr import RgCSRMatrix
    M = RgCSRMatrix.from_csr(rowptr, col, val, n_cols, group_size=config["group_size"], dtype=dtype,
                             row_order=config.get("row_order"))
    if "long_rows" in config:
        M.split_long_rows(*config["long_rows"])
    if "tiles" in config:
        M.tile_groups(*config["tiles"])
    return M, {k: v for k, v in config.items() if k in ("kernel", "variant")}


# relative margin by which a candidate must beat the default configuration
PREFER_DEFAULT = 0.02


def pick(results: list[dict]) -> dict:
    """The fastest timed configuration, except that the library's default
    (G = 32, automatic kernel) stays unless another is more than
    PREFER_DEFAULT faster: configurations within the timer's noise of each
    other would otherwise trade places from run to run."""
    best = min(results, key=lambda r: r["us"])
    default = next((r for r in results if r.get("kernel") == L.KERNEL_AUTO
                    and set(r) == {"group_size", "kernel", "us"} and r["group_size"] == 32), None)
    if default is not None and default["us"] <= best["us"] * (1.0 + PREFER_DEFAULT):
        return default
    return best


def tune(rowptr, col, val, n_cols: int, dtype: torch.dtype = torch.float32, reps: int = 10,
         use_cache: bool = True) -> dict:
    """Fastest configuration for this matrix on this GPU, e.g.
    {"group_size": 32, "kernel": 3, "variant": 0, "us": 30.6}; the default
    configuration (G = 32, automatic kernel) unless another is more than
    PREFER_DEFAULT faster."""
    from .rgcsr import RgCSRMatrix
    key = signature(rowptr, col, n_cols, dtype)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return cache[key]
    flush = torch.ones(64 << 20, dtype=torch.float32, device="cuda")      # 256 MB > L2
    x = torch.rand(n_cols, dtype=torch.float64 if dtype == torch.float64 else torch.float32, device="cuda")
    built = {}
    results = []
    for c in candidates(rowptr, dtype):
        fmt = (c["group_size"], c.get("row_order"))
        if fmt not in built:
            built[fmt] = RgCSRMatrix.from_csr(rowptr, col, val, n_cols, group_size=fmt[0], dtype=dtype,
                                              row_order=fmt[1])
        M = built[fmt]
        M._long = M._tiles = None
        if "long_rows" in c:
            M.split_long_rows(*c["long_rows"])
        if "tiles" in c:
            M.tile_groups(*c["tiles"])
        kw = {k: v for k, v in c.items() if k in ("kernel", "variant")}
        try:
            y = M.spmv(x, **kw)
        except L.RgCSRError:
            continue                      # configuration not valid for this matrix
        us = _time(lambda: M.spmv(x, out=y, **kw), reps, flush)
        results.append(dict(c, us=us))
        M._long = M._tiles = None
    best = pick(results)
    if use_cache:
        cache = _load_cache()
        cache[key] = best
        _store_cache(cache)
    return best


def tune_hyb_width(rowptr, col, val, n_cols: int, dtype: torch.dtype = torch.float32, reps: int = 10) -> dict:
    """Times ELL widths around the byte-cost rule's choice."""
    from .rgcsr import HybMatrix
    base = HybMatrix.from_csr(rowptr, col, val, n_cols, dtype=dtype)
    k0, kmax = base.ell_width, base.s.max_row_len
    widths = sorted({w for w in (k0 - 2, k0 - 1, k0, k0 + 1, k0 + 2, 2 * k0) if 0 <= w <= kmax})
    flush = torch.ones(64 << 20, dtype=torch.float32, device="cuda")
    x = torch.rand(n_cols, dtype=torch.float64 if dtype == torch.float64 else torch.float32, device="cuda")
    results = []
    for w in widths:
        H = base if w == k0 else HybMatrix.from_csr(rowptr, col, val, n_cols, ell_width=w, dtype=dtype)
        y = H.spmv(x)
        results.append(dict(ell_width=w, us=_time(lambda: H.spmv(x, out=y), reps, flush), rule=(w == k0)))
        del H
    return min(results, key=lambda r: r["us"])
