"""Seeded synthetic sparse matrices and vectors.

This module only *generates inputs*; it contains none of the RgCSR method's
arithmetic (no layout, no SpMV), so both the CUDA path and the CPU oracle can
take their inputs from it.  Matrices come back as plain CSR in host
memory: ``rowptr`` int64 [n+1], ``col`` int32 [nnz] (ascending within a row),
``val`` float64 [nnz] -- except ``uniform_rows_device``, a matrix past 2^31
entries given by closed forms, which is generated on the device.

The shapes stand in for the paper's test collection (University of Florida
and Matrix Market matrices, Sec. 4.1, which are not redistributable here):
PDE stencils with nearly uniform rows, power-law rows with a heavy tail (the
"second group" matrices of Sec. 4.4.2 such as trans4 and Raj1), banded
matrices, and mixes of small and large matrices.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np


@dataclass
class CSRMatrix:
    n_rows: int
    n_cols: int
    rowptr: np.ndarray   # int64 [n_rows + 1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr)


def _from_offsets(shape_rows: int, offsets_cols: np.ndarray, valid: np.ndarray,
                  n_cols: int, name: str) -> CSRMatrix:
    """offsets_cols/valid: [n, w] arrays, columns ascending along axis 1."""
    lengths = valid.sum(axis=1).astype(np.int64)
    rowptr = np.zeros(shape_rows + 1, np.int64)
    np.cumsum(lengths, out=rowptr[1:])
    col = offsets_cols[valid].astype(np.int32)
    return CSRMatrix(shape_rows, n_cols, rowptr, col, np.empty(0), name)


def stencil_3d(nx: int, ny: int, nz: int, points: int) -> CSRMatrix:
    """Lexicographic grid numbering i = (z*ny + y)*nx + x; Dirichlet
    truncation (neighbours outside the grid are dropped).  points = 7 (face
    neighbours) or 27 (full 3x3x3 neighbourhood).  Values are left empty."""
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    if points == 7:
        offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    elif points == 27:
        offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    else:
        raise ValueError(points)
    w = len(offs)
    cols = np.empty((n, w), np.int64)
    valid = np.empty((n, w), bool)
    for k, (dz, dy, dx) in enumerate(offs):
        valid[:, k] = ((x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
                       & (z + dz >= 0) & (z + dz < nz))
        cols[:, k] = idx + (dz * ny + dy) * nx + dx
    return _from_offsets(n, cols, valid, n, f"stencil{points}_{nx}x{ny}x{nz}")


def stencil_2d(nx: int, ny: int) -> CSRMatrix:
    """5-point stencil, row-major numbering i = y*nx + x, Dirichlet."""
    n = nx * ny
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = idx // nx
    offs = [(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)]
    cols = np.empty((n, 5), np.int64)
    valid = np.empty((n, 5), bool)
    for k, (dy, dx) in enumerate(offs):
        valid[:, k] = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
        cols[:, k] = idx + dy * nx + dx
    return _from_offsets(n, cols, valid, n, f"stencil5_{nx}x{ny}")


def _laplacian_values(A: CSRMatrix, diag: float) -> np.ndarray:
    rows = np.repeat(np.arange(A.n_rows, dtype=np.int64), A.row_lengths())
    return np.where(A.col.astype(np.int64) == rows, diag, -1.0).astype(np.float64)


def laplacian_2d(nx: int, ny: int | None = None) -> CSRMatrix:
    """2D 5-point Laplacian: 4 on the diagonal, -1 off (Dirichlet)."""
    A = stencil_2d(nx, ny or nx)
    A.val = _laplacian_values(A, 4.0)
    A.name = f"laplace2d_{nx}x{ny or nx}"
    return A


def laplacian_3d(nx: int, ny: int | None = None, nz: int | None = None) -> CSRMatrix:
    """3D 7-point Laplacian: 6 on the diagonal, -1 off (Dirichlet)."""
    A = stencil_3d(nx, ny or nx, nz or nx, 7)
    A.val = _laplacian_values(A, 6.0)
    A.name = f"laplace3d_{nx}x{ny or nx}x{nz or nx}"
    return A


def stencil27_random(nx: int, seed: int = 0) -> CSRMatrix:
    """27-point stencil on an nx^3 grid with values uniform in [-1, 1]."""
    A = stencil_3d(nx, nx, nx, 27)
    rng = np.random.default_rng(seed)
    A.val = rng.uniform(-1.0, 1.0, A.nnz)
    A.name = f"stencil27_{nx}^3"
    return A


def _distinct_sorted_columns(rng, lengths: np.ndarray, n_cols: int) -> np.ndarray:
    """Per row, lengths[i] distinct columns uniform in [0, n_cols), sorted.

    Rows longer than n_cols / 8 draw a partial permutation; the others draw
    with replacement and redraw duplicates until none are left."""
    lengths = np.asarray(lengths, dtype=np.int64)
    n = lengths.size
    dense = lengths > n_cols // 8
    Ls = np.where(dense, 0, lengths)
    nnz = int(Ls.sum())
    rows = np.repeat(np.arange(n, dtype=np.int64), Ls)
    cols = rng.integers(0, n_cols, nnz, dtype=np.int64)
    while nnz:
        key = rows * n_cols + cols
        order = np.argsort(key, kind="stable")
        key = key[order]
        cols = cols[order]
        dup = np.zeros(nnz, bool)
        dup[1:] = key[1:] == key[:-1]
        nd = int(dup.sum())
        if nd == 0:
            break
        cols[dup] = rng.integers(0, n_cols, nd, dtype=np.int64)
    if not dense.any():
        return cols.astype(np.int32)
    out = np.empty(int(lengths.sum()), np.int32)
    ptr = np.zeros(n + 1, np.int64)
    np.cumsum(lengths, out=ptr[1:])
    sparse_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(Ls, out=sparse_ptr[1:])
    for i in range(n):
        if dense[i]:
            out[ptr[i]:ptr[i + 1]] = np.sort(rng.choice(n_cols, int(lengths[i]), replace=False))
        else:
            out[ptr[i]:ptr[i + 1]] = cols[sparse_ptr[i]:sparse_ptr[i + 1]]
    return out


def power_law_lengths(n: int, rng, s: float = 2.0, scale: float = 2.69,
                      lmax: int = 10000) -> np.ndarray:
    """Row lengths L = clip(ceil(scale * k), 1, lmax) with k ~ Zipf(s)
    truncated to [1, lmax] (draws above lmax are redrawn)."""
    k = rng.zipf(s, n)
    bad = k > lmax
    while bad.any():
        k[bad] = rng.zipf(s, int(bad.sum()))
        bad = k > lmax
    return np.clip(np.ceil(scale * k).astype(np.int64), 1, lmax)


def power_law(n: int, seed: int = 0, s: float = 2.0, scale: float = 2.69,
              lmax: int = 10000, n_cols: int | None = None) -> CSRMatrix:
    """Power-law rows (mean length ~16, longest 10,000 at n = 10^6), distinct
    uniform random columns, values N(0, 1), rows in natural order."""
    m = n if n_cols is None else n_cols
    rng = np.random.default_rng(seed)
    L = power_law_lengths(n, rng, s, scale, min(lmax, m))
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(L, out=rowptr[1:])
    col = _distinct_sorted_columns(rng, L, m)
    val = rng.standard_normal(int(rowptr[-1]))
    return CSRMatrix(n, m, rowptr, col, val, f"powerlaw_{n}_s{seed}")


def banded(n: int, bandwidth: int, seed: int = 0) -> CSRMatrix:
    """Centred band of `bandwidth` (odd) diagonals, values U[-1, 1]."""
    h = bandwidth // 2
    idx = np.arange(n, dtype=np.int64)
    offs = np.arange(-h, h + 1, dtype=np.int64)
    cols = idx[:, None] + offs[None, :]
    valid = (cols >= 0) & (cols < n)
    A = _from_offsets(n, cols, valid, n, f"banded_{n}_bw{bandwidth}")
    A.val = np.random.default_rng(seed).uniform(-1.0, 1.0, A.nnz)
    return A


def random_csr(n: int, m: int, lengths, seed: int = 0, values: str = "normal") -> CSRMatrix:
    """Given row lengths (each <= m), distinct sorted uniform columns."""
    rng = np.random.default_rng(seed)
    L = np.asarray(lengths, dtype=np.int64)
    assert L.size == n and (L <= m).all() and (L >= 0).all()
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(L, out=rowptr[1:])
    col = _distinct_sorted_columns(rng, L, m) if rowptr[-1] else np.zeros(0, np.int32)
    nnz = int(rowptr[-1])
    if values == "normal":
        val = rng.standard_normal(nnz)
    elif values == "uniform":
        val = rng.uniform(-1.0, 1.0, nnz)
    else:
        raise ValueError(values)
    return CSRMatrix(n, m, rowptr, col, val, f"random_{n}x{m}_s{seed}")


def uniform_vector(n: int, seed: int = 0, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, n)


def uniform_matrix(n: int, k: int, seed: int = 0) -> np.ndarray:
    """Row-major [n, k] block of right-hand sides, U[-1, 1]."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, (n, k))


# Row statistics of the four matrices that Sec. 4.4.2 (Table 6) analyses:
# rows, longest, mean and shortest row length.  The matrices themselves
# (Hohn/fd18, AMD/G2_circuit, IBM_EDA/trans4 and Rajat/Raj1 of the UF
# collection) are not available here; the stand-ins match these numbers.
TABLE6_ROWS = {
    "fd18": (16_248, 6, 3.860, 1),
    "G2_circuit": (150_102, 6, 4.841, 2),
    "trans4": (116_835, 114_190, 6.600, 1),
    "Raj1": (263_743, 40_468, 4.938, 1),
}


def row_statistics_lengths(n: int, lmax: int, mean: float, lmin: int, rng) -> np.ndarray:
    """n row lengths with longest lmax, shortest lmin and total round(mean n):
    one row of lmax at a random position; the others lmin + Geometric - 1
    with the mean the total needs, clipped to [lmin, min(lmax, 64)] and then
    moved one entry at a time (random rows) until the total is met."""
    total = int(round(mean * n))
    cap = min(lmax, 64)
    rest = total - lmax
    if not (lmin * (n - 1) <= rest <= cap * (n - 1)):
        raise ValueError("statistics not reachable")
    target = rest / (n - 1)
    L = np.clip(lmin - 1 + rng.geometric(1.0 / (target - lmin + 1.0), n - 1), lmin, cap).astype(np.int64)
    diff = rest - int(L.sum())
    while diff:
        cand = np.flatnonzero(L < cap) if diff > 0 else np.flatnonzero(L > lmin)
        pick = rng.choice(cand, min(abs(diff), cand.size), replace=False)
        L[pick] += 1 if diff > 0 else -1
        diff = rest - int(L.sum())
    if L.min() > lmin:                       # keep one shortest row (moving its entries elsewhere)
        i = int(np.argmin(L))
        extra = int(L[i]) - lmin
        L[i] = lmin
        room = np.flatnonzero(L < cap)
        L[rng.choice(room, extra, replace=False)] += 1
    return np.insert(L, int(rng.integers(0, n)), lmax)


def table6_standin(name: str, seed: int = 0, window: int = 65) -> CSRMatrix:
    """Square stand-in for a Table 6 matrix.  Rows of at most 64 entries take
    distinct sorted columns from a window of `window` columns around the
    diagonal (local coupling, as in these PDE and circuit matrices); the
    longest row takes distinct columns over the whole range.  Values
    U[-1, 1]."""
    n, lmax, mean, lmin = TABLE6_ROWS[name]
    rng = np.random.default_rng(seed)
    L = row_statistics_lengths(n, lmax, mean, lmin, rng)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(L, out=rowptr[1:])
    col = np.empty(int(rowptr[-1]), np.int32)
    short = L <= min(64, window)
    rows = np.flatnonzero(short)
    local = _distinct_sorted_columns(rng, L[short], window).astype(np.int64)
    start = np.clip(rows - window // 2, 0, max(0, n - window))
    dst = np.concatenate([np.arange(rowptr[i], rowptr[i + 1]) for i in rows]) if rows.size else np.zeros(0, np.int64)
    col[dst] = (np.repeat(start, L[short]) + local).astype(np.int32)
    for i in np.flatnonzero(~short):
        col[rowptr[i]:rowptr[i + 1]] = np.sort(rng.choice(n, int(L[i]), replace=False))
    val = rng.uniform(-1.0, 1.0, int(rowptr[-1]))
    return CSRMatrix(n, n, rowptr, col, val, f"table6_{name}_s{seed}")


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------
def workload_small_laplacian() -> CSRMatrix:
    """2D 5-point Laplacian on a 64 x 64 grid (n = 4,096, nnz = 20,224)."""
    return laplacian_2d(64, 64)


def workload_a(scale: int = 128) -> CSRMatrix:
    """(a) 3D 7-point Laplacian 128^3 (n = 2,097,152, nnz = 14,581,760)."""
    return laplacian_3d(scale)


def workload_b(n: int = 1_000_000, seed: int = 0) -> CSRMatrix:
    """(b) power-law rows, n = 10^6, Zipf(2) lengths clipped to [1, 10^4]."""
    return power_law(n, seed)


def workload_c(scale: int = 96, seed: int = 0) -> CSRMatrix:
    """(c) 27-point stencil 96^3, values U[-1, 1] (nnz = 286^3)."""
    return stencil27_random(scale, seed)


def batch_member(i: int, seed_base: int = 1000, n_min: int = 1000,
                 n_max: int = 200_000) -> CSRMatrix:
    """Member i of the uneven batch: n log-uniform in [n_min, n_max]; kind by
    i mod 3: banded (odd bandwidth 5..101), stencil (2D 5-point if n is a
    perfect square, else 3D 7-point on the largest cube <= n), power-law."""
    rng = np.random.default_rng(seed_base + i)
    n = int(math.floor(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
    kind = i % 3
    if kind == 0:
        bw = int(rng.integers(2, 51)) * 2 + 1          # odd, 5..101
        A = banded(n, bw, seed=seed_base + i)
    elif kind == 1:
        r = int(math.isqrt(n))
        if r * r == n:
            A = laplacian_2d(r, r)
        else:
            c = int(round(n ** (1.0 / 3.0)))
            while c ** 3 > n:
                c -= 1
            A = laplacian_3d(c, c, c)
        A.val = np.random.default_rng(seed_base + i).uniform(-1.0, 1.0, A.nnz)
    else:
        A = power_law(n, seed=seed_base + i)
    A.name = f"batch{i}_{A.name}"
    return A


def workload_batch(count: int = 512, seed_base: int = 1000, n_min: int = 1000,
                   n_max: int = 200_000) -> list[CSRMatrix]:
    return [batch_member(i, seed_base, n_min, n_max) for i in range(count)]


# ---------------------------------------------------------------------------
# A matrix with more than 2^31 stored slots (the 64-bit slot offsets of the
# group pointers).  Every row holds exactly `length` entries given by closed
# forms, so that the whole matrix can be generated on the device in bulk
# (host arrays of that size would be unwieldy) and any sampled row again on
# the host.
# ---------------------------------------------------------------------------
_UA, _UB = 7919, 104729


def uniform_rows_entries(rows, length: int, n_cols: int) -> tuple[np.ndarray, np.ndarray]:
    """Columns [len(rows), length] int32 and values float64 of the given rows:
    entry j of row i has column (7919 i + 104729 j) mod n_cols and value
    ((i + 3 j) mod 17 - 8) / 16 (exact in binary32 and below)."""
    i = np.asarray(rows, dtype=np.int64)[:, None]
    j = np.arange(length, dtype=np.int64)[None, :]
    col = ((_UA * i + _UB * j) % n_cols).astype(np.int32)
    val = (((i + 3 * j) % 17) - 8).astype(np.float64) / 16.0
    return col, val


def uniform_rows_device(n: int, length: int, n_cols: int, device="cuda", chunk: int = 1 << 22):
    """The n-row matrix of uniform_rows_entries as torch tensors on `device`:
    rowptr int64 [n+1], col int32 [n*length], val float32 [n*length]."""
    import torch
    rowptr = torch.arange(n + 1, dtype=torch.int64, device=device) * length
    col = torch.empty(n * length, dtype=torch.int32, device=device)
    val = torch.empty(n * length, dtype=torch.float32, device=device)
    j = torch.arange(length, dtype=torch.int64, device=device)[None, :]
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        i = torch.arange(r0, r1, dtype=torch.int64, device=device)[:, None]
        col[r0 * length:r1 * length] = ((_UA * i + _UB * j) % n_cols).to(torch.int32).reshape(-1)
        val[r0 * length:r1 * length] = ((((i + 3 * j) % 17) - 8).to(torch.float32) / 16.0).reshape(-1)
    return rowptr, col, val


def uniform_x(n: int, shift: int = 0) -> np.ndarray:
    """x_k = ((5 k + shift) mod 23 - 11) / 32, float32 (exact)."""
    k = np.arange(n, dtype=np.int64)
    return ((((5 * k + shift) % 23) - 11) / 32.0).astype(np.float32)
