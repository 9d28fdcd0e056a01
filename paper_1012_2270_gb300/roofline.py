"""Algorithmic byte counts of one SpMV, the quantity the HBM roofline is
measured in.  They extend the paper's peak model (Sec. 3.4, peak-estimate
table: 2 flops per non-zero; per non-zero one value, one column index and
one x element, or no x element when x is served from a cache) with the
format's metadata and the one pass over x and y that any SpMV needs.
Padding (artificial zeros) is excluded: it is overhead of the format, not
work of the method."""
from __future__ import annotations

INDEX_BYTES = 4

# nominal HBM3e bandwidth used for the "% of 8 TB/s" figure
NOMINAL_HBM_GBS = 8000.0

# nominal FP64 rate of a GB300 (vector and tensor alike): an FP64 SpMV does
# one FMA (2 flops) per non-zero, so this is its arithmetic ceiling
NOMINAL_FP64_TFLOPS = 1.25


def rgcsr_spmv_bytes(n_rows: int, n_cols: int, nnz: int, n_groups: int, value_bytes: int,
                     x_bytes: int | None = None, row_scale: bool = False) -> int:
    """values + columns of the non-zeros, rowLengths, groupPointers, x once,
    y once (+ one float scale per row for reduced-precision storage)."""
    xb = value_bytes if x_bytes is None else x_bytes
    b = (nnz * (value_bytes + INDEX_BYTES) + n_rows * 4 + (n_groups + 1) * 8
         + n_cols * xb + n_rows * xb)
    if row_scale:
        b += n_rows * 4
    return b


def hyb_spmv_bytes(n_rows: int, n_cols: int, nnz: int, nnz_coo: int, value_bytes: int) -> int:
    """The same count for HYB: ELL and COO entries carry value + column, COO
    entries also their row index; x once, y once."""
    return (nnz * (value_bytes + INDEX_BYTES) + nnz_coo * INDEX_BYTES
            + n_cols * value_bytes + n_rows * value_bytes)


def spmm_bytes(n_rows: int, n_cols: int, nnz: int, n_groups: int, value_bytes: int, k: int,
               x_bytes: int | None = None) -> int:
    """Multiple right-hand sides: matrix once, X [n_cols x k] once, Y once
    (X and Y elements of the value type, or x_bytes for reduced-precision
    storage)."""
    xb = value_bytes if x_bytes is None else x_bytes
    return (nnz * (value_bytes + INDEX_BYTES) + n_rows * 4 + (n_groups + 1) * 8
            + k * (n_cols + n_rows) * xb)


def peak_gflops(bandwidth_gbs: float, value_bytes: int, x_cached: bool = False) -> float:
    """The paper's model: 2 flops per non-zero at (value + index [+ x]) bytes."""
    per_nnz = value_bytes + INDEX_BYTES + (0 if x_cached else value_bytes)
    return 2.0 * bandwidth_gbs / per_nnz
