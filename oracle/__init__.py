"""CPU oracle for Row-grouped CSR (RgCSR) SpMV -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct FP64 reference for everything the GPU path
computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the product library never does,
and this package never imports the product.  The arithmetic lives in
``oracle.c`` (plain C loops); this module only marshals numpy arrays.

Paper sections followed (Oberhuber, Suzuki, Vacata, "New Row-grouped CSR
format for storing the sparse matrices on GPU with implementation in CUDA"):

* Sec. 3.1  -- CSR format and the sequential CSR SpMV (``csr_spmv``).
* Sec. 3.3  -- Hybrid ELLPACK + COO (``hyb_layout``, ``hyb_spmv``).
* Sec. 3.4  -- RgCSR layout, its SpMV kernel semantics, sliced ELLPACK
  (``rgcsr_layout``, ``rgcsr_spmv``, ``sliced_ell_spmv``).
* Sec. 4.3  -- artificial-zero percentage (``artificial_zero_percent``).
* Sec. 4.4.2, Table 7 -- descending row-length ordering (``descending_order``)
  and layouts over reordered rows (``permute_rows``, ``rgcsr_layout(row_order=)``).
* Not in the paper (forms added on top of the method): per-row-scaled
  bf16/fp16 value storage, transposition and gradients, damped Jacobi,
  conjugate gradients.

Parity status: all functions are pinned by ``tests/test_oracle_*.py`` against
the paper's worked-example counts, dense products, closed forms, brute force
and finite differences.  The HYB default ELL width is a project rule (the
paper gives none); its layout for any given width is pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    # -ffp-contract=off: no fused multiply-add, every product is rounded
    # before the sum, exactly as the loops are written.
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    sig = {
        "orc_csr_spmv": (None, [I64, P, P, P, P, P, P]),
        "orc_csr_spmm": (None, [I64, I64, P, P, P, P, P, P]),
        "orc_rgcsr_sizes": (I64, [I64, P, I64, P, P]),
        "orc_rgcsr_fill": (None, [I64, P, P, P, I64, I64, P, P, P, P, P]),
        "orc_rgcsr_spmv": (None, [I64, I64, P, P, P, P, P, P]),
        "orc_sliced_ell_spmv": (None, [I64, I64, P, P, P, P, P]),
        "orc_descending_order": (None, [I64, P, P]),
        "orc_hyb_coo_count": (I64, [I64, P, I64]),
        "orc_hyb_choose_k1": (I64, [I64, P, I64, I64]),
        "orc_hyb_fill": (None, [I64, P, P, P, I64, I64, P, P, P, P, P]),
        "orc_hyb_spmv": (None, [I64, I64, P, P, I64, P, P, P, P, P]),
        "orc_row_scale": (ctypes.c_float, [ctypes.c_double]),
        "orc_round_bf16": (ctypes.c_uint16, [ctypes.c_double]),
        "orc_round_f16": (ctypes.c_uint16, [ctypes.c_double]),
        "orc_decode_bf16": (ctypes.c_double, [ctypes.c_uint16]),
        "orc_decode_f16": (ctypes.c_double, [ctypes.c_uint16]),
        "orc_quantize_rows": (None, [I64, P, P, ctypes.c_int, P, P]),
        "orc_csr_transpose": (None, [I64, I64, P, P, P, P, P]),
        "orc_spmm_grad_values": (None, [I64, I64, P, P, P, P, P]),
        "orc_jacobi": (None, [I64, P, P, P, P, P, ctypes.c_double, I64, P]),
        "orc_jacobi_grad": (ctypes.c_double, [I64, P, P, P, P, P, ctypes.c_double, I64, P, P]),
        "orc_jacobi_grad_bound": (None, [I64, P, P, P, P, P, ctypes.c_double, I64, ctypes.c_double, P, P]),
        "orc_cg": (I64, [I64, P, P, P, P, ctypes.c_double, I64, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(rowptr, col, val=None):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if val is None:
        return rowptr, col
    return rowptr, col, np.ascontiguousarray(val, dtype=np.float64)


# --------------------------------------------------------------------------
# Sec. 3.1: CSR SpMV (and the same definition for k right-hand sides)
# --------------------------------------------------------------------------
def csr_spmv(rowptr, col, val, x):
    """y = A x in FP64, summed in stored order; also returns |A||x|."""
    rowptr, col, val = _csr(rowptr, col, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = rowptr.size - 1
    y = np.empty(n, np.float64)
    ay = np.empty(n, np.float64)
    _load().orc_csr_spmv(n, _p(rowptr), _p(col), _p(val), _p(x), _p(y), _p(ay))
    return y, ay


def csr_spmm(rowptr, col, val, X):
    """Y = A X for row-major X [m, k]; also returns |A||X|."""
    rowptr, col, val = _csr(rowptr, col, val)
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = rowptr.size - 1
    k = X.shape[1]
    Y = np.empty((n, k), np.float64)
    aY = np.empty((n, k), np.float64)
    _load().orc_csr_spmm(n, k, _p(rowptr), _p(col), _p(val), _p(X), _p(Y), _p(aY))
    return Y, aY


# --------------------------------------------------------------------------
# Sec. 3.4: RgCSR layout and SpMV
# --------------------------------------------------------------------------
@dataclass
class RgCSRLayout:
    n: int
    group_size: int
    row_lengths: np.ndarray   # int32 [n]
    group_ptr: np.ndarray     # int64 [n_groups + 1]
    values: np.ndarray        # [n_stored], dtype of the input values
    columns: np.ndarray       # int32 [n_stored]
    slot_to_csr: np.ndarray   # int64 [n_stored], -1 for padding
    row_perm: np.ndarray | None = None   # stored row k holds CSR row row_perm[k]

    @property
    def n_stored(self) -> int:
        return int(self.group_ptr[-1])


def rgcsr_sizes(rowptr, group_size: int):
    """rowLengths and groupPointers only (Sec. 3.4), without the slabs."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    n = rowptr.size - 1
    G = int(group_size)
    rl = np.empty(n, np.int32)
    gp = np.empty((n + G - 1) // G + 1, np.int64)
    _load().orc_rgcsr_sizes(n, _p(rowptr), G, _p(rl), _p(gp))
    return rl, gp


def permute_rows(rowptr, col, val, perm):
    """The CSR of P A: row k of the result is row perm[k] of A, its entries
    in their CSR order.  Also returns, per entry of the result, its position
    in A's arrays."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    perm = np.ascontiguousarray(perm, dtype=np.int64)
    n = rowptr.size - 1
    if perm.size != n or not np.array_equal(np.sort(perm), np.arange(n)):
        raise ValueError("perm is not a permutation of the rows")
    new_ptr = np.zeros(n + 1, np.int64)
    source = []
    for k in range(n):
        i = perm[k]
        source.append(np.arange(rowptr[i], rowptr[i + 1], dtype=np.int64))
        new_ptr[k + 1] = new_ptr[k] + (rowptr[i + 1] - rowptr[i])
    source = np.concatenate(source) if n else np.zeros(0, np.int64)
    return new_ptr, np.asarray(col)[source], np.asarray(val)[source], source


def rgcsr_layout(rowptr, col, val, group_size: int, row_order=None) -> RgCSRLayout:
    """CSR -> RgCSR (Sec. 3.4).  ``val`` keeps its dtype; values are copied
    bit for bit, padding is all-zero bits with column 0.

    ``row_order`` (a permutation; Sec. 4.4.2, Table 7): the groups are
    formed over the rows in that order, i.e. the layout is that of P A
    (``permute_rows``), and slot_to_csr still points into A's arrays."""
    if row_order is not None:
        prp, pcol, pval, source = permute_rows(rowptr, col, val, row_order)
        lay = rgcsr_layout(prp, pcol, pval, group_size)
        s2c = np.where(lay.slot_to_csr >= 0, source[np.maximum(lay.slot_to_csr, 0)], -1)
        return RgCSRLayout(lay.n, lay.group_size, lay.row_lengths, lay.group_ptr, lay.values,
                           lay.columns, s2c, np.ascontiguousarray(row_order, dtype=np.int64))
    rowptr, col = _csr(rowptr, col)
    val = np.ascontiguousarray(val)
    n = rowptr.size - 1
    G = int(group_size)
    if G < 1:
        raise ValueError("group size must be >= 1")
    n_groups = (n + G - 1) // G
    rl = np.empty(n, np.int32)
    gp = np.empty(n_groups + 1, np.int64)
    lib = _load()
    n_stored = lib.orc_rgcsr_sizes(n, _p(rowptr), G, _p(rl), _p(gp))
    values = np.empty(n_stored, val.dtype)
    columns = np.empty(n_stored, np.int32)
    s2c = np.empty(n_stored, np.int64)
    lib.orc_rgcsr_fill(n, _p(rowptr), _p(col), _p(val), val.itemsize, G,
                       _p(gp), _p(rl), _p(values), _p(columns), _p(s2c))
    return RgCSRLayout(n, G, rl, gp, values, columns, s2c)


def rgcsr_spmv(layout: RgCSRLayout, x):
    """The Sec. 3.4 kernel's addressing, evaluated on the CPU in FP64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    vals = np.ascontiguousarray(layout.values, dtype=np.float64)
    y = np.empty(layout.n, np.float64)
    _load().orc_rgcsr_spmv(layout.n, layout.group_size, _p(layout.group_ptr),
                           _p(layout.row_lengths), _p(vals),
                           _p(layout.columns), _p(x), _p(y))
    if layout.row_perm is not None:      # stored row k is CSR row row_perm[k]
        out = np.empty_like(y)
        out[layout.row_perm] = y
        return out
    return y


def sliced_ell_spmv(layout: RgCSRLayout, x):
    """Sliced ELLPACK on the same slabs: all K_g slots of every row."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    vals = np.ascontiguousarray(layout.values, dtype=np.float64)
    y = np.empty(layout.n, np.float64)
    _load().orc_sliced_ell_spmv(layout.n, layout.group_size, _p(layout.group_ptr),
                                _p(vals), _p(layout.columns), _p(x), _p(y))
    return y


def artificial_zero_percent(nnz: int, n_stored: int) -> float:
    """Sec. 4.3: 100% means as many artificial zeros as non-zeros."""
    return 100.0 * (n_stored - nnz) / nnz if nnz else 0.0


def descending_order(rowptr):
    """Stable permutation putting the longest rows first (Table 7)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    n = rowptr.size - 1
    perm = np.empty(n, np.int64)
    _load().orc_descending_order(n, _p(rowptr), _p(perm))
    return perm


# --------------------------------------------------------------------------
# Sec. 3.3: Hybrid ELLPACK + COO
# --------------------------------------------------------------------------
@dataclass
class HybLayout:
    n: int
    ell_width: int
    ell_val: np.ndarray   # [ell_width * n], column-major: slot j of row i at j*n+i
    ell_col: np.ndarray   # int32, -1 = padding
    coo_row: np.ndarray   # int32 [nnz_coo]
    coo_col: np.ndarray   # int32 [nnz_coo]
    coo_val: np.ndarray   # [nnz_coo]


def hyb_choose_ell_width(rowptr, value_bytes: int, index_bytes: int = 4) -> int:
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    return int(_load().orc_hyb_choose_k1(rowptr.size - 1, _p(rowptr), value_bytes, index_bytes))


def hyb_coo_count(rowptr, ell_width: int) -> int:
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    return int(_load().orc_hyb_coo_count(rowptr.size - 1, _p(rowptr), ell_width))


def hyb_layout(rowptr, col, val, ell_width: int) -> HybLayout:
    rowptr, col = _csr(rowptr, col)
    val = np.ascontiguousarray(val)
    n = rowptr.size - 1
    K1 = int(ell_width)
    nc = hyb_coo_count(rowptr, K1)
    ev = np.empty(K1 * n, val.dtype)
    ec = np.empty(K1 * n, np.int32)
    cr = np.empty(nc, np.int32)
    cc = np.empty(nc, np.int32)
    cv = np.empty(nc, val.dtype)
    _load().orc_hyb_fill(n, _p(rowptr), _p(col), _p(val), val.itemsize, K1,
                         _p(ev), _p(ec), _p(cr), _p(cc), _p(cv))
    return HybLayout(n, K1, ev, ec, cr, cc, cv)


def hyb_spmv(h: HybLayout, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    ev = np.ascontiguousarray(h.ell_val, dtype=np.float64)
    cv = np.ascontiguousarray(h.coo_val, dtype=np.float64)
    y = np.empty(h.n, np.float64)
    _load().orc_hyb_spmv(h.n, h.ell_width, _p(ev), _p(h.ell_col), h.coo_row.size,
                         _p(h.coo_row), _p(h.coo_col), _p(cv), _p(x), _p(y))
    return y


# --------------------------------------------------------------------------
# Reduced-precision value storage with a per-row power-of-two scale
# --------------------------------------------------------------------------
BF16, F16 = 0, 1


def row_scale(maxabs: float) -> float:
    return float(_load().orc_row_scale(float(maxabs)))


def round_bf16(v: float) -> int:
    return int(_load().orc_round_bf16(float(v)))


def round_f16(v: float) -> int:
    return int(_load().orc_round_f16(float(v)))


def decode(bits, fmt: int):
    lib = _load()
    f = lib.orc_decode_bf16 if fmt == BF16 else lib.orc_decode_f16
    bits = np.asarray(bits, dtype=np.uint16).ravel()
    return np.array([f(int(b)) for b in bits], dtype=np.float64)


def quantize_rows(rowptr, val, fmt: int):
    """Returns (q bits uint16 [nnz] in CSR order, scale float32 [n])."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    val = np.ascontiguousarray(val, dtype=np.float64)
    n = rowptr.size - 1
    q = np.empty(val.size, np.uint16)
    s = np.empty(n, np.float32)
    _load().orc_quantize_rows(n, _p(rowptr), _p(val), int(fmt), _p(q), _p(s))
    return q, s


def dequantized_values(rowptr, q, scale, fmt: int):
    """a_ij ~= s_i * decode(q_ij), in CSR order, FP64."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    dec = _decode_vec(q, fmt)
    rows = np.repeat(np.arange(rowptr.size - 1), np.diff(rowptr))
    return dec * scale.astype(np.float64)[rows]


def _decode_vec(q, fmt):
    # Bit-level decode for large arrays (same definition as the C decoder):
    # bf16 bits are the top half of a binary32; fp16 is IEEE binary16.
    q = np.asarray(q, dtype=np.uint16)
    if fmt == BF16:
        return (q.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return q.view(np.float16).astype(np.float64)


# --------------------------------------------------------------------------
# Transposition and gradients
# --------------------------------------------------------------------------
def csr_transpose(rowptr, col, n_cols: int):
    """CSR of A^T: (t_rowptr int64[m+1], t_col int32[nnz], perm int64[nnz])."""
    rowptr, col = _csr(rowptr, col)
    n = rowptr.size - 1
    nnz = int(rowptr[-1])
    trp = np.empty(n_cols + 1, np.int64)
    tc = np.empty(nnz, np.int32)
    perm = np.empty(nnz, np.int64)
    _load().orc_csr_transpose(n, n_cols, _p(rowptr), _p(col), _p(trp), _p(tc), _p(perm))
    return trp, tc, perm


def spmm_grads(rowptr, col, val, X, Gy, n_cols: int):
    """Gradients of Y = A X: (dX = A^T Gy, dval[p] = sum_b Gy[row_p,b] X[col_p,b])."""
    rowptr, col, val = _csr(rowptr, col, val)
    X = np.ascontiguousarray(X, dtype=np.float64)
    Gy = np.ascontiguousarray(Gy, dtype=np.float64)
    n = rowptr.size - 1
    k = X.shape[1]
    trp, tc, perm = csr_transpose(rowptr, col, n_cols)
    dX, _ = csr_spmm(trp, tc, val[perm], Gy)
    dval = np.empty(val.size, np.float64)
    _load().orc_spmm_grad_values(n, k, _p(rowptr), _p(col), _p(Gy), _p(X), _p(dval))
    return dX, dval


# --------------------------------------------------------------------------
# Repeated-SpMV workloads: damped Jacobi and CG (Krylov context of Sec. 1)
# --------------------------------------------------------------------------
def jacobi(rowptr, col, val, dinv, b, omega: float, steps: int):
    rowptr, col, val = _csr(rowptr, col, val)
    dinv = np.ascontiguousarray(dinv, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = rowptr.size - 1
    x = np.empty(n, np.float64)
    _load().orc_jacobi(n, _p(rowptr), _p(col), _p(val), _p(dinv), _p(b),
                       float(omega), int(steps), _p(x))
    return x


def jacobi_grad(rowptr, col, val, dinv, b, omega: float, steps: int):
    """loss = ||x_steps||^2 and (d loss/d b, d loss/d values) by the adjoint."""
    rowptr, col, val = _csr(rowptr, col, val)
    dinv = np.ascontiguousarray(dinv, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = rowptr.size - 1
    db = np.empty(n, np.float64)
    dval = np.empty(val.size, np.float64)
    loss = _load().orc_jacobi_grad(n, _p(rowptr), _p(col), _p(val), _p(dinv), _p(b),
                                   float(omega), int(steps), _p(db), _p(dval))
    return float(loss), db, dval


def jacobi_grad_bound(rowptr, col, val, dinv, b, omega: float, steps: int, u: float):
    """Elementwise bounds on the error of (d loss/d b, d loss/d values) of
    ``jacobi_grad`` when they are computed in a floating-point format with
    unit roundoff u (2**-24 for float), any summation order: the running
    error recursions of oracle.c (first order in u)."""
    rowptr, col, val = _csr(rowptr, col, val)
    dinv = np.ascontiguousarray(dinv, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = rowptr.size - 1
    db = np.empty(n, np.float64)
    dval = np.empty(val.size, np.float64)
    _load().orc_jacobi_grad_bound(n, _p(rowptr), _p(col), _p(val), _p(dinv), _p(b), float(omega), int(steps),
                                  float(u), _p(db), _p(dval))
    return db, dval


def cg(rowptr, col, val, b, tol: float, maxit: int):
    rowptr, col, val = _csr(rowptr, col, val)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = rowptr.size - 1
    x = np.empty(n, np.float64)
    it = _load().orc_cg(n, _p(rowptr), _p(col), _p(val), _p(b), float(tol), int(maxit), _p(x))
    return x, int(it)


# --------------------------------------------------------------------------
# Peak-performance model (Sec. 3.4, the peak-estimate table)
# --------------------------------------------------------------------------
def peak_gflops(bandwidth_gbs: float, value_bytes: int, index_bytes: int = 4,
                x_cached: bool = False) -> float:
    """Two flops per non-zero; bytes per non-zero = value + column index, plus
    one x element unless x is served from a cache."""
    per_nnz = value_bytes + index_bytes + (0 if x_cached else value_bytes)
    return 2.0 * bandwidth_gbs / per_nnz
