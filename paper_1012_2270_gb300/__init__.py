"""Row-grouped CSR (RgCSR) sparse matrix-vector multiplication for NVIDIA
GB300 (sm_103a): hand-written CUDA kernels behind a C ABI (librgcsr.so,
declared in include/rgcsr.h) and a thin PyTorch-facing layer.

    from paper_1012_2270_gb300 import RgCSRMatrix
    A = RgCSRMatrix.from_csr(rowptr, col, val, n_cols, group_size=32, dtype=torch.float32)
    y = A @ x
"""
__all__ = ["RgCSRMatrix", "HybMatrix", "synth", "build"]


def __getattr__(name):
    if name in ("RgCSRMatrix", "HybMatrix"):
        from . import rgcsr
        return getattr(rgcsr, name)
    raise AttributeError(name)
