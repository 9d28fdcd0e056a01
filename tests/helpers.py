"""Shared helpers of the parity tests: moving oracle inputs to the GPU and the
elementwise error bound |y - y_ref|_i <= tau * (|A||x|)_i."""
import numpy as np

# tolerances of the parity bar, per storage type of the values
TAU = {"f64": 1e-12, "f32": 2e-6, "bf16": 1e-2, "f16": 1e-2}


def rounded_values(val: np.ndarray, dtype: str) -> np.ndarray:
    """The values the GPU actually stores, promoted back to float64."""
    if dtype == "f32":
        return val.astype(np.float32).astype(np.float64)
    return val.astype(np.float64)


def assert_within_bound(y, y_ref, absy, tau, what=""):
    y = np.asarray(y, dtype=np.float64)
    err = np.abs(y - y_ref)
    bound = tau * absy
    bad = err > bound
    if bad.any():
        i = int(np.argmax(err - bound))
        raise AssertionError(
            f"{what}: {int(bad.sum())} rows exceed tau*|A||x| (tau={tau}); worst row {i}: "
            f"y={y[i]!r} ref={y_ref[i]!r} err={err[i]:.3e} bound={bound[i]:.3e}")
    zero = absy == 0
    assert (y[zero] == 0).all(), f"{what}: rows with |A||x| = 0 must be exactly 0"
