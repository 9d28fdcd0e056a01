"""Pins for the oracle's per-row power-of-two scale and round-to-nearest-even
bf16/fp16 encoders: closed forms, exhaustive round trips over every 16-bit
pattern, numpy's independent double->half conversion, a direct-vs-double
rounding case, and the quantisation error bound."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("mx,s", [(0.0, 1.0), (1.0, 1.0), (0.75, 1.0), (1.5, 2.0), (3.0, 4.0),
                                  (4.0, 4.0), (4.000001, 8.0), (1e-3, 2.0 ** -9),
                                  (2.0 ** -20, 2.0 ** -20), (6.0, 8.0), (1e30, 2.0 ** 100),
                                  # exponent clamped to the binary32 normal range
                                  (1e-45, 2.0 ** -126), (2.0 ** -126, 2.0 ** -126),
                                  (2.0 ** 127, 2.0 ** 127), (1e300, 2.0 ** 127)])
def test_row_scale_closed_form(mx, s):
    assert oracle.row_scale(mx) == s


def test_decode_all_patterns_match_ieee():
    bits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    dec16 = oracle.decode(bits, oracle.F16)
    ref16 = bits.view(np.float16).astype(np.float64)
    same = (dec16 == ref16) | (np.isnan(dec16) & np.isnan(ref16))
    assert same.all()
    decb = oracle.decode(bits, oracle.BF16)
    with np.errstate(invalid="ignore"):            # signalling-NaN patterns widen to quiet NaNs
        refb = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    same = (decb == refb) | (np.isnan(decb) & np.isnan(refb))
    assert same.all()


@pytest.mark.parametrize("fmt", [oracle.BF16, oracle.F16])
def test_round_trip_every_finite_pattern(fmt):
    rnd = oracle.round_bf16 if fmt == oracle.BF16 else oracle.round_f16
    for b in range(65536):
        v = oracle.decode([b], fmt)[0]
        if np.isfinite(v):
            assert rnd(v) == b, (b, v)


def test_f16_matches_numpy_on_midpoints_and_randoms():
    bits = np.arange(0, 0x7C00, dtype=np.uint16)            # positive finite halves
    v = bits.view(np.float16).astype(np.float64)
    mids = (v[:-1] + v[1:]) / 2                              # exact ties
    rng = np.random.default_rng(0)
    rand = rng.uniform(-1, 1, 20000) * 2.0 ** rng.integers(-30, 1, 20000)
    for arr in (mids, -mids, rand, mids * (1 + 2 ** -40), mids * (1 - 2 ** -40)):
        for a in arr:
            assert oracle.round_f16(a) == int(np.float16(a).view(np.uint16)), a


def test_bf16_is_direct_rounding_not_double_rounding():
    # 1 + 2^-8 + 2^-30 lies just above the bf16 midpoint 1 + 2^-8; rounding
    # through binary32 first would drop 2^-30 and tie to 1.0.
    assert oracle.round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -30) == 0x3F81
    assert oracle.round_bf16(1.0 + 2.0 ** -8) == 0x3F80           # tie to even
    assert oracle.round_bf16(1.0 + 3 * 2.0 ** -8) == 0x3F82       # tie to even (up)
    assert oracle.round_bf16(-0.0) == 0x8000
    # the textbook float32 -> bf16 rule agrees on binary32 inputs
    rng = np.random.default_rng(1)
    f = (rng.standard_normal(20000) * 2.0 ** rng.integers(-40, 40, 20000)).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    ref = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    got = np.array([oracle.round_bf16(float(a)) for a in f], dtype=np.uint16)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("fmt,ulp", [(oracle.BF16, 2.0 ** -9), (oracle.F16, 2.0 ** -11)])
def test_quantize_rows_error_bound(fmt, ulp):
    rng = np.random.default_rng(2)
    n = 200
    L = rng.integers(0, 40, n)
    rowptr = np.concatenate([[0], np.cumsum(L)])
    val = rng.standard_normal(int(rowptr[-1])) * 2.0 ** rng.integers(-3, 4, int(rowptr[-1]))
    q, s = oracle.quantize_rows(rowptr, val, fmt)
    deq = oracle.dequantized_values(rowptr, q, s, fmt)
    for i in range(n):
        seg = slice(rowptr[i], rowptr[i + 1])
        if L[i] == 0:
            assert s[i] == 1.0
            continue
        mx = np.abs(val[seg]).max()
        assert s[i] >= mx and s[i] < 2 * mx
        err = np.abs(deq[seg] - val[seg])
        if fmt == oracle.F16:
            # below the fp16 normal range the quantum is fixed at 2^-24 * s
            tiny = np.abs(val[seg]) < 2.0 ** -14 * s[i]
            assert (err[tiny] <= 2.0 ** -25 * s[i]).all()
            err = err[~tiny]
        assert (err <= ulp * s[i] * 1.0000001).all()
