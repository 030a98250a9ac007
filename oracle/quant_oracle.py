"""Oracle of the lossy vector storage forms: what a stored row decodes to.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` may import this module.  It shares no code with
the CUDA library in ``paper_1603_09320_gb300``.

The paper defines no reduced-precision storage (Section 5.4 only mentions
integer distance functions for its SIFT 200M run); the storage forms are an
addition of this library.  Each is written out here from its number format:

* bf16: the fp32 value rounded to 8 significant bits (1 sign, 8 exponent,
  7 stored mantissa bits), round to nearest, ties to even;
* f16: IEEE-754 binary16, round to nearest, ties to even (numpy's conversion
  is that definition and serves as the step);
* fp8-e4m3 (the "fn" variant: 1 sign, 4 exponent bits with bias 7, 3 mantissa
  bits, no infinities, S.1111.111 is NaN, so the largest finite value is
  1.75 * 2^8 = 448; exponent field 0 holds the subnormals m/8 * 2^-6), with
  one fp32 scale per row: s = max_i |x_i| / 448 in fp32 (1 for an all-zero
  row), code_i = e4m3(x_i / s) with the fp32 quotient rounded to nearest,
  ties to even, and magnitudes above 448 saturated to 448; the row decodes to
  fp32(value(code_i) * s).

Search distances over a quantised index are the distances to these decoded
rows, accumulated in fp32 by the kernel (fp64 here).  parity pinned by
tests/test_quant_oracle.py: library conversions (torch's bfloat16 and
float8_e4m3fn casts) and hand-worked values of each format.
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def bf16_round(x) -> np.ndarray:
    """fp32 -> the nearest bf16 value (ties to even), returned as fp32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    hi, lo = u >> 16, u & 0xFFFF
    up = (lo > 0x8000) | ((lo == 0x8000) & ((hi & 1) == 1))
    return ((hi + up.astype(np.uint64)) << 16).astype(np.uint32).view(np.float32)


def f16_round(x) -> np.ndarray:
    """fp32 -> the nearest binary16 value (ties to even), returned as fp32."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def e4m3_magnitudes() -> np.ndarray:
    """Value of every non-negative finite e4m3 code 0..126 (ascending), fp64."""
    c = np.arange(127)
    e, m = c >> 3, c & 7
    return np.where(e == 0, m / 8.0 * 2.0 ** -6, (1.0 + m / 8.0) * 2.0 ** (e - 7.0))


def e4m3_encode(v) -> np.ndarray:
    """fp32 values -> e4m3 codes (uint8): nearest magnitude, ties to the even
    code, magnitudes of 448 and above saturated to 448, sign in bit 7."""
    v = np.asarray(v, dtype=np.float32)
    a = np.abs(v).astype(np.float64).ravel()
    mags = e4m3_magnitudes()
    code = np.empty(a.shape, dtype=np.int64)
    sat = a >= E4M3_MAX
    code[sat] = 126
    b = a[~sat]
    hi = np.searchsorted(mags, b, side="left")  # mags[hi-1] < b <= mags[hi]
    lo = np.maximum(hi - 1, 0)
    exact = mags[hi] == b
    d_lo, d_hi = b - mags[lo], mags[hi] - b  # exact: b has 24 bits, mags 4
    pick_hi = (d_hi < d_lo) | ((d_hi == d_lo) & (hi % 2 == 0))
    code[~sat] = np.where(exact | pick_hi, hi, lo)
    code = code.reshape(v.shape)
    return (code | np.where(np.signbit(v), 0x80, 0)).astype(np.uint8)


def e4m3_decode(code) -> np.ndarray:
    """e4m3 codes (never the NaN codes 0x7F / 0xFF) -> fp64 values."""
    code = np.asarray(code, dtype=np.int64)
    mag = e4m3_magnitudes()[code & 0x7F]
    return np.where(code & 0x80, -mag, mag)


def fp8_rows(X):
    """Row-scaled e4m3 quantisation of fp32 rows X[N][d]: (codes u8[N][d], s f32[N])."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    m = np.abs(X).max(axis=1) if X.shape[1] else np.zeros(X.shape[0], np.float32)
    s = np.where(m > 0, m / np.float32(E4M3_MAX), np.float32(1.0)).astype(np.float32)
    q = (X / s[:, None]).astype(np.float32)
    return e4m3_encode(q), s


def decoded_rows(storage: str, X) -> np.ndarray:
    """The fp32 rows a search over `storage` ("f32", "bf16", "f16", "fp8") reads."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    if storage == "f32":
        return X.copy()
    if storage == "bf16":
        return bf16_round(X)
    if storage == "f16":
        return f16_round(X)
    if storage == "fp8":
        codes, s = fp8_rows(X)
        return (e4m3_decode(codes).astype(np.float32) * s[:, None]).astype(np.float32)
    raise ValueError(f"unknown storage {storage!r}")
