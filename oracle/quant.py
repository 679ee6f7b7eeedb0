"""ORACLE (test infrastructure): BF16 and FP8 E4M3 encoders from the formats' definitions.

BF16: the top 16 bits of an IEEE-754 binary32; rounding is to nearest, ties to even.
FP8 E4M3 (the OCP "FN" variant): 1 sign bit, 4 exponent bits (bias 7), 3 mantissa bits; no
infinities; exponent 15 with mantissa 7 is NaN, so the largest finite value is 1.75 * 2^8 = 448;
exponent 0 encodes subnormals m * 2^-9. Encoding rounds to nearest, ties to even, and saturates
finite values beyond 448 to +-448.
"""
from __future__ import annotations

import numpy as np


def bf16_bits(x) -> np.ndarray:
    """uint16 BF16 codes of float32 inputs (round to nearest even; NaN -> quiet NaN)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    nan = np.isnan(np.asarray(x, dtype=np.float32))
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) & 0xFFFF
    r = np.where(nan, ((u >> 16) | 0x40) & 0xFFFF, r)
    return r.astype(np.uint16)


def bf16_value(bits) -> np.ndarray:
    return (np.asarray(bits, dtype=np.uint32) << 16).view(np.float32)


def bf16_round(x) -> np.ndarray:
    """float32 values rounded to the nearest BF16 value."""
    return bf16_value(bf16_bits(x))


def bf16_round64(x) -> np.ndarray:
    """float64 values rounded once, to nearest with ties to even, to the nearest BF16 value (8
    significant bits), returned as float64. Rounding a float64 to float32 first and then to BF16
    can differ (double rounding); this does not. Inputs stay inside BF16's normal range here."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                     # x = m * 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)   # np.rint rounds halves to even


E4M3_MAX = 448.0


def e4m3_bits(x) -> np.ndarray:
    """uint8 E4M3 codes (round to nearest even, saturating; NaN -> 0x7F with the input's sign)."""
    x = np.asarray(x, dtype=np.float64)
    sign = (np.signbit(x)).astype(np.uint8) << 7
    a = np.abs(x)
    out = np.zeros(a.shape, dtype=np.uint8)
    nan = np.isnan(a)
    sub = a < 2.0 ** -6
    # subnormals (and zero): m * 2^-9, m in 0..8 (m == 8 is the smallest normal, code 0x08)
    m_sub = np.rint(np.where(sub, a, 0.0) / 2.0 ** -9).astype(np.int64)
    # normals: (1 + m/8) * 2^e, e in -6..8
    safe = np.where(sub | nan, 1.0, a)
    e = np.floor(np.log2(safe)).astype(np.int64)
    # guard against log2 rounding at exact powers of two
    e = np.where(safe < 2.0 ** e, e - 1, e)
    e = np.where(safe >= 2.0 ** (e + 1), e + 1, e)
    frac = safe / 2.0 ** e * 8.0 - 8.0
    m = np.rint(frac).astype(np.int64)
    carry = m == 8
    e = np.where(carry, e + 1, e)
    m = np.where(carry, 0, m)
    over = (e > 8) | ((e == 8) & (m > 6))
    e = np.where(over, 8, e)
    m = np.where(over, 6, m)
    code_norm = ((e + 7) << 3) | m
    code = np.where(sub, m_sub, code_norm)
    code = np.where(nan, 0x7F, code)
    out[...] = code.astype(np.uint8)
    return out | sign


def e4m3_value(bits) -> np.ndarray:
    b = np.asarray(bits, dtype=np.int64)
    s = np.where(b & 0x80, -1.0, 1.0)
    e = (b >> 3) & 0xF
    m = b & 0x7
    val = np.where(e == 0, m * 2.0 ** -9, (1.0 + m / 8.0) * 2.0 ** (e - 7))
    val = np.where((e == 15) & (m == 7), np.nan, val)
    return s * val


def e4m3_round(x) -> np.ndarray:
    return e4m3_value(e4m3_bits(x))
