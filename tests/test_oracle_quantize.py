"""Pins for the oracle's reduced-precision storage: FP64 -> FP32 against
numpy's conversion, FP64 -> BF16 against exact rational rounding (ties to
even), including values placed exactly on and one FP64 ulp beside BF16
midpoints, where rounding through FP32 first would go wrong."""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def bf16_exact(d: float) -> int:
    """Nearest BF16 (8 significant bits), ties to even, by exact arithmetic."""
    if d == 0.0:
        return 0x8000 if math.copysign(1.0, d) < 0 else 0
    m, e = math.frexp(abs(d))                   # |d| = m * 2^e, 0.5 <= m < 1
    q = Fraction(abs(d)) / (Fraction(2) ** (e - 8))   # in [128, 256)
    k = math.floor(q)
    rem = q - k
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and k % 2 == 1):
        k += 1
    value = math.ldexp(k, e - 8) * (1.0 if d > 0 else -1.0)
    bits = int(np.array([value], np.float32).view(np.uint32)[0])
    assert (bits & 0xFFFF) == 0
    return bits >> 16


def _cases():
    rng_vals = list(synth.vector_normal(4000, seed=5)) + list(synth.vector_uniform(2000, -1e3, 1e3))
    ties = []
    for k in range(128, 256, 3):
        for e in (-20, -1, 0, 1, 7, 30):
            mid = math.ldexp(k + 0.5, e - 8)          # exactly between two BF16 values
            ties += [mid, -mid, math.nextafter(mid, math.inf), math.nextafter(mid, -math.inf)]
            # one FP64 ulp above a midpoint but within FP32 rounding of it
            ties.append(mid + math.ldexp(1.0, e - 40))
    return np.array(rng_vals + ties, np.float64)


def test_f32_matches_numpy_round_to_nearest_even():
    v = _cases()
    assert np.array_equal(oracle.quantize(v, "f32").view(np.uint32),
                          v.astype(np.float32).view(np.uint32))


def test_bf16_matches_exact_rounding():
    v = _cases()
    got = oracle.quantize(v, "bf16")
    expect = np.array([bf16_exact(float(d)) for d in v], np.uint16)
    bad = np.flatnonzero(got != expect)
    assert bad.size == 0, [(float(v[i]), int(got[i]), int(expect[i])) for i in bad[:5]]


def test_bf16_round_trip_and_error_bound():
    v = synth.vector_normal(10000, seed=8)
    back = oracle.bf16_to_f64(oracle.quantize(v, "bf16"))
    assert np.all(np.abs(back - v) <= np.abs(v) * 2.0 ** -8)   # half a unit of the 8-bit significand
    exact = oracle.bf16_to_f64(oracle.quantize(back, "bf16"))
    assert np.array_equal(exact, back)                          # representable values are fixed points
