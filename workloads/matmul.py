"""Seeded synthetic matrices for the paper's matrix-multiplication workload
(Cannon's algorithm, section 5: square N x N matrices, 30240 x 30240 in the
paper's runs, whose values it does not publish).

Only inputs are drawn here: BF16 numbers as raw 16-bit patterns, plus the
same values as float64 for the oracle.  No product is formed.

Recipes:

* dyadic: k / 16 with k uniform on the integers -16 .. 16.  Every value is a
  BF16 number, every product a multiple of 1/256 of magnitude <= 1, so any
  FP32 accumulation of up to 65536 products is exact, in any order.
* uniform: uniform on [-1, 1), rounded to the nearest BF16 (ties to even).

The second operand is drawn as B^T (B in column-major order: each row of
the returned array is one column of B, K contiguous), the layout of the
stripes that travel around the ring.
"""

from __future__ import annotations

import numpy as np

_DYADIC_BITS = None


def _dyadic_table() -> np.ndarray:
    global _DYADIC_BITS
    if _DYADIC_BITS is None:
        v = (np.arange(-16, 17, dtype=np.float32) / np.float32(16.0))
        _DYADIC_BITS = (v.view(np.uint32) >> 16).astype(np.uint16)
    return _DYADIC_BITS


def dyadic_codes(n: int, m: int, seed: int) -> np.ndarray:
    """An n x m int8 array of k in -16 .. 16 (value k / 16)."""
    rng = np.random.default_rng(seed)
    return rng.integers(-16, 17, size=(n, m), dtype=np.int8)


def dyadic_bits(codes: np.ndarray) -> np.ndarray:
    """BF16 bit patterns of k / 16."""
    return np.take(_dyadic_table(), codes.astype(np.intp) + 16)


def dyadic_values(codes: np.ndarray) -> np.ndarray:
    return codes.astype(np.float64) / 16.0


def round_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Nearest BF16 (ties to even) of finite float32 values, as bits."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    bias = ((u >> 16) & 1) + np.uint32(0x7FFF)
    return ((u + bias) >> 16).astype(np.uint16)


def bf16_values(bits: np.ndarray) -> np.ndarray:
    """float64 values of BF16 bit patterns."""
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def uniform_bits(n: int, m: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return round_bf16_bits(rng.uniform(-1.0, 1.0, size=(n, m)).astype(np.float32))


def pair(n: int, seed: int, kind: str = "dyadic"):
    """(A bits, B^T bits, A values, B values) for an N x N product; the
    float64 values only for n <= 4096 (None above)."""
    if kind == "dyadic":
        ka = dyadic_codes(n, n, seed)
        kb = dyadic_codes(n, n, seed + 1)
        a_bits, bt_bits = dyadic_bits(ka), dyadic_bits(kb)
        if n > 4096:
            return a_bits, bt_bits, None, None
        return a_bits, bt_bits, dyadic_values(ka), dyadic_values(kb).T.copy()
    if kind == "uniform":
        a_bits = uniform_bits(n, n, seed)
        bt_bits = uniform_bits(n, n, seed + 1)
        if n > 4096:
            return a_bits, bt_bits, None, None
        return a_bits, bt_bits, bf16_values(a_bits), bf16_values(bt_bits).T.copy()
    raise ValueError(f"unknown kind {kind!r}")
