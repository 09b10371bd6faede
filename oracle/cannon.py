"""FP64 oracle for the paper's matrix-multiplication workload (section 5,
"Matrix Multiplication"): Cannon's ring exchange computing C = A x B.

TEST INFRASTRUCTURE ONLY: used by the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; the library never imports it.

The paper's setting: P ranks in a ring, matrix size N, stripe width
Ns = N / P.  Rank r owns the row stripe A_r (rows r*Ns .. r*Ns + Ns - 1 of
A, all N columns) and one column stripe of B (N x Ns) at a time, plus one
spare stripe buffer so the next stripe can arrive while the current one is
used.  In each of P steps a rank multiplies its A stripe by the B stripe it
holds, giving one Ns x Ns block of its row stripe of C (N * Ns * Ns
multiply-adds), and passes the B stripe along the ring.

Reading (the paper gives no direction): at step s rank r holds column
stripe (r + s) mod P and sends it to rank (r - 1) mod P.

Inputs are the values the GPU receives (BF16 numbers, held here as float64);
the products and sums are exact FP64 arithmetic on them.  A block product
is a library matmul (a plain definition, no blocking beyond the stripes).
"""

from __future__ import annotations

import numpy as np


def stripe_width(n: int, p: int) -> int:
    if p < 1 or n % p:
        raise ValueError(f"N = {n} is not a multiple of P = {p}")
    return n // p


def schedule(p: int) -> list[list[tuple[int, int]]]:
    """Per step s, the (rank, B column stripe) pairs multiplied."""
    return [[(r, (r + s) % p) for r in range(p)] for s in range(p)]


def cannon(a: np.ndarray, b: np.ndarray, p: int):
    """C = A B by P ring steps.  Returns (C, blocks), blocks the list of
    (step, rank, stripe) in the order they were computed."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.shape[0]
    if a.shape != (n, n) or b.shape != (n, n):
        raise ValueError("square N x N matrices expected")
    ns = stripe_width(n, p)
    c = np.zeros((n, n), dtype=np.float64)
    # what each rank holds: its A row stripe and, initially, B column
    # stripe r (with the stripe's index travelling alongside)
    a_loc = [a[r * ns:(r + 1) * ns, :] for r in range(p)]
    b_loc = [b[:, r * ns:(r + 1) * ns].copy() for r in range(p)]
    b_idx = list(range(p))
    blocks = []
    for s in range(p):
        for r in range(p):
            j = b_idx[r]
            c[r * ns:(r + 1) * ns, j * ns:(j + 1) * ns] = a_loc[r] @ b_loc[r]
            blocks.append((s, r, j))
        # ring exchange: rank r receives the stripe of rank r + 1 into its
        # spare buffer, which then becomes the current one
        spare = [b_loc[(r + 1) % p].copy() for r in range(p)]
        b_idx = [b_idx[(r + 1) % p] for r in range(p)]
        b_loc = spare
    return c, blocks


def entry(a: np.ndarray, b: np.ndarray, i: int, j: int) -> float:
    """One element of A B, summed in FP64 (exact for the dyadic inputs of
    the tests), for sampled checks at sizes the full product does not fit."""
    return float(np.dot(np.asarray(a[i, :], dtype=np.float64),
                        np.asarray(b[:, j], dtype=np.float64)))


def entry_abs(a: np.ndarray, b: np.ndarray, i: int, j: int) -> float:
    """sum_k |A_ik B_kj|, the scale of the FP32 accumulation error bound."""
    return float(np.dot(np.abs(np.asarray(a[i, :], dtype=np.float64)),
                        np.abs(np.asarray(b[:, j], dtype=np.float64))))


def fp32_sum_bound(k: int, abs_sum):
    """Worst-case error of a length-k sum of exact products accumulated in
    FP32 in any order: (k - 1) u / (1 - (k - 1) u) * sum |terms| with
    u = 2^-24 (Higham, Accuracy and Stability of Numerical Algorithms,
    eq. 3.5), doubled to cover accumulators that truncate instead of
    rounding to nearest."""
    u = 2.0 ** -24
    g = (k - 1) * u
    return 2.0 * g / (1.0 - g) * np.asarray(abs_sum, dtype=np.float64)
