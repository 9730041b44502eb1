"""Channel messages p_v^(0)(x) = Pr(X_v = x | Y_v = y_v) from bit LLRs (test infrastructure only).

Section 2.1, initialisation: p_v^(0)(x) is the a-posteriori probability of symbol x. With the
m bits of a symbol sent independently (one BPSK use each) and a uniform prior, it factors over
the coordinates of the m-bit representation:

    p(x) = prod_{i=1..m} Pr(b_i = x_i | y_i),
    Pr(b = 0 | y) = 1 / (1 + exp(-L)),  Pr(b = 1 | y) = 1 / (1 + exp(L)),

with L = ln Pr(b=0|y)/Pr(b=1|y) and coordinate i stored at bit i-1 of the symbol integer.
Pinned by: sum_x p(x) = 1 and bit marginals equal to the logistic of L (tests/test_oracle_*).
"""

from __future__ import annotations

import numpy as np


def bit_probabilities(llr: np.ndarray):
    """(Pr(b=0), Pr(b=1)) for each LLR, computed without overflow."""
    L = np.asarray(llr, dtype=np.float64)
    p0 = np.where(L >= 0, 1.0 / (1.0 + np.exp(-np.abs(L))), np.exp(-np.abs(L)) / (1.0 + np.exp(-np.abs(L))))
    p1 = np.where(L >= 0, np.exp(-np.abs(L)) / (1.0 + np.exp(-np.abs(L))), 1.0 / (1.0 + np.exp(-np.abs(L))))
    return p0, p1


def symbol_probabilities(llr: np.ndarray) -> np.ndarray:
    """llr: (..., m) -> p^(0): (..., 2^m) with p[x] = prod_i Pr(b_i = bit_{i-1}(x))."""
    llr = np.asarray(llr, dtype=np.float64)
    m = llr.shape[-1]
    q = 1 << m
    pb0, pb1 = bit_probabilities(llr)
    xs = np.arange(q)
    p = np.ones(llr.shape[:-1] + (q,), dtype=np.float64)
    for i in range(m):
        bit = (xs >> i) & 1
        p = p * np.where(bit == 1, pb1[..., i:i + 1], pb0[..., i:i + 1])
    return p
