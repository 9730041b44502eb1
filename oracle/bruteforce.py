"""Brute-force MAP over all codewords of tiny codes (test infrastructure only).

Section 2.1: sum-product is symbol-MAP when the Tanner graph is a tree; Section 3.1: the bit-MAP
decision compares q_{v,i}(0) with q_{v,i}(1). Here both are computed by enumerating every word of
GF(2^m)^N, keeping those with Hx = 0, and summing prod_v p_v^(0)(x_v) over them. Exponential in
N*m: only for N*m <= 20.
"""

from __future__ import annotations

import numpy as np

from .channel import symbol_probabilities
from .code import OracleCode


def codewords(code: OracleCode) -> np.ndarray:
    """All x in GF(2^m)^N with Hx = 0, as an (n_words, N) integer array."""
    q, N = code.q, code.N
    if N * code.m > 20:
        raise ValueError("code too large for enumeration")
    idx = np.arange(q ** N, dtype=np.int64)
    words = np.empty((q ** N, N), dtype=np.int64)
    for v in range(N):
        words[:, v] = (idx // (q ** v)) % q
    s = code.syndrome(words)
    return words[~np.any(s != 0, axis=1)]


def symbol_marginals(code: OracleCode, llr: np.ndarray, cw: np.ndarray | None = None) -> np.ndarray:
    """Exact Pr(X_v = a | y) for every v, a: (N, q)."""
    if cw is None:
        cw = codewords(code)
    p0 = symbol_probabilities(llr)  # (N, q)
    w = np.ones(len(cw))
    for v in range(code.N):
        w = w * p0[v, cw[:, v]]
    out = np.zeros((code.N, code.q))
    for v in range(code.N):
        np.add.at(out[v], cw[:, v], w)
    return out / w.sum()


def bit_map(code: OracleCode, marg: np.ndarray) -> np.ndarray:
    """Bitwise MAP decisions (as symbol integers) and the biases q_{v,i}(0) - q_{v,i}(1)."""
    xs = np.arange(code.q)
    bias = np.empty((code.N, code.m))
    x = np.zeros(code.N, dtype=np.int64)
    for i in range(code.m):
        sgn = np.where((xs >> i) & 1, -1.0, 1.0)
        bias[:, i] = marg @ sgn
        x |= (bias[:, i] < 0).astype(np.int64) << i
    return x, bias
