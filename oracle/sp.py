"""Probability-domain sum-product decoder, FP64 (test infrastructure only).

Section 2.1 ("Conventional Sum-Product Algorithm"), step by step:

* INITIALIZATION: p_vc^(0) = p_v^(0) = Pr(X_v = x | Y_v = y_v).
* CHECK TO VARIABLE (Eq. (1) of the check-node update): p~_vc(x) = p_vc(h_cv^{-1} x);
  p~_cv = convolution over v' in V_c \\ {v} of p~_v'c; p_cv(x) = p~_cv(h_cv x).
  The convolution (p1 (x) p2)(x) = sum_{x1 + x2 = x} p1(x1) p2(x2) is evaluated from its
  definition (O(q^2) per pair, no transform), the k-1 factors folded left to right.
* VARIABLE TO CHECK: p_vc(x) = p_v^(0)(x) prod_{c' in C_v \\ {c}} p_c'v(x), normalised to sum 1.
* TENTATIVE DECISION: q_v(x) = p_v^(0)(x) prod_{c in C_v} p_cv(x); x_hat = argmax (ties: lowest x).
  The bitwise marginals q_{v,i}(0) - q_{v,i}(1) of Section 3.1 are returned as well.
* Stop when x_hat is a codeword (Hx = 0), else repeat; FAIL after max_iter iterations.

Independent of ``logfourier`` except for the channel factorisation and the graph view.
Pinned by: exact marginals on cycle-free graphs against brute-force enumeration, and equality of
every message with the Log-Fourier decoder (after the transform) on loopy graphs.
"""

from __future__ import annotations

import numpy as np

from .channel import symbol_probabilities
from .code import OracleCode
from .transforms import xor_conv


def init(code: OracleCode, llr: np.ndarray):
    """llr (N, m) -> (p0 (N, q), v2c (E, q))."""
    p0 = symbol_probabilities(llr)
    return p0, p0[code.edge_var].copy()


def check_update(code: OracleCode, v2c: np.ndarray) -> np.ndarray:
    gf = code.gf
    q = code.q
    xs = np.arange(q)
    c2v = np.empty_like(v2c)
    delta0 = np.zeros(q)
    delta0[0] = 1.0  # identity of the convolution (empty product)
    for c in range(code.M):
        edges = code.V[c]
        perm_in = []
        for e in edges:
            hinv = int(gf.inv(int(code.edge_h[e])))
            perm_in.append(v2c[e][gf.mul(hinv, xs)])  # p~_vc(x) = p_vc(h^{-1} x)
        for i, e in enumerate(edges):
            acc = None
            for j in range(len(edges)):
                if j == i:
                    continue
                acc = perm_in[j] if acc is None else xor_conv(acc, perm_in[j])
            if acc is None:
                acc = delta0
            c2v[e] = acc[gf.mul(int(code.edge_h[e]), xs)]  # p_cv(x) = p~_cv(h x)
    return c2v


def var_update(code: OracleCode, p0: np.ndarray, c2v: np.ndarray) -> np.ndarray:
    v2c = np.empty_like(c2v)
    for v in range(code.N):
        for e in code.C[v]:
            prod = p0[v].copy()
            for e2 in code.C[v]:
                if e2 != e:
                    prod = prod * c2v[e2]
            v2c[e] = prod / prod.sum()
    return v2c


def marginals(code: OracleCode, p0: np.ndarray, c2v: np.ndarray) -> np.ndarray:
    """q_v(x) normalised to sum 1, (N, q)."""
    qv = p0.copy()
    for e in range(code.E):
        qv[code.edge_var[e]] = qv[code.edge_var[e]] * c2v[e]
    return qv / qv.sum(axis=-1, keepdims=True)


def bit_bias(qv: np.ndarray, m: int) -> np.ndarray:
    """q_{v,i}(0) - q_{v,i}(1) for i = 1..m, shape (N, m) (Section 3.1)."""
    xs = np.arange(qv.shape[-1])
    out = np.empty(qv.shape[:-1] + (m,))
    for i in range(m):
        sgn = np.where((xs >> i) & 1, -1.0, 1.0)
        out[..., i] = qv @ sgn
    return out


def decode(code: OracleCode, llr: np.ndarray, max_iter: int):
    """One frame. Returns dict(symbols, ok, iters) with symbol-argmax decisions."""
    p0, v2c = init(code, llr)
    x_hat = np.argmax(p0, axis=-1)
    ok = False
    it = 0
    for it in range(1, max_iter + 1):
        c2v = check_update(code, v2c)
        v2c = var_update(code, p0, c2v)
        qv = marginals(code, p0, c2v)
        x_hat = np.argmax(qv, axis=-1)
        if not np.any(code.syndrome(x_hat)):
            ok = True
            break
    return {"symbols": x_hat, "ok": ok, "iters": it}
