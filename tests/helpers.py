"""Helpers shared by the parity tests: the library's one-float Gamma encoding on the host side,
teacher-forced inputs made by the oracle, and the tolerance metric.

Tolerances (FP32 path against the FP64 oracle fed the same FP32-rounded inputs):
* linear domain, every entry:          |P_gpu - P_oracle| <= LIN_ATOL
* log-magnitude where |P_oracle| >= 2^-7: |ln|P_gpu| - ln|P_oracle|| <= LOG_ATOL, signs equal.
FP32 transforms / sums of q terms bounded by 1 carry an absolute error of a few ulp(1) times
sqrt(q) per entry, so the log-magnitude bound is only feasible where |P| is not tiny; at
|P| >= 2^-7 an absolute error of 7.8e-7 in P is 1e-4 in ln|P|.
"""

from __future__ import annotations

import numpy as np

from oracle import logfourier as LF
from oracle.transforms import gamma_inv

LIN_ATOL = 1e-5
LOG_ATOL = 1e-4
LOG_FLOOR = 2.0 ** -7
MARGIN = 1e-3


def encode(s, l) -> np.ndarray:
    """Oracle Gamma pair (s, l = ln|P|) -> the library's float32 (sign bit = s, |value| = -l)."""
    mag = (-np.asarray(l, dtype=np.float64)).astype(np.float32)
    return np.where(np.asarray(s).astype(bool), -mag, mag).astype(np.float32)


def decode_pair(g: np.ndarray):
    """Library float32 -> oracle Gamma pair in float64 (exact)."""
    g = np.asarray(g, dtype=np.float32)
    return np.signbit(g).astype(np.uint8), -np.abs(g).astype(np.float64)


def to_linear(g: np.ndarray) -> np.ndarray:
    s, l = decode_pair(g)
    return gamma_inv(s, l)


def compare(gpu: np.ndarray, s_o: np.ndarray, l_o: np.ndarray, lin_atol=LIN_ATOL, log_atol=LOG_ATOL):
    """Returns (ok, stats) for GPU messages against oracle Gamma pairs of the same shape."""
    P_o = gamma_inv(s_o, l_o)
    P_g = to_linear(gpu)
    lin = float(np.max(np.abs(P_g - P_o))) if P_o.size else 0.0
    mask = np.abs(P_o) >= LOG_FLOOR
    sg, lg = decode_pair(gpu)
    logerr = float(np.max(np.abs(lg[mask] - l_o[mask]))) if mask.any() else 0.0
    sign_bad = int(np.sum(sg[mask] != s_o[mask]))
    nan = int(np.isnan(gpu).sum())
    ok = lin <= lin_atol and logerr <= log_atol and sign_bad == 0 and nan == 0
    return ok, {"lin_max": lin, "log_max": logerr, "sign_bad": sign_bad, "nan": nan,
                "n_log": int(mask.sum())}


def oracle_state(oc, llr: np.ndarray, n_iter: int):
    """Run the oracle n_iter iterations; returns (lam0, v2c, c2v) Gamma pairs (c2v None if 0)."""
    lam0, v2c = LF.init(oc, llr)
    c2v = None
    for _ in range(n_iter):
        c2v = LF.check_update(oc, v2c)
        v2c = LF.var_update(oc, lam0, c2v)
    return lam0, v2c, c2v


def vn_margins(oc, M) -> np.ndarray:
    """Per variable: min over its 3m read-out points of |M(z)| / M(0) (FP64)."""
    Ms, Ml = M
    out = np.min(Ml[:, [1 << i for i in range(oc.m)]] - Ml[:, :1], axis=1)
    for e in range(oc.E):
        v = oc.edge_var[e]
        pts = oc.perm[e, [1 << i for i in range(oc.m)]]
        out[v] = min(out[v], np.min(Ml[v, pts] - Ml[v, 0]))
    return np.exp(out)
