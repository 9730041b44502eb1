"""Helpers shared by the parity tests: the library's one-float Gamma encoding on the host side,
teacher-forced inputs made by the oracle, and the tolerance metric.

Tolerances (FP32 path against the FP64 oracle fed the same FP32-rounded inputs):
* linear domain, every entry:  |P_gpu - P_oracle| <= max(LIN_ATOL, U32 * kappa)
* log-magnitude, on entries with |P_oracle| >= 2^-7 of vectors with U32 * kappa * 2^7 <= LOG_ATOL:
  |ln|P_gpu| - ln|P_oracle|| <= LOG_ATOL, and the signs agree.
kappa is the condition number of the normalised output of a signed sum,
kappa = max_z sum_i |t_i(z)| / |U(0)| (1 for the transform of a probability vector and for the
check node's products), widened at the variable node by the FP32 error of the channel message the
kernel rebuilds (conv_condition). An FP32 sum of q terms followed by division by U(0) carries an error of
order U32 * kappa (U32 = 2^-24) however it is evaluated, because every input is itself an FP32
value: with conflicting channel and check messages U(0) is tiny and kappa large. At
|P| >= 2^-7 an absolute error of 7.8e-7 in P is 1e-4 in ln|P|.
"""

from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from oracle import logfourier as LF
from oracle.transforms import gamma_inv, xor_conv

U32 = 2.0 ** -24
LIN_ATOL = 1e-5
LOG_ATOL = 1e-4
LOG_FLOOR = 2.0 ** -7
MARGIN = 1e-3


def encode(s, l) -> np.ndarray:
    """Oracle Gamma pair (s, l = ln|P|) -> the library's float32 (sign bit = s, |value| = -l)."""
    neg_l = -np.asarray(l, dtype=np.float64)
    mag = np.where(neg_l > 0, neg_l, 0.0).astype(np.float32)  # +0.0 for P = 1, clamp |P| > 1
    return np.where(np.asarray(s).astype(bool), -mag, mag).astype(np.float32)


def decode_pair(g: np.ndarray):
    """Library float32 -> oracle Gamma pair in float64 (exact)."""
    g = np.asarray(g, dtype=np.float32)
    return np.signbit(g).astype(np.uint8), -np.abs(g).astype(np.float64)


def to_linear(g: np.ndarray) -> np.ndarray:
    s, l = decode_pair(g)
    return gamma_inv(s, l)


def compare(gpu: np.ndarray, s_o: np.ndarray, l_o: np.ndarray, kappa=None, lin_atol=LIN_ATOL,
            log_atol=LOG_ATOL, kappa_log=None):
    """Returns (ok, stats) for GPU messages against oracle Gamma pairs of the same shape
    (..., q); kappa (shape (...)) is the per-vector condition number (None: 1). kappa_log
    (shape (..., q)), if given, replaces the per-vector rule of the log-magnitude check by a
    per-entry one: entry z is checked where |P(z)| >= 2^-7 and U32 kappa_log(z) / |P(z)| <=
    log_atol. stats["exempt"] is the share of the entries with |P| >= 2^-7 left out."""
    P_o = gamma_inv(s_o, l_o)
    P_g = to_linear(gpu)
    k = np.ones(P_o.shape[:-1]) if kappa is None else np.asarray(kappa, dtype=np.float64)
    tol = np.maximum(lin_atol, U32 * k)[..., None]
    err = np.abs(P_g - P_o)
    lin_bad = int(np.sum(err > tol))
    lin = float(np.max(err)) if P_o.size else 0.0
    floor = np.abs(P_o) >= LOG_FLOOR
    if kappa_log is None:
        well = (U32 * k * 2.0 ** 7 <= log_atol)[..., None]
    else:
        with np.errstate(divide="ignore", invalid="ignore"):
            well = U32 * np.asarray(kappa_log, dtype=np.float64) <= log_atol * np.abs(P_o)
    mask = floor & well
    n_floor = int(floor.sum())
    sg, lg = decode_pair(gpu)
    logerr = float(np.max(np.abs(lg[mask] - l_o[mask]))) if mask.any() else 0.0
    sign_mask = np.abs(P_o) > np.maximum(2 * tol, LOG_FLOOR)  # a sign is decided where |P| > error
    sign_bad = int(np.sum(sg[sign_mask] != s_o[sign_mask]))
    nan = int(np.isnan(gpu).sum())
    ok = lin_bad == 0 and logerr <= log_atol and sign_bad == 0 and nan == 0
    return ok, {"lin_max": lin, "lin_bad": lin_bad, "log_max": logerr, "sign_bad": sign_bad, "nan": nan,
                "n_log": int(mask.sum()), "kappa_max": float(k.max()) if k.size else 1.0,
                "exempt": 1.0 - int(mask.sum()) / n_floor if n_floor else 0.0}


def conv_condition(a_lin: np.ndarray, b_lin: np.ndarray, m: int) -> np.ndarray:
    """kappa of the normalised XOR convolution a (*) b where `a` is the channel message that the
    kernel rebuilds in FP32 (absolute error up to 2m ulp(1) per entry: m products and an m-stage
    tree of additions over a probability vector):
    kappa = (max_z sum |a||b| + 2m sum |b|) / |(a (*) b)(0)|."""
    S = xor_conv(np.abs(a_lin), np.abs(b_lin))
    U0 = xor_conv(a_lin, b_lin)[..., 0]
    with np.errstate(divide="ignore"):
        return (np.max(S, axis=-1) + 2 * m * np.abs(b_lin).sum(-1)) / np.abs(U0)


def var_conditions(oc, lam0, c2v) -> np.ndarray:
    """kappa of every V->C output (edge e: channel of its variable (*) message of the other edge)."""
    a = gamma_inv(*lam0)
    b = gamma_inv(*c2v)
    other = np.empty(oc.E, dtype=np.int64)
    for v in range(oc.N):
        e1, e2 = oc.C[v]
        other[e1], other[e2] = e2, e1
    return conv_condition(a[oc.edge_var], b[other], oc.m)


def var_log_conditions(oc, lam0, c2v) -> np.ndarray:
    """Per entry of every V->C output (E, q), the condition that decides whether the entry's
    log-magnitude is held to LOG_ATOL: kappa_log(z) = 2m (sum_z' |b(z')| / |U(0)|) (1 + |P(z)|),
    b the message of the other edge, U = a (*) b, P = U / U(0). It is the channel-term part of
    conv_condition taken per entry: an absolute error of 2m ulp(1) in every entry of the channel
    term a moves U(z) and U(0) by at most 2m u sum|b| each, so P(z) by at most u kappa_log(z);
    since |a| <= 1 it also dominates the operand-rounding part. Measured on every FP32 form
    (teacher-forced, GF(16), GF(64), GF(256), 0.5-3 dB) the linear error stays below
    8.6 u sum|b| / |U(0)| (1 + |P(z)|), so the bound holds with room to spare; an entry is held
    to LOG_ATOL where u kappa_log(z) / |P(z)| <= LOG_ATOL."""
    a = gamma_inv(*lam0)[oc.edge_var]
    b = gamma_inv(*c2v)
    other = np.empty(oc.E, dtype=np.int64)
    for v in range(oc.N):
        e1, e2 = oc.C[v]
        other[e1], other[e2] = e2, e1
    b = b[other]
    U = xor_conv(a, b)
    with np.errstate(divide="ignore", invalid="ignore"):
        P = U / U[:, :1]
        return 2 * oc.m * (np.abs(b).sum(-1) / np.abs(U[:, 0]))[:, None] * (1.0 + np.abs(P))


def log_exempt_cap(m: int) -> float:
    """Largest share of the entries with |P| >= 2^-7 that a variable-node comparison may leave
    out of the log-magnitude check (kappa_log rule): measured 0-6% at GF(16), 3-10% at GF(64) and
    10-33% at GF(256) on oracle states at 0.5-3 dB and 1-4 iterations."""
    return 0.10 if m <= 5 else (0.15 if m <= 7 else 0.40)


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


# ---- half-precision message storage (NBFD_STORE_F16) ----------------------------------------
# A stored Gamma word is the float32 word rounded to IEEE half (round to nearest even): the sign
# bit is kept and the log-magnitude m = -ln|P| gets an 11-bit significand, so the stored value
# carries |dm| <= U16 * m, i.e. |dP| = |P| (1 - e^{-dm}) <= U16 * |P| * m <= U16 / e.
U16 = 2.0 ** -11


def to_half(g32: np.ndarray) -> np.ndarray:
    """Library float32 Gamma words -> the half words the library stores (as float16)."""
    return np.asarray(g32, dtype=np.float32).astype(np.float16)


def compare_store16(gpu16: np.ndarray, s_o: np.ndarray, l_o: np.ndarray, kappa=None, kappa_log=None):
    """compare() for half-stored outputs: the FP32 bounds plus the output rounding,
    linear |dP| <= max(LIN_ATOL, U32 kappa) + U16 |P| |ln|P||, log-magnitude
    |d ln|P|| <= LOG_ATOL + U16 |ln|P|| on the entries compare() checks (with kappa_log, the
    per-entry rule of compare()); signs where |P| exceeds twice the linear bound."""
    g = np.asarray(gpu16, dtype=np.float16).astype(np.float32)
    P_o = gamma_inv(s_o, l_o)
    P_g = to_linear(g)
    k = np.ones(P_o.shape[:-1]) if kappa is None else np.asarray(kappa, dtype=np.float64)
    with np.errstate(invalid="ignore"):
        store = np.where(np.isfinite(l_o), U16 * np.abs(P_o) * np.abs(l_o), 0.0)
    tol = np.maximum(LIN_ATOL, U32 * k)[..., None] + store
    err = np.abs(P_g - P_o)
    lin_bad = int(np.sum(err > tol * (1 + 1e-9)))
    if kappa_log is None:
        well = (U32 * k * 2.0 ** 7 <= LOG_ATOL)[..., None]
    else:
        with np.errstate(divide="ignore", invalid="ignore"):
            well = U32 * np.asarray(kappa_log, dtype=np.float64) <= LOG_ATOL * np.abs(P_o)
    floor = np.abs(P_o) >= LOG_FLOOR
    mask = floor & well
    sg, lg = decode_pair(g)
    log_bound = LOG_ATOL + U16 * np.abs(l_o)
    log_bad = int(np.sum(np.abs(lg[mask] - l_o[mask]) > log_bound[mask])) if mask.any() else 0
    sign_mask = np.abs(P_o) > np.maximum(2 * tol, LOG_FLOOR)
    sign_bad = int(np.sum(sg[sign_mask] != s_o[sign_mask]))
    nan = int(np.isnan(g).sum())
    ok = lin_bad == 0 and log_bad == 0 and sign_bad == 0 and nan == 0
    return ok, {"lin_max": float(err.max()) if err.size else 0.0, "lin_bad": lin_bad, "log_bad": log_bad,
                "sign_bad": sign_bad, "nan": nan, "n_log": int(mask.sum()),
                "exempt": 1.0 - int(mask.sum()) / int(floor.sum()) if floor.any() else 0.0}


# ---- oracle decodes of many frames, in a spawn process pool -----------------------------------

def _oracle_decode_worker(args):
    code, llr, max_iter, decision = args
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle.code import OracleCode
    r = LF.decode(OracleCode.from_dict(code), np.asarray(llr, dtype=np.float64), max_iter, decision=decision)
    return {k: r[k] for k in ("symbols", "ok", "iters", "margins", "fourier_only")}


def oracle_decodes(code: dict, llr_rows: np.ndarray, max_iter: int, decision: str = "bitwise"):
    """LF.decode of every row of llr_rows, one frame per task on a spawn pool (a pool forked from
    a process that has used the GPU can hang; spawn starts clean interpreters)."""
    n = len(llr_rows)
    procs = max(1, min(n, os.cpu_count() or 1))
    if procs == 1:
        return [_oracle_decode_worker((code, llr_rows[i], max_iter, decision)) for i in range(n)]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_oracle_decode_worker, [(code, llr_rows[i], max_iter, decision) for i in range(n)],
                        chunksize=1)
