"""Log-Fourier sum-product decoder, FP64, written from Section 3.2 (test infrastructure only).

Messages are Gamma-form vectors over z in GF(2^m): pairs (s, l), s in {0,1} (sign in GF(2)),
l = ln|P(z)| in [-inf, 0].

* INITIALIZATION: P_v^(0) = Fourier transform of p_v^(0) (Section 2.1 definition);
  Lambda_v^(0) = Gamma(P_v^(0)); Lambda_vc^(0) = Lambda_v^(0) on every edge of v.
* CHECK TO VARIABLE: Lambda~_vc(z) = Lambda_vc(H_cv z); Lambda~_cv = sum over v' in V_c \\ {v}
  of Lambda~_v'c (Gamma-form sum: signs XOR, log-magnitudes add); Lambda_cv(z) =
  Lambda~_cv(H_cv^{-1} z). H_cv = (A^i)^T for h_cv = alpha^i (Appendix A).
* VARIABLE TO CHECK: Lambda_vc = Lambda_v^(0) [+] (the boxplus of Lambda_c'v, c' in C_v \\ {c}),
  the log-convolution of the boxplus definition, evaluated term by term; then normalised to
  Lambda_vc(0) = (0, 0) (the Fourier-SP normalisation P(0) = 1 of Section 3.1 carried over to
  Gamma form: l -= l(0), s ^= s(0)).
* TENTATIVE DECISION: M_v = Lambda_v^(0) [+] Lambda_c1v [+] Lambda_c2v (all checks of v);
  bit i of x_hat_v is the sign entry of M_v(alpha^{i-1}); syndrome bit i of check c is the XOR
  over v in V_c of the sign entries of M_v(H_cv alpha^{i-1}).
* Stop rule (reading of Section 3.2 together with the Section 2 definition of a codeword): a frame
  stops at iteration l when every Fourier-domain syndrome bit is 0 AND the GF(2^m) syndrome
  H x_hat is 0; syndrome_ok reports the GF(2^m) syndrome. No check at l = 0.

sgn(0) is taken as 0 (the paper chooses at random); a bit whose M value is exactly 0 decides 0.
Pinned by: equality with the probability-domain decoder ``sp`` (messages and bit decisions),
brute-force bit-MAP on cycle-free graphs, and the transform/Gamma pins of ``transforms``.
"""

from __future__ import annotations

import numpy as np

from .channel import symbol_probabilities
from .code import OracleCode
from .transforms import gamma, gamma_inv, iwht, logconv, normalize_at_zero, wht

_CHUNK_ELEMS = 1 << 22  # bound on the q*q*batch temporaries of the literal log-convolution


def _logconv_batched(a, b):
    sa, la = a
    sb, lb = b
    n, q = la.shape
    step = max(1, _CHUNK_ELEMS // (q * q))
    out_s = np.empty((n, q), dtype=np.uint8)
    out_l = np.empty((n, q), dtype=np.float64)
    for i in range(0, n, step):
        s, l = logconv((sa[i:i + step], la[i:i + step]), (sb[i:i + step], lb[i:i + step]))
        out_s[i:i + step] = s
        out_l[i:i + step] = l
    return out_s, out_l


def init(code: OracleCode, llr: np.ndarray):
    """llr (N, m) -> (Lambda0, v2c) as Gamma pairs of shapes (N, q) and (E, q)."""
    p0 = symbol_probabilities(llr)
    lam0 = gamma(wht(p0))
    v2c = (lam0[0][code.edge_var].copy(), lam0[1][code.edge_var].copy())
    return lam0, v2c


def check_update(code: OracleCode, v2c, checks=None):
    """Gamma-form C->V messages for all edges (or only the edges of `checks`)."""
    s_in, l_in = v2c
    s_out = np.zeros_like(s_in)
    l_out = np.full_like(l_in, np.nan)
    q = code.q
    for c in (range(code.M) if checks is None else checks):
        edges = code.V[c]
        # Lambda~_vc(z) = Lambda_vc(H_cv z)
        ts = [s_in[e][code.perm[e]] for e in edges]
        tl = [l_in[e][code.perm[e]] for e in edges]
        for i, e in enumerate(edges):
            acc_s = np.zeros(q, dtype=np.uint8)  # Gamma(1) = (0, 0): the empty sum
            acc_l = np.zeros(q, dtype=np.float64)
            for j in range(len(edges)):
                if j != i:
                    acc_s = acc_s ^ ts[j]
                    acc_l = acc_l + tl[j]
            # Lambda_cv(z) = Lambda~_cv(H_cv^{-1} z)
            s_out[e] = acc_s[code.perm_inv[e]]
            l_out[e] = acc_l[code.perm_inv[e]]
    return s_out, l_out


def _edges_of(code: OracleCode, vars_):
    return [e for v in vars_ for e in code.C[v]]


def var_update(code: OracleCode, lam0, c2v, vars=None):
    """Gamma-form V->C messages (normalised) for all edges (or the edges of `vars`)."""
    s0, l0 = lam0
    sc, lc = c2v
    vars_ = range(code.N) if vars is None else vars
    s_out = np.zeros_like(sc)
    l_out = np.full_like(lc, np.nan)
    # group the output edges by the number of other checks of their variable
    groups = {}
    for v in vars_:
        for e in code.C[v]:
            others = [e2 for e2 in code.C[v] if e2 != e]
            groups.setdefault(len(others), []).append((e, v, others))
    for d, items in groups.items():
        es = np.array([t[0] for t in items], dtype=np.int64)
        vs = np.array([t[1] for t in items], dtype=np.int64)
        acc = (s0[vs].copy(), l0[vs].copy())
        for t in range(d):
            oth = np.array([it[2][t] for it in items], dtype=np.int64)
            acc = _logconv_batched(acc, (sc[oth], lc[oth]))
        ns, nl = normalize_at_zero(acc)
        s_out[es] = ns
        l_out[es] = nl
    return s_out, l_out


def tentative(code: OracleCode, lam0, c2v, vars=None):
    """M_v = Lambda_v^(0) [+] (boxplus over all checks of v) for `vars` (default all), (n, q)."""
    s0, l0 = lam0
    sc, lc = c2v
    vars_ = list(range(code.N) if vars is None else vars)
    Ms = np.zeros((code.N, code.q), dtype=np.uint8)
    Ml = np.full((code.N, code.q), np.nan)
    groups = {}
    for v in vars_:
        groups.setdefault(len(code.C[v]), []).append(v)
    for d, vs in groups.items():
        vs = np.array(vs, dtype=np.int64)
        acc = (s0[vs].copy(), l0[vs].copy())
        for t in range(d):
            es = np.array([code.C[v][t] for v in vs], dtype=np.int64)
            acc = _logconv_batched(acc, (sc[es], lc[es]))
        Ms[vs] = acc[0]
        Ml[vs] = acc[1]
    return Ms, Ml


def bit_decisions(code: OracleCode, M) -> np.ndarray:
    """x_hat_v as integers: bit i-1 = sign entry of M_v(alpha^{i-1})."""
    Ms, _ = M
    x = np.zeros(code.N, dtype=np.int64)
    for i in range(code.m):
        x |= Ms[:, 1 << i].astype(np.int64) << i
    return x


def symbol_decisions(code: OracleCode, M) -> np.ndarray:
    """x_hat_v = argmax_x mu_v(x), mu_v = inverse transform of M_v (Section 3.2, TENTATIVE
    DECISION, first form); ties go to the lowest symbol."""
    mu = iwht(gamma_inv(*M))
    return np.argmax(mu, axis=-1)


def symbol_margin(code: OracleCode, M) -> float:
    """Smallest (mu(top1) - mu(top2)) / sum |mu| over the variables."""
    mu = iwht(gamma_inv(*M))
    srt = np.sort(mu, axis=-1)
    return float(np.min((srt[:, -1] - srt[:, -2]) / np.abs(mu).sum(axis=-1)))


def fourier_syndrome_words(code: OracleCode, M) -> np.ndarray:
    """Per edge (c, v): m-bit word, bit i-1 = sign entry of M_v(H_cv alpha^{i-1}). (E,)"""
    Ms, _ = M
    w = np.zeros(code.E, dtype=np.int64)
    for i in range(code.m):
        z = code.perm[:, 1 << i]  # H_cv alpha^{i-1} for every edge
        w |= Ms[code.edge_var, z].astype(np.int64) << i
    return w


def fourier_syndrome(code: OracleCode, M) -> np.ndarray:
    """s_hat_c for every check: XOR over v in V_c of the per-edge words. (M,)"""
    w = fourier_syndrome_words(code, M)
    s = np.zeros(code.M, dtype=np.int64)
    for e in range(code.E):
        s[code.edge_check[e]] ^= w[e]
    return s


def decision_margin(code: OracleCode, M) -> float:
    """Smallest |M_v(z)| / M_v(0) over the points that decide bits and Fourier syndrome bits."""
    Ms, Ml = M
    worst = np.min(Ml[:, [1 << i for i in range(code.m)]] - Ml[:, :1])
    for i in range(code.m):
        z = code.perm[:, 1 << i]
        worst = min(worst, np.min(Ml[code.edge_var, z] - Ml[code.edge_var, 0]))
    return float(np.exp(worst))


def decode(code: OracleCode, llr: np.ndarray, max_iter: int, trace: bool = False,
           decision: str = "bitwise"):
    """One frame. Returns dict(symbols, ok, iters, fourier_ok, margins[, trace]).

    decision="bitwise": the Section 3.2 read-out of M_v(alpha^{i-1}); stop on a zero Fourier-domain
    syndrome and a zero GF(2^m) syndrome. decision="symbol": x_hat_v = argmax mu_v (the first
    form of the TENTATIVE DECISION); stop on a zero GF(2^m) syndrome (the Fourier-domain syndrome
    describes bitwise decisions and is not used)."""
    lam0, v2c = init(code, llr)
    x_hat = None
    ok = False
    fok = False
    margins = []
    hist = []
    fourier_only = 0  # iterations whose Fourier-domain syndrome cleared while H x_hat != 0
    it = 0
    for it in range(1, max_iter + 1):
        c2v = check_update(code, v2c)
        v2c = var_update(code, lam0, c2v)
        M = tentative(code, lam0, c2v)
        if decision == "symbol":
            x_hat = symbol_decisions(code, M)
            margins.append(symbol_margin(code, M))
            fok = True
        else:
            x_hat = bit_decisions(code, M)
            fs = fourier_syndrome(code, M)
            margins.append(decision_margin(code, M))
            fok = not np.any(fs)
        es = code.syndrome(x_hat)
        ok = not np.any(es)
        if decision != "symbol" and fok and not ok:
            fourier_only += 1
        if trace:
            hist.append({"c2v": c2v, "v2c": v2c, "M": M, "x": x_hat.copy()})
        if fok and ok:
            break
    out = {"symbols": x_hat, "ok": bool(ok), "iters": it, "fourier_ok": bool(fok), "margins": margins,
           "fourier_only": fourier_only}
    if trace:
        out["trace"] = hist
    return out
