"""Pins of the oracle's two margin helpers, which decide which frames and variables the GPU
decision tests compare (a frame or variable is compared where its FP64 margin exceeds 1e-3).

On a cycle-free graph the converged M_v is the Fourier transform of the exact symbol marginal
(Section 2.1: SP is exact on trees; Section 3.2: M_v is the transform of mu_v), so:
* decision_margin = the smallest |E[(-1)^{z.x_v}]| over the points that decide something: bit i
  of x_v (Section 3.1), and bit i of h_cv x_v for every edge (c, v) (the Fourier-domain syndrome
  of Section 3.2, since bit i of s_c is the XOR over v of bit i of h_cv x_v);
* symbol_margin = the smallest gap between the two most probable symbols of a variable.
Both are recomputed here from brute-force marginals, with the syndrome parities taken through a
bit-serial GF(2^m) multiply of every symbol (no index map), so a helper that reads M at the wrong
point (say z instead of H_cv z) or divides by the wrong total fails.
"""

import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import logfourier as LF
from oracle.code import OracleCode
from paper_1008_4370_gb300 import synth


def _gf_mul_bitserial(a: int, b: int, m: int, poly: int) -> int:
    r = 0
    for i in range(m):
        if (b >> i) & 1:
            r ^= a
        a <<= 1
        if a >> m:
            a ^= poly
    return r


def _converged_tree(m, n_checks, k, seed, trial):
    code = synth.tree_code(n_checks, k, m, seed=seed)
    oc = OracleCode.from_dict(code)
    rng = np.random.default_rng(100 * seed + trial)
    llr = rng.normal(0.8, 2.0, size=(oc.N, m))
    lam0, v = LF.init(oc, llr)
    for _ in range(2 * n_checks + 2):  # more than the graph diameter
        c = LF.check_update(oc, v)
        v = LF.var_update(oc, lam0, c)
    M = LF.tentative(oc, lam0, c)
    marg = BF.symbol_marginals(oc, llr, BF.codewords(oc))
    return code, oc, M, marg


def _bruteforce_decision_margin(code, oc, marg):
    m, q, poly = oc.m, oc.q, int(code["poly"])
    xs = np.arange(q)
    worst = np.inf
    for i in range(m):  # bit decisions: E[(-1)^{bit i of x_v}]
        sgn = np.where((xs >> i) & 1, -1.0, 1.0)
        worst = min(worst, np.min(np.abs(marg @ sgn)))
    for e in range(oc.E):  # syndrome bits: E[(-1)^{bit i of h x_v}]
        h, v = int(oc.edge_h[e]), int(oc.edge_var[e])
        hx = np.array([_gf_mul_bitserial(h, int(x), m, poly) for x in xs])
        for i in range(m):
            sgn = np.where((hx >> i) & 1, -1.0, 1.0)
            worst = min(worst, abs(float(marg[v] @ sgn)))
    return worst


CASES = [(2, 3, 3, 3), (3, 2, 3, 5), (4, 2, 3, 2), (2, 4, 2, 9)]


@pytest.mark.parametrize("m,n_checks,k,seed", CASES)
def test_decision_margin_equals_bruteforce(m, n_checks, k, seed):
    for trial in range(3):
        code, oc, M, marg = _converged_tree(m, n_checks, k, seed, trial)
        assert abs(LF.decision_margin(oc, M) - _bruteforce_decision_margin(code, oc, marg)) < 1e-10


@pytest.mark.parametrize("m,n_checks,k,seed", CASES)
def test_symbol_margin_equals_bruteforce(m, n_checks, k, seed):
    for trial in range(3):
        _, oc, M, marg = _converged_tree(m, n_checks, k, seed, trial)
        srt = np.sort(marg, axis=1)
        assert abs(LF.symbol_margin(oc, M) - float(np.min(srt[:, -1] - srt[:, -2]))) < 1e-10


def test_planted_wrong_readout_point_fails_the_pin():
    """A decision margin that reads the syndrome points at alpha^{i-1} instead of H_cv
    alpha^{i-1} (identity index map) differs from brute force on some tree case, so the pin above
    would catch that slip."""
    differs = 0
    for m, n_checks, k, seed in CASES:
        for trial in range(3):
            code, oc, M, marg = _converged_tree(m, n_checks, k, seed, trial)
            planted = OracleCode.from_dict(code)
            planted.perm = np.tile(np.arange(oc.q), (oc.E, 1))
            bf = _bruteforce_decision_margin(code, oc, marg)
            differs += abs(LF.decision_margin(planted, M) - bf) > 1e-6
    assert differs >= 1
