"""Pins of the two FP64 oracle decoders against each other and against brute force.

Section 2.1 (SP), Section 3.1 (Fourier SP and its bit / syndrome read-out), Section 3.2
(Log-Fourier SP). The Log-Fourier decoder is designed to output what SP outputs (Section 3), so
its Gamma-form messages must be the Fourier transforms of SP's probability messages; on
cycle-free graphs SP is exact symbol-MAP (Section 2.1) and the Fourier read-out is exact bit-MAP
(Section 3.1).
"""

import copy

import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import logfourier as LF
from oracle import sp
from oracle.code import OracleCode
from oracle.transforms import gamma_inv, wht
from paper_1008_4370_gb300 import synth


def _run_both(oc, llr, iters):
    p0, v_sp = sp.init(oc, llr)
    lam0, v_lf = LF.init(oc, llr)
    out = []
    for _ in range(iters):
        c_sp = sp.check_update(oc, v_sp)
        c_lf = LF.check_update(oc, v_lf)
        v_sp = sp.var_update(oc, p0, c_sp)
        v_lf = LF.var_update(oc, lam0, c_lf)
        out.append((c_sp, c_lf, v_sp, v_lf, p0, lam0))
    return out


def _max_msg_gap(oc, llr, iters):
    gap = 0.0
    for c_sp, c_lf, v_sp, v_lf, _, _ in _run_both(oc, llr, iters):
        gap = max(gap, np.abs(gamma_inv(*c_lf) - wht(c_sp)).max())
        gap = max(gap, np.abs(gamma_inv(*v_lf) - wht(v_sp)).max())
    return gap


@pytest.mark.parametrize("name,ebn0", [("gf16_n32_k4", 1.0), ("gf4_n8_k4", 0.0)])
def test_logfourier_messages_equal_sp_messages(name, ebn0):
    code = synth.named_code(name)
    oc = OracleCode.from_dict(code)
    _, llr = synth.frames(code, 3, ebn0)
    for f in range(3):
        assert _max_msg_gap(oc, llr[f], 5) < 1e-10


def test_logfourier_messages_equal_sp_messages_gf64_k6():
    code = synth.regular_code(24, 6, 6, seed=11)
    code["seed"] = 11
    oc = OracleCode.from_dict(code)
    _, llr = synth.frames(code, 1, 1.0)
    assert _max_msg_gap(oc, llr[0], 3) < 1e-10


def test_fourier_bit_readout_equals_bit_marginals():
    """Section 3.1: M_v(alpha^{i-1}) / M_v(0) = q_{v,i}(0) - q_{v,i}(1)."""
    code = synth.named_code("gf16_n32_k4")
    oc = OracleCode.from_dict(code)
    _, llr = synth.frames(code, 2, 1.5)
    for f in range(2):
        p0, v_sp = sp.init(oc, llr[f])
        lam0, v_lf = LF.init(oc, llr[f])
        for _ in range(3):
            c_sp = sp.check_update(oc, v_sp)
            c_lf = LF.check_update(oc, v_lf)
            v_sp = sp.var_update(oc, p0, c_sp)
            v_lf = LF.var_update(oc, lam0, c_lf)
            bias = sp.bit_bias(sp.marginals(oc, p0, c_sp), oc.m)
            Ms, Ml = LF.tentative(oc, lam0, c_lf)
            M = gamma_inv(Ms, Ml)
            for i in range(oc.m):
                np.testing.assert_allclose(M[:, 1 << i] / M[:, 0], bias[:, i], atol=1e-10)
            x_lf = LF.bit_decisions(oc, (Ms, Ml))
            clear = np.all(np.abs(bias) > 1e-9, axis=1)
            x_bias = ((bias < 0).astype(np.int64) << np.arange(oc.m)).sum(1)
            assert np.array_equal(x_lf[clear], x_bias[clear])


@pytest.mark.parametrize("m,n_checks,k,seed", [(2, 3, 3, 3), (3, 2, 3, 5), (4, 2, 3, 2), (2, 4, 2, 9)])
def test_tree_marginals_are_exact(m, n_checks, k, seed):
    """Cycle-free graph: SP marginals equal brute-force symbol marginals; the Log-Fourier bit
    decisions equal brute-force bit-MAP."""
    code = synth.tree_code(n_checks, k, m, seed=seed)
    oc = OracleCode.from_dict(code)
    cw = BF.codewords(oc)
    rng = np.random.default_rng(seed)
    for trial in range(3):
        llr = rng.normal(0.8, 2.0, size=(oc.N, m))
        marg = BF.symbol_marginals(oc, llr, cw)
        p0, v = sp.init(oc, llr)
        lam0, vl = LF.init(oc, llr)
        for _ in range(2 * n_checks + 2):  # more than the graph diameter
            c = sp.check_update(oc, v)
            v = sp.var_update(oc, p0, c)
            cl = LF.check_update(oc, vl)
            vl = LF.var_update(oc, lam0, cl)
        np.testing.assert_allclose(sp.marginals(oc, p0, c), marg, atol=1e-12)
        x_map, bias = BF.bit_map(oc, marg)
        M = LF.tentative(oc, lam0, cl)
        x_lf = LF.bit_decisions(oc, M)
        clear = np.all(np.abs(bias) > 1e-9, axis=1)
        assert np.array_equal(x_lf[clear], x_map[clear])
        Mlin = gamma_inv(*M)
        for i in range(m):
            np.testing.assert_allclose(Mlin[:, 1 << i] / Mlin[:, 0], bias[:, i], atol=1e-10)


def test_gf4_n8_loopy_decisions_vs_bruteforce_symbol_map():
    """Loopy graph: BP is not MAP, so only the agreement rate is pinned (it must be high at a
    moderate SNR; brute force enumerates all 4^8 words)."""
    code = synth.named_code("gf4_n8_k4")
    oc = OracleCode.from_dict(code)
    cw = BF.codewords(oc)
    enc = synth.Encoder(code)
    assert len(cw) == 4 ** enc.info_symbols
    tx, llr = synth.frames(code, 40, 2.0)
    agree = 0
    for f in range(40):
        marg = BF.symbol_marginals(oc, llr[f], cw)
        r = sp.decode(oc, llr[f], 20)
        agree += int(np.array_equal(r["symbols"], np.argmax(marg, axis=1)))
    assert agree >= 34


def test_decode_recovers_codeword_at_high_snr():
    code = synth.named_code("gf16_n32_k4")
    oc = OracleCode.from_dict(code)
    tx, llr = synth.frames(code, 6, 4.0)
    for f in range(6):
        r = LF.decode(oc, llr[f], 50)
        assert r["ok"] and r["fourier_ok"] and 1 <= r["iters"] <= 50
        assert np.array_equal(r["symbols"], tx[f])


def test_fourier_syndrome_is_exact_when_decisions_are_confident():
    """Section 3.2: when every q_v concentrates on one symbol, the Fourier-domain syndrome bits
    are the bits of sum_v h_cv x_hat_v."""
    code = synth.named_code("gf16_n32_k4")
    oc = OracleCode.from_dict(code)
    tx, llr = synth.frames(code, 4, 1.0)
    for f in range(4):
        r = LF.decode(oc, llr[f], 30, trace=True)
        for step in r["trace"]:
            if LF.decision_margin(oc, step["M"]) > 0.5:
                assert np.array_equal(LF.fourier_syndrome(oc, step["M"]), oc.syndrome(step["x"]))


def test_fourier_parity_differs_from_xor_of_bits_counterexample():
    """Reading of Section 3.2: sign M(z) for a multi-bit z is the MAP of the parity z.x, not the
    XOR of the bitwise decisions. q = (.3, .35, .35, 0) over GF(4)."""
    qv = np.array([0.3, 0.35, 0.35, 0.0])
    Q = wht(qv)
    assert Q[1] > 0 and Q[2] > 0  # both bit decisions are 0
    assert Q[3] < 0  # but the parity of the two bits decides 1


# --- planted mistakes: each must make one of the pins above fail --------------------------

def test_planted_untransposed_index_map_breaks_sp_equality():
    code = synth.named_code("gf16_n32_k4")
    oc = OracleCode.from_dict(code)
    bad = copy.copy(oc)
    xs = np.arange(oc.q)
    bad.perm = np.stack([oc.gf.mul(int(h), xs) for h in oc.edge_h])
    bad.perm_inv = np.stack([oc.gf.mul(int(oc.gf.inv(int(h))), xs) for h in oc.edge_h])
    _, llr = synth.frames(code, 1, 1.0)
    assert _max_msg_gap(oc, llr[0], 2) < 1e-10
    assert _max_msg_gap(bad, llr[0], 2) > 1e-3


def test_planted_missing_normalisation_breaks_sp_equality(monkeypatch):
    code = synth.named_code("gf16_n32_k4")
    oc = OracleCode.from_dict(code)
    _, llr = synth.frames(code, 1, 1.0)
    monkeypatch.setattr(LF, "normalize_at_zero", lambda v: v)
    assert _max_msg_gap(oc, llr[0], 2) > 1e-6


def test_planted_leave_one_out_error_breaks_sp_equality(monkeypatch):
    code = synth.named_code("gf16_n32_k4")
    oc = OracleCode.from_dict(code)
    _, llr = synth.frames(code, 1, 1.0)
    real = LF.check_update

    def include_self(code_, v2c, checks=None):
        s, l = real(code_, v2c, checks)
        s2, l2 = v2c
        return s ^ s2, l + l2  # adds the edge's own message (a dropped "v' != v")

    monkeypatch.setattr(LF, "check_update", include_self)
    assert _max_msg_gap(oc, llr[0], 2) > 1e-3


def test_symbol_decisions_equal_sp_argmax():
    """Section 3.2 first form: argmax of mu_v (inverse transform of M_v) is SP's symbol decision."""
    code = synth.named_code("gf16_n32_k4")
    oc = OracleCode.from_dict(code)
    _, llr = synth.frames(code, 2, 1.0)
    for f in range(2):
        p0, v_sp = sp.init(oc, llr[f])
        lam0, v_lf = LF.init(oc, llr[f])
        for _ in range(3):
            c_sp = sp.check_update(oc, v_sp)
            c_lf = LF.check_update(oc, v_lf)
            v_sp = sp.var_update(oc, p0, c_sp)
            v_lf = LF.var_update(oc, lam0, c_lf)
            qv = sp.marginals(oc, p0, c_sp)
            x = LF.symbol_decisions(oc, LF.tentative(oc, lam0, c_lf))
            srt = np.sort(qv, axis=1)
            clear = (srt[:, -1] - srt[:, -2]) > 1e-9
            assert np.array_equal(x[clear], np.argmax(qv, axis=1)[clear])


def test_symbol_decisions_are_symbol_map_on_trees():
    code = synth.tree_code(3, 3, 2, seed=3)
    oc = OracleCode.from_dict(code)
    cw = BF.codewords(oc)
    rng = np.random.default_rng(8)
    for _ in range(3):
        llr = rng.normal(0.8, 2.0, size=(oc.N, 2))
        marg = BF.symbol_marginals(oc, llr, cw)
        lam0, v = LF.init(oc, llr)
        for _ in range(8):
            c = LF.check_update(oc, v)
            v = LF.var_update(oc, lam0, c)
        x = LF.symbol_decisions(oc, LF.tentative(oc, lam0, c))
        srt = np.sort(marg, axis=1)
        clear = (srt[:, -1] - srt[:, -2]) > 1e-9
        assert np.array_equal(x[clear], np.argmax(marg, axis=1)[clear])
        r = LF.decode(oc, llr, 8, decision="symbol")
        assert r["iters"] >= 1
