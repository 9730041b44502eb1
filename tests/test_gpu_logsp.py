"""GPU parity of the conventional Log-SP steps (Section 2.2) against the FP64 oracle.

Log-SP messages are the logarithms of the probability-domain SP messages of Section 2.1 up to a
constant per vector (the paper shows the outputs are the same), so each step is teacher-forced on
oracle SP states: the GPU's log-domain output, exponentiated and scaled to a maximum of 1, must
match the oracle's (``oracle.sp``, O(q^2) convolutions from the definition, pinned to the
Log-Fourier decoder at 1e-10) scaled the same way. Every term of a log-convolution is positive,
so there is no cancellation: the FP32 error is a few ulp per level of the prefix / suffix
products (relative), held to |dP| <= 1e-5 everywhere and |d ln P| <= 1e-4 where P >= 2^-7.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1008_4370_gb300 as nb  # noqa: E402
from oracle import sp  # noqa: E402
from oracle.channel import symbol_probabilities  # noqa: E402
from oracle.code import OracleCode  # noqa: E402
from paper_1008_4370_gb300 import build as nbuild  # noqa: E402
from paper_1008_4370_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

LIN_ATOL, LOG_ATOL, LOG_FLOOR = 1e-5, 1e-4, 2.0 ** -7


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    nbuild.build()
    return torch.device("cuda:0")


def _code(spec):
    if isinstance(spec, str):
        return synth.named_code(spec)
    m, N, k, seed = spec
    c = synth.regular_code(N, k, m, seed=seed)
    c["seed"] = seed
    return c


CODES = [(3, 12, 4, 21), "gf16_n32_k4", (6, 24, 6, 23), (8, 16, 4, 25), "gf256_n512_k4", (8, 64, 16, 27)]


def _sp_states(oc, llr, iters):
    """(p0, v2c, c2v) of the oracle SP decoder after `iters` iterations (c2v None at 0)."""
    p0, v2c = sp.init(oc, llr)
    c2v = None
    for _ in range(iters):
        c2v = sp.check_update(oc, v2c)
        v2c = sp.var_update(oc, p0, c2v)
    return p0, v2c, c2v


def _log32(p):
    with np.errstate(divide="ignore"):
        return np.log(p).astype(np.float32)


def _compare(lam_gpu, p_ref):
    """Both sides scaled to max 1 per vector; returns (ok, stats)."""
    with np.errstate(over="ignore", invalid="ignore"):
        g = np.exp(lam_gpu.astype(np.float64) - np.max(lam_gpu, axis=-1, keepdims=True))
    r = p_ref / p_ref.max(axis=-1, keepdims=True)
    lin = np.abs(g - r)
    mask = r >= LOG_FLOOR
    with np.errstate(divide="ignore"):
        logerr = np.abs(np.log(g[mask]) - np.log(r[mask])) if mask.any() else np.zeros(1)
    st = {"lin_max": float(lin.max()), "log_max": float(logerr.max()), "nan": int(np.isnan(lam_gpu).sum())}
    return st["lin_max"] <= LIN_ATOL and st["log_max"] <= LOG_ATOL and st["nan"] == 0, st


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.mark.parametrize("spec", CODES)
def test_logsp_init(dev, spec):
    c = _code(spec)
    oc = OracleCode.from_dict(c)
    _, llr = synth.frames(c, 2, 1.0, batch_idx=4)
    code = nb.Code(c)
    v2c = torch.empty((2, oc.E, oc.q), dtype=torch.float32, device=dev)
    nb.nbfd_logsp_init(code.handle, 2, _t(llr, dev), v2c)
    torch.cuda.synchronize()
    g = v2c.cpu().numpy().astype(np.float64)
    for f in range(2):
        ref = np.log(symbol_probabilities(llr[f].astype(np.float64)))[oc.edge_var]
        assert np.max(np.abs(g[f] - ref) / np.maximum(1.0, np.abs(ref))) < 1e-5


@pytest.mark.parametrize("spec", CODES)
def test_logsp_check_parity(dev, spec):
    c = _code(spec)
    oc = OracleCode.from_dict(c)
    F = 3
    _, llr = synth.frames(c, F, 1.0, batch_idx=5)
    lam_in = np.empty((F, oc.E, oc.q), dtype=np.float32)
    for f in range(F):
        _, v2c, _ = _sp_states(oc, llr[f].astype(np.float64), f)  # iterations 0, 1, 2
        lam_in[f] = _log32(v2c)
    code = nb.Code(c)
    out = torch.empty_like(_t(lam_in, dev))
    nb.nbfd_logsp_check_update(code.handle, F, _t(lam_in, dev), out)
    torch.cuda.synchronize()
    g = out.cpu().numpy()
    for f in range(F):
        ref = sp.check_update(oc, np.exp(lam_in[f].astype(np.float64)))
        ok, st = _compare(g[f], ref)
        assert ok, (f, st)
        assert np.all(g[f] <= 0.0) and np.all(np.max(g[f], axis=-1) == 0.0)  # lambda in [-inf, 0]


@pytest.mark.parametrize("spec", CODES)
def test_logsp_var_parity(dev, spec):
    c = _code(spec)
    oc = OracleCode.from_dict(c)
    F = 2
    _, llr = synth.frames(c, F, 1.0, batch_idx=6)
    lam_in = np.empty((F, oc.E, oc.q), dtype=np.float32)
    for f in range(F):
        _, _, c2v = _sp_states(oc, llr[f].astype(np.float64), 1 + f)
        lam_in[f] = _log32(c2v / c2v.max(axis=-1, keepdims=True))
    code = nb.Code(c)
    v2c = torch.empty((F, oc.E, oc.q), dtype=torch.float32, device=dev)
    sym = torch.zeros((F, oc.N), dtype=torch.int16, device=dev)
    nb.nbfd_logsp_var_update(code.handle, F, _t(llr, dev), _t(lam_in, dev), v2c, sym)
    torch.cuda.synchronize()
    g, gs = v2c.cpu().numpy(), sym.cpu().numpy().astype(np.int64)
    n_dec = 0
    for f in range(F):
        p0 = symbol_probabilities(llr[f].astype(np.float64))
        c2v = np.exp(lam_in[f].astype(np.float64))
        ok, st = _compare(g[f], sp.var_update(oc, p0, c2v))
        assert ok, (f, st)
        assert np.all(g[f][:, 0] == 0.0)  # normalised to lambda(0) = 0
        qv = sp.marginals(oc, p0, c2v)
        srt = np.sort(qv, axis=-1)
        clear = (srt[:, -1] - srt[:, -2]) > 1e-3 * srt[:, -1]
        n_dec += int(clear.sum())
        assert np.array_equal(gs[f][clear], np.argmax(qv, axis=-1)[clear]), f
    assert n_dec > 0


def test_logsp_decisions_follow_the_oracle_over_iterations(dev):
    """Three whole Log-SP iterations on the GPU (init, check, variable, repeated) against the
    oracle SP decoder on the tiny configuration's code: the argmax decisions agree wherever the
    oracle's top two symbols are apart, at every iteration."""
    c = synth.named_code("gf16_n32_k4")
    oc = OracleCode.from_dict(c)
    code = nb.Code(c)
    F = 8
    _, llr = synth.frames(c, F, 2.0, zero_codeword=True, batch_idx=8)
    x = _t(llr, dev)
    v2c = torch.empty((F, oc.E, oc.q), dtype=torch.float32, device=dev)
    c2v = torch.empty_like(v2c)
    sym = torch.zeros((F, oc.N), dtype=torch.int16, device=dev)
    nb.nbfd_logsp_init(code.handle, F, x, v2c)
    states = [sp.init(oc, llr[f].astype(np.float64)) for f in range(F)]
    n_cmp = 0
    for _ in range(3):
        nb.nbfd_logsp_check_update(code.handle, F, v2c, c2v)
        nb.nbfd_logsp_var_update(code.handle, F, x, c2v, v2c, sym)
        torch.cuda.synchronize()
        gs = sym.cpu().numpy().astype(np.int64)
        for f in range(F):
            p0, vf = states[f]
            cf = sp.check_update(oc, vf)
            states[f] = (p0, sp.var_update(oc, p0, cf))
            qv = sp.marginals(oc, p0, cf)
            srt = np.sort(qv, axis=-1)
            clear = (srt[:, -1] - srt[:, -2]) > 1e-3
            n_cmp += int(clear.sum())
            assert np.array_equal(gs[f][clear], np.argmax(qv, axis=-1)[clear])
    assert n_cmp > 3 * F * oc.N // 2


def test_logsp_rejects_unsupported_fields(dev):
    c = synth.named_code("gf4_n8_k4")
    code = nb.Code(c)
    v = torch.zeros((1, 16, 4), dtype=torch.float32, device=dev)
    with pytest.raises(nb.NbfdError) as ei:
        nb.nbfd_logsp_check_update(code.handle, 1, v, v.clone())
    assert ei.value.status == -10
