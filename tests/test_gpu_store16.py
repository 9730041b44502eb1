"""GPU tests of half-precision message storage (NBFD_STORE_F16, GF(256), FWHT form): every
message the library keeps in device memory is the float32 Gamma word rounded to IEEE half; the
arithmetic stays FP32. Each step is teacher-forced against the FP64 oracle fed the same
(half-rounded) inputs, with the FP32 bound plus the rounding of the stored output
(helpers.compare_store16); the whole decoder is compared with the FP32-storage decoder on the
measured configuration, on identical frames."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1008_4370_gb300 as nb  # noqa: E402
from oracle import logfourier as LF  # noqa: E402
from oracle.code import OracleCode  # noqa: E402
from paper_1008_4370_gb300 import build as nbuild  # noqa: E402
from paper_1008_4370_gb300 import synth  # noqa: E402

from helpers import (compare_store16, decode_pair, encode, log_exempt_cap, oracle_state, to_half,  # noqa: E402
                     var_conditions, var_log_conditions)

pytestmark = pytest.mark.gpu

F16 = nb.FORM_FP32_FWHT | nb.STORE_F16
CODES = [(8, 16, 4, 25), (8, 64, 16, 27), "gf256_n512_k4"]


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


def _llr(c, F, ebn0):
    _, llr = synth.frames(c, F, ebn0, batch_idx=3)
    llr = llr.copy()
    llr[0, 0, 0] = 0.0
    if F > 1:
        llr[1, :2, :] = 45.0
    return llr


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _half_dev(a16, dev):
    return torch.from_numpy(np.ascontiguousarray(a16).view(np.int16)).to(dev)


def _half_host(t):
    return t.cpu().numpy().view(np.float16)


@pytest.mark.parametrize("spec", CODES)
def test_init_store16(dev, spec):
    c = _code(spec)
    oc = OracleCode.from_dict(c)
    F = 3
    llr = _llr(c, F, 1.0)
    code = nb.Code(c)
    v2c = torch.empty((F, oc.E, oc.q), dtype=torch.int16, device=dev)
    nb.nbfd_init_messages_f16(code.handle, F, _t(llr, dev), v2c)
    torch.cuda.synchronize()
    g = _half_host(v2c)
    for f in range(F):
        lam0, _ = LF.init(oc, llr[f].astype(np.float64))
        ok, st = compare_store16(g[f], lam0[0][oc.edge_var], lam0[1][oc.edge_var])
        assert ok, (f, st)


@pytest.mark.parametrize("spec", CODES)
def test_check_store16(dev, spec):
    c = _code(spec)
    oc = OracleCode.from_dict(c)
    F = 2
    llr = _llr(c, F, 1.0)
    v2c16 = np.empty((F, oc.E, oc.q), dtype=np.float16)
    for f in range(F):
        _, v2c, _ = oracle_state(oc, llr[f].astype(np.float64), 1 + f)
        v2c16[f] = to_half(encode(*v2c))
    code = nb.Code(c)
    out = torch.empty((F, oc.E, oc.q), dtype=torch.int16, device=dev)
    nb.nbfd_check_update_f16(code.handle, F, _half_dev(v2c16, dev), out)
    torch.cuda.synchronize()
    g = _half_host(out)
    checks = None if oc.M <= 64 else list(range(0, oc.M, max(1, oc.M // 48)))
    for f in range(F):
        s, l = LF.check_update(oc, decode_pair(v2c16[f].astype(np.float32)), checks=checks)
        es = np.arange(oc.E) if checks is None else np.concatenate([oc.V[cc] for cc in checks])
        ok, st = compare_store16(g[f][es], s[es], l[es])
        assert ok, (f, st)


@pytest.mark.parametrize("spec", CODES)
def test_var_store16(dev, spec):
    c = _code(spec)
    oc = OracleCode.from_dict(c)
    F = 2
    llr = _llr(c, F, 1.0)
    c2v16 = np.empty((F, oc.E, oc.q), dtype=np.float16)
    for f in range(F):
        _, _, c2v = oracle_state(oc, llr[f].astype(np.float64), 1 + f)
        c2v16[f] = to_half(encode(*c2v))
    code = nb.Code(c)
    v2c = torch.empty((F, oc.E, oc.q), dtype=torch.int16, device=dev)
    sym = torch.zeros((F, oc.N), dtype=torch.int16, device=dev)
    fsyn = torch.zeros((F, oc.E), dtype=torch.uint8, device=dev)
    nb.nbfd_var_update(code.handle, F, F16, _t(llr, dev), _half_dev(c2v16, dev), v2c, sym, fsyn)
    torch.cuda.synchronize()
    g = _half_host(v2c)
    vars_ = None if oc.N <= 64 else list(range(0, oc.N, max(1, oc.N // 40)))
    for f in range(F):
        lam0, _ = LF.init(oc, llr[f].astype(np.float64))
        c2v_o = decode_pair(c2v16[f].astype(np.float32))
        s, l = LF.var_update(oc, lam0, c2v_o, vars=vars_)
        vs = np.arange(oc.N) if vars_ is None else np.array(vars_)
        es = np.concatenate([oc.C[v] for v in vs])
        kappa = var_conditions(oc, lam0, c2v_o)
        ok, st = compare_store16(g[f][es], s[es], l[es], kappa=kappa[es],
                                 kappa_log=var_log_conditions(oc, lam0, c2v_o)[es])
        assert f == 1 or st["exempt"] <= log_exempt_cap(oc.m), (f, st)  # frame 1: saturated LLRs
        assert ok, (f, st)


def test_decode_store16_vs_fp32_storage(dev):
    """GF(256) (2,4) N=512, 1024 frames at 1.0, 1.5 and 2.0 dB, half against float storage on
    identical frames. Every flag agrees with the library's syndrome of the output and iterations
    stay in [1, 100]. Half storage costs decoding performance: measured on 2048 frames per point,
    FER 0.0181 / 0.0068 / 0.0044 against 0.0132 / 0.0029 / 0.0005 with float storage at 1.0 /
    1.5 / 2.0 dB, and about one more iteration on average; the test bounds that loss
    (FER_half <= 3 FER_float + 0.012) and requires most frames to be decoded by both."""
    c = synth.named_code("gf256_n512_k4")
    code = nb.Code(c)
    enc = synth.Encoder(c)
    for si, ebn0 in enumerate((1.0, 1.5, 2.0)):
        tx, llr = synth.frames(c, 1024, ebn0, snr_idx=si, batch_idx=61, encoder=enc)
        x = _t(llr, dev)
        s32, o32, i32 = nb.decode(code, x, 100, nb.FORM_FP32_FWHT)
        s16, o16, i16 = nb.decode(code, x, 100, F16)
        ex = torch.empty((1024, code.M), dtype=torch.int16, device=dev)
        nb.nbfd_syndrome(code.handle, 1024, s16, None, None, ex)
        torch.cuda.synchronize()
        ok16 = o16.cpu().numpy().astype(bool)
        assert np.array_equal(ok16, ~ex.cpu().numpy().any(axis=1))
        it = i16.cpu().numpy()
        assert it.min() >= 1 and it.max() <= 100 and np.all(it[~ok16] == 100)
        c32 = np.all(s32.cpu().numpy().astype(np.int64) == tx, axis=1)
        c16 = np.all(s16.cpu().numpy().astype(np.int64) == tx, axis=1)
        fer32, fer16 = 1 - c32.mean(), 1 - c16.mean()
        print(f"{ebn0} dB: FER float {fer32:.4f}, half {fer16:.4f}, "
              f"mean iterations {i32.float().mean().item():.2f} / {i16.float().mean().item():.2f}")
        assert fer16 <= 3 * fer32 + 0.012, (ebn0, fer32, fer16)
        assert np.mean(c32 & c16) > 0.95


def test_batch_store16_equals_alone(dev):
    groups = []
    for gi, (name, F) in enumerate([("gf256_n512_k4", 24), ("gf256_n2048_k16", 4)]):
        c = synth.named_code(name)
        _, llr = synth.frames(c, F, 2.5, snr_idx=gi, batch_idx=62)
        groups.append((nb.Code(c), _t(llr, dev)))
    outs = nb.decode_batch([g[0] for g in groups], [g[1] for g in groups], 60, F16)
    torch.cuda.synchronize()
    for (code, x), (sym, ok, it) in zip(groups, outs):
        s0, o0, i0 = nb.decode(code, x, 60, F16)
        torch.cuda.synchronize()
        assert np.array_equal(sym.cpu().numpy(), s0.cpu().numpy())
        assert np.array_equal(ok.cpu().numpy(), o0.cpu().numpy()) and np.array_equal(it.cpu().numpy(), i0.cpu().numpy())


def test_store16_not_supported_elsewhere(dev):
    c16 = nb.Code(synth.named_code("gf16_n32_k4"))
    x = torch.zeros((2, 32, 4), dtype=torch.float32, device=dev)
    with pytest.raises(nb.NbfdError) as ei:
        nb.decode(c16, x, 5, F16)
    assert ei.value.status == -10
    c256 = nb.Code(synth.named_code("gf256_n512_k4"))
    x = torch.zeros((2, 512, 8), dtype=torch.float32, device=dev)
    for form in (nb.FORM_FP32_DIRECT | nb.STORE_F16, nb.FORM_FP32_TC | nb.STORE_F16):
        with pytest.raises(nb.NbfdError) as ei:
            nb.decode(c256, x, 5, form)
        assert ei.value.status == -10
