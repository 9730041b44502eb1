"""GPU parity: every step of the CUDA path against the FP64 oracle, called through the C ABI.

Per-step tests are teacher-forced: the oracle produces realistic message states, they are rounded
to the library's float32 encoding, and both sides compute one step from those same inputs.
Decode tests run the whole loop on both sides from the same seeded LLRs.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1008_4370_gb300 as nb  # noqa: E402
from oracle import logfourier as LF  # noqa: E402
from oracle.code import OracleCode  # noqa: E402
from paper_1008_4370_gb300 import build as nbuild  # noqa: E402
from paper_1008_4370_gb300 import synth  # noqa: E402

from helpers import (MARGIN, compare, decode_pair, encode, log_exempt_cap, oracle_decodes, oracle_state,  # noqa: E402
                     var_conditions, var_log_conditions, vn_margins)

pytestmark = pytest.mark.gpu


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
    c["name"] = f"gf{1 << m}_n{N}_k{k}"
    return c


# small codes over every field size the kernels are instantiated for, plus the configured codes
STEP_CODES = [
    "gf4_n8_k4", (3, 12, 4, 21), "gf16_n32_k4", (5, 20, 4, 22), (6, 24, 6, 23), (6, 30, 6, 28),
    (7, 16, 4, 24),
    (8, 16, 4, 25), (4, 80, 20, 26), (8, 64, 16, 27),
]


def _llr(code, F, ebn0, special=True, batch=0):
    _, llr = synth.frames(code, F, ebn0, batch_idx=batch)
    if special:
        llr = llr.copy()
        llr[0, 0, 0] = 0.0  # a bit with no information: P0(z) = 0 wherever z_1 = 1
        if F > 1:
            llr[1, :2, :] = 45.0  # saturated channel
            llr[1, 2, :] = -45.0
    return llr


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def test_code_tables_roundtrip(dev):
    c = synth.named_code("gf256_n512_k4")
    code = nb.Code(c)
    assert nb.nbfd_code_info(code.handle) == (512, 256, 4, 8)
    assert np.array_equal(nb.nbfd_code_edge_order(code.handle, code.E), np.arange(code.E))
    oc = OracleCode.from_dict(c)
    tab = nb.nbfd_code_index_map(code.handle, 256)
    for h in range(1, 256, 17):
        assert np.array_equal(tab[h], oc.gf.fourier_index_map(h))
    # edges given in a shuffled order come back check-major
    rng = np.random.default_rng(0)
    p = rng.permutation(code.E)
    c2 = dict(c, edge_check=c["edge_check"][p], edge_var=c["edge_var"][p], edge_h=c["edge_h"][p])
    code2 = nb.Code(c2)
    order = nb.nbfd_code_edge_order(code2.handle, code.E)
    assert np.array_equal(c2["edge_check"][order], c["edge_check"])
    assert sorted(order.tolist()) == list(range(code.E))


@pytest.mark.parametrize("spec", STEP_CODES + ["gf256_n512_k4"])
def test_init_parity(dev, spec):
    c = _code(spec)
    oc = OracleCode.from_dict(c)
    F = 3
    llr = _llr(c, F, 1.0)
    code = nb.Code(c)
    lam0 = torch.empty((F, oc.N, oc.q), dtype=torch.float32, device=dev)
    v2c = torch.empty((F, oc.E, oc.q), dtype=torch.float32, device=dev)
    nb.nbfd_init_messages(code.handle, F, _t(llr, dev), lam0, v2c)
    torch.cuda.synchronize()
    g_lam0, g_v2c = lam0.cpu().numpy(), v2c.cpu().numpy()
    for f in range(F):
        o_lam0, _ = LF.init(oc, llr[f].astype(np.float64))
        ok, st = compare(g_lam0[f], *o_lam0)
        assert ok, (f, st)
        assert np.array_equal(g_v2c[f].view(np.uint32), g_lam0[f][oc.edge_var].view(np.uint32))
        assert np.all(g_lam0[f][:, 0] == 0.0) and not np.any(np.signbit(g_lam0[f][:, 0]))


# row weights above 8 at q >= 128 run the check kernel's team variant (a block shares one
# pipeline of whole checks): GF(128) k = 10 and GF(256) k = 20 beside (8, 64, 16, 27) above
@pytest.mark.parametrize("spec", STEP_CODES + ["gf256_n512_k4", "gf64_n1200_k6", (7, 40, 10, 29),
                                  (8, 60, 20, 30)])
def test_check_parity(dev, spec):
    c = _code(spec)
    oc = OracleCode.from_dict(c)
    F = 2
    llr = _llr(c, F, 1.0)
    v2c_in = np.empty((F, oc.E, oc.q), dtype=np.float32)
    for f in range(F):
        _, v2c, _ = oracle_state(oc, llr[f].astype(np.float64), 1 + f)
        v2c_in[f] = encode(*v2c)
    code = nb.Code(c)
    out = torch.empty((F, oc.E, oc.q), dtype=torch.float32, device=dev)
    nb.nbfd_check_update(code.handle, F, _t(v2c_in, dev), out)
    torch.cuda.synchronize()
    g = out.cpu().numpy()
    checks = None if oc.M <= 64 else list(range(0, oc.M, max(1, oc.M // 48)))
    for f in range(F):
        s, l = LF.check_update(oc, decode_pair(v2c_in[f]), checks=checks)
        es = np.arange(oc.E) if checks is None else np.concatenate([oc.V[cc] for cc in checks])
        ok, st = compare(g[f][es], s[es], l[es])
        assert ok, (f, st)


FORMS = [nb.FORM_FP32_DIRECT, nb.FORM_FP32_FWHT]
TC_FORMS = [nb.FORM_BF16_HGEMM, nb.FORM_FP16_HGEMM, nb.FORM_FP32_TC]
# unit roundoff of the operands each form rounds to (FP32 forms: 2^-24)
FORM_UNIT = {nb.FORM_FP32_DIRECT: 2.0 ** -24, nb.FORM_FP32_FWHT: 2.0 ** -24, nb.FORM_FP32_TC: 2.0 ** -24,
             nb.FORM_FP64_DIRECT: 2.0 ** -24,
             nb.FORM_BF16_HGEMM: 2.0 ** -9, nb.FORM_FP16_HGEMM: 2.0 ** -12}
VAR_CASES = ([(sp, f) for sp in STEP_CODES + ["gf256_n512_k4", "gf64_n1200_k6"] for f in FORMS]
             + [(sp, nb.FORM_FP64_DIRECT) for sp in ["gf16_n32_k4", (6, 24, 6, 23), (8, 16, 4, 25), "gf256_n512_k4"]]
             + [(sp, f | path) for sp in [(8, 16, 4, 25), (8, 64, 16, 27), "gf256_n512_k4"] for f in TC_FORMS
                for path in (nb.MMA_SYNC, nb.TCGEN05)])


def _tolerances(form):
    """(linear floor, kappa factor, log bound, decision margin) for a form: the FP32 forms use the
    FP32 bounds of helpers.py; the BF16 / FP16 operand forms a bound scaled by their unit
    roundoff u_p: |dP| <= max(16 u_p, 4 u_p kappa), decisions compared where the FP64 margin
    exceeds 0.1."""
    u = FORM_UNIT[form & 0xff]
    if u == 2.0 ** -24:
        return None, None, 1e-4, MARGIN
    return 16 * u, 4 * u, 1e9, 0.1


@pytest.mark.parametrize("spec,form", VAR_CASES)
def test_var_parity(dev, spec, form):
    c = _code(spec)
    oc = OracleCode.from_dict(c)
    F = 2
    llr = _llr(c, F, 1.0)
    c2v_in = np.empty((F, oc.E, oc.q), dtype=np.float32)
    for f in range(F):
        _, _, c2v = oracle_state(oc, llr[f].astype(np.float64), 1 + f)
        c2v_in[f] = encode(*c2v)
    code = nb.Code(c)
    v2c = torch.empty((F, oc.E, oc.q), dtype=torch.float32, device=dev)
    sym = torch.zeros((F, oc.N), dtype=torch.int16, device=dev)
    fsyn = torch.zeros((F, oc.E), dtype=torch.uint8, device=dev)
    nb.nbfd_var_update(code.handle, F, form, _t(llr, dev), _t(c2v_in, dev), v2c, sym, fsyn)
    torch.cuda.synchronize()
    g, gs, gw = v2c.cpu().numpy(), sym.cpu().numpy().astype(np.int64), fsyn.cpu().numpy().astype(np.int64)
    vars_ = None if oc.N <= 64 else list(range(0, oc.N, max(1, oc.N // 40)))
    n_cmp = 0
    for f in range(F):
        lam0, _ = LF.init(oc, llr[f].astype(np.float64))
        c2v_o = decode_pair(c2v_in[f])
        s, l = LF.var_update(oc, lam0, c2v_o, vars=vars_)
        vs = np.arange(oc.N) if vars_ is None else np.array(vars_)
        es = np.concatenate([oc.C[v] for v in vs])
        kappa = var_conditions(oc, lam0, c2v_o)
        floor, kf, logb, margin = _tolerances(form)
        if floor is None:
            ok, st = compare(g[f][es], s[es], l[es], kappa=kappa[es],
                             kappa_log=var_log_conditions(oc, lam0, c2v_o)[es])
            # frame 1 carries saturated +-45 LLRs against its check messages on purpose (U(0) tiny):
            # its share of entries left out of the log check is not capped
            assert f == 1 or st["exempt"] <= log_exempt_cap(oc.m), (f, st)
        else:
            ok, st = compare(g[f][es], s[es], l[es], kappa=kappa[es] * kf / 2.0 ** -24, lin_atol=floor,
                             log_atol=logb)
        assert ok, (f, st)
        M = LF.tentative(oc, lam0, c2v_o, vars=vs)
        x = LF.bit_decisions(oc, M)
        w = LF.fourier_syndrome_words(oc, M)
        marg = vn_margins(oc, M)
        for v in vs:
            if marg[v] > margin:
                n_cmp += 1
                assert gs[f, v] == x[v], (f, v)
                for e in oc.C[v]:
                    assert gw[f, e] == w[e], (f, v, e)
    assert n_cmp > 0


def test_syndrome_parity(dev):
    c = synth.named_code("gf64_n1200_k6")
    oc = OracleCode.from_dict(c)
    F = 5
    rng = np.random.default_rng(1)
    sym = rng.integers(0, oc.q, size=(F, oc.N)).astype(np.int16)
    sym[0] = synth.Encoder(c).random_codewords(1, rng)[0]
    fsyn = rng.integers(0, oc.q, size=(F, oc.E)).astype(np.uint8)
    code = nb.Code(c)
    fo = torch.empty((F, oc.M), dtype=torch.int16, device=dev)
    ex = torch.empty((F, oc.M), dtype=torch.int16, device=dev)
    nb.nbfd_syndrome(code.handle, F, _t(sym, dev), _t(fsyn, dev), fo, ex)
    torch.cuda.synchronize()
    for f in range(F):
        assert np.array_equal(ex.cpu().numpy()[f], oc.syndrome(sym[f].astype(np.int64)))
        ref = np.zeros(oc.M, dtype=np.int64)
        for e in range(oc.E):
            ref[oc.edge_check[e]] ^= fsyn[f, e]
        assert np.array_equal(fo.cpu().numpy()[f], ref)
    assert not ex.cpu().numpy()[0].any()


_ORACLE_CACHE = {}


def _decode_vs_oracle(dev, c, llr, max_iter, frames=None, min_frac=0.5, form=nb.FORM_FP32_DIRECT,
                      decision="bitwise"):
    """Whole decodes on both sides. Bit-exact symbols and syndrome flags are required on frames
    the oracle decodes (or runs to max_iter) whose last-iteration margin exceeds MARGIN; equal
    iteration counts on frames whose margin exceeds MARGIN at every iteration. Messages do not
    depend on earlier decisions, so only low-margin read-outs can make the two sides differ."""
    oc = OracleCode.from_dict(c)
    code = nb.Code(c)
    F = llr.shape[0]
    sym, ok, it = nb.decode(code, _t(llr, dev), max_iter, form)
    torch.cuda.synchronize()
    sym, ok, it = sym.cpu().numpy().astype(np.int64), ok.cpu().numpy(), it.cpu().numpy()
    n_sym = n_it = 0
    fl = list(range(F) if frames is None else frames)
    key = (c.get("name"), max_iter, decision, tuple(fl), hash(llr[fl].tobytes()))
    if key not in _ORACLE_CACHE:  # the same frames are decoded with several forms
        _ORACLE_CACHE[key] = oracle_decodes(c, llr[fl], max_iter, decision) if len(fl) > 8 else \
            [LF.decode(oc, llr[f].astype(np.float64), max_iter, decision=decision) for f in fl]
    res = _ORACLE_CACHE[key]
    for f, r in zip(fl, res):
        if r["margins"][-1] > MARGIN and (r["ok"] or r["iters"] == max_iter and max_iter <= 4):
            n_sym += 1
            assert np.array_equal(sym[f], r["symbols"]), f
            assert int(ok[f]) == int(r["ok"]), f
        if min(r["margins"]) > MARGIN:
            n_it += 1
            assert int(it[f]) == r["iters"], (f, it[f], r["iters"])
    n = F if frames is None else len(frames)
    assert n_sym >= min_frac * n, (n_sym, n)
    return sym, ok, it, n_sym, n_it


@pytest.mark.parametrize("form", FORMS)
def test_decode_parity_tiny_gf16(dev, form):
    """Tiny configuration: GF(16) (2,4) N=32, all-zero codeword at Eb/N0 = 2 dB, 100 frames,
    at most 50 iterations."""
    c = synth.named_code("gf16_n32_k4")
    _, llr = synth.frames(c, 100, 2.0, zero_codeword=True)
    sym, ok, it, n_sym, n_it = _decode_vs_oracle(dev, c, llr, 50, min_frac=0.6, form=form)
    assert ok.mean() > 0.5 and it.min() >= 1 and it.max() <= 50


@pytest.mark.parametrize("form", FORMS)
def test_fourier_only_clears_count(dev, form):
    """nbfd_last_decode_stats counts the (frame, iteration) pairs where the Fourier-domain
    syndrome cleared while H x_hat != 0 (reading of Section 3.2: the stop test needs both); one
    frame per call, compared with the oracle's count on frames whose margins are clear."""
    c = synth.named_code("gf4_n8_k4")
    oc = OracleCode.from_dict(c)
    code = nb.Code(c)
    _, llr = synth.frames(c, 100, -1.0, batch_idx=5)  # low SNR: the case occurs
    n_cmp = n_hit = total = 0
    for f in range(100):
        nb.decode(code, _t(llr[f:f + 1], dev), 20, form)
        torch.cuda.synchronize()
        got = nb.nbfd_last_decode_stats()
        assert got >= 0
        total += got
        r = LF.decode(oc, llr[f].astype(np.float64), 20)
        if min(r["margins"]) > MARGIN:
            n_cmp += 1
            n_hit += r["fourier_only"] > 0
            assert got == r["fourier_only"], (f, got, r["fourier_only"])
    assert n_cmp > 30 and n_hit >= 2, (n_cmp, n_hit)
    print(f"fourier-only clears: {total} over 100 frames")


@pytest.mark.parametrize("spec,ebn0", [((8, 64, 16, 27), 4.0), ((7, 40, 10, 29), 3.5)])
def test_decode_parity_high_row_weight(dev, spec, ebn0):
    """Whole decodes of codes whose check node runs the team variant (q >= 128, k > 8: a block's
    warps share one pipeline of whole checks), random codewords, against the oracle's decodes."""
    c = _code(spec)
    _, llr = synth.frames(c, 24, ebn0, batch_idx=13)
    sym, ok, it, n_sym, n_it = _decode_vs_oracle(dev, c, llr, 20, min_frac=0.5, form=nb.FORM_FP32_FWHT)
    assert ok.any() and it.max() <= 20
    print(f"\n{spec}: decoded {ok.mean():.3f}, {n_sym} frames compared, {n_it} iteration counts")


@pytest.mark.parametrize("form", FORMS)
def test_decode_parity_gf4_n8(dev, form):
    c = synth.named_code("gf4_n8_k4")
    _, llr = synth.frames(c, 64, 1.0)
    _decode_vs_oracle(dev, c, llr, 20, min_frac=0.6, form=form)


def test_decode_edge_cases(dev):
    c = synth.named_code("gf16_n32_k4")
    code = nb.Code(c)
    _, llr = synth.frames(c, 33, 1.0)
    x = _t(llr, dev)
    # empty batch
    nb.nbfd_decode(code.handle, 0, x, 10, nb.FORM_FP32_DIRECT, 0, 0, 0)
    # max_iter = 1, ragged batch, library-allocated workspace
    sym = torch.empty((33, 32), dtype=torch.int16, device=dev)
    ok = torch.empty(33, dtype=torch.uint8, device=dev)
    it = torch.empty(33, dtype=torch.int32, device=dev)
    nb.nbfd_decode(code.handle, 33, x, 1, nb.FORM_FP32_DIRECT, sym, ok, it)
    torch.cuda.synchronize()
    assert np.all(it.cpu().numpy() == 1)
    oc = OracleCode.from_dict(c)
    for f in range(33):
        r = LF.decode(oc, llr[f].astype(np.float64), 1)
        if min(r["margins"]) > MARGIN:
            assert np.array_equal(sym.cpu().numpy()[f].astype(np.int64), r["symbols"])
            assert int(ok.cpu().numpy()[f]) == int(r["ok"])
    with pytest.raises(nb.NbfdError) as ei:
        nb.nbfd_decode(code.handle, 33, x, 0, nb.FORM_FP32_DIRECT, sym, ok, it)
    assert ei.value.status == -1
    with pytest.raises(nb.NbfdError) as ei:
        nb.nbfd_decode(code.handle, 33, x, 5, nb.FORM_FP32_DIRECT, sym, ok, it,
                       torch.empty(64, dtype=torch.uint8, device=dev), 64)
    assert ei.value.status == -6
    with pytest.raises(nb.NbfdError) as ei:
        nb.nbfd_decode(code.handle, 33, x, 5, 99, sym, ok, it)
    assert ei.value.status == -10


# 16 frames spread over a batch, first and last included
SPREAD_1024 = [int(x) for x in np.linspace(0, 1023, 16)]
SPREAD_4096 = [int(x) for x in np.linspace(0, 4095, 16)]


@pytest.mark.parametrize("form", FORMS + [nb.FORM_FP32_TC | nb.MMA_SYNC, nb.FORM_FP32_TC | nb.TCGEN05])
def test_decode_full_size_gf256_n512(dev, form):
    """The measured configuration: GF(256) (2,4) N=512, 1024 frames at Eb/N0 = 1.5 dB. With at
    most 10 iterations 16 frames spread over the batch (so over the grid's waves and the
    bulk-copy pipelines' stages) are decoded by the oracle as well, and compared wherever they
    converged with a clear margin; with 100 iterations every frame is checked for properties
    that hold at any size."""
    c = synth.named_code("gf256_n512_k4")
    tx, llr = synth.frames(c, 1024, 1.5)
    _decode_vs_oracle(dev, c, llr, 10, frames=SPREAD_1024, min_frac=0.6, form=form)
    code = nb.Code(c)
    sym, ok, it = nb.decode(code, _t(llr, dev), 100, form)
    # self-consistency on every frame: the library's own syndrome of its output is 0 iff ok
    ex = torch.empty((1024, code.M), dtype=torch.int16, device=dev)
    nb.nbfd_syndrome(code.handle, 1024, sym, None, None, ex)
    torch.cuda.synchronize()
    ok_h = ok.cpu().numpy().astype(bool)
    zero = ~ex.cpu().numpy().any(axis=1)
    assert np.array_equal(ok_h, zero)
    sym_h = sym.cpu().numpy().astype(np.int64)
    # decoded frames carry the transmitted codeword (undetected errors are vanishingly rare)
    assert np.mean(np.all(sym_h[ok_h] == tx[ok_h], axis=1)) > 0.999
    assert ok_h.mean() > 0.5
    it_h = it.cpu().numpy()
    assert it_h.min() >= 1 and it_h.max() <= 100 and np.all(it_h[~ok_h] == 100)


@pytest.mark.parametrize("form", FORMS)
def test_decode_full_size_gf64_n1200(dev, form):
    """The plain batched configuration: GF(64) (2,6) N=1200, 4096 frames per launch, Eb/N0 over
    1.0 .. 3.0 dB (here 2.5 dB, where most frames decode), random codewords. 16 frames spread
    over the batch are decoded by the oracle too (at most 10 iterations); with 100 iterations
    every frame is checked for what holds at any size."""
    c = synth.named_code("gf64_n1200_k6")
    enc = synth.Encoder(c)
    tx, llr = synth.frames(c, 4096, 2.5, snr_idx=3, encoder=enc)
    _decode_vs_oracle(dev, c, llr, 10, frames=SPREAD_4096, min_frac=0.6, form=form)
    code = nb.Code(c)
    sym, ok, it = nb.decode(code, _t(llr, dev), 100, form)
    ex = torch.empty((4096, code.M), dtype=torch.int16, device=dev)
    nb.nbfd_syndrome(code.handle, 4096, sym, None, None, ex)
    torch.cuda.synchronize()
    ok_h = ok.cpu().numpy().astype(bool)
    assert np.array_equal(ok_h, ~ex.cpu().numpy().any(axis=1))
    it_h = it.cpu().numpy()
    assert it_h.min() >= 1 and it_h.max() <= 100 and np.all(it_h[~ok_h] == 100)
    sym_h = sym.cpu().numpy().astype(np.int64)
    assert np.mean(np.all(sym_h[ok_h] == tx[ok_h], axis=1)) > 0.999
    assert ok_h.mean() > 0.9


@pytest.mark.parametrize("form", [nb.FORM_BF16_HGEMM, nb.FORM_FP16_HGEMM])
def test_decode_low_precision_forms_gf256_n512(dev, form):
    """BF16 / FP16 operand forms on the measured configuration. What holds at any precision is
    checked exactly: a frame is flagged decoded iff H x = 0, iterations stay in [1, 100]. Their
    error rates are the precision study's subject (the x-domain check messages come out of signed
    sums of O(1) Fourier coefficients, which 8 or 11 significant bits resolve poorly: at 1.5 dB
    about half of the frames fail with BF16 operands and a few percent with FP16), so here only
    progress is required: a fifth of the frames or more come out as the transmitted codeword
    (the channel's hard decisions alone give none), and wrong codewords stay rare."""
    c = synth.named_code("gf256_n512_k4")
    tx, llr = synth.frames(c, 1024, 1.5)
    code = nb.Code(c)
    x = _t(llr, dev)
    sym, ok, it = nb.decode(code, x, 100, form)
    ex = torch.empty((1024, code.M), dtype=torch.int16, device=dev)
    nb.nbfd_syndrome(code.handle, 1024, sym, None, None, ex)
    torch.cuda.synchronize()
    ok_h = ok.cpu().numpy().astype(bool)
    assert np.array_equal(ok_h, ~ex.cpu().numpy().any(axis=1))
    it_h = it.cpu().numpy()
    assert it_h.min() >= 1 and it_h.max() <= 100
    sym_h = sym.cpu().numpy().astype(np.int64)
    correct = np.all(sym_h == tx, axis=1)
    print(f"form {form}: flagged {ok_h.mean():.4f}, correct {correct.mean():.4f}, "
          f"undetected {np.mean(ok_h & ~correct):.4f}")
    assert correct.mean() > 0.2
    assert np.mean(ok_h & ~correct) < 0.02


def test_tc_forms_need_m8(dev):
    c = synth.named_code("gf16_n32_k4")
    code = nb.Code(c)
    _, llr = synth.frames(c, 4, 2.0)
    for form in TC_FORMS + [f | nb.TCGEN05 for f in TC_FORMS] + [nb.FORM_FP32_FWHT | nb.TCGEN05,
                                                                nb.FORM_FP32_FWHT | nb.MMA_SYNC]:
        with pytest.raises(nb.NbfdError) as ei:
            nb.decode(code, _t(llr, dev), 5, form)
        assert ei.value.status == -10


@pytest.mark.parametrize("form", [nb.FORM_FP32_FWHT])
def test_decode_parity_symbol_decisions_tiny(dev, form):
    """Symbol-MAP tentative decisions (argmax of mu_v) against the oracle's, GF(16) N=32."""
    c = synth.named_code("gf16_n32_k4")
    _, llr = synth.frames(c, 100, 2.0, zero_codeword=True)
    _decode_vs_oracle(dev, c, llr, 50, min_frac=0.6, form=form | nb.DECIDE_SYMBOL, decision="symbol")


@pytest.mark.parametrize("form", [nb.FORM_FP32_FWHT, nb.FORM_FP32_TC])
def test_decode_parity_symbol_decisions_gf256(dev, form):
    c = synth.named_code("gf256_n512_k4")
    tx, llr = synth.frames(c, 256, 1.5)
    _decode_vs_oracle(dev, c, llr, 4, frames=[0, 99], min_frac=0.5, form=form | nb.DECIDE_SYMBOL,
                      decision="symbol")
    code = nb.Code(c)
    sym, ok, it = nb.decode(code, _t(llr, dev), 100, form | nb.DECIDE_SYMBOL)
    ex = torch.empty((256, code.M), dtype=torch.int16, device=dev)
    nb.nbfd_syndrome(code.handle, 256, sym, None, None, ex)
    torch.cuda.synchronize()
    ok_h = ok.cpu().numpy().astype(bool)
    assert np.array_equal(ok_h, ~ex.cpu().numpy().any(axis=1))
    assert np.mean(np.all(sym.cpu().numpy().astype(np.int64)[ok_h] == tx[ok_h], axis=1)) > 0.99
    assert ok_h.mean() > 0.9


def test_symbol_decisions_not_supported_by_direct_form(dev):
    c = synth.named_code("gf16_n32_k4")
    code = nb.Code(c)
    _, llr = synth.frames(c, 2, 2.0)
    with pytest.raises(nb.NbfdError) as ei:
        nb.decode(code, _t(llr, dev), 5, nb.FORM_FP32_DIRECT | nb.DECIDE_SYMBOL)
    assert ei.value.status == -10
