"""GPU tests of nbfd_decode_batch (several codes of uneven N, k and q in one call, the iteration
loop replayed from a CUDA graph) and of the launch-shape autotuner.

Frames never interact and every kernel computes a frame the same way whatever the launch shape,
so each group's result must equal nbfd_decode of that group alone, bit for bit; nbfd_decode is
itself compared with the oracle in test_gpu_parity.py, and two small groups are compared with the
oracle here as well."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1008_4370_gb300 as nb  # noqa: E402
from oracle import logfourier as LF  # noqa: E402
from oracle.code import OracleCode  # noqa: E402
from paper_1008_4370_gb300 import build as nbuild  # noqa: E402
from paper_1008_4370_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

# the uneven-batch configuration: codes and frame counts
UNEVEN = [("gf16_n96_k4", 8192), ("gf64_n1200_k6", 2048), ("gf64_n4096_k8", 512),
          ("gf256_n512_k4", 1024), ("gf256_n2048_k16", 256)]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    nbuild.build()
    return torch.device("cuda:0")


def _groups(spec, batch_idx, lo=1.0, hi=3.5):
    """Per-frame Eb/N0 uniform in [lo, hi] (seeded), random codewords."""
    out = []
    for gi, (name, F) in enumerate(spec):
        c = synth.named_code(name)
        rng = synth.rng_for(97, gi, batch_idx)
        ebn0 = rng.uniform(lo, hi, size=F)
        tx, llr = synth.frames(c, F, ebn0, snr_idx=gi, batch_idx=batch_idx)
        out.append((c, tx, llr))
    return out


def _alone(code, llr, max_iter, form):
    sym, ok, it = nb.decode(code, llr, max_iter, form)
    torch.cuda.synchronize()
    return sym.cpu().numpy(), ok.cpu().numpy(), it.cpu().numpy()


def _check_equal_alone(groups, codes, xs, outs, max_iter, form):
    for (c, tx, _), code, x, (sym, ok, it) in zip(groups, codes, xs, outs):
        s1, o1, i1 = sym.cpu().numpy(), ok.cpu().numpy(), it.cpu().numpy()
        s0, o0, i0 = _alone(code, x, max_iter, form)
        assert np.array_equal(s1, s0), c["name"] if "name" in c else c["N"]
        assert np.array_equal(o1, o0) and np.array_equal(i1, i0)


@pytest.mark.parametrize("form", [nb.FORM_FP32_FWHT, nb.FORM_FP32_DIRECT])
def test_batch_equals_alone_small(dev, form):
    spec = [("gf16_n96_k4", 64), ("gf64_n1200_k6", 12), ("gf256_n512_k4", 10), ("gf16_n32_k4", 0),
            ("gf256_n2048_k16", 3)]
    groups = _groups(spec, batch_idx=5)
    codes = [nb.Code(c) for c, _, _ in groups]
    xs = [torch.from_numpy(llr).to(dev) for _, _, llr in groups]
    outs = nb.decode_batch(codes, xs, 60, form)
    torch.cuda.synchronize()
    _check_equal_alone(groups, codes, xs, outs, 60, form)


def test_batch_vs_oracle_small_codes(dev):
    """Two groups through the batch path against the oracle's whole decode (3 iterations)."""
    groups = _groups([("gf16_n96_k4", 3), ("gf64_n1200_k6", 1)], batch_idx=6, lo=2.0, hi=3.0)
    codes = [nb.Code(c) for c, _, _ in groups]
    xs = [torch.from_numpy(llr).to(dev) for _, _, llr in groups]
    outs = nb.decode_batch(codes, xs, 3, nb.FORM_FP32_FWHT)
    torch.cuda.synchronize()
    for (c, _, llr), (sym, ok, it) in zip(groups, outs):
        oc = OracleCode.from_dict(c)
        for f in range(llr.shape[0]):
            r = LF.decode(oc, llr[f].astype(np.float64), 3)
            if min(r["margins"]) > 1e-3:
                assert np.array_equal(sym.cpu().numpy()[f].astype(np.int64), r["symbols"])
                assert int(ok.cpu().numpy()[f]) == int(r["ok"]) and int(it.cpu().numpy()[f]) == r["iters"]


def test_uneven_batch_full_config_with_autotune(dev):
    """The configured uneven batch (8192 / 2048 / 512 / 1024 / 256 frames of five codes, per-frame
    Eb/N0 uniform in 1.0-3.5 dB, max 100 iterations), autotuned: every group equals its own
    nbfd_decode, flags agree with the library's syndrome of the output, iterations in range."""
    groups = _groups(UNEVEN, batch_idx=7)
    codes = [nb.Code(c) for c, _, _ in groups]
    xs = [torch.from_numpy(llr).to(dev) for _, _, llr in groups]
    outs = nb.decode_batch(codes, xs, 100, nb.FORM_FP32_FWHT, nb.BATCH_AUTOTUNE)
    torch.cuda.synchronize()
    for (c, tx, _), code, (sym, ok, it) in zip(groups, codes, outs):
        F = tx.shape[0]
        if c["m"] == 4:  # the GF(16) group runs as one fused launch: no shapes to tune
            with pytest.raises(nb.NbfdError):
                nb.nbfd_autotune_result(code.handle, F, nb.FORM_FP32_FWHT)
        else:
            shape = nb.nbfd_autotune_result(code.handle, F, nb.FORM_FP32_FWHT)
            # check_warps < 0: the team variant (q >= 128 only)
            assert (1 <= shape[0] <= 8 or (shape[0] == -4 and c["m"] >= 7)) and shape[1] >= 3
            assert shape[2] >= 1 and shape[3] >= 1
        ex = torch.empty((F, code.M), dtype=torch.int16, device=dev)
        nb.nbfd_syndrome(code.handle, F, sym, None, None, ex)
        torch.cuda.synchronize()
        ok_h = ok.cpu().numpy().astype(bool)
        assert np.array_equal(ok_h, ~ex.cpu().numpy().any(axis=1))
        it_h = it.cpu().numpy()
        assert it_h.min() >= 1 and it_h.max() <= 100 and np.all(it_h[~ok_h] == 100)
        correct = np.all(sym.cpu().numpy().astype(np.int64) == tx, axis=1)
        print(f"{c['name']}: {F} frames, decoded {ok_h.mean():.4f}, correct {correct.mean():.4f}, "
              f"mean iterations {it_h.mean():.2f}")
        assert correct.sum() > 0 and np.mean(ok_h & ~correct) < 0.05
    # the tuned shapes are used by nbfd_decode too: each group alone gives the same result
    _check_equal_alone(groups, codes, xs, outs, 100, nb.FORM_FP32_FWHT)


def test_batch_symbol_decisions(dev):
    groups = _groups([("gf16_n96_k4", 32), ("gf256_n512_k4", 8)], batch_idx=8)
    codes = [nb.Code(c) for c, _, _ in groups]
    xs = [torch.from_numpy(llr).to(dev) for _, _, llr in groups]
    form = nb.FORM_FP32_FWHT | nb.DECIDE_SYMBOL
    outs = nb.decode_batch(codes, xs, 50, form)
    torch.cuda.synchronize()
    _check_equal_alone(groups, codes, xs, outs, 50, form)


def test_autotune_keeps_results(dev):
    c = synth.named_code("gf64_n1200_k6")
    code = nb.Code(c)
    _, llr = synth.frames(c, 64, 2.5, batch_idx=9)
    x = torch.from_numpy(llr).to(dev)
    before = _alone(code, x, 40, nb.FORM_FP32_FWHT)
    nb.nbfd_autotune(code.handle, 64, nb.FORM_FP32_FWHT)
    after = _alone(code, x, 40, nb.FORM_FP32_FWHT)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)


def test_batch_errors(dev):
    c16 = nb.Code(synth.named_code("gf16_n32_k4"))
    x = torch.zeros((2, 32, 4), dtype=torch.float32, device=dev)
    with pytest.raises(nb.NbfdError) as ei:  # tensor-core forms need GF(256)
        nb.decode_batch([c16], [x], 5, nb.FORM_FP32_TC)
    assert ei.value.status == -10
    with pytest.raises(nb.NbfdError) as ei:
        nb.nbfd_decode_batch([], [], [], 5, nb.FORM_FP32_FWHT, 0, [], [], [])
    assert ei.value.status == -1
