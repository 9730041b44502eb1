"""The fused small-code kernel (whole GF(16) decodes in one launch, each frame's messages in
shared memory) against the per-iteration kernels (NBFD_UNFUSED): the same Section 3.2 arithmetic
in the same order, so symbols, syndrome flags, iteration counts and the Fourier-only clear count
must be bit-identical, for bitwise and symbol decisions, at every row weight the kernel is
instantiated for, at the configured batch size and at the edges (one frame, max_iter = 1). The
oracle comparison of GF(16) decodes lives in test_gpu_parity.py (its FWHT cases now take this
path)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1008_4370_gb300 as nb  # noqa: E402
from paper_1008_4370_gb300 import build as nbuild  # noqa: E402
from paper_1008_4370_gb300 import synth  # noqa: E402

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
    return c


def _both(code, x, max_iter, form):
    out = []
    for f in (form, form | nb.UNFUSED):
        sym, ok, it = nb.decode(code, x, max_iter, f)
        torch.cuda.synchronize()
        out.append((sym.cpu().numpy(), ok.cpu().numpy(), it.cpu().numpy(), nb.nbfd_last_decode_stats()))
    return out


CASES = [("gf16_n96_k4", 8192, 100), ("gf16_n32_k4", 777, 50), ((4, 48, 8, 31), 300, 60),
         ((4, 80, 20, 26), 200, 60), ((4, 40, 2, 32), 123, 40)]


@pytest.mark.parametrize("spec,F,max_iter", CASES)
@pytest.mark.parametrize("decision", [0, nb.DECIDE_SYMBOL])
def test_fused_equals_per_iteration_kernels(dev, spec, F, max_iter, decision):
    c = _code(spec)
    code = nb.Code(c)
    enc = synth.Encoder(c)
    rng = synth.rng_for(5, F)
    _, llr = synth.frames(c, F, rng.uniform(1.0, 3.5, size=F), batch_idx=7, encoder=enc)
    (s1, o1, i1, q1), (s2, o2, i2, q2) = _both(code, torch.from_numpy(llr).to(dev), max_iter,
                                               nb.FORM_FP32_FWHT | decision)
    assert np.array_equal(s1, s2) and np.array_equal(o1, o2) and np.array_equal(i1, i2)
    assert q1 == q2
    assert i1.min() >= 1 and i1.max() <= max_iter and o1.any()
    print(f"\n{c.get('name', spec)} F={F}: decoded {o1.mean():.4f}, mean iterations {i1.mean():.2f}, "
          f"Fourier-only clears {q1}")


def test_fused_edges(dev):
    c = synth.named_code("gf16_n96_k4")
    code = nb.Code(c)
    _, llr = synth.frames(c, 5, 1.0, batch_idx=9)
    x = torch.from_numpy(llr).to(dev)
    for F, max_iter in ((1, 20), (5, 1), (5, 2)):
        (s1, o1, i1, q1), (s2, o2, i2, q2) = _both(code, x[:F], max_iter, nb.FORM_FP32_FWHT)
        assert np.array_equal(s1, s2) and np.array_equal(o1, o2) and np.array_equal(i1, i2) and q1 == q2
        assert i1.max() <= max_iter


def test_fused_kernel_is_timed_and_used(dev):
    """The fused launch shows up under its own timer, once per decode, covering every frame; with
    NBFD_UNFUSED the per-iteration kernels run instead."""
    c = synth.named_code("gf16_n96_k4")
    code = nb.Code(c)
    _, llr = synth.frames(c, 1000, 2.0, batch_idx=3)
    x = torch.from_numpy(llr).to(dev)
    nb.nbfd_prof_enable(0x3F)
    nb.decode(code, x, 100, nb.FORM_FP32_FWHT)
    torch.cuda.synchronize()
    ms, launches, units = nb.nbfd_prof_get(nb.KERNEL_FUSED)
    assert launches == 1 and units == 1000 and ms > 0
    assert nb.nbfd_prof_get(nb.KERNEL_CHECK)[1] == 0
    nb.nbfd_prof_enable(0x3F)
    nb.decode(code, x, 100, nb.FORM_FP32_FWHT | nb.UNFUSED)
    torch.cuda.synchronize()
    assert nb.nbfd_prof_get(nb.KERNEL_FUSED)[1] == 0 and nb.nbfd_prof_get(nb.KERNEL_CHECK)[1] > 0
    nb.nbfd_prof_enable(0)


def test_batch_with_a_fused_group_equals_the_graph_path(dev):
    """nbfd_decode_batch runs a GF(16) group as one fused launch beside the graph replays of the
    other groups; with NBFD_UNFUSED that group joins the graph. Both give the same bits."""
    groups = [("gf16_n96_k4", 2048), ("gf64_n1200_k6", 256), ("gf16_n32_k4", 300)]
    codes, xs = [], []
    for gi, (name, F) in enumerate(groups):
        c = synth.named_code(name)
        rng = synth.rng_for(11, gi)
        _, llr = synth.frames(c, F, rng.uniform(1.0, 3.5, size=F), batch_idx=gi, encoder=synth.Encoder(c))
        codes.append(nb.Code(c))
        xs.append(torch.from_numpy(llr).to(dev))
    a = nb.decode_batch(codes, xs, 100, nb.FORM_FP32_FWHT)
    b = nb.decode_batch(codes, xs, 100, nb.FORM_FP32_FWHT | nb.UNFUSED)
    torch.cuda.synchronize()
    for (s1, o1, i1), (s2, o2, i2) in zip(a, b):
        assert torch.equal(s1, s2) and torch.equal(o1, o2) and torch.equal(i1, i2)
