"""GPU test of nbfd_decode_noalloc, the entry point for callers that must not allocate device
memory while they decode (their memory is reserved by another runtime, or allocation is banned
in their real-time loop). It must give exactly what nbfd_decode gives -- the outputs are integers
(symbols, syndrome flags, iteration counts), so the tolerance is equality -- on consecutive calls
that share its fixed scratch array, and it must refuse a batch that does not fit.

Named so that pytest collects it after every other test file."""

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


def _outputs(F, N, dev):
    # filled with junk so that a field the call forgets to write shows up
    return (torch.full((F, N), 0x5A5A, dtype=torch.int16, device=dev),
            torch.full((F,), 7, dtype=torch.uint8, device=dev),
            torch.full((F,), -3, dtype=torch.int32, device=dev))


def _check_against_decode(code, llr, max_iter, dev, form=nb.FORM_FP32_DIRECT):
    F = llr.shape[0]
    x = torch.from_numpy(llr).to(dev)
    ref_sym, ref_ok, ref_it = nb.decode(code, x, max_iter, form)
    sym, ok, it = _outputs(F, code.N, dev)
    nb.nbfd_decode_noalloc(code.handle, F, x, max_iter, form, sym, ok, it)
    torch.cuda.synchronize()
    assert torch.equal(sym, ref_sym)
    assert torch.equal(ok, ref_ok)
    assert torch.equal(it, ref_it)
    return ok.cpu().numpy(), it.cpu().numpy()


@pytest.mark.parametrize("form", [nb.FORM_FP32_DIRECT, nb.FORM_FP32_FWHT])
def test_noalloc_matches_decode_on_consecutive_calls(dev, form):
    """With the FWHT form both entry points finish the last GF(256) frames in the tail kernel."""
    c = synth.named_code("gf256_n512_k4")
    code = nb.Code(c)
    enc = synth.Encoder(c)
    # first call: 24 frames (50 MiB of scratch); second call: fewer frames at another SNR, so it
    # runs on whatever the first call left in the shared array
    _, llr1 = synth.frames(c, 24, 1.5, batch_idx=51, encoder=enc)
    ok1, it1 = _check_against_decode(code, llr1, 60, dev, form)
    _, llr2 = synth.frames(c, 7, 0.75, batch_idx=52, encoder=enc)
    ok2, it2 = _check_against_decode(code, llr2, 60, dev, form)
    assert it1.min() >= 1 and it2.min() >= 1
    # and a different code and field through the same array
    t = synth.named_code("gf16_n32_k4")
    _, llr3 = synth.frames(t, 100, 2.0, zero_codeword=True)
    _check_against_decode(nb.Code(t), llr3, 50, dev, form)


def test_noalloc_rejects_a_batch_larger_than_its_scratch(dev):
    c = synth.named_code("gf256_n512_k4")
    code = nb.Code(c)
    F = 64
    need = nb.nbfd_decode_workspace_size(code.handle, F, 100, nb.FORM_FP32_DIRECT)
    assert need > nb.NOALLOC_SCRATCH_BYTES
    _, llr = synth.frames(c, F, 1.5)
    sym, ok, it = _outputs(F, code.N, dev)
    with pytest.raises(nb.NbfdError) as ei:
        nb.nbfd_decode_noalloc(code.handle, F, torch.from_numpy(llr).to(dev), 100, nb.FORM_FP32_DIRECT,
                               sym, ok, it)
    assert ei.value.status == -6 and "scratch" in str(ei.value)
