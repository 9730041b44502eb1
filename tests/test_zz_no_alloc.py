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
    torch.cuda.synchronize()
    ref_stats = nb.nbfd_last_decode_stats()
    sym, ok, it = _outputs(F, code.N, dev)
    nb.nbfd_decode_noalloc(code.handle, F, x, max_iter, form, sym, ok, it)
    torch.cuda.synchronize()
    assert torch.equal(sym, ref_sym)
    assert torch.equal(ok, ref_ok)
    assert torch.equal(it, ref_it)
    assert nb.nbfd_last_decode_stats() == ref_stats
    return ok.cpu().numpy(), it.cpu().numpy()


def _largest_batch(code, max_iter, form):
    """The most frames whose scratch fits the fixed array (its layout is nbfd_decode's)."""
    F = 1
    while nb.nbfd_decode_workspace_size(code.handle, F + 1, max_iter, form) <= nb.NOALLOC_SCRATCH_BYTES:
        F += 1
    return F


NOALLOC_FORMS = [nb.FORM_FP32_DIRECT, nb.FORM_FP32_FWHT, nb.FORM_FP32_FWHT | nb.STORE_F16,
                 nb.FORM_FP32_FWHT | nb.DECIDE_SYMBOL]


@pytest.mark.parametrize("form", NOALLOC_FORMS)
def test_noalloc_matches_decode_on_consecutive_calls(dev, form):
    """With the FWHT form both entry points finish the last GF(256) frames in the tail kernel;
    with half storage the messages take 2 bytes per entry, so the same array holds twice the
    frames. The first call fills the array to within one frame of its size."""
    c = synth.named_code("gf256_n512_k4")
    code = nb.Code(c)
    enc = synth.Encoder(c)
    F1 = _largest_batch(code, 60, form)
    need = nb.nbfd_decode_workspace_size(code.handle, F1, 60, form)
    one = need - nb.nbfd_decode_workspace_size(code.handle, F1 - 1, 60, form)
    assert nb.NOALLOC_SCRATCH_BYTES - one < need <= nb.NOALLOC_SCRATCH_BYTES
    # first call: as many frames as fit; second call: fewer frames at another SNR, so it runs on
    # whatever the first call left in the shared array
    _, llr1 = synth.frames(c, F1, 1.5, batch_idx=51, encoder=enc)
    ok1, it1 = _check_against_decode(code, llr1, 60, dev, form)
    _, llr2 = synth.frames(c, 7, 0.75, batch_idx=52, encoder=enc)
    ok2, it2 = _check_against_decode(code, llr2, 60, dev, form)
    assert it1.min() >= 1 and it2.min() >= 1 and ok1.mean() > 0.5
    if form & nb.STORE_F16:
        return  # half storage is a GF(256) form
    # and a different code and field through the same array
    t = synth.named_code("gf16_n32_k4")
    _, llr3 = synth.frames(t, 100, 2.0, zero_codeword=True)
    _check_against_decode(nb.Code(t), llr3, 50, dev, form)


@pytest.mark.parametrize("form", [nb.FORM_FP32_DIRECT, nb.FORM_FP32_FWHT])
def test_noalloc_reports_its_status_word(dev, form):
    """A status word that comes back nonzero (what a kernel whose bounded wait expired leaves)
    is returned as NBFD_ETIMEDOUT, on the iteration path (GF(16)) and on the tail-kernel path
    (GF(256), FWHT). The word is preset on the host, so nothing faults; the call after it is
    clean again."""
    for name, F in (("gf16_n32_k4", 20), ("gf256_n512_k4", 4)):
        c = synth.named_code(name)
        code = nb.Code(c)
        _, llr = synth.frames(c, F, 2.0)
        x = torch.from_numpy(llr).to(dev)
        sym, ok, it = _outputs(F, code.N, dev)
        nb.nbfd_diag_preset_status(-8)
        with pytest.raises(nb.NbfdError) as ei:
            nb.nbfd_decode_noalloc(code.handle, F, x, 30, form, sym, ok, it)
        assert ei.value.status == -8 and "bounded" in str(ei.value)
        nb.nbfd_decode_noalloc(code.handle, F, x, 30, form, sym, ok, it)
        torch.cuda.synchronize()
        assert it.cpu().numpy().min() >= 1


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
