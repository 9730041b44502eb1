"""The expiry path of the kernels' bounded waits, on a GPU without a fault: a wait for bulk-copy
bytes that nobody sends runs out after a short budget, the status reaches the host as
NBFD_ETIMEDOUT, and the context stays usable (a decode right after gives the same result as
before)."""

import time

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


def test_bounded_wait_expires_and_context_survives(dev):
    c = synth.named_code("gf16_n32_k4")
    code = nb.Code(c)
    _, llr = synth.frames(c, 16, 2.0)
    x = torch.from_numpy(llr).to(dev)
    before = [t.cpu().numpy() for t in nb.decode(code, x, 20, nb.FORM_FP32_FWHT)]
    t0 = time.time()
    with pytest.raises(nb.NbfdError) as ei:
        nb.nbfd_diag_wait_expiry(2_000_000)  # about 1 ms of SM cycles
    assert ei.value.status == -8
    assert time.time() - t0 < 30.0
    with pytest.raises(nb.NbfdError) as ei:
        nb.nbfd_diag_wait_expiry(-1)
    assert ei.value.status == -1
    after = [t.cpu().numpy() for t in nb.decode(code, x, 20, nb.FORM_FP32_FWHT)]
    for a, b in zip(before, after):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("form", [nb.FORM_FP32_DIRECT, nb.FORM_FP32_FWHT])
def test_decode_reports_its_status_word(dev, form):
    """nbfd_decode returns NBFD_ETIMEDOUT when its status word comes back nonzero, on the
    iteration path and on the tail-kernel path. The word is preset on the host
    (nbfd_diag_preset_status), so no kernel waits in vain and nothing faults; the preset is
    one-shot, so the next decode is clean."""
    for name, F in (("gf16_n32_k4", 20), ("gf256_n512_k4", 4)):
        c = synth.named_code(name)
        code = nb.Code(c)
        _, llr = synth.frames(c, F, 2.0)
        x = torch.from_numpy(llr).to(dev)
        nb.nbfd_diag_preset_status(-8)
        with pytest.raises(nb.NbfdError) as ei:
            nb.decode(code, x, 30, form)
        assert ei.value.status == -8 and "bounded" in str(ei.value)
        sym, ok, it = nb.decode(code, x, 30, form)
        torch.cuda.synchronize()
        assert it.cpu().numpy().min() >= 1
