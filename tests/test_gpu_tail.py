"""GPU tests of the tail kernel (k_tail_x2): once the GF(256) frames still active fit the
thread-block clusters that can be resident at once, nbfd_decode runs all their remaining
iterations in one launch, one cluster per frame.

The tail kernel calls the per-lane check arithmetic and the per-unit variable-node arithmetic of
the iteration kernels, so its results must equal, bit for bit, those of a path that never uses
it: nbfd_decode_batch (the graph-replayed loop of per-iteration kernels). A batch small enough
to run wholly inside the tail kernel is compared with the oracle as well."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1008_4370_gb300 as nb  # noqa: E402
from oracle import logfourier as LF  # noqa: E402
from oracle.code import OracleCode  # noqa: E402
from paper_1008_4370_gb300 import build as nbuild  # noqa: E402
from paper_1008_4370_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

MARGIN = 1e-3


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    nbuild.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("decide", [0, nb.DECIDE_SYMBOL])
@pytest.mark.parametrize("frames,ebn0", [(96, 1.0), (5, 0.5)])
def test_tail_equals_iteration_kernels(dev, decide, frames, ebn0):
    """96 frames at 1.0 dB: the per-iteration kernels run until 7 or fewer frames are left, the
    tail kernel finishes them (some converge late, some run to max_iter); 5 frames at 0.5 dB:
    the tail kernel runs the whole decode. Symbols, flags and iteration counts must equal those
    of the batch path, which has no tail kernel."""
    c = synth.named_code("gf256_n512_k4")
    code = nb.Code(c)
    _, llr = synth.frames(c, frames, ebn0, batch_idx=71)
    x = torch.from_numpy(np.ascontiguousarray(llr, np.float32)).to(dev)
    form = nb.FORM_FP32_FWHT | decide
    sym0, ok0, it0 = nb.decode(code, x, 60, form)
    torch.cuda.synchronize()
    [(sym1, ok1, it1)] = nb.decode_batch([code], [x], 60, form)
    torch.cuda.synchronize()
    it0_h = it0.cpu().numpy()
    assert np.array_equal(sym0.cpu().numpy(), sym1.cpu().numpy())
    assert np.array_equal(ok0.cpu().numpy(), ok1.cpu().numpy())
    assert np.array_equal(it0_h, it1.cpu().numpy())
    # the workload reaches the tail: frames that need many iterations (and, of 96, frames that
    # stop before max_iter)
    assert it0_h.max() >= 20
    if frames > 7:
        assert (it0_h < 60).any()


def test_tail_only_decode_vs_oracle(dev):
    """Three frames: the tail kernel runs every iteration; compared with the FP64 oracle at 4
    iterations (bit-exact symbols and flags where the oracle's margins are clear)."""
    c = synth.named_code("gf256_n512_k4")
    oc = OracleCode.from_dict(c)
    code = nb.Code(c)
    _, llr = synth.frames(c, 3, 1.5, batch_idx=72)
    x = torch.from_numpy(np.ascontiguousarray(llr, np.float32)).to(dev)
    sym, ok, it = nb.decode(code, x, 4, nb.FORM_FP32_FWHT)
    torch.cuda.synchronize()
    sym, ok, it = sym.cpu().numpy().astype(np.int64), ok.cpu().numpy(), it.cpu().numpy()
    n_cmp = 0
    for f in range(3):
        r = LF.decode(oc, llr[f].astype(np.float64), 4)
        if r["margins"][-1] > MARGIN:
            n_cmp += 1
            assert np.array_equal(sym[f], r["symbols"]), f
            assert int(ok[f]) == int(r["ok"]), f
        if min(r["margins"]) > MARGIN:
            assert int(it[f]) == r["iters"], f
    assert n_cmp >= 2


def test_tail_kernel_timer(dev):
    """The kernel timers attribute the tail launch to NBFD_KERNEL_TAIL, with its frames."""
    c = synth.named_code("gf256_n512_k4")
    code = nb.Code(c)
    _, llr = synth.frames(c, 4, 0.5, batch_idx=73)
    x = torch.from_numpy(np.ascontiguousarray(llr, np.float32)).to(dev)
    nb.nbfd_prof_enable(1 << nb.KERNEL_TAIL)
    try:
        nb.decode(code, x, 30, nb.FORM_FP32_FWHT)
        torch.cuda.synchronize()
        ms, launches, units = nb.nbfd_prof_get(nb.KERNEL_TAIL)
    finally:
        nb.nbfd_prof_enable(0)
    assert launches == 1 and units == 4 and ms > 0
