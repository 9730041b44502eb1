"""GPU tests of the serving loop (nbfd_srv_*): continuous batching of single-frame requests of
different codes, admitted while others are in flight, retired on a clear syndrome. Each frame's
result must equal the result of decoding that frame alone with nbfd_decode (the frames never
interact, so equality is exact)."""

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


def _wait_all(srv, tickets, n_of, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            r = nb.nbfd_srv_poll(srv, t, n_of[t])
            if r is not None:
                out[t] = r
        if time.time() - t0 > timeout:
            raise TimeoutError(f"{len(tickets) - len(out)} requests did not retire")
        time.sleep(0.001)
    return out


@pytest.mark.parametrize("form", [nb.FORM_FP32_FWHT, nb.FORM_FP32_DIRECT])
def test_serving_results_equal_decoding_alone(dev, form):
    specs = [("gf256_n512_k4", 24, 1.5, 60), ("gf64_n1200_k6", 12, 2.5, 60), ("gf16_n32_k4", 40, 2.0, 50)]
    codes, frames = {}, []
    for name, n, ebn0, max_iter in specs:
        c = synth.named_code(name)
        code = nb.Code(c)
        codes[name] = code
        _, llr = synth.frames(c, n, ebn0, batch_idx=31)
        frames += [(name, llr[i], max_iter) for i in range(n)]
    rng = np.random.default_rng(5)
    order = rng.permutation(len(frames))
    srv = nb.nbfd_srv_create(8 << 30, form)
    try:
        tickets, info, n_of = [], {}, {}
        # first wave, then the rest while the first is in flight
        for wave in (order[: len(order) // 3], order[len(order) // 3:]):
            for i in wave:
                name, llr, max_iter = frames[i]
                t = nb.nbfd_srv_submit(srv, codes[name].handle, llr, max_iter)
                tickets.append(t)
                info[t] = i
                n_of[t] = codes[name].N
            time.sleep(0.002)
        res = _wait_all(srv, tickets, n_of)
        rounds, queued, in_flight, dev_bytes = nb.nbfd_srv_stats(srv)
        assert rounds > 0 and queued == 0 and in_flight == 0 and dev_bytes > 0
    finally:
        nb.nbfd_srv_destroy(srv)
    lat = []
    for t in tickets:
        name, llr, max_iter = frames[info[t]]
        sym, ok, it, latency = res[t]
        ref_sym, ref_ok, ref_it = nb.decode(codes[name], torch.from_numpy(llr[None]).to(dev), max_iter, form)
        torch.cuda.synchronize()
        assert np.array_equal(sym.astype(np.int64), ref_sym.cpu().numpy()[0].astype(np.int64)), (name, info[t])
        assert ok == int(ref_ok.cpu().numpy()[0]) and it == int(ref_it.cpu().numpy()[0]), (name, info[t])
        lat.append(latency)
    assert min(lat) > 0


def test_serving_refuses_when_no_pool_fits_the_budget(dev):
    code = nb.Code(synth.named_code("gf256_n512_k4"))
    srv = nb.nbfd_srv_create(4096, nb.FORM_FP32_FWHT)
    try:
        with pytest.raises(nb.NbfdError) as ei:
            nb.nbfd_srv_submit(srv, code.handle, np.zeros((512, 8), np.float32), 10)
        assert ei.value.status == -9
    finally:
        nb.nbfd_srv_destroy(srv)


def test_serving_poll_unknown_ticket(dev):
    srv = nb.nbfd_srv_create(1 << 20, nb.FORM_FP32_FWHT)
    try:
        with pytest.raises(nb.NbfdError):
            nb.nbfd_srv_poll(srv, 12345, 8)
    finally:
        nb.nbfd_srv_destroy(srv)


def test_registered_pool_and_chunked_submit_many(dev):
    """A pool created by nbfd_srv_register serves a submit_many of several copy chunks (600
    frames, queued 256 at a time while the worker already runs); every frame equals its decoding
    in one nbfd_decode batch, tickets come back in order, and the worker's phase times add up."""
    c = synth.named_code("gf16_n32_k4")
    code = nb.Code(c)
    _, llr = synth.frames(c, 600, 1.0, batch_idx=41)
    form = nb.FORM_FP32_FWHT
    srv = nb.nbfd_srv_create(1 << 30, form)
    try:
        nb.nbfd_srv_register(srv, code.handle)
        nb.nbfd_srv_register(srv, code.handle)  # a second registration is a no-op
        _, _, _, dev_bytes = nb.nbfd_srv_stats(srv)
        assert dev_bytes > 0
        tickets = nb.nbfd_srv_submit_many(srv, code.handle, llr, 30)
        assert np.array_equal(np.diff(tickets.astype(np.int64)), np.ones(599, np.int64))
        res = _wait_all(srv, tickets.tolist(), {int(t): code.N for t in tickets})
        rounds, queued, in_flight, dev_bytes2 = nb.nbfd_srv_stats(srv)
        assert queued == 0 and in_flight == 0 and dev_bytes2 == dev_bytes and rounds > 0
        times = nb.nbfd_srv_worker_times(srv)
        assert set(times) == {"admission", "issue", "wait", "retire", "idle"}
        assert min(times.values()) >= 0 and times["issue"] > 0 and times["wait"] > 0
    finally:
        nb.nbfd_srv_destroy(srv)
    ref_sym, ref_ok, ref_it = nb.decode(code, torch.from_numpy(llr).to(dev), 30, form)
    torch.cuda.synchronize()
    ref_sym, ref_ok, ref_it = ref_sym.cpu().numpy(), ref_ok.cpu().numpy(), ref_it.cpu().numpy()
    for i, t in enumerate(tickets.tolist()):
        sym, ok, it, _ = res[t]
        assert np.array_equal(sym.astype(np.int64), ref_sym[i].astype(np.int64)), i
        assert ok == int(ref_ok[i]) and it == int(ref_it[i]), i
