"""The seeded input generators: graph structure, encoder and channel statistics."""

import numpy as np
import pytest

from oracle.code import OracleCode
from paper_1008_4370_gb300 import synth


@pytest.mark.parametrize("name", ["gf16_n32_k4", "gf256_n512_k4", "gf64_n1200_k6", "gf4_n8_k4"])
def test_regular_code_structure(name):
    c = synth.named_code(name)
    N, M, k = c["N"], c["M"], c["k"]
    assert M * k == 2 * N == len(c["edge_var"])
    assert np.array_equal(c["edge_check"], np.repeat(np.arange(M), k))
    assert np.all(np.bincount(c["edge_var"], minlength=N) == 2)
    rows = c["edge_var"].reshape(M, k)
    assert all(len(set(r.tolist())) == k for r in rows)  # no double edge
    assert c["edge_h"].min() >= 1 and c["edge_h"].max() < (1 << c["m"])
    c2 = synth.named_code(name)
    assert np.array_equal(c["edge_var"], c2["edge_var"]) and np.array_equal(c["edge_h"], c2["edge_h"])


@pytest.mark.parametrize("name", ["gf16_n32_k4", "gf256_n512_k4", "gf4_n8_k4"])
def test_encoder_outputs_codewords(name):
    c = synth.named_code(name)
    oc = OracleCode.from_dict(c)
    enc = synth.Encoder(c)
    assert enc.rank <= c["M"] and enc.info_symbols >= c["N"] - c["M"]
    x = enc.random_codewords(5, np.random.default_rng(0))
    assert not np.any(oc.syndrome(x))
    assert np.any(x)


def test_tree_code_is_cycle_free():
    c = synth.tree_code(5, 4, 2, seed=1)
    deg = np.bincount(c["edge_var"], minlength=c["N"])
    assert set(deg.tolist()) <= {1, 2}
    # a connected bipartite graph is a tree iff |edges| = |nodes| - 1
    assert len(c["edge_var"]) == c["N"] + c["M"] - 1


def test_channel_llr_statistics():
    rng = np.random.default_rng(0)
    cw = rng.integers(0, 256, size=(400, 64))
    ebn0, R = 1.5, 0.5
    llr = synth.bpsk_awgn_llr(cw, 8, ebn0, R, rng)
    assert llr.dtype == np.float32 and llr.shape == (400, 64, 8)
    bits = (cw[..., None] >> np.arange(8)) & 1
    sgn = 1 - 2 * bits
    sigma2 = 1 / (2 * R * 10 ** (ebn0 / 10))
    z = llr * sgn  # consistent Gaussian: mean 2/s^2, variance 4/s^2
    assert abs(z.mean() - 2 / sigma2) < 0.05 * (2 / sigma2)
    assert abs(z.var() - 4 / sigma2) < 0.05 * (4 / sigma2)


def test_frames_are_seeded():
    c = synth.named_code("gf16_n32_k4")
    a = synth.frames(c, 3, 2.0, snr_idx=1, batch_idx=2)
    b = synth.frames(c, 3, 2.0, snr_idx=1, batch_idx=2)
    d = synth.frames(c, 3, 2.0, snr_idx=1, batch_idx=3)
    assert np.array_equal(a[1], b[1]) and not np.array_equal(a[1], d[1])


def test_every_gpu_test_code_can_be_built():
    """The GPU tests build these codes; construct them here so input problems show up on CPU."""
    specs = [(2, 8, 4, 7), (3, 12, 4, 21), (4, 32, 4, 1), (5, 20, 4, 22), (6, 24, 6, 23), (6, 30, 6, 28),
             (7, 16, 4, 24),
             (8, 16, 4, 25), (4, 80, 20, 26), (8, 64, 16, 27)]
    for m, N, k, seed in specs:
        c = synth.regular_code(N, k, m, seed=seed)
        oc = OracleCode.from_dict(c)
        assert oc.E == 2 * N
    for name in synth.CODES:
        if name != "gf64_n4096_k8":
            synth.named_code(name)
