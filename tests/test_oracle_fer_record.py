"""Pins of the stored FP64 frame-error record (oracle/fer_fp64.json) that the GPU FER test reads.

* The tiny configuration's record (GF(16) (2,4) N=32, all-zero codeword, 2.0 dB, 100 frames, max
  50 iterations) is decoded again here with the oracle: every frame's outcome and iteration count
  must be the stored one, so the record is the oracle's own output and not an edited file.
* Every record matches its configuration (frame count, iterations, code, Eb/N0) and its interval
  is the exact binomial (Clopper-Pearson) interval of its error count.
* The interval helpers (the oracle's and bench.py's, both through the beta quantile) are checked
  against the interval's definition evaluated with exact binomial sums: at the lower bound the
  probability of k or more errors is alpha/2, at the upper bound that of k or fewer is alpha/2;
  and against the closed forms at k = 0 and k = n.
"""

import json
import math

import numpy as np
import pytest

pytest.importorskip("scipy")

from oracle import fer_study  # noqa: E402
from oracle import logfourier as LF  # noqa: E402
from oracle.code import OracleCode  # noqa: E402


@pytest.fixture(scope="module")
def record():
    with open(fer_study.OUT) as f:
        return json.load(f)


def test_tiny_record_is_reproduced_by_the_oracle(record):
    name = "gf16_n32_2.0dB"
    rec = record[name]
    c, tx, llr, max_iter = fer_study.make_frames(name)
    oc = OracleCode.from_dict(c)
    failed, iters, flagged = [], [], []
    for f in range(llr.shape[0]):
        r = LF.decode(oc, llr[f].astype(np.float64), max_iter)
        if not np.array_equal(np.asarray(r["symbols"], dtype=np.int64), tx[f].astype(np.int64)):
            failed.append(f)
        iters.append(int(r["iters"]))
        flagged.append(int(r["ok"]))
    assert failed == rec["failed_frames"]
    assert iters == rec["iterations"]
    assert flagged == rec["flagged_ok"]


def test_every_record_matches_its_configuration(record):
    assert set(fer_study.CONFIGS) <= set(record)
    for name, (code, F, ebn0, snr_idx, batch_idx, zero, max_iter) in fer_study.CONFIGS.items():
        rec = record[name]
        assert (rec["code"], rec["frames"], rec["ebn0_db"], rec["max_iter"]) == (code, F, ebn0, max_iter)
        assert (rec["snr_idx"], rec["batch_idx"], rec["zero_codeword"]) == (snr_idx, batch_idx, zero)
        k = len(rec["failed_frames"])
        assert rec["frame_errors"] == k and rec["fer"] == k / F
        assert len(rec["iterations"]) == F and max(rec["iterations"]) <= max_iter
        lo, hi = fer_study.clopper_pearson(k, F)
        assert rec["ci95"] == pytest.approx([lo, hi], abs=1e-12)


def _tail_ge(k, n, p):
    return sum(math.comb(n, i) * p ** i * (1 - p) ** (n - i) for i in range(k, n + 1))


def _tail_le(k, n, p):
    return sum(math.comb(n, i) * p ** i * (1 - p) ** (n - i) for i in range(0, k + 1))


@pytest.mark.parametrize("k,n", [(0, 100), (9, 100), (8, 512), (1, 20), (20, 20), (3, 256)])
def test_clopper_pearson_matches_its_definition(k, n):
    import bench

    alpha = 0.05
    for lo, hi in (fer_study.clopper_pearson(k, n), tuple(bench.clopper_pearson(k, n))):
        if k == 0:
            assert lo == 0.0 and hi == pytest.approx(1 - (alpha / 2) ** (1 / n), rel=1e-9)
        else:
            assert _tail_ge(k, n, lo) == pytest.approx(alpha / 2, rel=1e-6)
        if k == n:
            assert hi == 1.0 and lo == pytest.approx((alpha / 2) ** (1 / n), rel=1e-9)
        else:
            assert _tail_le(k, n, hi) == pytest.approx(alpha / 2, rel=1e-6)
        assert lo <= k / n <= hi
