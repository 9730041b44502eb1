"""Frame error rate of the FP64 oracle (test infrastructure).

Decodes seeded synthetic frames with the FP64 Log-Fourier SP decoder of Section 3.2
(``logfourier.decode``: literal log-domain boxplus at the variable nodes, bitwise tentative
decisions, stop on a zero Fourier-domain syndrome and a zero GF(2^m) syndrome) and writes, per
configuration, every frame's outcome (decoded to the transmitted codeword, syndrome flag,
iterations) and the FER with its 95% Clopper-Pearson interval to oracle/fer_fp64.json. The GPU
test tests/test_gpu_fer_vs_oracle.py decodes the very same frames (same generator keys and batch
sizes) with each FP32 variable-node form and checks that its FER lies inside this interval: the
paper designs Log-Fourier SP to compute exactly what SP computes (Section 3), so a faithful FP32
implementation must decode at the FP64 decoder's error rate.

Calls nothing but oracle/ and the seeded input generators. Frames run in a ``spawn`` process
pool; each configuration is written as soon as it is done, and configurations already in the
file are skipped unless --redo names them.

    python -m oracle.fer_study [--procs 8] [--only NAME ...] [--redo NAME ...]
"""

from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

# one BLAS thread per process: the pool already runs one process per core (set before numpy is
# imported here or in a spawned child, which inherits the environment)
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fer_fp64.json")

# name -> (code, frames, Eb/N0 dB, snr_idx, batch_idx, all-zero codeword, max iterations)
CONFIGS = {
    # the tiny configuration: GF(16) (2,4) N=32, all-zero codeword, 2.0 dB, 100 frames, max 50
    "gf16_n32_2.0dB": ("gf16_n32_k4", 100, 2.0, 0, 0, True, 50),
    # the precision-study code, GF(256) (2,4) N=512, random codewords, max 100
    "gf256_n512_1.0dB": ("gf256_n512_k4", 512, 1.0, 2, 80, False, 100),
    "gf256_n512_1.5dB": ("gf256_n512_k4", 256, 1.5, 4, 80, False, 100),
    # the plain batched code, GF(64) (2,6) N=1200, random codewords, max 100
    "gf64_n1200_2.0dB": ("gf64_n1200_k6", 512, 2.0, 2, 80, False, 100),
}


def clopper_pearson(k: int, n: int, alpha: float = 0.05):
    """Exact binomial interval for k failures in n trials."""
    from scipy.stats import beta
    lo = 0.0 if k == 0 else float(beta.ppf(alpha / 2, k, n - k + 1))
    hi = 1.0 if k == n else float(beta.ppf(1 - alpha / 2, k + 1, n - k))
    return lo, hi


def make_frames(name: str):
    """(code dict, transmitted symbols [F][N], LLRs [F][N][m] float32, max_iter) of a
    configuration; the GPU test calls this too, so both sides decode the same frames."""
    from paper_1008_4370_gb300 import synth
    code_name, F, ebn0, snr_idx, batch_idx, zero, max_iter = CONFIGS[name]
    c = synth.named_code(code_name)
    enc = None if zero else synth.Encoder(c)
    tx, llr = synth.frames(c, F, ebn0, snr_idx=snr_idx, batch_idx=batch_idx, zero_codeword=zero,
                           encoder=enc)
    return c, tx, llr, max_iter


def _one(args):
    name, f, llr, tx = args
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    import numpy as np

    from oracle import logfourier as LF
    from oracle.code import OracleCode
    from paper_1008_4370_gb300 import synth

    oc = OracleCode.from_dict(synth.named_code(CONFIGS[name][0]))
    t0 = time.perf_counter()
    r = LF.decode(oc, llr.astype(np.float64), CONFIGS[name][6])
    correct = bool(np.array_equal(np.asarray(r["symbols"], dtype=np.int64), tx.astype(np.int64)))
    return f, bool(r["ok"]), correct, int(r["iters"]), time.perf_counter() - t0


def run(name: str, procs: int) -> dict:
    c, tx, llr, max_iter = make_frames(name)
    F = llr.shape[0]
    t0 = time.time()
    res = []
    with mp.get_context("spawn").Pool(procs) as pool:
        for r in pool.imap_unordered(_one, [(name, f, llr[f], tx[f]) for f in range(F)], chunksize=1):
            res.append(r)
            if len(res) % 32 == 0:
                print(f"  {name}: {len(res)}/{F} frames, {time.time() - t0:.0f} s", flush=True)
    res.sort()
    failed = [r[0] for r in res if not r[2]]
    lo, hi = clopper_pearson(len(failed), F)
    code_name, _, ebn0, snr_idx, batch_idx, zero, _ = CONFIGS[name]
    return {
        "code": code_name, "ebn0_db": ebn0, "snr_idx": snr_idx, "batch_idx": batch_idx,
        "zero_codeword": zero, "frames": F, "max_iter": max_iter, "decision": "bitwise",
        "frame_errors": len(failed), "fer": len(failed) / F, "ci95": [lo, hi],
        "failed_frames": failed,
        "flagged_ok": [int(r[1]) for r in res],
        "iterations": [r[3] for r in res],
        "mean_iterations": sum(r[3] for r in res) / F,
        "cpu_seconds": sum(r[4] for r in res), "wall_seconds": time.time() - t0, "procs": procs,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--redo", nargs="*", default=[])
    a = ap.parse_args()
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in CONFIGS:
        if a.only is not None and name not in a.only:
            continue
        if name in data and name not in a.redo:
            continue
        data[name] = run(name, a.procs)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1)
        d = data[name]
        print(f"{name}: FER {d['fer']:.4f} [{d['ci95'][0]:.4f}, {d['ci95'][1]:.4f}] over {d['frames']} frames, "
              f"mean iterations {d['mean_iterations']:.2f}, {d['wall_seconds']:.0f} s", flush=True)


if __name__ == "__main__":
    main()
