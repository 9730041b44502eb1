"""Mean decoding iterations of the FP64 oracle on the measured workload (test infrastructure).

Writes oracle/workload_iterations.json, which bench.py's CPU legs use to turn the oracle's
frame-iterations per second into decoded Mbit/s. Calls nothing but oracle/ and the seeded
input generators.

    python -m oracle.measure_iterations [--frames 32] [--procs 8]
"""

from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CODE = "gf256_n512_k4"
EBN0 = 1.5
MAX_ITER = 100
BATCH = 900  # batch index of the sample (distinct from the benchmark's GPU batches)


def _one(args):
    f, llr = args
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    import numpy as np

    from oracle import logfourier as LF
    from oracle.code import OracleCode
    from paper_1008_4370_gb300 import synth

    oc = OracleCode.from_dict(synth.named_code(CODE))
    t0 = time.perf_counter()
    r = LF.decode(oc, llr.astype(np.float64), MAX_ITER)
    return f, r["iters"], bool(r["ok"]), time.perf_counter() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--frames", type=int, default=32)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    from paper_1008_4370_gb300 import synth

    code = synth.named_code(CODE)
    _, llr = synth.frames(code, a.frames, EBN0, snr_idx=0, batch_idx=BATCH)
    with mp.get_context("spawn").Pool(a.procs) as pool:
        res = pool.map(_one, [(f, llr[f]) for f in range(a.frames)])
    iters = [r[1] for r in res]
    out = {
        "workload": f"{CODE}, Eb/N0 {EBN0} dB, max {MAX_ITER} iterations, batch index {BATCH}",
        "frames": a.frames,
        "mean_iterations": sum(iters) / len(iters),
        "iterations": iters,
        "decoded": sum(r[2] for r in res),
        "seconds_per_frame_iteration": sum(r[3] for r in res) / sum(iters),
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
