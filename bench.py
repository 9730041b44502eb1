"""Benchmark: decoded Mbit/s of the Log-Fourier decoder on GF(256) (2,4) N=512.

A step is one nbfd_decode call on a batch of 1024 frames (INITIALIZATION, then up to 100
iterations of check update, variable update, tentative decision and syndrome test, frames
retiring as soon as their syndrome clears). Inputs are seeded synthetic BPSK/AWGN LLRs of random
codewords at Eb/N0 = 1.5 dB (the middle of the 0.5-2.5 dB sweep), resident in HBM before the
timed region. `value` = information bits of all frames (decoded or not) / device time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--form fwht|direct] [--impl reference]

Under torchrun each rank decodes its own batches (frames shard with no data exchange; weak
scaling); the barrier and the max over ranks are the only collectives.
"""

from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1008_4370_gb300 import synth  # noqa: E402

CODE_NAME = "gf256_n512_k4"
FORMS = {"direct": 0, "bf16": 1, "fp16": 2, "fwht": 3, "tc32": 4}

# DRAM bytes per frame of one launch, from one ncu capture of a 256-frame launch with every frame
# active (dram__bytes_read.sum + dram__bytes_write.sum, divided by 256), keyed by (kernel, form,
# code), with the sources the kernel was built from and the first 16 hex digits of the SHA-256 of
# their concatenation at capture time. A changed source voids the figure (reported as null).
# Capture: ncu --set full --clock-control none -k regex:<kernel> -s 2 -c 1 python bench.py
#          --frames 256 --steps 1 --warmup 1 --batches 1 --form fwht --no-cpu-baseline
#          --serve-requests 0 --plain-steps 0 --store16-steps 0 --uneven-steps 0 --gf64-steps 0
#          --fused-steps 0 --table1-reps 0 --serve-mix-loads
MEASURED_TRAFFIC = {
    ("var", "fwht", "gf256_n512_k4"): {
        "bytes_per_frame": (272720384 + 220069888) / 256,
        "sources": ["kernels_var_fwht8x2.cu", "check_math.cuh", "device_common.cuh", "bulk_copy.cuh"],
        "sha256_16": "e2a889c55c3da656"},
    ("check", "fwht", "gf256_n512_k4"): {
        "bytes_per_frame": (268668672 + 215507968) / 256,
        "sources": ["kernels_check.cu", "check_math.cuh", "device_common.cuh", "bulk_copy.cuh"],
        "sha256_16": "2f182015a8af3ca6"},
}


def measured_traffic(kernel, form_name, code_name):
    """Per-frame DRAM bytes of the capture above, or None if absent or its sources changed."""
    import hashlib
    rec = MEASURED_TRAFFIC.get((kernel, form_name, code_name))
    if rec is None:
        return None
    h = hashlib.sha256()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, "paper_1008_4370_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return rec["bytes_per_frame"] if h.hexdigest()[:16] == rec["sha256_16"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=80)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="fwht", choices=sorted(FORMS))
    ap.add_argument("--plain-steps", type=int, default=3, help="steps of the plain FP32 direct form")
    ap.add_argument("--code", default=CODE_NAME,
                    help="named code of the main decode (the measured workload is GF(256) N=512; other codes "
                         "serve kernel captures)")
    ap.add_argument("--frames", type=int, default=1024)
    ap.add_argument("--ebn0", type=float, default=1.5)
    ap.add_argument("--max-iter", type=int, default=100)
    ap.add_argument("--batches", type=int, default=4)
    ap.add_argument("--store16-steps", type=int, default=10,
                    help="steps of the half-precision message storage leg (0: skip)")
    ap.add_argument("--uneven-steps", type=int, default=3,
                    help="steps of the uneven five-code batch leg (0: skip)")
    ap.add_argument("--gf64-steps", type=int, default=2,
                    help="timed steps per point of the GF(64) N=1200 plain batched sweep (0: skip)")
    ap.add_argument("--fused-steps", type=int, default=3,
                    help="timed steps of the fused vs per-iteration GF(16) comparison (0: skip)")
    ap.add_argument("--table1-reps", type=int, default=3,
                    help="timed launches per kernel of the Log-SP vs Log-Fourier comparison (0: skip)")
    ap.add_argument("--table1-frames", type=int, default=1024, help="frames of the Table 1 comparison")
    ap.add_argument("--prof-steps", type=int, default=8,
                    help="leading steps of the timed region with per-launch kernel timers")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=16384, help="requests of the serving leg (0: skip)")
    ap.add_argument("--serve-load", type=float, default=30000.0, help="Poisson offered load, frames/s")
    ap.add_argument("--serve-sweep", action="store_true", help="serving sweep over loads and the code mix")
    ap.add_argument("--serve-sweep-requests", type=int, default=100000, help="requests per load of the sweep")
    ap.add_argument("--serve-mix-loads", type=float, nargs="*", default=[1e4, 1e5],
                    help="offered loads (frames/s) of the five-code serving mix in the default run")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---- CPU oracle timing (the only place besides tests that runs oracle/) ---------------------

def _oracle_worker(args):
    name, llr, n_iter = args
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle import logfourier as LF
    from oracle.code import OracleCode
    oc = OracleCode.from_dict(synth.named_code(name))
    t0 = time.perf_counter()
    lam0, v2c = LF.init(oc, llr.astype(np.float64))
    done = 0
    for _ in range(n_iter):
        c2v = LF.check_update(oc, v2c)
        v2c = LF.var_update(oc, lam0, c2v)
        M = LF.tentative(oc, lam0, c2v)
        x = LF.bit_decisions(oc, M)
        done += 1
        if not LF.fourier_syndrome(oc, M).any() and not oc.syndrome(x).any():
            break
    return time.perf_counter() - t0, done


def oracle_frame_iterations(llr_frames: np.ndarray, n_iter: int, cores: int):
    """Wall time and frame-iterations of the FP64 oracle on `cores` processes."""
    ctx = mp.get_context("spawn")
    env_prev = os.environ.get("OPENBLAS_NUM_THREADS")
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        with ctx.Pool(cores) as pool:
            pool.map(_oracle_worker, [(CODE_NAME, llr_frames[0], 0)] * cores)  # import + setup
            t0 = time.perf_counter()
            res = pool.map(_oracle_worker, [(CODE_NAME, l, n_iter) for l in llr_frames])
            wall = time.perf_counter() - t0
    finally:
        if env_prev is None:
            os.environ.pop("OPENBLAS_NUM_THREADS", None)
        else:
            os.environ["OPENBLAS_NUM_THREADS"] = env_prev
    return wall, sum(r[1] for r in res)


# ---- clocks sampling ------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---- the arms ---------------------------------------------------------------------------------

def aggregate(local_seconds: float, local_frames: int, info_bits: int, dist=None, device=None):
    """Whole-job throughput: frames of all ranks / the slowest rank's time (max over ranks)."""
    import torch

    t = torch.tensor([local_seconds], dtype=torch.float64, device=device)
    n = torch.tensor([float(local_frames)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    t_max, frames = float(t.item()), float(n.item())
    return t_max, frames * info_bits / t_max / 1e6


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(a):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    code = synth.named_code(CODE_NAME)
    enc = synth.Encoder(code)
    info_bits = enc.info_symbols * code["m"]
    cores = os.cpu_count() or 1
    _, llr = synth.frames(code, cores, a.ebn0, snr_idx=0, batch_idx=900)
    it_mean = reference_mean_iterations()
    if it_mean is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle/workload_iterations.json is missing "
                          "(run python -m oracle.measure_iterations)"}), flush=True)
        return
    times = []
    fi = 0
    for s in range(a.warmup + a.steps):
        wall, n = oracle_frame_iterations(llr, 1, cores)
        if s >= a.warmup:
            times.append(wall)
            fi += n
    tot = sum(times)
    value = info_bits * (fi / tot) / it_mean / 1e6
    line = {
        "impl": "reference", "metric": "decoded Mbit/s (GF(256) (2,4) N=512)", "value": value,
        "unit": "Mbit/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": ("GF(256) (2,4) N=512, 1024 frames per step, Eb/N0 1.5 dB, random codewords, "
                                "max 100 iterations, early stop") if a.frames == 1024 else
                   f"{CODE_NAME}, {a.frames} frames per step, Eb/N0 {a.ebn0} dB, random codewords, "
                   f"max {a.max_iter} iterations",
                   "frames_per_step": a.frames, "ebn0_db": a.ebn0, "max_iter": a.max_iter,
                   "form": "FP64 oracle (literal log-domain boxplus)", "info_bits_per_frame": info_bits,
                   "sample_frames_per_step": cores, "parallelism": f"{cores} host processes"},
        "cpu_baseline": {"value": value, "unit": "Mbit/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} frames x 1 iteration per step on {cores} processes; "
                                   f"converted at {it_mean:.2f} mean iterations per frame"},
        "e2e": {"value": value, "unit": "Mbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def reference_mean_iterations():
    p = os.path.join(ROOT, "oracle", "workload_iterations.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["mean_iterations"])
    return None


def clopper_pearson(k: int, n: int, alpha: float = 0.05):
    """Exact 95% interval of a frame error rate (None without scipy)."""
    try:
        from scipy.stats import beta
    except ImportError:
        return None
    lo = 0.0 if k == 0 else float(beta.ppf(alpha / 2, k, n - k + 1))
    hi = 1.0 if k == n else float(beta.ppf(1 - alpha / 2, k + 1, n - k))
    return [lo, hi]


def fp32_peak(nb):
    """Measured FP32 FMA rate (TFLOP/s) with scalar and packed (f32x2) FMA chains."""
    out = {}
    for name, packed in (("scalar", 0), ("packed_f32x2", 1)):
        t, ms = nb.nbfd_diag_fp32_rate(packed, 4, 1 << 20)
        out[name] = {"tflops": t, "ms": ms}
    out["peak_tflops"] = max(v["tflops"] for v in out.values())
    return out


def fused_leg(nb, torch, dev, steps, max_iter, F=8192):
    """The uneven batch's GF(16) (2,4) N=96 group alone (8192 frames, per-frame Eb/N0 uniform in
    1.0-3.5 dB): nbfd_decode with the fused small-code kernel (each frame's messages in shared
    memory for all its iterations) against the per-iteration kernels (NBFD_UNFUSED), device time
    from CUDA events, and the message bytes the per-iteration path streams (36 N q per
    frame-iteration) that the fused launch keeps on chip."""
    c = synth.named_code("gf16_n96_k4")
    enc = synth.Encoder(c)
    code = nb.Code(c)
    rng = synth.rng_for(97, 0, 11)
    _, llr = synth.frames(c, F, rng.uniform(1.0, 3.5, size=F), snr_idx=0, batch_idx=11, encoder=enc)
    x = torch.from_numpy(llr).to(dev)
    bits = enc.info_symbols * c["m"]
    stream = torch.cuda.current_stream()
    out = {"code": "gf16_n96_k4", "frames": F, "max_iter": max_iter}
    for name, form in (("fused", FORMS["fwht"]), ("per_iteration", FORMS["fwht"] | nb.UNFUSED)):
        sym, ok, it = nb.decode(code, x, max_iter, form)  # warm (and the outputs' buffers)
        need = nb.nbfd_decode_workspace_size(code.handle, F, max_iter, form)
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            ev[i][0].record(stream)
            nb.nbfd_decode(code.handle, F, x, max_iter, form, sym.data_ptr(), ok, it, ws, need, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a_.elapsed_time(b_) for a_, b_ in ev) / steps
        out[name] = {"ms_per_step": ms, "mbit_s": bits * F / (ms / 1e3) / 1e6,
                     "mean_iterations": float(it.float().mean()), "decoded_frac": float(ok.float().mean())}
    fi = out["per_iteration"]["mean_iterations"] * F
    out["unfused_message_bytes_per_step"] = fi * 36 * c["N"] * (1 << c["m"])
    out["speedup"] = out["per_iteration"]["ms_per_step"] / out["fused"]["ms_per_step"]
    return out


def table1_leg(nb, torch, dev, reps, F=1024, ebn0=1.5):
    """Table 1 of the paper on the GPU: per-launch device time of the check node and of the
    variable node for conventional Log-SP (Section 2.2: (k-1)-fold log-convolutions at the check,
    additions at the variable) against Log-Fourier SP (Section 3.2: additions at the check,
    2-fold convolutions at the degree-2 variable; FWHT and direct forms), 1024 frames of GF(256)
    (2,4) N=512, first-iteration inputs. CUDA events on the launching stream, mean of reps."""
    c = synth.named_code(CODE_NAME)
    code = nb.Code(c)
    N, E, q, m, k = c["N"], 2 * c["N"], 1 << c["m"], c["m"], c["k"]
    M = E // k
    _, llr = synth.frames(c, F, ebn0, snr_idx=0, batch_idx=31)
    x = torch.from_numpy(llr).to(dev)
    a = torch.empty((F, E, q), dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    sym = torch.empty((F, N), dtype=torch.int16, device=dev)
    fsyn = torch.empty((F, E), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for i in range(reps):
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(s_.elapsed_time(e_) for s_, e_ in ev) / reps

    out = {"code": CODE_NAME, "frames": F, "ebn0_db": ebn0, "reps": reps}
    nb.nbfd_logsp_init(code.handle, F, x, a)
    lsp_check = timed(lambda: nb.nbfd_logsp_check_update(code.handle, F, a, b))
    lsp_var = timed(lambda: nb.nbfd_logsp_var_update(code.handle, F, x, b, a, sym))
    out["log_sp"] = {"check_ms": lsp_check, "var_ms": lsp_var,
                     "check_fma_per_frame": 3 * (k - 2) * M * q * q, "var_adds_per_frame": 3 * N * q}
    nb.nbfd_init_messages(code.handle, F, x, None, a)
    lf_check = timed(lambda: nb.nbfd_check_update(code.handle, F, a, b))
    out["log_fourier"] = {"check_ms": lf_check, "check_adds_per_frame": 3 * k * M * q}
    for fname in ("fwht", "direct"):
        ms = timed(lambda: nb.nbfd_var_update(code.handle, F, FORMS[fname], x, b, a, sym, fsyn))
        out["log_fourier"][f"var_{fname}_ms"] = ms
    out["log_fourier"]["var_direct_fma_per_frame"] = E * q * q + 3 * m * q * N
    # the tensor-core forms on both paths: warp-level mma.sync and tcgen05 (TMEM accumulators)
    forms = {}
    for fname in ("tc32", "bf16", "fp16"):
        for path, flag in (("mma_sync", nb.MMA_SYNC), ("tcgen05", nb.TCGEN05)):
            forms[f"{fname}_{path}_ms"] = timed(
                lambda: nb.nbfd_var_update(code.handle, F, FORMS[fname] | flag, x, b, a, sym, fsyn))
    out["variable_node_tensor_core_paths"] = forms
    return out


GF64_POINTS = (1.0, 1.5, 2.0, 2.5, 3.0)


def gf64_leg(nb, torch, dev, steps, max_iter, peak_gbs, F=4096):
    """The plain batched configuration: GF(64) (2,6) N=1200, 4096 frames per launch, random
    codewords, Eb/N0 over 1.0 .. 3.0 dB, max_iter iterations with early stop. Per point and form:
    decoded Mbit/s (device time, CUDA events), FER with its 95% Clopper-Pearson interval, mean
    iterations, and the HBM fraction of the iteration kernels (check + variable node, algorithmic
    bytes / their launch time)."""
    c = synth.named_code("gf64_n1200_k6")
    enc = synth.Encoder(c)
    code = nb.Code(c)
    m, N, E, q = c["m"], c["N"], 2 * c["N"], 1 << c["m"]
    bits = enc.info_symbols * m
    stream = torch.cuda.current_stream()
    sym = torch.empty((F, N), dtype=torch.int16, device=dev)
    ok = torch.empty(F, dtype=torch.uint8, device=dev)
    its = torch.empty(F, dtype=torch.int32, device=dev)
    need = max(nb.nbfd_decode_workspace_size(code.handle, F, max_iter, f) for f in (FORMS["fwht"], FORMS["direct"]))
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    rows = []
    for si, ebn0 in enumerate(GF64_POINTS):
        tx, llr = synth.frames(c, F, ebn0, snr_idx=si, batch_idx=500, encoder=enc)
        x = torch.from_numpy(llr).to(dev)
        for fname in ("fwht", "direct"):
            form = FORMS[fname]

            def dec():
                nb.nbfd_decode(code.handle, F, x, max_iter, form, sym, ok, its, ws, need, stream)

            nb.nbfd_prof_enable((1 << nb.KERNEL_CHECK) | (1 << nb.KERNEL_VAR))
            dec()
            torch.cuda.synchronize()
            (cms, _, cu), (vms, _, vu) = nb.nbfd_prof_get(nb.KERNEL_CHECK), nb.nbfd_prof_get(nb.KERNEL_VAR)
            nb.nbfd_prof_enable(0)
            wrong = int((~np.all(sym.cpu().numpy().astype(np.int64) == tx, axis=1)).sum())
            mean_it = float(its.float().mean())
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for i in range(steps):
                ev[i][0].record(stream)
                dec()
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            ms = sum(a_.elapsed_time(b_) for a_, b_ in ev) / steps
            it_bytes = cu * 2 * E * q * 4 + vu * (2 * E * q * 4 + N * m * 4 + N * 2 + E)
            rows.append({"ebn0_db": ebn0, "form": fname, "mbit_s": bits * F / (ms / 1e3) / 1e6, "ms_per_step": ms,
                         "fer": wrong / F, "fer_ci95": clopper_pearson(wrong, F), "mean_iterations": mean_it,
                         "iteration_kernels_hbm_frac": it_bytes / ((cms + vms) / 1e3) / 1e9 / peak_gbs,
                         "check_ms": cms, "var_ms": vms})
    return {"code": "gf64_n1200_k6", "frames": F, "max_iter": max_iter, "steps_per_point": steps,
            "info_bits_per_frame": bits, "points": rows}


UNEVEN = [("gf16_n96_k4", 8192), ("gf64_n1200_k6", 2048), ("gf64_n4096_k8", 512),
          ("gf256_n512_k4", 1024), ("gf256_n2048_k16", 256)]


def uneven_leg(nb, torch, dev, form, steps, max_iter):
    """The uneven-batch configuration (five codes, per-frame Eb/N0 ~ U[1.0, 3.5], max_iter):
    one nbfd_decode_batch per step (graph-replayed loop, autotuned shapes) against the same
    frames decoded by one nbfd_decode call per code. Device time per step from CUDA events."""
    codes, xs, bits, frames = [], [], 0, 0
    for gi, (name, F) in enumerate(UNEVEN):
        c = synth.named_code(name)
        enc = synth.Encoder(c)
        rng = synth.rng_for(97, gi, 11)
        _, llr = synth.frames(c, F, rng.uniform(1.0, 3.5, size=F), snr_idx=gi, batch_idx=11, encoder=enc)
        codes.append(nb.Code(c))
        xs.append(torch.from_numpy(llr).to(dev))
        bits += F * enc.info_symbols * c["m"]
        frames += F
    handles = [c.handle for c in codes]
    ns = [int(x.shape[0]) for x in xs]
    need = nb.nbfd_decode_batch_workspace_size(handles, ns, max_iter, form)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    outs = [(torch.empty((n, c.N), dtype=torch.int16, device=dev), torch.empty(n, dtype=torch.uint8, device=dev),
             torch.empty(n, dtype=torch.int32, device=dev)) for c, n in zip(codes, ns)]
    stream = torch.cuda.current_stream()

    def batch(flags=0):
        nb.nbfd_decode_batch(handles, ns, xs, max_iter, form, flags, [o[0].data_ptr() for o in outs],
                             [o[1] for o in outs], [o[2] for o in outs], ws, need, stream)

    def per_code():
        for c, x, n, o in zip(codes, xs, ns, outs):
            nb.nbfd_decode(c.handle, n, x, max_iter, form, o[0].data_ptr(), o[1], o[2], ws, need, stream)

    batch(nb.BATCH_AUTOTUNE)  # tunes every shape once, then warm
    batch()
    torch.cuda.synchronize()
    res = {}
    for name, fn in (("batch", batch), ("per_code", per_code)):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(x.elapsed_time(y) for x, y in ev) / steps
        res[name] = {"ms_per_step": ms, "mbit_s": bits / (ms / 1e3) / 1e6}
    oks = [float(o[1].float().mean()) for o in outs]
    its = [float(o[2].float().mean()) for o in outs]
    tunes = []
    for h, n in zip(handles, ns):
        try:
            tunes.append(nb.nbfd_autotune_result(h, n, form))
        except nb.NbfdError:  # a group decoded by the fused small-code kernel has no shapes
            tunes.append(None)
    return {"codes": [n for n, _ in UNEVEN], "frames": ns, "info_bits_per_step": bits,
            "value": res["batch"]["mbit_s"], "unit": "Mbit/s", "ms_per_step": res["batch"]["ms_per_step"],
            "per_code_calls": res["per_code"], "steps": steps, "decoded_frac": oks, "mean_iterations": its,
            "tuned_shapes": [{"check_warps": abs(t[0]), "check_team": t[0] < 0, "check_stages": t[1],
                              "check_blocks_per_sm": t[2],
                              "var_blocks_per_sm": t[3], "var_warps": t[4]} if t else "fused small-code kernel"
                             for t in tunes],
            "ebn0_db": "per frame U[1.0, 3.5]", "max_iter": max_iter}


def serve_run(nb, streams, form, budget, poll_sleep=2e-4, timeout=300.0):
    """Drive the serving loop. streams: list of (code, llr [R][N][m], arrivals (s, relative, sorted)
    or None for 'all at t = 0', max_iter, info_bits). Returns per-request (ok, iters, latency, bits),
    the wall time from the first arrival to the last retirement and the worker's time per phase.
    The codes' pools are created before the clock starts (a server registers its codes at
    start-up)."""
    srv = nb.nbfd_srv_create(budget, form)
    try:
        for code, _, _, _, _ in streams:
            nb.nbfd_srv_register(srv, code.handle)
        t0 = nb.nbfd_srv_clock()
        events = []  # (arrival, stream index, frame index)
        for si, (_, llr, arr, _, _) in enumerate(streams):
            for i in range(llr.shape[0]):
                events.append((0.0 if arr is None else float(arr[i]), si, i))
        events.sort()
        total = len(events)
        bits_of = {}
        got = []
        pos = 0
        while pos < total or len(got) < total:
            now = nb.nbfd_srv_clock() - t0
            # submit every request that has arrived, per stream in one call
            end = pos
            while end < total and events[end][0] <= now:
                end += 1
            if end > pos:
                by = {}
                for arr_t, si, i in events[pos:end]:
                    by.setdefault(si, []).append((arr_t, i))
                for si, lst in by.items():
                    code, llr, _, max_iter, bits = streams[si]
                    idx = np.array([i for _, i in lst])
                    run = len(idx) > 0 and idx[-1] - idx[0] + 1 == len(idx) and bool(np.all(np.diff(idx) == 1))
                    x = llr[idx[0]:idx[-1] + 1] if run else llr[idx]  # a view when the frames are consecutive
                    tk = nb.nbfd_srv_submit_many(srv, code.handle, x, max_iter,
                                                 np.array([t0 + t for t, _ in lst]))
                    for t in tk.tolist():
                        bits_of[t] = bits
                pos = end
            tk, ok, it, lat = nb.nbfd_srv_collect(srv, 65536)
            for j in range(len(tk)):
                got.append((int(ok[j]), int(it[j]), float(lat[j]), bits_of[int(tk[j])]))
            if now > timeout:
                raise TimeoutError("serving run did not finish")
            if len(tk) == 0:
                time.sleep(poll_sleep)
        wall = nb.nbfd_srv_clock() - t0
        phases = nb.nbfd_srv_worker_times(srv)
    finally:
        nb.nbfd_srv_destroy(srv)
    return got, wall, phases


def serve_summary(got, wall, phases, offered=None):
    lat = np.array([g[2] for g in got])
    bits = sum(g[3] for g in got)
    return {"requests": len(got), "mbit_s": bits / wall / 1e6, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "fer": float(np.mean([1 - g[0] for g in got])),
            "mean_iterations": float(np.mean([g[1] for g in got])), "offered_frames_s": offered,
            "wall_s": wall, "worker_s": {k: round(v, 4) for k, v in phases.items()}}


SERVE_MIX = [("gf16_n96_k4", 0.1), ("gf64_n1200_k6", 0.3), ("gf64_n4096_k8", 0.2), ("gf256_n512_k4", 0.3),
             ("gf256_n2048_k16", 0.1)]


def serve_mix_codes(nb):
    codes = {}
    for name, _ in SERVE_MIX:
        c = synth.named_code(name)
        enc = synth.Encoder(c)
        codes[name] = (c, nb.Code(c), enc.info_symbols * c["m"], enc)
    return codes


def serve_mix_point(nb, codes, form, lam, n_req, pool_frames=8192):
    """One offered load of the serving configuration: n_req Poisson arrivals at lam frames/s, each
    request a single frame of one of five codes (weights .1/.3/.2/.3/.1), per-request Eb/N0
    uniform in 1.5-3.5 dB, max 100 iterations, a 40 GB budget for resident messages. Each code's
    requests draw from a pool of up to pool_frames distinct frames (each with its own Eb/N0), so
    that long runs need not synthesise every frame; requests beyond the pool reuse its frames in
    order."""
    rng = synth.rng_for(17, int(lam))
    dur = n_req / lam
    arr = np.sort(rng.uniform(0.0, dur, size=n_req))
    which = rng.choice(len(SERVE_MIX), size=n_req, p=[w for _, w in SERVE_MIX])
    streams = []
    for ci, (name, _) in enumerate(SERVE_MIX):
        sel = np.nonzero(which == ci)[0]
        if len(sel) == 0:
            continue
        c, code, bits, enc = codes[name]
        n_pool = min(len(sel), pool_frames)
        ebn0 = rng.uniform(1.5, 3.5, size=n_pool)
        _, pool = synth.frames(c, n_pool, ebn0, snr_idx=ci, batch_idx=int(lam) % 100000, encoder=enc)
        llr = pool if n_pool == len(sel) else np.ascontiguousarray(pool[np.arange(len(sel)) % n_pool])
        streams.append((code, llr, arr[sel], 100, bits))
    got, wall, ph = serve_run(nb, streams, form, 40 << 30)
    out = serve_summary(got, wall, ph, lam)
    out["distinct_frames"] = int(sum(min(int(np.sum(which == ci)), pool_frames) for ci in range(len(SERVE_MIX))))
    return out


def run_serve_sweep(a):
    """Serving sweep of the configured mix over offered loads 1e4 .. 1e6 frames/s."""
    import torch

    import paper_1008_4370_gb300 as nb
    from paper_1008_4370_gb300 import build as nbuild

    nbuild.build()
    torch.cuda.init()
    codes = serve_mix_codes(nb)
    form = FORMS[a.form] if FORMS[a.form] in (0, 3) else FORMS["fwht"]
    for lam in [1e4, 3e4, 1e5, 3e5, 1e6]:
        print(json.dumps({"serving_sweep": serve_mix_point(nb, codes, form, lam, a.serve_sweep_requests),
                          "form": a.form}), flush=True)


def run_ours(a):
    import torch
    import torch.distributed as dist

    import paper_1008_4370_gb300 as nb
    from paper_1008_4370_gb300 import build as nbuild

    world, rank, local = dist_setup()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        nbuild.build()
    if world > 1:
        dist.barrier()
    nb.lib()
    form = FORMS[a.form]

    code_d = synth.named_code(a.code)
    enc = synth.Encoder(code_d)
    m, N, E, q = code_d["m"], code_d["N"], 2 * code_d["N"], 1 << code_d["m"]
    info_bits = enc.info_symbols * m
    F = a.frames
    batches = []
    for b in range(a.batches):
        tx, llr = synth.frames(code_d, F, a.ebn0, snr_idx=0, batch_idx=rank * 1000 + b, encoder=enc)
        batches.append((tx, torch.from_numpy(llr).to(dev)))
    code = nb.Code(code_d)
    need = nb.nbfd_decode_workspace_size(code.handle, F, a.max_iter, form)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    sym = torch.empty((F, N), dtype=torch.int16, device=dev)
    ok = torch.empty(F, dtype=torch.uint8, device=dev)
    its = torch.empty(F, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step(i):
        nb.nbfd_decode(code.handle, F, batches[i % len(batches)][1], a.max_iter, form, sym, ok, its, ws, need,
                       stream)

    for i in range(a.warmup):
        step(i)
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = Clocks(uuid) if rank == 0 else None
    # Event timers around the two candidate dominant kernels only, during the first prof_steps
    # steps of the timed region (each timed launch adds two event records to the stream, which
    # also cost time between launches; those steps stay in the timed region).
    prof_steps = max(1, min(a.prof_steps, a.steps))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(a.steps):
        if i == 0:
            nb.nbfd_prof_enable((1 << nb.KERNEL_CHECK) | (1 << nb.KERNEL_VAR))
        elif i == prof_steps:  # totals are final: each decode call flushes its timers on return
            prof = {k: nb.nbfd_prof_get(k) for k in range(4)}
            nb.nbfd_prof_enable(0)
        evs[i][0].record(stream)
        step(i)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - t0
    step_ms = [s.elapsed_time(e) for s, e in evs]
    if prof_steps == a.steps:
        prof = {k: nb.nbfd_prof_get(k) for k in range(4)}
    nb.nbfd_prof_enable(0)
    clk = clocks.stop() if clocks else None
    dev_s = sum(step_ms) / 1e3
    t_max, value = aggregate(dev_s, F * a.steps, info_bits, dist if world > 1 else None, dev)

    # decoding statistics of every batch (outside the timed region)
    fails, iters_all = 0, []
    for b in range(len(batches)):
        step(b)
        torch.cuda.synchronize()
        ok_h = ok.cpu().numpy().astype(bool)
        fails += int((~ok_h).sum())
        iters_all.append(its.cpu().numpy())
    iters_all = np.concatenate(iters_all)
    mean_iters = float(iters_all.mean())
    fer = fails / (F * len(batches))

    # end to end: pinned host LLRs -> device -> decode -> symbols/flags/iterations back to host
    host_llr = [torch.from_numpy(synth.frames(code_d, F, a.ebn0, snr_idx=0, batch_idx=rank * 1000 + b,
                                              encoder=enc)[1]).pin_memory() for b in range(2)]
    dllr = torch.empty_like(batches[0][1])
    hsym = torch.empty((F, N), dtype=torch.int16).pin_memory()
    hok = torch.empty(F, dtype=torch.uint8).pin_memory()
    hit = torch.empty(F, dtype=torch.int32).pin_memory()
    e2e_steps = max(2, a.steps // 2)
    torch.cuda.synchronize()
    te = time.perf_counter()
    for i in range(e2e_steps):
        dllr.copy_(host_llr[i % 2], non_blocking=True)
        nb.nbfd_decode(code.handle, F, dllr, a.max_iter, form, sym, ok, its, ws, need, stream)
        hsym.copy_(sym, non_blocking=True)
        hok.copy_(ok, non_blocking=True)
        hit.copy_(its, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - te
    _, e2e_value = aggregate(e2e_s, F * e2e_steps, info_bits, dist if world > 1 else None, dev)

    # the plain FP32 direct form on the same batches (the "plain" side of served vs plain)
    plain = None
    if a.plain_steps > 0 and form != FORMS["direct"]:
        pe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(a.plain_steps)]
        nb.nbfd_decode(code.handle, F, batches[0][1], a.max_iter, FORMS["direct"], sym, ok, its, ws, need, stream)
        torch.cuda.synchronize()
        for i in range(a.plain_steps):
            pe[i][0].record(stream)
            nb.nbfd_decode(code.handle, F, batches[i % len(batches)][1], a.max_iter, FORMS["direct"], sym, ok,
                           its, ws, need, stream)
            pe[i][1].record(stream)
        torch.cuda.synchronize()
        p_s = sum(x.elapsed_time(y) for x, y in pe) / 1e3
        p_t, p_value = aggregate(p_s, F * a.plain_steps, info_bits, dist if world > 1 else None, dev)
        # FER of the plain form on every batch, and its variable-node launches timed (one decode)
        p_fail = 0
        for b in range(len(batches)):
            nb.nbfd_decode(code.handle, F, batches[b][1], a.max_iter, FORMS["direct"], sym, ok, its, ws, need,
                           stream)
            torch.cuda.synchronize()
            p_fail += int((ok == 0).sum().item())
        nb.nbfd_prof_enable(1 << nb.KERNEL_VAR)
        nb.nbfd_decode(code.handle, F, batches[0][1], a.max_iter, FORMS["direct"], sym, ok, its, ws, need, stream)
        torch.cuda.synchronize()
        pv_ms, pv_launches, pv_units = nb.nbfd_prof_get(nb.KERNEL_VAR)
        nb.nbfd_prof_enable(0)
        plain = {"form": "direct", "value": p_value, "unit": "Mbit/s", "steps": a.plain_steps,
                 "ms_per_step": 1e3 * p_t / a.plain_steps, "fer": p_fail / (F * len(batches)),
                 "var_kernel": {"ms": pv_ms, "launches": pv_launches, "frame_units": pv_units}}
    # serving leg: continuous batching of single-frame requests of this code
    # the same workload with half-precision message storage (FP32 arithmetic): a lower-precision
    # form of its own, reported beside the FP32 headline
    store16 = None
    if a.store16_steps > 0 and form == FORMS["fwht"] and world == 1:
        f16 = form | nb.STORE_F16
        need16 = nb.nbfd_decode_workspace_size(code.handle, F, a.max_iter, f16)
        for i in range(2):
            nb.nbfd_decode(code.handle, F, batches[i][1], a.max_iter, f16, sym, ok, its, ws, need16, stream)
        torch.cuda.synchronize()
        ev16 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(a.store16_steps)]
        fails16 = 0
        for i in range(a.store16_steps):
            ev16[i][0].record(stream)
            nb.nbfd_decode(code.handle, F, batches[i % len(batches)][1], a.max_iter, f16, sym, ok, its, ws,
                           need16, stream)
            ev16[i][1].record(stream)
            if i < len(batches):
                torch.cuda.synchronize()
                fails16 += int((ok == 0).sum().item())
        torch.cuda.synchronize()
        ms16 = sum(x.elapsed_time(y) for x, y in ev16) / a.store16_steps
        store16 = {"form": "fwht + half message storage", "value": info_bits * F / (ms16 / 1e3) / 1e6,
                   "unit": "Mbit/s", "ms_per_step": ms16, "steps": a.store16_steps,
                   "fer": fails16 / (F * min(len(batches), a.store16_steps)),
                   "message_bytes_per_frame_iteration": 4 * E * q * 2 + N * m * 4}
    served = None
    if a.serve_requests > 0 and world == 1:
        R = a.serve_requests
        pool = [batches[b][1].cpu().numpy() for b in range(len(batches))]
        llr_all = np.concatenate(pool, axis=0)
        reps = (R + llr_all.shape[0] - 1) // llr_all.shape[0]
        llr_req = np.concatenate([llr_all] * reps, axis=0)[:R]
        got, swall, ph = serve_run(nb, [(code, llr_req, None, a.max_iter, info_bits)], form, 32 << 30)
        sat = serve_summary(got, swall, ph)
        rng = synth.rng_for(23, R)
        arr = np.cumsum(rng.exponential(1.0 / a.serve_load, size=R))
        got2, wall2, ph2 = serve_run(nb, [(code, llr_req, arr, a.max_iter, info_bits)], form, 32 << 30)
        ld = serve_summary(got2, wall2, ph2, a.serve_load)
        served = {"form": a.form, "saturation": sat, "poisson": ld}
        if a.serve_mix_loads:
            # the configured five-code mix at a few offered loads (the full sweep: --serve-sweep)
            codes_mix = serve_mix_codes(nb)
            served["mix"] = [serve_mix_point(nb, codes_mix, form, lam, int(lam * min(1.0, max(0.2, 10000.0 / lam))))
                             for lam in a.serve_mix_loads]
    peaks, peak_kind = load_peaks()
    gf64 = None
    if a.gf64_steps > 0 and world == 1:
        gf64 = gf64_leg(nb, torch, dev, a.gf64_steps, a.max_iter, float(peaks["hbm_gbs"]))
    fused = fused_leg(nb, torch, dev, a.fused_steps, a.max_iter) if a.fused_steps > 0 and world == 1 else None
    fp32 = fp32_peak(nb) if rank == 0 else None
    table1 = (table1_leg(nb, torch, dev, a.table1_reps, F=a.table1_frames)
              if a.table1_reps > 0 and world == 1 else None)
    # the uneven five-code batch last: it holds about 9 GB while it runs
    uneven = None
    if a.uneven_steps > 0 and world == 1 and (form & 0xff) in (FORMS["fwht"], FORMS["direct"]):
        uneven = uneven_leg(nb, torch, dev, form, a.uneven_steps, a.max_iter)
        torch.cuda.empty_cache()
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return

    # roofline of the dominant kernel
    names = {0: "init", 1: "check", 2: "var", 3: "syndrome"}
    dom = max(prof, key=lambda k: prof[k][0])
    ms, launches, units = prof[dom]
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    flops_per_frame = 2.0 * (E * q * q + 3 * m * q * N)  # the direct form's q^2 FMAs per edge
    if dom == 2 and form == 0:
        achieved = flops_per_frame * units / (ms / 1e3) / 1e12
        peak = fp32["peak_tflops"]
        roof = {"bound": "alu", "kernel": "k_var_direct", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": "measured FP32 FMA rate (nbfd_diag_fp32_rate)"}
    else:
        bytes_per_frame = {
            0: N * m * 4 + E * q * 4,
            1: 2 * E * q * 4,
            2: 2 * E * q * 4 + N * m * 4 + N * 2 + E,
            3: E * 3 + N * 2,
        }[dom]
        achieved = bytes_per_frame * units / (ms / 1e3) / 1e9
        peak = float(peaks["hbm_gbs"])
        tpf = measured_traffic(names[dom], a.form, a.code) if a.frames >= 256 else None
        roof = {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None if tpf is None else tpf * units / launches,
                "algorithmic_bytes_per_launch": bytes_per_frame * units / launches,
                "peak_source": f"{peak_kind} hbm_gbs"}
    timed = {k: prof[k] for k in (1, 2)}
    roof["timed_kernel_ms_share"] = {names[k]: timed[k][0] / max(1e-9, sum(v[0] for v in timed.values()))
                                     for k in timed}
    roof["launches"] = int(launches)
    roof["timed_steps"] = f"launches of the first {prof_steps} of the {a.steps} timed steps"
    # per decode: one INIT launch, then per iteration one check, one variable and one stop launch
    launches_total = int(round(3 * prof[1][1] * a.steps / prof_steps)) + a.steps

    cpu = None
    if world == 1 and not a.no_cpu_baseline and a.code == CODE_NAME:
        cores = os.cpu_count() or 1
        sample = batches[0][1][:cores].cpu().numpy()
        wall_c, fi = oracle_frame_iterations(sample, 2, cores)
        it_ref, it_src = reference_mean_iterations(), "the oracle's own mean (oracle/workload_iterations.json)"
        if it_ref is None:
            it_ref, it_src = mean_iters, "the GPU run's mean"
        cpu_val = info_bits * (fi / wall_c) / it_ref / 1e6
        cpu = {"value": cpu_val, "unit": "Mbit/s", "cores": cores, "kind": "oracle",
               "sample": f"{cores} frames of the workload x up to 2 iterations on {cores} processes: "
                         f"{fi} frame-iterations in {wall_c:.1f} s, converted at {it_ref:.2f} "
                         f"iterations per frame ({it_src})"}

    if plain is not None and plain["var_kernel"]["ms"] > 0:
        pv = plain["var_kernel"]
        achieved = flops_per_frame * pv["frame_units"] / (pv["ms"] / 1e3) / 1e12
        plain["roofline"] = {"bound": "alu", "kernel": "k_var_direct", "achieved": achieved,
                             "peak": fp32["peak_tflops"], "unit": "TFLOP/s", "frac": achieved / fp32["peak_tflops"],
                             "peak_source": "measured FP32 FMA rate (nbfd_diag_fp32_rate)"}
    line = {
        "metric": "decoded Mbit/s (GF(256) (2,4) N=512)" if a.code == CODE_NAME else f"decoded Mbit/s ({a.code})",
        "value": value, "unit": "Mbit/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t_max / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": ("GF(256) (2,4) N=512, 1024 frames per step, Eb/N0 1.5 dB, random codewords, "
                                "max 100 iterations, early stop") if a.code == CODE_NAME and F == 1024 else
                   f"{a.code}, {F} frames per step, Eb/N0 {a.ebn0} dB, random codewords, max {a.max_iter} iterations",
                   "frames_per_step": F, "ebn0_db": a.ebn0, "max_iter": a.max_iter, "form": a.form,
                   "info_bits_per_frame": info_bits, "design_info_bits": int(N * m * (1 - 2 / code_d["k"])),
                   "l2": "working set > L2 (messages 2 x 1.07 GB streamed every iteration)",
                   "parallelism": f"replicas x{world}"},
        "fer": fer, "mean_iterations": mean_iters,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "e2e": {"value": e2e_value, "unit": "Mbit/s", "h2d_bytes_per_step": F * N * m * 4,
                "d2h_bytes_per_step": F * N * 2 + F + F * 4},
        "plain_fp32": plain,
        "store16": store16,
        "uneven_batch": uneven,
        "plain_batch_gf64": gf64,
        "fused_gf16": fused,
        "table1_check_vs_var": table1,
        "fp32_peak": fp32,
        "served": served,
        "gpu_launches": launches_total,
        "roofline": roof,
        "clocks": clk,
        "cpu_baseline": cpu,
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.serve_sweep:
        run_serve_sweep(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
