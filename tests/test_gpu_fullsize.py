"""Full-size teacher-forced parity of the check-node and variable-node kernels: GF(256) (2,4)
N=512 at 1024 frames and GF(64) (2,6) N=1200 at 4096 frames, the batch sizes the configurations
name, and for the check node also GF(256) (2,16) N=2048 at 256 frames, through the step-level C
ABI calls (the kernels, grids and pipelines nbfd_decode launches).

Inputs are distinct per frame and still checkable everywhere. A handful of oracle message states
(G "virtual frames": several Eb/N0, iterations and saturated / zero-information LLRs) form a pool;
every unit of every frame -- a check with its k incoming messages, or a variable with its LLRs and
two incoming messages -- takes its inputs from a pool state drawn at random per (frame, unit).
Frames 0..G-1 are the pool states themselves. Then
  * frames 0..G-1 are compared with the FP64 oracle element by element, every unit;
  * every other unit's outputs must equal, bit for bit, the outputs of the same unit in the frame
    whose state it copied (the kernels' arithmetic does not depend on where a unit sits in the
    grid); a unit that differs is compared with the oracle directly instead.
So every output of the full-size launch -- all grid waves, all warps, every bulk-copy pipeline
stage -- is checked against the oracle (Section 3.2 CHECK TO VARIABLE and VARIABLE TO CHECK /
TENTATIVE DECISION), and a unit corrupted anywhere in the grid fails.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1008_4370_gb300 as nb  # noqa: E402
from oracle import logfourier as LF  # noqa: E402
from oracle.code import OracleCode  # noqa: E402
from paper_1008_4370_gb300 import build as nbuild  # noqa: E402
from paper_1008_4370_gb300 import synth  # noqa: E402

from helpers import (MARGIN, compare, decode_pair, encode, log_exempt_cap, oracle_state,  # noqa: E402
                     var_conditions, var_log_conditions, vn_margins)

pytestmark = pytest.mark.gpu

# (code, frames per launch) of the configurations
FULL = [("gf256_n512_k4", 1024), ("gf64_n1200_k6", 4096)]
# pool states: (Eb/N0 dB, oracle iterations before the state is taken, special LLRs)
STATES = [(0.5, 0, True), (1.0, 1, False), (1.5, 2, False), (2.5, 1, False), (0.75, 3, True),
          (2.0, 2, False)]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    nbuild.build()
    return torch.device("cuda:0")


def _llr(c, ebn0, special, batch):
    _, llr = synth.frames(c, 1, ebn0, batch_idx=batch)
    llr = llr[0].copy()
    if special:
        llr[0, 0] = 0.0          # a bit with no information: P0(z) = 0 wherever z_1 = 1
        llr[1:3, :] = 45.0       # saturated channel
        llr[3, :] = -45.0
    return llr


def _assign(F, units, G, seed):
    """Pool state of every (frame, unit): frames 0..G-1 are the states themselves."""
    g = np.random.default_rng(seed).integers(0, G, size=(F, units))
    g[:G] = np.arange(G)[:, None]
    return g


def _mismatch(o, g, unit_of_slot=None):
    """(F, units) bool on the device: outputs that differ from those of the same unit in the
    frame whose pool state they copied. o: (F, units, w) int32 view."""
    F, U = g.shape
    gt = torch.from_numpy(g).to(o.device)
    if unit_of_slot is None:
        rep = o[gt, torch.arange(U, device=o.device)[None, :]]
        return (rep != o).any(-1)
    us = torch.from_numpy(unit_of_slot).to(o.device)
    src = gt[:, us]  # (F, slots): frame whose state slot's unit copied
    rep = o[src, torch.arange(o.shape[1], device=o.device)[None, :]]
    return (rep != o).reshape(F, o.shape[1], -1).any(-1)


# the uneven batch's GF(256) (2,16) N=2048 group (256 frames): the check kernel's team variant
FULL_CHECK = FULL + [("gf256_n2048_k16", 256)]


@pytest.mark.parametrize("name,F", FULL_CHECK)
def test_check_update_full_size(dev, name, F):
    c = synth.named_code(name)
    oc = OracleCode.from_dict(c)
    k, q, M = int(c["k"]), oc.q, oc.M
    pool = []
    for i, (ebn0, iters, special) in enumerate(STATES):
        llr = _llr(c, ebn0, special, 60 + i)
        if iters == 0:
            _, v2c = LF.init(oc, llr.astype(np.float64))
        else:
            _, v2c, _ = oracle_state(oc, llr.astype(np.float64), iters)
        pool.append(encode(*v2c))
    pool = np.stack(pool)  # (G, E, q), check-major slots
    G = len(pool)
    g = _assign(F, M, G, seed=7)
    x = pool.reshape(G, M, k * q)[g, np.arange(M)[None, :]]  # (F, M, k q)
    code = nb.Code(c)
    xin = torch.from_numpy(x).to(dev)
    del x
    out = torch.empty((F, oc.E, q), dtype=torch.float32, device=dev)
    nb.nbfd_check_update(code.handle, F, xin, out)
    torch.cuda.synchronize()
    del xin
    o = out.view(F, M, k * q).view(torch.int32)
    bad = _mismatch(o, g).cpu().numpy()
    exp = [LF.check_update(oc, decode_pair(pool[r])) for r in range(G)]
    stats = []
    for r in range(G):
        ok, st = compare(out[r].cpu().numpy(), *exp[r])
        assert ok and st["exempt"] == 0.0, (r, st)  # products of Gamma values: condition 1
        stats.append(st)
    # units that are not bit-identical to their copy: compared with the oracle directly
    fb, cb = np.nonzero(bad)
    cslots = np.asarray([oc.V[cc] for cc in range(M)])  # (M, k)
    for r in range(G):
        sel = g[fb, cb] == r
        if sel.any():
            fe = np.repeat(fb[sel], k)
            es = cslots[cb[sel]].reshape(-1)
            got = out[torch.from_numpy(fe).to(dev), torch.from_numpy(es).to(dev)].cpu().numpy()
            ok, st = compare(got, exp[r][0][es], exp[r][1][es])
            assert ok, (r, st)
    print(f"\n{name} check node, {F} frames: {G} pool states vs oracle, "
          f"{F * M - G * M} copied checks, {int(bad.sum())} not bit-identical to their copy; "
          f"max lin err {max(s['lin_max'] for s in stats):.2e}, max log err {max(s['log_max'] for s in stats):.2e}")


VAR_FORMS = {"gf256_n512_k4": [nb.FORM_FP32_DIRECT, nb.FORM_FP32_FWHT, nb.FORM_FP32_TC | nb.MMA_SYNC,
                               nb.FORM_FP32_TC | nb.TCGEN05],
             "gf64_n1200_k6": [nb.FORM_FP32_DIRECT, nb.FORM_FP32_FWHT]}
VAR_STATES = [(0.5, 1, True), (1.0, 2, False), (1.5, 1, False), (2.5, 3, False), (2.0, 2, True)]


@pytest.fixture(scope="module")
def var_pools():
    """Per code: (LLR pool (G, N, m), C->V pool (G, E, q) float32, oracle V->C, tentative
    outputs and conditions per state)."""
    out = {}
    for name, _ in FULL:
        c = synth.named_code(name)
        oc = OracleCode.from_dict(c)
        L, C, ref = [], [], []
        for i, (ebn0, iters, special) in enumerate(VAR_STATES):
            llr = _llr(c, ebn0, special, 70 + i)
            _, _, c2v = oracle_state(oc, llr.astype(np.float64), iters)
            cin = encode(*c2v)
            c2v_o = decode_pair(cin)
            lam0, _ = LF.init(oc, llr.astype(np.float64))
            v2c = LF.var_update(oc, lam0, c2v_o)
            Mv = LF.tentative(oc, lam0, c2v_o)
            ref.append({"v2c": v2c, "x": LF.bit_decisions(oc, Mv), "w": LF.fourier_syndrome_words(oc, Mv),
                        "margin": vn_margins(oc, Mv), "kappa": var_conditions(oc, lam0, c2v_o),
                        "kappa_log": var_log_conditions(oc, lam0, c2v_o)})
            L.append(llr)
            C.append(cin)
        out[name] = (np.stack(L), np.stack(C), ref)
    return out


@pytest.mark.parametrize("name,F,form", [(n, F, f) for n, F in FULL for f in VAR_FORMS[n]])
def test_var_update_full_size(dev, var_pools, name, F, form):
    c = synth.named_code(name)
    oc = OracleCode.from_dict(c)
    N, E, q, m = oc.N, oc.E, oc.q, oc.m
    L, C, ref = var_pools[name]
    G = len(L)
    g = _assign(F, N, G, seed=11)
    ev = np.asarray(oc.edge_var)
    llr = L[g, np.arange(N)[None, :]]                       # (F, N, m)
    c2v = C[g[:, ev], np.arange(E)[None, :]]                # (F, E, q)
    code = nb.Code(c)
    x = torch.from_numpy(np.ascontiguousarray(llr)).to(dev)
    cin = torch.from_numpy(c2v).to(dev)
    del c2v
    v2c = torch.empty((F, E, q), dtype=torch.float32, device=dev)
    sym = torch.zeros((F, N), dtype=torch.int16, device=dev)
    fsyn = torch.zeros((F, E), dtype=torch.uint8, device=dev)
    nb.nbfd_var_update(code.handle, F, form, x, cin, v2c, sym, fsyn)
    torch.cuda.synchronize()
    del cin
    bad_msg = _mismatch(v2c.view(torch.int32).view(F, E, q), g, unit_of_slot=ev).cpu().numpy()  # (F, E)
    bad_sym = _mismatch(sym.view(F, N, 1), g).cpu().numpy()                                      # (F, N)
    bad_w = _mismatch(fsyn.view(F, E, 1), g, unit_of_slot=ev).cpu().numpy()                     # (F, E)
    gs = sym.cpu().numpy().astype(np.int64)
    gw = fsyn.cpu().numpy().astype(np.int64)
    worst = {"lin_max": 0.0, "log_max": 0.0, "exempt": 0.0}
    n_dec = 0
    vslots = np.asarray([oc.C[v] for v in range(N)])  # (N, 2)

    def check_units(fs, vs, r):
        """Outputs of variables vs in frames fs (same length) against pool state r's oracle."""
        nonlocal n_dec
        R = ref[r]
        fe = np.repeat(fs, 2)
        es = vslots[vs].reshape(-1)
        got = v2c[torch.from_numpy(fe).to(dev), torch.from_numpy(es).to(dev)].cpu().numpy()
        ok, st = compare(got, R["v2c"][0][es], R["v2c"][1][es], kappa=R["kappa"][es],
                         kappa_log=R["kappa_log"][es])
        assert ok, (r, st)
        for key in ("lin_max", "log_max", "exempt"):
            worst[key] = max(worst[key], st[key])
        clear = R["margin"][vs] > MARGIN
        n_dec += int(clear.sum())
        assert np.array_equal(gs[fs[clear], vs[clear]], R["x"][vs[clear]]), r
        ec = vslots[vs[clear]]
        fc = fs[clear]
        for j in range(2):
            assert np.array_equal(gw[fc, ec[:, j]], R["w"][ec[:, j]]), r

    for r in range(G):  # the pool states themselves, every variable
        check_units(np.full(N, r), np.arange(N), r)
    # units that differ from their copy anywhere (message, decision or syndrome word)
    bad_var = bad_sym.copy()
    for arr in (bad_msg, bad_w):
        fi, ei = np.nonzero(arr)
        bad_var[fi, ev[ei]] = True
    fb, vb = np.nonzero(bad_var)
    for r in range(G):
        sel = g[fb, vb] == r
        if sel.any():
            check_units(fb[sel], vb[sel], r)
    assert worst["exempt"] <= log_exempt_cap(m), worst
    print(f"\n{name} variable node form {form}, {F} frames: {G} pool states vs oracle, {F * N - G * N} copied "
          f"variables, {int(bad_var.sum())} not bit-identical to their copy; max lin err {worst['lin_max']:.2e}, "
          f"max log err {worst['log_max']:.2e}, log-exempt share {worst['exempt']:.4f}; {n_dec} decisions compared")
    assert n_dec > G * N // 4
