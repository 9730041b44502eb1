"""Precision study on GF(256) (2,4) N=512: message error against FP64 and frame error rate of every
variable-node form (FP32 direct, FP32 FWHT, FP32 tensor-core bf16x3, BF16 and FP16 tensor-core
operands). Prints the tables (run with -s to see them) and checks the claims made about them:
  * message error: every form within its stated bound (FP32: u32 * kappa, BF16 / FP16:
    max(16 u_p, 4 u_p kappa)), teacher-forced on oracle message states at 0.5 / 1.5 / 2.5 dB;
  * FER, over the 0.5 - 2.5 dB sweep of the configuration, paired on identical frames: the two
    fast FP32 forms decode the same frames, and neither decodes fewer than the plain direct form."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1008_4370_gb300 as nb  # noqa: E402
from oracle import logfourier as LF  # noqa: E402
from oracle.code import OracleCode  # noqa: E402
from oracle.transforms import gamma_inv  # noqa: E402
from paper_1008_4370_gb300 import build as nbuild  # noqa: E402
from paper_1008_4370_gb300 import synth  # noqa: E402

from helpers import LOG_FLOOR, U32, decode_pair, encode, oracle_state, to_linear, var_conditions  # noqa: E402

pytestmark = pytest.mark.gpu

FORMS = [("fp32_direct", nb.FORM_FP32_DIRECT, U32), ("fp32_fwht", nb.FORM_FP32_FWHT, U32),
         ("fp32_tc", nb.FORM_FP32_TC | nb.MMA_SYNC, U32), ("bf16_tc", nb.FORM_BF16_HGEMM | nb.MMA_SYNC, 2.0 ** -9),
         ("fp16_tc", nb.FORM_FP16_HGEMM | nb.MMA_SYNC, 2.0 ** -12)]
# the tensor-core forms again on tcgen05 (message error only: the same operand precision)
TC5_FORMS = [("fp32_tc5", nb.FORM_FP32_TC | nb.TCGEN05, U32), ("bf16_tc5", nb.FORM_BF16_HGEMM | nb.TCGEN05, 2.0 ** -9),
             ("fp16_tc5", nb.FORM_FP16_HGEMM | nb.TCGEN05, 2.0 ** -12)]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    nbuild.build()
    return torch.device("cuda:0")


def clopper_pearson(k, n, alpha=0.05):
    from scipy.stats import beta
    lo = 0.0 if k == 0 else beta.ppf(alpha / 2, k, n - k + 1)
    hi = 1.0 if k == n else beta.ppf(1 - alpha / 2, k + 1, n - k)
    return lo, hi


def test_message_error_per_form(dev):
    c = synth.named_code("gf256_n512_k4")
    oc = OracleCode.from_dict(c)
    code = nb.Code(c)
    vs = np.arange(0, oc.N, 8)
    es = np.concatenate([oc.C[v] for v in vs])
    rows = []
    for ebn0 in (0.5, 1.5, 2.5):
        _, llr = synth.frames(c, 1, ebn0, batch_idx=41)
        lam0, _, c2v = oracle_state(oc, llr[0].astype(np.float64), 2)
        c2v_in = encode(*c2v)
        c2v_o = decode_pair(c2v_in)
        s_ref, l_ref = LF.var_update(oc, lam0, c2v_o, vars=vs)
        P_ref = gamma_inv(s_ref[es], l_ref[es])
        kappa = var_conditions(oc, lam0, c2v_o)[es]
        x = torch.from_numpy(llr).to(dev)
        cin = torch.from_numpy(c2v_in[None]).to(dev)
        for name, form, u in FORMS + TC5_FORMS:
            out = torch.empty_like(cin)
            nb.nbfd_var_update(code.handle, 1, form, x, cin, out)
            torch.cuda.synchronize()
            g = out.cpu().numpy()[0][es]
            err = np.abs(to_linear(g) - P_ref)
            mask = np.abs(P_ref) >= LOG_FLOOR
            lerr = np.abs(-np.abs(g.astype(np.float64))[mask] - l_ref[es][mask])
            bound = np.maximum(1e-5, u * kappa) if u == U32 else np.maximum(16 * u, 4 * u * kappa)
            ratio = float(np.max(err / bound[:, None]))
            rows.append((ebn0, name, float(err.max()), float(np.percentile(err, 99)), float(np.median(err)),
                         float(lerr.max()), float(np.percentile(lerr, 99)), ratio))
            assert ratio <= 1.0, (ebn0, name, ratio)
    print("\nV->C message error against FP64 (teacher-forced, 64 variables x 2 edges x 256 entries)")
    print("Eb/N0  form          lin max   lin p99   lin p50   ln|P| max  ln|P| p99  max err/bound")
    for r in rows:
        print(f"{r[0]:4.1f}   {r[1]:12s} {r[2]:.2e}  {r[3]:.2e}  {r[4]:.2e}  {r[5]:.2e}   {r[6]:.2e}   {r[7]:.3f}")


def test_fer_per_form(dev):
    c = synth.named_code("gf256_n512_k4")
    code = nb.Code(c)
    enc = synth.Encoder(c)
    F = 1024
    snrs = [0.5 + 0.25 * i for i in range(9)]
    results = {}
    for si, ebn0 in enumerate(snrs):
        tx, llr = synth.frames(c, F, ebn0, snr_idx=si, batch_idx=77, encoder=enc)
        x = torch.from_numpy(llr).to(dev)
        for name, form, _ in FORMS:
            sym, ok, it = nb.decode(code, x, 100, form)
            torch.cuda.synchronize()
            correct = np.all(sym.cpu().numpy().astype(np.int64) == tx, axis=1)
            results[(ebn0, name)] = (correct, float(it.float().mean()))
    print("\nFER (1024 frames per point, max 100 iterations; 95% Clopper-Pearson interval)")
    print("Eb/N0 " + "".join(f"{n:>26s}" for n, _, _ in FORMS))
    for ebn0 in snrs:
        cells = []
        for name, _, _ in FORMS:
            corr, itm = results[(ebn0, name)]
            k = int((~corr).sum())
            lo, hi = clopper_pearson(k, F)
            cells.append(f"{k / F:.4f} [{lo:.4f},{hi:.4f}] {itm:4.1f}")
        print(f"{ebn0:4.2f}  " + "  ".join(f"{cl:>24s}" for cl in cells))
    # Paired comparisons on identical frames (exact binomial tests on the discordant frames):
    #  * the two fast FP32 forms (butterflies, tensor-core bf16x3) decode the same frames;
    #  * neither decodes fewer frames than the plain FP32 direct form (which carries more FP32
    #    rounding in its q^2-term sums and has no x-domain projection).
    from scipy.stats import binomtest
    for ebn0 in snrs:
        fw = results[(ebn0, "fp32_fwht")][0]
        tc = results[(ebn0, "fp32_tc")][0]
        dr = results[(ebn0, "fp32_direct")][0]
        n01, n10 = int(np.sum(fw & ~tc)), int(np.sum(~fw & tc))
        if n01 + n10 > 8:
            assert binomtest(n01, n01 + n10, 0.5).pvalue > 0.001, (ebn0, n01, n10)
        for fast in (fw, tc):
            worse, better = int(np.sum(~fast & dr)), int(np.sum(fast & ~dr))
            if worse + better > 8:
                assert binomtest(worse, worse + better, 0.5, alternative="greater").pvalue > 0.001, \
                    (ebn0, worse, better)
    assert math.isfinite(sum(v[1] for v in results.values()))
