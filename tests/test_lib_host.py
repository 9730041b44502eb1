"""Host-side checks of libnbfd that need no GPU: it builds for sm_103a, loads, exports every
symbol include/nbfd.h declares, validates codes, and its index maps equal the oracle's."""

import os
import re

import numpy as np
import pytest

import paper_1008_4370_gb300 as nb
from oracle.gf import GF
from paper_1008_4370_gb300 import build as nbuild
from paper_1008_4370_gb300 import synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "nbfd.h")


@pytest.fixture(scope="module")
def L():
    nbuild.build()
    return nb.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nbfd_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    # and the binding declares a signature for each
    assert sorted(s[0] for s in nb.SIGNATURES) == names


def _args(code):
    return (code["N"], code["M"], code["k"], code["m"], code["poly"], code["edge_check"],
            code["edge_var"], code["edge_h"])


def _expect_status(status, *args):
    with pytest.raises(nb.NbfdError) as ei:
        nb.nbfd_code_create(*args)
    assert ei.value.status == status, str(ei.value)
    assert nb.nbfd_status_string(status) in {"NBFD_EINVAL", "NBFD_ENOTREG", "NBFD_EPOLY", "NBFD_EDUP",
                                              "NBFD_EZERO"}


def test_code_create_rejects_bad_codes(L):
    c = synth.named_code("gf16_n32_k4")
    N, M, k, m, poly, ec, ev, eh = _args(c)
    _expect_status(-3, N, M, k, m, 0x1F, ec, ev, eh)  # not primitive
    _expect_status(-3, N, M, k, m, 0x25, ec, ev, eh)  # wrong degree
    eh0 = eh.copy()
    eh0[5] = 0
    _expect_status(-5, N, M, k, m, poly, ec, ev, eh0)
    eh16 = eh.copy()
    eh16[3] = 16
    _expect_status(-5, N, M, k, m, poly, ec, ev, eh16)
    ev_dup = ev.copy()
    ev_dup[1] = ev_dup[0]  # two edges (0, v) on check 0
    _expect_status(-4, N, M, k, m, poly, ec, ev_dup, eh)
    ev_deg = ev.copy()
    # move one socket of variable a to variable b: a gets degree 1, b degree 3
    a, b = int(ev[0]), int([v for v in ev if v not in set(ev[:k].tolist())][0])
    ev_deg[0] = b
    with pytest.raises(nb.NbfdError) as ei:
        nb.nbfd_code_create(N, M, k, m, poly, ec, ev_deg, eh)
    assert ei.value.status in (-2, -4)
    _expect_status(-2, N, M, k + 1, m, poly, ec, ev, eh)  # counts disagree
    _expect_status(-1, N, M, k, 9, poly, ec, ev, eh)  # m out of range
    _expect_status(-1, N, M, k, 1, 0x3, ec, ev, eh)
    ev_oob = ev.copy()
    ev_oob[2] = N
    _expect_status(-1, N, M, k, m, poly, ec, ev_oob, eh)
    assert "not" in nb.nbfd_last_error() or nb.nbfd_last_error()


@pytest.mark.parametrize("m,poly", [(2, 0x7), (3, 0xB), (4, 0x13), (5, 0x25), (6, 0x43), (7, 0x89), (8, 0x11D)])
def test_library_index_map_equals_oracle(L, m, poly):
    """Bit-exact: the C++ map (parities of z AND h*alpha^j) equals the oracle's GF(2) product with
    (A^i)^T built from the companion matrix of Appendix A."""
    tab = nb.nbfd_field_index_map(m, poly)
    g = GF(m, poly)
    assert not tab[0].any()
    for h in range(1, g.q):
        assert np.array_equal(tab[h], g.fourier_index_map(h).astype(np.uint8)), h


def test_field_index_map_rejects_bad_polynomial(L):
    with pytest.raises(nb.NbfdError) as ei:
        nb.nbfd_field_index_map(4, 0x1F)
    assert ei.value.status == -3


def test_python_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(nb, "_lib", None)
    monkeypatch.setattr(nb, "LIB_PATH", "/nonexistent/libnbfd.so")
    with pytest.raises(ImportError):
        nb.lib()


def header_defines():
    """Integer #define NBFD_* values of include/nbfd.h."""
    text = open(HEADER).read()
    out = {}
    for m in re.finditer(r"#define\s+(NBFD_[A-Z0-9_]+)\s+\(?\s*(-?(?:0x[0-9A-Fa-f]+|\d+))\s*\)?", text):
        out[m.group(1)] = int(m.group(2), 0)
    return out


def test_binding_constants_equal_the_header():
    """The Python binding passes forms, flags and kernel ids as plain integers: each must equal
    the value include/nbfd.h defines."""
    d = header_defines()
    pairs = {
        "NBFD_FORM_FP32_DIRECT": nb.FORM_FP32_DIRECT, "NBFD_FORM_BF16_HGEMM": nb.FORM_BF16_HGEMM,
        "NBFD_FORM_FP16_HGEMM": nb.FORM_FP16_HGEMM, "NBFD_FORM_FP32_FWHT": nb.FORM_FP32_FWHT,
        "NBFD_FORM_FP32_TC": nb.FORM_FP32_TC, "NBFD_FORM_FP64_DIRECT": nb.FORM_FP64_DIRECT,
        "NBFD_DECIDE_SYMBOL": nb.DECIDE_SYMBOL,
        "NBFD_STORE_F16": nb.STORE_F16, "NBFD_BATCH_AUTOTUNE": nb.BATCH_AUTOTUNE,
        "NBFD_KERNEL_INIT": nb.KERNEL_INIT, "NBFD_KERNEL_CHECK": nb.KERNEL_CHECK,
        "NBFD_KERNEL_VAR": nb.KERNEL_VAR, "NBFD_KERNEL_SYNDROME": nb.KERNEL_SYNDROME,
        "NBFD_KERNEL_TAIL": nb.KERNEL_TAIL, "NBFD_KERNEL_FUSED": nb.KERNEL_FUSED, "NBFD_UNFUSED": nb.UNFUSED, "NBFD_TCGEN05": nb.TCGEN05, "NBFD_MMA_SYNC": nb.MMA_SYNC,
    }
    for name, value in pairs.items():
        assert d[name] == value, name
    # every kernel id has a timer bit in NBFD_PROF_ALL, and the ids are 0 .. COUNT-1
    kernels = sorted(v for k, v in d.items() if k.startswith("NBFD_KERNEL_") and k != "NBFD_KERNEL_COUNT")
    assert kernels == list(range(d["NBFD_KERNEL_COUNT"]))
    assert d["NBFD_PROF_ALL"] == (1 << d["NBFD_KERNEL_COUNT"]) - 1
    # status codes are distinct and negative, NBFD_OK is 0
    errs = [v for k, v in d.items() if k.startswith("NBFD_E")]
    assert d["NBFD_OK"] == 0 and len(set(errs)) == len(errs) and max(errs) < 0
