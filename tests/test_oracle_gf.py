"""Pins of the oracle's GF(2^m) layer (Section 2 representation, Appendix A)."""

import os

import numpy as np
import pytest

from oracle.gf import GF, clmul_mod
from oracle.transforms import wht

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
POLYS = {2: 0x7, 3: 0xB, 4: 0x13, 6: 0x43, 8: 0x11D}


def test_gf8_table_matches_paper():
    g = GF(3, 0xB)  # alpha^3 + alpha + 1 = 0
    rows = []
    with open(os.path.join(GOLDEN, "gf8_table.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, *bits = line.split()
            rows.append((name, [int(b) for b in bits]))
    assert len(rows) == 8
    for name, bits in rows:
        if name == "0":
            sym = 0
        elif name == "1":
            sym = g.alpha_pow(0)
        elif name == "alpha":
            sym = g.alpha_pow(1)
        else:
            sym = g.alpha_pow(int(name.split("^")[1]))
        assert g.to_bits(sym).tolist() == bits, name


@pytest.mark.parametrize("m", sorted(POLYS))
def test_primitive_polynomials_have_order_q_minus_1(m):
    g = GF(m, POLYS[m])
    q = g.q
    powers = {g.alpha_pow(i) for i in range(q - 1)}
    assert powers == set(range(1, q))
    assert g.alpha_pow(q - 1) == 1


def test_rejects_non_primitive_and_wrong_degree():
    with pytest.raises(ValueError):
        GF(4, 0x1F)  # x^4+x^3+x^2+x+1: irreducible, alpha has order 5
    with pytest.raises(ValueError):
        GF(4, 0x15)  # x^4+x^2+1 = (x^2+x+1)^2: reducible
    with pytest.raises(ValueError):
        GF(4, 0x25)  # degree 5


@pytest.mark.parametrize("m", [2, 3, 4, 6])
def test_tables_match_bitserial_multiply_all_pairs(m):
    g = GF(m, POLYS[m])
    a, b = np.meshgrid(np.arange(g.q), np.arange(g.q), indexing="ij")
    tab = g.mul(a, b)
    brute = np.vectorize(lambda x, y: clmul_mod(int(x), int(y), g.poly, m))(a, b)
    assert np.array_equal(tab, brute)


def test_tables_match_bitserial_multiply_gf256_sample():
    g = GF(8, 0x11D)
    rng = np.random.default_rng(1)
    a = rng.integers(0, 256, 4000)
    b = rng.integers(0, 256, 4000)
    brute = np.array([clmul_mod(int(x), int(y), 0x11D, 8) for x, y in zip(a, b)])
    assert np.array_equal(g.mul(a, b), brute)
    nz = np.arange(1, 256)
    assert np.all(g.mul(nz, g.inv(nz)) == 1)


@pytest.mark.parametrize("m", [2, 3, 4, 6, 8])
def test_companion_matrix_power_multiplies_by_alpha_power(m):
    """Appendix A: A^i alpha^j = alpha^{i+j} on m-bit column vectors."""
    g = GF(m, POLYS[m])
    idx = range(g.q - 1) if m <= 4 else range(0, g.q - 1, 7)
    for i in idx:
        Ai = g.companion_power(i)
        for j in (range(g.q - 1) if m <= 4 else range(0, g.q - 1, 11)):
            got = g.from_bits((Ai @ g.to_bits(g.alpha_pow(j))) & 1)
            assert got == g.alpha_pow(i + j)
            # and the product with the tables / the bit-serial multiply agree
            assert got == clmul_mod(g.alpha_pow(i), g.alpha_pow(j), g.poly, m)


@pytest.mark.parametrize("m", [2, 3, 4, 6, 8])
def test_fourier_permutation_identity_appendix_a(m):
    """Appendix A: the transform of p~(x) = p(h^{-1} x) is P(H_cv z), H_cv = (A^i)^T."""
    g = GF(m, POLYS[m])
    rng = np.random.default_rng(m)
    xs = np.arange(g.q)
    hs = range(1, g.q) if m <= 6 else rng.integers(1, g.q, 24)
    for h in hs:
        h = int(h)
        p = rng.random(g.q)
        p /= p.sum()
        p_tilde = p[g.mul(g.inv(h), xs)]
        lhs = wht(p_tilde)
        rhs = wht(p)[g.fourier_index_map(h)]
        np.testing.assert_allclose(lhs, rhs, atol=1e-12, rtol=0)


def test_transpose_matters():
    """Indexing by h*z (the un-transposed matrix) breaks the identity for most h in GF(16):
    the pin above would catch that mistake."""
    g = GF(4, 0x13)
    xs = np.arange(16)
    rng = np.random.default_rng(0)
    p = rng.random(16)
    wrong_ok = 0
    differ = 0
    for h in range(1, 16):
        naive = g.mul(h, xs)
        if not np.array_equal(naive, g.fourier_index_map(h)):
            differ += 1
        lhs = wht(p[g.mul(g.inv(h), xs)])
        if np.allclose(lhs, wht(p)[naive], atol=1e-12):
            wrong_ok += 1
    assert differ >= 10
    assert wrong_ok < 15


@pytest.mark.parametrize("m", [2, 4, 8])
def test_inverse_index_map_is_map_of_inverse(m):
    g = GF(m, POLYS[m])
    for h in range(1, g.q, max(1, g.q // 32)):
        inv = g.fourier_index_map_inverse(h)
        assert np.array_equal(inv, g.fourier_index_map(int(g.inv(h))))
        # the map is GF(2)-linear: image of z is the XOR of the images of its bits
        fwd = g.fourier_index_map(h)
        for z in range(g.q):
            acc = 0
            for b in range(m):
                if (z >> b) & 1:
                    acc ^= int(fwd[1 << b])
            assert fwd[z] == acc
