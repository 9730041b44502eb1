"""Pins of the oracle's transform, channel and Gamma layer (Sections 2.1 and 3.2)."""

import os

import numpy as np
import pytest

from oracle.channel import symbol_probabilities
from oracle.transforms import (dot, gamma, gamma_add, gamma_inv, iwht, logconv, signed_logsumexp,
                               walsh_matrix, wht, xor_conv)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bits_to_int(bits):
    return sum(int(b) << i for i, b in enumerate(bits))


def test_dot_product_example_from_paper():
    with open(os.path.join(GOLDEN, "dot_example.txt")) as f:
        line = [ln for ln in f if not ln.startswith("#")][0]
    zb, xb, val = [part.split() for part in line.split("|")]
    z, x = _bits_to_int(zb), _bits_to_int(xb)
    assert dot(z, x) == int(val[0]) == 3
    W = walsh_matrix(8)
    assert W[z, x] == (-1) ** 3


@pytest.mark.parametrize("m", [1, 2, 4, 6, 8])
def test_transform_is_involution_up_to_q(m):
    q = 1 << m
    W = walsh_matrix(m)
    np.testing.assert_array_equal(W @ W, q * np.eye(q))
    rng = np.random.default_rng(m)
    p = rng.random((5, q))
    np.testing.assert_allclose(iwht(wht(p)), p, atol=1e-13)


@pytest.mark.parametrize("m", [2, 4, 8])
def test_parseval(m):
    rng = np.random.default_rng(10 + m)
    p = rng.random((7, 1 << m))
    P = wht(p)
    np.testing.assert_allclose((P ** 2).sum(-1), (1 << m) * (p ** 2).sum(-1), rtol=1e-12)
    # P(0) = sum p (the normalisation point) and |P(z)| <= P(0) for non-negative p
    np.testing.assert_allclose(P[:, 0], p.sum(-1), rtol=1e-13)
    assert np.all(np.abs(P) <= P[:, :1] * (1 + 1e-12))


def test_transform_of_delta_and_uniform():
    q = 16
    d = np.zeros(q)
    d[5] = 1.0
    P = wht(d)
    assert np.array_equal(P, np.array([(-1.0) ** dot(z, 5) for z in range(q)]))
    u = np.full(q, 1.0 / q)
    np.testing.assert_allclose(wht(u), np.eye(q)[0], atol=1e-15)


@pytest.mark.parametrize("m", [2, 4, 6, 8])
def test_channel_transform_tanh_closed_form(m):
    """P^(0)(z) = prod_{i: z_i = 1} tanh(L_i / 2) for a product channel (from the definitions of
    p^(0) and the transform; cf. the Gallager-f remark of Section 5)."""
    rng = np.random.default_rng(20 + m)
    L = rng.normal(0.5, 3.0, size=(9, m))
    L[0, 0] = 0.0  # a bit with no information makes P(z) = 0 wherever z_1 = 1
    P = wht(symbol_probabilities(L))
    q = 1 << m
    for z in range(q):
        expect = np.ones(L.shape[0])
        for i in range(m):
            if (z >> i) & 1:
                expect = expect * np.tanh(L[:, i] / 2)
        np.testing.assert_allclose(P[:, z], expect, atol=1e-13)


def test_channel_probabilities_marginals():
    rng = np.random.default_rng(3)
    L = rng.normal(0, 4, size=(11, 6))
    p = symbol_probabilities(L)
    np.testing.assert_allclose(p.sum(-1), 1.0, rtol=1e-13)
    xs = np.arange(64)
    for i in range(6):
        pb0 = p[:, ((xs >> i) & 1) == 0].sum(-1)
        np.testing.assert_allclose(pb0, 1 / (1 + np.exp(-L[:, i])), rtol=1e-12)
    # huge LLRs stay finite
    p = symbol_probabilities(np.array([[800.0, -800.0]]))
    assert np.all(np.isfinite(p)) and p[0, 2] == pytest.approx(1.0)


def test_gamma_homomorphism_and_inverse():
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, 1000)
    y = rng.uniform(-1, 1, 1000)
    s, l = gamma_add(gamma(x), gamma(y))
    np.testing.assert_allclose(gamma_inv(s, l), x * y, rtol=1e-13)
    np.testing.assert_allclose(gamma_inv(*gamma(x)), x, rtol=1e-15)
    s0, l0 = gamma(np.array([0.0, -0.5, 0.5]))
    assert s0.tolist() == [0, 1, 0] and l0[0] == -np.inf


def test_xor_convolution_matches_double_loop():
    rng = np.random.default_rng(5)
    q = 8
    a, b = rng.random(q), rng.random(q)
    ref = np.zeros(q)
    for x1 in range(q):
        for x2 in range(q):
            ref[x1 ^ x2] += a[x1] * b[x2]
    np.testing.assert_allclose(xor_conv(a, b), ref, rtol=1e-14)


@pytest.mark.parametrize("m", [2, 4, 6])
def test_logconv_equals_linear_convolution_theorem(m):
    """The signed log-convolution of two Fourier vectors equals q times the transform of the
    product of their inverse transforms (convolution theorem)."""
    q = 1 << m
    rng = np.random.default_rng(30 + m)
    A = wht(rng.random((6, q)))
    B = wht(rng.random((6, q)))
    got = gamma_inv(*logconv(gamma(A), gamma(B)))
    ref = q * wht(iwht(A) * iwht(B))
    np.testing.assert_allclose(got, ref, atol=1e-12 * q)
    direct = np.array([[sum(A[r, z1] * B[r, z ^ z1] for z1 in range(q)) for z in range(q)] for r in range(6)])
    np.testing.assert_allclose(got, direct, atol=1e-12 * q)


def test_signed_logsumexp_edge_cases():
    s, l = signed_logsumexp(np.array([[0, 0]]), np.array([[-np.inf, -np.inf]]))
    assert s[0] == 0 and l[0] == -np.inf
    s, l = signed_logsumexp(np.array([[0, 1]]), np.array([[np.log(0.5), np.log(0.5)]]))
    assert l[0] == -np.inf  # exact cancellation -> Gamma(0) = (0, -inf)
    s, l = signed_logsumexp(np.array([[1, 1]]), np.array([[-800.0, -800.0]]))
    assert s[0] == 1 and l[0] == pytest.approx(-800 + np.log(2))
