"""Fourier transform over the additive group of GF(2^m), the Gamma map and the log-convolution.

Test infrastructure only (FP64 oracle).

* Section 2.1: P(z) = sum_x p(x) (-1)^{z.x}, where z.x is the dot product of the m-bit
  representations; the inverse transform carries the factor 1/2^m. Written here from the
  definition as a q x q matrix product (no butterflies), so it is checked against nothing but
  its definition, W.W = qI and Parseval.
* Section 3.2: Gamma(x) = (sgn(x), ln|x|) with sgn in GF(2); Gamma(xy) = Gamma(x) + Gamma(y).
  sgn(0) is "chosen randomly" in the paper; the oracle takes 0 (with ln|0| = -inf).
* Section 3.2, the boxplus definition: (l1 [+] l2)(x) = Gamma( sum_{x1 + x2 = x}
  Gamma^{-1}(l1(x1) + l2(x2)) ), the sum over GF(2^m) addition (XOR of bit vectors).
  Evaluated literally: q terms per output, each a signed exponential, summed after a
  per-output max shift (the shift is exact algebra, exp(a)*sum exp(l-a)).

A Gamma-form vector is a pair (s, l): s uint8 in {0,1}, l float64 in [-inf, 0] (or any real
for unnormalised vectors).
"""

from __future__ import annotations

import numpy as np


def dot(z: int, x: int) -> int:
    """z.x of Section 2.1: number of coordinates where both bit vectors are 1."""
    return bin(int(z) & int(x)).count("1")


def walsh_matrix(m: int) -> np.ndarray:
    """W[z, x] = (-1)^{z.x} for z, x in GF(2^m), built entry by entry from the definition."""
    q = 1 << m
    zs = np.arange(q)
    pc = np.zeros((q, q), dtype=np.int64)
    for b in range(m):
        pc += ((zs[:, None] >> b) & 1) * ((zs[None, :] >> b) & 1)
    return np.where(pc % 2 == 0, 1.0, -1.0)


def wht(p: np.ndarray) -> np.ndarray:
    """Fourier transform along the last axis: P(z) = sum_x p(x)(-1)^{z.x}."""
    p = np.asarray(p, dtype=np.float64)
    W = walsh_matrix(int(p.shape[-1]).bit_length() - 1)
    return p @ W.T


def iwht(P: np.ndarray) -> np.ndarray:
    """Inverse transform: p(x) = 2^{-m} sum_z P(z)(-1)^{z.x}."""
    P = np.asarray(P, dtype=np.float64)
    q = int(P.shape[-1])
    W = walsh_matrix(q.bit_length() - 1)
    return (P @ W.T) / q


def gamma(x: np.ndarray):
    """Gamma(x) = (sgn_GF(2)(x), ln|x|); sgn(0) := 0, ln 0 = -inf."""
    x = np.asarray(x, dtype=np.float64)
    s = (x < 0).astype(np.uint8)
    with np.errstate(divide="ignore"):
        l = np.log(np.abs(x))
    return s, l


def gamma_inv(s: np.ndarray, l: np.ndarray) -> np.ndarray:
    """Gamma^{-1}(s, l) = (-1)^s exp(l)."""
    s = np.asarray(s)
    return np.where(s.astype(bool), -1.0, 1.0) * np.exp(np.asarray(l, dtype=np.float64))


def gamma_add(a, b):
    """Gamma(x) + Gamma(y) = (s_x XOR s_y, l_x + l_y) = Gamma(xy) for non-zero x, y."""
    return (a[0] ^ b[0]).astype(np.uint8), a[1] + b[1]


def signed_logsumexp(s: np.ndarray, l: np.ndarray, axis: int = -1):
    """Gamma( sum_i Gamma^{-1}(s_i, l_i) ) along `axis`, with a max shift for range safety."""
    l = np.asarray(l, dtype=np.float64)
    lmax = np.max(l, axis=axis, keepdims=True)
    finite = np.isfinite(lmax)
    shift = np.where(finite, lmax, 0.0)
    terms = np.where(np.asarray(s).astype(bool), -1.0, 1.0) * np.exp(l - shift)
    tot = np.sum(terms, axis=axis, keepdims=True)
    so, lo = gamma(tot)
    lo = np.where(finite, lo + shift, -np.inf)
    so = np.where(finite, so, 0).astype(np.uint8)
    return np.squeeze(so, axis=axis), np.squeeze(lo, axis=axis)


def _xor_index(q: int) -> np.ndarray:
    xs = np.arange(q)
    return xs[:, None] ^ xs[None, :]  # [x, x1] -> x XOR x1 (= x - x1 in GF(2^m))


def logconv(a, b):
    """(a [+] b)(x) of the boxplus definition (Section 3.2), literal q-term sum per output.

    a, b: Gamma-form pairs with arrays of shape (..., q). Returns a Gamma-form pair.
    """
    sa, la = a
    sb, lb = b
    q = int(np.asarray(la).shape[-1])
    X = _xor_index(q)
    # term (x, x1) = Gamma(a(x1)) + Gamma(b(x - x1))
    ts = np.asarray(sa)[..., None, :] ^ np.asarray(sb)[..., X]
    tl = np.asarray(la)[..., None, :] + np.asarray(lb)[..., X]
    return signed_logsumexp(ts, tl, axis=-1)


def xor_conv(p1: np.ndarray, p2: np.ndarray) -> np.ndarray:
    """(p1 (x) p2)(x) = sum_{x1 + x2 = x} p1(x1) p2(x2), the Section 2.1 convolution, O(q^2)."""
    p1 = np.asarray(p1, dtype=np.float64)
    p2 = np.asarray(p2, dtype=np.float64)
    q = int(p1.shape[-1])
    X = _xor_index(q)
    return np.einsum("...j,...ij->...i", p1, p2[..., X])


def normalize_at_zero(v):
    """Divide a Gamma-form vector by its value at z = 0: l -= l(0), s ^= s(0)."""
    s, l = v
    s = np.asarray(s)
    l = np.asarray(l, dtype=np.float64)
    return (s ^ s[..., :1]).astype(np.uint8), l - l[..., :1]
