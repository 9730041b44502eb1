"""GF(2^m) arithmetic for the FP64 oracle (test infrastructure only).

Representation (Section 2, the GF(8) example with alpha^3 + alpha + 1 = 0): a symbol is an
m-bit vector whose coordinate i (i = 1..m) is the coefficient of alpha^(i-1). As an integer,
coordinate i is bit i-1, so 1 = 0b001, alpha = 0b010, alpha^2 = 0b100, alpha^3 = 0b011 for GF(8).

Appendix A: the companion matrix A of the primitive polynomial
pi(x) = pi_0 + pi_1 x + ... + pi_{m-1} x^{m-1} + x^m has ones on the sub-diagonal and the
column (pi_0, ..., pi_{m-1}) as its last column; A^i alpha^j = alpha^{i+j} on column bit
vectors. For h = alpha^i the paper defines H_cv = (A^i)^T, and the Fourier-domain messages are
re-indexed as P(H_cv z) (Section 3.1, check-to-variable step; proof in Appendix A).

Pinned by: the printed GF(8) table, A^i alpha^j = alpha^{i+j} against an independent bit-serial
carry-less multiply, multiplicative order q-1 for the five polynomials used, and the Fourier
permutation identity of Appendix A (tests/test_oracle_gf.py).
"""

from __future__ import annotations

import numpy as np


def clmul_mod(a: int, b: int, poly: int, m: int) -> int:
    """Product a*b in GF(2)[x] / poly(x), by shift-and-add over the bits of b.

    Used as the library-free brute-force multiplication against which the tables are pinned.
    """
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if (a >> m) & 1:
            a ^= poly
    return r


class GF:
    """GF(2^m) defined by a primitive polynomial given as an integer (bit j = coeff of x^j)."""

    def __init__(self, m: int, poly: int):
        if not (1 <= m <= 16):
            raise ValueError("m out of range")
        if poly.bit_length() - 1 != m:
            raise ValueError(f"polynomial 0x{poly:x} is not of degree {m}")
        self.m = m
        self.q = q = 1 << m
        self.poly = poly
        exp = np.zeros(2 * q, dtype=np.int64)
        log = np.full(q, -1, dtype=np.int64)
        x = 1
        for i in range(q - 1):
            if log[x] != -1:
                raise ValueError(f"polynomial 0x{poly:x} is not primitive")
            exp[i] = x
            log[x] = i
            x <<= 1
            if x & q:
                x ^= poly
        if x != 1:
            raise ValueError(f"polynomial 0x{poly:x} is not primitive")
        exp[q - 1:2 * (q - 1)] = exp[0:q - 1]
        self.exp = exp
        self.log = log

    # --- scalar / vector field operations -----------------------------------------------
    def mul(self, a, b):
        a = np.asarray(a, dtype=np.int64)
        b = np.asarray(b, dtype=np.int64)
        nz = (a != 0) & (b != 0)
        la = np.where(nz, self.log[np.where(a == 0, 1, a)], 0)
        lb = np.where(nz, self.log[np.where(b == 0, 1, b)], 0)
        return np.where(nz, self.exp[(la + lb) % (self.q - 1)], 0)

    def inv(self, a):
        a = np.asarray(a, dtype=np.int64)
        if np.any(a == 0):
            raise ZeroDivisionError("inverse of 0 in GF(2^m)")
        return self.exp[(self.q - 1 - self.log[a]) % (self.q - 1)]

    def alpha_pow(self, i: int) -> int:
        return int(self.exp[i % (self.q - 1)])

    # --- bit-vector views (coordinate i <-> bit i-1) ------------------------------------
    def to_bits(self, x):
        """Column bit vectors: x (...,) -> (..., m) with [..., i-1] = coefficient of alpha^(i-1)."""
        x = np.asarray(x, dtype=np.int64)
        return ((x[..., None] >> np.arange(self.m)) & 1).astype(np.int64)

    def from_bits(self, bits):
        bits = np.asarray(bits, dtype=np.int64) & 1
        return (bits << np.arange(self.m)).sum(axis=-1)

    # --- Appendix A ----------------------------------------------------------------------
    def companion(self) -> np.ndarray:
        """Companion matrix A (m x m over GF(2)) exactly as printed in Appendix A."""
        m = self.m
        A = np.zeros((m, m), dtype=np.int64)
        for r in range(1, m):
            A[r, r - 1] = 1
        for r in range(m):
            A[r, m - 1] = (self.poly >> r) & 1
        return A

    @staticmethod
    def _matmul2(X, Y):
        return (X @ Y) & 1

    def companion_power(self, i: int) -> np.ndarray:
        """A^i over GF(2) (i >= 0), by repeated multiplication."""
        A = self.companion()
        R = np.eye(self.m, dtype=np.int64)
        for _ in range(i % (self.q - 1)):
            R = self._matmul2(A, R)
        return R

    def H_matrix(self, h: int) -> np.ndarray:
        """H_cv = (A^i)^T for h_cv = alpha^i (Appendix A definition)."""
        if h == 0:
            raise ValueError("H_cv is defined for non-zero entries only")
        return self.companion_power(int(self.log[h])).T.copy()

    def fourier_index_map(self, h: int) -> np.ndarray:
        """Table z -> H_cv z for all z in GF(2^m) (the index map of the check-node step).

        Computed as a GF(2) matrix-vector product with the Appendix A matrix.
        """
        H = self.H_matrix(h)
        zs = np.arange(self.q)
        zb = self.to_bits(zs)  # (q, m)
        return self.from_bits((zb @ H.T) & 1)

    def fourier_index_map_inverse(self, h: int) -> np.ndarray:
        """Table z -> H_cv^{-1} z, as the inverse of the bijection fourier_index_map(h)."""
        fwd = self.fourier_index_map(h)
        inv = np.empty_like(fwd)
        inv[fwd] = np.arange(self.q)
        return inv
