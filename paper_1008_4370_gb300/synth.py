"""Seeded synthetic workloads: Tanner graphs, codewords and BPSK/AWGN channel LLRs.

This module is the only code shared by the CUDA path's callers (tests, bench) and the FP64
oracle's callers. It holds none of the decoder's arithmetic: it draws graphs and field entries,
encodes random information symbols (with a small GF(2^m) table of its own, used for nothing
but encoding) and adds channel noise.

Code construction (not in the paper, which assumes a given (j=2, k)-regular H, Section 2):
socket permutation -- each variable node owns two sockets, the 2N sockets are shuffled and dealt
k at a time to the M = 2N/k check nodes; a draw that puts both sockets of a variable on one check
(a double edge) is rejected whole and redrawn. Non-zero entries h_cv are uniform over
GF(2^m) \\ {0}. Edges are listed check-major (edge e = c*k + slot).

Channel: symbol bit i-1 (coefficient of alpha^(i-1)) is sent as BPSK 0 -> +1, 1 -> -1 over AWGN
with sigma^2 = 1 / (2 R 10^(Eb/N0 / 10)), R = 1 - 2/k the design rate; the LLR
L = ln Pr(b=0|y)/Pr(b=1|y) = 2y/sigma^2 is returned as float32, laid out [frame][symbol][bit].
"""

from __future__ import annotations

import numpy as np

# primitive polynomials used by the workloads (bit j = coefficient of x^j)
PRIMITIVE_POLY = {2: 0x7, 3: 0xB, 4: 0x13, 5: 0x25, 6: 0x43, 7: 0x89, 8: 0x11D}


def rng_for(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(list(int(k) for k in key)))


def regular_code(N: int, k: int, m: int, poly: int | None = None, seed: int = 1,
                 max_draws: int = 1_000_000) -> dict:
    """Random (2, k)-regular code over GF(2^m) by socket permutation with double-edge rejection."""
    if (2 * N) % k:
        raise ValueError("2N must be a multiple of k")
    poly = PRIMITIVE_POLY[m] if poly is None else poly
    q = 1 << m
    M = 2 * N // k
    rng = rng_for(seed, N, k, m)
    sockets = np.repeat(np.arange(N, dtype=np.int32), 2)
    for _ in range(max_draws):
        checks = rng.permutation(sockets).reshape(M, k)
        srt = np.sort(checks, axis=1)
        if not np.any(srt[:, 1:] == srt[:, :-1]):
            break
    else:
        raise RuntimeError("no simple graph found")
    E = M * k
    return {
        "N": N, "M": M, "k": k, "m": m, "poly": poly,
        "edge_check": np.repeat(np.arange(M, dtype=np.int32), k),
        "edge_var": checks.reshape(-1).astype(np.int32),
        "edge_h": rng.integers(1, q, size=E).astype(np.uint16),
    }


def tree_code(n_checks: int, k: int, m: int, poly: int | None = None, seed: int = 1) -> dict:
    """Cycle-free Tanner graph: check c > 0 shares exactly one degree-1 variable with the
    checks before it and adds k-1 new variables. Variable degrees are 1 or 2."""
    poly = PRIMITIVE_POLY[m] if poly is None else poly
    q = 1 << m
    rng = rng_for(seed, n_checks, k, m, 7)
    edge_check, edge_var = [], []
    deg = []
    for c in range(n_checks):
        vs = []
        if c > 0:
            leaves = [v for v, d in enumerate(deg) if d == 1]
            shared = int(rng.choice(leaves))
            vs.append(shared)
            deg[shared] += 1
        while len(vs) < k:
            vs.append(len(deg))
            deg.append(1)
        for v in vs:
            edge_check.append(c)
            edge_var.append(v)
    E = len(edge_check)
    return {
        "N": len(deg), "M": n_checks, "k": k, "m": m, "poly": poly,
        "edge_check": np.array(edge_check, dtype=np.int32),
        "edge_var": np.array(edge_var, dtype=np.int32),
        "edge_h": rng.integers(1, q, size=E).astype(np.uint16),
    }


class _EncoderField:
    """Multiplication / inverse tables of GF(2^m), for the encoder only."""

    def __init__(self, m: int, poly: int):
        q = 1 << m
        exp = np.zeros(2 * q, dtype=np.int64)
        log = np.zeros(q, dtype=np.int64)
        x = 1
        for i in range(q - 1):
            exp[i] = x
            log[x] = i
            x <<= 1
            if x & q:
                x ^= poly
        exp[q - 1:2 * q - 2] = exp[:q - 1]
        a = np.arange(q)
        la, lb = np.meshgrid(log, log, indexing="ij")
        mul = exp[(la + lb) % (q - 1)]
        mul[0, :] = 0
        mul[:, 0] = 0
        self.mul = mul
        self.inv = np.zeros(q, dtype=np.int64)
        self.inv[1:] = exp[(q - 1 - log[a[1:]]) % (q - 1)]


class Encoder:
    """Codewords of {x : Hx = 0} from the reduced row-echelon form of H (Gaussian elimination
    over GF(2^m), column pivoting; rank-deficient H is handled: pivot columns are parity)."""

    def __init__(self, code: dict):
        m, poly = int(code["m"]), int(code["poly"])
        N, M = int(code["N"]), int(code["M"])
        F = _EncoderField(m, poly)
        H = np.zeros((M, N), dtype=np.int64)
        H[np.asarray(code["edge_check"]), np.asarray(code["edge_var"])] = np.asarray(code["edge_h"])
        rank = 0
        pivots = []
        for col in range(N):
            if rank == M:
                break
            nz = np.nonzero(H[rank:, col])[0]
            if len(nz) == 0:
                continue
            r = rank + int(nz[0])
            if r != rank:
                H[[rank, r]] = H[[r, rank]]
            H[rank] = F.mul[F.inv[H[rank, col]], H[rank]]
            rows = np.nonzero(H[:, col])[0]
            rows = rows[rows != rank]
            if len(rows):
                H[rows] ^= F.mul[H[rows, col][:, None], H[rank][None, :]]
            pivots.append(col)
            rank += 1
        self.field = F
        self.rank = rank
        self.pivots = np.array(pivots, dtype=np.int64)
        self.free = np.setdiff1d(np.arange(N), self.pivots)
        self.A = H[:rank][:, self.free]  # x_pivot[r] = sum_j A[r, j] x_free[j]  (char 2)
        self.N = N
        self.m = m

    @property
    def info_symbols(self) -> int:
        return self.N - self.rank

    def encode(self, info: np.ndarray) -> np.ndarray:
        info = np.asarray(info, dtype=np.int64)
        F = info.shape[0]
        x = np.zeros((F, self.N), dtype=np.int64)
        x[:, self.free] = info
        step = max(1, (1 << 24) // max(1, self.A.size))
        for i in range(0, F, step):
            prod = self.field.mul[self.A[None, :, :], info[i:i + step, None, :]]
            x[i:i + step][:, self.pivots] = np.bitwise_xor.reduce(prod, axis=2) if prod.shape[2] else 0
        return x

    def random_codewords(self, n: int, rng: np.random.Generator) -> np.ndarray:
        q = 1 << self.m
        return self.encode(rng.integers(0, q, size=(n, self.info_symbols)))


def design_rate(k: int) -> float:
    return 1.0 - 2.0 / k


def bpsk_awgn_llr(codewords: np.ndarray, m: int, ebn0_db, rate: float,
                  rng: np.random.Generator) -> np.ndarray:
    """LLRs (F, N, m) float32 for the given codewords; ebn0_db scalar or per-frame (F,)."""
    x = np.asarray(codewords, dtype=np.int64)
    bits = (x[..., None] >> np.arange(m)) & 1
    s = 1.0 - 2.0 * bits
    ebn0 = np.asarray(ebn0_db, dtype=np.float64)
    sigma2 = 1.0 / (2.0 * rate * 10.0 ** (ebn0 / 10.0))
    if sigma2.ndim == 1:
        sigma2 = sigma2[:, None, None]
    y = s + np.sqrt(sigma2) * rng.standard_normal(s.shape)
    return (2.0 * y / sigma2).astype(np.float32)


# Named workloads: (field m, N, k, code seed). Code seeds are fixed per code.
CODES = {
    "gf16_n32_k4": (4, 32, 4, 1),
    "gf64_n1200_k6": (6, 1200, 6, 2),
    "gf256_n512_k4": (8, 512, 4, 3),
    "gf16_n96_k4": (4, 96, 4, 4),
    "gf64_n4096_k8": (6, 4096, 8, 5),
    "gf256_n2048_k16": (8, 2048, 16, 6),
    "gf4_n8_k4": (2, 8, 4, 7),
}


def named_code(name: str) -> dict:
    m, N, k, seed = CODES[name]
    c = regular_code(N, k, m, seed=seed)
    c["name"] = name
    c["seed"] = seed
    return c


def frames(code: dict, n_frames: int, ebn0_db, *, snr_idx: int = 0, batch_idx: int = 0,
           zero_codeword: bool = False, encoder: Encoder | None = None):
    """(codewords (F, N) int64, llr (F, N, m) float32) for a code; noise seeded by
    PCG64([code seed, snr_idx, batch_idx])."""
    rng = rng_for(int(code.get("seed", 0)), snr_idx, batch_idx)
    if zero_codeword:
        cw = np.zeros((n_frames, int(code["N"])), dtype=np.int64)
    else:
        enc = encoder if encoder is not None else Encoder(code)
        cw = enc.random_codewords(n_frames, rng)
    llr = bpsk_awgn_llr(cw, int(code["m"]), ebn0_db, design_rate(int(code["k"])), rng)
    return cw, llr
