"""Tanner-graph view of a non-binary LDPC code for the oracle (test infrastructure only).

Section 2: H = {h_cv} is an M x N matrix over GF(2^m); check c and variable v are adjacent iff
h_cv != 0; V_c is the set of variables of check c and C_v the set of checks of variable v.
The code is {x in GF(2^m)^N : Hx = 0}. The oracle accepts any column weight (degree-1 leaves
are needed for the cycle-free graphs on which belief propagation is exact, Section 2.1).

Built directly from the plain edge list (edge_check, edge_var, edge_h); shares nothing with the
C++ host code of the library.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .gf import GF


@dataclass
class OracleCode:
    N: int
    M: int
    m: int
    poly: int
    edge_check: np.ndarray
    edge_var: np.ndarray
    edge_h: np.ndarray
    gf: GF = field(init=False)
    V: list = field(init=False)  # V[c] = list of edge ids of check c, in edge-list order
    C: list = field(init=False)  # C[v] = list of edge ids of variable v, in edge-list order
    perm: np.ndarray = field(init=False)      # perm[e] = table z -> H_e z
    perm_inv: np.ndarray = field(init=False)  # perm_inv[e] = table z -> H_e^{-1} z

    def __post_init__(self):
        self.edge_check = np.asarray(self.edge_check, dtype=np.int64)
        self.edge_var = np.asarray(self.edge_var, dtype=np.int64)
        self.edge_h = np.asarray(self.edge_h, dtype=np.int64)
        self.gf = GF(self.m, self.poly)
        E = len(self.edge_check)
        if not (len(self.edge_var) == E == len(self.edge_h)):
            raise ValueError("edge arrays differ in length")
        if np.any(self.edge_h <= 0) or np.any(self.edge_h >= self.gf.q):
            raise ValueError("edge entries must be non-zero field elements")
        pairs = set()
        for c, v in zip(self.edge_check.tolist(), self.edge_var.tolist()):
            if (c, v) in pairs:
                raise ValueError("double edge")
            pairs.add((c, v))
        self.V = [[] for _ in range(self.M)]
        self.C = [[] for _ in range(self.N)]
        for e in range(E):
            self.V[int(self.edge_check[e])].append(e)
            self.C[int(self.edge_var[e])].append(e)
        maps = {}
        for h in np.unique(self.edge_h).tolist():
            maps[h] = (self.gf.fourier_index_map(h), self.gf.fourier_index_map_inverse(h))
        self.perm = np.stack([maps[int(h)][0] for h in self.edge_h]) if E else np.zeros((0, self.gf.q), np.int64)
        self.perm_inv = np.stack([maps[int(h)][1] for h in self.edge_h]) if E else np.zeros((0, self.gf.q), np.int64)

    @property
    def q(self) -> int:
        return self.gf.q

    @property
    def E(self) -> int:
        return len(self.edge_check)

    @classmethod
    def from_dict(cls, d: dict) -> "OracleCode":
        return cls(N=int(d["N"]), M=int(d["M"]), m=int(d["m"]), poly=int(d["poly"]),
                   edge_check=d["edge_check"], edge_var=d["edge_var"], edge_h=d["edge_h"])

    def dense_H(self) -> np.ndarray:
        H = np.zeros((self.M, self.N), dtype=np.int64)
        H[self.edge_check, self.edge_var] = self.edge_h
        return H

    def syndrome(self, x: np.ndarray) -> np.ndarray:
        """s_c = sum_{v in V_c} h_cv x_v over GF(2^m) (Section 3.1). x: (..., N) -> (..., M)."""
        x = np.asarray(x, dtype=np.int64)
        prod = self.gf.mul(self.edge_h, x[..., self.edge_var])  # (..., E)
        s = np.zeros(x.shape[:-1] + (self.M,), dtype=np.int64)
        for e in range(self.E):
            s[..., self.edge_check[e]] ^= prod[..., e]
        return s
