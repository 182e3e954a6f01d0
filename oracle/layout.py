"""Register layout and the embedding of physics indices into the qubit register.

Test infrastructure only.  Registers, little-endian from bit 0: t, s, iL, q1,
a1, then (N_C = 2) q2, a2, ord, then k and m.  A basis state is physical when
t, s and iL are 0, every velocity is at most 2 and, for N_C = 2 and ord = 0,
q2 = a2 = 0.  The register sizes follow
the paper: n_alpha = ceil(log2 Nx) (Sec. II.D.2), n_k = ceil(log2(K+1)),
n_m = ceil(log2(Nt)+1), n_i^L = max(1 + n_i^A, 2 + n_k) (Sec. II.D.4), and the
I/O qubit count reproduces Table qubit-count (plus one signal qubit).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import physics as P


@dataclass
class Layout:
    Nx: int
    NC: int
    K: int
    Nt: int
    na: int = field(init=False)
    nk: int = field(init=False)
    nm: int = field(init=False)
    niA: int = field(init=False)
    niL: int = field(init=False)
    regs: dict = field(init=False)
    n: int = field(init=False)

    def __post_init__(self):
        if self.Nx < 2 or self.Nx & (self.Nx - 1):
            raise ValueError("Nx must be a power of two >= 2")
        if self.NC not in (1, 2) or self.K < 1 or self.Nt < 1:
            raise ValueError("bad parameters")
        self.na = P.n_alpha(self.Nx)
        self.nk = P.n_k_bits(self.K)
        self.nm = P.n_m_bits(self.Nt)
        self.niA = 2 if self.NC == 1 else 4
        self.niL = max(1 + self.niA, 2 + self.nk)
        order = [("t", 1), ("s", 1), ("iL", self.niL), ("q1", 2), ("a1", self.na)]
        if self.NC == 2:
            order += [("q2", 2), ("a2", self.na), ("ord", 1)]
        order += [("k", self.nk), ("m", self.nm)]
        pos = 0
        self.regs = {}
        for name, w in order:
            self.regs[name] = list(range(pos, pos + w))
            pos += w
        self.n = pos
        iL = self.regs["iL"]
        self.regs["i"] = iL[0:2]
        if self.NC == 2:
            self.regs["case"] = iL[2:4]
        self.regs["e"] = iL[self.niA:]
        self.regs["l"] = iL[0:self.nk]
        self.regs["unused"] = iL[self.nk:self.niL - 2]
        self.regs["km"] = self.regs["k"] + self.regs["m"]
        self.top = iL[self.niL - 1]
        self.sel = iL[self.niL - 2]

    # ------------------------------------------------------------- helpers
    def bits(self, name):
        return self.regs[name]

    def field_value(self, index: int, name: str) -> int:
        v = 0
        for j, b in enumerate(self.regs[name]):
            v |= ((index >> b) & 1) << j
        return v

    def place(self, **values) -> int:
        """Register values -> basis index."""
        idx = 0
        for name, v in values.items():
            bits = self.regs[name]
            if v >> len(bits):
                raise ValueError(f"{name}={v} does not fit")
            for j, b in enumerate(bits):
                idx |= ((v >> j) & 1) << b
        return idx

    def carleman_dim(self) -> int:
        n1 = 3 * self.Nx
        return n1 if self.NC == 1 else n1 + n1 * n1

    def n_slots(self) -> int:
        return 1 << (self.nk + self.nm)

    def embed_index(self, slot: int, j: int) -> int:
        """(slot (m,k), physics index j) -> basis index with t = s = iL = 0."""
        m, k = slot >> self.nk, slot & ((1 << self.nk) - 1)
        n1 = 3 * self.Nx
        if j < n1:
            a, q = divmod(j, 3)
            if self.NC == 1:
                return self.place(a1=a, q1=q, k=k, m=m)
            return self.place(a1=a, q1=q, a2=0, q2=0, ord=0, k=k, m=m)
        p1, p2 = divmod(j - n1, n1)
        a1, q1 = divmod(p1, 3)
        a2, q2 = divmod(p2, 3)
        return self.place(a1=a1, q1=q1, a2=a2, q2=q2, ord=1, k=k, m=m)

    def physical_indices(self) -> np.ndarray:
        """Basis index of every physical (slot, j), ordered like L's rows."""
        D = self.carleman_dim()
        out = np.empty(self.n_slots() * D, dtype=np.int64)
        for s in range(self.n_slots()):
            for j in range(D):
                out[s * D + j] = self.embed_index(s, j)
        return out

    def system_bits(self):
        """Qubits of the system register (everything except t, s and iL)."""
        anc = set(self.regs["t"] + self.regs["s"] + self.regs["iL"])
        return [b for b in range(self.n) if b not in anc]
