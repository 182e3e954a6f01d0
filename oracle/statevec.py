"""O2 -- naive FP64 state-vector simulation, plus dense and sparse brute force.

Test infrastructure only.  Three independent ways to apply a gate list:

* ``DenseSim``     -- one vectorised NumPy pass per elementary gate over a
                      complex128 state (the "naive simulator"), with an
                      optional norm check after every gate.
* ``gate_unitary`` -- the full 2^n x 2^n matrix of one gate, written out column
                      by column from the gate's definition (n <= 10).
* ``AxisSim``      -- the same gate semantics on the state seen as an n-axis
                      tensor of 2 x ... x 2: the controls select a sub-tensor
                      by basic indexing, the 2x2 matrix acts along the
                      target's axis (for states of 20-26 qubits, where the
                      index tables of ``DenseSim`` become too large).
* ``SparseColumns``-- exact simulation of many basis-state inputs at once,
                      storing only non-zero amplitudes (used for the
                      block-encoding sweep of App. B).

Gate semantics: the 2x2 matrix G acts on the target
qubit of every basis pair whose index satisfies (index & cmask) == cval.
"""
from __future__ import annotations

import math

import numpy as np

OP_X, OP_H, OP_RY, OP_ZPHASE = 0, 1, 2, 3
_S = 1.0 / math.sqrt(2.0)


def gate_2x2(op: int, angle: float) -> np.ndarray:
    if op == OP_X:
        return np.array([[0, 1], [1, 0]], dtype=np.complex128)
    if op == OP_H:
        return np.array([[_S, _S], [_S, -_S]], dtype=np.complex128)
    if op == OP_RY:
        c, s = math.cos(angle / 2.0), math.sin(angle / 2.0)
        return np.array([[c, -s], [s, c]], dtype=np.complex128)
    if op == OP_ZPHASE:
        return np.array([[complex(math.cos(angle), math.sin(angle)), 0],
                         [0, complex(math.cos(angle), -math.sin(angle))]], dtype=np.complex128)
    raise ValueError(op)


class DenseSim:
    """Naive gate-by-gate simulator on a dense complex128 vector of 2^n amplitudes."""

    def __init__(self, n: int, check_norm: bool = False, norm_tol: float = 1e-13):
        self.n = n
        self.check_norm = check_norm
        self.norm_tol = norm_tol
        self._cache = {}

    def _pairs(self, target, cmask, cval):
        key = (target, cmask, cval)
        hit = self._cache.get(key)
        if hit is None:
            idx = np.arange(1 << self.n, dtype=np.int64)
            sel = ((idx & cmask) == cval) & (((idx >> target) & 1) == 0)
            i0 = idx[sel]
            hit = (i0, i0 | (1 << target))
            if len(self._cache) > 4096:
                self._cache.clear()
            self._cache[key] = hit
        return hit

    def apply(self, psi: np.ndarray, gate) -> None:
        op, t, cm, cv, ang = gate[0], gate[1], gate[2], gate[3], gate[4]
        i0, i1 = self._pairs(t, cm, cv)
        a = psi[i0]
        b = psi[i1]
        if op == OP_X:
            psi[i0] = b
            psi[i1] = a
        elif op == OP_H:
            psi[i0] = (a + b) * _S
            psi[i1] = (a - b) * _S
        elif op == OP_RY:
            c, s = math.cos(ang / 2.0), math.sin(ang / 2.0)
            psi[i0] = c * a - s * b
            psi[i1] = s * a + c * b
        elif op == OP_ZPHASE:
            psi[i0] = a * complex(math.cos(ang), math.sin(ang))
            psi[i1] = b * complex(math.cos(ang), -math.sin(ang))
        else:
            raise ValueError(op)

    def run(self, psi: np.ndarray, gates) -> np.ndarray:
        for g in gates:
            self.apply(psi, g)
            if self.check_norm:
                nrm = float(np.vdot(psi, psi).real)
                if abs(1.0 - nrm) >= self.norm_tol:
                    raise AssertionError(f"norm drifted to {nrm!r} after gate {g}")
        return psi


class AxisSim:
    """Gate-by-gate simulator on the state viewed as a tensor with one axis
    per qubit (axis n-1-q holds qubit q, since index bit q has stride 2^q).

    For a gate with target t and controls (cmask, cval): index every control
    axis with its required value and keep the others whole (a view of the
    sub-tensor where the controls hold), split that view along the target
    axis into the halves a, b with the target 0 and 1, and write back
    G[0,0] a + G[0,1] b and G[1,0] a + G[1,1] b.  The sub-tensor is cut
    along up to three further axes into independent pieces, which a few
    threads update at once (NumPy releases the GIL inside its loops)."""

    def __init__(self, n: int, threads: int = 0):
        import os
        self.n = n
        self.threads = threads or min(8, os.cpu_count() or 1)
        self._pool = None

    @staticmethod
    def _update(a, b, op, G):
        if op == OP_ZPHASE:  # diagonal
            a *= G[0, 0]
            b *= G[1, 1]
            return
        a0 = a.copy()
        if op == OP_X:
            a[...] = b
            b[...] = a0
            return
        a *= G[0, 0]
        a += G[0, 1] * b
        b *= G[1, 1]
        b += G[1, 0] * a0

    def apply(self, psi: np.ndarray, gate) -> None:
        op, t, cm, cv, ang = gate[0], gate[1], gate[2], gate[3], gate[4]
        n = self.n
        sel = [slice(None)] * n
        for q in range(n):
            if (cm >> q) & 1:
                sel[n - 1 - q] = (cv >> q) & 1
        # free axes (neither control nor target) cut the work into pieces
        free = [n - 1 - q for q in range(n) if q != t and not (cm >> q) & 1][:3]
        if (1 << n) >> bin(cm).count("1") < (1 << 16):
            free = []
        G = gate_2x2(op, ang)
        T = psi.reshape((2,) * n)
        jobs = []
        for k in range(1 << len(free)):
            s = list(sel)
            for j, axis in enumerate(free):
                s[axis] = (k >> j) & 1
            s0, s1 = list(s), list(s)
            s0[n - 1 - t] = 0
            s1[n - 1 - t] = 1
            jobs.append((T[tuple(s0)], T[tuple(s1)]))  # views into the state
        if len(jobs) == 1 or self.threads == 1:
            for a, b in jobs:
                self._update(a, b, op, G)
            return
        if self._pool is None:
            from concurrent.futures import ThreadPoolExecutor
            self._pool = ThreadPoolExecutor(self.threads)
        list(self._pool.map(lambda ab: self._update(ab[0], ab[1], op, G), jobs))

    def run(self, psi: np.ndarray, gates) -> np.ndarray:
        if not psi.flags.c_contiguous:
            raise ValueError("AxisSim needs a contiguous state")
        for g in gates:
            self.apply(psi, g)
        return psi


def gate_unitary(gate, n: int) -> np.ndarray:
    """Dense unitary of one gate, built column by column (brute force, n <= 10)."""
    if n > 10:
        raise ValueError("brute force only up to 10 qubits")
    op, t, cm, cv, ang = gate[0], gate[1], gate[2], gate[3], gate[4]
    G = gate_2x2(op, ang)
    N = 1 << n
    U = np.zeros((N, N), dtype=np.complex128)
    for col in range(N):
        if (col & cm) == cv:
            b = (col >> t) & 1
            base = col & ~(1 << t)
            U[base, col] += G[0, b]
            U[base | (1 << t), col] += G[1, b]
        else:
            U[col, col] = 1.0
    return U


def circuit_unitary(gates, n: int) -> np.ndarray:
    U = np.eye(1 << n, dtype=np.complex128)
    for g in gates:
        U = gate_unitary(g, n) @ U
    return U


class SparseColumns:
    """Simulate many basis-state inputs at once, keeping only non-zero entries.

    State: arrays (col, key, amp); entry means amplitude ``amp`` on basis
    ``key`` of the output column ``col``.
    """

    def __init__(self, n: int, inputs: np.ndarray):
        self.n = n
        inputs = np.asarray(inputs, dtype=np.int64)
        self.col = np.arange(inputs.shape[0], dtype=np.int64)
        self.key = inputs.copy()
        self.amp = np.ones(inputs.shape[0], dtype=np.complex128)

    def apply(self, gate) -> None:
        op, t, cm, cv, ang = gate[0], gate[1], gate[2], gate[3], gate[4]
        hit = (self.key & cm) == cv
        if op == OP_X:
            self.key = np.where(hit, self.key ^ (1 << t), self.key)
            return
        G = gate_2x2(op, ang)
        if not hit.any():
            return
        kc, cc, ac = self.key[hit], self.col[hit], self.amp[hit]
        bit = (kc >> t) & 1
        base = kc & ~(1 << t)
        new_key = np.concatenate([self.key[~hit], base, base | (1 << t)])
        new_col = np.concatenate([self.col[~hit], cc, cc])
        new_amp = np.concatenate([self.amp[~hit], G[0, bit] * ac, G[1, bit] * ac])
        comb = new_col * (1 << self.n) + new_key
        uniq, inv = np.unique(comb, return_inverse=True)
        re = np.bincount(inv, weights=new_amp.real, minlength=uniq.shape[0])
        im = np.bincount(inv, weights=new_amp.imag, minlength=uniq.shape[0])
        amp = re + 1j * im
        keep = amp != 0
        self.col = (uniq >> self.n)[keep]
        self.key = (uniq & ((1 << self.n) - 1))[keep]
        self.amp = amp[keep]

    def run(self, gates):
        for g in gates:
            self.apply(g)
        return self
