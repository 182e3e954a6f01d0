"""O3 -- the oracle's own gate compiler (U_A inside U_L, QSVT wrapper, mask).

Test infrastructure only.  Written independently of the product's compiler,
in plain Python, from the same gate-level construction (registers as in
``layout.py``; U_A as one permutation of site, velocity and label followed by
the RY value encodings on t).  The construction realises, with multi-controlled elementary gates
and no work ancillas, the sparse-oracle block encoding of Eq. UM-structure
(Sec. II.D.1) for the Carleman matrix of Eq. carleman-system and the Taylor
matrix L of Fig. L (Sec. II.D.4), wrapped in the QSVT sequence of
Fig. circuit-qsvt with Hadamards on the signal qubit (reading R13).

A gate is a tuple ``(op, target, cmask, cval, angle, tag)`` with Python ints
and a Python float; op 0=X, 1=H, 2=RY, 3=ZPHASE (e^{i phi Z}).
"""
from __future__ import annotations

import math

from . import physics as P
from .layout import Layout

OP_X, OP_H, OP_RY, OP_ZPHASE = 0, 1, 2, 3
TAG_HPREP, TAG_PERM, TAG_VALUE, TAG_HUNPREP, TAG_TFLIP, TAG_PHASE, TAG_SIGNAL = 1, 2, 3, 4, 5, 6, 7


def _ctrl(*parts):
    """Merge control specs given as dicts {qubit: value}."""
    out = {}
    for p in parts:
        for b, v in p.items():
            if b in out and out[b] != v:
                raise ValueError("conflicting controls")
            out[b] = v
    return out


def _reg_eq(bits, value):
    """Control spec: register `bits` (LSB first) equals `value`."""
    return {b: (value >> j) & 1 for j, b in enumerate(bits)}


def _mask(ctrl):
    cmask = 0
    cval = 0
    for b, v in ctrl.items():
        cmask |= 1 << b
        cval |= (v & 1) << b
    return cmask, cval


def _gate(op, target, ctrl=None, angle=0.0, tag=0):
    ctrl = ctrl or {}
    if target in ctrl:
        raise ValueError("target used as control")
    cmask, cval = _mask(ctrl)
    return (op, target, cmask, cval, float(angle), tag)


def prefix_patterns(lo, hi, w):
    """Aligned dyadic cover of [lo, hi) over a w-bit register: list of (value>>j, j)."""
    out = []
    while lo < hi:
        j = 0
        while j < w and lo % (1 << (j + 1)) == 0 and lo + (1 << (j + 1)) <= hi:
            j += 1
        out.append((lo >> j, j))
        lo += 1 << j
    return out


def _pattern_ctrl(bits, pat):
    hi_val, j = pat
    return {b: (hi_val >> (idx - j)) & 1 for idx, b in enumerate(bits) if idx >= j}


def _inc(bits, ctrl, tag):
    g = []
    for j in range(len(bits) - 1, -1, -1):
        c = _ctrl(ctrl, {b: 1 for b in bits[:j]})
        g.append(_gate(OP_X, bits[j], c, tag=tag))
    return g


def _dec(bits, ctrl, tag):
    g = []
    for j in range(len(bits) - 1, -1, -1):
        c = _ctrl(ctrl, {b: 0 for b in bits[:j]})
        g.append(_gate(OP_X, bits[j], c, tag=tag))
    return g


def _bounce(a, v, X, tag):
    """Bounce-back fix-up after periodic streaming of the site register `a` by
    the velocity register `v` (value 0: e=+1, 1: e=-1).  Periodic streaming
    leaves the populations that left the lattice at (a=0, v=0) (from the right
    wall) and (a=Nx-1, v=1) (from the left wall); exchanging these two
    patterns returns each to its own site with the opposite velocity (the wall
    rule of reading R2).  The exchange: flip a where v=1, flip v where a=0,
    flip a where v=1 again (all with v's high bit 0)."""
    v0, v1 = v
    base = _ctrl(X, {v1: 0})
    g = [_gate(OP_X, b, _ctrl(base, {v0: 1}), tag=tag) for b in a]
    g.append(_gate(OP_X, v0, _ctrl(base, {b: 0 for b in a}), tag=tag))
    g += [_gate(OP_X, b, _ctrl(base, {v0: 1}), tag=tag) for b in a]
    return g


def _p11(a, q, i, X, tag, bc="periodic"):
    """Collide-then-stream index map of Eq. A11-elements on (a, q) with label i."""
    q0, q1 = q
    i0, i1 = i
    g = []
    g += _inc(a, _ctrl(X, _reg_eq(i, 0)), tag)
    g += _dec(a, _ctrl(X, _reg_eq(i, 1)), tag)
    if bc == "bounceback":
        g += _bounce(a, i, X, tag)
    # T1: (q,i) = (0,1) <-> (1,0)
    g.append(_gate(OP_X, q0, _ctrl(X, {i0: 1}), tag=tag))
    g.append(_gate(OP_X, i0, _ctrl(X, {q0: 1, q1: 0, i1: 0}), tag=tag))
    g.append(_gate(OP_X, q0, _ctrl(X, {i0: 1}), tag=tag))
    # T2: (0,2) <-> (2,0)
    g.append(_gate(OP_X, q1, _ctrl(X, {i1: 1}), tag=tag))
    g.append(_gate(OP_X, i1, _ctrl(X, {q1: 1, q0: 0, i0: 0}), tag=tag))
    g.append(_gate(OP_X, q1, _ctrl(X, {i1: 1}), tag=tag))
    # T3: (1,2) <-> (2,1)
    for tgt in (q1, i0, i1):
        g.append(_gate(OP_X, tgt, _ctrl(X, {q0: 1}), tag=tag))
    g.append(_gate(OP_X, q0, _ctrl(X, {q1: 1, i0: 1, i1: 0}), tag=tag))
    for tgt in (q1, i0, i1):
        g.append(_gate(OP_X, tgt, _ctrl(X, {q0: 1}), tag=tag))
    return g


def _pi3(lay: Layout, X, tag, bc="periodic"):
    """A12 branch (Eq. A12-elements): a2 <- a2 - a1, label bookkeeping, stream, ord flip."""
    r = lay.regs
    a1, a2, q1, q2, i = r["a1"], r["a2"], r["q1"], r["q2"], r["i"]
    g = []
    for j in range(lay.na):
        g += _dec(a2[j:], _ctrl(X, {a1[j]: 1}), tag)
    for b in range(2):
        g.append(_gate(OP_X, q1[b], _ctrl(X, {i[b]: 1}), tag=tag))
        g.append(_gate(OP_X, i[b], _ctrl(X, {q1[b]: 1}), tag=tag))
        g.append(_gate(OP_X, q1[b], _ctrl(X, {i[b]: 1}), tag=tag))
    g.append(_gate(OP_X, i[1], _ctrl(X, {q2[0]: 1}), tag=tag))
    g.append(_gate(OP_X, q2[0], _ctrl(X, {i[1]: 1}), tag=tag))
    g.append(_gate(OP_X, i[1], _ctrl(X, {q2[0]: 1}), tag=tag))
    g += _inc(a1, _ctrl(X, _reg_eq(q1, 0)), tag)
    g += _dec(a1, _ctrl(X, _reg_eq(q1, 1)), tag)
    if bc == "bounceback":
        g += _bounce(a1, q1, X, tag)
    g.append(_gate(OP_X, r["ord"][0], X, tag=tag))
    return g


# ----------------------------------------------------------- value tables
def v11(qo, io, tau):
    """Value encoded for A11 at output (q'=qo, stored input velocity io)."""
    if qo <= 2 and io <= 2:
        v = P.collision_coeff(qo, io, tau)
        if qo == 2 and io == 2:
            v = v - 1.0
        return v
    if qo <= 1 and io == 3:
        return -1.0
    return 0.0


def max_abs_A(tau, NC, bc="periodic"):
    """max |A_ij| of the assembled Carleman matrix, from its distinct entries.
    Bounce-back walls add one diagonal entry per wall, c(q', qbar') - 1 (the
    bounced coefficient lands on the same row and column as the -1 of the
    A11 diagonal), and its sums with the second copy's diagonal in A22."""
    vals = []
    for qp in range(3):
        for q in range(3):
            if (qp, q) != (2, 2):
                vals.append(P.collision_coeff(qp, q, tau))
    c22m1 = P.collision_coeff(2, 2, tau) - 1.0
    vals += [c22m1, -1.0]
    if NC == 2:
        for qp in range(3):
            for q1 in range(3):
                for q2 in range(3):
                    vals.append(P.k12(qp, q1, q2, tau))
        vals += [-1.0 + -1.0, -1.0 + c22m1, c22m1 + c22m1]
    if bc == "bounceback":
        walls = [P.collision_coeff(0, 1, tau) - 1.0, P.collision_coeff(1, 0, tau) - 1.0]
        vals += walls
        if NC == 2:
            for w in walls:
                vals += [w + -1.0, w + c22m1]
                vals += [w + w2 for w2 in walls]
    return max(abs(v) for v in vals)


def lmax_value(tau, NC, dt, bc="periodic"):
    return max(1.0, dt * max_abs_A(tau, NC, bc))


def _theta(v, ko, dt, Lmax):
    return 2.0 * math.asin((((-dt) * v) / (ko + 1.0)) / Lmax)


def _theta0(v, ko, dt, Lmax):
    return _theta(v, ko, dt, Lmax) if v != 0.0 else 0.0


def _wall(lay: Layout, areg, qo):
    """Site value of the wall whose bounced population lands on output
    velocity qo: qo = 1 at the right wall (a = Nx-1), qo = 0 at the left (a = 0)."""
    return _reg_eq(areg, lay.Nx - 1 if qo == 1 else 0)


def _wall_fix(lay, base, areg, qreg, vfun, ios, ko, dt, Lmax, t):
    """Bounce-back value corrections: an output (qo, io) at its wall site
    carries the entry of the opposite velocity, v(1-qo, io), instead of
    v(qo, io); a second RY on t adds the angle difference there."""
    g = []
    for qo in (0, 1):
        for io in ios:
            tw = _theta0(vfun(1 - qo, io), ko, dt, Lmax)
            tg = _theta0(vfun(qo, io), ko, dt, Lmax)
            if tw != tg:
                c = _ctrl(base, _reg_eq(qreg, qo), _wall(lay, areg, qo))
                g.append(_gate(OP_RY, t, _ctrl(c, ios[io]), tw - tg, TAG_VALUE))
    return g


# -------------------------------------------------------------------- U_L
def build_UL(Nx, tau, NC, K, dt, Nt, bc="periodic"):
    """Gate list of U_L in time order (Fig. L's block structure); bc "periodic" or
    "bounceback" (reading R2)."""
    if bc not in ("periodic", "bounceback"):
        raise ValueError(bc)
    lay = Layout(Nx, NC, K, Nt)
    r = lay.regs
    Lmax = lmax_value(tau, NC, dt, bc)
    t = r["t"][0]
    T = {b: 0 for b in r["e"]}
    C = {lay.top: 1, lay.sel: 0}
    g = []
    for b in r["iL"]:
        g.append(_gate(OP_H, b, tag=TAG_HPREP))
    # ---- permutation
    if NC == 2:
        cs, od = r["case"], r["ord"][0]
        g += _p11(r["a1"], r["q1"], r["i"], _ctrl(T, _reg_eq(cs, 0), {od: 0}), TAG_PERM, bc)
        g += _p11(r["a1"], r["q1"], r["i"], _ctrl(T, _reg_eq(cs, 1), {od: 1}), TAG_PERM, bc)
        g += _p11(r["a2"], r["q2"], r["i"], _ctrl(T, _reg_eq(cs, 2), {od: 1}), TAG_PERM, bc)
        g += _pi3(lay, _ctrl(T, _reg_eq(cs, 3)), TAG_PERM, bc)
    else:
        g += _p11(r["a1"], r["q1"], r["i"], dict(T), TAG_PERM, bc)
    g += _inc(r["k"], T, TAG_PERM)
    k, l = r["k"], r["l"]
    for p in prefix_patterns(0, Nt, lay.nm):
        pc = _pattern_ctrl(r["m"], p)
        for b in range(lay.nk):
            g.append(_gate(OP_X, l[b], _ctrl(C, pc, {k[b]: 1}), tag=TAG_PERM))
        for b in range(lay.nk):
            g.append(_gate(OP_X, k[b], _ctrl(C, pc, {l[b]: 1}), tag=TAG_PERM))
        for b in range(lay.nk):
            g.append(_gate(OP_X, k[b], _ctrl(C, pc), tag=TAG_PERM))
    g += _inc(r["km"], C, TAG_PERM)
    # ---- value encoding
    for kn in range(1, K + 1):
        for p in prefix_patterns(0, Nt, lay.nm):
            base = _ctrl(T, _reg_eq(k, kn), _pattern_ctrl(r["m"], p))
            if NC == 2:
                cs, od = r["case"], r["ord"][0]
                for cval, ordv, qreg in ((0, 0, "q1"), (1, 1, "q1"), (2, 1, "q2")):
                    for qo in range(3):
                        for io in range(4):
                            v = v11(qo, io, tau)
                            if v != 0.0:
                                c = _ctrl(base, _reg_eq(cs, cval), {od: ordv},
                                          _reg_eq(r[qreg], qo), _reg_eq(r["i"], io))
                                g.append(_gate(OP_RY, t, c, _theta(v, kn - 1, dt, Lmax), TAG_VALUE))
                    if bc == "bounceback":
                        areg = r["a1"] if qreg == "q1" else r["a2"]
                        g += _wall_fix(lay, _ctrl(base, _reg_eq(cs, cval), {od: ordv}), areg,
                                       r[qreg], lambda qo, io: v11(qo, io, tau),
                                       {io: _reg_eq(r["i"], io) for io in range(3)},
                                       kn - 1, dt, Lmax, t)
                for qo in range(3):
                    for io in range(4):
                        v = P.k12(qo, io & 1, io >> 1, tau)
                        if v != 0.0:
                            c = _ctrl(base, _reg_eq(cs, 3), {od: 0}, _reg_eq(r["a2"], 0),
                                      _reg_eq(r["q2"], 0), _reg_eq(r["q1"], qo), _reg_eq(r["i"], io))
                            g.append(_gate(OP_RY, t, c, _theta(v, kn - 1, dt, Lmax), TAG_VALUE))
                if bc == "bounceback":
                    g += _wall_fix(lay, _ctrl(base, _reg_eq(cs, 3), {od: 0}, _reg_eq(r["a2"], 0),
                                              _reg_eq(r["q2"], 0)),
                                   r["a1"], r["q1"], lambda qo, io: P.k12(qo, io & 1, io >> 1, tau),
                                   {io: _reg_eq(r["i"], io) for io in range(4)}, kn - 1, dt, Lmax, t)
            else:
                for qo in range(3):
                    for io in range(4):
                        v = v11(qo, io, tau)
                        if v != 0.0:
                            c = _ctrl(base, _reg_eq(r["q1"], qo), _reg_eq(r["i"], io))
                            g.append(_gate(OP_RY, t, c, _theta(v, kn - 1, dt, Lmax), TAG_VALUE))
                if bc == "bounceback":
                    g += _wall_fix(lay, base, r["a1"], r["q1"], lambda qo, io: v11(qo, io, tau),
                                   {io: _reg_eq(r["i"], io) for io in range(3)}, kn - 1, dt, Lmax, t)
    unused0 = {b: 0 for b in r["unused"]}
    th_m1 = 2.0 * math.asin(-1.0 / Lmax)
    for pm in prefix_patterns(1, Nt + 1, lay.nm):
        for pl in prefix_patterns(0, K + 1, lay.nk):
            c = _ctrl(C, unused0, _reg_eq(k, 0), _pattern_ctrl(r["m"], pm), _pattern_ctrl(l, pl))
            g.append(_gate(OP_RY, t, c, th_m1, TAG_VALUE))
    for pc in prefix_patterns(Nt * (1 << lay.nk) + 1, 1 << (lay.nk + lay.nm), lay.nk + lay.nm):
        c = _ctrl(C, unused0, _reg_eq(l, 0), _pattern_ctrl(r["km"], pc))
        g.append(_gate(OP_RY, t, c, th_m1, TAG_VALUE))
    g.append(_gate(OP_RY, t, {b: 1 for b in r["iL"]}, 2.0 * math.asin(1.0 / Lmax), TAG_VALUE))
    for b in r["iL"]:
        g.append(_gate(OP_H, b, tag=TAG_HUNPREP))
    g.append(_gate(OP_X, t, tag=TAG_TFLIP))
    return g


def dagger(gates):
    """Adjoint gate list: reversed order, angles negated (H, X self-inverse)."""
    return [(op, tg, cm, cv, -ang if op in (OP_RY, OP_ZPHASE) else ang, tag)
            for (op, tg, cm, cv, ang, tag) in reversed(gates)]


def phase_gates(lay: Layout, phi):
    r = lay.regs
    anc0 = {b: 0 for b in r["iL"] + r["t"]}
    s = r["s"][0]
    return [_gate(OP_X, s, anc0, tag=TAG_PHASE),
            _gate(OP_ZPHASE, s, {}, phi, tag=TAG_PHASE),
            _gate(OP_X, s, anc0, tag=TAG_PHASE)]


def build_qsvt(Nx, tau, NC, K, dt, Nt, phases, bc="periodic"):
    """Fig. circuit-qsvt with signal Hadamards: H, PHI(phi_0), [U_L^dag or U_L, PHI]*d, H.

    The first oracle call on b is U_L^dag (the block encoding of L^T): an odd
    polynomial P ~ 1/x applied this way gives P^{SV}(L^T/lambda) ~ lambda L^{-1},
    the inverse that Sec. II.D.5 states the circuit implements.  Starting
    with U_L, as the figure is drawn, would give (L^T)^{-1} instead.
    """
    d = len(phases) - 1
    if d < 1 or d % 2 == 0:
        raise ValueError("need an odd degree d >= 1 (d+1 phases)")
    lay = Layout(Nx, NC, K, Nt)
    UL = build_UL(Nx, tau, NC, K, dt, Nt, bc)
    ULd = dagger(UL)
    s = lay.regs["s"][0]
    g = [_gate(OP_H, s, tag=TAG_SIGNAL)]
    g += phase_gates(lay, float(phases[0]))
    for j in range(1, d + 1):
        g += ULd if j % 2 == 1 else UL
        g += phase_gates(lay, float(phases[j]))
    g.append(_gate(OP_H, s, tag=TAG_SIGNAL))
    return g


def postselect_patterns(lay: Layout):
    """Mask of Sec. "Postselection mask": list of (cmask, cval) pairs."""
    r = lay.regs
    base = {b: 0 for b in r["s"] + r["t"] + r["iL"]}
    out = []
    for p in prefix_patterns(lay.Nt, 1 << lay.nm, lay.nm):
        out.append(_mask(_ctrl(base, _pattern_ctrl(r["m"], p))))
    return out


def initial_state(lay: Layout, f0):
    """b of Sec. II.D.5 in the register basis (normalised), as {index: amplitude}."""
    import numpy as np
    f0 = np.asarray(f0, dtype=np.float64).reshape(lay.Nx, 3)
    vec = P.carleman_vector(f0.reshape(-1), lay.NC)
    nrm = math.sqrt(float(np.sum(vec * vec)))
    out = {}
    for j, v in enumerate(vec):
        if v != 0.0:
            out[lay.embed_index(0, j)] = v / nrm
    return out, nrm
