"""Gate-count report of the compiled circuits (Sec. III.F.2, "Gate count").

The paper compiles its circuits to {TOFFOLI, CNOT, H, X, RY, S, S^dag},
removes adjacent identical Toffoli pairs and X-X pairs with a peephole pass,
and, because a QSVT circuit is linear in its degree, counts it at d = 3 and
d = 13 and interpolates linearly in d to the target degree.  This module does
the same for the library's gate lists (multi-controlled X, H, RY and Z-phase
gates, ``Circuit.export_gates``):

* ``histogram`` counts the records by kind and number of controls;
* ``expand`` writes each record out as elementary gates with the standard
  clean-ancilla V-chain, as gate records of the same format on the register
  plus ancilla qubits n, n+1, ...:

  - a control on value 0 is conjugated by X on that qubit;
  - X with c controls is X (c = 0), CNOT (c = 1), TOFFOLI (c = 2), or for
    c >= 3 a chain of Toffolis that ANDs the controls into c - 2 ancillas, one
    Toffoli onto the target, and the chain undone (2c - 3 Toffolis);
  - RY or a Z phase with c >= 1 controls: the AND of the controls in one
    ancilla (c - 1 Toffolis to compute and again to uncompute, c >= 2), then
    the singly controlled rotation as rotation(theta/2), CNOT,
    rotation(-theta/2), CNOT;
  - H is uncontrolled in these circuits.

  The ancilla chain always takes the controls in ascending qubit order and
  the same ancillas, so consecutive gates that share controls produce
  identical Toffolis back to back;
* ``peephole`` removes adjacent identical pairs of Toffolis and of X gates
  (both self-inverse): a gate cancels the latest gate still alive on all of
  its qubits when that gate is identical and nothing else touched those
  qubits in between; removal exposes earlier gates, so nested pairs go too;
* ``elementary_counts`` counts the expanded list (optionally after the
  peephole pass) in {TOFFOLI, CNOT, X, H, RY, RZ} (a Z phase is an RZ up to
  sign convention; S and S^dag do not occur in this construction);
* ``interpolated_counts`` counts QSVT circuits of degree 3 and 13 and
  interpolates linearly in d, as the paper does.

The expansion describes this repository's ancilla-free construction (no work
ancillas in the simulated register); the paper's circuits carry work ancillas
and case flags, so the counts are of a different decomposition of the same
operator, not the paper's numbers.
"""
from __future__ import annotations

from collections import Counter

OPS = {0: "X", 1: "H", 2: "RY", 3: "ZPHASE"}
OP_X, OP_H, OP_RY, OP_ZPHASE = 0, 1, 2, 3


def _records(gates):
    for g in gates:
        if isinstance(g, tuple):
            yield int(g[0]), int(g[1]), int(g[2]), int(g[3]), float(g[4])
        else:
            yield int(g["op"]), int(g["target"]), int(g["cmask"]), int(g["cval"]), float(g["angle"])


def histogram(gates):
    """Counter over (kind, number of controls)."""
    h = Counter()
    for op, _, cm, _, _ in _records(gates):
        h[(OPS[op], bin(cm).count("1"))] += 1
    return h


def _bits(mask):
    out = []
    b = 0
    while mask:
        if mask & 1:
            out.append(b)
        mask >>= 1
        b += 1
    return out


def _x(t, *ctrl):
    cm = 0
    for c in ctrl:
        cm |= 1 << c
    return (OP_X, t, cm, cm, 0.0)


def _and_chain(ctrl, anc):
    """Toffolis that leave AND(ctrl) in anc[len(ctrl) - 2] (len(ctrl) >= 2)."""
    out = [_x(anc[0], ctrl[0], ctrl[1])]
    for j in range(2, len(ctrl)):
        out.append(_x(anc[j - 1], ctrl[j], anc[j - 2]))
    return out


def expand(gates, n):
    """Elementary gate records (op, target, cmask, cval, angle) of the V-chain
    expansion; ancillas are qubits n, n+1, ... and start and end in 0.
    Returns (list, number of ancillas used)."""
    out = []
    n_anc = 0
    for op, t, cm, cv, ang in _records(gates):
        ctrl = _bits(cm)
        zeros = [q for q in ctrl if not (cv >> q) & 1]
        c = len(ctrl)
        pre = [_x(q) for q in zeros]
        body = []
        if op == OP_X:
            if c <= 2:
                body.append(_x(t, *ctrl))
            else:
                anc = [n + j for j in range(c - 2)]
                n_anc = max(n_anc, c - 2)
                chain = _and_chain(ctrl[:-1], anc)
                body += chain
                body.append(_x(t, ctrl[-1], anc[c - 3]))
                body += chain[::-1]
        elif op == OP_H:
            if c:
                raise ValueError("controlled H does not occur in these circuits")
            body.append((OP_H, t, 0, 0, 0.0))
        else:
            if c == 0:
                body.append((op, t, 0, 0, ang))
            else:
                if c == 1:
                    q = ctrl[0]
                    chain = []
                else:
                    anc = [n + j for j in range(c - 1)]
                    n_anc = max(n_anc, c - 1)
                    chain = _and_chain(ctrl, anc)
                    q = anc[c - 2]
                body += chain
                body += [(op, t, 0, 0, ang / 2.0), _x(t, q), (op, t, 0, 0, -ang / 2.0), _x(t, q)]
                body += chain[::-1]
        out += pre + body + pre
    return out, n_anc


def _kind(g):
    op, _, cm, _, _ = g
    if op == OP_X:
        return ("X", "CNOT", "TOFFOLI")[bin(cm).count("1")]
    if op == OP_H:
        return "H"
    return "RY" if op == OP_RY else "RZ"


def peephole(elem):
    """Remove adjacent identical Toffoli pairs and X-X pairs (see module doc)."""
    alive = [True] * len(elem)
    top = {}      # qubit -> stack of indices of live gates touching it
    for i, g in enumerate(elem):
        qubits = [g[1]] + _bits(g[2])
        kind = _kind(g)
        if kind in ("TOFFOLI", "X"):
            stacks = [top.get(q) for q in qubits]
            if all(s for s in stacks):
                j = stacks[0][-1]
                h = elem[j]
                if all(s[-1] == j for s in stacks) and h[:4] == g[:4]:
                    for s in stacks:
                        s.pop()
                    alive[j] = False
                    alive[i] = False
                    continue
        for q in qubits:
            top.setdefault(q, []).append(i)
    return [g for g, a in zip(elem, alive) if a]


def elementary_counts(gates, n=None, peephole_pass=False):
    """Counts in {TOFFOLI, CNOT, X, H, RY, RZ} of the V-chain expansion, after
    the peephole pass when asked (n, the register width, places the
    ancillas; any value above the highest qubit will do)."""
    if n is None:
        n = 1 + max(max([t] + _bits(cm)) for _, t, cm, _, _ in _records(gates)) if len(gates) else 0
    elem, _ = expand(gates, n)
    if peephole_pass:
        elem = peephole(elem)
    return Counter(_kind(g) for g in elem)


def interpolated_counts(build, d_target, peephole_pass=True):
    """The paper's procedure: elementary counts of the whole QSVT circuit at
    d = 3 and d = 13, interpolated linearly in d to d_target.  `build(d)`
    returns the gate list of the degree-d circuit."""
    c3 = elementary_counts(build(3), peephole_pass=peephole_pass)
    c13 = elementary_counts(build(13), peephole_pass=peephole_pass)
    out = {}
    for k in set(c3) | set(c13):
        slope = (c13.get(k, 0) - c3.get(k, 0)) / 10.0
        out[k] = c3.get(k, 0) + slope * (d_target - 3)
    return out
