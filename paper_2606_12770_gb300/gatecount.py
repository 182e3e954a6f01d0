"""Gate-count report of the compiled circuits (the paper's gate-count figures,
Sec. III.F, report counts in a Toffoli + Clifford + rotation gate set).

The library's gate lists are made of multi-controlled X, H, RY and Z-phase
gates (``Circuit.export_gates``).  ``histogram`` counts them by kind and number
of controls; ``elementary_counts`` expands them into the gate set
{TOFFOLI, CNOT, X, H, RY, RZ} with the standard clean-ancilla V-chain:

* a control on value 0 costs two X (conjugation);
* X with c controls: X (c = 0), CNOT (c = 1), TOFFOLI (c = 2), and 2c - 3
  TOFFOLIs for c >= 3 (c - 2 ancillas computed, used and uncomputed);
* RY or a Z phase with c >= 1 controls: the AND of the controls in one
  ancilla (2(c - 1) TOFFOLIs to compute and uncompute for c >= 2), then the
  singly controlled rotation as two CNOTs and two rotations;
* H is uncontrolled in these circuits.

This is an expansion of this repository's own construction (no work ancillas
in the simulated register); the paper's circuits differ (they carry work
ancillas and case flags), so the counts describe a different decomposition
of the same operator, not the paper's numbers.
"""
from __future__ import annotations

from collections import Counter

OPS = {0: "X", 1: "H", 2: "RY", 3: "ZPHASE"}


def _records(gates):
    for g in gates:
        if isinstance(g, tuple):
            yield int(g[0]), int(g[2]), int(g[3])
        else:
            yield int(g["op"]), int(g["cmask"]), int(g["cval"])


def histogram(gates):
    """Counter over (kind, number of controls)."""
    h = Counter()
    for op, cm, _ in _records(gates):
        h[(OPS[op], bin(cm).count("1"))] += 1
    return h


def elementary_counts(gates):
    """Counts in {TOFFOLI, CNOT, X, H, RY, RZ} under the V-chain expansion."""
    out = Counter()
    for op, cm, cv in _records(gates):
        c = bin(cm).count("1")
        zeros = c - bin(cv & cm).count("1")
        if zeros:
            out["X"] += 2 * zeros
        if op == 0:
            if c == 0:
                out["X"] += 1
            elif c == 1:
                out["CNOT"] += 1
            elif c == 2:
                out["TOFFOLI"] += 1
            else:
                out["TOFFOLI"] += 2 * c - 3
        elif op == 1:
            if c:
                raise ValueError("controlled H does not occur in these circuits")
            out["H"] += 1
        else:
            rot = "RY" if op == 2 else "RZ"
            if c == 0:
                out[rot] += 1
            else:
                if c >= 2:
                    out["TOFFOLI"] += 2 * (c - 1)
                out["CNOT"] += 2
                out[rot] += 2
    return out
