"""Gate-count report: the V-chain expansion on hand-checked gates, and the
growth of the U_L counts with Nx (more site bits: longer increment cascades
and wider controls)."""
import paper_2606_12770_gb300 as G
from paper_2606_12770_gb300 import gatecount as GC


def test_expansion_of_single_gates():
    X, H, RY, ZP = 0, 1, 2, 3
    assert GC.elementary_counts([(X, 0, 0, 0, 0.0, 0)]) == {"X": 1}
    assert GC.elementary_counts([(X, 0, 0b10, 0b10, 0.0, 0)]) == {"CNOT": 1}
    assert GC.elementary_counts([(X, 0, 0b110, 0b110, 0.0, 0)]) == {"TOFFOLI": 1}
    # five controls, two of them on value 0
    c = GC.elementary_counts([(X, 0, 0b111110, 0b001110, 0.0, 0)])
    assert c["TOFFOLI"] == 2 * 5 - 3 and c["X"] == 4
    c = GC.elementary_counts([(RY, 0, 0b1110, 0b1110, 0.3, 0)])
    assert c == {"TOFFOLI": 4, "CNOT": 2, "RY": 2}
    assert GC.elementary_counts([(ZP, 1, 0, 0, 0.1, 0)]) == {"RZ": 1}
    assert GC.elementary_counts([(H, 3, 0, 0, 0.0, 0)]) == {"H": 1}
    h = GC.histogram([(X, 0, 0b110, 0b110, 0.0, 0), (X, 1, 0b100, 0, 0.0, 0)])
    assert h[("X", 2)] == 1 and h[("X", 1)] == 1


def test_counts_grow_with_grid_size():
    tot = []
    for Nx in (4, 8, 16, 32):
        c = G.Circuit(Nx, 0.8, 2, 2, 0.1, 4, kappa_qsvt=10.0, d=3)
        g = c.export_gates(0)
        e = GC.elementary_counts(g)
        assert sum(GC.histogram(g).values()) == len(g)
        tot.append(e["TOFFOLI"])
    assert all(b > a for a, b in zip(tot, tot[1:]))
