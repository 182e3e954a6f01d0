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


def _small_ul():
    c = G.Circuit(2, 0.8, 1, 1, 0.1, 1, kappa_qsvt=10.0, d=3)
    return c.export_gates(0), c.info()["n_qubits"]


def test_expansion_and_peephole_preserve_the_operator():
    """The V-chain expansion of one U_L (N_C = 1, Nx = 2: 10 qubits plus the
    chain's ancillas), before and after the peephole pass, applied by the
    oracle's naive simulator to a random register state with the ancillas in
    0, equals the compiled gate list applied to the register alone, and
    leaves every ancilla in 0."""
    import numpy as np
    from oracle import statevec as S
    g, n = _small_ul()
    elem, na = GC.expand(g, n)
    pe = GC.peephole(elem)
    assert 0 < len(pe) < len(elem)
    rng = np.random.default_rng(5)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    ref = S.DenseSim(n).run(psi.copy(), [tuple(x) for x in
                                          ((int(r["op"]), int(r["target"]), int(r["cmask"]),
                                            int(r["cval"]), float(r["angle"]), 0) for r in g)])
    for lst in (elem, pe):
        big = np.zeros(1 << (n + na), dtype=complex)
        big[: 1 << n] = psi
        out = S.DenseSim(n + na).run(big, [x + (0,) for x in lst])
        assert np.linalg.norm(out[1 << n:]) < 1e-13
        assert np.linalg.norm(out[: 1 << n] - ref) < 1e-12


def test_peephole_cancels_only_identical_adjacent_pairs():
    X = 0
    tof = (X, 5, 0b11, 0b11, 0.0)
    # T T -> nothing; X X -> nothing; T (X on another qubit) T -> nothing
    assert GC.peephole([tof, tof]) == []
    assert GC.peephole([(X, 2, 0, 0, 0.0), (X, 2, 0, 0, 0.0)]) == []
    assert GC.peephole([tof, (X, 7, 0, 0, 0.0), tof]) == [(X, 7, 0, 0, 0.0)]
    # a gate on a shared qubit in between blocks the pair
    blk = (X, 0, 0, 0, 0.0)
    assert GC.peephole([tof, blk, tof]) == [tof, blk, tof]
    # nested pairs: T1 T2 T2 T1 -> nothing
    tof2 = (X, 6, 0b101, 0b101, 0.0)
    assert GC.peephole([tof, tof2, tof2, tof]) == []
    # CNOT pairs and rotations are left alone (the paper's pass removes
    # Toffoli and X-X pairs only)
    cn = (X, 3, 0b1, 0b1, 0.0)
    assert GC.peephole([cn, cn]) == [cn, cn]


def test_interpolated_count_matches_direct_count():
    """Sec. III.F.2: the QSVT gate count is linear in d, so the counts at
    d = 3 and d = 13 interpolate to any odd degree; checked against a direct
    count at d = 31, with and without the peephole pass."""
    def build(d):
        return G.Circuit(4, 0.8, 1, 2, 0.1, 2, kappa_qsvt=10.0, d=d).export_gates(1)
    for pp in (False, True):
        est = GC.interpolated_counts(build, 31, peephole_pass=pp)
        direct = GC.elementary_counts(build(31), peephole_pass=pp)
        assert set(est) == set(direct)
        for k, v in direct.items():
            assert abs(est[k] - v) < 1e-9, (pp, k, est[k], v)
    # the peephole pass removes Toffolis in the whole circuit
    full = GC.elementary_counts(build(13))
    pp = GC.elementary_counts(build(13), peephole_pass=True)
    assert pp["TOFFOLI"] < full["TOFFOLI"] and pp["RY"] == full["RY"]
