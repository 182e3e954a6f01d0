"""Pins for the oracle's gate compiler (O3), layout, simulator (O2) and extractor (O4)."""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import blockenc as B
from oracle import circuit as C
from oracle import physics as P
from oracle import statevec as S
from oracle.layout import Layout


def test_qubit_count_table():
    """Table tab:qubit-count: I/O qubits of the L block encoding (+1 signal for QSVT)."""
    for row in read_golden("qubit_count.txt"):
        NC, K, formula = int(row[0]), int(row[1]), " ".join(row[2:])
        for Nx in (4, 8, 64):
            for Nt in (2, 4, 5, 16):
                lay = Layout(Nx, NC, K, Nt)
                n_a, n_m = lay.na, (2 * Nt - 1).bit_length()
                expect = eval(formula, {}, {"n_a": n_a, "n_m": n_m})
                assert lay.n == expect + 1, (NC, K, Nx, Nt)


@pytest.mark.parametrize("NC,K", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 3), (2, 4)])
@pytest.mark.parametrize("tau", [0.55, 0.8, 1.5, 0.09375])
def test_max_abs_entries_match_assembled_A(NC, K, tau):
    """The compiler's max|A| from distinct entries equals the assembled matrix's."""
    A = P.carleman_A(4, tau, NC, "periodic")
    assert C.max_abs_A(tau, NC) == P.max_abs_entry(A)


def test_prefix_patterns_cover_exactly():
    rng = np.random.default_rng(0)
    for _ in range(200):
        w = int(rng.integers(1, 8))
        lo = int(rng.integers(0, 1 << w))
        hi = int(rng.integers(lo, (1 << w) + 1))
        covered = []
        for v, j in C.prefix_patterns(lo, hi, w):
            covered += [(v << j) + r for r in range(1 << j)]
        assert covered == list(range(lo, hi))


@pytest.mark.parametrize("args", [(2, 0.8, 1, 1, 0.1, 1), (4, 0.8, 1, 2, 0.1, 2),
                                  (8, 0.6, 1, 3, 0.3, 3), (4, 0.55, 1, 4, 0.2, 5)])
def test_block_encoding_nc1(args):
    """App. B method: lambda_L <0|U_L|0> = L on physical states, zero cross terms."""
    tol = float(read_golden("blockenc_app_b.txt")[1][1])
    err, cross, lam = B.compare_with_L(*args)
    assert err < tol and cross == 0.0


@pytest.mark.parametrize("args", [(2, 0.8, 2, 1, 0.1, 1), (4, 0.8, 2, 1, 0.1, 1),
                                  (2, 1.3, 2, 3, 0.2, 3), (4, 0.8, 2, 2, 0.1, 2)])
def test_block_encoding_nc2(args):
    """Same at N_C=2 over every basis input (A11, A12, A22 blocks inside L)."""
    tol = float(read_golden("blockenc_app_b.txt")[1][1])
    err, cross, lam = B.compare_with_L(*args)
    assert err < tol and cross == 0.0


def test_block_encoding_lmax_above_one():
    """tau small enough that dt*max|A| > 1, so the RY angles use L_max > 1."""
    tau, dt = 0.09375, 0.2
    assert C.lmax_value(tau, 2, dt) > 1.0
    err, cross, lam = B.compare_with_L(2, tau, 2, 2, dt, 2)
    assert err < 1e-13 and cross == 0.0


def test_gate_list_well_formed():
    g = C.build_UL(4, 0.8, 2, 2, 0.1, 2)
    lay = Layout(4, 2, 2, 2)
    for op, t, cm, cv, ang, tag in g:
        assert 0 <= t < lay.n and not (cm >> t) & 1 and (cv & ~cm) == 0
        assert cm < (1 << lay.n)
        if op in (C.OP_X, C.OP_H):
            assert ang == 0.0
    d = C.dagger(g)
    assert C.dagger(d) == g


def _random_gates(n, count, rng):
    g = []
    for _ in range(count):
        op = int(rng.integers(0, 4))
        t = int(rng.integers(n))
        others = [b for b in range(n) if b != t]
        nc = int(rng.integers(0, min(4, n - 1) + 1))
        cs = rng.choice(others, nc, replace=False) if nc else []
        cm = sum(1 << int(c) for c in cs)
        cv = sum((int(rng.integers(2)) << int(c)) for c in cs)
        ang = float(rng.uniform(-math.pi, math.pi)) if op in (2, 3) else 0.0
        g.append((op, t, cm, cv, ang, 0))
    return g


def test_dense_sim_matches_brute_force_random():
    """O2 vs dense 2^n x 2^n gate matrices, random controlled gates, n <= 10."""
    rng = np.random.default_rng(5)
    for n in (3, 6, 9):
        gates = _random_gates(n, 40, rng)
        psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
        psi0 /= np.linalg.norm(psi0)
        U = S.circuit_unitary(gates, n)
        assert np.max(np.abs(U.conj().T @ U - np.eye(1 << n))) < 1e-12
        psi = S.DenseSim(n, check_norm=True).run(psi0.copy(), gates)
        assert np.max(np.abs(psi - U @ psi0)) < 1e-13


def test_dense_sim_matches_brute_force_UL():
    """O2 vs brute force on the whole U_L of the 10-qubit instance (N_C=1, Nx=2, K=1, Nt=1)."""
    lay = Layout(2, 1, 1, 1)
    assert lay.n == 10
    gates = C.build_UL(2, 0.8, 1, 1, 0.1, 1)
    U = S.circuit_unitary(gates, lay.n)
    rng = np.random.default_rng(2)
    psi0 = rng.standard_normal(1 << 10) + 1j * rng.standard_normal(1 << 10)
    psi0 /= np.linalg.norm(psi0)
    psi = S.DenseSim(10, check_norm=True).run(psi0.copy(), gates)
    assert np.max(np.abs(psi - U @ psi0)) < 1e-13


def test_sparse_columns_match_dense():
    rng = np.random.default_rng(9)
    n = 8
    gates = _random_gates(n, 30, rng)
    inputs = np.array([3, 17, 200, 0, 255])
    sim = S.SparseColumns(n, inputs).run(gates)
    for c, inp in enumerate(inputs):
        psi = np.zeros(1 << n, dtype=complex)
        psi[inp] = 1.0
        S.DenseSim(n).run(psi, gates)
        got = np.zeros(1 << n, dtype=complex)
        sel = sim.col == c
        got[sim.key[sel]] = sim.amp[sel]
        assert np.max(np.abs(got - psi)) < 1e-14


def test_norm_drift_is_detected():
    """The per-gate norm check fires when a planted mistake breaks unitarity."""

    class Leaky(S.DenseSim):
        def apply(self, psi, gate):
            super().apply(psi, gate)
            psi *= 1.0 + 1e-9

    n = 4
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1.0
    S.DenseSim(n, check_norm=True).run(psi, [(1, 0, 0, 0, 0.0, 0)])
    with pytest.raises(AssertionError):
        Leaky(n, check_norm=True).run(psi, [(1, 0, 0, 0, 0.0, 0)])


def test_initial_state_embedding():
    lay = Layout(4, 2, 2, 2)
    f0 = np.arange(12, dtype=float).reshape(4, 3) + 1.0
    init, nrm = C.initial_state(lay, f0)
    vec = P.carleman_vector(f0.reshape(-1), 2)
    assert abs(nrm - np.linalg.norm(vec)) < 1e-12
    for j, v in enumerate(vec):
        assert abs(init[lay.embed_index(0, j)] - v / nrm) < 1e-15
    # f2 entry (a1,q1,a2,q2) = f0[a1,q1] f0[a2,q2]
    idx = lay.place(a1=1, q1=2, a2=3, q2=0, ord=1)
    assert abs(init[idx] * nrm - f0[1, 2] * f0[3, 0]) < 1e-12


def test_axis_simulator_matches_brute_force_and_index_simulator():
    """AxisSim (sub-tensor views along qubit axes) against the dense unitary
    brute force at 6 qubits and against DenseSim at 12 and 18 qubits (the
    latter large enough to be cut into pieces for threads), on seeded
    streams of every gate kind with controls on either value; a transposed
    axis, a wrong control value or a swapped matrix entry changes the state."""
    import numpy as np
    import lbm_inputs as I
    from oracle import statevec as S
    rng = np.random.default_rng(4)
    for n, count in ((6, 60), (12, 300), (18, 80)):  # 18: the threaded pieces
        gates = []
        for _ in range(count):
            op = int(rng.integers(4))
            t = int(rng.integers(n))
            others = [q for q in range(n) if q != t]
            nc = int(rng.integers(0, 4))
            cs = [int(q) for q in rng.choice(others, nc, replace=False)]
            cm = sum(1 << q for q in cs)
            cv = sum((int(rng.integers(2)) << q) for q in cs)
            gates.append((op, t, cm, cv, float(rng.uniform(-3, 3)), 0))
        psi = I.random_unit_state(n, 9)
        got = S.AxisSim(n).run(psi.copy(), gates)
        if n <= 6:
            ref = S.circuit_unitary(gates, n) @ psi
        else:
            ref = S.DenseSim(n).run(psi.copy(), gates)
        assert np.linalg.norm(got - ref) < 1e-12
