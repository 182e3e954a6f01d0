"""The fused-program format executed on the host (csim_emulate_fused) against the oracle.

The same fuser output runs on the GPU; these CPU tests check the fuser's
lookup-table permutations, multiplexed rotations and warp-tile gates."""
import math

import numpy as np
import pytest

import lbm_inputs as I
from oracle import circuit as OC
from oracle import statevec as S
from oracle.layout import Layout
from paper_2606_12770_gb300 import _native as N


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def random_gates(n, count, seed, ops=(0, 1, 2, 3), maxc=4, targets=None):
    rng = np.random.default_rng(seed)
    g = []
    for _ in range(count):
        op = int(rng.choice(ops))
        t = int(rng.choice(targets)) if targets is not None else int(rng.integers(n))
        others = [b for b in range(n) if b != t]
        nc = int(rng.integers(0, maxc + 1))
        cs = rng.choice(others, nc, replace=False) if nc else []
        cm = sum(1 << int(c) for c in cs)
        cv = sum(int(rng.integers(2)) << int(c) for c in cs)
        ang = float(rng.uniform(-math.pi, math.pi)) if op in (2, 3) else 0.0
        g.append((op, t, cm, cv, ang, 0))
    return g


@pytest.mark.parametrize("n,seed", [(7, 1), (9, 2), (12, 3), (15, 4)])
def test_random_lists(n, seed):
    g = random_gates(n, 250, seed)
    psi = I.random_unit_state(n, seed)
    got, st = N.emulate_fused(g, n, psi)
    assert rel(got, S.DenseSim(n).run(psi.copy(), g)) < 1e-13


def test_long_permutation_runs_split_into_tables():
    """Only multi-controlled X on qubits >= 2: one gather, several lookup tables."""
    n = 20
    g = random_gates(n, 300, 7, ops=(0,), maxc=6, targets=list(range(2, 20)))
    g = [x for x in g if x[2] & 3 == 0]
    psi = I.random_unit_state(n, 7)
    got, st = N.emulate_fused(g, n, psi)
    # at most 32 steps fit one kernel parameter block; longer runs take more passes
    assert st["segments"] > 1 and st["max_support"] <= 14
    assert st["passes"] == -(-st["segments"] // 32)
    assert rel(got, S.DenseSim(n).run(psi.copy(), g)) < 1e-14


@pytest.mark.parametrize("target", [0, 1])
def test_multiplexed_rotations(target):
    """Runs of RY on an in-thread qubit, controls anywhere (incl. the other low qubit)."""
    n = 14
    g = random_gates(n, 200, 11 + target, ops=(2,), maxc=7, targets=[target])
    psi = I.random_unit_state(n, 3)
    got, st = N.emulate_fused(g, n, psi)
    # one multiplexer per distinct control pattern on the other in-thread qubit
    assert 1 <= st["mux"] <= 3 and st["mux_gates"] == 200
    assert rel(got, S.DenseSim(n).run(psi.copy(), g)) < 1e-13


def test_microbench_stream():
    n = 16
    g = I.microbench_gates(n, 400, 1)
    psi = I.random_unit_state(n, 1)
    got, _ = N.emulate_fused(g, n, psi)
    assert rel(got, S.DenseSim(n).run(psi.copy(), g)) < 1e-13


@pytest.mark.parametrize("cfg,d", [((4, 0.8, 2, 2, 0.1, 2), 3), ((8, 0.7, 1, 3, 0.2, 3), 5)])
def test_qsvt_circuit_one_sweep_per_call(cfg, d):
    lay = Layout(cfg[0], cfg[2], cfg[3], cfg[5])
    f0, _ = I.lbm_instance(cfg[0], 0, tau=cfg[1])
    gates = OC.build_qsvt(*cfg, list(I.random_phases(d, 5)))
    psi = np.zeros(1 << lay.n, dtype=complex)
    init, _ = OC.initial_state(lay, f0)
    for k, v in init.items():
        psi[k] = v
    got, st = N.emulate_fused(gates, lay.n, psi)
    assert st["passes"] == d + 1 and st["single"] == 0
    if cfg[2] == 2:  # five label qubits = all lane bits: projector phases become averaging blocks
        assert st["reflect"] == d - 1  # every phase between two oracle calls
    # the multiplexer that ends U_L and its inverse that starts the next U_L^dag
    # share one sweep: the second reuses the first's rotation
    assert st["mux_inverse"] == (d - 1) // 2
    # the label Hadamard layers of the first and the last call are fused
    assert st["wht"] == 2
    # each U_L^dag permutation is undone by the next U_L: one in-place sweep
    # (P^-1, projector, P); the multiplexer sweeps between need no gather
    assert st["conjugated"] == (d - 1) // 2
    assert rel(got, S.DenseSim(lay.n).run(psi.copy(), gates)) < 1e-13


def test_lane_walsh_hadamard_fused():
    """Uncontrolled H gates on distinct lane bits run as one Walsh-Hadamard op;
    a repeated bit or a controlled H ends the run."""
    n = 11
    g = [(1, b, 0, 0, 0.0, 0) for b in (6, 4, 2, 3)]          # one op (4 bits)
    g += [(1, 3, 0, 0, 0.0, 0), (1, 5, 0, 0, 0.0, 0)]         # bit 3 again: a second op
    g += [(1, 2, 1 << 9, 1 << 9, 0.0, 0), (1, 4, 0, 0, 0.0, 0)]  # controlled: single gates
    g += [(2, 0, 1 << 8, 0, 0.7, 0), (1, 5, 0, 0, 0.0, 0), (1, 6, 0, 0, 0.0, 0), (1, 2, 0, 0, 0.0, 0)]
    psi = I.random_unit_state(n, 8)
    got, st = N.emulate_fused(g, n, psi)
    assert st["wht"] == 3
    assert rel(got, S.DenseSim(n).run(psi.copy(), g)) < 1e-14


def test_conjugated_sweep_random_permutation():
    """A run of multi-controlled X gates, tile-local gates, then the same X gates
    in reverse: one in-place conjugated sweep, P^-1 . ops . P, then the local
    gates that follow need no gather.  Every X gate is controlled by lane bit 2,
    on which the local run has an H, so no X gate commutes across it (as in
    the QSVT circuit, where U_L's permutation reads the label).  Against the
    dense simulator."""
    n = 14
    rng = np.random.default_rng(21)
    perm = []
    for _ in range(40):
        t = int(rng.integers(7, n))  # above the tile: a permutation gate, never tile-local
        others = [b for b in range(3, n) if b != t]
        cs = list(rng.choice(others, int(rng.integers(0, 4)), replace=False)) + [2]
        cm = sum(1 << int(c) for c in cs)
        cv = sum(int(rng.integers(2)) << int(c) for c in cs)
        perm.append((0, t, cm, cv, 0.0, 0))
    local = [(1, 2, 0, 0, 0.0, 0)] + random_gates(n, 30, 22, ops=(1, 2, 3), maxc=3,
                                                   targets=list(range(7)))
    after = random_gates(n, 30, 23, ops=(1, 2, 3), maxc=3, targets=list(range(7)))
    g = perm + local + perm[::-1] + after
    psi = I.random_unit_state(n, 9)
    got, st = N.emulate_fused(g, n, psi)
    assert st["conjugated"] == 1
    assert rel(got, S.DenseSim(n).run(psi.copy(), g)) < 1e-13


def test_averaging_block_detection_general():
    """H layer on lane bits, tile-internal diagonal/controlled gates, H layer: one block."""
    n = 12
    lanes = [2, 3, 4, 5, 6]
    g = [(1, b, 0, 0, 0.0, 0) for b in lanes]
    anc = sum(1 << b for b in lanes) | 1
    g += [(0, 0, 0, 0, 0.0, 0), (0, 1, anc, 0, 0.0, 0), (3, 1, 0, 0, 0.37, 0), (0, 1, anc, 0, 0.0, 0),
          (0, 0, 0, 0, 0.0, 0)]
    g += [(1, b, 0, 0, 0.0, 0) for b in lanes]
    psi = I.random_unit_state(n, 4)
    got, st = N.emulate_fused(g, n, psi)
    assert st["reflect"] == 1
    assert rel(got, S.DenseSim(n).run(psi.copy(), g)) < 1e-13


def test_staged_sweeps_match_oracle_on_host():
    """Gates on qubits above the warp tile join sweeps that hold 2^k tiles per
    warp (k <= 3 staged qubits): the host executor of the fused program
    against the dense oracle on seeded vocabulary streams, and the 30-qubit
    stream needs far fewer passes than its 1505 gates."""
    import numpy as np
    import lbm_inputs as I
    from oracle import statevec as S
    from paper_2606_12770_gb300 import _native as N
    for n, count, seed in ((12, 200, 1), (14, 300, 2)):
        gates = I.microbench_gates(n, count, seed)
        psi = I.random_unit_state(n, seed)
        ref = S.DenseSim(n).run(psi.copy(), gates)
        got, st = N.emulate_fused(gates, n, psi)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13
        assert st["staged_sweeps"] > 0 and st["staged_gates"] > 0
    _, st = N.emulate_fused(I.microbench_gates(30, 1000, 0), 30, None)
    assert st["passes"] <= 200


def test_dense_blocks_match_oracle_on_host():
    """Runs of at least ten gates on at most five qubits that mix amplitudes
    across the warp tile become dense blocks (the host executor applies their
    composed 32 x 32 matrices in FP64): the
    fused program against the dense oracle on a seeded stream of 5-qubit
    blocks, one block per run; the vocabulary stream, whose gates spread over
    all qubits, forms at most a couple."""
    import numpy as np
    import lbm_inputs as I
    from oracle import statevec as S
    from paper_2606_12770_gb300 import _native as N
    n = 14
    gates = I.dense_block_gates(n, 12, 3)
    psi = I.random_unit_state(n, 3)
    ref = S.DenseSim(n).run(psi.copy(), gates)
    got, st = N.emulate_fused(gates, n, psi)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13
    # one pass per block: a dense block, or a sweep for a block that stays
    # inside the warp tile (the sweep applies it without a pass of its own)
    assert st["passes"] == 12 and st["dense_blocks"] + st["sweeps"] == 12
    assert st["dense_blocks"] >= 10 and st["dense_gates"] == 16 * st["dense_blocks"]
    _, st = N.emulate_fused(I.microbench_gates(30, 1000, 0), 30, None)
    assert st["dense_blocks"] <= 2


def test_dense_blocks_with_selector_qubits_on_host():
    """A run on six qubits whose matrix never mixes the two values of one of
    them (a phase on that qubit, controlled by the others, between two layers
    of gates on the other five) becomes one dense block with that qubit as
    its selector: one 32 x 32 matrix per selector value.  Host executor
    against the dense oracle."""
    import numpy as np
    import lbm_inputs as I
    from oracle import statevec as S
    from paper_2606_12770_gb300 import _native as N
    n = 14
    rng = np.random.default_rng(6)
    q = [8, 9, 10, 11, 12]
    sel = 3
    gates = [(2, t, 0, 0, float(rng.uniform(0, 6.28)), 0) for t in q]
    gates += [(0, q[1], 1 << q[0], 1 << q[0], 0.0, 0)]
    m = (1 << q[2]) | (1 << q[4])
    gates += [(0, sel, m, m, 0.0, 0), (3, sel, 0, 0, 0.37, 0), (0, sel, m, m, 0.0, 0)]
    gates += [(1, t, 0, 0, 0.0, 0) for t in q]
    psi = I.random_unit_state(n, 6)
    ref = S.DenseSim(n).run(psi.copy(), gates)
    got, st = N.emulate_fused(gates, n, psi)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13
    assert st["dense_blocks"] == 1 and st["passes"] == 1
