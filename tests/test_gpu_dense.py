"""Dense 5-qubit blocks on the tensor cores (tcgen05, split BF16x3, FP32
accumulation) and on the CUDA cores (FP32).

* One block applied through csim_sv_apply_dense to a seeded random complex64
  state, against the block's matrix applied by NumPy in FP64 along the five
  qubit axes (the definition of the operation), for qubit sets low, high,
  mixed and given out of order.  Tolerances: FP32, 1e-6 relative L2 (32-term
  complex sums at 2^-24); split BF16x3, 3e-5: each factor is the sum of two
  BF16 values (16 significant bits), so one product keeps a relative error of
  at most about 3 * 2^-18 = 1.1e-5, and the errors of the 64 terms of an
  output add with random signs.
* The fused program of a stream of 5-qubit blocks (one dense block per run)
  against the oracle's naive simulator on the elementary gates, both engines,
  at 20 and 24 qubits; tolerance 1e-4, the complex64 bound.
* The tensor-core kernel's bounded wait: with CSIM_DENSE_SPIN=0 it gives up at
  once, lets its products finish, frees its TMEM and returns; the next read
  reports CSIM_ERR_TIMEOUT and the context stays usable.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import lbm_inputs as I
import paper_2606_12770_gb300 as G
from oracle import statevec as S

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TC, FP32 = 0, 1


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def random_unitary(seed):
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def apply_block(psi, n, qubits, u):
    """y = U x over the five qubit axes (element bit j of U's index = qubits[j])."""
    T = psi.reshape((2,) * n)
    axes = [n - 1 - q for q in reversed(qubits)]  # element bit 4 is the slowest
    rest = [a for a in range(n) if a not in axes]
    X = np.transpose(T, axes + rest).reshape(32, -1)
    Y = u @ X
    out = np.empty_like(T)
    np.transpose(out, axes + rest)[...] = Y.reshape((2,) * 5 + (2,) * (n - 5))
    return out.reshape(-1)


@pytest.mark.parametrize("qubits", [[0, 1, 2, 3, 4], [15, 16, 17, 18, 19], [3, 9, 14, 17, 19],
                                    [17, 2, 11, 0, 8]])
@pytest.mark.parametrize("engine,tol", [(TC, 3e-5), (FP32, 1e-6)])
def test_single_block_against_definition(qubits, engine, tol):
    n = 20
    psi = I.random_unit_state(n, 2)
    u = random_unitary(sum(qubits))
    ref = apply_block(psi, n, qubits, u)
    sv = G.StateVector(n, G.CSIM_C64)
    sv.load(psi)
    sv.apply_dense(qubits, u, engine)
    got = sv.read()
    err = rel_l2(got, ref)
    print(f"dense block {qubits} engine {engine}: rel L2 {err:.3e}")
    assert err < tol


@pytest.fixture(scope="module")
def block_streams():
    out = {}
    for n in (20, 24):
        gates = I.dense_block_gates(n, 24, n)
        psi0 = I.random_unit_state(n, n)
        out[n] = (gates, psi0, S.AxisSim(n).run(psi0.copy(), gates))
    return out


@pytest.mark.parametrize("n", [20, 24])
@pytest.mark.parametrize("engine", ["tc", "fp32"])
def test_block_stream_against_oracle(block_streams, n, engine, monkeypatch):
    gates, psi0, ref = block_streams[n]
    if engine == "fp32":
        monkeypatch.setenv("CSIM_DENSE_ENGINE", "fp32")
    sv = G.StateVector(n, G.CSIM_C64)
    sv.load(psi0)
    sv.compile(G.gates_to_records(gates), G.CSIM_EXEC_FUSED)
    st = sv.stats()
    assert st["dense_blocks"] == 24 and st["passes"] == 24
    sv.run(1)
    err = rel_l2(sv.read(), ref)
    print(f"{n}-qubit block stream, {engine}: rel L2 {err:.3e}")
    assert err < 1e-4


TIMEOUT_SCRIPT = r'''
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import lbm_inputs as I, paper_2606_12770_gb300 as G
n = 14
sv = G.StateVector(n, G.CSIM_C64)
sv.load(I.random_unit_state(n, 1))
sv.apply_dense([0, 3, 5, 7, 9], np.eye(32), 0)
try:
    sv.read()
    print("no timeout")
except G.CsimError as e:
    assert e.status == -6, e.status
    print("timeout reported")
# the context is still usable: a gate stream runs and reads back
sv2 = G.StateVector(n, G.CSIM_C64)
psi = I.random_unit_state(n, 4)
sv2.load(psi)
sv2.compile(G.gates_to_records(I.microbench_gates(n, 50, 4)), G.CSIM_EXEC_GATE)
sv2.run(1)
out = sv2.read()
assert abs(np.linalg.norm(out) - 1.0) < 1e-5
print("ok")
'''


def test_tensor_core_wait_times_out_cleanly():
    env = dict(os.environ, CSIM_DENSE_SPIN="0")
    r = subprocess.run([sys.executable, "-c", TIMEOUT_SCRIPT, ROOT], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "timeout reported" in r.stdout and r.stdout.strip().endswith("ok"), r.stdout


def _label_layer(n_x=4):
    """The label layer of the precision circuit's family member (between the
    first U_L^dag and the next U_L): 13 gates on the five label qubits, the
    signal and the value-encoding target; the latter two only select the
    matrix (it is diagonal in them)."""
    import bench
    f0, tau = I.lbm_instance(n_x, 1, tau_range=(0.6, 1.2))
    c = G.Circuit(n_x, tau, 2, 4, 0.1, 16, kappa_qsvt=1000.0, d=13)
    return bench.label_layer(c.export_gates(1)), c.info()["n_qubits"]


@pytest.mark.parametrize("engine,tol", [("tc", 3e-5), ("fp32", 1e-6)])
def test_label_layer_as_selector_block(engine, tol, monkeypatch):
    """The QSVT label layer as one dense block with two selector qubits (a
    32 x 32 matrix per value of t and s) against the warp reduction the sweeps
    use and against the oracle's naive simulator, at 24 qubits."""
    layer, n = _label_layer()
    gates = [(int(g["op"]), int(g["target"]), int(g["cmask"]), int(g["cval"]),
              float(g["angle"]), 0) for g in layer]
    psi0 = I.random_unit_state(n, 3)
    ref = S.AxisSim(n).run(psi0.copy(), gates)
    monkeypatch.setenv("CSIM_DENSE_ENGINE", engine)
    sv = G.StateVector(n, G.CSIM_C64)
    sv.load(psi0)
    sv.compile(layer, stage=0, dense=2)
    st = sv.stats()
    assert st["dense_blocks"] == 1 and st["passes"] == 1
    sv.run(1)
    dense = sv.read()
    sv.load(psi0)
    sv.compile(layer, stage=0, dense=0)
    assert sv.stats()["dense_blocks"] == 0
    sv.run(1)
    warp = sv.read()
    e1, e2 = rel_l2(dense, ref), rel_l2(dense, warp)
    print(f"label layer as a selector block, {engine}: vs oracle {e1:.3e}, vs warp reduction {e2:.3e}")
    assert e1 < tol and e2 < tol and rel_l2(warp, ref) < 1e-6


@pytest.mark.parametrize("engine,tol", [("tc", 3e-5), ("fp32", 1e-6)])
def test_selector_block_above_the_tile(engine, tol, monkeypatch):
    """A run on five qubits above the tile and one selector qubit (a phase on
    it controlled by two of the five, between layers of RY and H) as one dense
    block, at 20 qubits, against the oracle."""
    n = 20
    rng = np.random.default_rng(12)
    q = [8, 11, 13, 16, 19]
    sel = 9
    gates = [(2, t, 0, 0, float(rng.uniform(0, 6.28)), 0) for t in q]
    gates += [(0, q[1], 1 << q[0], 1 << q[0], 0.0, 0)]
    m = (1 << q[2]) | (1 << q[4])
    gates += [(0, sel, m, m, 0.0, 0), (3, sel, 0, 0, 0.37, 0), (0, sel, m, m, 0.0, 0)]
    gates += [(1, t, 0, 0, 0.0, 0) for t in q]
    psi0 = I.random_unit_state(n, 12)
    ref = S.DenseSim(n).run(psi0.copy(), gates)
    monkeypatch.setenv("CSIM_DENSE_ENGINE", engine)
    sv = G.StateVector(n, G.CSIM_C64)
    sv.load(psi0)
    sv.compile(gates)
    assert sv.stats()["dense_blocks"] == 1
    sv.run(1)
    err = rel_l2(sv.read(), ref)
    print(f"selector block above the tile, {engine}: rel L2 {err:.3e}")
    assert err < tol
