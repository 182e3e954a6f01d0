"""Sweeps that stage qubits above the warp tile (the gate-vocabulary stream).

* The vocabulary microbenchmark stream at 24 qubits (1000 seeded gates: 1505
  records after the increments are written out as MCX cascades) against the
  oracle's tensor-axis naive simulator (O2), complex64 and complex128, in the
  launch configuration of the benchmark (fused, staged).  Tolerances: complex128
  1e-12 relative L2 (about 200 passes of at most 40 ops, 2^-53 each);
  complex64 1e-5 (2^-24 per op, the same count).
* Every staging width (CSIM_STAGE = 0..3, i.e. 1, 2, 4 and 8 tiles per warp)
  against the index-table simulator at 20 qubits, each in a fresh process
  (the switch is read once per process).
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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def stream24():
    n = 24
    gates = I.microbench_gates(n, 1000, 0)
    psi0 = I.random_unit_state(n, 0)
    ref = S.AxisSim(n).run(psi0.copy(), gates)
    return n, gates, psi0, ref


@pytest.mark.parametrize("prec,tol", [(G.CSIM_C128, 1e-12), (G.CSIM_C64, 1e-5)])
def test_vocabulary_stream_24_qubits_against_oracle(stream24, prec, tol):
    n, gates, psi0, ref = stream24
    sv = G.StateVector(n, prec)
    sv.load(psi0)
    sv.compile(G.gates_to_records(gates), G.CSIM_EXEC_FUSED)
    st = sv.stats()
    sv.run(1)
    err = rel_l2(sv.read(), ref)
    print(f"24-qubit vocabulary stream prec={prec}: {st['passes']} passes, rel L2 {err:.3e}")
    assert err < tol
    # staging fuses the stream into a fraction of the 1505 gates
    assert st["passes"] < 300


STAGE_SCRIPT = r'''
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import lbm_inputs as I, paper_2606_12770_gb300 as G
from oracle import statevec as S
from paper_2606_12770_gb300 import _native as N
n = 20
gates = I.microbench_gates(n, 400, 5)
psi = I.random_unit_state(n, 5)
ref = S.DenseSim(n).run(psi.copy(), gates)
_, fs = N.emulate_fused(gates, n, None)
for prec, tol in ((G.CSIM_C128, 1e-12), (G.CSIM_C64, 1e-5)):
    sv = G.StateVector(n, prec)
    sv.load(psi)
    sv.compile(G.gates_to_records(gates), G.CSIM_EXEC_FUSED)
    sv.run(1)
    err = np.linalg.norm(sv.read() - ref) / np.linalg.norm(ref)
    assert err < tol, (prec, err)
print("passes", fs["passes"], "staged", fs["staged_sweeps"], "ok")
'''


@pytest.mark.parametrize("k", ["0", "1", "2", "3"])
def test_every_staging_width(k):
    env = dict(os.environ, CSIM_STAGE=k)
    r = subprocess.run([sys.executable, "-c", STAGE_SCRIPT, ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
    staged = int(r.stdout.split("staged")[1].split()[0])
    assert (staged == 0) == (k == "0")


def test_autotune_picks_a_trial_and_keeps_the_state():
    """csim_sv_autotune times the stream at every staging width (and with
    dense blocks) on the loaded state, restores that state, and leaves the
    fastest program compiled: its result equals the oracle's."""
    n = 20
    gates = I.microbench_gates(n, 300, 8) + I.dense_block_gates(n, 4, 8)
    psi0 = I.random_unit_state(n, 8)
    ref = S.DenseSim(n).run(psi0.copy(), gates)
    sv = G.StateVector(n, G.CSIM_C64)
    sv.load(psi0)
    tune = sv.autotune(gates, reps=2)
    assert len(tune["trials"]) >= 5
    assert (tune["stage"], tune["dense"]) in [(t["stage"], t["dense"]) for t in tune["trials"]]
    assert tune["ms"] == min(t["ms"] for t in tune["trials"])
    assert np.array_equal(sv.read(), psi0.astype(np.complex64).astype(np.complex128))
    sv.run(1)
    assert rel_l2(sv.read(), ref) < 1e-4
