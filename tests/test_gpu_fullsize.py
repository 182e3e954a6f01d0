"""Parity at the full benchmark sizes, in the launch configuration the bench times.

* The 32-qubit precision circuit (Nx=64, N_C=2, K=4, Nt=16, d=13), complex64 and
  complex128.  Every physical entry with s = t = label = 0 (all time slots,
  9.5 million amplitudes) is compared with the classical QSVT evaluator of the
  oracle on the same phases.  The phases are the oracle-fitted 1/x phases for
  kappa_QSVT = 1000, d = 13.  The whole-state norm is checked as well.
  Tolerances: complex64 1e-4 relative L2 (the complex64 bound); complex128 1e-11
  (about 5e3 gate applications at 2^-53 each).
* The vocabulary microbenchmark at 30 and 33 qubits (complex64), from a seeded
  random state.  Properties that hold at any size are checked: the stream
  followed by its inverse returns the initial state, and at 30 qubits the fused
  and the gate-by-gate executors agree.
"""
import math
import os

import numpy as np
import pytest

import lbm_inputs as I
import paper_2606_12770_gb300 as G
from oracle import qsvt as Q
from oracle.layout import Layout

HERE = os.path.dirname(os.path.abspath(__file__))
C2 = dict(Nx=64, N_C=2, K=4, Nt=16, dt=0.1)
PHASES_C2 = np.loadtxt(os.path.join(HERE, "golden", "phases_k1000_d13.txt"))


def physical_indices_fast(lay):
    """Vectorised physical index table, equal to Layout.physical_indices()."""
    D = lay.carleman_dim()
    base = np.array([lay.embed_index(0, j) for j in range(D)], dtype=np.int64)
    slots = np.arange(lay.n_slots())
    off = np.array([lay.place(k=int(s) & ((1 << lay.nk) - 1), m=int(s) >> lay.nk) for s in slots],
                   dtype=np.int64)
    return (off[:, None] | base[None, :]).reshape(-1)


def test_fast_physical_indices_match_layout():
    for args in ((4, 2, 2, 2), (8, 2, 3, 5), (4, 1, 4, 3)):
        lay = Layout(*args)
        assert np.array_equal(physical_indices_fast(lay), lay.physical_indices())


def _sample(ds, idx):
    import torch
    t = torch.as_tensor(ds, device="cuda")
    sel = t[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    return sel[:, 0] + 1j * sel[:, 1]


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [(G.CSIM_C64, 1e-4), (G.CSIM_C128, 1e-11)])
def test_precision_circuit_full_size(prec, tol):
    torch = pytest.importorskip("torch")
    f0, tau = I.lbm_instance(C2["Nx"], 1, tau_range=(0.6, 1.2))
    cfg = (C2["Nx"], tau, C2["N_C"], C2["K"], C2["dt"], C2["Nt"])
    c = G.Circuit(*cfg, phases=PHASES_C2)
    assert c.info()["n_qubits"] == 32
    c.init(f0, prec, torch.cuda.current_stream())
    c.run()
    _, p, tot = c.postselect(want_amplitudes=False)
    assert abs(tot - 1.0) < (1e-5 if prec == G.CSIM_C64 else 1e-12)
    # d = 13 calls cannot reach the slots m >= Nt = 16 from b: the final block is 0
    assert p == 0.0
    y, lay, _, _ = Q.qsvt_postselected(*cfg, f0, PHASES_C2)
    idx = physical_indices_fast(lay)
    got = _sample(c.device_state(), idx)
    err = float(np.linalg.norm(got - y) / np.linalg.norm(y))
    print(f"32-qubit precision circuit prec={prec}: rel L2 over {idx.size} physical entries "
          f"{err:.3e}; block norm^2 {float(np.sum(y * y)):.4e}")
    assert err < tol


def _inverse(gates):
    out = []
    for op, t, cm, cv, ang, tag in reversed(gates):
        out.append((op, t, cm, cv, -ang if op in (2, 3) else ang, tag))
    return out


def _rel_l2_device(torch, a, b, chunk=1 << 26):
    """||a - b|| / ||b|| in FP64, chunked so no state-sized temporary is made."""
    num = 0.0
    den = 0.0
    for i in range(0, a.shape[0], chunk):
        da = a[i:i + chunk].double()
        db = b[i:i + chunk].double()
        num += float(torch.sum((da - db) ** 2))
        den += float(torch.sum(db * db))
    return math.sqrt(num / den)


def _random_device_state(torch, n, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    x = torch.randn((1 << n, 2), generator=g, device="cuda", dtype=torch.float32)
    x /= torch.linalg.vector_norm(x)
    return x


@pytest.mark.gpu
@pytest.mark.parametrize("n", [30, 33])
def test_microbench_full_size_inverse_round_trip(n):
    torch = pytest.importorskip("torch")
    free, _ = torch.cuda.mem_get_info()
    need = 3 * (8 << n) + (1 << 30)
    if free < need:
        pytest.skip(f"needs {need / 2**30:.0f} GiB free, {free / 2**30:.0f} GiB available")
    gates = I.microbench_gates(n, 1000, 0)
    x = _random_device_state(torch, n, 0)
    sv = G.StateVector(n, G.CSIM_C64, torch.cuda.current_stream())
    sv.load_device(x.data_ptr())
    sv.compile(gates, G.CSIM_EXEC_FUSED)
    sv.run()
    fwd_info = sv.info()
    sv.compile(_inverse(gates), G.CSIM_EXEC_FUSED)
    sv.run()
    torch.cuda.synchronize()
    back = torch.as_tensor(sv.device_state(), device="cuda")
    err = _rel_l2_device(torch, back, x)
    print(f"n={n}: fused passes {fwd_info['n_sweeps']}, round-trip rel L2 {err:.3e}")
    assert err < 1e-4
    assert math.isfinite(err)


@pytest.mark.gpu
def test_microbench_30_fused_equals_gate_by_gate():
    torch = pytest.importorskip("torch")
    n = 30
    gates = I.microbench_gates(n, 1000, 0)
    x = _random_device_state(torch, n, 1)
    st = torch.cuda.current_stream()
    sf = G.StateVector(n, G.CSIM_C64, st)
    sf.load_device(x.data_ptr())
    sf.compile(gates, G.CSIM_EXEC_FUSED)
    sf.run()
    torch.cuda.synchronize()
    fused = torch.as_tensor(sf.device_state(), device="cuda").clone()
    sf.close()
    sg = G.StateVector(n, G.CSIM_C64, st)
    sg.load_device(x.data_ptr())
    sg.compile(gates, G.CSIM_EXEC_GATE)
    sg.run()
    torch.cuda.synchronize()
    plain = torch.as_tensor(sg.device_state(), device="cuda")
    err = _rel_l2_device(torch, fused, plain)
    print(f"n=30 fused vs gate-by-gate rel L2 {err:.3e}")
    assert err < 1e-5
