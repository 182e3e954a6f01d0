"""Checkpointed and long QSVT runs.

* A run split into step ranges with a checkpoint round trip through the host
  into a second handle gives the same final state as one csim_run, bit for bit
  (complex128 and complex64; the kernels are deterministic).
* The paper's walled N_C = 1 run of Sec. III.E.3 (Nx = 32, K = 1, dt = 0.04375,
  Nt = 128, nu = 2): kappa(L) = 3283 as printed, d = 25771 from Eq. d-star with
  eps = 1e-3, phases from the fixed-point solver.  The run goes through ten
  checkpointed chunks in complex128.  Its postselected block equals the
  classical evaluation of the same phases within 50 G 2^-53 / sqrt(p) (G the
  gate applications), and scale * lambda_L * L^{-1} b within the polynomial's
  residual bound (Sec. II.D.5).
"""
import math
import os
import time

import numpy as np
import pytest

import lbm_inputs as I
import paper_2606_12770_gb300 as G
from oracle import physics as P
from oracle import qsvt as Q

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
C1 = (4, 0.8, 2, 2, 0.1, 2)
PH31 = np.loadtxt(os.path.join(HERE, "golden", "phases_k10_d31.txt"))


@pytest.mark.parametrize("prec", [G.CSIM_C128, G.CSIM_C64])
def test_checkpointed_run_equals_plain_run(prec):
    f0, _ = I.lbm_instance(4, 0, tau=0.8)
    a = G.Circuit(*C1, phases=PH31)
    a.init(f0, prec)
    a.run()
    ref = a.read_state()
    total = a.info()["n_sweeps_run"]
    assert total > 12
    b = G.Circuit(*C1, phases=PH31)
    b.init(f0, prec)
    assert b.run_steps(5) == 5
    psi, nxt = b.checkpoint()
    assert nxt == 5
    b.close()
    c = G.Circuit(*C1, phases=PH31)
    c.restore(psi, nxt, prec)
    assert c.run_steps(7) == 12
    c.run()  # finishes the run that run_steps started
    assert np.array_equal(c.read_state(), ref)
    with pytest.raises(G.CsimError):
        c.run_steps(1)  # the run is complete


def test_paper_long_run_nc1_checkpointed():
    Nx = 32
    tau = P.tau_from_nu(Nx, 2.0)
    cfg = (Nx, tau, 1, 1, 0.04375, 128)
    t0 = time.perf_counter()
    c = G.Circuit(*cfg, bc="bounceback")
    inf = c.info()
    t_build = time.perf_counter() - t0
    assert abs(inf["kappa_qsvt"] - 3283.0) / 3283.0 < 5e-3
    d = inf["d"]
    assert d == Q.degree_from_kappa(inf["kappa_qsvt"], 1e-3)
    ph = c.export_phases()
    f0, _ = I.lbm_instance(Nx, 0, tau=tau)
    c.init(f0, G.CSIM_C128)
    assert c.run_steps(0) == 0  # fuses the program, runs nothing
    total = c.info()["n_sweeps_run"]
    assert total >= d  # one fused sweep per U_L call
    chunk = total // 10 + 1
    t0 = time.perf_counter()
    nxt = c.run_steps(chunk)
    psi, nxt = c.checkpoint()
    c.restore(psi, nxt, G.CSIM_C128)
    while nxt < total:
        nxt = c.run_steps(chunk)
    c.sync()
    t_run = time.perf_counter() - t0
    amps, p, tot = c.postselect()
    print(f"long run: d={d}, {total} steps, build {t_build:.1f} s, GPU run {t_run:.2f} s, "
          f"p={p:.3e}")
    assert abs(tot - 1.0) < 1e-9
    # the classical evaluation of the same phases (O5)
    y, lay, M, b = Q.qsvt_postselected(*cfg, f0, ph, "bounceback")
    final = Q.final_slot_mask(lay)
    phys = lay.physical_indices()
    sel = phys[final]
    fs, ms = 2 + lay.niL, lay.regs["m"][0]
    pos = ((sel >> ms) - lay.Nt) * (1 << (ms - fs)) + ((sel >> fs) & ((1 << (ms - fs)) - 1))
    got = amps[pos]
    ref = y[final]
    p_ref = float(np.sum(ref * ref))
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    bound = 50 * inf["n_gates_total"] * 2.0 ** -53 / math.sqrt(p_ref)
    print(f"long run vs O5: rel L2 {err:.3e} (bound {bound:.3e}), p_ref {p_ref:.3e}")
    assert err < bound
    # physics: scale * lambda_L * L^{-1} b within the residual of the 1/x polynomial
    A = P.carleman_A(Nx, tau, 1, "bounceback")
    L = P.l_matrix(A, cfg[4], cfg[3], cfg[5])
    vec = P.carleman_vector(np.asarray(f0).reshape(-1), 1)
    bb = P.rhs_vector(vec / np.linalg.norm(vec), cfg[3], cfg[5])
    x = inf["poly_scale"] * inf["lambda_L"] * P.solve_l(L, bb)
    a = 1.0 / inf["kappa_qsvt"]
    delta = 1.0 / math.cosh(((d + 1) // 2) * math.acosh((1 + a * a) / (1 - a * a)))
    phys_err = float(np.linalg.norm(got.real - x[final]) / np.linalg.norm(x[final]))
    print(f"long run vs classical Taylor solve: rel L2 {phys_err:.3e} (residual {delta:.3e})")
    assert phys_err < 1.01 * delta
