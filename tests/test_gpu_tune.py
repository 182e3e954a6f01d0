"""Launch-shape autotuner of the fused sweeps (csim_tune_launch) and the
per-class launch shapes it sets (csim_set_launch_shape).

* The tuner times candidate shapes on a scratch state, returns a valid choice
  with its trials (the default shape among them), and leaves the circuit's
  own state alone: a run after tuning equals the run before it within the
  precision's rounding (the chosen variant may be the general interpreter
  instead of the shaped op lists): 1e-12 relative in complex128, 1e-6 in
  complex64.
* Every kernel variant set directly gives the same result within the same
  tolerances, at the default grid and at one and eight waves.
* A sparse init followed by a tuned run still equals the plain run (the
  sweeps that complete the init keep the default variant).
Each test clears the shapes it set: they are process-wide.
"""
import numpy as np
import pytest

import lbm_inputs as I
import paper_2606_12770_gb300 as G

pytestmark = pytest.mark.gpu

CFG = (4, 0.8, 2, 2, 0.1, 2)  # 20 qubits


def _run(c, f0, prec):
    c.init(f0, prec)
    c.run()
    return c.postselect()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec,tol", [(G.CSIM_C128, 1e-12), (G.CSIM_C64, 1e-6)])
def test_tuner_choice_and_result(prec, tol):
    f0, _ = I.lbm_instance(CFG[0], 3, tau=CFG[1])
    c = G.Circuit(*CFG, kappa_qsvt=10.0, d=31)
    n = c.info()["n_qubits"]
    try:
        amps0, p0, t0 = _run(c, f0, prec)
        t = c.tune_launch(prec, max_steps=40, reps=2)
        print(f"tuned {n} qubits, precision {prec}: u {t['u']} minb {t['minb']} waves {t['waves']}, "
              f"{t['ms']:.3f} ms against {t['ms_default']:.3f} ms default, {len(t['trials'])} trials")
        assert 1 <= t["steps"] <= 40 and len(t["trials"]) >= 8
        assert t["ms"] <= t["ms_default"] and t["ms"] > 0
        assert (t["u"], t["minb"], t["waves"]) in {(x["u"], x["minb"], x["waves"]) for x in t["trials"]}
        amps, p, tot = _run(c, f0, prec)
        assert _rel(amps, amps0) < tol and abs(p - p0) <= tol * p0 and abs(tot - t0) < tol
    finally:
        G.set_launch_shape(prec, n, 0)
        c.close()


@pytest.mark.parametrize("prec,tol", [(G.CSIM_C128, 1e-12), (G.CSIM_C64, 1e-6)])
def test_every_shape_agrees(prec, tol):
    f0, _ = I.lbm_instance(CFG[0], 4, tau=CFG[1])
    c = G.Circuit(*CFG, kappa_qsvt=10.0, d=15)
    n = c.info()["n_qubits"]
    shapes = [(u, m, 4) for u in (1, 2, 4) for m in (1, 2, 4) if not (u == 4 and m == 4)]
    shapes += [(2, 4, 1), (1, 2, 8)]
    try:
        amps0, p0, t0 = _run(c, f0, prec)
        for u, m, w in shapes:
            G.set_launch_shape(prec, n, u, m, w)
            amps, p, tot = _run(c, f0, prec)
            assert _rel(amps, amps0) < tol, (u, m, w)
            assert abs(tot - t0) < tol, (u, m, w)
    finally:
        G.set_launch_shape(prec, n, 0)
        c.close()


def test_bad_shapes_rejected():
    for args in [(G.CSIM_C64, 20, 4, 4, 4), (G.CSIM_C64, 20, 3, 2, 4), (G.CSIM_C64, 20, 2, 2, 0),
                 (G.CSIM_C64, 3, 2, 2, 4)]:
        with pytest.raises(G.CsimError):
            G.set_launch_shape(*args)
