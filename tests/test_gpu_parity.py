"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (derived from the arithmetic of each path):
  * complex128, truncated d, full state vs the naive simulator: 1e-12 relative L2;
  * complex64, full state: 1e-4 relative L2 (the complex64 bound), expected ~1e-6;
  * complex128 at the full QSVT degree, postselected block vs the classical
    evaluator: rounding grows with the number of gate applications G as about
    G * 2^-53 on a unit-norm state, relative to the block norm sqrt(p).
"""
import math

import numpy as np
import pytest

import lbm_inputs as I
import paper_2606_12770_gb300 as G
from oracle import circuit as OC
from oracle import qsvt as Q
from oracle import statevec as S
from oracle.layout import Layout

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_full_state(cfg, f0, phases):
    Nx, tau, NC, K, dt, Nt = cfg
    lay = Layout(Nx, NC, K, Nt)
    psi = np.zeros(1 << lay.n, dtype=complex)
    init, _ = OC.initial_state(lay, f0)
    for k, v in init.items():
        psi[k] = v
    S.DenseSim(lay.n).run(psi, OC.build_qsvt(*cfg, list(phases)))
    return psi, lay


def gpu_full_state(cfg, f0, phases, prec, mode):
    c = G.Circuit(*cfg, phases=phases)
    c.set_exec(mode)
    c.init(f0, prec)
    c.run()
    return c.read_state(), c


C1 = (4, 0.8, 2, 2, 0.1, 2)
SMALL = [((2, 0.8, 1, 1, 0.1, 1), 3), ((4, 0.8, 1, 2, 0.1, 2), 5), ((8, 0.7, 1, 3, 0.2, 3), 3),
         ((2, 1.1, 2, 3, 0.1, 2), 3), ((4, 0.6, 2, 1, 0.15, 3), 1)]


@pytest.mark.parametrize("d", [1, 3])
@pytest.mark.parametrize("mode", [G.CSIM_EXEC_FUSED, G.CSIM_EXEC_GATE])
def test_c1_full_state_c128(d, mode):
    f0, _ = I.lbm_instance(4, 0, tau=0.8)
    ph = I.random_phases(d, 100 + d)
    ref, lay = oracle_full_state(C1, f0, ph)
    got, c = gpu_full_state(C1, f0, ph, G.CSIM_C128, mode)
    assert rel_l2(got, ref) < 1e-12
    amps, p, tot = c.postselect()
    assert abs(tot - 1.0) < 1e-12


@pytest.mark.parametrize("cfg,d", SMALL)
def test_small_configs_full_state_c128_and_c64(cfg, d):
    f0, _ = I.lbm_instance(cfg[0], 5, tau=cfg[1])
    ph = I.random_phases(d, 7)
    ref, lay = oracle_full_state(cfg, f0, ph)
    got, _ = gpu_full_state(cfg, f0, ph, G.CSIM_C128, G.CSIM_EXEC_FUSED)
    assert rel_l2(got, ref) < 1e-12
    got64, _ = gpu_full_state(cfg, f0, ph, G.CSIM_C64, G.CSIM_EXEC_FUSED)
    assert rel_l2(got64, ref) < 1e-4


def _postselected_reference(cfg, f0, phases, bc="periodic"):
    y, lay, M, b = Q.qsvt_postselected(*cfg, f0, phases, bc)
    final = Q.final_slot_mask(lay)
    phys = lay.physical_indices()
    return y, lay, phys, final


def _gpu_postselected_by_index(c, lay):
    amps, p, tot = c.postselect()
    free_shift = 2 + lay.niL
    m_shift = lay.regs["m"][0]
    free_bits = m_shift - free_shift
    return amps, p, tot, free_shift, free_bits, m_shift


def _compare_postselect(c, cfg, f0, phases, bc="periodic"):
    """Errors of the GPU postselected block against the classical evaluator.

    Returns (max abs error of the physical entries on the unit-norm state,
    relative L2 error of the block, relative error of p, max |non-physical
    entry|, total norm, p_ref)."""
    y, lay, phys, final = _postselected_reference(cfg, f0, phases, bc)
    amps, p, tot, free_shift, free_bits, m_shift = _gpu_postselected_by_index(c, lay)
    sel = phys[final]
    m = sel >> m_shift
    f = (sel >> free_shift) & ((1 << free_bits) - 1)
    pos = ((m - lay.Nt) << free_bits) + f
    got = amps[pos]
    ref = y[final]
    p_ref = float(np.sum(ref * ref))
    mask = np.ones(amps.shape[0], dtype=bool)
    mask[pos] = False
    leak = float(np.max(np.abs(amps[mask]), initial=0.0))
    return (float(np.max(np.abs(got - ref))), rel_l2(got, ref), abs(p - p_ref) / p_ref, leak, tot,
            p_ref)


GOLDEN_PHASES = np.loadtxt(__import__("os").path.join(
    __import__("os").path.dirname(__file__), "golden", "phases_k10_d31.txt"))


@pytest.mark.parametrize("prec,abs_tol", [(G.CSIM_C128, 1e-13), (G.CSIM_C64, 1e-6)])
@pytest.mark.parametrize("mode", [G.CSIM_EXEC_FUSED, G.CSIM_EXEC_GATE])
def test_c1_postselect_truncated(prec, abs_tol, mode):
    """1/x phases fitted by the oracle (kappa_QSVT = 10, d = 31) on the 20-qubit circuit."""
    f0, _ = I.lbm_instance(4, 0, tau=0.8)
    c = G.Circuit(*C1, phases=GOLDEN_PHASES)
    c.set_exec(mode)
    c.init(f0, prec)
    c.run()
    e_abs, e_rel, e_p, leak, tot, p_ref = _compare_postselect(c, C1, f0, GOLDEN_PHASES)
    print(f"prec {prec} mode {mode}: abs {e_abs:.2e} block-rel {e_rel:.2e} p-rel {e_p:.2e} "
          f"leak {leak:.2e} p {p_ref:.3e}")
    assert e_abs < abs_tol and leak < abs_tol
    assert abs(tot - 1.0) < (1e-12 if prec == G.CSIM_C128 else 1e-5)
    if prec == G.CSIM_C128:
        assert e_rel < 1e-9


@pytest.mark.parametrize("prec,abs_tol", [(G.CSIM_C128, 1e-13), (G.CSIM_C64, 1e-6)])
def test_bounceback_postselect_truncated(prec, abs_tol):
    """The walled circuit (reading R2) against the classical evaluator of the
    walled L, on the 20-qubit configuration with the oracle-fitted 1/x phases;
    and its full state against the naive simulator of the oracle's walled
    gate list."""
    f0, _ = I.lbm_instance(4, 0, tau=0.8)
    c = G.Circuit(*C1, phases=GOLDEN_PHASES, bc="bounceback")
    c.init(f0, prec)
    c.run()
    e_abs, e_rel, e_p, leak, tot, p_ref = _compare_postselect(c, C1, f0, GOLDEN_PHASES,
                                                              "bounceback")
    print(f"bounce-back prec {prec}: abs {e_abs:.2e} block-rel {e_rel:.2e} p {p_ref:.3e}")
    assert e_abs < abs_tol and leak < abs_tol
    assert abs(tot - 1.0) < (1e-12 if prec == G.CSIM_C128 else 1e-5)
    if prec == G.CSIM_C128:
        ph = I.random_phases(3, 11)
        cfg = (2, 1.1, 2, 3, 0.1, 2)
        lay = Layout(2, 2, 3, 2)
        f2, _ = I.lbm_instance(2, 1, tau=1.1)
        psi = np.zeros(1 << lay.n, dtype=complex)
        for k, v in OC.initial_state(lay, f2)[0].items():
            psi[k] = v
        S.DenseSim(lay.n).run(psi, OC.build_qsvt(*cfg, list(ph), bc="bounceback"))
        c2 = G.Circuit(*cfg, phases=ph, bc="bounceback")
        c2.init(f2, G.CSIM_C128)
        c2.run()
        assert rel_l2(c2.read_state(), psi) < 1e-12


def test_c1_full_degree_postselect_c128():
    """Full Eq. d-star degree (d = 1957) with the build's own kappa and phases.

    Two checks: the GPU block equals the classical evaluation of the same
    phases, and (oracle only) it equals scale * lambda_L * L^{-1} b within the
    residual bound of the 1/x polynomial."""
    f0, _ = I.lbm_instance(4, 0, tau=0.8)
    c = G.Circuit(*C1)
    inf = c.info()
    assert inf["d"] == 1957
    ph = c.export_phases()
    c.init(f0, G.CSIM_C128)
    c.run()
    e_abs, e_amp, e_p, leak, tot, p_ref = _compare_postselect(c, C1, f0, ph)
    G_gates = inf["n_gates_total"]
    bound = 50 * G_gates * 2.0 ** -53 / math.sqrt(p_ref)
    print(f"full-degree c128: rel L2 {e_amp:.3e}, p rel {e_p:.3e}, bound {bound:.3e}, p {p_ref:.3e}")
    assert e_amp < bound and abs(tot - 1.0) < 1e-9
    # physics: the final-time block is scale * lambda_L * L^{-1} b up to the
    # polynomial's residual 1/T_n(z0) (Sec. II.D.5; classical forward substitution)
    from oracle import physics as P
    A = P.carleman_A(4, 0.8, 2)
    L = P.l_matrix(A, 0.1, 2, 2)
    vec = P.carleman_vector(np.asarray(f0).reshape(-1), 2)
    b = P.rhs_vector(vec / np.linalg.norm(vec), 2, 2)
    x = inf["poly_scale"] * inf["lambda_L"] * P.solve_l(L, b)
    y, lay, phys, final = _postselected_reference(C1, f0, ph)
    a = 1.0 / inf["kappa_qsvt"]
    delta = 1.0 / math.cosh(((inf["d"] + 1) // 2) * math.acosh((1 + a * a) / (1 - a * a)))
    amps, p, tot = c.postselect()
    sel = phys[final]
    fs, ms = 2 + lay.niL, lay.regs["m"][0]
    pos = ((sel >> ms) - lay.Nt) * (1 << (ms - fs)) + ((sel >> fs) & ((1 << (ms - fs)) - 1))
    phys_err = rel_l2(amps[pos].real, x[final])
    print(f"QSVT vs classical Taylor solve at T: rel L2 {phys_err:.3e} (polynomial residual {delta:.3e})")
    assert phys_err < 1.01 * delta


def _random_gates(n, count, seed, high_h=True):
    rng = np.random.default_rng(seed)
    g = []
    for _ in range(count):
        op = int(rng.integers(0, 4))
        t = int(rng.integers(n)) if (high_h or op == 0) else int(rng.integers(min(n, 7)))
        others = [b for b in range(n) if b != t]
        nc = int(rng.integers(0, 5))
        cs = rng.choice(others, nc, replace=False) if nc else []
        cm = sum(1 << int(c) for c in cs)
        cv = sum(int(rng.integers(2)) << int(c) for c in cs)
        ang = float(rng.uniform(-math.pi, math.pi)) if op in (2, 3) else 0.0
        g.append((op, t, cm, cv, ang, 0))
    return g


@pytest.mark.parametrize("n,seed", [(5, 1), (7, 2), (12, 3), (16, 4)])
@pytest.mark.parametrize("mode", [G.CSIM_EXEC_FUSED, G.CSIM_EXEC_GATE])
def test_random_gate_lists(n, seed, mode):
    gates = _random_gates(n, 120, seed)
    psi0 = I.random_unit_state(n, seed)
    ref = S.DenseSim(n).run(psi0.copy(), gates)
    for prec, tol in ((G.CSIM_C128, 1e-12), (G.CSIM_C64, 1e-5)):
        sv = G.StateVector(n, prec)
        sv.load(psi0)
        sv.compile(gates, mode)
        sv.run(1)
        assert rel_l2(sv.read(), ref) < tol


def test_microbench_vocabulary_parity():
    """The gate-vocabulary microbenchmark stream at n = 20, checked against O2."""
    n = 20
    gates = I.microbench_gates(n, 300, 0)
    psi0 = I.random_unit_state(n, 0)
    ref = S.DenseSim(n).run(psi0.copy(), gates)
    for prec, tol in ((G.CSIM_C128, 1e-12), (G.CSIM_C64, 1e-5)):
        sv = G.StateVector(n, prec)
        sv.load(psi0)
        sv.compile(gates, G.CSIM_EXEC_FUSED)
        sv.run(1)
        assert rel_l2(sv.read(), ref) < tol


def test_empty_program_and_reuse():
    n = 9
    psi0 = I.random_unit_state(n, 9)
    sv = G.StateVector(n, G.CSIM_C128)
    sv.load(psi0)
    sv.compile([], G.CSIM_EXEC_FUSED)
    sv.run(3)
    assert np.array_equal(sv.read(), psi0)
    gates = _random_gates(n, 40, 9)
    sv.compile(gates, G.CSIM_EXEC_FUSED)
    sv.run(2)
    ref = S.DenseSim(n).run(S.DenseSim(n).run(psi0.copy(), gates), gates)
    assert rel_l2(sv.read(), ref) < 1e-12


def test_state_machine_errors():
    f0, _ = I.lbm_instance(4, 0, tau=0.8)
    c = G.Circuit(*C1, phases=I.random_phases(5, 0))
    c.init(f0, G.CSIM_C64)
    c.run()
    with pytest.raises(G.CsimError) as e:
        c.run()
    assert e.value.status == -5
    c.init(f0, G.CSIM_C64)  # re-init reuses the allocation
    c.run()
    _, p, tot = c.postselect(False)
    assert 0.0 < p < 1.0 and abs(tot - 1.0) < 1e-5
    with pytest.raises(G.CsimError):
        c.init(np.full((4, 3), np.nan), G.CSIM_C64)


VARIANT_SCRIPT = r'''
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import lbm_inputs as I, paper_2606_12770_gb300 as G
from oracle import statevec as S, circuit as OC
from oracle.layout import Layout
cfg = (4, 0.8, 2, 2, 0.1, 2)
lay = Layout(4, 2, 2, 2)
f0, _ = I.lbm_instance(4, 0, tau=0.8)
ph = I.random_phases(5, 2)
gates = OC.build_qsvt(*cfg, list(ph))
psi = np.zeros(1 << lay.n, dtype=complex)
init, _ = OC.initial_state(lay, f0)
for k, v in init.items():
    psi[k] = v
ref = S.DenseSim(lay.n).run(psi.copy(), gates)
for prec, tol in ((G.CSIM_C128, 1e-12), (G.CSIM_C64, 1e-5)):
    sv = G.StateVector(lay.n, prec)
    sv.load(psi)
    sv.compile(gates, G.CSIM_EXEC_FUSED)
    sv.run(1)
    err = np.linalg.norm(sv.read() - ref) / np.linalg.norm(ref)
    assert err < tol, (prec, err)
print("ok")
'''


def _variant_cases():
    """The launch variants worth running: every (tiles per iteration, blocks
    per SM) variant in both forms with four resident waves; single-wave grids
    on three variants; the lookup-table chain on the default gather variant;
    separate permutation sweeps (no conjugation) on the two default
    variants."""
    cfgs = ["1,1", "2,1", "4,1", "1,2", "2,2", "4,2", "1,4", "2,4"]
    out = []
    for form in ("gather", "scatter"):
        for cfg in cfgs:
            out.append((cfg, form, "4", "1", "1"))
        for cfg in ("1,4", "2,4", "4,2"):
            out.append((cfg, form, "1", "1", "1"))
    out.append(("2,4", "gather", "4", "0", "1"))
    out.append(("2,4", "gather", "1", "0", "1"))
    out.append(("2,4", "gather", "4", "1", "0"))
    out.append(("1,2", "gather", "4", "1", "0"))
    out.append(("2,4", "gather", "4", "0", "0"))
    return out


@pytest.mark.parametrize("cfg,form,waves,src,conj", _variant_cases())
def test_sweep_kernel_variants(cfg, form, waves, src, conj):
    """Every compiled sweep-kernel variant (tiles per iteration, blocks per SM,
    form); one resident wave makes each warp loop over several tiles at 20
    qubits.  Gather sweeps run with source-index tables and, on the default
    variant, with the lookup-table chain; the default variants also run with
    the permutation pairs as separate gathers instead of in-place conjugated
    sweeps."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CSIM_SWEEP_CFG=cfg, CSIM_SWEEP_FORM=form, CSIM_SWEEP_WAVES=waves,
               CSIM_SRC_INDEX=src, CSIM_CONJUGATE=conj)
    r = subprocess.run([sys.executable, "-c", VARIANT_SCRIPT, root], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


SRC_SCRIPT = r'''
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import lbm_inputs as I, paper_2606_12770_gb300 as G
ph = np.loadtxt(sys.argv[1] + "/tests/golden/phases_k10_d31.txt")
f0, _ = I.lbm_instance(4, 0, tau=0.8)
out = {}
for name, prec in (("c128", G.CSIM_C128), ("c64", G.CSIM_C64)):
    c = G.Circuit(4, 0.8, 2, 2, 0.1, 2, phases=ph)
    c.init(f0, prec)
    c.run()
    out[name] = c.read_state()
    out[name + "_tables"] = np.array(c.info()["n_src_tables"])
np.savez(sys.argv[2], **out)
print("ok")
'''


def test_source_index_tables_equal_lookup_chain(tmp_path):
    """The gather sweeps give the same state, bit for bit, whether they load the
    precomputed source index of each chunk or walk the lookup-table chain (the
    same index, the same arithmetic), with the indices loaded one iteration
    ahead or not, with four or two tiles per warp iteration in the averaging
    sweeps, and in the scatter form (destination indices); the table
    path is the one in use by default (one table: the U_L^dag chain, which the
    conjugated sweeps and the last gather share).  The kernels specialised on
    the sweep shape agree with the generic op interpreter within rounding."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    modes = {"chain": ("0", "1", "gather", "1"), "src-nopre": ("1", "0", "gather", "1"),
             "default": ("1", "1", "gather", "1"), "chain-scatter": ("0", "1", "scatter", "1"),
             "scatter": ("1", "1", "scatter", "1"), "generic": ("1", "1", "gather", "0"),
             "avg-2,4": ("1", "1", "gather", "1")}
    for name, (flag, pre, form, shapes) in modes.items():
        path = str(tmp_path / f"{name}.npz")
        env = dict(os.environ, CSIM_SRC_INDEX=flag, CSIM_SRC_PREFETCH=pre, CSIM_SWEEP_FORM=form,
                   CSIM_SWEEP_SHAPES=shapes)
        if name == "avg-2,4":
            env["CSIM_AVG_CFG"] = "2,4"
        else:
            env.pop("CSIM_AVG_CFG", None)
        r = subprocess.run([sys.executable, "-c", SRC_SCRIPT, root, path], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
        res[name] = np.load(path)
    assert int(res["chain"]["c128_tables"]) == 0 and int(res["default"]["c128_tables"]) == 1
    for prec in ("c128", "c64"):
        assert np.array_equal(res["chain"][prec], res["default"][prec]), prec
        assert np.array_equal(res["src-nopre"][prec], res["default"][prec]), prec
        assert np.array_equal(res["chain-scatter"][prec], res["scatter"][prec]), prec
        # four tiles per warp iteration in the averaging sweeps (the default)
        # or two: the same arithmetic per tile
        assert np.array_equal(res["avg-2,4"][prec], res["default"][prec]), prec
        # shaped kernels against the generic op interpreter: the same operations,
        # compiled in other instantiations (contraction may differ)
        a, b = res["default"][prec], res["generic"][prec]
        tol = 1e-14 if prec == "c128" else 1e-6
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < tol, prec


SPARSE_SCRIPT = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import lbm_inputs as I, paper_2606_12770_gb300 as G
ph = np.loadtxt(sys.argv[1] + "/tests/golden/phases_k10_d31.txt")
f0, _ = I.lbm_instance(4, 0, tau=0.8)
out = {}
for name, prec in (("c128", G.CSIM_C128), ("c64", G.CSIM_C64)):
    c = G.Circuit(4, 0.8, 2, 2, 0.1, 2, phases=ph)
    c.init(f0, prec)
    out[name + "_sparse"] = np.array(c.info()["sparse_init"])
    out[name + "_b"] = c.read_state()           # read before the first sweep
    c.init(f0, prec)
    c.run()
    out[name + "_final"] = c.read_state()
    c.init(f0, prec)                             # stepped run with a checkpoint
    c.run_steps(1)
    out[name + "_ck"] = c.checkpoint()[0]
    c.run()
    out[name + "_stepped"] = c.read_state()
    c.init(f0, prec)                             # the two leading sweeps one by one
    c.run_steps(1)
    c.run_steps(1)
    out[name + "_ck2"] = c.checkpoint()[0]
    c.run()
    out[name + "_stepped2"] = c.read_state()
    c.init(f0, prec)                             # postselection before any sweep
    a, p, t = c.postselect()
    out[name + "_post0"] = np.array([p, t])
    c.init(f0, prec)                             # the mode changes after csim_init
    c.set_exec(G.CSIM_EXEC_GATE)
    c.run()
    out[name + "_gate"] = c.read_state()
np.savez(sys.argv[2], **out)
print("ok")
"""


def test_sparse_init_is_invisible(tmp_path):
    """csim_init that writes only the tiles of b (the first in-place sweep
    leaves the other tiles unwritten and the first conjugated gather reads
    zeros for them) gives, bit for bit, the states of the whole zero-filled
    init: after a full run, after one or two steps and a checkpoint, when the
    state is read or postselected before any sweep, and when the execution
    mode changes between init and run."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    for name, flag in (("sparse", "1"), ("whole", "0")):
        path = str(tmp_path / f"{name}.npz")
        env = dict(os.environ, CSIM_SPARSE_INIT=flag)
        r = subprocess.run([sys.executable, "-c", SPARSE_SCRIPT, root, path], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
        res[name] = np.load(path)
    for prec in ("c128", "c64"):
        # the first sweep and the first conjugated gather complete the zeros
        assert int(res["sparse"][prec + "_sparse"]) == 2, prec
        assert int(res["whole"][prec + "_sparse"]) == 0, prec
        for key in ("_b", "_final", "_ck", "_stepped", "_ck2", "_stepped2", "_post0", "_gate"):
            assert np.array_equal(res["sparse"][prec + key], res["whole"][prec + key]), prec + key
        b = res["sparse"][prec + "_b"]
        assert abs(np.linalg.norm(b) - 1.0) < 1e-6
        assert 0 < np.count_nonzero(b) < b.size // 64


AVG_SCRIPT = r"""
import sys, hashlib, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import lbm_inputs as I, paper_2606_12770_gb300 as G
Nx = int(sys.argv[2])
f0, tau = I.lbm_instance(Nx, 1, tau=None, tau_range=(0.6, 1.2))
c = G.Circuit(Nx, tau, 2, 4, 0.1, 16, kappa_qsvt=1000.0, d=13)
c.init(f0, G.CSIM_C64, torch.cuda.current_stream())
c.run()
_, p, t = c.postselect(want_amplitudes=False)
x = torch.as_tensor(c.device_state(), device="cuda")
h = hashlib.sha256()
for i in range(0, x.shape[0], 1 << 26):
    h.update(x[i:i + (1 << 26)].cpu().numpy().tobytes())
np.savez(sys.argv[3], pt=np.array([p, t]), digest=np.frombuffer(h.digest(), dtype=np.uint8))
print("ok")
"""


@pytest.mark.parametrize("Nx", [8, 32])
def test_averaging_sweep_launch_shapes_agree(tmp_path, Nx):
    """The conjugated averaging sweeps of the precision circuit give the same
    final state, bit for bit (a SHA-256 of the whole complex64 state), with
    four tiles per warp iteration (the default) and with two
    (CSIM_AVG_CFG=2,4): at 26 qubits in the natural tile order and at 30
    qubits with four fast tile bits."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    for name, cfg in (("four", None), ("two", "2,4")):
        path = str(tmp_path / f"{name}.npz")
        env = dict(os.environ)
        env.pop("CSIM_AVG_CFG", None)
        if cfg:
            env["CSIM_AVG_CFG"] = cfg
        r = subprocess.run([sys.executable, "-c", AVG_SCRIPT, root, str(Nx), path], env=env,
                           capture_output=True, text=True, timeout=900)
        assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
        res[name] = np.load(path)
    assert np.array_equal(res["four"]["digest"], res["two"]["digest"])
    assert np.array_equal(res["four"]["pt"], res["two"]["pt"])
    # unitary circuit: the total norm stays 1 (complex64 rounding)
    assert abs(res["four"]["pt"][1] - 1.0) < 1e-4
