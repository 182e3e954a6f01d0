"""Host-side (no GPU) tests of the C-ABI library: symbols, gate lists, masks, phases."""
import math
import os
import re
import struct

import numpy as np
import pytest

import paper_2606_12770_gb300 as G
from paper_2606_12770_gb300 import _native as N
from oracle import circuit as OC
from oracle import physics as P
from oracle import qsvt as Q
from oracle.layout import Layout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_header_symbol():
    lib = G.load()
    header = open(os.path.join(ROOT, "include", "csim.h")).read()
    declared = set(re.findall(r"\b(csim_[a-z_]+)\s*\(", header))
    assert declared == set(N.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name


def _same_gate(a, b):
    return ((int(a["op"]), int(a["target"]), int(a["cmask"]), int(a["cval"]), int(a["tag"]))
            == (b[0], b[1], b[2], b[3], b[5])
            and struct.pack("<d", float(a["angle"])) == struct.pack("<d", b[4]))


CONFIGS = [(4, 0.8, 2, 2, 0.1, 2), (64, 0.93, 2, 4, 0.1, 16), (8, 0.6, 1, 3, 0.3, 5),
           (4, 0.09375, 2, 3, 0.2, 3), (16, 1.3, 2, 6, 0.1, 37), (32, 0.375, 1, 1, 0.1, 32),
           (2, 0.55, 2, 7, 0.05, 1), (8, 1.5, 2, 8, 0.1, 4)]


@pytest.mark.parametrize("cfg", CONFIGS)
def test_ul_gate_list_bit_exact(cfg):
    c = G.Circuit(*cfg, kappa_qsvt=20.0, d=3)
    got = c.export_gates(0)
    ref = OC.build_UL(*cfg)
    assert len(got) == len(ref)
    assert all(_same_gate(a, b) for a, b in zip(got, ref))
    assert c.info()["n_qubits"] == Layout(cfg[0], cfg[2], cfg[3], cfg[5]).n


@pytest.mark.parametrize("cfg", CONFIGS[:4])
def test_qsvt_gate_list_and_mask_bit_exact(cfg):
    ph = np.random.default_rng(1).uniform(-math.pi, math.pi, 6)
    c = G.Circuit(*cfg, phases=ph)
    got = c.export_gates(1)
    ref = OC.build_qsvt(*cfg, list(ph))
    assert len(got) == len(ref) == c.info()["n_gates_total"]
    assert all(_same_gate(a, b) for a, b in zip(got, ref))
    m, v = c.export_mask()
    lay = Layout(cfg[0], cfg[2], cfg[3], cfg[5])
    assert [(int(a), int(b)) for a, b in zip(m, v)] == OC.postselect_patterns(lay)


def test_default_build_c1_kappa_degree_phases():
    """Default path: kappa(L) -> Eq. d-star -> Newton phases; pinned by the oracle."""
    c = G.Circuit(4, 0.8, 2, 2, 0.1, 2)
    inf = c.info()
    kap = P.kappa_L(4, 0.8, 2, 2, 0.1, 2, "periodic")
    assert abs(inf["kappa_qsvt"] - kap) / kap < 1e-9
    assert inf["d"] == Q.degree_from_kappa(kap, 1e-3) == 1957
    assert inf["lambda_L"] == 32.0
    ph = c.export_phases()
    Pf, scale = Q.inverse_target(inf["kappa_qsvt"], inf["d"])
    assert abs(inf["poly_scale"] - scale) < 1e-15
    x = Q.chebyshev_nodes(3001)
    assert np.max(np.abs(Q.qsp_poly(ph, x).real - Pf(x))) < 1e-9


@pytest.mark.parametrize("kappa,d", [(3.0, 1), (5.0, 7), (40.0, 101), (1000.0, 13)])
def test_phases_reproduce_target(kappa, d):
    c = G.Circuit(4, 0.8, 2, 2, 0.1, 2, kappa_qsvt=kappa, d=d)
    ph = c.export_phases()
    assert ph.shape == (d + 1,)
    Pf, _ = Q.inverse_target(kappa, d)
    x = np.linspace(-1, 1, 801)
    x = x[x != 0]
    assert np.max(np.abs(Q.qsp_poly(ph, x).real - Pf(x))) < 1e-11


def test_argument_errors():
    with pytest.raises(N.CsimError) as e:
        G.Circuit(6, 0.8, 2, 2, 0.1, 2, kappa_qsvt=10, d=3)
    assert e.value.status == N.CSIM_ERR_ARG
    for bad in [(4, -1.0, 2, 2, 0.1, 2), (4, 0.8, 3, 2, 0.1, 2), (4, 0.8, 2, 0, 0.1, 2),
                (4, 0.8, 2, 2, 0.0, 2), (4, 0.8, 2, 2, 0.1, 0)]:
        with pytest.raises(N.CsimError) as e:
            G.Circuit(*bad, kappa_qsvt=10, d=3)
        assert e.value.status == N.CSIM_ERR_ARG
    with pytest.raises(N.CsimError) as e:
        G.Circuit(256, 0.8, 2, 2, 0.1, 16, kappa_qsvt=10, d=3)
    assert e.value.status == N.CSIM_ERR_TOO_LARGE
    with pytest.raises(N.CsimError) as e:
        G.Circuit(4, 0.8, 2, 2, 0.1, 2, phases=np.zeros(3))
    assert e.value.status == N.CSIM_ERR_ARG
    with pytest.raises(N.CsimError) as e:
        G.Circuit(4, 0.8, 2, 2, 0.1, 2, kappa_qsvt=10, d=4)
    assert e.value.status == N.CSIM_ERR_ARG


def test_launch_shape_arguments():
    """csim_set_launch_shape (host only): the kernel variants that exist are
    accepted and cleared again; the others, waves outside 1..64 and qubit
    counts outside 7..63 are argument errors.  csim_tune_launch refuses a
    circuit in gate-by-gate mode before touching the device."""
    for u, m, w in [(1, 1, 1), (2, 4, 4), (4, 2, 64), (1, 4, 8)]:
        G.set_launch_shape(G.CSIM_C64, 30, u, m, w)
        G.set_launch_shape(G.CSIM_C64, 30, 0)
    for args in [(G.CSIM_C64, 30, 4, 4, 4), (G.CSIM_C64, 30, 3, 2, 4), (G.CSIM_C64, 30, 2, 3, 4),
                 (G.CSIM_C64, 30, 2, 4, 0), (G.CSIM_C64, 30, 2, 4, 65), (G.CSIM_C128, 6, 1, 2, 4),
                 (G.CSIM_C128, 64, 1, 2, 4), (7, 30, 1, 2, 4)]:
        with pytest.raises(N.CsimError) as e:
            G.set_launch_shape(*args)
        assert e.value.status == N.CSIM_ERR_ARG
    c = G.Circuit(4, 0.8, 2, 2, 0.1, 2, kappa_qsvt=10, d=3)
    c.set_exec(G.CSIM_EXEC_GATE)
    with pytest.raises(N.CsimError) as e:
        c.tune_launch(G.CSIM_C64)
    assert e.value.status == N.CSIM_ERR_ARG


def test_run_before_init_is_state_error():
    c = G.Circuit(4, 0.8, 2, 2, 0.1, 2, kappa_qsvt=10, d=3)
    with pytest.raises(N.CsimError) as e:
        c.run()
    assert e.value.status == N.CSIM_ERR_STATE


def test_amp_update_count():
    """Algorithmic work: sum over gates of 2^(n - #controls)."""
    c = G.Circuit(4, 0.8, 2, 2, 0.1, 2, kappa_qsvt=10, d=3)
    n = c.info()["n_qubits"]
    g = c.export_gates(1)
    expect = sum(2.0 ** (n - bin(int(x)).count("1")) for x in g["cmask"])
    assert c.info()["amp_updates_run"] == expect


def test_final_distribution_matches_oracle():
    """csim_final_distribution reads f(T) from a postselected block and rescales
    it to physical units.  The block here is the oracle's own (O5, the exact
    target polynomial) laid out as csim_postselect compacts it; the densities
    must equal the oracle's, whose rescaling uses the oracle's own scale and
    lambda_L (Sec. II.D.5)."""
    import paper_claims as PC
    kq, d = 1200.0, 1201
    c = G.Circuit(*PC.cfg(PC.K3), kappa_qsvt=kq, d=d, bc="bounceback")
    rho_q, _, y, lay, _, _, _ = PC.oracle_run(PC.K3, kq, d)
    final = PC.Q.final_slot_mask(lay)
    sel = lay.physical_indices()[final]
    fs, ms = 2 + lay.niL, lay.regs["m"][0]
    pos = ((sel >> ms) - lay.Nt) * (1 << (ms - fs)) + ((sel >> fs) & ((1 << (ms - fs)) - 1))
    amps = np.zeros(c.postselect_count(), dtype=complex)
    amps[pos] = y[final]
    f = c.final_distribution(PC.f0(), amps)
    assert f.shape == (PC.NX, 3)
    rho = f.sum(axis=1)
    assert np.max(np.abs(rho - rho_q)) < 1e-8 * np.max(np.abs(rho_q))
    with pytest.raises(G.CsimError):
        c.final_distribution(PC.f0(), amps[:-1])
