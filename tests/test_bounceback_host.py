"""Bounce-back walls in the circuit (reading R2): the C++ compiler against the
oracle's compiler (bit-exact gate lists), the oracle's circuit against the
classical L with walls (block-encoding extraction, App. B method), and the
library's own kappa(L) against the values the paper prints for its
bounce-back runs."""
import struct

import numpy as np
import pytest

import paper_2606_12770_gb300 as G
from conftest import read_golden
from oracle import blockenc as B
from oracle import circuit as OC
from oracle import physics as P

CONFIGS = [(4, 0.8, 2, 2, 0.1, 2), (64, 0.93, 2, 4, 0.1, 16), (8, 0.6, 1, 3, 0.3, 5),
           (4, 0.09375, 2, 3, 0.2, 3), (16, 1.3, 2, 6, 0.1, 37), (2, 0.55, 2, 7, 0.05, 1),
           (8, 1.5, 2, 8, 0.1, 4), (2, 0.8, 1, 1, 0.1, 1), (4, 0.3, 2, 1, 0.7, 2)]


def _same(a, b):
    return ((int(a["op"]), int(a["target"]), int(a["cmask"]), int(a["cval"]), int(a["tag"]))
            == (b[0], b[1], b[2], b[3], b[5])
            and struct.pack("<d", float(a["angle"])) == struct.pack("<d", b[4]))


@pytest.mark.parametrize("cfg", CONFIGS)
def test_bounceback_gate_list_bit_exact(cfg):
    c = G.Circuit(*cfg, kappa_qsvt=20.0, d=3, bc="bounceback")
    got = c.export_gates(0)
    ref = OC.build_UL(*cfg, bc="bounceback")
    assert len(got) == len(ref)
    assert all(_same(a, b) for a, b in zip(got, ref))
    # the walls add gates: the periodic list is shorter
    assert len(ref) > len(OC.build_UL(*cfg))


def test_lmax_list_equals_assembled_matrix():
    """max|A| from the distinct entries (used for the angles) equals the
    maximum over the assembled matrix, with and without walls (reading R8)."""
    for tau in (0.8, 0.5, 0.3, 0.09375, 1.5, 2.0):
        for NC in (1, 2):
            for bc in ("periodic", "bounceback"):
                A = P.carleman_A(4, tau, NC, bc)
                assert abs(OC.max_abs_A(tau, NC, bc) - np.max(np.abs(A.data))) < 1e-13


@pytest.mark.parametrize("cfg", [(4, 0.8, 1, 2, 0.1, 2), (8, 0.7, 1, 3, 0.2, 3),
                                 (2, 1.1, 2, 1, 0.1, 2), (4, 0.8, 2, 1, 0.1, 1),
                                 (4, 0.3, 2, 1, 0.7, 1)])
def test_bounceback_block_encoding_is_L(cfg):
    err, cross, _ = B.compare_with_L(*cfg, bc="bounceback")
    tol = float(dict((r[0], r[1]) for r in read_golden("blockenc_app_b.txt"))["tolerance"])
    assert err < tol and cross == 0.0
    # and it differs from the periodic operator (the walls are really there)
    M, inputs, lam, lay = B.extract_UL(*cfg, bc="periodic")
    A = P.carleman_A(cfg[0], cfg[1], cfg[2], "bounceback")
    L = P.l_matrix(A, cfg[4], cfg[3], cfg[5]).toarray()
    pos = {int(v): i for i, v in enumerate(inputs)}
    pidx = np.array([pos[int(v)] for v in lay.physical_indices()])
    assert np.max(np.abs(M.toarray()[np.ix_(pidx, pidx)] - L)) > 1e-3


def test_library_kappa_matches_paper_with_walls():
    """The library's Lanczos kappa(L) for the walled system reproduces the
    kappa values the paper prints (rounded there, hence 5e-3 relative)."""
    for NC, Nx, K, dt, Nt, kap, lam, *_ in read_golden("kappa.txt"):
        NC, Nx, K, Nt = int(NC), int(Nx), int(K), int(Nt)
        dt, kap = float(dt), float(kap)
        tau = P.tau_from_nu(Nx, 2.0)
        c = G.Circuit(Nx, tau, NC, K, dt, Nt, d=3, bc="bounceback")
        inf = c.info()
        if lam != "-":
            assert inf["lambda_L"] == float(lam)
        assert abs(inf["kappa_qsvt"] - kap) / kap < 5e-3, (NC, Nx, K, dt, Nt, inf["kappa_qsvt"], kap)
