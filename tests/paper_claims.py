"""The paper's QSVT runs on the N_C = 1 path and what the paper states about them.

Shared by tests/test_oracle_paper_runs.py (the oracle alone) and
tests/test_gpu_paper_runs.py (the CUDA path through the C ABI).  All runs
use bounce-back walls, nu = 2 (tau from Eq. tau-nu), Nx = 32, and the step
initial condition with drho = 0.4 (lbm_inputs.step_instance).

Degree scan (Sec. III.E.1, Fig. qsvt-d-comparison): K = 1, dt = 0.1, Nt = 32,
kappa(L) about 800, kappa_QSVT in {400, 1000}, d = r kappa_QSVT + 1 for
r in {5, 10, 15}.
  * kappa_QSVT = 1000 >= kappa: the output converges to the classical
    reference as d grows.  At r = 10 the error is about 1e-4 (the figure that
    Sec. III.E.2 quotes for this run; Sec. III.E.1 says "1e-5 or below").
  * kappa_QSVT = 400 < kappa: the output is under-inverted (reduced
    amplitude at r = 5), and the deficit shrinks as d grows.

K trade-off (Sec. III.E.3, Fig. qsvt-K-comparison): T = 5.6,
kappa_QSVT = 1200, d = 12001.
  * K = 3, dt = 0.7, Nt = 8: kappa about 1058.  The output matches the
    classical Taylor solve to an L-infinity error of about 8e-4, within the
    1e-3 target.
  * K = 1, dt = 0.04375, Nt = 128: kappa about 3283.  The density profile
    collapses to about half its amplitude.
"""
import numpy as np
import scipy.fft

import lbm_inputs as I
from oracle import physics as P
from oracle import qsvt as Q

NX = 32
DRHO = 0.4
TAU = P.tau_from_nu(NX, 2.0)

# (K, dt, Nt)
SCAN = (1, 0.1, 32)
K3 = (3, 0.7, 8)
K1 = (1, 0.04375, 128)

PAPER_KAPPA = {SCAN: 800.0, K3: 1058.0, K1: 3283.0}
PAPER_K3_LINF = 8e-4      # Sec. III.E.3, against the classical Taylor solve
TARGET_LINF = 1e-3        # the accuracy target of Sec. III.E.3
PAPER_SCAN_R10 = 1e-4     # Sec. III.E.2, kappa_QSVT = 1000, d = 10 kappa_QSVT


def cfg(kdn):
    K, dt, Nt = kdn
    return (NX, TAU, 1, K, dt, Nt)


def f0():
    return I.step_instance(NX, DRHO)


def exact_poly_coeffs(kappa_qsvt, d):
    """Chebyshev coefficients of the oracle's target polynomial (inverse_target),
    from its values at the d + 1 Chebyshev-Gauss nodes (a DCT-II: exact for a
    degree-d polynomial), and its scale."""
    Pf, scale = Q.inverse_target(kappa_qsvt, d)
    x = Q.chebyshev_nodes(d + 1)
    c = scipy.fft.dct(Pf(x), type=2) / (d + 1)
    c[0] *= 0.5
    c[0::2] = 0.0  # the target is odd; its even coefficients are rounding noise
    return c, scale


def first_final_density(rows, lay):
    """Density profile of the first postselected slot (m = Nt, k = 0) of a vector
    over L's rows; N_C = 1, so the slot holds f^(1)[alpha*3 + q]."""
    D = lay.carleman_dim()
    final = Q.final_slot_mask(lay)
    blk = np.asarray(rows)[final][:D].real
    return blk.reshape(NX, 3).sum(axis=1)


def oracle_run(kdn, kappa_qsvt, d):
    """The oracle's QSVT output (the exact target polynomial, O5) and the classical
    Taylor solve, both as densities in physical units, plus the O5 rows.

    The postselected block approximates scale * lambda_L * L^{-1} b with b the
    normalised Carleman vector, so dividing by scale * lambda_L and multiplying by
    |f^(1)(0)| gives f(T)."""
    c_ = cfg(kdn)
    f = f0()
    coeffs, scale = exact_poly_coeffs(kappa_qsvt, d)
    y, lay, M, b = Q.qsvt_postselected(*c_, f, None, "bounceback", coeffs=coeffs)
    A = P.carleman_A(NX, TAU, 1, "bounceback")
    lam = P.lambda_L(1, kdn[0], P.l_max(A, kdn[1]))
    nv = np.linalg.norm(P.carleman_vector(f.reshape(-1), 1))
    L = P.l_matrix(A, kdn[1], kdn[0], kdn[2])
    x = P.solve_l(L, b)
    rho_q = first_final_density(y, lay) / (scale * lam) * nv
    rho_x = first_final_density(x, lay) * nv
    return rho_q, rho_x, y, lay, scale, lam, nv


def linf(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


def amplitude_ratio(rho_q, rho_x):
    """Ratio of the mean densities (the collapse factor of an under-inverted run)."""
    return float(np.mean(rho_q) / np.mean(rho_x))


def compacted_rows(amps, lay):
    """The entries of csim_postselect's compacted block (signal, label and target
    0; slots m >= Nt), reordered like the final-slot rows of L."""
    final = Q.final_slot_mask(lay)
    sel = lay.physical_indices()[final]
    fs, ms = 2 + lay.niL, lay.regs["m"][0]
    pos = ((sel >> ms) - lay.Nt) * (1 << (ms - fs)) + ((sel >> fs) & ((1 << (ms - fs)) - 1))
    return np.asarray(amps)[pos]
