"""Pins for oracle/physics.py (O1) against what the paper and mathematics fix."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.linalg import expm

from conftest import read_golden
from oracle import physics as P


def test_spectral_radius_table_app_d():
    """App. D table: mu(A11) for Nx = 4..256 at nu = 2, both boundary conditions."""
    for Nx, tau_p, mu1, mu2 in read_golden("spectral_radius.txt"):
        Nx, tau_p, mu1, mu2 = int(Nx), float(tau_p), float(mu1), float(mu2)
        tau = P.tau_from_nu(Nx, 2.0)
        assert abs(tau - tau_p) <= 5e-4 + 1e-12
        for bc in ("bounceback", "periodic"):
            mu = P.spectral_radius(P.a11(Nx, tau, bc))
            assert abs(mu - mu1) <= 0.05 + 1e-9, (Nx, bc, mu)
            # Kronecker sum: mu(A22) = 2 mu(A11) (App. D text) -> N_C=2 column
            assert abs(2 * mu - mu2) <= 0.1 + 1e-9


@pytest.mark.parametrize("Nx", [4, 8])
def test_spectral_radius_nc2_assembled(Nx):
    """mu of the assembled N_C=2 matrix equals the App. D N_C=2 column and 2 mu(A11)."""
    table = {int(r[0]): float(r[3]) for r in read_golden("spectral_radius.txt")}
    tau = P.tau_from_nu(Nx, 2.0)
    A = P.carleman_A(Nx, tau, 2, "bounceback")
    mu = P.spectral_radius(A)
    assert abs(mu - table[Nx]) <= 0.05
    assert abs(mu - 2 * P.spectral_radius(P.a11(Nx, tau, "bounceback"))) < 1e-9


def test_kappa_pins():
    """kappa(L) values printed in Sec. III.E (bounce-back, nu = 2)."""
    for NC, Nx, K, dt, Nt, kap, lam, *_ in read_golden("kappa.txt"):
        NC, Nx, K, Nt = int(NC), int(Nx), int(K), int(Nt)
        dt, kap = float(dt), float(kap)
        tau = P.tau_from_nu(Nx, 2.0)
        A = P.carleman_A(Nx, tau, NC, "bounceback")
        if lam != "-":
            assert P.lambda_L(NC, K, P.l_max(A, dt)) == float(lam)
        k = P.kappa_L(Nx, tau, NC, K, dt, Nt, "bounceback")
        assert abs(k - kap) / kap < 5e-3, (NC, Nx, K, dt, Nt, k, kap)


def test_lambda_L_growth_nc1_to_nc2():
    """Sec. III.D.3: lambda_L grows 8 -> 32 from N_C=1 to N_C=2 at K=1 (L_max = 1)."""
    Nx = 64
    tau = P.tau_from_nu(Nx, 2.0)
    for NC, expect in ((1, 8.0), (2, 32.0)):
        A = P.carleman_A(Nx, tau, NC, "bounceback")
        assert P.l_max(A, 0.1) == 1.0
        assert P.lambda_L(NC, 1, P.l_max(A, 0.1)) == expect


def test_lambda_L_nc2_nx8():
    """L_max = dt * max|A| = 0.1/tau = 1.0667 at Nx = 8, nu = 2 -> lambda_L = 34.13."""
    tau = P.tau_from_nu(8, 2.0)
    A = P.carleman_A(8, tau, 2, "bounceback")
    assert abs(P.max_abs_entry(A) - 1.0 / tau) < 1e-12
    assert abs(P.lambda_L(2, 3, P.l_max(A, 0.1)) - 32 * 0.1 / tau) < 1e-12


@pytest.mark.parametrize("bc", ["periodic", "bounceback"])
def test_mass_momentum_conservation(bc):
    """Column sums of A11 vanish (mass); periodic: momentum-weighted sums vanish."""
    Nx, tau = 8, 0.7
    A = P.a11(Nx, tau, bc).toarray()
    assert np.max(np.abs(A.sum(axis=0))) < 1e-14
    if bc == "periodic":
        e = np.tile(np.array(P.E, dtype=float), Nx)
        assert np.max(np.abs(e @ A)) < 1e-14
    for q1 in range(3):
        for q2 in range(3):
            ks = [P.k12(qp, q1, q2, tau) for qp in range(3)]
            assert abs(sum(ks)) < 1e-15
            assert abs(sum(P.E[qp] * ks[qp] for qp in range(3))) < 1e-15


def test_k12_closed_form():
    """Eq. A12-kernel in D1Q3: e1 e2/(2 tau) for q' in {0,1}; -e1 e2/tau for q'=2."""
    tau = 0.9
    for q1 in range(3):
        for q2 in range(3):
            ee = P.E[q1] * P.E[q2]
            assert abs(P.k12(0, q1, q2, tau) - ee / (2 * tau)) < 1e-15
            assert abs(P.k12(1, q1, q2, tau) - ee / (2 * tau)) < 1e-15
            assert abs(P.k12(2, q1, q2, tau) + ee / tau) < 1e-15


@pytest.mark.parametrize("NC", [1, 2])
def test_uniform_equilibrium_is_fixed_point(NC):
    """f = w rho0 (rest equilibrium) is a stationary point of Eq. carleman-system."""
    Nx, tau, rho0 = 4, 0.8, 1.3
    f1 = np.tile(np.array(P.W), Nx) * rho0
    A = P.carleman_A(Nx, tau, NC)
    x = P.carleman_vector(f1, NC)
    assert np.max(np.abs(A @ x)) < 1e-14
    g, _ = P.taylor_recurrence(A, x, 0.1, 3, 5)
    assert np.max(np.abs(g - x)) < 1e-14


@pytest.mark.parametrize("NC,Nx,K,Nt", [(2, 4, 2, 2), (1, 8, 3, 5), (2, 2, 4, 3)])
def test_forward_substitution_matches_recurrence(NC, Nx, K, Nt):
    """L x = b (Fig. L, full idle chain) reproduces Eqs. taylor-recurrence/step-transition."""
    rng = np.random.default_rng(3)
    tau, dt = 0.8, 0.1
    A = P.carleman_A(Nx, tau, NC)
    f1 = np.tile(np.array(P.W), Nx) * (1 + 0.05 * rng.uniform(-1, 1, 3 * Nx))
    f = P.carleman_vector(f1, NC)
    gN, hist = P.taylor_recurrence(A, f, dt, K, Nt)
    L = P.l_matrix(A, dt, K, Nt)
    x = P.solve_l(L, P.rhs_vector(f, K, Nt))
    D = f.shape[0]
    nk, nm = P.n_k_bits(K), P.n_m_bits(Nt)
    scale = np.max(np.abs(f))
    for m in range(Nt):
        for k in range(K + 1):
            s = P.slot(m, k, K)
            assert np.max(np.abs(x[s * D:(s + 1) * D] - hist[m][k])) < 1e-14 * scale
        for k in range(K + 1, 1 << nk):
            s = P.slot(m, k, K)
            assert np.max(np.abs(x[s * D:(s + 1) * D])) == 0.0
    for s in range(P.slot(Nt, 0, K), 1 << (nk + nm)):
        assert np.max(np.abs(x[s * D:(s + 1) * D] - gN)) < 1e-13 * scale


def test_a11_fourier_symbol():
    """Periodic A11 is block circulant with symbol e^{-i th e_q'} c(q',q) - delta_{q'q}."""
    Nx, tau = 8, 0.65
    A = P.a11(Nx, tau, "periodic").toarray()
    alpha = np.arange(Nx)
    for j in range(Nx):
        th = 2 * np.pi * j / Nx
        S = np.array([[np.exp(-1j * th * P.E[qp]) * P.collision_coeff(qp, q, tau) - (qp == q)
                       for q in range(3)] for qp in range(3)])
        for q in range(3):
            v = np.zeros((Nx, 3), dtype=complex)
            v[:, q] = np.exp(1j * th * alpha)
            lhs = (A @ v.reshape(-1)).reshape(Nx, 3)
            rhs = np.outer(np.exp(1j * th * alpha), S[:, q])
            assert np.max(np.abs(lhs - rhs)) < 1e-13


@pytest.mark.parametrize("K", [1, 2, 3])
def test_taylor_converges_to_expm(K):
    """Sec. III.C: the Taylor solve tends to e^{TA} f(0); global error O(dt^K)."""
    Nx, tau, T = 8, 0.7, 0.8
    A = P.a11(Nx, tau, "periodic")
    rng = np.random.default_rng(1)
    f = np.tile(np.array(P.W), Nx) * (1 + 0.1 * rng.uniform(-1, 1, 3 * Nx))
    # Fourier closed form of e^{TA} f, mode by mode
    fh = np.fft.fft(f.reshape(Nx, 3), axis=0)
    out = np.empty_like(fh)
    for j in range(Nx):
        th = 2 * np.pi * j / Nx
        S = np.array([[np.exp(-1j * th * P.E[qp]) * P.collision_coeff(qp, q, tau) - (qp == q)
                       for q in range(3)] for qp in range(3)])
        out[j] = expm(T * S) @ fh[j]
    exact = np.fft.ifft(out, axis=0).real.reshape(-1)
    errs = []
    for Nt in (8, 16, 32):
        g, _ = P.taylor_recurrence(A, f, T / Nt, K, Nt)
        errs.append(np.max(np.abs(g - exact)))
    for e0, e1 in zip(errs, errs[1:]):
        assert 0.6 * 2 ** K < e0 / e1 < 1.5 * 2 ** K, errs


def _carleman_vs_bgk_error(delta, kernel_scale):
    Nx, tau, T = 4, 0.8, 1.0
    rho = 1.0 + delta * np.sin(2 * np.pi * np.arange(Nx) / Nx)
    f0 = np.outer(rho, np.array(P.W))
    exact = P.rk4(lambda y: P.bgk_rhs_collide_stream(y.reshape(Nx, 3), tau).reshape(-1),
                  f0.reshape(-1), 1e-3, 1000)
    A1 = P.a11(Nx, tau)
    A2 = kernel_scale * P.a12(Nx, tau)
    n1 = A1.shape[0]
    A = sp.bmat([[A1, A2], [sp.csr_matrix((n1 * n1, n1)), P.a22(A1)]], format="csc")
    x = spla.expm_multiply(T * A, P.carleman_vector(f0.reshape(-1), 2))
    return np.max(np.abs(x[:n1] - exact))


def test_nc2_kernel_reading():
    """Reading R4: the printed Eq. A12-kernel is the N_C=2 coupling.

    With it the N_C=2 Carleman error against the exact-1/rho BGK flow falls at
    least as delta^3 when the density perturbation delta halves (observed
    delta^4); with the 2-rho (doubled) or a halved kernel the quadratic
    source is wrong at O(delta^2) and the error ratio is 4.
    """
    r_printed = _carleman_vs_bgk_error(0.04, 1.0) / _carleman_vs_bgk_error(0.02, 1.0)
    r_doubled = _carleman_vs_bgk_error(0.04, 2.0) / _carleman_vs_bgk_error(0.02, 2.0)
    r_halved = _carleman_vs_bgk_error(0.04, 0.5) / _carleman_vs_bgk_error(0.02, 0.5)
    assert r_printed > 7.0, r_printed
    assert 3.5 < r_doubled < 4.5, r_doubled
    assert 3.5 < r_halved < 4.5, r_halved
