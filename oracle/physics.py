"""O1 -- classical Carleman-Taylor physics, written from the paper's equations.

Test infrastructure only (see ``oracle/__init__``).  Every matrix here is
assembled entry by entry from the printed formulas, in the paper's own index
convention: f^(1) is indexed ``alpha*Q + q`` (Sec. II.B, the vector below
Eq. ode) and f^(2) = f^(1) (x) f^(1) is indexed ``p1*(Q*Nx) + p2``.

Readings of the paper used here:

* Velocity order e_0=+1, e_1=-1, e_2=0 and weights (1/6, 1/6, 2/3): Sec. II.A.
* Boundary: ``periodic`` wraps alpha+e mod Nx; ``bounceback`` sends the
  collided population whose streaming target alpha+e_{q'} leaves [0, Nx-1]
  back to the same site with reversed velocity (alpha, qbar') -- the wall
  rule of Sec. II.A applied to the collide-then-stream update of
  Eq. A11-elements.
* The N_C=2 quadratic coupling is the printed kernel Eq. A12-kernel (the
  1/rho -> 1 evaluation that Sec. II.B calls the halved coupling).
* L uses the "full idle chain": every (m, k) slot with m >= Nt, taken in
  lexicographic (m, k) order, copies its predecessor (Fig. L, Sec. II.D.4:
  the idle rows fill all register values m >= Nt).  Slots (m < Nt, k > K)
  carry only the identity and are decoupled.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# ---------------------------------------------------------------- D1Q3 model
E = (1, -1, 0)                       # e_0=+1, e_1=-1, e_2=0          (Sec. II.A)
W = (1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0)  # lattice weights                 (Eq. feq)
Q = 3
CS2 = 1.0 / 3.0                      # c_s^2 = 1/3
QBAR = (1, 0, 2)                     # velocity reversal for bounce-back


def tau_from_nu(Nx: int, nu: float) -> float:
    """Eq. tau-nu: tau = (Nx/512) * nu / c_s^2."""
    return (Nx / 512.0) * nu / CS2


def n_alpha(Nx: int) -> int:
    """n_alpha = ceil(log2 Nx) (Sec. II.D.2)."""
    return (Nx - 1).bit_length()


def n_k_bits(K: int) -> int:
    """n_k = ceil(log2(K+1)) (Sec. II.C, last paragraph)."""
    return K.bit_length()


def n_m_bits(Nt: int) -> int:
    """n_m = ceil(log2(Nt) + 1) (Sec. II.D.4)."""
    return (Nt - 1).bit_length() + 1


def stream_target(alpha: int, qp: int, Nx: int, bc: str):
    """Where collide-then-stream sends the output population q' of site alpha."""
    ap = alpha + E[qp]
    if bc == "periodic":
        return ap % Nx, qp
    if bc == "bounceback":
        if 0 <= ap < Nx:
            return ap, qp
        return alpha, QBAR[qp]
    raise ValueError(bc)


def collision_coeff(qp: int, q: int, tau: float) -> float:
    """Bracket of Eq. A11-elements: (1-1/tau) delta_{q'q} + (w_q'/tau)(1 + 3 e_q' e_q)."""
    return (1.0 - 1.0 / tau) * (1.0 if qp == q else 0.0) + W[qp] / tau * (1.0 + 3.0 * E[qp] * E[q])


def k12(qp: int, q1: int, q2: int, tau: float) -> float:
    """Eq. A12-kernel: (w_q'/tau) * (9/2 (e_q1 e_q')(e_q2 e_q') - 3/2 e_q1 e_q2)."""
    return W[qp] / tau * (4.5 * (E[q1] * E[qp]) * (E[q2] * E[qp]) - 1.5 * (E[q1] * E[q2]))


def a11(Nx: int, tau: float, bc: str = "periodic") -> sp.csr_matrix:
    """Eq. A11-elements, entry by entry.  Shape (3Nx, 3Nx); duplicates are summed."""
    rows, cols, vals = [], [], []
    for a in range(Nx):
        for q in range(Q):
            col = a * Q + q
            for qp in range(Q):
                ao, qo = stream_target(a, qp, Nx, bc)
                rows.append(ao * Q + qo)
                cols.append(col)
                vals.append(collision_coeff(qp, q, tau))
            rows.append(col)
            cols.append(col)
            vals.append(-1.0)
    n = Q * Nx
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def a12(Nx: int, tau: float, bc: str = "periodic") -> sp.csr_matrix:
    """Eq. A12-elements with the kernel of Eq. A12-kernel.  Shape (3Nx, 9Nx^2)."""
    rows, cols, vals = [], [], []
    n1 = Q * Nx
    for a in range(Nx):                      # alpha1 == alpha2 == a (the delta)
        for q1 in range(Q):
            for q2 in range(Q):
                col = (a * Q + q1) * n1 + (a * Q + q2)
                for qp in range(Q):
                    v = k12(qp, q1, q2, tau)
                    if v == 0.0:
                        continue
                    ao, qo = stream_target(a, qp, Nx, bc)
                    rows.append(ao * Q + qo)
                    cols.append(col)
                    vals.append(v)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n1, n1 * n1))


def a22(A11: sp.spmatrix) -> sp.csr_matrix:
    """A22 = A11 (x) I + I (x) A11 (Eq. carleman-second)."""
    n = A11.shape[0]
    I = sp.identity(n, format="csr")
    return (sp.kron(A11, I) + sp.kron(I, A11)).tocsr()


def carleman_A(Nx: int, tau: float, NC: int, bc: str = "periodic") -> sp.csr_matrix:
    """Eq. carleman-system for N_C=2 ([[A11, A12], [0, A22]]); A11 alone for N_C=1."""
    A1 = a11(Nx, tau, bc)
    if NC == 1:
        return A1
    if NC != 2:
        raise ValueError("N_C must be 1 or 2")
    A2 = a12(Nx, tau, bc)
    A3 = a22(A1)
    n1 = A1.shape[0]
    Z = sp.csr_matrix((n1 * n1, n1))
    return sp.bmat([[A1, A2], [Z, A3]], format="csr")


def carleman_vector(f1: np.ndarray, NC: int) -> np.ndarray:
    """(f^(1), f^(1) (x) f^(1)) for N_C=2; f^(1) for N_C=1 (Sec. II.B)."""
    f1 = np.asarray(f1, dtype=np.float64).reshape(-1)
    if NC == 1:
        return f1.copy()
    return np.concatenate([f1, np.kron(f1, f1)])


def max_abs_entry(A: sp.spmatrix) -> float:
    """max_ij |A_ij| over the assembled matrix (L_max definition, Sec. II.D.4)."""
    A = sp.csr_matrix(A)
    A.sum_duplicates()
    return float(np.max(np.abs(A.data))) if A.nnz else 0.0


# ------------------------------------------------------------- Taylor solver
def taylor_recurrence(A: sp.spmatrix, f0: np.ndarray, dt: float, K: int, Nt: int):
    """Eqs. taylor-recurrence and step-transition, applied sequentially.

    Returns (g_Nt^(0), history) where history[m][k] = g_m^(k).
    """
    g = np.asarray(f0, dtype=np.float64).copy()
    history = []
    for _m in range(Nt):
        terms = [g]
        for k in range(K):
            terms.append(dt * (A @ terms[-1]) / (k + 1))
        history.append(terms)
        g = np.sum(terms, axis=0)
    return g, history


def slot(m: int, k: int, K: int) -> int:
    """Slot index of block (m, k): k is the fast digit over 2^{n_k} values."""
    return m * (1 << n_k_bits(K)) + k


def l_matrix(A: sp.spmatrix, dt: float, K: int, Nt: int) -> sp.csr_matrix:
    """Berry et al.'s C_{Nt,K,p}(dt A) in the full-idle-chain register layout.

    Block rows/columns are the 2^{n_m+n_k} slots (m, k).  For m < Nt:
    row (m, k+1) holds -dt A/(k+1) at column (m, k) (k < K); row (m+1, 0)
    holds -I at columns (m, 0..K).  Every slot after (Nt, 0) holds -I at its
    predecessor.  All diagonal blocks are I.  (Fig. L; Sec. II.D.4.)
    """
    D = A.shape[0]
    nk, nm = n_k_bits(K), n_m_bits(Nt)
    S = 1 << (nk + nm)
    I = sp.identity(D, format="csr")
    A = sp.csr_matrix(A)
    blocks = [[None] * S for _ in range(S)]
    for s in range(S):
        blocks[s][s] = I
    for m in range(Nt):
        for k in range(K):
            blocks[slot(m, k + 1, K)][slot(m, k, K)] = (-dt / (k + 1)) * A
        for k in range(K + 1):
            blocks[slot(m + 1, 0, K)][slot(m, k, K)] = -I
    for s in range(slot(Nt, 0, K) + 1, S):
        blocks[s][s - 1] = -I
    return sp.bmat(blocks, format="csr")


def rhs_vector(f_init: np.ndarray, K: int, Nt: int) -> np.ndarray:
    """b: the initial Carleman vector in slot (0, 0), zero elsewhere (Sec. II.D.5)."""
    D = f_init.shape[0]
    S = 1 << (n_k_bits(K) + n_m_bits(Nt))
    b = np.zeros(S * D)
    b[:D] = f_init
    return b


def solve_l(L: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    """x = L^{-1} b by forward substitution (L is unit lower triangular)."""
    return spla.spsolve_triangular(sp.csr_matrix(L), b, lower=True, unit_diagonal=True)


def lambda_L(NC: int, K: int, Lmax: float) -> float:
    """lambda_L = 2^{n_i^L} L_max with n_i^L = max(1 + n_i^A, 2 + n_k) (Sec. II.D.4)."""
    n_iA = 2 if NC == 1 else 4
    n_iL = max(1 + n_iA, 2 + n_k_bits(K))
    return float(1 << n_iL) * Lmax


def l_max(A: sp.spmatrix, dt: float) -> float:
    """L_max = max(1, dt * max|A_ij|) (Sec. II.D.4)."""
    return max(1.0, dt * max_abs_entry(A))


def sigma_min(L: sp.spmatrix) -> float:
    """Smallest singular value of L, as 1 / ||L^{-1}||_2 (ARPACK on L^{-1})."""
    Lc = sp.csc_matrix(L)
    lu = spla.splu(Lc, permc_spec="NATURAL", diag_pivot_thresh=0.0,
                   options={"SymmetricMode": True})
    n = L.shape[0]
    op = spla.LinearOperator((n, n), matvec=lambda v: lu.solve(v),
                             rmatvec=lambda v: lu.solve(v, trans="T"), dtype=np.float64)
    s = spla.svds(op, k=1, which="LM", return_singular_vectors=False, tol=1e-12,
                  maxiter=20000, random_state=0)
    return 1.0 / float(s[0])


def kappa_L(Nx: int, tau: float, NC: int, K: int, dt: float, Nt: int, bc: str = "periodic") -> float:
    """Effective condition number kappa = lambda_L / sigma_min(L) (Sec. II.D.5)."""
    A = carleman_A(Nx, tau, NC, bc)
    L = l_matrix(A, dt, K, Nt)
    return lambda_L(NC, K, l_max(A, dt)) / sigma_min(L)


def spectral_radius(A: sp.spmatrix) -> float:
    """mu(A) = max |eigenvalue| (App. D), dense."""
    return float(np.max(np.abs(np.linalg.eigvals(A.toarray()))))


# ------------------------------------------------- nonlinear reference flows
def feq(rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Eq. feq for every site; returns shape (Nx, 3)."""
    out = np.empty((rho.shape[0], Q))
    for q in range(Q):
        eu = E[q] * u
        out[:, q] = W[q] * rho * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - u * u / (2.0 * CS2))
    return out


def bgk_rhs_collide_stream(f: np.ndarray, tau: float, bc: str = "periodic") -> np.ndarray:
    """Exact-1/rho BGK in the collide-then-stream form whose Carleman expansion
    is Eqs. A11/A12: df_q'(a')/dt = [f + (feq - f)/tau]_q'(upstream) - f_q'(a')."""
    Nx = f.shape[0]
    rho = f.sum(axis=1)
    u = (f @ np.asarray(E, dtype=np.float64)) / rho
    post = f + (feq(rho, u) - f) / tau
    out = -f.copy()
    for a in range(Nx):
        for qp in range(Q):
            ao, qo = stream_target(a, qp, Nx, bc)
            out[ao, qo] += post[a, qp]
    return out


def rk4(rhs, y0: np.ndarray, dt: float, nsteps: int) -> np.ndarray:
    y = np.array(y0, dtype=np.float64)
    for _ in range(nsteps):
        k1 = rhs(y)
        k2 = rhs(y + 0.5 * dt * k1)
        k3 = rhs(y + 0.5 * dt * k2)
        k4 = rhs(y + dt * k3)
        y = y + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return y
