"""O5 -- classical evaluation of the QSVT circuit's postselected output.

Test infrastructure only.  QSP convention of the circuit (Fig. circuit-qsvt):
with the reflection R(x) = [[x, sqrt(1-x^2)], [sqrt(1-x^2), -x]] that U_L
realises on each singular-value plane, a phase list (phi_0..phi_d) defines

    W(x) = e^{i phi_0 Z} R(x) e^{i phi_1 Z} R(x) ... R(x) e^{i phi_d Z},
    P(x) = <0| W(x) |0>.

The signal-qubit Hadamards average the +phi and -phi branches, and the first
oracle call on b is U_L^dag, so the block (s=0, ancillas=0) of the circuit is
Re(P)^{SV}(L^T/lambda_L) applied to b (reading R13 for the real part), where
Re(P) is the real odd polynomial x -> Re P(x); for P ~ 1/x this is
~ lambda_L L^{-1} b, the solution of L x = b (Sec. II.D.5).  This
module computes that vector directly from L (``physics.l_matrix``) using
Chebyshev coefficients of Re(P) and the singular-value Chebyshev recurrence

    A_0 = I,  A_1 = M,  A_{k+1} = 2 M^T A_k - A_{k-1} (k odd),
                         A_{k+1} = 2 M   A_k - A_{k-1} (k even),

which is T_k^{SV}(M) for odd k (Gilyen et al., QSVT Def. of the singular
value transform).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import circuit as C
from . import physics as P
from .layout import Layout


def qsp_poly(phases, x) -> np.ndarray:
    """P(x) = <0|W(x)|0> for an array of x in [-1, 1]."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    r0 = np.full(x.shape, complex(math.cos(phases[0]), math.sin(phases[0])))
    r1 = np.zeros(x.shape, dtype=np.complex128)
    for phi in phases[1:]:
        n0 = r0 * x + r1 * s
        n1 = r0 * s - r1 * x
        r0 = n0 * complex(math.cos(phi), math.sin(phi))
        r1 = n1 * complex(math.cos(phi), -math.sin(phi))
    return r0


def chebyshev_nodes(N: int) -> np.ndarray:
    return np.cos(np.pi * (np.arange(N) + 0.5) / N)


def cheb_coeffs(values_at_nodes: np.ndarray) -> np.ndarray:
    """Chebyshev coefficients c_0..c_{N-1} from values at the N Chebyshev-Gauss nodes."""
    N = values_at_nodes.shape[0]
    theta = np.pi * (np.arange(N) + 0.5) / N
    k = np.arange(N)
    c = (2.0 / N) * (np.cos(np.outer(k, theta)) @ values_at_nodes)
    c[0] *= 0.5
    return c


def re_poly_coeffs(phases) -> np.ndarray:
    """Chebyshev coefficients of Re P for the phase list (degree d = len-1)."""
    d = len(phases) - 1
    x = chebyshev_nodes(d + 1)
    return cheb_coeffs(qsp_poly(phases, x).real)


def apply_odd_sv_poly(c: np.ndarray, M: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    """sum over odd k of c_k T_k^{SV}(M) b (the even coefficients must vanish)."""
    M = sp.csr_matrix(M)
    MT = M.T.tocsr()
    d = c.shape[0] - 1
    a_prev = b.astype(np.float64)
    a_cur = M @ a_prev
    y = c[1] * a_cur
    for k in range(1, d):
        if k % 2 == 1:
            a_next = 2.0 * (MT @ a_cur) - a_prev
        else:
            a_next = 2.0 * (M @ a_cur) - a_prev
        a_prev, a_cur = a_cur, a_next
        if (k + 1) % 2 == 1:
            y = y + c[k + 1] * a_cur
    return y


def qsvt_postselected(Nx, tau, NC, K, dt, Nt, f0, phases, bc="periodic", coeffs=None):
    """Postselected (s=0, ancillas=0) amplitudes on every physical (slot, j).

    y = Re(P)^{SV}((L/lambda_L)^T) b.  Returns (y, lay, L/lambda_L, b), y ordered
    like L's rows.
    """
    lay = Layout(Nx, NC, K, Nt)
    A = P.carleman_A(Nx, tau, NC, bc)
    L = P.l_matrix(A, dt, K, Nt)
    lam = P.lambda_L(NC, K, P.l_max(A, dt))
    f0 = np.asarray(f0, dtype=np.float64).reshape(Nx, 3)
    vec = P.carleman_vector(f0.reshape(-1), NC)
    b = P.rhs_vector(vec / np.linalg.norm(vec), K, Nt)
    c = re_poly_coeffs(phases) if coeffs is None else np.asarray(coeffs)
    if np.max(np.abs(c[0::2])) > 1e-10:
        raise ValueError("Re P is not odd")
    M = L / lam
    y = apply_odd_sv_poly(c, M.T.tocsr(), b)
    return y, lay, M, b


def final_slot_mask(lay: Layout) -> np.ndarray:
    """Boolean over L's rows: True for slots with m >= Nt (the postselected time)."""
    D = lay.carleman_dim()
    m_of_slot = np.arange(lay.n_slots()) >> lay.nk
    return np.repeat(m_of_slot >= lay.Nt, D)


# --------------------------------------------- target polynomial for 1/x
def inverse_target(kappa: float, d: int):
    """Odd degree-d polynomial approximating 1/x on [1/kappa, 1], scaled to |P| <= 1/2.

    p(x) = (1 - r(x^2)) / x with r(y) = T_n((1 + a^2 - 2y)/(1 - a^2)) / T_n((1+a^2)/(1-a^2)),
    a = 1/kappa, n = (d+1)/2 (the shifted-Chebyshev minimal-residual polynomial).
    The scale is 1 / (2 max |p|) over 8(d+1) Chebyshev-Gauss nodes.
    Returns (callable P, scale).
    """
    if d % 2 == 0:
        raise ValueError("odd d")
    a = 1.0 / kappa
    n = (d + 1) // 2
    z0 = (1.0 + a * a) / (1.0 - a * a)
    tn_z0 = math.cosh(n * math.acosh(z0))

    def tn(z):
        z = np.asarray(z, dtype=np.float64)
        out = np.empty_like(z)
        inside = np.abs(z) <= 1.0
        out[inside] = np.cos(n * np.arccos(z[inside]))
        zo = z[~inside]
        out[~inside] = np.cosh(n * np.arccosh(np.abs(zo))) * np.where(zo < 0, (-1.0) ** n, 1.0)
        return out

    def p(x):
        x = np.asarray(x, dtype=np.float64)
        y = x * x
        z = (1.0 + a * a - 2.0 * y) / (1.0 - a * a)
        return (1.0 - tn(z) / tn_z0) / x

    grid = chebyshev_nodes(8 * (d + 1))
    scale = 1.0 / (2.0 * float(np.max(np.abs(p(grid)))))
    return (lambda x: scale * p(x)), scale


def degree_from_kappa(kappa: float, eps: float) -> int:
    """Eq. d-star: d = kappa * log(2 kappa / eps) / 2, rounded up to the next odd integer."""
    d = int(math.ceil(kappa * math.log(2.0 * kappa / eps) / 2.0))
    return d if d % 2 == 1 else d + 1


def fit_phases(target, d: int, seed: int = 0, tol: float = 1e-12):
    """Phases (reflection convention) with Re P = target on [-1, 1], by least squares.

    Plain Levenberg-Marquardt (scipy) over all d+1 phases, matching Re P at
    the d+1 Chebyshev-Gauss nodes (a degree-d odd polynomial is fixed by its
    values there).  Slow and only meant for small d; raises if the fit does
    not reach ``tol``.  Restarts from seeded random points.
    """
    from scipy.optimize import least_squares

    x = chebyshev_nodes(d + 1)
    f = target(x)
    rng = np.random.default_rng(seed)
    best = None
    for _ in range(20):
        p0 = rng.uniform(-math.pi, math.pi, d + 1)
        r = least_squares(lambda ph: qsp_poly(ph, x).real - f, p0, method="lm",
                          xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=200 * (d + 1))
        err = float(np.max(np.abs(r.fun)))
        if best is None or err < best[1]:
            best = (r.x, err)
        if err < tol:
            return r.x
    raise RuntimeError(f"phase fit did not converge (best max error {best[1]:.2e})")
