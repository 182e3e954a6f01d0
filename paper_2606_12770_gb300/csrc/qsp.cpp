// Host FP64 pieces that choose the QSVT polynomial:
//  * kappa(L) = lambda_L / sigma_min(L) (Sec. II.D.5, Sec. III.D), with
//    sigma_min from restarted Lanczos on (L^{-1})^T L^{-1}; L^{-1} and L^{-T}
//    are applied matrix-free by the Taylor recurrence of Eqs.
//    taylor-recurrence/step-transition in the slot layout of Fig. L;
//  * the degree of Eq. d-star;
//  * an odd polynomial ~ 1/x on [1/kappa, 1] (shifted-Chebyshev minimal
//    residual: p(x) = (1 - T_n((1+a^2-2x^2)/(1-a^2)) / T_n((1+a^2)/(1-a^2))) / x);
//  * QSP phases by Newton's method on symmetric phases (Dong, Lin, Ni, Wang,
//    "robust iterative method for symmetric quantum signal processing"), solved
//    in the e^{i arccos(x) X} convention and converted to the reflection
//    convention that the circuit's U_L realises (Fig. circuit-qsvt).
#include <cmath>
#include <complex>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace csim {
namespace {

using cd = std::complex<double>;
const int E[3] = {1, -1, 0};

// Matrix-free Carleman operator A of Eq. carleman-system, periodic or with
// bounce-back walls (a population leaving the lattice returns to its own site
// with the opposite velocity, reading R2).
struct CarlemanOp {
  int Nx, NC;
  bool bounce = false;
  double tau;
  int n1;      // 3 Nx
  int D;       // n1 (N_C=1) or n1 + n1^2
  double c[3][3];
  double kk[3][3][3];

  CarlemanOp(int Nx_, int NC_, double tau_) : Nx(Nx_), NC(NC_), tau(tau_) {
    n1 = 3 * Nx;
    D = NC == 1 ? n1 : n1 + n1 * n1;
    for (int qp = 0; qp < 3; ++qp)
      for (int q = 0; q < 3; ++q) {
        c[qp][q] = collision_coeff(qp, q, tau);
        for (int q2 = 0; q2 < 3; ++q2) kk[qp][q][q2] = k12(qp, q, q2, tau);
      }
  }
  int wrap(int a) const { return ((a % Nx) + Nx) % Nx; }
  // flat index (site * 3 + velocity) that the output population qp of site a streams to
  int tgt(int a, int qp) const {
    const int ap = a + E[qp];
    if (!bounce || (ap >= 0 && ap < Nx)) return wrap(ap) * 3 + qp;
    return a * 3 + (qp == 0 ? 1 : (qp == 1 ? 0 : qp));
  }

  // y = A11 x on a 3Nx vector (Eq. A11-elements, periodic).
  void a11(const double* x, double* y) const {
    for (int r = 0; r < n1; ++r) y[r] = -x[r];
    for (int a = 0; a < Nx; ++a)
      for (int q = 0; q < 3; ++q) {
        const double xv = x[a * 3 + q];
        if (xv == 0.0) continue;
        for (int qp = 0; qp < 3; ++qp) y[tgt(a, qp)] += c[qp][q] * xv;
      }
  }
  void a11T(const double* x, double* y) const {
    for (int r = 0; r < n1; ++r) y[r] = -x[r];
    for (int a = 0; a < Nx; ++a)
      for (int q = 0; q < 3; ++q) {
        double acc = 0.0;
        for (int qp = 0; qp < 3; ++qp) acc += c[qp][q] * x[tgt(a, qp)];
        y[a * 3 + q] += acc;
      }
  }
  // y = A x
  void apply(const double* x, double* y, std::vector<double>& tmp) const {
    a11(x, y);
    if (NC == 1) return;
    const double* X2 = x + n1;
    double* Y2 = y + n1;
    // A12: y1[a + e_q', q'] += K[q'][q1][q2] X2[(a q1),(a q2)]
    for (int a = 0; a < Nx; ++a)
      for (int q1 = 0; q1 < 3; ++q1)
        for (int q2 = 0; q2 < 3; ++q2) {
          const double xv = X2[(size_t)(a * 3 + q1) * n1 + (a * 3 + q2)];
          if (xv == 0.0) continue;
          for (int qp = 0; qp < 3; ++qp) y[tgt(a, qp)] += kk[qp][q1][q2] * xv;
        }
    // A22 = A11 (x) I + I (x) A11 on the row-major matrix X2[p1][p2]
    tmp.assign(n1, 0.0);
    std::vector<double> col(n1), out(n1);
    for (int p1 = 0; p1 < n1; ++p1) a11(X2 + (size_t)p1 * n1, Y2 + (size_t)p1 * n1);
    for (int p2 = 0; p2 < n1; ++p2) {
      for (int p1 = 0; p1 < n1; ++p1) col[p1] = X2[(size_t)p1 * n1 + p2];
      a11(col.data(), out.data());
      for (int p1 = 0; p1 < n1; ++p1) Y2[(size_t)p1 * n1 + p2] += out[p1];
    }
  }
  void applyT(const double* x, double* y, std::vector<double>& tmp) const {
    a11T(x, y);
    if (NC == 1) return;
    double* Y2 = y + n1;
    const double* X2 = x + n1;
    std::vector<double> col(n1), out(n1);
    for (int p1 = 0; p1 < n1; ++p1) a11T(X2 + (size_t)p1 * n1, Y2 + (size_t)p1 * n1);
    for (int p2 = 0; p2 < n1; ++p2) {
      for (int p1 = 0; p1 < n1; ++p1) col[p1] = X2[(size_t)p1 * n1 + p2];
      a11T(col.data(), out.data());
      for (int p1 = 0; p1 < n1; ++p1) Y2[(size_t)p1 * n1 + p2] += out[p1];
    }
    // A12^T: Y2[(a q1),(a q2)] += sum_q' K[q'][q1][q2] x1[a + e_q', q']
    for (int a = 0; a < Nx; ++a)
      for (int q1 = 0; q1 < 3; ++q1)
        for (int q2 = 0; q2 < 3; ++q2) {
          double acc = 0.0;
          for (int qp = 0; qp < 3; ++qp) acc += kk[qp][q1][q2] * x[tgt(a, qp)];
          Y2[(size_t)(a * 3 + q1) * n1 + (a * 3 + q2)] += acc;
        }
    (void)tmp;
  }
};

// L^{-1} v (forward substitution of Fig. L, full idle chain) and L^{-T} v.
struct LInverse {
  const CarlemanOp& A;
  int K, Nt, nk, nm, S;
  double dt;
  size_t D;
  LInverse(const CarlemanOp& A_, int K_, int Nt_, int nk_, int nm_, double dt_)
      : A(A_), K(K_), Nt(Nt_), nk(nk_), nm(nm_), dt(dt_) {
    S = 1 << (nk + nm);
    D = (size_t)A.D;
  }
  int slot(int m, int k) const { return (m << nk) + k; }
  size_t size() const { return (size_t)S * D; }

  void solve(const std::vector<double>& v, std::vector<double>& x) const {
    x = v;
    std::vector<double> tmp, ax(D);
    for (int m = 0; m < Nt; ++m) {
      if (m > 0)
        for (int k = 0; k <= K; ++k) {
          const double* src = &x[slot(m - 1, k) * D];
          double* dst = &x[slot(m, 0) * D];
          for (size_t j = 0; j < D; ++j) dst[j] += src[j];
        }
      for (int k = 0; k < K; ++k) {
        A.apply(&x[slot(m, k) * D], ax.data(), tmp);
        double* dst = &x[slot(m, k + 1) * D];
        const double f = dt / (k + 1);
        for (size_t j = 0; j < D; ++j) dst[j] += f * ax[j];
      }
    }
    for (int k = 0; k <= K; ++k) {
      const double* src = &x[slot(Nt - 1, k) * D];
      double* dst = &x[slot(Nt, 0) * D];
      for (size_t j = 0; j < D; ++j) dst[j] += src[j];
    }
    for (int s = slot(Nt, 0) + 1; s < S; ++s)
      for (size_t j = 0; j < D; ++j) x[s * D + j] += x[(s - 1) * D + j];
  }

  void solveT(const std::vector<double>& v, std::vector<double>& y) const {
    y = v;
    std::vector<double> tmp, ax(D);
    for (int s = S - 2; s >= slot(Nt, 0); --s)
      for (size_t j = 0; j < D; ++j) y[s * D + j] += y[(s + 1) * D + j];
    for (int m = Nt - 1; m >= 0; --m) {
      for (int k = K; k >= 0; --k) {
        double* dst = &y[slot(m, k) * D];
        if (k < K) {
          A.applyT(&y[slot(m, k + 1) * D], ax.data(), tmp);
          const double f = dt / (k + 1);
          for (size_t j = 0; j < D; ++j) dst[j] += f * ax[j];
        }
        const double* up = &y[slot(m + 1, 0) * D];
        for (size_t j = 0; j < D; ++j) dst[j] += up[j];
      }
    }
  }
};

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  long double s = 0;
  for (size_t i = 0; i < a.size(); ++i) s += (long double)a[i] * b[i];
  return (double)s;
}

// Largest eigenvalue of the symmetric PSD operator B = L^{-T} L^{-1}
// by Lanczos with full reorthogonalisation, restarted from the Ritz vector.
double lanczos_top(const LInverse& Li, int m_steps, int restarts, std::string* err) {
  const size_t N = Li.size();
  std::mt19937_64 rng(12345);
  std::normal_distribution<double> nd;
  std::vector<double> q(N);
  for (auto& x : q) x = nd(rng);
  double nq = std::sqrt(dot(q, q));
  for (auto& x : q) x /= nq;
  double last = 0.0;
  std::vector<std::vector<double>> V;
  std::vector<double> w, t1, alpha, beta;
  for (int rs = 0; rs < restarts; ++rs) {
    V.clear();
    alpha.clear();
    beta.clear();
    V.push_back(q);
    int mstep = std::min<int>(m_steps, (int)N);
    for (int j = 0; j < mstep; ++j) {
      Li.solve(V[j], t1);
      Li.solveT(t1, w);
      const double a = dot(w, V[j]);
      alpha.push_back(a);
      for (int pass = 0; pass < 2; ++pass)
        for (size_t i = 0; i < V.size(); ++i) {
          const double h = dot(w, V[i]);
          for (size_t r = 0; r < N; ++r) w[r] -= h * V[i][r];
        }
      const double b = std::sqrt(dot(w, w));
      if (j + 1 == mstep || b < 1e-14 * std::fabs(a)) break;
      beta.push_back(b);
      for (auto& x : w) x /= b;
      V.push_back(w);
    }
    // eigen-decomposition of the tridiagonal (Jacobi sweeps on a small dense matrix)
    const int m = (int)alpha.size();
    std::vector<double> T((size_t)m * m, 0.0), Q((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) {
      T[i * m + i] = alpha[i];
      Q[i * m + i] = 1.0;
      if (i + 1 < m) T[i * m + i + 1] = T[(i + 1) * m + i] = beta[i];
    }
    for (int sweep = 0; sweep < 100; ++sweep) {
      double off = 0.0;
      for (int p = 0; p < m; ++p)
        for (int r = p + 1; r < m; ++r) off += T[p * m + r] * T[p * m + r];
      if (off < 1e-30) break;
      for (int p = 0; p < m; ++p)
        for (int r = p + 1; r < m; ++r) {
          const double apr = T[p * m + r];
          if (std::fabs(apr) < 1e-300) continue;
          const double th = (T[r * m + r] - T[p * m + p]) / (2.0 * apr);
          const double tt = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
          const double cs = 1.0 / std::sqrt(tt * tt + 1.0), sn = tt * cs;
          for (int k = 0; k < m; ++k) {
            const double tkp = T[k * m + p], tkr = T[k * m + r];
            T[k * m + p] = cs * tkp - sn * tkr;
            T[k * m + r] = sn * tkp + cs * tkr;
          }
          for (int k = 0; k < m; ++k) {
            const double tpk = T[p * m + k], trk = T[r * m + k];
            T[p * m + k] = cs * tpk - sn * trk;
            T[r * m + k] = sn * tpk + cs * trk;
          }
          for (int k = 0; k < m; ++k) {
            const double qkp = Q[k * m + p], qkr = Q[k * m + r];
            Q[k * m + p] = cs * qkp - sn * qkr;
            Q[k * m + r] = sn * qkp + cs * qkr;
          }
        }
    }
    int best = 0;
    for (int i = 1; i < m; ++i)
      if (T[i * m + i] > T[best * m + best]) best = i;
    const double top = T[best * m + best];
    std::fill(q.begin(), q.end(), 0.0);
    for (int i = 0; i < m; ++i)
      for (size_t r = 0; r < N; ++r) q[r] += Q[i * m + best] * V[i][r];
    nq = std::sqrt(dot(q, q));
    for (auto& x : q) x /= nq;
    if (rs > 0 && std::fabs(top - last) <= 1e-12 * top) return top;
    last = top;
  }
  *err = "kappa(L): Lanczos did not converge";
  return last;
}

}  // namespace

double kappa_of_L(const Layout& L, double tau, double dt, std::string* err) {
  CarlemanOp A(L.Nx, L.NC, tau);
  A.bounce = L.bc == CSIM_BC_BOUNCEBACK;
  LInverse Li(A, L.K, L.Nt, L.nk, L.nm, dt);
  const size_t N = Li.size();
  if (N > (size_t)4 << 20) {
    *err = "kappa(L) estimation needs more than 4M unknowns; pass kappa_qsvt explicitly";
    return -1.0;
  }
  std::string lerr;
  const double top = lanczos_top(Li, 60, 40, &lerr);
  if (!lerr.empty()) {
    *err = lerr;
    return -1.0;
  }
  const double sigma_min = 1.0 / std::sqrt(top);
  const double lambda = std::ldexp(1.0, L.niL) * lmax_value(tau, L.NC, dt, L.bc);
  return lambda / sigma_min;
}

int degree_from_kappa(double kappa, double eps) {
  int d = (int)std::ceil(kappa * std::log(2.0 * kappa / eps) / 2.0);
  return (d % 2 == 1) ? d : d + 1;
}

namespace {

double cheb_t(int n, double z) {
  if (std::fabs(z) <= 1.0) return std::cos(n * std::acos(z));
  const double v = std::cosh(n * std::acosh(std::fabs(z)));
  return (z < 0 && (n % 2 == 1)) ? -v : v;
}

double p_raw(double kappa, int d, double x) {
  const double a = 1.0 / kappa;
  const int n = (d + 1) / 2;
  const double z0 = (1.0 + a * a) / (1.0 - a * a);
  const double tn0 = std::cosh(n * std::acosh(z0));
  const double y = x * x;
  const double z = (1.0 + a * a - 2.0 * y) / (1.0 - a * a);
  return (1.0 - cheb_t(n, z) / tn0) / x;
}

}  // namespace

double inverse_target_scale(double kappa, int d) {
  const int N = 8 * (d + 1);
  double mx = 0.0;
  for (int j = 0; j < N; ++j) {
    const double x = std::cos(M_PI * (j + 0.5) / N);
    mx = std::max(mx, std::fabs(p_raw(kappa, d, x)));
  }
  return 1.0 / (2.0 * mx);
}

double inverse_target_value(double kappa, int d, double scale, double x) {
  return scale * p_raw(kappa, d, x);
}

namespace {

// Re <0| e^{i psi_0 Z} W(x) e^{i psi_1 Z} ... W(x) e^{i psi_d Z} |0> and its
// gradient with respect to every psi_j, W(x) = [[x, i s], [i s, x]].
void qsp_w_value_grad(const std::vector<double>& psi, double x, double* val,
                      std::vector<double>* grad) {
  const int d = (int)psi.size() - 1;
  const double s = std::sqrt(std::max(0.0, 1.0 - x * x));
  std::vector<cd> r0(d + 1), r1(d + 1), c0(d + 1), c1(d + 1);
  // rows: r_j = <0| e^{i psi_0 Z} W ... W e^{i psi_j Z}
  r0[0] = std::polar(1.0, psi[0]);
  r1[0] = 0.0;
  for (int j = 1; j <= d; ++j) {
    const cd a = r0[j - 1] * x + r1[j - 1] * cd(0, s);
    const cd b = r0[j - 1] * cd(0, s) + r1[j - 1] * x;
    r0[j] = a * std::polar(1.0, psi[j]);
    r1[j] = b * std::polar(1.0, -psi[j]);
  }
  // columns: c_j = W e^{i psi_{j+1} Z} ... W e^{i psi_d Z} |0>, c_d = |0>
  c0[d] = 1.0;
  c1[d] = 0.0;
  for (int j = d - 1; j >= 0; --j) {
    const cd u0 = c0[j + 1] * std::polar(1.0, psi[j + 1]);
    const cd u1 = c1[j + 1] * std::polar(1.0, -psi[j + 1]);
    c0[j] = u0 * x + u1 * cd(0, s);
    c1[j] = u0 * cd(0, s) + u1 * x;
  }
  *val = (r0[d] * c0[d] + r1[d] * c1[d]).real();
  if (grad) {
    grad->assign(d + 1, 0.0);
    for (int j = 0; j <= d; ++j)
      (*grad)[j] = (cd(0, 1) * (r0[j] * c0[j] - r1[j] * c1[j])).real();
  }
}

bool lu_solve(std::vector<double>& M, std::vector<double>& b, int n) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(M[(size_t)r * n + c]) > std::fabs(M[(size_t)piv * n + c])) piv = r;
    if (std::fabs(M[(size_t)piv * n + c]) < 1e-300) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(M[(size_t)c * n + k], M[(size_t)piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    const double inv = 1.0 / M[(size_t)c * n + c];
    for (int r = c + 1; r < n; ++r) {
      const double f = M[(size_t)r * n + c] * inv;
      if (f == 0.0) continue;
      for (int k = c; k < n; ++k) M[(size_t)r * n + k] -= f * M[(size_t)c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double acc = b[r];
    for (int k = r + 1; k < n; ++k) acc -= M[(size_t)r * n + k] * b[k];
    b[r] = acc / M[(size_t)r * n + r];
  }
  return true;
}

// Re <0| e^{i psi_0 Z} W(x) ... W(x) e^{i psi_d Z} |0> at every node, spread
// over the host's hardware threads (O(d) per node).
void qsp_w_values(const std::vector<double>& psi, const std::vector<double>& xs,
                  std::vector<double>* out) {
  const int d = (int)psi.size() - 1;
  const size_t nn = xs.size();
  out->assign(nn, 0.0);
  std::vector<cd> ph(d + 1);
  for (int j = 0; j <= d; ++j) ph[j] = std::polar(1.0, psi[j]);
  auto work = [&](size_t lo, size_t hi) {
    for (size_t l = lo; l < hi; ++l) {
      const double x = xs[l], sn = std::sqrt(std::max(0.0, 1.0 - x * x));
      cd a = ph[0], b = 0.0;
      for (int j = 1; j <= d; ++j) {
        const cd na = a * x + b * cd(0, sn), nb = a * cd(0, sn) + b * x;
        a = na * ph[j];
        b = nb * std::conj(ph[j]);
      }
      (*out)[l] = a.real();
    }
  };
  unsigned nt = std::max(1u, std::thread::hardware_concurrency());
  if ((size_t)nt > nn / 64 + 1) nt = (unsigned)(nn / 64 + 1);
  std::vector<std::thread> pool;
  for (unsigned k = 0; k < nt; ++k)
    pool.emplace_back(work, nn * k / nt, nn * (k + 1) / nt);
  for (std::thread& t : pool) t.join();
}

// Coefficients c_k of sum_k c_k T_{2k+1}(x) from values at the nodes
// x_l = cos((2l + 1) pi / (4 n)): the matrix cos((2l+1)(2k+1) pi / (4n)) is a
// DCT-IV, orthogonal up to the factor n / 2.
void odd_cheb_coeffs(const std::vector<double>& v, std::vector<double>* c) {
  const size_t n = v.size();
  c->assign(n, 0.0);
  auto work = [&](size_t lo, size_t hi) {
    for (size_t k = lo; k < hi; ++k) {
      double acc = 0.0;
      for (size_t l = 0; l < n; ++l)
        acc += v[l] * std::cos(M_PI * (double)((2 * l + 1) * (2 * k + 1) % (8 * n)) / (4.0 * n));
      (*c)[k] = 2.0 * acc / (double)n;
    }
  };
  unsigned nt = std::max(1u, std::thread::hardware_concurrency());
  if ((size_t)nt > n / 64 + 1) nt = (unsigned)(n / 64 + 1);
  std::vector<std::thread> pool;
  for (unsigned k = 0; k < nt; ++k) pool.emplace_back(work, n * k / nt, n * (k + 1) / nt);
  for (std::thread& t : pool) t.join();
}

// Fixed-point iteration for symmetric phases (Dong, Lin, Ni, Wang): the
// reduced phase j moves by half the gap between the target's and the current
// polynomial's coefficients of T_{d-2j}.  Near zero phases the map from
// reduced phases to those coefficients is -2 times the identity, so the
// iteration contracts when the target is small (|P| <= 1/2 here).  Each step
// costs O(d^2), against the O(d^3) LU solve of the Newton step.
bool fixed_point_phases(int d, const std::vector<double>& xs, const std::vector<double>& f,
                        std::vector<double>* th, double* res_out) {
  const int dr = (int)xs.size();
  std::vector<double> cf, cv, v, psi(d + 1);
  odd_cheb_coeffs(f, &cf);
  th->assign(dr, 0.0);
  double res = 1.0;
  for (int it = 0; it < 200; ++it) {
    for (int j = 0; j <= d; ++j) psi[j] = (*th)[std::min(j, d - j)];
    psi[0] += M_PI / 4;
    psi[d] += M_PI / 4;
    qsp_w_values(psi, xs, &v);
    res = 0.0;
    for (int l = 0; l < dr; ++l) res = std::max(res, std::fabs(v[l] - f[l]));
    if (res < 1e-12) break;
    odd_cheb_coeffs(v, &cv);
    for (int k = 0; k < dr; ++k) (*th)[(d - 1) / 2 - k] -= 0.5 * (cf[k] - cv[k]);
  }
  *res_out = res;
  return std::isfinite(res);
}

}  // namespace

bool solve_phases(double kappa, int d, std::vector<double>* phases, double* scale_out,
                  std::string* err) {
  if (d < 1 || d % 2 == 0) {
    *err = "degree must be odd";
    return false;
  }
  const double scale = inverse_target_scale(kappa, d);
  const int dr = (d + 1) / 2;
  std::vector<double> xs(dr), f(dr);
  for (int l = 0; l < dr; ++l) {
    xs[l] = std::cos((2.0 * (l + 1) - 1.0) * M_PI / (4.0 * dr));
    f[l] = inverse_target_value(kappa, d, scale, xs[l]);
  }
  std::vector<double> th(dr, 0.0), psi(d + 1), g;
  auto expand = [&]() {
    for (int j = 0; j <= d; ++j) psi[j] = th[std::min(j, d - j)];
    psi[0] += M_PI / 4;
    psi[d] += M_PI / 4;
  };
  double res = 1.0;
  // Newton (dense Jacobian) up to kNewtonMax reduced phases; the fixed-point
  // iteration beyond, where the Jacobian no longer fits
  const int kNewtonMax = 1024;
  if (dr > kNewtonMax) {
    if (!fixed_point_phases(d, xs, f, &th, &res) || !(res < 1e-9)) {
      *err = "phase solver (fixed point) did not converge, residual " + std::to_string(res);
      return false;
    }
  }
  for (int it = 0; it < 60 && dr <= kNewtonMax; ++it) {
    expand();
    std::vector<double> J((size_t)dr * dr), F(dr);
    res = 0.0;
    for (int l = 0; l < dr; ++l) {
      double v;
      qsp_w_value_grad(psi, xs[l], &v, &g);
      F[l] = f[l] - v;
      res = std::max(res, std::fabs(F[l]));
      for (int j = 0; j < dr; ++j) J[(size_t)l * dr + j] = g[j] + g[d - j];
    }
    if (res < 1e-14) break;
    if (!lu_solve(J, F, dr)) {
      *err = "phase solver: singular Jacobian";
      return false;
    }
    for (int j = 0; j < dr; ++j) th[j] += F[j];
  }
  if (!(res < (dr > kNewtonMax ? 1e-9 : 1e-11))) {
    *err = "phase solver did not converge";
    return false;
  }
  expand();
  // e^{i pi/2 Z} in front turns Re into Im; then R = -i e^{i pi Z/4} W e^{i pi Z/4}.
  std::vector<double> phi(d + 1);
  psi[0] += M_PI / 2;
  phi[0] = psi[0] - M_PI / 4;
  phi[d] = psi[d] - M_PI / 4;
  for (int j = 1; j < d; ++j) phi[j] = psi[j] - M_PI / 2;
  if (((d - 1) / 2) % 2 == 1) phi[0] += M_PI;
  *phases = phi;
  *scale_out = scale;
  return true;
}

}  // namespace csim
