// Host-side circuit compiler: register layout, value tables and the canonical
// gate list of U_L, U_L^dag and the QSVT wrapper.
//
// The construction is this library's own ancilla-free realisation of the
// sparse-oracle block encoding of Eq. UM-structure (Sec. II.D.1) for the
// Carleman rate matrix of Eq. carleman-system (A11 of Eq. A11-elements, A12 of
// Eqs. A12-elements/A12-kernel, A22 = A11 (x) I + I (x) A11) and for the Taylor
// matrix L of Fig. L (Sec. II.D.4, idle rows filling every m >= Nt).  The gate
// order and every floating-point expression are fixed so that the list is
// reproducible bit for bit (compile with -ffp-contract=off).
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "internal.h"

namespace csim {
namespace {

const int E[3] = {1, -1, 0};                            // e_0=+1, e_1=-1, e_2=0
const double W[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};  // D1Q3 weights

struct Ctrl {
  uint64_t mask = 0, val = 0;
};

Ctrl merge(Ctrl a, const Ctrl& b) {
  uint64_t both = a.mask & b.mask;
  if ((a.val & both) != (b.val & both)) throw std::logic_error("conflicting controls");
  a.mask |= b.mask;
  a.val |= b.val;
  return a;
}
Ctrl merge(Ctrl a, const Ctrl& b, const Ctrl& c) { return merge(merge(a, b), c); }
Ctrl merge(Ctrl a, const Ctrl& b, const Ctrl& c, const Ctrl& d) {
  return merge(merge(merge(a, b), c), d);
}

Ctrl bit_eq(int q, int v) {
  Ctrl c;
  c.mask = 1ull << q;
  c.val = (uint64_t)(v & 1) << q;
  return c;
}

Ctrl reg_eq(const std::vector<int>& bits, uint64_t value) {
  Ctrl c;
  for (size_t j = 0; j < bits.size(); ++j) c = merge(c, bit_eq(bits[j], (int)((value >> j) & 1)));
  return c;
}

Ctrl all_eq(const std::vector<int>& bits, int v) {
  Ctrl c;
  for (int b : bits) c = merge(c, bit_eq(b, v));
  return c;
}

Gate gate(uint8_t op, int target, Ctrl c, double angle, uint16_t tag) {
  if ((c.mask >> target) & 1ull) throw std::logic_error("target used as control");
  Gate g;
  std::memset(&g, 0, sizeof(g));
  g.op = op;
  g.target = (uint8_t)target;
  g.tag = tag;
  g.cmask = c.mask;
  g.cval = c.val;
  g.angle = angle;
  return g;
}

struct Pattern {
  uint64_t hi;
  int j;
};

// Aligned dyadic cover of [lo, hi) over a w-bit register, increasing lo.
std::vector<Pattern> prefix_patterns(uint64_t lo, uint64_t hi, int w) {
  std::vector<Pattern> out;
  while (lo < hi) {
    int j = 0;
    while (j < w && lo % (1ull << (j + 1)) == 0 && lo + (1ull << (j + 1)) <= hi) ++j;
    out.push_back({lo >> j, j});
    lo += 1ull << j;
  }
  return out;
}

Ctrl pattern_ctrl(const std::vector<int>& bits, const Pattern& p) {
  Ctrl c;
  for (size_t idx = 0; idx < bits.size(); ++idx)
    if ((int)idx >= p.j) c = merge(c, bit_eq(bits[idx], (int)((p.hi >> (idx - p.j)) & 1)));
  return c;
}

void inc(std::vector<Gate>& g, const std::vector<int>& bits, Ctrl ctrl, uint16_t tag) {
  for (int j = (int)bits.size() - 1; j >= 0; --j) {
    Ctrl c = ctrl;
    for (int b = 0; b < j; ++b) c = merge(c, bit_eq(bits[b], 1));
    g.push_back(gate(OP_X, bits[j], c, 0.0, tag));
  }
}

void dec(std::vector<Gate>& g, const std::vector<int>& bits, Ctrl ctrl, uint16_t tag) {
  for (int j = (int)bits.size() - 1; j >= 0; --j) {
    Ctrl c = ctrl;
    for (int b = 0; b < j; ++b) c = merge(c, bit_eq(bits[b], 0));
    g.push_back(gate(OP_X, bits[j], c, 0.0, tag));
  }
}

// Collide-then-stream index map on (a, q) with label i: (a, q, i) with q,i <= 2
// maps to (a + e_i, i, q); label 3 (the subtracted identity) is left in place.
// Bounce-back fix-up after periodic streaming of the site register a by the
// velocity register v (value 0: e = +1, 1: e = -1).  Periodic streaming leaves
// the populations that left the lattice at (a = 0, v = 0) (right wall) and
// (a = Nx-1, v = 1) (left wall); exchanging the two patterns returns each to
// its own site with the opposite velocity (reading R2): flip a where v = 1,
// flip v where a = 0, flip a where v = 1 again (v's high bit 0 throughout).
void bounce(std::vector<Gate>& g, const std::vector<int>& a, const std::vector<int>& v, Ctrl X,
            uint16_t tag) {
  const Ctrl base = merge(X, bit_eq(v[1], 0));
  for (int b : a) g.push_back(gate(OP_X, b, merge(base, bit_eq(v[0], 1)), 0.0, tag));
  g.push_back(gate(OP_X, v[0], merge(base, all_eq(a, 0)), 0.0, tag));
  for (int b : a) g.push_back(gate(OP_X, b, merge(base, bit_eq(v[0], 1)), 0.0, tag));
}

void p11(std::vector<Gate>& g, const std::vector<int>& a, const std::vector<int>& q,
         const std::vector<int>& i, Ctrl X, uint16_t tag, bool bb) {
  const int q0 = q[0], q1 = q[1], i0 = i[0], i1 = i[1];
  inc(g, a, merge(X, reg_eq(i, 0)), tag);
  dec(g, a, merge(X, reg_eq(i, 1)), tag);
  if (bb) bounce(g, a, i, X, tag);
  // (q,i) = (0,1) <-> (1,0)
  g.push_back(gate(OP_X, q0, merge(X, bit_eq(i0, 1)), 0.0, tag));
  g.push_back(gate(OP_X, i0, merge(X, bit_eq(q0, 1), bit_eq(q1, 0), bit_eq(i1, 0)), 0.0, tag));
  g.push_back(gate(OP_X, q0, merge(X, bit_eq(i0, 1)), 0.0, tag));
  // (0,2) <-> (2,0)
  g.push_back(gate(OP_X, q1, merge(X, bit_eq(i1, 1)), 0.0, tag));
  g.push_back(gate(OP_X, i1, merge(X, bit_eq(q1, 1), bit_eq(q0, 0), bit_eq(i0, 0)), 0.0, tag));
  g.push_back(gate(OP_X, q1, merge(X, bit_eq(i1, 1)), 0.0, tag));
  // (1,2) <-> (2,1)
  for (int tgt : {q1, i0, i1}) g.push_back(gate(OP_X, tgt, merge(X, bit_eq(q0, 1)), 0.0, tag));
  g.push_back(gate(OP_X, q0, merge(X, bit_eq(q1, 1), bit_eq(i0, 1), bit_eq(i1, 0)), 0.0, tag));
  for (int tgt : {q1, i0, i1}) g.push_back(gate(OP_X, tgt, merge(X, bit_eq(q0, 1)), 0.0, tag));
}

// A12 branch (Eq. A12-elements): a2 <- a2 - a1 (zero iff the sites match),
// move (q1, q2) into the label, q' into q1, stream a1 by e_{q'}, ord 1 -> 0.
void pi3(std::vector<Gate>& g, const Layout& L, Ctrl X, uint16_t tag, bool bb) {
  for (int j = 0; j < L.na; ++j) {
    std::vector<int> sub(L.a2.begin() + j, L.a2.end());
    dec(g, sub, merge(X, bit_eq(L.a1[j], 1)), tag);
  }
  for (int b = 0; b < 2; ++b) {
    g.push_back(gate(OP_X, L.q1[b], merge(X, bit_eq(L.i[b], 1)), 0.0, tag));
    g.push_back(gate(OP_X, L.i[b], merge(X, bit_eq(L.q1[b], 1)), 0.0, tag));
    g.push_back(gate(OP_X, L.q1[b], merge(X, bit_eq(L.i[b], 1)), 0.0, tag));
  }
  g.push_back(gate(OP_X, L.i[1], merge(X, bit_eq(L.q2[0], 1)), 0.0, tag));
  g.push_back(gate(OP_X, L.q2[0], merge(X, bit_eq(L.i[1], 1)), 0.0, tag));
  g.push_back(gate(OP_X, L.i[1], merge(X, bit_eq(L.q2[0], 1)), 0.0, tag));
  inc(g, L.a1, merge(X, reg_eq(L.q1, 0)), tag);
  dec(g, L.a1, merge(X, reg_eq(L.q1, 1)), tag);
  if (bb) bounce(g, L.a1, L.q1, X, tag);
  g.push_back(gate(OP_X, L.ord[0], X, 0.0, tag));
}

double theta(double v, int ko, double dt, double Lmax) {
  return 2.0 * std::asin((((-dt) * v) / (ko + 1.0)) / Lmax);
}

int bitlen(uint64_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

}  // namespace

bool make_layout(int Nx, int NC, int K, int Nt, Layout* out, std::string* err) {
  if (Nx < 2 || (Nx & (Nx - 1))) {
    *err = "Nx must be a power of two >= 2";
    return false;
  }
  if (NC != 1 && NC != 2) {
    *err = "N_C must be 1 or 2";
    return false;
  }
  if (K < 1 || Nt < 1) {
    *err = "K and Nt must be >= 1";
    return false;
  }
  Layout L;
  L.Nx = Nx;
  L.NC = NC;
  L.K = K;
  L.Nt = Nt;
  L.na = bitlen((uint64_t)Nx - 1);
  L.nk = bitlen((uint64_t)K);
  L.nm = bitlen((uint64_t)Nt - 1) + 1;
  L.niA = NC == 1 ? 2 : 4;
  L.niL = std::max(1 + L.niA, 2 + L.nk);
  int pos = 0;
  auto alloc = [&](std::vector<int>& r, int w) {
    r.clear();
    for (int j = 0; j < w; ++j) r.push_back(pos++);
  };
  alloc(L.t, 1);
  alloc(L.s, 1);
  alloc(L.iL, L.niL);
  alloc(L.q1, 2);
  alloc(L.a1, L.na);
  if (NC == 2) {
    alloc(L.q2, 2);
    alloc(L.a2, L.na);
    alloc(L.ord, 1);
  }
  alloc(L.k, L.nk);
  alloc(L.m, L.nm);
  L.n = pos;
  L.i.assign(L.iL.begin(), L.iL.begin() + 2);
  if (NC == 2) L.cs.assign(L.iL.begin() + 2, L.iL.begin() + 4);
  L.e.assign(L.iL.begin() + L.niA, L.iL.end());
  L.l.assign(L.iL.begin(), L.iL.begin() + L.nk);
  L.unused.assign(L.iL.begin() + L.nk, L.iL.begin() + (L.niL - 2));
  L.km = L.k;
  L.km.insert(L.km.end(), L.m.begin(), L.m.end());
  L.top = L.iL[L.niL - 1];
  L.sel = L.iL[L.niL - 2];
  *out = L;
  return true;
}

double collision_coeff(int qp, int q, double tau) {
  return (1.0 - 1.0 / tau) * (qp == q ? 1.0 : 0.0) + W[qp] / tau * (1.0 + 3.0 * E[qp] * E[q]);
}

double k12(int qp, int q1, int q2, double tau) {
  return W[qp] / tau * (4.5 * (E[q1] * E[qp]) * (E[q2] * E[qp]) - 1.5 * (E[q1] * E[q2]));
}

double v11(int qo, int io, double tau) {
  if (qo <= 2 && io <= 2) {
    double v = collision_coeff(qo, io, tau);
    if (qo == 2 && io == 2) v = v - 1.0;
    return v;
  }
  if (qo <= 1 && io == 3) return -1.0;
  return 0.0;
}

// max |A_ij| of the assembled Carleman matrix.  Bounce-back walls add one
// diagonal entry per wall, c(q', qbar') - 1, and its sums with the second
// copy's diagonal in A22.
double max_abs_A(double tau, int NC, int bc) {
  std::vector<double> vals;
  for (int qp = 0; qp < 3; ++qp)
    for (int q = 0; q < 3; ++q)
      if (!(qp == 2 && q == 2)) vals.push_back(collision_coeff(qp, q, tau));
  const double c22m1 = collision_coeff(2, 2, tau) - 1.0;
  vals.push_back(c22m1);
  vals.push_back(-1.0);
  if (NC == 2) {
    for (int qp = 0; qp < 3; ++qp)
      for (int q1 = 0; q1 < 3; ++q1)
        for (int q2 = 0; q2 < 3; ++q2) vals.push_back(k12(qp, q1, q2, tau));
    vals.push_back(-1.0 + -1.0);
    vals.push_back(-1.0 + c22m1);
    vals.push_back(c22m1 + c22m1);
  }
  if (bc == CSIM_BC_BOUNCEBACK) {
    const double walls[2] = {collision_coeff(0, 1, tau) - 1.0, collision_coeff(1, 0, tau) - 1.0};
    for (double w : walls) vals.push_back(w);
    if (NC == 2)
      for (double w : walls) {
        vals.push_back(w + -1.0);
        vals.push_back(w + c22m1);
        for (double w2 : walls) vals.push_back(w + w2);
      }
  }
  double m = 0.0;
  for (double v : vals) m = std::max(m, std::fabs(v));
  return m;
}

double lmax_value(double tau, int NC, double dt, int bc) {
  return std::max(1.0, dt * max_abs_A(tau, NC, bc));
}

namespace {
double theta0(double v, int ko, double dt, double Lmax) {
  return v != 0.0 ? theta(v, ko, dt, Lmax) : 0.0;
}

// Bounce-back value corrections: an output (qo, io) at its wall site (a = Nx-1
// for qo = 1, a = 0 for qo = 0) carries the entry of the opposite velocity,
// v(1 - qo, io), instead of v(qo, io); a second RY on t adds the angle
// difference there.  nio input labels (3 for A11, 4 for A12).
template <typename F>
void wall_fix(std::vector<Gate>& g, const Layout& L, const Ctrl& base, const std::vector<int>& areg,
              const std::vector<int>& qreg, F vfun, int nio, int ko, double dt, double Lmax) {
  const int t = L.t[0];
  for (int qo = 0; qo < 2; ++qo)
    for (int io = 0; io < nio; ++io) {
      const double tw = theta0(vfun(1 - qo, io), ko, dt, Lmax);
      const double tg = theta0(vfun(qo, io), ko, dt, Lmax);
      if (tw != tg) {
        Ctrl c = merge(base, reg_eq(qreg, (uint64_t)qo),
                       reg_eq(areg, qo == 1 ? (uint64_t)(L.Nx - 1) : 0));
        c = merge(c, reg_eq(L.i, (uint64_t)io));
        g.push_back(gate(OP_RY, t, c, tw - tg, TAG_VALUE));
      }
    }
}
}  // namespace

std::vector<Gate> build_UL(const Layout& L, double tau, double dt) {
  const double Lmax = lmax_value(tau, L.NC, dt, L.bc);
  const bool bb = L.bc == CSIM_BC_BOUNCEBACK;
  const int t = L.t[0];
  const Ctrl T = all_eq(L.e, 0);
  const Ctrl C = merge(bit_eq(L.top, 1), bit_eq(L.sel, 0));
  std::vector<Gate> g;
  for (int b : L.iL) g.push_back(gate(OP_H, b, Ctrl{}, 0.0, TAG_HPREP));
  // permutation
  if (L.NC == 2) {
    const int od = L.ord[0];
    p11(g, L.a1, L.q1, L.i, merge(T, reg_eq(L.cs, 0), bit_eq(od, 0)), TAG_PERM, bb);
    p11(g, L.a1, L.q1, L.i, merge(T, reg_eq(L.cs, 1), bit_eq(od, 1)), TAG_PERM, bb);
    p11(g, L.a2, L.q2, L.i, merge(T, reg_eq(L.cs, 2), bit_eq(od, 1)), TAG_PERM, bb);
    pi3(g, L, merge(T, reg_eq(L.cs, 3)), TAG_PERM, bb);
  } else {
    p11(g, L.a1, L.q1, L.i, T, TAG_PERM, bb);
  }
  inc(g, L.k, T, TAG_PERM);
  for (const Pattern& p : prefix_patterns(0, (uint64_t)L.Nt, L.nm)) {
    const Ctrl pc = pattern_ctrl(L.m, p);
    for (int b = 0; b < L.nk; ++b)
      g.push_back(gate(OP_X, L.l[b], merge(C, pc, bit_eq(L.k[b], 1)), 0.0, TAG_PERM));
    for (int b = 0; b < L.nk; ++b)
      g.push_back(gate(OP_X, L.k[b], merge(C, pc, bit_eq(L.l[b], 1)), 0.0, TAG_PERM));
    for (int b = 0; b < L.nk; ++b) g.push_back(gate(OP_X, L.k[b], merge(C, pc), 0.0, TAG_PERM));
  }
  inc(g, L.km, C, TAG_PERM);
  // value encoding on the post-permutation state
  for (int kn = 1; kn <= L.K; ++kn) {
    for (const Pattern& p : prefix_patterns(0, (uint64_t)L.Nt, L.nm)) {
      const Ctrl base = merge(T, reg_eq(L.k, (uint64_t)kn), pattern_ctrl(L.m, p));
      if (L.NC == 2) {
        const int od = L.ord[0];
        struct Case {
          int cval, ordv;
          const std::vector<int>* q;
        };
        const Case cases[3] = {{0, 0, &L.q1}, {1, 1, &L.q1}, {2, 1, &L.q2}};
        auto vA11 = [tau](int qo, int io) { return v11(qo, io, tau); };
        auto vA12 = [tau](int qo, int io) { return k12(qo, io & 1, io >> 1, tau); };
        for (const Case& cc : cases) {
          for (int qo = 0; qo < 3; ++qo)
            for (int io = 0; io < 4; ++io) {
              const double v = v11(qo, io, tau);
              if (v != 0.0) {
                Ctrl c = merge(base, reg_eq(L.cs, (uint64_t)cc.cval), bit_eq(od, cc.ordv),
                               reg_eq(*cc.q, (uint64_t)qo));
                c = merge(c, reg_eq(L.i, (uint64_t)io));
                g.push_back(gate(OP_RY, t, c, theta(v, kn - 1, dt, Lmax), TAG_VALUE));
              }
            }
          if (bb)
            wall_fix(g, L, merge(base, reg_eq(L.cs, (uint64_t)cc.cval), bit_eq(od, cc.ordv)),
                     cc.q == &L.q1 ? L.a1 : L.a2, *cc.q, vA11, 3, kn - 1, dt, Lmax);
        }
        for (int qo = 0; qo < 3; ++qo)
          for (int io = 0; io < 4; ++io) {
            const double v = k12(qo, io & 1, io >> 1, tau);
            if (v != 0.0) {
              Ctrl c = merge(base, reg_eq(L.cs, 3), bit_eq(od, 0), reg_eq(L.a2, 0));
              c = merge(c, reg_eq(L.q2, 0), reg_eq(L.q1, (uint64_t)qo), reg_eq(L.i, (uint64_t)io));
              g.push_back(gate(OP_RY, t, c, theta(v, kn - 1, dt, Lmax), TAG_VALUE));
            }
          }
        if (bb)
          wall_fix(g, L,
                   merge(merge(base, reg_eq(L.cs, 3), bit_eq(od, 0)), reg_eq(L.a2, 0),
                         reg_eq(L.q2, 0)),
                   L.a1, L.q1, vA12, 4, kn - 1, dt, Lmax);
      } else {
        for (int qo = 0; qo < 3; ++qo)
          for (int io = 0; io < 4; ++io) {
            const double v = v11(qo, io, tau);
            if (v != 0.0) {
              Ctrl c = merge(base, reg_eq(L.q1, (uint64_t)qo), reg_eq(L.i, (uint64_t)io));
              g.push_back(gate(OP_RY, t, c, theta(v, kn - 1, dt, Lmax), TAG_VALUE));
            }
          }
        if (bb)
          wall_fix(g, L, base, L.a1, L.q1, [tau](int qo, int io) { return v11(qo, io, tau); }, 3,
                   kn - 1, dt, Lmax);
      }
    }
  }
  const Ctrl unused0 = all_eq(L.unused, 0);
  const double th_m1 = 2.0 * std::asin(-1.0 / Lmax);
  for (const Pattern& pm : prefix_patterns(1, (uint64_t)L.Nt + 1, L.nm))
    for (const Pattern& pl : prefix_patterns(0, (uint64_t)L.K + 1, L.nk)) {
      Ctrl c = merge(C, unused0, reg_eq(L.k, 0), pattern_ctrl(L.m, pm));
      c = merge(c, pattern_ctrl(L.l, pl));
      g.push_back(gate(OP_RY, t, c, th_m1, TAG_VALUE));
    }
  for (const Pattern& pc : prefix_patterns((uint64_t)L.Nt * (1ull << L.nk) + 1,
                                           1ull << (L.nk + L.nm), L.nk + L.nm)) {
    Ctrl c = merge(C, unused0, reg_eq(L.l, 0), pattern_ctrl(L.km, pc));
    g.push_back(gate(OP_RY, t, c, th_m1, TAG_VALUE));
  }
  g.push_back(gate(OP_RY, t, all_eq(L.iL, 1), 2.0 * std::asin(1.0 / Lmax), TAG_VALUE));
  for (int b : L.iL) g.push_back(gate(OP_H, b, Ctrl{}, 0.0, TAG_HUNPREP));
  g.push_back(gate(OP_X, t, Ctrl{}, 0.0, TAG_TFLIP));
  return g;
}

std::vector<Gate> dagger(const std::vector<Gate>& g) {
  std::vector<Gate> out(g.rbegin(), g.rend());
  for (Gate& x : out)
    if (x.op == OP_RY || x.op == OP_ZPHASE) x.angle = -x.angle;
  return out;
}

std::vector<Gate> phase_gates(const Layout& L, double phi) {
  Ctrl anc0 = merge(all_eq(L.iL, 0), all_eq(L.t, 0));
  const int s = L.s[0];
  return {gate(OP_X, s, anc0, 0.0, TAG_PHASE), gate(OP_ZPHASE, s, Ctrl{}, phi, TAG_PHASE),
          gate(OP_X, s, anc0, 0.0, TAG_PHASE)};
}

std::vector<Gate> build_qsvt(const Layout& L, const std::vector<Gate>& UL,
                             const std::vector<double>& phases) {
  const int d = (int)phases.size() - 1;
  const std::vector<Gate> ULd = dagger(UL);
  std::vector<Gate> g;
  g.reserve((size_t)d * (UL.size() + 3) + 8);
  const int s = L.s[0];
  g.push_back(gate(OP_H, s, Ctrl{}, 0.0, TAG_SIGNAL));
  for (const Gate& x : phase_gates(L, phases[0])) g.push_back(x);
  for (int j = 1; j <= d; ++j) {
    // the first call on b is U_L^dag: P^{SV}(L^T/lambda) ~ lambda L^{-1} (Sec. II.D.5)
    const std::vector<Gate>& U = (j % 2 == 1) ? ULd : UL;
    g.insert(g.end(), U.begin(), U.end());
    for (const Gate& x : phase_gates(L, phases[j])) g.push_back(x);
  }
  g.push_back(gate(OP_H, s, Ctrl{}, 0.0, TAG_SIGNAL));
  return g;
}

void postselect_patterns(const Layout& L, std::vector<uint64_t>* masks,
                         std::vector<uint64_t>* vals) {
  masks->clear();
  vals->clear();
  Ctrl base = merge(all_eq(L.s, 0), all_eq(L.t, 0), all_eq(L.iL, 0));
  for (const Pattern& p : prefix_patterns((uint64_t)L.Nt, 1ull << L.nm, L.nm)) {
    Ctrl c = merge(base, pattern_ctrl(L.m, p));
    masks->push_back(c.mask);
    vals->push_back(c.val);
  }
}

double gate_amp_updates(const Gate& g, int n) {
  // amplitudes the gate changes: all 2^{n-c} matching amplitudes for a dense or
  // diagonal 2x2 (H, RY, ZPHASE); for X the same (both halves of each pair move)
  int c = __builtin_popcountll(g.cmask);
  return std::ldexp(1.0, n - c);
}

}  // namespace csim
