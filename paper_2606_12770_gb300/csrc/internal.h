// Internal declarations shared by the host compiler, the fuser, the C ABI and
// the CUDA kernels.  Not part of the public interface (include/csim.h is).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/csim.h"

namespace csim {

enum : uint8_t { OP_X = 0, OP_H = 1, OP_RY = 2, OP_ZPHASE = 3 };
enum : uint16_t {
  TAG_HPREP = 1, TAG_PERM = 2, TAG_VALUE = 3, TAG_HUNPREP = 4,
  TAG_TFLIP = 5, TAG_PHASE = 6, TAG_SIGNAL = 7
};

using Gate = csim_gate;

// Register layout of Sec. II.D (bit positions, little-endian registers).
struct Layout {
  int Nx = 0, NC = 0, K = 0, Nt = 0;
  int bc = CSIM_BC_PERIODIC;  // boundary condition of the streaming step (reading R2)
  int na = 0, nk = 0, nm = 0, niA = 0, niL = 0, n = 0;
  std::vector<int> t, s, iL, i, cs, e, l, unused, q1, a1, q2, a2, ord, k, m, km;
  int top = -1, sel = -1;
};

bool make_layout(int Nx, int NC, int K, int Nt, Layout* out, std::string* err);

// Physics constants and value tables (Eqs. A11-elements, A12-kernel).
double collision_coeff(int qp, int q, double tau);
double k12(int qp, int q1, int q2, double tau);
double v11(int qo, int io, double tau);
double max_abs_A(double tau, int NC, int bc = CSIM_BC_PERIODIC);
double lmax_value(double tau, int NC, double dt, int bc = CSIM_BC_PERIODIC);

// Gate lists of the ancilla-free construction: U_A as one permutation of
// (site, velocity, label) followed by RY value encodings on t, U_L as the
// Taylor / coupling / identity label classes over (k, m), the QSVT wrapper
// with signal Hadamards and projector phases (Fig. circuit-qsvt).
std::vector<Gate> build_UL(const Layout& L, double tau, double dt);
std::vector<Gate> dagger(const std::vector<Gate>& g);
std::vector<Gate> phase_gates(const Layout& L, double phi);
std::vector<Gate> build_qsvt(const Layout& L, const std::vector<Gate>& UL,
                             const std::vector<double>& phases);
void postselect_patterns(const Layout& L, std::vector<uint64_t>* masks,
                         std::vector<uint64_t>* vals);

// Classical pieces needed to choose the QSVT polynomial (host, FP64).
double kappa_of_L(const Layout& L, double tau, double dt, std::string* err);
int degree_from_kappa(double kappa, double eps);
// Target odd polynomial ~ 1/x on [1/kappa, 1] (values at given x) and its scale.
double inverse_target_scale(double kappa, int d);
double inverse_target_value(double kappa, int d, double scale, double x);
// Phases (reflection convention of Fig. circuit-qsvt) with Re P = target.
bool solve_phases(double kappa, int d, std::vector<double>* phases, double* scale,
                  std::string* err);

// Number of amplitudes a gate changes (the algorithmic work unit).
double gate_amp_updates(const Gate& g, int n);

}  // namespace csim
