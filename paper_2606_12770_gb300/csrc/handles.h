// Handle structures behind the opaque types of include/csim.h, and the
// helpers that the C ABI (capi.cpp) and the request pool (pool.cpp) share.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "fuse.h"
#include "internal.h"

struct csim_circuit {
  csim::Layout L;
  double tau = 0, dt = 0, eps = 1e-3, kappa = 0, scale = 0, Lmax = 0, lambda = 0;
  int d = 0, max_qubits = 34;
  std::vector<csim::Gate> UL;
  std::vector<double> phases;
  std::vector<uint64_t> pm, pv;
  // device side
  int prec = -1;
  cudaStream_t stream = nullptr;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  size_t bytes = 0;
  csim_exec exec = CSIM_EXEC_FUSED;
  bool loaded = false, ran = false;
  int64_t next_step = 0;  // next program step of a run in progress (csim_run_steps)
  // sparse csim_init: only the tiles of b were written (d_zmap marks them);
  // the program's first zero_steps sweeps (1 or 2) write the zeros of the
  // others.  Until they have run, zero_fill is set, and reading the state
  // zeroes the unmarked tiles first.
  bool zero_fill = false;
  int zero_steps = 0;
  int sparse_init = 0;  // zero_steps of the last csim_init, 0 if plain (csim_info)
  uint32_t* d_zmap = nullptr;
  csim::Program prog;
  bool prog_built = false;
  uint64_t* d_pat = nullptr;  // masks then values
  double* d_partial = nullptr;
  double* d_out = nullptr;
  double* d_compact = nullptr;
  size_t compact_cap = 0;
  // the last sweep's |a|^2 partials (kNormPartCap doubles), and whether they
  // hold the total of the current state (set by a run that ended with a
  // fused last sweep, cleared by anything else that writes the state)
  double* d_npart = nullptr;
  bool norm_fused = false;
};

struct csim_sv {
  int n = 0, prec = 0;
  cudaStream_t stream = nullptr;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  size_t bytes = 0;
  csim::Program prog;
  bool compiled = false;
  csim::DenseBlock dense;            // the block of the latest csim_sv_apply_dense
  unsigned int timeouts_seen = 0;    // the tensor-core wait timeouts already reported
  int tune_stage = -1, tune_dense = -1;  // csim_sv_autotune's choice (-1: defaults)
};

namespace csim {

uint64_t place_bits(const std::vector<int>& bits, uint64_t v);
// Build (once, host only) the fused or gate-by-gate program of the circuit.
void ensure_built(csim_circuit* c);
// ensure_built, then upload the program's tables to the device (once).
bool ensure_program(csim_circuit* c, cudaStream_t st, std::string* err);
// Leading sweeps of the fused program that complete a sparse init (0, 1, 2).
int zero_fill_steps(const csim_circuit* c, int prec);
bool sparse_init_enabled();
// Normalised right-hand side b = (f, f (x) f) as (state index, value) pairs
// (Sec. II.D.5); false with a message for a non-finite or zero f0.
bool circuit_rhs(const csim_circuit* c, const double* f0, std::vector<uint64_t>* idx,
                 std::vector<double>* val, std::string* err);
// Lowest index bits that every postselection pattern fixes to the same value.
void mask_low_bits(const csim_circuit* c, int* lowk, uint64_t* lowv);
// Geometry of the compacted postselected block (m >= Nt, s = t = label = 0).
struct CompactGeom {
  int free_shift = 0, free_bits = 0, m_shift = 0;
  uint64_t count = 0;
};
CompactGeom compact_geom(const csim_circuit* c);

}  // namespace csim
