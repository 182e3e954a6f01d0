// Gate-list -> executable program (the fuser) and its executor.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "dense.h"
#include "internal.h"
#include "kernels.h"

namespace csim {

struct Step {
  int kind = 0;    // 0 = fused sweep, 1 = single gate, 2 = dense 5-qubit block
  int param = -1;  // index into Program::params (sweeps) or Program::dense (blocks)
  bool gather = false;  // the sweep has segments (moves data)
  bool inplace = false;  // ... and stores back to the gathered addresses (in == out)
  csim_gate g{};
};

struct FuseStats {
  int64_t sweeps = 0, single = 0, perm_gates = 0, segments = 0, local_gates = 0, mux = 0;
  int64_t mux_gates = 0, mux_entries = 0, max_bucket = 0, lut_entries = 0, max_support = 0;
  int64_t reflect = 0;
  int64_t mux_inverse = 0;  // multiplexers run as the inverse of the sweep's previous one
  int64_t wht = 0;          // Walsh-Hadamard ops (H on several lane bits)
  int64_t conjugated = 0;   // in-place P^-1 . ops . P sweeps
  int64_t staged_sweeps = 0;  // sweeps that stage qubits above the tile
  int64_t staged_gates = 0;   // gates on staged qubits
  int64_t dense_blocks = 0;   // runs of gates on at most 5 qubits applied as one dense block
  int64_t dense_gates = 0;    // gates in those runs
};

struct Program {
  int n = 0;
  csim_exec mode = CSIM_EXEC_FUSED;
  bool scatter = false;  // sweep form: [ops][scatter] instead of [gather][ops]
  std::vector<Step> steps;
  std::vector<SweepParams> params;
  std::vector<uint16_t> lut;
  std::vector<uint32_t> mtab;
  std::vector<MuxEntryF> mentf;
  std::vector<MuxEntryD> mentd;
  std::vector<float2> angf;
  std::vector<double2> angd;
  // device copies of the tables
  uint16_t* d_lut = nullptr;
  uint32_t* d_mtab = nullptr;
  MuxEntryF* d_mentf = nullptr;
  MuxEntryD* d_mentd = nullptr;
  float2* d_angf = nullptr;
  double2* d_angd = nullptr;
  int64_t passes = 0;        // HBM passes per execution
  double pass_amps = 0.0;    // amplitudes the passes read (and write) at minimum: 2^n per
                             // sweep, the changed amplitudes per single-gate step
  double amp_updates = 0.0;  // sum over elementary gates of amplitudes changed
  bool pingpong = false;     // some step moves data out of place
  bool uploaded = false;
  FuseStats stats;
  // identical permutation runs and multiplexers (every U_L call of a QSVT
  // circuit repeats them) share one table: content -> table offset
  std::unordered_map<std::string, uint32_t> lut_cache, mux_cache;
  std::vector<MuxDesc> mux_descs;  // compiled multiplexers, indexed by mux_cache
  // mux_inv[i]: the compiled multiplexer whose gates are those of i with the
  // angles negated (its inverse; the gates commute), or -1.  mux_sig maps the
  // order-free gate content of each multiplexer to its index.
  std::vector<int> mux_inv;
  std::unordered_map<std::string, uint32_t> mux_sig;
  std::unordered_map<std::string, std::string> order_cache;  // segments -> fast tile bits
  // source-index tables of the gather sweeps (build_src_index), one per
  // distinct segment chain
  std::vector<uint32_t*> d_src;
  bool src_tried = false;
  // plan_src_index: the table of each sweep's chain (by params index, -1 for
  // none) and the first sweep of each table
  std::vector<int> src_tab, src_first;
  bool src_planned = false;
  // dense 5-qubit blocks (complex64 programs only; Step kind 2) and the
  // engine that applies them (DENSE_TC or DENSE_FP32)
  std::vector<DenseBlock> dense;
  int dense_engine = DENSE_TC;
  int stage_k = kMaxStage;  // most qubits a sweep stages above the tile
  bool dense_on = false;    // runs on <= 5 qubits were eligible for dense blocks
};

// Build the program for `gates` on an n-qubit state.  FUSED mode needs
// 7 <= n <= 34 (the warp tile and 32-bit chunk indices); other sizes fall
// back to one launch per gate.  The sweep form is gather unless
// CSIM_SWEEP_FORM=scatter.
// With allow_dense (complex64 states of at least 12 qubits), a run of at
// least CSIM_DENSE_MIN (default 10) consecutive gates that touch at most five
// qubits becomes one dense block on the tensor cores (CSIM_DENSE=0 turns
// this off; CSIM_DENSE_ENGINE=fp32 applies the blocks on the CUDA cores).
// stage_k (0..3) overrides the staging width (CSIM_STAGE, default 3);
// dense_mode overrides CSIM_DENSE (0 off, 1 runs that mix across the warp
// tile, 2 every long run, -1 the switch).
void build_program(const std::vector<csim_gate>& gates, int n, csim_exec mode, Program* p,
                   bool allow_dense = false, int stage_k = -1, int dense_mode = -1);
cudaError_t upload_program(Program* p, cudaStream_t st);
void free_program(Program* p);
// After upload_program: precompute the source-index table of each distinct
// gather chain (2^(n-2) uint32 entries, 2^n bytes each), so that the sweeps
// load one index per chunk instead of walking the lookup-table chain.  Skipped
// (the sweeps keep the chain) when CSIM_SRC_INDEX=0, when the program has more
// than max_tables distinct chains, or when the tables would take more than a
// quarter of the free device memory.  Runs once per program.
cudaError_t build_src_index(Program* p, cudaStream_t st, int max_tables);
// The distinct chains of the program's data-moving sweeps (cached): returns
// how many source-index tables the program takes, 0 when it keeps the chain
// (CSIM_SRC_INDEX=0, more than max_tables chains, n < 7).
int plan_src_index(Program* p, int max_tables);
// Fill caller-owned tables (2^(n-2) uint32 each, one per planned chain) on st.
cudaError_t launch_src_tables(const Program& p, uint32_t* const* tables, cudaStream_t st);
// Run the program on buf[*cur] (and buf[1 - *cur] when it moves data); *cur
// tracks which buffer holds the state afterwards.
// With src_tables (caller-owned, from launch_src_tables), the sweeps load
// their source indices from those tables instead of the program's own.
cudaError_t run_program(const Program& p, void* buf[2], int* cur, int prec, cudaStream_t st,
                        const uint32_t* const* src_tables = nullptr);
// Steps [first, last) of the program only (checkpointed runs).  zero_map
// (launch_init_sparse) goes to the first zero_steps steps, when they are
// among them: with zero_steps = 1, step 0 in mode 1; with 2, step 0 in mode 2
// and step 1 in mode 3 (SweepParams::zero_mode).
// With norm_part (kNormPartCap doubles) and program_fuses_norm, the
// program's last sweep also sums |a|^2 of the final state into it, when it
// is among the steps run (launch_norms_fused then takes the total from it).
cudaError_t run_program_steps(const Program& p, void* buf[2], int* cur, int prec, cudaStream_t st,
                              int64_t first, int64_t last,
                              const uint32_t* const* src_tables = nullptr,
                              const uint32_t* zero_map = nullptr, int zero_steps = 0,
                              double* norm_part = nullptr);
// Whether the program's last step is a sweep that can sum the final state's
// |a|^2 (sweep_fuses_norm).
bool program_fuses_norm(const Program& p, int prec);
// Host executor of a fused program (FP64, kernel semantics) for testing.
void emulate_program(const Program& p, std::vector<double>* amps);

}  // namespace csim
