// Gate-list -> executable program (the fuser) and its executor.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "internal.h"
#include "kernels.h"

namespace csim {

struct Step {
  int kind = 0;  // 0 = fused sweep, 1 = single gate
  int perm_off = 0, perm_cnt = 0, op_off = 0, op_cnt = 0;
  csim_gate g{};
};

struct Program {
  int n = 0;
  csim_exec mode = CSIM_EXEC_FUSED;
  std::vector<Step> steps;
  std::vector<PermOp> perm;
  std::vector<LocalOp> ops;
  PermOp* d_perm = nullptr;
  LocalOp* d_ops = nullptr;
  int64_t passes = 0;         // HBM passes per execution
  double amp_updates = 0.0;   // sum over elementary gates of amplitudes changed
  bool pingpong = false;      // some step gathers out of place
  bool uploaded = false;
};

// Build the program for `gates` on an n-qubit state.  FUSED mode needs n >= 7
// (the warp tile); smaller states fall back to one launch per gate.
void build_program(const std::vector<csim_gate>& gates, int n, csim_exec mode, Program* p);
cudaError_t upload_program(Program* p, cudaStream_t st);
void free_program(Program* p);
// Run the program on buf[*cur] (and buf[1 - *cur] when it gathers); *cur tracks
// which buffer holds the state afterwards.
cudaError_t run_program(const Program& p, void* buf[2], int* cur, int prec, cudaStream_t st);

}  // namespace csim
