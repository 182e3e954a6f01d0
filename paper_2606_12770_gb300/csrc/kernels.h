// Host-side launch interface of the CUDA kernels in kernels.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/csim.h"

namespace csim {

// One multi-controlled X of a fused permutation, in chunk-index space
// (state index >> 2; the two lowest qubits never take part).
struct PermOp {
  uint64_t mask, val, tbit;
};

// One gate acting inside the 128-amplitude warp tile (target qubit 0..6);
// controls may sit on any qubit.  c, s: RY cos/sin(theta/2), ZPHASE cos/sin(phi).
struct LocalOp {
  uint64_t cmask, cval;
  int32_t op, target;
  double c, s;
};

cudaError_t launch_init(void* state, int prec, uint64_t n_amps, const uint64_t* d_idx,
                        const double* d_val, int64_t count, cudaStream_t st);
cudaError_t launch_gate(void* state, int prec, int n, const csim_gate& g, cudaStream_t st);
cudaError_t launch_sweep(const void* in, void* out, int prec, int n, const PermOp* d_perm,
                         int nperm, const LocalOp* d_ops, int nops, cudaStream_t st);
int norm_partials_needed();
cudaError_t launch_norms(const void* state, int prec, int n, const uint64_t* d_pm,
                         const uint64_t* d_pv, int npat, double* d_partial, double* d_out,
                         cudaStream_t st);
cudaError_t launch_compact(const void* state, int prec, double* d_out, uint64_t count,
                           int free_shift, int free_bits, uint64_t m_first, int m_shift,
                           cudaStream_t st);

}  // namespace csim
