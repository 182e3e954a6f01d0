// Host-side launch interface of the CUDA kernels in kernels.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/csim.h"

namespace csim {

// Bits [lo, lo+len) of a 32-bit chunk index (state index >> 2) are bits
// [off, off+len) of a table key.
struct BitRun {
  uint8_t lo, len, off, pad;
};

constexpr int kMaxRuns = 8;

// A run of multi-controlled X gates compiled to a lookup table over the
// chunk-index bits they read or write (their support): the table maps the
// support bits of an index to the support bits of its image.
struct PermSeg {
  uint32_t supmask;
  uint32_t lut_off;  // into the uint16 table array
  uint32_t nruns;
  BitRun runs[kMaxRuns];
};

// One gate inside the 128-amplitude warp tile.  Controls are split into the
// chunk-index part (state bits >= 2) and state bits 0-1.
// op: 0 X, 1 H, 2 RY, 3 ZPHASE, 4 multiplexed RY (cm = index of its MuxDesc),
// 5 averaging block (cm = index of its ReflectDesc).
struct LocalOp {
  uint32_t cm, cv;
  uint8_t lm, lv, op, target;
  float cf, sf;   // RY cos/sin(theta/2); ZPHASE cos/sin(phi)
  double cd, sd;  // the same in FP64
};

// Multiplexed RY on an in-thread qubit: key bits of the chunk index select a
// bucket of candidate gates; each candidate's chunk controls are checked in
// full.  All candidates share the controls (lm, lv) on state bits 0-1.
struct MuxDesc {
  uint32_t nruns;
  BitRun runs[kMaxRuns];
  uint32_t tab_off;  // into the bucket table: entry start << 8 | count
  uint8_t target, lm, lv, pad;
};
struct MuxEntryF {
  uint32_t cm, cv;
  float c, s;
};
struct MuxEntryD {
  uint32_t cm, cv;
  uint32_t pad0, pad1;
  double c, s;
};

// A window of tile-local gates whose 128 x 128 matrix is I (x) A + J (x) B on
// (lane bits) x (bits 0-1), J the summing matrix over the lane bits in
// `lanemask`: out[l][y] = sum_y' A[y][y'] v[l][y'] + B[y][y'] sum_l'(v[l'][y']),
// the sum running over the lanes that differ from l only in `lanemask` bits.
// A and B are dense 4 x 4 (index y*4+y'); nzA / nzB flag the non-zero entries.
struct ReflectDesc {
  uint32_t lanemask;
  uint32_t nzA, nzB;
  uint32_t pad;
  float2 af[16], bf[16];
  double2 ad[16], bd[16];
};

// Everything one sweep launch needs, passed by value in the kernel parameter
// block (constant bank): the permutation segments, the tile-local ops and
// their descriptors.  Large tables stay in global memory.
constexpr int kMaxSeg = 12, kMaxOps = 40, kMaxRefl = 4, kMaxMux = 8;
struct SweepParams {
  int nseg, nops, scatter, pad;
  PermSeg segs[kMaxSeg];
  LocalOp ops[kMaxOps];
  ReflectDesc refl[kMaxRefl];
  MuxDesc mux[kMaxMux];
  const uint16_t* lut;
  const uint32_t* mtab;
  const MuxEntryF* mentf;
  const MuxEntryD* mentd;
};

cudaError_t launch_init(void* state, int prec, uint64_t n_amps, const uint64_t* d_idx,
                        const double* d_val, int64_t count, cudaStream_t st);
cudaError_t launch_gate(void* state, int prec, int n, const csim_gate& g, cudaStream_t st);
cudaError_t launch_sweep(const void* in, void* out, int prec, int n, const SweepParams& a,
                         cudaStream_t st);
int norm_partials_needed();
cudaError_t launch_norms(const void* state, int prec, int n, const uint64_t* d_pm,
                         const uint64_t* d_pv, int npat, double* d_partial, double* d_out,
                         cudaStream_t st);
cudaError_t launch_compact(const void* state, int prec, double* d_out, uint64_t count,
                           int free_shift, int free_bits, uint64_t m_first, int m_shift,
                           cudaStream_t st);

}  // namespace csim
