// Dense 5-qubit blocks (dense.cu): host-side launch interface.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace csim {

// Kernel parameters of one dense block on an n-qubit complex64 state.
struct DenseParams {
  // A tile is 128 groups of 32 amplitudes.  Its 12 local index bits (7 for
  // the group within the tile, 5 for the element of the group) in ascending
  // order of their state bit: pos[m] is the state bit of local bit m, tag[m]
  // its role (0-6: bit of the group in the tile; 8-12: element bit tag - 8).
  uint8_t pos[12];
  uint8_t tag[12];
  uint8_t nonq[32];  // state bits outside the block and its selectors, ascending
  uint8_t q[5];      // the block's qubits, ascending (element bits)
  // Selector qubits (at most 2): the block applies matrix y to the groups
  // whose selector bits read y.  They are the lowest bits of the tile index,
  // and the grid is a multiple of 2^nsel, so each CTA keeps one y.
  uint8_t nsel;
  uint8_t sel[2];
  int n;
  uint32_t ntiles;   // 2^(n - 12)
  // tensor-core path: per selector value, W^T in two BF16 planes (hi then
  // lo, 8 KB each) in the operand layout the MMA reads; FP32 path: per
  // selector value, U as 32 x 32 float2, row-major
  const uint4* bimg;
  const float2* uf;
  uint32_t spin;           // iterations of the mbarrier wait before it gives up
  unsigned int* timeouts;  // incremented (device) once per CTA that gave up
};

enum DenseEngine : int { DENSE_TC = 0, DENSE_FP32 = 1 };

// Everything the device needs for one block, built on the host from U (32 x
// 32 complex, row-major, interleaved re/im doubles) and the block's qubits.
struct DenseBlock {
  uint8_t q[5];
  uint8_t nsel = 0, sel[2] = {0, 0};  // selector qubits (matrix y acts where they read y)
  std::vector<double> u;        // 2^nsel x (2 x 32 x 32)
  std::vector<uint16_t> bimg;   // 2^nsel x (2 x 4096 BF16 bits: hi plane, lo plane)
  std::vector<float> uf;        // 2^nsel x (2 x 32 x 32)
  uint4* d_bimg = nullptr;      // device copies (upload_dense)
  float2* d_uf = nullptr;
  size_t d_bimg_bytes = 0, d_uf_bytes = 0;
};

// Fill bimg and uf from u.
void make_dense_block(DenseBlock* b);
cudaError_t upload_dense(DenseBlock* b, cudaStream_t st);
void free_dense(DenseBlock* b);
// Apply the block to the n-qubit complex64 state (n >= 12 + nsel for the
// tensor cores; the FP32 engine takes n >= 5 + nsel).
cudaError_t launch_dense(void* state, int n, const DenseBlock& b, int engine, cudaStream_t st);
// Timeouts counted by the tensor-core kernel's bounded waits since the
// library loaded (a device counter, read synchronously).
cudaError_t dense_timeouts(unsigned int* out);
// Kernel load and occupancy cache (before any stream capture).
cudaError_t warm_dense();

}  // namespace csim
