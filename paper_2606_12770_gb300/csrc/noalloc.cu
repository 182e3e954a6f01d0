// csim_norms_noalloc: the FP64 norm reduction for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside another
// framework's memory pool that forbids side allocations, or a host that must
// keep its device footprint fixed after start-up. csim_postselect cannot
// serve them, because it needs a library-allocated buffer of per-block
// partial sums. This variant keeps those partial sums in a fixed
// file-scope device array instead.
//
// The array is a static module variable, so every GPU that loads the library
// holds it (kNoAllocBlocks partial pairs, 32 KiB) until the process exits.
// The entry point allocates nothing: no cudaMalloc, no cudaFree, and no
// library routine that allocates.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/csim.h"

namespace csim {
void record_last_error(const std::string& msg);  // capi.cpp: the text csim_last_error returns
}

namespace {

constexpr int kNoAllocBlocks = 2048;    // partial (total, masked) pairs the array holds
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxPatterns = 16; // patterns travel by value in the launch
constexpr int kNoAllocMaxQubits = 34;
constexpr int kMaxDevices = 64;

// Scratch: one (total, masked) pair per block of the reduction. In host code
// this name is only a stand-in for the symbol; the device address comes
// from cudaGetSymbolAddress (see scratch_on_current_device).
static __device__ __align__(256) double g_norm_scratch[2 * kNoAllocBlocks];

struct Patterns {
  uint64_t m[kNoAllocMaxPatterns];
  uint64_t v[kNoAllocMaxPatterns];
};

csim_status na_fail(csim_status s, const std::string& msg) {
  csim::record_last_error(msg);
  return s;
}

template <typename R>
struct Amp;
template <>
struct Amp<float> {
  using T = float2;
  using V = float4;  // two amplitudes per 16-byte load
};
template <>
struct Amp<double> {
  using T = double2;
  using V = double2;
};

// |a|^2 of the amplitudes in one 16-byte vector, every product in FP64 (the
// reduction is bandwidth-bound, so widening first costs nothing measurable).
__device__ __forceinline__ double sq16(const float4 v) {
  const double x = v.x, y = v.y, z = v.z, w = v.w;
  return (x * x + y * y) + (z * z + w * w);
}
__device__ __forceinline__ double sq16(const double2 v) { return v.x * v.x + v.y * v.y; }

// Block b writes its sums to scratch[2b], scratch[2b+1]. Every pair that the
// final pass reads was written by the same launch sequence, so nothing in the
// array has to start at zero.
template <typename R>
__global__ void __launch_bounds__(kNoAllocThreads)
    norms_partial_noalloc(const typename Amp<R>::T* __restrict__ st, uint64_t N,
                          const __grid_constant__ Patterns pat, int npat, int lowk, uint64_t lowv,
                          double* __restrict__ scratch) {
  using V = typename Amp<R>::V;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const V* vp = reinterpret_cast<const V*>(st);
  const uint64_t nv = N * sizeof(typename Amp<R>::T) / sizeof(V);
  double tot = 0.0, sel = 0.0;
  for (uint64_t i = tid; i < nv; i += stride) tot += sq16(__ldcs(vp + i));
  const uint64_t ncand = N >> lowk;
  for (uint64_t j = tid; j < ncand; j += stride) {
    const uint64_t i = lowv | (j << lowk);
    bool hit = false;
    for (int k = 0; k < npat; ++k) hit |= ((i & pat.m[k]) == pat.v[k]);
    if (hit) {
      const auto a = st[i];
      sel += (double)a.x * (double)a.x + (double)a.y * (double)a.y;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    sel += __shfl_xor_sync(0xffffffffu, sel, o);
  }
  __shared__ double sh[2][kNoAllocThreads / 32];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[0][w] = tot;
    sh[1][w] = sel;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < kNoAllocThreads / 32; ++k) {
      a += sh[0][k];
      b += sh[1][k];
    }
    scratch[2 * blockIdx.x] = a;
    scratch[2 * blockIdx.x + 1] = b;
  }
}

// Sums the first nblocks pairs in block order (deterministic).
__global__ void norms_final_noalloc(const double* __restrict__ scratch, int nblocks,
                                    double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nblocks; ++k) {
      a += scratch[2 * k];
      b += scratch[2 * k + 1];
    }
    out[0] = a;
    out[1] = b;
  }
}

// Device address of g_norm_scratch on the current device, looked up while
// that device is current.  The lookup can load the module on that device,
// which is not allowed while a stream is being captured; hence the first
// call on each device should come before any capture.  Only a successful
// lookup is cached: after a failure (a capture in progress, say) the next
// call tries again, and the failure's non-sticky error is cleared so that it
// does not surface in the caller's next cudaGetLastError.
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu[kMaxDevices];

cudaError_t scratch_on_current_device(int dev, double** out) {
  std::lock_guard<std::mutex> lk(g_scratch_mu[dev]);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_norm_scratch);
    if (e != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();
      *out = nullptr;
      return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<double*>(g_scratch_ptr[dev]);
  return cudaSuccess;
}

}  // namespace

extern "C" csim_status csim_norms_noalloc(const void* d_state, int32_t n, csim_precision prec,
                                          const uint64_t* pm, const uint64_t* pv, int32_t npat,
                                          double* d_out, void* cuda_stream) {
  if (!d_state || !d_out) return na_fail(CSIM_ERR_ARG, "csim_norms_noalloc: null device pointer");
  if (prec != CSIM_C64 && prec != CSIM_C128)
    return na_fail(CSIM_ERR_ARG, "csim_norms_noalloc: unknown precision");
  if (n < 1) return na_fail(CSIM_ERR_ARG, "csim_norms_noalloc: n must be at least 1");
  if (n > kNoAllocMaxQubits)
    return na_fail(CSIM_ERR_TOO_LARGE, "csim_norms_noalloc: n = " + std::to_string(n) +
                                           " exceeds the maximum of " +
                                           std::to_string(kNoAllocMaxQubits) + " qubits");
  if (npat < 0 || (npat > 0 && (!pm || !pv)))
    return na_fail(CSIM_ERR_ARG, "csim_norms_noalloc: bad pattern arrays");
  if (npat > kNoAllocMaxPatterns)
    return na_fail(CSIM_ERR_TOO_LARGE, "csim_norms_noalloc: " + std::to_string(npat) +
                                           " patterns exceed the maximum of " +
                                           std::to_string(kNoAllocMaxPatterns));
  if ((reinterpret_cast<uintptr_t>(d_state) & 15) != 0)
    return na_fail(CSIM_ERR_ARG, "csim_norms_noalloc: state must be 16-byte aligned");
  if ((reinterpret_cast<uintptr_t>(d_out) & 7) != 0)
    return na_fail(CSIM_ERR_ARG, "csim_norms_noalloc: d_out must be 8-byte aligned");
  const uint64_t N = 1ull << n;
  Patterns pat{};
  for (int k = 0; k < npat; ++k) {
    if ((pv[k] & ~pm[k]) != 0 || (pm[k] >> n) != 0)
      return na_fail(CSIM_ERR_ARG, "csim_norms_noalloc: pattern value outside its mask or state");
    pat.m[k] = pm[k];
    pat.v[k] = pv[k];
  }
  // the low index bits that every pattern fixes to the same value
  int lowk = 0;
  uint64_t lowv = 0;
  while (npat > 0 && lowk < n) {
    const uint64_t b = 1ull << lowk;
    bool all = true;
    for (int k = 0; k < npat; ++k) all = all && (pm[k] & b) && ((pv[k] & b) == (pv[0] & b));
    if (!all) break;
    lowv |= pv[0] & b;
    ++lowk;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return na_fail(CSIM_ERR_CUDA, std::string("csim_norms_noalloc: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return na_fail(CSIM_ERR_ARG, "csim_norms_noalloc: device ordinal out of range");
  double* scratch = nullptr;
  e = scratch_on_current_device(dev, &scratch);
  if (e != cudaSuccess)
    return na_fail(CSIM_ERR_CUDA, std::string("csim_norms_noalloc: scratch lookup: ") +
                                      cudaGetErrorString(e));
  // one thread per 16-byte vector at most, clamped to the scratch capacity
  const uint64_t nvec = (prec == CSIM_C64) ? N / 2 : N;
  uint64_t want = (nvec + kNoAllocThreads - 1) / kNoAllocThreads;
  if (want < 1) want = 1;
  const int grid = (int)(want < (uint64_t)kNoAllocBlocks ? want : (uint64_t)kNoAllocBlocks);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (prec == CSIM_C64)
    norms_partial_noalloc<float><<<grid, kNoAllocThreads, 0, st>>>(
        static_cast<const float2*>(d_state), N, pat, npat, lowk, lowv, scratch);
  else
    norms_partial_noalloc<double><<<grid, kNoAllocThreads, 0, st>>>(
        static_cast<const double2*>(d_state), N, pat, npat, lowk, lowv, scratch);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    norms_final_noalloc<<<1, 32, 0, st>>>(scratch, grid, d_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess)
    return na_fail(CSIM_ERR_CUDA, std::string("csim_norms_noalloc: ") + cudaGetErrorString(e));
  return CSIM_OK;
}
