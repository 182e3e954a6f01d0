// CUDA kernels (sm_103a) of the state-vector path.
//
// State layout: 2^n complex amplitudes (float2 for complex64, double2 for
// complex128), index bit b = qubit b.  A "warp tile" is 128 consecutive
// amplitudes: bits 0-1 live in one thread (4 amplitudes, 32 B or 64 B),
// bits 2-6 select the lane.  In the register layout of the circuit these
// seven bits are the value-encoding target t, the QSVT signal s and the five
// U_L label qubits, i.e. every qubit that is touched by a non-permutation gate.
//
//   init_scatter_kernel  -- scatter the normalised right-hand side b (after a
//                           memset, or after the sparse init's two kernels)
//   mark_tiles_kernel    -- sparse init: the tile map of b's 128-amplitude tiles
//   zero_tiles_kernel    -- sparse init: zero those tiles (the leading sweeps
//                           write the zeros of all others)
//   zero_unmarked_kernel -- write the zeros of a sparse init whole (state read early)
//   gate_kernel          -- one elementary gate over the 2^{n-1-c} matching pairs
//   sweep_kernel         -- one fused HBM pass: gather through an index
//                           permutation (a run of multi-controlled X gates; its
//                           precomputed source index, or its lookup-table
//                           chain), then a list of ops acting inside the warp
//                           tile (in-register for bits 0-1, warp shuffles for
//                           2-6), stored contiguously or back to the gathered
//                           addresses (conjugated, in place).  Specialised on
//                           the op list (SHAPE) for the QSVT circuit's sweeps.
//   perm_index_kernel    -- the source-index table of a permutation chain
//   norm_kernel          -- FP64 sum |a|^2 (total and under a pattern mask)
//   compact_kernel       -- gather the postselected block
#include <cuda_runtime.h>

#include <cstdint>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <utility>

#include "kernels.h"

namespace csim {
namespace {

template <typename R>
struct V2;
template <>
struct V2<float> {
  using T = float2;
};
template <>
struct V2<double> {
  using T = double2;
};

template <typename T>
__device__ __forceinline__ T mk(decltype(T::x) a, decltype(T::x) b) {
  T r;
  r.x = a;
  r.y = b;
  return r;
}

// ------------------------------------------------------------------ init
template <typename R>
__global__ void init_scatter_kernel(typename V2<R>::T* state, const uint64_t* idx,
                                    const double* val, int64_t count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) state[idx[i]] = mk<typename V2<R>::T>((R)val[i], (R)0);
}

// Sparse init: mark the tile of every entry, then zero the marked tiles (one
// warp per entry; tiles shared by several entries are zeroed repeatedly).
__global__ void mark_tiles_kernel(const uint64_t* __restrict__ idx, int64_t count,
                                  uint32_t* __restrict__ map) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    const uint64_t tile = idx[i] >> 7;
    atomicOr(map + (tile >> 5), 1u << (uint32_t)(tile & 31u));
  }
}
template <typename R>
__global__ void zero_tiles_kernel(typename V2<R>::T* __restrict__ state,
                                  const uint64_t* __restrict__ idx, int64_t count) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31u;
  if (w < count) {
    typename V2<R>::T* t = state + ((idx[w] >> 7) << 7);
#pragma unroll
    for (int j = 0; j < 4; ++j) t[(lane << 2) + j] = mk<typename V2<R>::T>((R)0, (R)0);
  }
}

// Zero every tile whose bit is clear in map (grid-stride, one warp per tile).
template <typename R>
__global__ void zero_unmarked_kernel(typename V2<R>::T* __restrict__ state,
                                     const uint32_t* __restrict__ map, uint32_t ntiles) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ntiles; w += nwarps) {
    if ((__ldg(map + (w >> 5)) >> (w & 31u)) & 1u) continue;
    typename V2<R>::T* t = state + ((size_t)w << 7);
#pragma unroll
    for (int j = 0; j < 4; ++j) t[(j << 5) + lane] = mk<typename V2<R>::T>((R)0, (R)0);
  }
}

// ------------------------------------------------------- gate-by-gate path
struct GateParams {
  uint64_t cmask, cval, tbit;
  uint64_t npairs;
  int nfixed;
  uint8_t fixed[64];  // sorted bit positions of controls + target
  int op;
  double c, s;        // RY: cos(th/2), sin(th/2); ZPHASE: cos(phi), sin(phi)
};

template <typename R>
__global__ void gate_kernel(typename V2<R>::T* __restrict__ st, GateParams p) {
  using T = typename V2<R>::T;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const R c = (R)p.c, s = (R)p.s;
  const R h = (R)0.70710678118654752440;
  for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < p.npairs; f += stride) {
    uint64_t idx = f;
    for (int k = 0; k < p.nfixed; ++k) {
      const int b = p.fixed[k];
      idx = ((idx >> b) << (b + 1)) | (idx & ((1ull << b) - 1));
    }
    const uint64_t i0 = idx | p.cval, i1 = i0 | p.tbit;
    const T a = st[i0], bb = st[i1];
    T na, nb;
    switch (p.op) {
      case 0:  // X
        na = bb;
        nb = a;
        break;
      case 1:  // H
        na = mk<T>((a.x + bb.x) * h, (a.y + bb.y) * h);
        nb = mk<T>((a.x - bb.x) * h, (a.y - bb.y) * h);
        break;
      case 2:  // RY
        na = mk<T>(c * a.x - s * bb.x, c * a.y - s * bb.y);
        nb = mk<T>(s * a.x + c * bb.x, s * a.y + c * bb.y);
        break;
      default:  // ZPHASE: diag(e^{i phi}, e^{-i phi})
        na = mk<T>(a.x * c - a.y * s, a.x * s + a.y * c);
        nb = mk<T>(bb.x * c + bb.y * s, -bb.x * s + bb.y * c);
        break;
    }
    st[i0] = na;
    st[i1] = nb;
  }
}

// ------------------------------------------------------------ fused sweep
template <typename T>
__device__ __forceinline__ T shfl_xor_c(T v, int lanemask);
template <>
__device__ __forceinline__ float2 shfl_xor_c(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
template <>
__device__ __forceinline__ double2 shfl_xor_c(double2 v, int m) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// Sums of the four complex values x[0..3] over all 32 lanes, returned in
// every lane: a reduce-scatter (each level halves the values a lane carries)
// followed by an all-gather, 16 shuffles instead of the 40 of four separate
// butterflies.
// Sums over all 32 lanes of two complex values (xa, xb): the same reduce-scatter
// then all-gather as lane_sum4 on four reals, 9 shuffles instead of the 20 of
// two separate butterflies.
template <typename T, typename R>
__device__ __forceinline__ void lane_sum2(const T xa, const T xb, T& Sa, T& Sb, uint32_t lane) {
  const unsigned full = 0xffffffffu;
  const R a[4] = {xa.x, xa.y, xb.x, xb.y};
  const bool h4 = (lane & 16u) != 0, h3 = (lane & 8u) != 0;
  R k[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {  // keep values (2 h4 + i)
    const R send = h4 ? a[i] : a[i + 2];
    k[i] = (h4 ? a[i + 2] : a[i]) + __shfl_xor_sync(full, send, 16);
  }
  R r = (h3 ? k[1] : k[0]) + __shfl_xor_sync(full, h3 ? k[0] : k[1], 8);
  r += __shfl_xor_sync(full, r, 4);
  r += __shfl_xor_sync(full, r, 2);
  r += __shfl_xor_sync(full, r, 1);  // total of value 2 h4 + h3
  const R p = __shfl_xor_sync(full, r, 8);
  const R q0 = h3 ? p : r, q1 = h3 ? r : p;  // values 2 h4 + {0, 1}
  const R z0 = __shfl_xor_sync(full, q0, 16), z1 = __shfl_xor_sync(full, q1, 16);
  Sa.x = h4 ? z0 : q0;
  Sa.y = h4 ? z1 : q1;
  Sb.x = h4 ? q0 : z0;
  Sb.y = h4 ? q1 : z1;
}

template <typename T, typename R>
__device__ __forceinline__ void lane_sum4(const T (&x)[4], T (&S)[4], uint32_t lane) {
  const unsigned full = 0xffffffffu;
  R a[8] = {x[0].x, x[0].y, x[1].x, x[1].y, x[2].x, x[2].y, x[3].x, x[3].y};
  const bool h4 = (lane & 16u) != 0, h3 = (lane & 8u) != 0, h2 = (lane & 4u) != 0;
  R k[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {  // keep values (4 h4 + i)
    const R send = h4 ? a[i] : a[i + 4];
    k[i] = (h4 ? a[i + 4] : a[i]) + __shfl_xor_sync(full, send, 16);
  }
  R m[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {  // keep (4 h4 + 2 h3 + i)
    const R send = h3 ? k[i] : k[i + 2];
    m[i] = (h3 ? k[i + 2] : k[i]) + __shfl_xor_sync(full, send, 8);
  }
  R r = (h2 ? m[1] : m[0]) + __shfl_xor_sync(full, h2 ? m[0] : m[1], 4);
  r += __shfl_xor_sync(full, r, 2);
  r += __shfl_xor_sync(full, r, 1);  // total of value 4 h4 + 2 h3 + h2
  const R p = __shfl_xor_sync(full, r, 4);
  const R q0 = h2 ? p : r, q1 = h2 ? r : p;  // values 4 h4 + 2 h3 + {0, 1}
  const R u0 = __shfl_xor_sync(full, q0, 8), u1 = __shfl_xor_sync(full, q1, 8);
  R w[4];  // values 4 h4 + {0..3}
  w[0] = h3 ? u0 : q0;
  w[1] = h3 ? u1 : q1;
  w[2] = h3 ? q0 : u0;
  w[3] = h3 ? q1 : u1;
  R z[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) z[i] = __shfl_xor_sync(full, w[i], 16);
  R t[8];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    t[i] = h4 ? z[i] : w[i];
    t[i + 4] = h4 ? w[i] : z[i];
  }
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    S[y].x = t[2 * y];
    S[y].y = t[2 * y + 1];
  }
}

template <typename R>
__device__ __forceinline__ void apply_pair(typename V2<R>::T& a, typename V2<R>::T& b, int op,
                                           R c, R s) {
  using T = typename V2<R>::T;
  const R h = (R)0.70710678118654752440;
  T na, nb;
  switch (op) {
    case 0:
      na = b;
      nb = a;
      break;
    case 1:
      na = mk<T>((a.x + b.x) * h, (a.y + b.y) * h);
      nb = mk<T>((a.x - b.x) * h, (a.y - b.y) * h);
      break;
    case 2:
      na = mk<T>(c * a.x - s * b.x, c * a.y - s * b.y);
      nb = mk<T>(s * a.x + c * b.x, s * a.y + c * b.y);
      break;
    default:
      na = mk<T>(a.x * c - a.y * s, a.x * s + a.y * c);
      nb = mk<T>(b.x * c + b.y * s, -b.x * s + b.y * c);
      break;
  }
  a = na;
  b = nb;
}

template <typename R>
struct Coef;
template <>
struct Coef<float> {
  template <typename O>
  static __device__ __forceinline__ float c(const O& o) { return o.cf; }
  template <typename O>
  static __device__ __forceinline__ float s(const O& o) { return o.sf; }
};
template <>
struct Coef<double> {
  template <typename O>
  static __device__ __forceinline__ double c(const O& o) { return o.cd; }
  template <typename O>
  static __device__ __forceinline__ double s(const O& o) { return o.sd; }
};

// key = x[lo0, lo0+w0) | x[lo1, lo1+w1) << w0
__device__ __forceinline__ uint32_t win_key(uint32_t x, KeyWin w) {
  const uint32_t k0 = (x >> w.lo0) & ((1u << w.w0) - 1u);
  const uint32_t k1 = (x >> w.lo1) & ((1u << w.w1) - 1u);
  return k0 | (k1 << w.w0);
}

// the inverse placement: x with its window bits replaced by the key v
__device__ __forceinline__ uint32_t win_put(uint32_t x, uint32_t v, KeyWin w) {
  const uint32_t m0 = (1u << w.w0) - 1u, m1 = (1u << w.w1) - 1u;
  x &= ~((m0 << w.lo0) | (m1 << w.lo1));
  return x | ((v & m0) << w.lo0) | (((v >> w.w0) & m1) << w.lo1);
}

// RY(c, s) on the in-thread pair (a, b) = (bit 0, bit 1) of the target qubit.
template <typename T, typename R>
__device__ __forceinline__ void rot(T& a, T& b, R c, R s) {
  const T na = mk<T>(c * a.x - s * b.x, c * a.y - s * b.y);
  b = mk<T>(s * a.x + c * b.x, s * a.y + c * b.y);
  a = na;
}

// A chunk is 32 bytes (complex64) or 64 bytes (complex128), 32-byte aligned
// (launch_sweep checks the buffers), and moves with 256-bit accesses: one
// L2 sector request per 32 bytes.
__device__ __forceinline__ void load_chunk(const float2* base, float2 (&v)[4]) {
  asm volatile("ld.global.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[1].x), "=f"(v[1].y), "=f"(v[2].x),
                 "=f"(v[2].y), "=f"(v[3].x), "=f"(v[3].y)
               : "l"(base));
}
__device__ __forceinline__ void load_chunk(const double2* base, double2 (&v)[4]) {
#pragma unroll
  for (int h = 0; h < 2; ++h)
    asm volatile("ld.global.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(v[2 * h].x), "=d"(v[2 * h].y), "=d"(v[2 * h + 1].x), "=d"(v[2 * h + 1].y)
                 : "l"(base + 2 * h));
}
// Complex64 chunk stores carry an L2 evict-first policy: a sweep's output is
// read again only by the next sweep, after the whole state has streamed
// through L2.  Measured on the 32-qubit precision circuit: 166.6 against
// 171.4 ms per step (evict-last gave the same 166.2 ms).
__device__ __forceinline__ void store_chunk(float2* base, const float2 (&v)[4]) {
  asm volatile(
      "{\n\t.reg .b64 pol;\n\t"
      "createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
      "st.global.L2::cache_hint.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8}, pol;\n\t}" ::"l"(base),
      "f"(v[0].x), "f"(v[0].y), "f"(v[1].x), "f"(v[1].y), "f"(v[2].x), "f"(v[2].y), "f"(v[3].x),
      "f"(v[3].y)
      : "memory");
}
__device__ __forceinline__ void store_chunk(double2* base, const double2 (&v)[4]) {
#pragma unroll
  for (int h = 0; h < 2; ++h)
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(base + 2 * h), "d"(v[2 * h].x),
                 "d"(v[2 * h].y), "d"(v[2 * h + 1].x), "d"(v[2 * h + 1].y)
                 : "memory");
}

// RY(c, s) on both in-thread pairs of target bit mt whose other low bit
// satisfies the controls (mlm, mlv).
template <typename T, typename R>
__device__ __forceinline__ void rot_pairs(T (&w)[4], uint32_t mt, uint32_t mlm, uint32_t mlv, R c,
                                          R s) {
  if (mt == 0) {
    if ((0u & mlm) == mlv) rot<T, R>(w[0], w[1], c, s);
    if ((2u & mlm) == mlv) rot<T, R>(w[2], w[3], c, s);
  } else {
    if ((0u & mlm) == mlv) rot<T, R>(w[0], w[2], c, s);
    if ((1u & mlm) == mlv) rot<T, R>(w[1], w[3], c, s);
  }
}

template <typename R>
struct CplxOf;
template <>
struct CplxOf<float> {
  static __device__ __forceinline__ float2 a(const ReflectDesc& d, int k) { return d.af[k]; }
  static __device__ __forceinline__ float2 b(const ReflectDesc& d, int k) { return d.bf[k]; }
  static __device__ __forceinline__ float2 angle(const SweepParams& p, uint32_t i) {
    return __ldg(p.angf + i);
  }
  static __device__ __forceinline__ void entry(const SweepParams& p, uint32_t e, uint32_t* cm,
                                               uint32_t* cv, float* c, float* s) {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(p.mentf) + e);
    *cm = w.x;
    *cv = w.y;
    *c = __uint_as_float(w.z);
    *s = __uint_as_float(w.w);
  }
};
template <>
struct CplxOf<double> {
  static __device__ __forceinline__ double2 a(const ReflectDesc& d, int k) { return d.ad[k]; }
  static __device__ __forceinline__ double2 b(const ReflectDesc& d, int k) { return d.bd[k]; }
  static __device__ __forceinline__ double2 angle(const SweepParams& p, uint32_t i) {
    return __ldg(p.angd + i);
  }
  static __device__ __forceinline__ void entry(const SweepParams& p, uint32_t e, uint32_t* cm,
                                               uint32_t* cv, double* c, double* s) {
    const MuxEntryD& E = p.mentd[e];
    *cm = E.cm;
    *cv = E.cv;
    *c = E.c;
    *s = E.s;
  }
};

// Bucket words of the first kPrefetchMux multiplexers are loaded early.
constexpr int kPrefetchMux = 2;

// Averaging block: I (x) A + J (x) B over the lane bits of rd.lanemask.
template <typename R, int U>
__device__ __forceinline__ void op_refl(const ReflectDesc& rd, typename V2<R>::T (&v)[U][4],
                                        uint32_t lane) {
  using T = typename V2<R>::T;
  const uint32_t lmask = rd.lanemask, nzA = rd.nzA, nzB = rd.nzB;
  if (((nzA | nzB) & ~0x8421u) == 0) {  // A and B diagonal
    if (lmask == 31u && __popc(nzB) == 2) {  // every lane, two y's: one joint reduction
      const int ya = (__ffs(nzB) - 1) / 5, yb = (31 - __clz(nzB)) / 5;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        T xa = v[u][0], xb = v[u][0];
#pragma unroll
        for (int y = 1; y < 4; ++y) {
          if (y == ya) xa = v[u][y];
          if (y == yb) xb = v[u][y];
        }
        T Sa, Sb;
        lane_sum2<T, R>(xa, xb, Sa, Sb, lane);
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const int q = y * 5;
          const T ca = CplxOf<R>::a(rd, q);
          const T x = v[u][y];
          T o = mk<T>(ca.x * x.x - ca.y * x.y, ca.x * x.y + ca.y * x.x);
          if (y == ya || y == yb) {
            const T cb = CplxOf<R>::b(rd, q);
            const T S = (y == ya) ? Sa : Sb;
            if (cb.x == (R)0) {  // purely imaginary (the QSVT projector phase)
              o.x -= cb.y * S.y;
              o.y += cb.y * S.x;
            } else {
              o.x += cb.x * S.x - cb.y * S.y;
              o.y += cb.x * S.y + cb.y * S.x;
            }
          }
          v[u][y] = o;
        }
      }
      return;
    }
    if (lmask == 31u && nzB == 0x8421u) {  // every lane and every y: one joint reduction
#pragma unroll
      for (int u = 0; u < U; ++u) {
        T S[4];
        lane_sum4<T, R>(v[u], S, lane);
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const int q = y * 5;
          const T ca = CplxOf<R>::a(rd, q), cb = CplxOf<R>::b(rd, q);
          const T x = v[u][y];
          v[u][y] = mk<T>(ca.x * x.x - ca.y * x.y + cb.x * S[y].x - cb.y * S[y].y,
                          ca.x * x.y + ca.y * x.x + cb.x * S[y].y + cb.y * S[y].x);
        }
      }
      return;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int q = y * 5;
        T S = v[u][y];
        if ((nzB >> q) & 1u) {
#pragma unroll
          for (int b = 0; b < 5; ++b) {
            if (!((lmask >> b) & 1u)) continue;
            const T w = shfl_xor_c(S, 1 << b);
            S.x += w.x;
            S.y += w.y;
          }
        }
        const T ca = CplxOf<R>::a(rd, q), cb = CplxOf<R>::b(rd, q);
        const T x = v[u][y];
        T o = mk<T>(ca.x * x.x - ca.y * x.y, ca.x * x.y + ca.y * x.x);
        if ((nzB >> q) & 1u) {
          o.x += cb.x * S.x - cb.y * S.y;
          o.y += cb.x * S.y + cb.y * S.x;
        }
        v[u][y] = o;
      }
    }
    return;
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    T S[4];
#pragma unroll
    for (int y = 0; y < 4; ++y) S[y] = v[u][y];
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      if (!((lmask >> b) & 1u)) continue;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const T w = shfl_xor_c(S[y], 1 << b);
        S[y].x += w.x;
        S[y].y += w.y;
      }
    }
    T o4[4];
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      o4[y] = mk<T>((R)0, (R)0);
#pragma unroll
      for (int yp = 0; yp < 4; ++yp) {
        const int q = y * 4 + yp;
        if ((nzA >> q) & 1u) {
          const T c = CplxOf<R>::a(rd, q);
          o4[y].x += c.x * v[u][yp].x - c.y * v[u][yp].y;
          o4[y].y += c.x * v[u][yp].y + c.y * v[u][yp].x;
        }
        if ((nzB >> q) & 1u) {
          const T c = CplxOf<R>::b(rd, q);
          o4[y].x += c.x * S[yp].x - c.y * S[yp].y;
          o4[y].y += c.x * S[yp].y + c.y * S[yp].x;
        }
      }
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) v[u][y] = o4[y];
  }
  return;
}

// Multiplexed RY (descriptor md, prefetched bucket words in wd when slot < 2):
// compose the rotation each chunk gets, apply it, and keep it in (mc, ms).
template <typename R, int U>
__device__ __forceinline__ void op_mux(const SweepParams& a, const MuxDesc& md, uint32_t slot,
                                       typename V2<R>::T (&v)[U][4], const uint32_t (&ci)[U],
                                       const uint32_t (&wd)[kPrefetchMux][U], R (&mc)[U],
                                       R (&ms)[U]) {
  using T = typename V2<R>::T;
  const KeyWin w = md.win;
  const uint32_t toff = md.tab_off, mt = md.target, mlm = md.lm, mlv = md.lv;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    uint32_t word;
    if (slot == 0) word = wd[0][u];
    else if (slot == 1 && kPrefetchMux > 1) word = wd[1][u];
    else word = __ldg(a.mtab + toff + win_key(ci[u], w));
    R c = (R)1, s = (R)0;
    if (word & 0x80000000u) {
      const T cs = CplxOf<R>::angle(a, word & 0x7fffffffu);
      c = cs.x;
      s = cs.y;
    } else if (word != 0u) {
      // the matching candidates' rotations commute: compose them, rotate once
      const uint32_t e0 = word >> 8, e1 = e0 + (word & 255u);
      for (uint32_t e = e0; e < e1; ++e) {
        uint32_t cm, cv;
        R ce, se;
        CplxOf<R>::entry(a, e, &cm, &cv, &ce, &se);
        if ((ci[u] & cm) == cv) {
          const R nc = c * ce - s * se;
          s = s * ce + c * se;
          c = nc;
        }
      }
    }
    mc[u] = c;
    ms[u] = s;
    if (word != 0u) rot_pairs<T, R>(v[u], mt, mlm, mlv, c, s);
  }
}

// The inverse of the latest multiplexer: the kept rotation with the sine negated.
template <typename R, int U>
__device__ __forceinline__ void op_mux_inverse(uint32_t tg, uint32_t lm, uint32_t lv,
                                               typename V2<R>::T (&v)[U][4], const R (&mc)[U],
                                               const R (&ms)[U]) {
  using T = typename V2<R>::T;
#pragma unroll
  for (int u = 0; u < U; ++u)
    if (ms[u] != (R)0 || mc[u] != (R)1) rot_pairs<T, R>(v[u], tg, lm, lv, mc[u], -ms[u]);
}

// Bucket words of the first multiplexers of the sweep: they depend only on
// the destination index, so they are loaded before the permutation chain.
template <int U>
__device__ __forceinline__ void prefetch_mux(const SweepParams& a, const uint32_t (&ci)[U],
                                             uint32_t (&wd)[kPrefetchMux][U]) {
#pragma unroll
  for (int m = 0; m < kPrefetchMux; ++m) {
    if (m >= a.nmux) break;
    const MuxDesc& md = a.mux[m];
#pragma unroll
    for (int u = 0; u < U; ++u) wd[m][u] = __ldg(a.mtab + md.tab_off + win_key(ci[u], md.win));
  }
}

// A gate of op code 0-3 (X, H, RY, ZPHASE) on an in-thread bit (target 0-1)
// or a lane bit (target 2-6), op 6 (ZPHASE above the tile) or op 8 (lane
// Walsh-Hadamard), with the descriptor o.  The op code is a parameter so that
// the shaped sweeps, which pass a constant, compile one path.
template <typename R, int U, bool WHT = true>
__device__ __forceinline__ void op_tile_gate(uint32_t op, const LocalOp& o,
                                             typename V2<R>::T (&v)[U][4], const uint32_t (&ci)[U],
                                             uint32_t lane) {
  using T = typename V2<R>::T;
  const uint32_t ocm = o.cm, ocv = o.cv, lm = o.lm, lv = o.lv, tg = o.target;
  if (WHT && op == 8) {  // H on each lane bit of the mask: butterflies, then one scale
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      if (!((ocm >> b) & 1u)) continue;
      const R sg = ((lane >> b) & 1u) ? (R)-1 : (R)1;
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const T w = shfl_xor_c(v[u][j], 1 << b);
          v[u][j] = mk<T>(fma(v[u][j].x, sg, w.x), fma(v[u][j].y, sg, w.y));
        }
    }
    const R sc = Coef<R>::c(o);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < 4; ++j) v[u][j] = mk<T>(v[u][j].x * sc, v[u][j].y * sc);
    return;
  }
  const R c = Coef<R>::c(o), s = Coef<R>::s(o);
  if (op == 6) {  // e^{i phi Z} on chunk-index bit tg (a qubit above the tile)
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if ((ci[u] & ocm) != ocv) continue;
      const R sg = ((ci[u] >> tg) & 1u) ? -s : s;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (((uint32_t)j & lm) == lv)
          v[u][j] = mk<T>(v[u][j].x * c - v[u][j].y * sg, v[u][j].x * sg + v[u][j].y * c);
    }
    return;
  }
  if (tg < 2) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if ((ci[u] & ocm) != ocv) continue;
      if (tg == 0) {
        if ((0u & lm) == lv) apply_pair<R>(v[u][0], v[u][1], op, c, s);
        if ((2u & lm) == lv) apply_pair<R>(v[u][2], v[u][3], op, c, s);
      } else {
        if ((0u & lm) == lv) apply_pair<R>(v[u][0], v[u][2], op, c, s);
        if ((1u & lm) == lv) apply_pair<R>(v[u][1], v[u][3], op, c, s);
      }
    }
    return;
  }
  const int lmask = 1 << (tg - 2);
  const bool hi = (lane & (uint32_t)lmask) != 0;
  const R h = (R)0.70710678118654752440;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const bool cok = (ci[u] & ocm) == ocv;
    if (op == 3) {  // diagonal: no partner needed
      if (!cok) continue;
      const R sg = hi ? -s : s;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (((uint32_t)j & lm) == lv)
          v[u][j] = mk<T>(v[u][j].x * c - v[u][j].y * sg, v[u][j].x * sg + v[u][j].y * c);
      continue;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T w = shfl_xor_c(v[u][j], lmask);
      if (!cok || (((uint32_t)j & lm) != lv)) continue;
      if (op == 0) {
        v[u][j] = w;
      } else if (op == 1) {
        v[u][j] = hi ? mk<T>((w.x - v[u][j].x) * h, (w.y - v[u][j].y) * h)
                     : mk<T>((v[u][j].x + w.x) * h, (v[u][j].y + w.y) * h);
      } else {
        v[u][j] = hi ? mk<T>(s * w.x + c * v[u][j].x, s * w.y + c * v[u][j].y)
                     : mk<T>(c * v[u][j].x - s * w.x, c * v[u][j].y - s * w.y);
      }
    }
  }
}

// X / H / RY (kind 0 / 1 / 2) on staged qubit J: the warp's tiles u and
// u | (1 << J) hold the amplitudes with that qubit 0 and 1 at the same lane
// and in-thread position, so the gate pairs their registers.  Controls come
// from the chunk index of the tile with the qubit clear (a control never
// includes the target) and from the in-thread bits.
template <typename R, int U, int J, int KIND>
__device__ __forceinline__ void stage_pairs(const LocalOp& o, typename V2<R>::T (&v)[U][4],
                                            const uint32_t (&ci)[U]) {
  const R c = Coef<R>::c(o), s = Coef<R>::s(o);
  const uint32_t ocm = o.cm, ocv = o.cv, lm = o.lm, lv = o.lv;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (u & (1 << J)) continue;
    if ((ci[u] & ocm) != ocv) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (((uint32_t)j & lm) == lv) apply_pair<R>(v[u][j], v[u | (1 << J)][j], KIND, c, s);
  }
}

// The gate kind is dispatched once per op, outside the tile loops.
template <typename R, int U, int J>
__device__ __forceinline__ void stage_kind(uint32_t kind, const LocalOp& o,
                                           typename V2<R>::T (&v)[U][4], const uint32_t (&ci)[U]) {
  if (kind == 2) return stage_pairs<R, U, J, 2>(o, v, ci);
  if (kind == 1) return stage_pairs<R, U, J, 1>(o, v, ci);
  stage_pairs<R, U, J, 0>(o, v, ci);
}

template <typename R, int U>
__device__ __forceinline__ void op_stage_gate(uint32_t kind, const LocalOp& o,
                                              typename V2<R>::T (&v)[U][4],
                                              const uint32_t (&ci)[U]) {
  const uint32_t j = o.target;
  if constexpr (U >= 2)
    if (j == 0) return stage_kind<R, U, 0>(kind, o, v, ci);
  if constexpr (U >= 4)
    if (j == 1) return stage_kind<R, U, 1>(kind, o, v, ci);
  if constexpr (U >= 8)
    if (j == 2) return stage_kind<R, U, 2>(kind, o, v, ci);
}

// Apply the tile-local ops of one sweep to U tiles held by the warp.
// Gates only (ops 0-3, 6 and the staged-qubit ops 9-11): the interpreter of
// gate streams, without the multiplexer, averaging-block and Walsh-Hadamard
// code and its registers (the kernels that stage 2^k tiles per warp).
template <typename R, int U>
__device__ __forceinline__ void apply_gates(const SweepParams& a, typename V2<R>::T (&v)[U][4],
                                            const uint32_t (&ci)[U], uint32_t lane) {
  for (int k = 0; k < a.nops; ++k) {
    const LocalOp& o = a.ops[k];
    // one specialised body per op code (the code is a constant inside each case)
    switch (o.op) {
      case 0: op_tile_gate<R, U, false>(0, o, v, ci, lane); break;
      case 1: op_tile_gate<R, U, false>(1, o, v, ci, lane); break;
      case 2: op_tile_gate<R, U, false>(2, o, v, ci, lane); break;
      case 3: op_tile_gate<R, U, false>(3, o, v, ci, lane); break;
      case 6: op_tile_gate<R, U, false>(6, o, v, ci, lane); break;
      default: op_stage_gate<R, U>((uint32_t)o.op - 9u, o, v, ci); break;
    }
  }
}

template <typename R, int U>
__device__ __forceinline__ void apply_ops(const SweepParams& a, typename V2<R>::T (&v)[U][4],
                                          const uint32_t (&ci)[U], uint32_t lane,
                                          const uint32_t (&wd)[kPrefetchMux][U]) {
  // rotation (cos, sin of half the summed angle) of the latest multiplexer, per tile
  R mc[U], ms[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    mc[u] = (R)1;
    ms[u] = (R)0;
  }
  for (int k = 0; k < a.nops; ++k) {
    const LocalOp& o = a.ops[k];
    const uint32_t ocm = o.cm, lm = o.lm, lv = o.lv, op = o.op, tg = o.target;
    if (op == 4) {  // multiplexed RY on bit tg (0 or 1)
      op_mux<R, U>(a, a.mux[ocm], ocm, v, ci, wd, mc, ms);
      continue;
    }
    if (op == 7) {  // inverse of the latest multiplexer: RY(-theta) with the same controls
      op_mux_inverse<R, U>(tg, lm, lv, v, mc, ms);
      continue;
    }
    if (op == 5) {  // I (x) A + J (x) B over the lane bits of lanemask
      op_refl<R, U>(a.refl[ocm], v, lane);
      continue;
    }
    if (op >= 9) {  // a gate on a staged qubit
      op_stage_gate<R, U>(op - 9, o, v, ci);
      continue;
    }
    op_tile_gate<R, U>(op, o, v, ci, lane);
  }
}

// Sweep shapes with a kernel of their own: the op list is fixed at compile
// time, so the descriptors sit at fixed parameter offsets and no op list is
// interpreted.  Shape 0 is any op list (apply_ops).  The op codes are those of
// LocalOp::op; the k-th multiplexer (averaging block) of a list uses mux[k]
// (refl[k]), as the fuser assigns them.
struct ShapeAvg {  // 1: one averaging block (the conjugated sweeps)
  static constexpr int n = 1;
  static constexpr int op[1] = {5};
};
struct ShapeMux {  // 2: multiplexer, averaging block, inverse multiplexer
  static constexpr int n = 3;
  static constexpr int op[3] = {4, 5, 7};
};
struct ShapeFirst {  // 3: the first QSVT sweep: H, X, ZPHASE, X, X in-thread, W-H, multiplexer
  static constexpr int n = 7;
  static constexpr int op[7] = {1, 0, 3, 0, 0, 8, 4};
};
struct ShapeLast {  // 4: the last sweep: W-H, X, ZPHASE, X, H
  static constexpr int n = 5;
  static constexpr int op[5] = {8, 0, 3, 0, 1};
};

template <typename S>
__host__ __device__ constexpr int count_before(int i, int code) {
  int c = 0;
  for (int j = 0; j < i; ++j) c += S::op[j] == code ? 1 : 0;
  return c;
}

template <typename R, int U, typename S, int I>
__device__ __forceinline__ void shaped_step(const SweepParams& a, typename V2<R>::T (&v)[U][4],
                                            const uint32_t (&ci)[U], uint32_t lane,
                                            const uint32_t (&wd)[kPrefetchMux][U], R (&mc)[U],
                                            R (&ms)[U]) {
  constexpr int code = S::op[I];
  if constexpr (code == 4) {
    constexpr int m = count_before<S>(I, 4);
    op_mux<R, U>(a, a.mux[m], (uint32_t)m, v, ci, wd, mc, ms);
  } else if constexpr (code == 5) {
    constexpr int r = count_before<S>(I, 5);
    op_refl<R, U>(a.refl[r], v, lane);
  } else if constexpr (code == 7) {
    op_mux_inverse<R, U>(a.ops[I].target, a.ops[I].lm, a.ops[I].lv, v, mc, ms);
  } else {
    op_tile_gate<R, U>((uint32_t)code, a.ops[I], v, ci, lane);
  }
}

template <typename R, int U, typename S, int... I>
__device__ __forceinline__ void apply_seq(std::integer_sequence<int, I...>, const SweepParams& a,
                                          typename V2<R>::T (&v)[U][4], const uint32_t (&ci)[U],
                                          uint32_t lane, const uint32_t (&wd)[kPrefetchMux][U]) {
  R mc[U], ms[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    mc[u] = (R)1;
    ms[u] = (R)0;
  }
  (shaped_step<R, U, S, I>(a, v, ci, lane, wd, mc, ms), ...);
}

template <typename R, int U, int SHAPE>
__device__ __forceinline__ void apply_shaped(const SweepParams& a, typename V2<R>::T (&v)[U][4],
                                             const uint32_t (&ci)[U], uint32_t lane,
                                             const uint32_t (&wd)[kPrefetchMux][U]) {
  if constexpr (SHAPE == 1) {
    apply_seq<R, U, ShapeAvg>(std::make_integer_sequence<int, ShapeAvg::n>{}, a, v, ci, lane, wd);
  } else if constexpr (SHAPE == 2) {
    apply_seq<R, U, ShapeMux>(std::make_integer_sequence<int, ShapeMux::n>{}, a, v, ci, lane, wd);
  } else if constexpr (SHAPE == 3) {
    apply_seq<R, U, ShapeFirst>(std::make_integer_sequence<int, ShapeFirst::n>{}, a, v, ci, lane,
                                wd);
  } else if constexpr (SHAPE == 4) {
    apply_seq<R, U, ShapeLast>(std::make_integer_sequence<int, ShapeLast::n>{}, a, v, ci, lane, wd);
  } else if constexpr (SHAPE == 5) {
    apply_gates<R, U>(a, v, ci, lane);
  } else {
    apply_ops<R, U>(a, v, ci, lane, wd);
  }
}

// Map chunk indices through the permutation segments of a sweep.
template <int U>
__device__ __forceinline__ void permute(const SweepParams& a, uint32_t (&x)[U]) {
  for (int k = 0; k < a.nseg; ++k) {
    const PermSeg& g = a.segs[k];
    const uint32_t kind = g.kind, m = g.m, v = g.v, t = g.t;
    if (kind == 0) {
      const KeyWin w = g.win;
      const uint16_t* lut = a.lut + t;
#pragma unroll
      for (int u = 0; u < U; ++u) x[u] = win_put(x[u], __ldg(lut + win_key(x[u], w)), w);
    } else if (kind == 1) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if ((x[u] & m) == v) x[u] ^= t;
    } else {
      const uint32_t base = g.base, rm = (1u << g.width) - 1u, step = g.neg ? rm : 1u;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if ((x[u] & m) != v) continue;
        const uint32_t r = (((x[u] >> base) & rm) + step) & rm;
        x[u] = (x[u] & ~(rm << base)) | (r << base);
      }
    }
  }
}

// One fused sweep over U tiles per warp iteration (one 4-amplitude chunk per
// lane and tile).  Gather form: the lane computes its source chunk through the
// segments (the inverse permutation), loads it, applies the tile-local ops,
// and stores contiguously.  Scatter form: the lane loads its own chunk, applies
// the tile-local ops, and stores to the chunk's image under the permutation.
//
// Tile order: warp w takes the tile counters c = w U + u + i (nwarps U).  With
// nfe > 0 fast bits, counter bit j goes to tile bit fast[j] (j < nfe) and the
// remaining counter bits fill the other tile bits in ascending order.  The
// stride is a multiple of 2^nfe, so a warp's low counter bits never change:
// their deposit L[u] is computed once, and the high part H advances by a
// masked add of hstep (the deposit of stride >> nfe).  nfe = 0 is the natural
// order.
// |a|^2 of one chunk (four amplitudes) for a fused norm: complex64 products
// added in FP32 (as the norm kernel does) and widened once; complex128 in FP64.
__device__ __forceinline__ double chunk_norm2(const float2 (&c)[4]) {
  const float s = ((c[0].x * c[0].x + c[0].y * c[0].y) + (c[1].x * c[1].x + c[1].y * c[1].y)) +
                  ((c[2].x * c[2].x + c[2].y * c[2].y) + (c[3].x * c[3].x + c[3].y * c[3].y));
  return (double)s;
}
__device__ __forceinline__ double chunk_norm2(const double2 (&c)[4]) {
  return ((c[0].x * c[0].x + c[0].y * c[0].y) + (c[1].x * c[1].x + c[1].y * c[1].y)) +
         ((c[2].x * c[2].x + c[2].y * c[2].y) + (c[3].x * c[3].x + c[3].y * c[3].y));
}

// A block's fused-norm partial: warp sums, then the warps in order.
template <int BLK>
__device__ __forceinline__ void store_norm_partial(double acc, double* part) {
  __shared__ double sh[BLK / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31u) == 0u) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < BLK / 32; ++k) t += sh[k];
    if (blockIdx.x + 1u < kNormPartCap) part[1 + blockIdx.x] = t;
    if (blockIdx.x == 0) part[0] = (double)gridDim.x;
  }
}

template <typename R, int U, int MINB, int SHAPE, int BLK = 256>
__global__ void __launch_bounds__(BLK, MINB)
    sweep_kernel(const typename V2<R>::T* in, typename V2<R>::T* out, uint32_t ntiles, int nfe,
                 uint32_t fmask, uint32_t hstep, const __grid_constant__ SweepParams a) {
  using T = typename V2<R>::T;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t c0 = warp * U;
  uint32_t L[U];
  uint32_t H = c0;
  if (nfe > 0) {
    const uint32_t lo = c0 & ((1u << nfe) - 1u);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      uint32_t d = 0;
      for (int j = 0; j < nfe; ++j) d |= (((lo + (uint32_t)u) >> j) & 1u) << a.fast[j];
      L[u] = d;
    }
    uint32_t hv = c0 >> nfe;
    H = 0;
    for (int b = 0; hv != 0u && b < 32; ++b) {
      if ((fmask >> b) & 1u) continue;
      H |= (hv & 1u) << b;
      hv >>= 1;
    }
  } else {
#pragma unroll
    for (int u = 0; u < U; ++u) L[u] = (uint32_t)u;
  }
  if constexpr (SHAPE == 3) {
    // zero mode 2 (the next sweep reads zeros for unmarked tiles): visit the
    // marked tiles only.  Warp w takes map words w, w + nwarps, ... (b's
    // tiles fill a run of consecutive words, which this spreads over the
    // warps) and the tiles of each set bit, U aligned tiles at a time; an
    // unmarked tile of such a group is read as zeros.
    if (a.zero_map && a.zero_mode == 2) {
      const uint32_t nwords = ntiles >> 5;
      for (uint32_t wi = warp; wi < nwords; wi += nwarps) {
        const uint32_t word = __ldg(a.zero_map + wi);
        uint32_t bits = word;
        while (bits != 0u) {
          const uint32_t b0 = (uint32_t)(__ffs((int)bits) - 1) & ~(uint32_t)(U - 1);
          bits &= ~(((1u << U) - 1u) << b0);
          uint32_t ci[U];
#pragma unroll
          for (int u = 0; u < U; ++u) ci[u] = (((wi << 5) + b0 + (uint32_t)u) << 5) | lane;
          uint32_t wd[kPrefetchMux][U];
          prefetch_mux<U>(a, ci, wd);
          T v[U][4];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if ((word >> (b0 + (uint32_t)u)) & 1u) {
              load_chunk(in + ((size_t)ci[u] << 2), v[u]);
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q) v[u][q] = mk<T>((R)0, (R)0);
            }
          }
          apply_shaped<R, U, SHAPE>(a, v, ci, lane, wd);
#pragma unroll
          for (int u = 0; u < U; ++u) store_chunk(out + ((size_t)ci[u] << 2), v[u]);
        }
      }
      return;
    }
  }
  // source indices of the warp's next tiles, loaded one iteration ahead
  const bool pre = a.src != nullptr && a.src_prefetch != 0 && !a.scatter;
  uint32_t nxt[U];
  if (pre && c0 < ntiles) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      nxt[u] = __ldcs(a.src + (((nfe > 0 ? (H | L[u]) : (H + L[u])) << 5) | lane));
  }
  double nacc = 0.0;  // fused norm of the last sweep (SHAPE 4)
  for (uint32_t t0 = c0; t0 < ntiles; t0 += nwarps * U) {
    uint32_t ci[U], mv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) mv[u] = ci[u] = ((nfe > 0 ? (H | L[u]) : (H + L[u])) << 5) | lane;
    H = nfe > 0 ? (((H | fmask) + hstep) & ~fmask) : (H + nwarps * U);
    T v[U][4];
    if constexpr (SHAPE == 3) {
      // first sweep after a sparse init: the sweep maps each tile to itself
      // linearly, so tiles that b does not touch stay zero.  Mode 1 writes
      // the zeros and skips the ops; mode 2 leaves them to the next sweep
      // (warp-uniform: a tile belongs to one warp).
      if (a.zero_map) {
        bool any = false;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const uint32_t tile = ci[u] >> 5;
          any |= ((__ldg(a.zero_map + (tile >> 5)) >> (tile & 31u)) & 1u) != 0u;
        }
        if (!any) {
          if (a.zero_mode == 1) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
              for (int j = 0; j < 4; ++j) v[u][j] = mk<T>((R)0, (R)0);
              store_chunk(out + ((size_t)ci[u] << 2), v[u]);
            }
          }
          continue;
        }
      }
    }
    uint32_t wd[kPrefetchMux][U];
    if constexpr (SHAPE != 1 && SHAPE != 5) prefetch_mux<U>(a, ci, wd);
    if (!a.scatter) {
      if (pre) {
#pragma unroll
        for (int u = 0; u < U; ++u) mv[u] = nxt[u];
        if (t0 + nwarps * U < ntiles) {
#pragma unroll
          for (int u = 0; u < U; ++u)
            nxt[u] = __ldcs(a.src + (((nfe > 0 ? (H | L[u]) : (H + L[u])) << 5) | lane));
        }
      } else if (a.src) {
#pragma unroll
        for (int u = 0; u < U; ++u) mv[u] = __ldcs(a.src + ci[u]);
      } else {
        permute<U>(a, mv);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if constexpr (SHAPE == 1 || SHAPE == 3) {  // chunks of unmarked tiles read as zeros
          if (a.zero_map) {
            const uint32_t tile = mv[u] >> 5;
            if (!((__ldg(a.zero_map + (tile >> 5)) >> (tile & 31u)) & 1u)) {
#pragma unroll
              for (int j = 0; j < 4; ++j) v[u][j] = mk<T>((R)0, (R)0);
              continue;
            }
          }
        }
        load_chunk(in + ((size_t)mv[u] << 2), v[u]);
      }
      apply_shaped<R, U, SHAPE>(a, v, ci, lane, wd);
#pragma unroll
      for (int u = 0; u < U; ++u)
        store_chunk(out + ((size_t)(a.inplace ? mv[u] : ci[u]) << 2), v[u]);
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) load_chunk(in + ((size_t)ci[u] << 2), v[u]);
      apply_shaped<R, U, SHAPE>(a, v, ci, lane, wd);
      if (a.src) {
#pragma unroll
        for (int u = 0; u < U; ++u) mv[u] = __ldcs(a.src + ci[u]);
      } else {
        permute<U>(a, mv);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) store_chunk(out + ((size_t)mv[u] << 2), v[u]);
    }
    if constexpr (SHAPE == 4) {
      if (a.norm_part) {
#pragma unroll
        for (int u = 0; u < U; ++u) nacc += chunk_norm2(v[u]);
      }
    }
  }
  if constexpr (SHAPE == 4) {
    if (a.norm_part) store_norm_partial<BLK>(nacc, a.norm_part);
  }
}

// Source-index table of a gather sweep: the segment chain applied to every
// chunk index once, so that the sweeps that share the chain load one index
// per chunk instead of walking the chain.  Each thread walks four chunks at a
// time (independent lookup chains in flight) and writes them coalesced.
constexpr int kPermIndexILP = 4;
__global__ void __launch_bounds__(256)
    perm_index_kernel(uint32_t* __restrict__ src, uint64_t nchunks,
                      const __grid_constant__ SweepParams a) {
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t stride = nthreads * kPermIndexILP;
  for (uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x0 < nchunks; x0 += stride) {
    uint32_t m[kPermIndexILP];
#pragma unroll
    for (int j = 0; j < kPermIndexILP; ++j) m[j] = (uint32_t)(x0 + (uint64_t)j * nthreads);
    permute<kPermIndexILP>(a, m);
#pragma unroll
    for (int j = 0; j < kPermIndexILP; ++j) {
      const uint64_t x = x0 + (uint64_t)j * nthreads;
      if (x < nchunks) src[x] = m[j];
    }
  }
}

// --------------------------------------------------------------- reductions
// |a|^2 of one 16-byte vector of the state: two complex64 amplitudes (each
// product in FP32, matching the data's precision) or one complex128.
__device__ __forceinline__ double vec_norm2(const float4 v) {
  return (double)(v.x * v.x + v.y * v.y) + (double)(v.z * v.z + v.w * v.w);
}
__device__ __forceinline__ double vec_norm2(const double2 v) { return v.x * v.x + v.y * v.y; }

// Sum of |a|^2 over four 16-byte vectors.  Complex64: the eight non-negative
// FP32 products are added in FP32 (relative error below 8 * 2^-24, the size
// of the products' own rounding) and converted once, so the FP64 pipe, a small
// fraction of the FP32 rate on this GPU, handles one addition per eight
// amplitudes.  Complex128: FP64 throughout.
__device__ __forceinline__ double vec_norm2_4(const float4 a, const float4 b, const float4 c,
                                              const float4 d) {
  const float s = ((a.x * a.x + a.y * a.y) + (a.z * a.z + a.w * a.w)) +
                  ((b.x * b.x + b.y * b.y) + (b.z * b.z + b.w * b.w)) +
                  (((c.x * c.x + c.y * c.y) + (c.z * c.z + c.w * c.w)) +
                   ((d.x * d.x + d.y * d.y) + (d.z * d.z + d.w * d.w)));
  return (double)s;
}
__device__ __forceinline__ double vec_norm2_4(const double2 a, const double2 b, const double2 c,
                                              const double2 d) {
  return (vec_norm2(a) + vec_norm2(b)) + (vec_norm2(c) + vec_norm2(d));
}

template <typename R>
struct Vec16;
template <>
struct Vec16<float> {
  using T = float4;
};
template <>
struct Vec16<double> {
  using T = double2;
};

// FP64 sums: the total over the state (streamed as 16-byte vectors) and the
// sum over the pattern mask.  When every pattern fixes the `lowk` lowest index
// bits to `lowv`, only the indices lowv + j 2^lowk are candidates.
// TOTAL = false: the masked sum only (the total comes from a fused sweep).
template <typename R, bool TOTAL = true>
__global__ void norm_kernel(const typename V2<R>::T* __restrict__ st, uint64_t N,
                            const uint64_t* __restrict__ pm, const uint64_t* __restrict__ pv,
                            int npat, int lowk, uint64_t lowv, double* __restrict__ partial) {
  using VT = typename Vec16<R>::T;
  double tot = 0.0, sel = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (TOTAL) {
    const VT* vp = reinterpret_cast<const VT*>(st);
    const uint64_t nv = N * sizeof(typename V2<R>::T) / sizeof(VT);
    uint64_t i = tid;
    // four independent 16-byte loads in flight per thread
    for (; i + 3 * stride < nv; i += 4 * stride) {
      const VT v0 = __ldcs(vp + i), v1 = __ldcs(vp + i + stride),
               v2 = __ldcs(vp + i + 2 * stride), v3 = __ldcs(vp + i + 3 * stride);
      tot += vec_norm2_4(v0, v1, v2, v3);
    }
    for (; i < nv; i += stride) tot += vec_norm2(__ldcs(vp + i));
  }
  const uint64_t ncand = N >> lowk;
  for (uint64_t j = tid; j < ncand; j += stride) {
    const uint64_t i = lowv | (j << lowk);
    bool hit = false;
    for (int k = 0; k < npat; ++k) hit |= ((i & pm[k]) == pv[k]);
    if (hit) {
      const auto a = st[i];
      sel += (double)a.x * (double)a.x + (double)a.y * (double)a.y;
    }
  }
  __shared__ double sh[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    sel += __shfl_xor_sync(0xffffffffu, sel, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sh[0][w] = tot;
    sh[1][w] = sel;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += sh[0][k];
      b += sh[1][k];
    }
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = b;
  }
}

__global__ void reduce_partials_kernel(const double* __restrict__ partial, int nblocks,
                                       double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nblocks; ++k) {
      a += partial[2 * k];
      b += partial[2 * k + 1];
    }
    out[0] = a;
    out[1] = b;
  }
}

// The total from a fused sweep's partials (norm_part[0] = their count), the
// masked sum from the norm kernel's partials; the same order as the plain
// reduction within each.
__global__ void reduce_fused_kernel(const double* __restrict__ norm_part,
                                    const double* __restrict__ partial, int nblocks,
                                    double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int m = (int)norm_part[0];
    double a = 0.0, b = 0.0;
    for (int k = 0; k < m; ++k) a += norm_part[1 + k];
    for (int k = 0; k < nblocks; ++k) b += partial[2 * k + 1];
    out[0] = a;
    out[1] = b;
  }
}

template <typename R>
__global__ void compact_kernel(const typename V2<R>::T* __restrict__ st, double2* __restrict__ out,
                               uint64_t count, int free_shift, int free_bits, uint64_t m_first,
                               int m_shift) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t o = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; o < count; o += stride) {
    const uint64_t f = o & ((1ull << free_bits) - 1);
    const uint64_t m = m_first + (o >> free_bits);
    const uint64_t idx = (m << m_shift) | (f << free_shift);
    const auto a = st[idx];
    out[o] = make_double2((double)a.x, (double)a.y);
  }
}

int device_sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 132;
  }
  return sms;
}

int grid_for(uint64_t work, int block) {
  const int sms = device_sm_count();
  uint64_t g = (work + block - 1) / block;
  const uint64_t cap = (uint64_t)sms * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t launch_init(void* state, int prec, uint64_t n_amps, const uint64_t* d_idx,
                        const double* d_val, int64_t count, cudaStream_t st) {
  const size_t bytes = n_amps * (prec == CSIM_C64 ? sizeof(float2) : sizeof(double2));
  cudaError_t e = cudaMemsetAsync(state, 0, bytes, st);
  if (e != cudaSuccess) return e;
  if (count <= 0) return cudaSuccess;
  const int blk = 256;
  const int grd = (int)((count + blk - 1) / blk);
  if (prec == CSIM_C64)
    init_scatter_kernel<float><<<grd, blk, 0, st>>>((float2*)state, d_idx, d_val, count);
  else
    init_scatter_kernel<double><<<grd, blk, 0, st>>>((double2*)state, d_idx, d_val, count);
  return cudaGetLastError();
}

cudaError_t launch_init_sparse(void* state, int prec, int n, const uint64_t* d_idx,
                               const double* d_val, int64_t count, uint32_t* map, cudaStream_t st) {
  if (n < 12) return cudaErrorInvalidValue;  // the map has 2^(n-12) words
  cudaError_t e = cudaMemsetAsync(map, 0, ((size_t)1 << (n - 12)) * sizeof(uint32_t), st);
  if (e != cudaSuccess || count <= 0) return e;
  const int blk = 256;
  mark_tiles_kernel<<<(int)((count + blk - 1) / blk), blk, 0, st>>>(d_idx, count, map);
  const int zgrd = (int)((count * 32 + blk - 1) / blk);
  if (prec == CSIM_C64)
    zero_tiles_kernel<float><<<zgrd, blk, 0, st>>>((float2*)state, d_idx, count);
  else
    zero_tiles_kernel<double><<<zgrd, blk, 0, st>>>((double2*)state, d_idx, count);
  const int grd = (int)((count + blk - 1) / blk);
  if (prec == CSIM_C64)
    init_scatter_kernel<float><<<grd, blk, 0, st>>>((float2*)state, d_idx, d_val, count);
  else
    init_scatter_kernel<double><<<grd, blk, 0, st>>>((double2*)state, d_idx, d_val, count);
  return cudaGetLastError();
}

cudaError_t launch_gate(void* state, int prec, int n, const csim_gate& g, cudaStream_t st) {
  GateParams p;
  p.cmask = g.cmask;
  p.cval = g.cval;
  p.tbit = 1ull << g.target;
  const uint64_t fixedmask = g.cmask | p.tbit;
  p.nfixed = 0;
  for (int b = 0; b < 64; ++b)
    if ((fixedmask >> b) & 1ull) p.fixed[p.nfixed++] = (uint8_t)b;
  p.npairs = 1ull << (n - p.nfixed);
  p.op = g.op;
  if (g.op == 2) {
    p.c = cos(g.angle / 2.0);
    p.s = sin(g.angle / 2.0);
  } else if (g.op == 3) {
    p.c = cos(g.angle);
    p.s = sin(g.angle);
  } else {
    p.c = p.s = 0.0;
  }
  const int blk = 256;
  const int grd = grid_for(p.npairs, blk);
  if (prec == CSIM_C64)
    gate_kernel<float><<<grd, blk, 0, st>>>((float2*)state, p);
  else
    gate_kernel<double><<<grd, blk, 0, st>>>((double2*)state, p);
  return cudaGetLastError();
}

namespace {

// Tiles per warp iteration (U) and minimum resident blocks per SM (MINB) of
// the sweep kernel; CSIM_SWEEP_CFG="U,MINB" overrides the defaults.
struct SweepCfg {
  int u64, minb64, u128, minb128;
};

SweepCfg sweep_cfg() {
  static SweepCfg cfg = [] {
    // measured defaults: complex64 two tiles per iteration at 4 blocks/SM;
    // complex128 one tile at 2 blocks/SM (the wider variants spill)
    SweepCfg c{2, 4, 1, 2};
    if (const char* e = std::getenv("CSIM_SWEEP_CFG")) {
      int u = 0, m = 0;
      if (std::sscanf(e, "%d,%d", &u, &m) == 2 && (u == 1 || u == 2 || u == 4) &&
          (m == 1 || m == 2 || m == 4)) {
        c.u64 = u;
        c.u128 = u;
        c.minb64 = m;
        c.minb128 = m;
      }
    }
    return c;
  }();
  return cfg;
}

// Grid of the sweep kernel in resident waves: blocks = SMs x co-resident
// blocks per SM x waves (CSIM_SWEEP_WAVES overrides; default 4).  Measured on
// the 32-qubit QSVT circuit: 4 waves is 3% faster than one persistent wave,
// which also reads more from DRAM.
// A tuned launch shape (launch_sweep) sets the waves of the launches it makes
// on this thread.
thread_local int t_waves = 0;

int sweep_waves() {
  static const int w = [] {
    const char* e = std::getenv("CSIM_SWEEP_WAVES");
    const int v = e ? std::atoi(e) : 4;
    return (v >= 1 && v <= 64) ? v : 4;
  }();
  return t_waves > 0 ? t_waves : w;
}

// Tuned launch shapes per (precision, qubit count): u | minb << 4 | waves << 8,
// 0 for none.
std::atomic<uint32_t> g_shapes[2][64];

struct WavesScope {
  explicit WavesScope(int w) { t_waves = w; }
  ~WavesScope() { t_waves = 0; }
};

// Co-resident blocks of one sweep-kernel instantiation on the device (cached).
template <typename R, int U, int MINB, int SHAPE = 0, int BLK = 256>
int sweep_resident() {
  static int resident = 0;
  if (!resident) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<R, U, MINB, SHAPE, BLK>,
                                                  BLK, 0);
    resident = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  }
  return resident;
}

template <typename R, int U, int MINB, int SHAPE = 0, int BLK = 256>
void launch_sweep_t(const void* in, void* out, uint32_t ntiles, const SweepParams& a, cudaStream_t st) {
  using T = typename V2<R>::T;
  const int blk = BLK;
  // the default-block variants share one occupancy figure per (U, MINB)
  uint64_t grd = (uint64_t)(BLK == 256 ? sweep_resident<R, U, MINB>()
                                       : sweep_resident<R, U, MINB, SHAPE, BLK>()) *
                 sweep_waves();
  const uint64_t need = ((uint64_t)ntiles / U * 32 + blk - 1) / blk;
  if (grd > need) grd = need;
  if (grd < 1) grd = 1;
  // effective fast bits: the warp stride must be a multiple of 2^nfe, and a
  // warp's U tiles must fit in one group of 2^nfe
  const uint32_t stride = (uint32_t)grd * (blk / 32) * U;
  int nfe = a.nfast;
  while (nfe > 0 && (stride & ((1u << nfe) - 1u)) != 0u) --nfe;
  if (nfe > 0 && (1 << nfe) < U) nfe = 0;
  uint32_t fmask = 0, hstep = 0;
  for (int j = 0; j < nfe; ++j) fmask |= 1u << a.fast[j];
  uint32_t hv = stride >> nfe;
  for (int b = 0; hv != 0u && b < 32; ++b) {
    if ((fmask >> b) & 1u) continue;
    hstep |= (hv & 1u) << b;
    hv >>= 1;
  }
  sweep_kernel<R, U, MINB, SHAPE, BLK><<<(int)grd, blk, 0, st>>>((const T*)in, (T*)out, ntiles,
                                                                  nfe, fmask, hstep, a);
}

// The sweep shape of a parameter block (see apply_shaped).
template <typename S>
bool has_ops(const SweepParams& a) {
  if (a.nops != S::n) return false;
  int nm = 0, nr = 0;
  for (int i = 0; i < S::n; ++i) {
    const LocalOp& o = a.ops[i];
    if ((int)o.op != S::op[i]) return false;
    if (o.op == 4 && (int)o.cm != nm++) return false;
    if (o.op == 5 && (int)o.cm != nr++) return false;
  }
  return true;
}
int sweep_shape(const SweepParams& a) {
  if (has_ops<ShapeAvg>(a)) return 1;
  if (has_ops<ShapeMux>(a)) return 2;
  if (has_ops<ShapeFirst>(a)) return 3;
  if (has_ops<ShapeLast>(a)) return 4;
  return 0;
}

// Shaped kernels exist for the default variants only (complex64 <2, 4>,
// complex128 <1, 2>); CSIM_SWEEP_SHAPES=0 keeps every sweep generic.
bool shapes_enabled() {
  static const bool v = [] {
    const char* e = std::getenv("CSIM_SWEEP_SHAPES");
    return !(e && e[0] == '0');
  }();
  return v;
}

// Complex64 averaging sweeps (ShapeAvg, the conjugated gathers) run four
// tiles per warp iteration at two blocks per SM: a warp then loads and stores
// the sibling tiles whose chunks share 128-byte lines together.  Not with
// exactly one fast tile bit: four tiles per warp need two, and would force
// the natural order.  CSIM_AVG_CFG=2,4 gives them the variant of the other
// shapes.
bool avg_four_tiles() {
  static const bool v = [] {
    const char* e = std::getenv("CSIM_AVG_CFG");
    return !(e && std::strcmp(e, "2,4") == 0);
  }();
  return v;
}

template <typename R, int U, int MINB>
void launch_shaped(const void* in, void* out, uint32_t ntiles, const SweepParams& a,
                   cudaStream_t st) {
  const int shape = shapes_enabled() ? sweep_shape(a) : 0;
  if constexpr (sizeof(R) == 4) {
    if (shape == 1 && a.nfast != 1 && ntiles >= 4 && avg_four_tiles())
      return launch_sweep_t<R, 4, 2, 1>(in, out, ntiles, a, st);
  }
  if (shape == 1) return launch_sweep_t<R, U, MINB, 1>(in, out, ntiles, a, st);
  if (shape == 2) return launch_sweep_t<R, U, MINB, 2>(in, out, ntiles, a, st);
  if (shape == 3) return launch_sweep_t<R, U, MINB, 3>(in, out, ntiles, a, st);
  if (shape == 4) return launch_sweep_t<R, U, MINB, 4>(in, out, ntiles, a, st);
  return launch_sweep_t<R, U, MINB, 0>(in, out, ntiles, a, st);
}

template <typename R>
void launch_sweep_r(const void* in, void* out, uint32_t ntiles, int u, int minb, const SweepParams& a,
                    cudaStream_t st) {
  while ((uint32_t)u > ntiles) u >>= 1;
  if (minb == 4) {
    if (u == 2) {
      if constexpr (sizeof(R) == 4) return launch_shaped<R, 2, 4>(in, out, ntiles, a, st);
      return launch_sweep_t<R, 2, 4>(in, out, ntiles, a, st);
    }
    return launch_sweep_t<R, 1, 4>(in, out, ntiles, a, st);
  }
  if (minb == 2) {
    if (u == 4) return launch_sweep_t<R, 4, 2>(in, out, ntiles, a, st);
    if (u == 2) return launch_sweep_t<R, 2, 2>(in, out, ntiles, a, st);
    if constexpr (sizeof(R) == 8) return launch_shaped<R, 1, 2>(in, out, ntiles, a, st);
    return launch_sweep_t<R, 1, 2>(in, out, ntiles, a, st);
  }
  if (u == 4) return launch_sweep_t<R, 4, 1>(in, out, ntiles, a, st);
  if (u == 2) return launch_sweep_t<R, 2, 1>(in, out, ntiles, a, st);
  return launch_sweep_t<R, 1, 1>(in, out, ntiles, a, st);
}

// A sweep with staged qubits runs 2^nstage tiles per warp iteration (the
// lean gate interpreter when it holds gates only); the resident blocks per SM
// fall as the registers hold 2^nstage x 4 amplitudes a thread.
// A sweep of gates only (no multiplexer, averaging block or Walsh-Hadamard
// op) runs the lean interpreter (SHAPE 5).
bool gates_only(const SweepParams& a) {
  for (int k = 0; k < a.nops; ++k) {
    const int op = a.ops[k].op;
    if (op == 4 || op == 5 || op == 7 || op == 8) return false;
  }
  return true;
}

// MINB / BLK: the lean kernel's launch shape; the generic interpreter keeps
// 256-thread blocks at MINB0.
template <typename R, int U, int MINB, int BLK, int MINB0>
void launch_staged_u(const void* in, void* out, uint32_t ntiles, const SweepParams& a,
                     cudaStream_t st) {
  if (gates_only(a)) return launch_sweep_t<R, U, MINB, 5, BLK>(in, out, ntiles, a, st);
  return launch_sweep_t<R, U, MINB0, 0>(in, out, ntiles, a, st);
}

template <typename R>
void launch_staged(const void* in, void* out, uint32_t ntiles, const SweepParams& a,
                   cudaStream_t st) {
  if (a.nstage == 1) {
    if constexpr (sizeof(R) == 4) return launch_staged_u<R, 2, 4, 256, 4>(in, out, ntiles, a, st);
    return launch_staged_u<R, 2, 2, 256, 2>(in, out, ntiles, a, st);
  }
  // 128-thread blocks: the register file, not the block size, sets how many
  // warps a 4- or 8-tile sweep keeps resident
  if (a.nstage == 2) {
    if constexpr (sizeof(R) == 4) return launch_staged_u<R, 4, 6, 128, 2>(in, out, ntiles, a, st);
    return launch_staged_u<R, 4, 4, 128, 1>(in, out, ntiles, a, st);
  }
  // eight tiles (32 complex64 or complex128 amplitudes a thread)
  if constexpr (sizeof(R) == 4) return launch_staged_u<R, 8, 3, 128, 1>(in, out, ntiles, a, st);
  return launch_staged_u<R, 8, 2, 128, 1>(in, out, ntiles, a, st);
}

}  // namespace

cudaError_t launch_sweep(const void* in, void* out, int prec, int n, const SweepParams& a,
                         cudaStream_t st) {
  // the 256-bit chunk accesses need 32-byte aligned buffers
  if (((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 31u) != 0)
    return cudaErrorInvalidValue;
  const uint32_t ntiles = 1u << (n - 7);
  if (a.nstage > 0) {
    // the staged qubits are the first fast bits, all below the tile count
    if (a.nstage > kMaxStage || a.nfast < a.nstage || a.scatter || (ntiles >> a.nstage) == 0)
      return cudaErrorInvalidValue;
    for (int j = 0; j < a.nstage; ++j)
      if ((1u << a.fast[j]) >= ntiles) return cudaErrorInvalidValue;
    if (prec == CSIM_C64)
      launch_staged<float>(in, out, ntiles, a, st);
    else
      launch_staged<double>(in, out, ntiles, a, st);
    return cudaGetLastError();
  }
  const SweepCfg c = sweep_cfg();
  int u = prec == CSIM_C64 ? c.u64 : c.u128, minb = prec == CSIM_C64 ? c.minb64 : c.minb128;
  // a tuned shape for this class, except on the sweeps that complete a sparse
  // init (their zero handling exists in the default variant only)
  LaunchShape t;
  const bool tuned = a.zero_map == nullptr && launch_shape_for(prec, n, &t);
  if (tuned) {
    u = t.u;
    minb = t.minb;
  }
  WavesScope ws(tuned ? t.waves : 0);
  if (prec == CSIM_C64)
    launch_sweep_r<float>(in, out, ntiles, u, minb, a, st);
  else
    launch_sweep_r<double>(in, out, ntiles, u, minb, a, st);
  return cudaGetLastError();
}

bool valid_launch_shape(int prec, const LaunchShape& s) {
  if (s.waves < 1 || s.waves > 64) return false;
  if (!(s.u == 1 || s.u == 2 || s.u == 4) || !(s.minb == 1 || s.minb == 2 || s.minb == 4))
    return false;
  if (s.u == 4 && s.minb == 4) return false;  // not a kernel variant
  (void)prec;
  return true;
}

void set_launch_shape(int prec, int n, const LaunchShape* s) {
  if (n < 0 || n >= 64) return;
  const int p = prec == CSIM_C64 ? 0 : 1;
  const uint32_t v = s ? (uint32_t)s->u | ((uint32_t)s->minb << 4) | ((uint32_t)s->waves << 8) : 0u;
  g_shapes[p][n].store(v, std::memory_order_relaxed);
}

bool launch_shape_for(int prec, int n, LaunchShape* s) {
  if (n < 0 || n >= 64) return false;
  const uint32_t v = g_shapes[prec == CSIM_C64 ? 0 : 1][n].load(std::memory_order_relaxed);
  if (v == 0u) return false;
  s->u = (int)(v & 15u);
  s->minb = (int)((v >> 4) & 15u);
  s->waves = (int)(v >> 8);
  return true;
}

LaunchShape default_launch_shape(int prec) {
  const SweepCfg c = sweep_cfg();
  const int save = t_waves;
  t_waves = 0;
  LaunchShape s{prec == CSIM_C64 ? c.u64 : c.u128, prec == CSIM_C64 ? c.minb64 : c.minb128,
                sweep_waves()};
  t_waves = save;
  return s;
}

cudaError_t launch_perm_index(uint32_t* src, int n, const SweepParams& a, cudaStream_t st) {
  const uint64_t nchunks = 1ull << (n - 2);
  const int blk = 256;
  const int grd = grid_for((nchunks + kPermIndexILP - 1) / kPermIndexILP, blk);
  perm_index_kernel<<<grd, blk, 0, st>>>(src, nchunks, a);
  return cudaGetLastError();
}

int sweep_zero_kind(int prec, int n, const SweepParams& a) {
  // the same choice as launch_sweep: a shaped kernel of the default variant
  // (ShapeFirst in place, or ShapeAvg gathering)
  if (n < 12 || !shapes_enabled() || a.scatter) return 0;
  const int shape = sweep_shape(a);
  int kind = 0;
  if (shape == 3 && a.nseg == 0) kind = 1;
  if (shape == 1 && a.nseg > 0) kind = 3;
  if (kind == 0) return 0;
  const SweepCfg c = sweep_cfg();
  const uint32_t ntiles = 1u << (n - 7);
  int u = prec == CSIM_C64 ? c.u64 : c.u128;
  while ((uint32_t)u > ntiles) u >>= 1;
  const bool shaped = prec == CSIM_C64 ? (u == 2 && c.minb64 == 4) : (u == 1 && c.minb128 == 2);
  return shaped ? kind : 0;
}

cudaError_t launch_zero_unmarked(void* state, int prec, int n, const uint32_t* map,
                                 cudaStream_t st) {
  if (n < 12) return cudaErrorInvalidValue;
  const uint32_t ntiles = 1u << (n - 7);
  const int blk = 256;
  const int grd = grid_for((uint64_t)ntiles * 32, blk);
  if (prec == CSIM_C64)
    zero_unmarked_kernel<float><<<grd, blk, 0, st>>>((float2*)state, map, ntiles);
  else
    zero_unmarked_kernel<double><<<grd, blk, 0, st>>>((double2*)state, map, ntiles);
  return cudaGetLastError();
}

int norm_partials_needed() { return 2048; }

namespace {
// Co-resident 256-thread blocks of the norm kernel on the device (cached).
int norm_resident(int prec) {
  static int resident[2] = {0, 0};
  int& res = resident[prec == CSIM_C64 ? 0 : 1];
  if (!res) {
    int per_sm = 0;
    if (prec == CSIM_C64)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, norm_kernel<float>, 256, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, norm_kernel<double>, 256, 0);
    res = device_sm_count() * (per_sm > 0 ? per_sm : 1);
  }
  return res;
}
}  // namespace

namespace {
template <typename R>
cudaError_t warm_r() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  chk(cudaFuncGetAttributes(&fa, init_scatter_kernel<R>));
  chk(cudaFuncGetAttributes(&fa, zero_tiles_kernel<R>));
  chk(cudaFuncGetAttributes(&fa, zero_unmarked_kernel<R>));
  chk(cudaFuncGetAttributes(&fa, gate_kernel<R>));
  chk(cudaFuncGetAttributes(&fa, norm_kernel<R>));
  chk(cudaFuncGetAttributes(&fa, compact_kernel<R>));
  if constexpr (sizeof(R) == 4) {
    chk(cudaFuncGetAttributes(&fa, sweep_kernel<R, 2, 4, 1>));
    chk(cudaFuncGetAttributes(&fa, sweep_kernel<R, 4, 2, 1>));
    chk(cudaFuncGetAttributes(&fa, sweep_kernel<R, 2, 4, 2>));
    chk(cudaFuncGetAttributes(&fa, sweep_kernel<R, 2, 4, 3>));
    chk(cudaFuncGetAttributes(&fa, sweep_kernel<R, 2, 4, 4>));
  } else {
    chk(cudaFuncGetAttributes(&fa, sweep_kernel<R, 1, 2, 1>));
    chk(cudaFuncGetAttributes(&fa, sweep_kernel<R, 1, 2, 2>));
    chk(cudaFuncGetAttributes(&fa, sweep_kernel<R, 1, 2, 3>));
    chk(cudaFuncGetAttributes(&fa, sweep_kernel<R, 1, 2, 4>));
  }
  sweep_resident<R, 1, 1>();
  sweep_resident<R, 2, 1>();
  sweep_resident<R, 4, 1>();
  sweep_resident<R, 1, 2>();
  sweep_resident<R, 2, 2>();
  sweep_resident<R, 4, 2>();
  sweep_resident<R, 1, 4>();
  sweep_resident<R, 2, 4>();
  if constexpr (sizeof(R) == 4) {
    sweep_resident<R, 4, 6, 5, 128>();
    sweep_resident<R, 8, 3, 5, 128>();
  } else {
    sweep_resident<R, 4, 4, 5, 128>();
    sweep_resident<R, 8, 2, 5, 128>();
  }
  return e;
}
}  // namespace

cudaError_t warm_kernels() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, reduce_partials_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, perm_index_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, mark_tiles_kernel);
  if (e == cudaSuccess) e = warm_r<float>();
  if (e == cudaSuccess) e = warm_r<double>();
  sweep_cfg();
  sweep_waves();
  grid_for(1, 256);
  norm_resident(CSIM_C64);
  norm_resident(CSIM_C128);
  return e;
}

cudaError_t launch_norms_fused(const void* state, int prec, int n, const uint64_t* d_pm,
                               const uint64_t* d_pv, int npat, int lowk, uint64_t lowv,
                               const double* d_norm_part, double* d_partial, double* d_out,
                               cudaStream_t st) {
  const uint64_t N = 1ull << n;
  const int blk = 256;
  const int res = norm_resident(prec);
  int grd = grid_for(N >> lowk, blk);
  if (grd > res) grd = res;
  if (grd > norm_partials_needed()) grd = norm_partials_needed();
  if (grd < 1) grd = 1;
  if (prec == CSIM_C64)
    norm_kernel<float, false><<<grd, blk, 0, st>>>((const float2*)state, N, d_pm, d_pv, npat,
                                                   lowk, lowv, d_partial);
  else
    norm_kernel<double, false><<<grd, blk, 0, st>>>((const double2*)state, N, d_pm, d_pv, npat,
                                                    lowk, lowv, d_partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_fused_kernel<<<1, 32, 0, st>>>(d_norm_part, d_partial, grd, d_out);
  return cudaGetLastError();
}

bool sweep_fuses_norm(int prec, int n, const SweepParams& a) {
  // the choice launch_sweep makes: the shaped last-sweep kernel of the
  // default variant (complex64 <2, 4>, complex128 <1, 2>)
  if (n < 12 || a.nstage > 0 || !shapes_enabled() || sweep_shape(a) != 4) return false;
  const SweepCfg c = sweep_cfg();
  int u = prec == CSIM_C64 ? c.u64 : c.u128, minb = prec == CSIM_C64 ? c.minb64 : c.minb128;
  LaunchShape t;
  if (a.zero_map == nullptr && launch_shape_for(prec, n, &t)) {
    u = t.u;
    minb = t.minb;
  }
  const uint32_t ntiles = 1u << (n - 7);
  while ((uint32_t)u > ntiles) u >>= 1;
  return prec == CSIM_C64 ? (u == 2 && minb == 4) : (u == 1 && minb == 2);
}

cudaError_t launch_norms(const void* state, int prec, int n, const uint64_t* d_pm,
                         const uint64_t* d_pv, int npat, int lowk, uint64_t lowv, double* d_partial,
                         double* d_out, cudaStream_t st) {
  const uint64_t N = 1ull << n;
  const int blk = 256;
  // one full wave of resident blocks (a partial second wave would finish
  // alone at reduced bandwidth), at most the partial-sum capacity
  const int res = norm_resident(prec);
  int grd = grid_for(N / 2, blk);
  if (grd > res) grd = res;
  if (grd > norm_partials_needed()) grd = norm_partials_needed();
  if (prec == CSIM_C64)
    norm_kernel<float><<<grd, blk, 0, st>>>((const float2*)state, N, d_pm, d_pv, npat, lowk, lowv,
                                            d_partial);
  else
    norm_kernel<double><<<grd, blk, 0, st>>>((const double2*)state, N, d_pm, d_pv, npat, lowk,
                                             lowv, d_partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_partials_kernel<<<1, 32, 0, st>>>(d_partial, grd, d_out);
  return cudaGetLastError();
}

cudaError_t launch_compact(const void* state, int prec, double* d_out, uint64_t count,
                           int free_shift, int free_bits, uint64_t m_first, int m_shift,
                           cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int blk = 256;
  const int grd = grid_for(count, blk);
  if (prec == CSIM_C64)
    compact_kernel<float><<<grd, blk, 0, st>>>((const float2*)state, (double2*)d_out, count,
                                               free_shift, free_bits, m_first, m_shift);
  else
    compact_kernel<double><<<grd, blk, 0, st>>>((const double2*)state, (double2*)d_out, count,
                                                free_shift, free_bits, m_first, m_shift);
  return cudaGetLastError();
}

}  // namespace csim

// ------------------------------------------------------ persistent batches
namespace csim {
namespace {

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

constexpr int kBatchThreads = 256;
constexpr uint64_t kBatchWaitNs = 2000000000ull;  // a dependency wait gives up after 2 s

// One persistent launch over the sweeps of many programs.  Every CTA takes
// the next item of a queue in global memory (a range of tile counters of one
// step) and waits, with a time limit, until every item of the step it
// depends on (the same program's previous step) has signalled; its warps
// apply the step to their tiles (the sweep kernels' op bodies for the four
// sweep op lists; the pool sends only such steps, gathers with source-index
// tables, and runs the sweeps that complete a sparse init before the launch)
// and the CTA signals.  An item waits only for items earlier in the queue,
// which running CTAs have taken, so the earliest unfinished item never waits
// and the launch progresses whether or not all its CTAs are resident at once
// (another launch may share the SMs).  While the queue's head waits, CTAs
// beyond the number of items left leave.  A wait that runs out (2 s) records
// the error and every CTA stops at its next wait.
template <typename R, int U, int MINB>
__global__ void __launch_bounds__(kBatchThreads, MINB)
    batch_kernel(const BatchStep* __restrict__ steps, const BatchItem* __restrict__ items,
                 uint32_t nitems, uint32_t* done, BatchCtl* ctl, int may_leave) {
  using T = typename V2<R>::T;
  __shared__ uint32_t s_item;
  __shared__ int s_ok;
  // the item's sweep parameters, copied once per item: the op bodies read
  // them from shared memory instead of holding global loads in registers
  __shared__ __align__(16) SweepParams s_a;
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  for (;;) {
    // thread 0 takes the next ticket of the queue (one atomic add) and waits
    // until every item of the step the ticket's item depends on has
    // signalled.  Before that, while the queue's head item cannot start yet,
    // CTAs beyond the number of items left in the queue leave the launch:
    // they would only wait, and their SMs go to other launches (the next
    // pass).
    if (threadIdx.x == 0) {
      uint32_t got = ~0u;
      int ok = 1;
      const uint32_t h = *reinterpret_cast<volatile uint32_t*>(&ctl->next);
      bool leave = h >= nitems;
      if (!leave && may_leave) {
        const BatchStep& hs = steps[items[h].step];
        if (hs.dep >= 0 &&
            *reinterpret_cast<volatile uint32_t*>(done + hs.dep) < steps[hs.dep].nitems) {
          const uint32_t gone = atomicAdd(&ctl->exited, 1u);
          leave = gridDim.x - gone > nitems - h;
          if (!leave) atomicSub(&ctl->exited, 1u);
        }
      }
      if (!leave) {
        const uint32_t t = atomicAdd(&ctl->next, 1u);
        if (t < nitems) {
          got = t;
          const BatchStep& ts = steps[items[t].step];
          if (ts.dep >= 0) {
            const uint32_t need = steps[ts.dep].nitems;
            const uint64_t t0 = global_ns();
            while (*reinterpret_cast<volatile uint32_t*>(done + ts.dep) < need) {
              if (*reinterpret_cast<volatile uint32_t*>(&ctl->error) != 0u) {
                ok = 0;
                break;
              }
              if (global_ns() - t0 > kBatchWaitNs) {
                atomicOr(&ctl->error, 1u);
                ok = 0;
                break;
              }
              __nanosleep(200);
            }
          }
        }
      }
      __threadfence();
      s_item = got;
      s_ok = ok;
    }
    __syncthreads();
    const uint32_t k = s_item;
    if (!s_ok || k == ~0u) break;
    const BatchItem it = items[k];
    const BatchStep& bs = steps[it.step];
    {
      const uint4* src = reinterpret_cast<const uint4*>(bs.sp);
      uint4* dst = reinterpret_cast<uint4*>(&s_a);
      for (uint32_t i = threadIdx.x; i < sizeof(SweepParams) / 16; i += kBatchThreads) dst[i] = src[i];
    }
    __syncthreads();
    const SweepParams& a = s_a;
    const T* in = static_cast<const T*>(bs.in);
    T* out = static_cast<T*>(bs.out);
    const int nfe = (int)bs.nfe;
    const uint32_t fmask = bs.fmask;
    // Counters: the step's items split its counter range into 2^li items of
    // 64 iterations of S = kBatchThreads / 32 * U counters.  Iteration j of
    // item k, warp w, tile u takes counter (w U + u) | k << s | j << (s + li)
    // (S = 2^s), so that while the CTAs holding the step's items run their
    // j-th iterations together, they cover a contiguous window of S 2^li
    // counters, as one iteration of the sweep kernel's grid does, and the
    // step's fast tile bits (at most s + li) give the same tile order.  The
    // low nfe counter bits are fixed per warp and item: their deposit L[u]
    // is computed once, and the high part H advances by the masked add of
    // hstep (the deposit of 2^(s + li - nfe)).
    constexpr uint32_t S = (kBatchThreads / 32) * U;
    constexpr int sb = U == 4 ? 5 : 4;
    static_assert((1u << sb) == S, "S is a power of two");
    const uint32_t li = bs.li;
    const uint32_t kk = it.c0 >> (sb + 6);
    const uint32_t nj = (it.c1 - it.c0) >> sb;
    const uint32_t cw = (wib * U) | (kk << sb);
    uint32_t L[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      uint32_t d = 0;
      for (int j = 0; j < nfe; ++j) d |= (((cw + (uint32_t)u) >> j) & 1u) << a.fast[j];
      L[u] = nfe > 0 ? d : (uint32_t)u;
    }
    uint32_t H = 0;
    if (nfe > 0) {
      uint32_t hv = cw >> nfe;
      for (int b = 0; hv != 0u && b < 32; ++b) {
        if ((fmask >> b) & 1u) continue;
        H |= (hv & 1u) << b;
        hv >>= 1;
      }
    } else {
      H = cw;
    }
    const uint32_t jstep = 1u << (sb + li);
    // source indices of the warp's next tiles, loaded one iteration ahead
    const bool pre = a.src != nullptr;
    uint32_t nxt[U];
    if (pre && nj > 0) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        nxt[u] = __ldcs(a.src + (((nfe > 0 ? (H | L[u]) : (H + L[u])) << 5) | lane));
    }
    double* const npart = bs.shape == 4 ? bs.norm_part : nullptr;
    double nacc = 0.0;
    for (uint32_t j = 0; j < nj; ++j) {
      uint32_t ci[U], mv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) mv[u] = ci[u] = ((nfe > 0 ? (H | L[u]) : (H + L[u])) << 5) | lane;
      H = nfe > 0 ? (((H | fmask) + bs.hstep) & ~fmask) : (H + jstep);
      uint32_t wd[kPrefetchMux][U];
      if (bs.shape != 1) prefetch_mux<U>(a, ci, wd);
      T v[U][4];
      // gathers load their source indices (one iteration ahead); the other
      // sweeps do not move data (mv = ci)
      if (pre) {
#pragma unroll
        for (int u = 0; u < U; ++u) mv[u] = nxt[u];
        if (j + 1 < nj) {
#pragma unroll
          for (int u = 0; u < U; ++u)
            nxt[u] = __ldcs(a.src + (((nfe > 0 ? (H | L[u]) : (H + L[u])) << 5) | lane));
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) load_chunk(in + ((size_t)mv[u] << 2), v[u]);
      // the sweep kernels' op bodies, so a request's result does not depend
      // on which path ran it
      switch (bs.shape) {
        case 1: apply_shaped<R, U, 1>(a, v, ci, lane, wd); break;
        case 2: apply_shaped<R, U, 2>(a, v, ci, lane, wd); break;
        case 3: apply_shaped<R, U, 3>(a, v, ci, lane, wd); break;
        default: apply_shaped<R, U, 4>(a, v, ci, lane, wd); break;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        store_chunk(out + ((size_t)(a.inplace ? mv[u] : ci[u]) << 2), v[u]);
      if (npart) {
#pragma unroll
        for (int u = 0; u < U; ++u) nacc += chunk_norm2(v[u]);
      }
    }
    if (npart) {  // the item's |a|^2, in a fixed order (CTA-uniform branch)
      __shared__ double s_norm[kBatchThreads / 32];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nacc += __shfl_xor_sync(0xffffffffu, nacc, o);
      if (lane == 0) s_norm[wib] = nacc;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kBatchThreads / 32; ++w) t += s_norm[w];
        if (kk + 1u < kNormPartCap) npart[1 + kk] = t;
        if (kk == 0) npart[0] = (double)bs.nitems;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (k != ctl->drop_item) atomicAdd(done + it.step, 1u);
    }
  }
}

}  // namespace

// Tiles per warp iteration and CTAs per SM of the persistent kernel
// (CSIM_BATCH_CFG="U,MINB"): 2,4 by default, as the sweep kernel's complex64
// variant, with a few of the op bodies' registers spilled; 2,2 keeps all of
// them at half the warps; 2,3 between; 4,2 holds four tiles a warp.
struct BatchCfg {
  int u, minb;
};

BatchCfg batch_cfg() {
  static const BatchCfg c = [] {
    BatchCfg v{2, 4};
    if (const char* e = std::getenv("CSIM_BATCH_CFG")) {
      int u = 0, m = 0;
      if (std::sscanf(e, "%d,%d", &u, &m) == 2 &&
          ((u == 2 && (m == 2 || m == 3 || m == 4)) || (u == 4 && m == 2)))
        v = BatchCfg{u, m};
    }
    return v;
  }();
  return c;
}

uint32_t batch_stride() { return (kBatchThreads / 32) * (uint32_t)batch_cfg().u; }

int batch_shape(const SweepParams& a) { return shapes_enabled() ? sweep_shape(a) : 0; }

void batch_order(const SweepParams& a, uint32_t ntiles, uint32_t* nfe, uint32_t* fmask,
                 uint32_t* hstep, uint32_t* li) {
  // tile order of the persistent kernel: items of 64 iterations of S
  // counters, 2^l of them; the fast bits that fit the window of S 2^l
  // counters the items' j-th iterations cover together
  const uint32_t S = batch_stride();
  int sb = 0;
  while ((1u << sb) < S) ++sb;
  const uint32_t items = ntiles / (S * 64u);
  int l = 0;
  while ((2u << l) <= items) ++l;
  int f = a.nstage > 0 ? 0 : a.nfast;
  if (f > sb + l) f = sb + l;
  if (f > 0 && (1u << f) < (uint32_t)batch_cfg().u) f = 0;
  uint32_t fm = 0, hs = 0;
  for (int j = 0; j < f; ++j) fm |= 1u << a.fast[j];
  uint32_t hv = 1u << (sb + l - f);
  for (int b = 0; hv != 0u && b < 32; ++b) {
    if ((fm >> b) & 1u) continue;
    hs |= (hv & 1u) << b;
    hv >>= 1;
  }
  *nfe = (uint32_t)f;
  *fmask = fm;
  *hstep = hs;
  *li = (uint32_t)l;
}

namespace {

template <int U, int MINB>
int batch_resident() {
  static int resident = 0;
  if (!resident) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel<float, U, MINB>,
                                                  kBatchThreads, 0);
    resident = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }
  return resident;
}

template <int U, int MINB>
void launch_batch_t(const BatchStep* d_steps, const BatchItem* d_items, uint32_t nitems,
                    uint32_t* d_done, BatchCtl* d_ctl, cudaStream_t st) {
  // the grid is the resident CTA count: more CTAs would only queue behind
  // the persistent ones.  (Progress does not depend on it: an item waits only
  // for items earlier in the queue, which running CTAs hold.)
  static const int leave = [] {
    const char* e = std::getenv("CSIM_BATCH_LEAVE");
    return e && e[0] == '0' ? 0 : 1;
  }();
  batch_kernel<float, U, MINB><<<batch_resident<U, MINB>(), kBatchThreads, 0, st>>>(
      d_steps, d_items, nitems, d_done, d_ctl, leave);
}

}  // namespace

cudaError_t warm_batch() {
  const BatchCfg c = batch_cfg();
  if (c.u == 4) batch_resident<4, 2>();
  if (c.u == 2 && c.minb == 2) batch_resident<2, 2>();
  if (c.u == 2 && c.minb == 3) batch_resident<2, 3>();
  if (c.u == 2 && c.minb == 4) batch_resident<2, 4>();
  return cudaGetLastError();
}

cudaError_t launch_batch(const BatchStep* d_steps, const BatchItem* d_items, uint32_t nitems,
                         uint32_t* d_done, BatchCtl* d_ctl, cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  const BatchCfg c = batch_cfg();
  if (c.u == 4)
    launch_batch_t<4, 2>(d_steps, d_items, nitems, d_done, d_ctl, st);
  else if (c.minb == 2)
    launch_batch_t<2, 2>(d_steps, d_items, nitems, d_done, d_ctl, st);
  else if (c.minb == 4)
    launch_batch_t<2, 4>(d_steps, d_items, nitems, d_done, d_ctl, st);
  else
    launch_batch_t<2, 3>(d_steps, d_items, nitems, d_done, d_ctl, st);
  return cudaGetLastError();
}

}  // namespace csim
