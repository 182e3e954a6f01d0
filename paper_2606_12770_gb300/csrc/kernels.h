// Host-side launch interface of the CUDA kernels in kernels.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/csim.h"

namespace csim {

// A table key made of at most two bit windows of a 32-bit chunk index
// (state index >> 2): key = bits [lo0, lo0+w0) | bits [lo1, lo1+w1) << w0.
struct KeyWin {
  uint8_t lo0, w0, lo1, w1;
};

// One step of a compiled permutation (chunk-index space):
//  kind 0: a run of multi-controlled X gates as a lookup table over the key
//          windows holding every bit the gates read or write; the table maps
//          the window bits of an index to those of its image (offset t);
//  kind 1: one gate applied directly: if ((x & m) == v) x ^= t;
//  kind 2: a controlled increment (neg = 0) or decrement (neg = 1) of the
//          register of `width` bits at `base`: if ((x & m) == v) r = r +- 1.
struct PermSeg {
  KeyWin win;
  uint8_t kind, base, width, neg;
  uint32_t m, v, t;
};

// One gate inside the 128-amplitude warp tile.  Controls are split into the
// chunk-index part (state bits >= 2) and state bits 0-1.
// op: 0 X, 1 H, 2 RY, 3 ZPHASE, 4 multiplexed RY (cm = index of its MuxDesc),
// 5 averaging block (cm = index of its ReflectDesc), 6 ZPHASE on a qubit above
// the tile (target = its chunk-index bit, state bit - 2), 7 the inverse of the
// sweep's latest multiplexed RY (the same rotation with the sine negated; its
// target and bit 0-1 controls in target, lm, lv), 8 H on every lane bit of the
// mask cm (no controls), followed by one scale 2^(-k/2) in cf / cd,
// 9 / 10 / 11 X / H / RY on the staged qubit `target` (an index into the
// sweep's staged qubits, see SweepParams::nstage): a 2 x 2 map between the
// warp's tiles u and u ^ (1 << target), held in registers.
struct LocalOp {
  uint32_t cm, cv;
  uint8_t lm, lv, op, target;
  float cf, sf;   // RY cos/sin(theta/2); ZPHASE cos/sin(phi)
  double cd, sd;  // the same in FP64
};

// Multiplexed RY on an in-thread qubit: key windows of the chunk index select
// a bucket-table word: 0 = no rotation; bit 31 set = the bucket's gates all
// match, rotate by the precomputed angle with index (word & 0x7fffffff);
// otherwise (start << 8 | count) candidates whose chunk controls are checked
// in full.  All gates of one multiplexer share the controls (lm, lv) on state
// bits 0-1.
struct MuxDesc {
  KeyWin win;
  uint32_t tab_off;
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
constexpr int kMaxSeg = 32, kMaxOps = 40, kMaxRefl = 4, kMaxMux = 8, kMaxFast = 12;
struct SweepParams {
  int nseg, nops, scatter, nmux;
  // Tile order (gather form): tile-index bits that vary fastest, most useful
  // first.  Tiles whose sources share 128-byte lines differ in these bits, so
  // they are processed together and the shared lines are read from DRAM once.
  int nfast;
  uint8_t fast[kMaxFast];
  PermSeg segs[kMaxSeg];
  LocalOp ops[kMaxOps];
  ReflectDesc refl[kMaxRefl];
  MuxDesc mux[kMaxMux];
  const uint16_t* lut;
  const uint32_t* mtab;
  const MuxEntryF* mentf;
  const MuxEntryD* mentd;
  const float2* angf;   // cos, sin of the summed angle of pure buckets
  const double2* angd;
  // When set, src[x] is the segments applied to chunk x, precomputed by
  // launch_perm_index: in the gather form the source chunk of destination x,
  // in the scatter form the destination of chunk x.  The kernel loads it
  // instead of walking the segment chain.
  const uint32_t* src;
  int src_prefetch;  // load the next iteration's source indices one iteration ahead
  // Gather form: store each chunk back to the address it was loaded from
  // (in == out), so that the sweep applies P^-1 . ops . P in place, P the
  // segments' permutation: a permutation, tile ops, and the inverse
  // permutation in one pass.
  int inplace;
  // The leading sweeps after a sparse csim_init.  Tiles (128 amplitudes)
  // whose bit is clear in zero_map (bit t of word t / 32) hold zeros that
  // were never written.  zero_mode says how the sweep treats them:
  //   1: in-place tile sweep (ShapeFirst).  The sweep maps each tile to
  //      itself linearly, so it writes zeros there without loading them or
  //      applying the ops;
  //   2: the same sweep, but unmarked tiles are left unwritten (the next
  //      sweep reads zeros for them);
  //   3: gather sweep (ShapeAvg): a gathered chunk in an unmarked tile is
  //      read as zeros.  The sweep writes every chunk, so the state is whole
  //      afterwards.
  // In modes 1 and 2 a tile that shares a warp iteration with a marked one
  // is read as zeros.
  const uint32_t* zero_map;
  int zero_mode;
  // Staged high qubits (gather or in-place sweeps; 0 = none, at most 3).  The
  // sweep runs 2^nstage tiles per warp iteration, and its first nstage fast
  // tile bits (fast[0..nstage-1], always honoured) are these qubits' tile
  // bits (state bit - 7): the warp's tile u has bit j of u in fast[j].  Gates
  // on those qubits (ops 9-11) then pair registers of two tiles of the warp.
  int nstage;
  // The last sweep of a program (ShapeLast, the shaped kernel) may also sum
  // |a|^2 of the state it writes: each block adds the FP64 sum of its
  // chunks (four complex64 amplitudes squared and added in FP32, or complex128
  // in FP64) into norm_part[1 + block], block 0 writes the block count into
  // norm_part[0].  nullptr: no sum.  (sweep_fuses_norm says when it applies.)
  double* norm_part;
  uint64_t norm_pad;  // keeps the size a multiple of 16 bytes
};
static_assert(sizeof(SweepParams) % 16 == 0, "SweepParams is copied as 16-byte words");
constexpr int kMaxStage = 3;
// Doubles of a norm_part buffer: the count and one partial per block of the
// largest sweep grid (8 blocks per SM, 64 resident waves, 152 SMs).
constexpr size_t kNormPartCap = size_t(1) << 17;

cudaError_t launch_init(void* state, int prec, uint64_t n_amps, const uint64_t* d_idx,
                        const double* d_val, int64_t count, cudaStream_t st);
// Sparse initialisation for a first sweep that takes a zero map: marks the
// tiles holding the count entries in map (2^(n-7) bits, cleared here), zeroes
// those tiles and scatters the entries.  The other tiles are left unwritten.
cudaError_t launch_init_sparse(void* state, int prec, int n, const uint64_t* d_idx,
                               const double* d_val, int64_t count, uint32_t* map, cudaStream_t st);
// Whether launch_sweep runs this sweep with a kernel that honours zero_map:
// 1 for an in-place tile sweep (modes 1, 2), 3 for a gather sweep (mode 3),
// 0 otherwise.
int sweep_zero_kind(int prec, int n, const SweepParams& a);
// Zero the tiles whose bit is clear in map (completes a sparse init early).
cudaError_t launch_zero_unmarked(void* state, int prec, int n, const uint32_t* map,
                                 cudaStream_t st);
cudaError_t launch_gate(void* state, int prec, int n, const csim_gate& g, cudaStream_t st);
// Launch shape of the sweeps of one (precision, qubit count) class: tiles per
// warp iteration, minimum resident blocks per SM, grid in resident waves.
// set_launch_shape (nullptr clears) makes launch_sweep use it for that class
// in this process; the sweeps that complete a sparse init keep the default.
struct LaunchShape {
  int u, minb, waves;
};
bool valid_launch_shape(int prec, const LaunchShape& s);
void set_launch_shape(int prec, int n, const LaunchShape* s);
bool launch_shape_for(int prec, int n, LaunchShape* s);
LaunchShape default_launch_shape(int prec);
// Whether launch_sweep runs this sweep with the kernel that sums |a|^2 into
// norm_part (the shaped last sweep of the default kernel variant).
bool sweep_fuses_norm(int prec, int n, const SweepParams& a);
// launch_norms with the total taken from a fused sweep's norm_part (the
// masked sum is computed here); the same output (d_out[0] total, d_out[1]
// masked).
cudaError_t launch_norms_fused(const void* state, int prec, int n, const uint64_t* d_pm,
                               const uint64_t* d_pv, int npat, int lowk, uint64_t lowv,
                               const double* d_norm_part, double* d_partial, double* d_out,
                               cudaStream_t st);
cudaError_t launch_sweep(const void* in, void* out, int prec, int n, const SweepParams& a,
                         cudaStream_t st);
// src[x] = the segments of `a` applied to chunk index x, for every chunk of an
// n-qubit state (2^(n-2) entries).
cudaError_t launch_perm_index(uint32_t* src, int n, const SweepParams& a, cudaStream_t st);
int norm_partials_needed();
// Load every kernel of this file and compute the cached launch shapes (before
// any stream capture).
cudaError_t warm_kernels();
// FP64 total norm and masked norm.  Every pattern must fix the lowk lowest
// index bits to the value lowv (lowk = 0 checks every index).
cudaError_t launch_norms(const void* state, int prec, int n, const uint64_t* d_pm,
                         const uint64_t* d_pv, int npat, int lowk, uint64_t lowv, double* d_partial,
                         double* d_out, cudaStream_t st);
// Persistent batch execution of many fused programs (complex64): one step of
// one program, cut into items of tile-counter ranges.
struct BatchStep {
  const SweepParams* sp;  // device copy of the step's parameters (source tables filled)
  const void* in;
  void* out;
  uint32_t nitems;        // items the step was cut into
  int32_t dep;            // step that must finish first (the program's previous step), or -1
  uint32_t nfe, fmask, hstep;  // tile order of the kernel's items (batch_order)
  int32_t shape;          // op list of a shaped sweep kernel (batch_shape), 0 for any other
  uint32_t li;            // log2 of the step's items (batch_order)
  // the request's last sweep (shape 4) may sum |a|^2 of what it writes:
  // item k adds its FP64 sum into norm_part[1 + k], item 0 writes the item
  // count into norm_part[0] (the layout of SweepParams::norm_part); nullptr:
  // no sum
  double* norm_part;
};
// Item k of a step covers the counters of iterations [0, (c1 - c0) / S) of
// that item, c0 = k * 64 S (S = batch_stride()); the kernel maps them to tile
// counters interleaved across the step's items (see batch_kernel).
struct BatchItem {
  uint32_t step;    // index into the step array
  uint32_t c0, c1;  // c0 = k * 64 S; c1 - c0 = 64 S, or the whole step when it has one item
};
struct BatchCtl {
  uint32_t next;       // queue head, 0 at launch
  uint32_t error;      // set when a dependency wait ran out
  uint32_t drop_item;  // an item that does not signal (tests of the timeout); ~0u: none
  uint32_t exited;     // CTAs that left the launch early, 0 at launch
};
uint32_t batch_stride();
int batch_shape(const SweepParams& a);
void batch_order(const SweepParams& a, uint32_t ntiles, uint32_t* nfe, uint32_t* fmask,
                 uint32_t* hstep, uint32_t* li);
// Kernel load and occupancy cache of the persistent kernel (before capture).
cudaError_t warm_batch();
// One launch of co-resident CTAs over all items; done[] (one counter per step)
// and ctl must be zeroed (drop_item set) before it.
cudaError_t launch_batch(const BatchStep* d_steps, const BatchItem* d_items, uint32_t nitems,
                         uint32_t* d_done, BatchCtl* d_ctl, cudaStream_t st);
cudaError_t launch_compact(const void* state, int prec, double* d_out, uint64_t count,
                           int free_shift, int free_bits, uint64_t m_first, int m_shift,
                           cudaStream_t st);

}  // namespace csim
