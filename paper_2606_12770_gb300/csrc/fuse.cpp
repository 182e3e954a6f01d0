// The fuser: groups consecutive elementary gates into sweeps, each one HBM pass.
//
// A sweep is  [permutation]  then  [tile-local gates]:
//  * permutation: a maximal run of multi-controlled X gates whose target is a
//    qubit >= 2 and whose controls avoid qubits 0-1.  Such a run maps every
//    4-amplitude chunk (qubits 0-1) to another chunk, so the kernel gathers
//    each destination chunk from the chunk obtained by applying the run's
//    gates in reverse order to the destination.  The reversed run is cut into
//    segments whose support (bits read or written) has at most kMaxSupport
//    bits; each segment becomes a lookup table over its support.
//  * tile-local gates: any gate whose target is one of the 7 lowest qubits
//    (the 128-amplitude warp tile); controls may sit anywhere.  Runs of RY
//    gates on the same in-thread qubit (0 or 1) commute and become one
//    multiplexed rotation: a few chunk-index bits select a bucket of
//    candidate gates, each checked in full.
// A gate fitting neither class (e.g. H on a high qubit) becomes its own
// single-gate step.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>

#include <cstring>

#include "fuse.h"

namespace csim {

namespace {

constexpr int kMaxSupport = 14;   // bits per permutation lookup table
constexpr int kMuxKeyBits = 11;   // bits of the multiplexer bucket key
constexpr int kMuxMinGates = 4;   // shorter RY runs stay individual gates

bool perm_eligible(const csim_gate& g) {
  return g.op == OP_X && g.target >= 2 && (g.cmask & 3ull) == 0;
}
bool local_eligible(const csim_gate& g) { return g.target <= 6; }

std::vector<BitRun> runs_of(uint32_t mask) {
  std::vector<BitRun> runs;
  int off = 0;
  for (int b = 0; b < 32;) {
    if (!((mask >> b) & 1u)) {
      ++b;
      continue;
    }
    int e = b;
    while (e < 32 && ((mask >> e) & 1u)) ++e;
    BitRun r;
    r.lo = (uint8_t)b;
    r.len = (uint8_t)(e - b);
    r.off = (uint8_t)off;
    r.pad = 0;
    runs.push_back(r);
    off += e - b;
    b = e;
  }
  return runs;
}

uint32_t deposit(uint32_t key, const std::vector<BitRun>& runs) {
  uint32_t x = 0;
  for (const BitRun& r : runs) x |= ((key >> r.off) & ((1u << r.len) - 1u)) << r.lo;
  return x;
}
uint32_t extract(uint32_t x, const std::vector<BitRun>& runs) {
  uint32_t k = 0;
  for (const BitRun& r : runs) k |= ((x >> r.lo) & ((1u << r.len) - 1u)) << r.off;
  return k;
}

struct ChunkGate {
  uint32_t m, v, t;
};

ChunkGate chunk_gate(const csim_gate& g) {
  return {(uint32_t)(g.cmask >> 2), (uint32_t)(g.cval >> 2), 1u << (g.target - 2)};
}

// Compile a run of X gates (time order) into lookup-table segments in
// evaluation order (the inverse permutation: gates taken from the last).
void compile_perm(const std::vector<csim_gate>& run, Program* p, Step* st) {
  st->seg_off = (int)p->segs.size();
  st->nseg = 0;
  size_t i = run.size();
  while (i > 0) {
    std::vector<ChunkGate> seg;
    uint32_t sup = 0;
    while (i > 0) {
      const ChunkGate cg = chunk_gate(run[i - 1]);
      const uint32_t ns = sup | cg.m | cg.t;
      if (!seg.empty() && (__builtin_popcount(ns) > kMaxSupport || (int)runs_of(ns).size() > kMaxRuns))
        break;
      sup = ns;
      seg.push_back(cg);
      --i;
    }
    const std::vector<BitRun> runs = runs_of(sup);
    const int w = __builtin_popcount(sup);
    PermSeg ps{};
    ps.supmask = sup;
    ps.lut_off = (uint32_t)p->lut.size();
    ps.nruns = (uint32_t)runs.size();
    for (size_t r = 0; r < runs.size(); ++r) ps.runs[r] = runs[r];
    for (uint32_t key = 0; key < (1u << w); ++key) {
      uint32_t x = deposit(key, runs);
      for (const ChunkGate& cg : seg)
        if ((x & cg.m) == cg.v) x ^= cg.t;
      p->lut.push_back((uint16_t)extract(x, runs));
    }
    p->segs.push_back(ps);
    ++st->nseg;
    p->stats.segments++;
    p->stats.max_support = std::max<int64_t>(p->stats.max_support, w);
  }
  p->stats.perm_gates += (int64_t)run.size();
}

LocalOp local_op(const csim_gate& g) {
  LocalOp o{};
  o.cm = (uint32_t)(g.cmask >> 2);
  o.cv = (uint32_t)(g.cval >> 2);
  o.lm = (uint8_t)(g.cmask & 3ull);
  o.lv = (uint8_t)(g.cval & 3ull);
  o.op = g.op;
  o.target = g.target;
  double c = 0.0, s = 0.0;
  if (g.op == OP_RY) {
    c = std::cos(g.angle / 2.0);
    s = std::sin(g.angle / 2.0);
  } else if (g.op == OP_ZPHASE) {
    c = std::cos(g.angle);
    s = std::sin(g.angle);
  }
  o.cd = c;
  o.sd = s;
  o.cf = (float)c;
  o.sf = (float)s;
  return o;
}

void compile_mux(const std::vector<csim_gate>& grp, Program* p) {
  // key bits: the chunk bits constrained by the most gates
  int freq[32] = {0};
  for (const csim_gate& g : grp) {
    const uint32_t m = (uint32_t)(g.cmask >> 2);
    for (int b = 0; b < 32; ++b) freq[b] += (m >> b) & 1u;
  }
  std::vector<int> order;
  for (int b = 0; b < 32; ++b)
    if (freq[b] > 0) order.push_back(b);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return freq[a] > freq[b]; });
  uint32_t keymask = 0;
  for (int b : order) {
    const uint32_t nk = keymask | (1u << b);
    if (__builtin_popcount(nk) > kMuxKeyBits || (int)runs_of(nk).size() > kMaxRuns) continue;
    keymask = nk;
  }
  const std::vector<BitRun> runs = runs_of(keymask);
  const int w = __builtin_popcount(keymask);
  std::vector<std::vector<int>> bucket((size_t)1 << w);
  for (size_t gi = 0; gi < grp.size(); ++gi) {
    const uint32_t m = (uint32_t)(grp[gi].cmask >> 2), v = (uint32_t)(grp[gi].cval >> 2);
    const uint32_t fixed_m = extract(m & keymask, runs), fixed_v = extract(v & keymask, runs);
    for (uint32_t key = 0; key < (1u << w); ++key)
      if ((key & fixed_m) == fixed_v) bucket[key].push_back((int)gi);
  }
  MuxDesc md{};
  md.nruns = (uint32_t)runs.size();
  for (size_t r = 0; r < runs.size(); ++r) md.runs[r] = runs[r];
  md.tab_off = (uint32_t)p->mtab.size();
  md.target = grp[0].target;
  for (uint32_t key = 0; key < (1u << w); ++key) {
    uint2 be;
    be.x = (uint32_t)p->ment.size();
    be.y = (uint32_t)bucket[key].size();
    p->mtab.push_back(be);
    p->stats.max_bucket = std::max<int64_t>(p->stats.max_bucket, be.y);
    for (int gi : bucket[key]) {
      const LocalOp o = local_op(grp[gi]);
      MuxEntry e{};
      e.cm = o.cm;
      e.cv = o.cv;
      e.lm = o.lm;
      e.lv = o.lv;
      e.cf = o.cf;
      e.sf = o.sf;
      e.cd = o.cd;
      e.sd = o.sd;
      p->ment.push_back(e);
    }
  }
  LocalOp mo{};
  mo.op = 4;
  mo.target = grp[0].target;
  mo.cm = (uint32_t)p->mux.size();
  p->mux.push_back(md);
  p->ops.push_back(mo);
  p->stats.mux++;
  p->stats.mux_gates += (int64_t)grp.size();
  p->stats.mux_entries = (int64_t)p->ment.size();
}

using cplx = std::complex<double>;

bool in_tile(const csim_gate& g) { return g.target <= 6 && (g.cmask >> 7) == 0; }

// Dense 128 x 128 matrix (column-major per input basis state) of a window of
// tile-only gates.
std::vector<cplx> tile_matrix(const std::vector<csim_gate>& run, size_t i, size_t j) {
  std::vector<cplx> U(128 * 128, 0.0);
  const double h = 0.70710678118654752440;
  for (int col = 0; col < 128; ++col) {
    cplx* v = &U[(size_t)col * 128];
    v[col] = 1.0;
    for (size_t k = i; k < j; ++k) {
      const csim_gate& g = run[k];
      const int tb = 1 << g.target;
      const double c2 = std::cos(g.angle / 2), s2 = std::sin(g.angle / 2);
      const cplx ph(std::cos(g.angle), std::sin(g.angle));
      for (int x = 0; x < 128; ++x) {
        if ((x & tb) || ((uint64_t)x & g.cmask) != g.cval) continue;
        cplx a0 = v[x], a1 = v[x | tb];
        switch (g.op) {
          case OP_X: v[x] = a1; v[x | tb] = a0; break;
          case OP_H: v[x] = (a0 + a1) * h; v[x | tb] = (a0 - a1) * h; break;
          case OP_RY: v[x] = c2 * a0 - s2 * a1; v[x | tb] = s2 * a0 + c2 * a1; break;
          default: v[x] = a0 * ph; v[x | tb] = a1 * std::conj(ph); break;
        }
      }
    }
  }
  return U;
}

// If the window's matrix is I (x) A + J (x) B over the lane bits in lanes
// (a 5-bit mask of lane-index bits), fill the descriptor and return true.
bool reflect_form(const std::vector<cplx>& U, uint32_t lanes, ReflectDesc* d) {
  auto at = [&](int row, int col) { return U[(size_t)col * 128 + row]; };
  const int cls = 1 << __builtin_popcount(lanes);
  int l1 = 0;
  for (int b = 0; b < 5; ++b)
    if ((lanes >> b) & 1u) { l1 = 1 << b; break; }
  cplx A[4][4], B[4][4];
  for (int y = 0; y < 4; ++y)
    for (int yp = 0; yp < 4; ++yp) {
      B[y][yp] = at((0 << 2) | y, (l1 << 2) | yp) * (double)cls;
      A[y][yp] = at(y, yp) - B[y][yp] / (double)cls;
    }
  for (int l = 0; l < 32; ++l)
    for (int lp = 0; lp < 32; ++lp) {
      const bool same_class = ((l ^ lp) & ~lanes & 31) == 0;
      for (int y = 0; y < 4; ++y)
        for (int yp = 0; yp < 4; ++yp) {
          cplx model = (l == lp ? A[y][yp] : 0.0) + (same_class ? B[y][yp] / (double)cls : 0.0);
          if (std::abs(at((l << 2) | y, (lp << 2) | yp) - model) > 1e-12) return false;
        }
    }
  std::memset(d, 0, sizeof(*d));
  d->lanemask = lanes;
  for (int y = 0; y < 4; ++y)
    for (int yp = 0; yp < 4; ++yp) {
      const int q = y * 4 + yp;
      const cplx av = A[y][yp], bv = B[y][yp] / (double)cls;
      d->ad[q] = make_double2(av.real(), av.imag());
      d->af[q] = make_float2((float)av.real(), (float)av.imag());
      d->bd[q] = make_double2(bv.real(), bv.imag());
      d->bf[q] = make_float2((float)bv.real(), (float)bv.imag());
      if (std::abs(av) > 1e-15) d->nzA |= 1u << q;
      if (std::abs(bv) > 1e-15) d->nzB |= 1u << q;
    }
  return true;
}

// Longest window starting at i (an H on a lane bit) with the averaging form.
size_t try_reflect(const std::vector<csim_gate>& run, size_t i, Program* p) {
  const csim_gate& g0 = run[i];
  if (!(g0.op == OP_H && g0.target >= 2 && g0.cmask == 0)) return 0;
  size_t end = i;
  while (end < run.size() && in_tile(run[end])) ++end;
  for (size_t j = end; j > i + 1; --j) {
    const csim_gate& gl = run[j - 1];
    if (!(gl.op == OP_H && gl.target >= 2 && gl.cmask == 0)) continue;
    uint32_t lanes = 0;
    for (size_t k = i; k < j; ++k)
      if (run[k].op == OP_H && run[k].target >= 2) lanes |= 1u << (run[k].target - 2);
    ReflectDesc d;
    if (!reflect_form(tile_matrix(run, i, j), lanes, &d)) continue;
    LocalOp mo{};
    mo.op = 5;
    mo.cm = (uint32_t)p->refl.size();
    p->refl.push_back(d);
    p->ops.push_back(mo);
    p->stats.reflect++;
    return j - i;
  }
  return 0;
}

void compile_local(const std::vector<csim_gate>& run, Program* p, Step* st) {
  st->op_off = (int)p->ops.size();
  size_t i = 0;
  while (i < run.size()) {
    const csim_gate& g = run[i];
    if (const size_t w = try_reflect(run, i, p)) {
      i += w;
      continue;
    }
    if (g.op == OP_RY && g.target < 2) {
      size_t j = i;
      while (j < run.size() && run[j].op == OP_RY && run[j].target == g.target) ++j;
      if ((int)(j - i) >= kMuxMinGates) {
        compile_mux(std::vector<csim_gate>(run.begin() + i, run.begin() + j), p);
        i = j;
        continue;
      }
    }
    p->ops.push_back(local_op(g));
    ++i;
  }
  st->nops = (int)p->ops.size() - st->op_off;
  p->stats.local_gates += (int64_t)run.size();
}

}  // namespace

void build_program(const std::vector<csim_gate>& gates, int n, csim_exec mode, Program* p) {
  *p = Program();
  p->n = n;
  p->mode = mode;
  for (const csim_gate& g : gates) p->amp_updates += gate_amp_updates(g, n);
  if (mode == CSIM_EXEC_GATE || n < 7 || n > 34) {
    for (const csim_gate& g : gates) {
      Step s;
      s.kind = 1;
      s.g = g;
      p->steps.push_back(s);
    }
    p->passes = (int64_t)p->steps.size();
    p->stats.single = p->passes;
    return;
  }
  std::vector<csim_gate> perm, local;
  bool open = false;
  auto close = [&]() {
    if (!open) return;
    Step st;
    st.kind = 0;
    compile_perm(perm, p, &st);
    compile_local(local, p, &st);
    p->steps.push_back(st);
    p->stats.sweeps++;
    perm.clear();
    local.clear();
    open = false;
  };
  for (const csim_gate& g : gates) {
    const bool pe = perm_eligible(g), le = local_eligible(g);
    if (open && local.empty() && pe) {
      perm.push_back(g);
      continue;
    }
    if (open && le) {
      local.push_back(g);
      continue;
    }
    close();
    if (pe || le) {
      open = true;
      (pe ? perm : local).push_back(g);
    } else {
      Step s;
      s.kind = 1;
      s.g = g;
      p->steps.push_back(s);
      p->stats.single++;
    }
  }
  close();
  p->passes = (int64_t)p->steps.size();
  for (const Step& s : p->steps)
    if (s.kind == 0 && s.nseg > 0) p->pingpong = true;
  p->stats.lut_entries = (int64_t)p->lut.size();
  if (std::getenv("CSIM_FUSE_STATS")) {
    const FuseStats& f = p->stats;
    std::fprintf(stderr,
                 "[csim fuse] n=%d sweeps=%lld single=%lld perm_gates=%lld segments=%lld "
                 "max_support=%lld lut=%lld local=%lld mux=%lld mux_gates=%lld entries=%lld "
                 "max_bucket=%lld reflect=%lld\n",
                 n, (long long)f.sweeps, (long long)f.single, (long long)f.perm_gates,
                 (long long)f.segments, (long long)f.max_support, (long long)f.lut_entries,
                 (long long)f.local_gates, (long long)f.mux, (long long)f.mux_gates,
                 (long long)f.mux_entries, (long long)f.max_bucket, (long long)f.reflect);
  }
}

namespace {
template <typename T>
cudaError_t up(T** d, const std::vector<T>& h, cudaStream_t st) {
  if (h.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)d, h.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}
}  // namespace

cudaError_t upload_program(Program* p, cudaStream_t st) {
  if (p->uploaded) return cudaSuccess;
  cudaError_t e = up(&p->d_segs, p->segs, st);
  if (e == cudaSuccess) e = up(&p->d_lut, p->lut, st);
  if (e == cudaSuccess) e = up(&p->d_ops, p->ops, st);
  if (e == cudaSuccess) e = up(&p->d_mux, p->mux, st);
  if (e == cudaSuccess) e = up(&p->d_mtab, p->mtab, st);
  if (e == cudaSuccess) e = up(&p->d_ment, p->ment, st);
  if (e == cudaSuccess) e = up(&p->d_refl, p->refl, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_program(p);
    return e;
  }
  p->uploaded = true;
  return cudaSuccess;
}

void free_program(Program* p) {
  void* ptrs[] = {p->d_segs, p->d_lut, p->d_ops, p->d_mux, p->d_mtab, p->d_ment, p->d_refl};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  p->d_segs = nullptr;
  p->d_lut = nullptr;
  p->d_ops = nullptr;
  p->d_mux = nullptr;
  p->d_mtab = nullptr;
  p->d_ment = nullptr;
  p->d_refl = nullptr;
  p->uploaded = false;
}

cudaError_t run_program(const Program& p, void* buf[2], int* cur, int prec, cudaStream_t st) {
  for (const Step& s : p.steps) {
    cudaError_t e;
    if (s.kind == 1) {
      e = launch_gate(buf[*cur], prec, p.n, s.g, st);
    } else {
      SweepArgs a;
      a.segs = p.d_segs + s.seg_off;
      a.nseg = s.nseg;
      a.ops = p.d_ops + s.op_off;
      a.nops = s.nops;
      a.lut = p.d_lut;
      a.mux = p.d_mux;
      a.mtab = p.d_mtab;
      a.ment = p.d_ment;
      a.refl = p.d_refl;
      if (s.nseg == 0) {
        e = launch_sweep(buf[*cur], buf[*cur], prec, p.n, a, st);
      } else {
        e = launch_sweep(buf[*cur], buf[1 - *cur], prec, p.n, a, st);
        *cur = 1 - *cur;
      }
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Host executor of a fused program with the kernel's semantics (FP64), used to
// test the fuser without a GPU.  amps: 2^n interleaved complex values.
void emulate_program(const Program& p, std::vector<double>* amps) {
  const int n = p.n;
  const size_t N = (size_t)1 << n;
  std::vector<double> other(2 * N);
  std::vector<double>* cur = amps;
  std::vector<double>* nxt = &other;
  const double h = 0.70710678118654752440;
  auto pair = [&](double* a, double* b, int op, double c, double s) {
    double ar = a[0], ai = a[1], br = b[0], bi = b[1];
    switch (op) {
      case 0:
        a[0] = br; a[1] = bi; b[0] = ar; b[1] = ai;
        break;
      case 1:
        a[0] = (ar + br) * h; a[1] = (ai + bi) * h; b[0] = (ar - br) * h; b[1] = (ai - bi) * h;
        break;
      case 2:
        a[0] = c * ar - s * br; a[1] = c * ai - s * bi; b[0] = s * ar + c * br; b[1] = s * ai + c * bi;
        break;
      default:
        a[0] = ar * c - ai * s; a[1] = ar * s + ai * c; b[0] = br * c + bi * s; b[1] = -br * s + bi * c;
        break;
    }
  };
  for (const Step& st : p.steps) {
    if (st.kind == 1) {
      const csim_gate& g = st.g;
      double c = 0, s = 0;
      if (g.op == OP_RY) { c = std::cos(g.angle / 2); s = std::sin(g.angle / 2); }
      if (g.op == OP_ZPHASE) { c = std::cos(g.angle); s = std::sin(g.angle); }
      const uint64_t tb = 1ull << g.target;
      for (uint64_t i = 0; i < N; ++i)
        if (!(i & tb) && (i & g.cmask) == g.cval) pair(&(*cur)[2 * i], &(*cur)[2 * (i | tb)], g.op, c, s);
      continue;
    }
    const bool gather = st.nseg > 0;
    std::vector<double>& dst = gather ? *nxt : *cur;
    const uint32_t nchunks = (uint32_t)(N >> 2);
    for (uint32_t tile = 0; tile < (nchunks >> 5); ++tile) {
      double v[32][4][2];
      for (uint32_t lane = 0; lane < 32; ++lane) {
        const uint32_t ci = (tile << 5) | lane;
        uint32_t src = ci;
        for (int k = 0; k < st.nseg; ++k) {
          const PermSeg& g = p.segs[st.seg_off + k];
          std::vector<BitRun> runs(g.runs, g.runs + g.nruns);
          const uint32_t key = extract(src, runs);
          const uint32_t val = p.lut[g.lut_off + key];
          src = (src & ~g.supmask) | deposit(val, runs);
        }
        for (int j = 0; j < 4; ++j) {
          v[lane][j][0] = (*cur)[2 * (((size_t)src << 2) + j)];
          v[lane][j][1] = (*cur)[2 * (((size_t)src << 2) + j) + 1];
        }
      }
      for (int k = 0; k < st.nops; ++k) {
        const LocalOp& o = p.ops[st.op_off + k];
        if (o.op == 4) {
          const MuxDesc& md = p.mux[o.cm];
          std::vector<BitRun> runs(md.runs, md.runs + md.nruns);
          for (uint32_t lane = 0; lane < 32; ++lane) {
            const uint32_t ci = (tile << 5) | lane;
            const uint2 bk = p.mtab[md.tab_off + extract(ci, runs)];
            for (uint32_t e = bk.x; e < bk.x + bk.y; ++e) {
              const MuxEntry& E = p.ment[e];
              if ((ci & E.cm) != E.cv) continue;
              for (int j0 = 0; j0 < 4; ++j0) {
                if (j0 & (1 << md.target)) continue;
                if (((uint32_t)j0 & E.lm) != E.lv) continue;
                pair(v[lane][j0], v[lane][j0 | (1 << md.target)], 2, E.cd, E.sd);
              }
            }
          }
          continue;
        }
        if (o.op == 5) {
          const ReflectDesc& rd = p.refl[o.cm];
          double S[32][4][2];
          for (uint32_t lane = 0; lane < 32; ++lane)
            for (int y = 0; y < 4; ++y) {
              S[lane][y][0] = S[lane][y][1] = 0.0;
              for (uint32_t l2 = 0; l2 < 32; ++l2)
                if (((lane ^ l2) & ~rd.lanemask & 31u) == 0) {
                  S[lane][y][0] += v[l2][y][0];
                  S[lane][y][1] += v[l2][y][1];
                }
            }
          for (uint32_t lane = 0; lane < 32; ++lane) {
            double o4[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
            for (int y = 0; y < 4; ++y)
              for (int yp = 0; yp < 4; ++yp) {
                const int q = y * 4 + yp;
                if ((rd.nzA >> q) & 1u) {
                  o4[y][0] += rd.ad[q].x * v[lane][yp][0] - rd.ad[q].y * v[lane][yp][1];
                  o4[y][1] += rd.ad[q].x * v[lane][yp][1] + rd.ad[q].y * v[lane][yp][0];
                }
                if ((rd.nzB >> q) & 1u) {
                  o4[y][0] += rd.bd[q].x * S[lane][yp][0] - rd.bd[q].y * S[lane][yp][1];
                  o4[y][1] += rd.bd[q].x * S[lane][yp][1] + rd.bd[q].y * S[lane][yp][0];
                }
              }
            for (int y = 0; y < 4; ++y) {
              v[lane][y][0] = o4[y][0];
              v[lane][y][1] = o4[y][1];
            }
          }
          continue;
        }
        if (o.target < 2) {
          for (uint32_t lane = 0; lane < 32; ++lane) {
            const uint32_t ci = (tile << 5) | lane;
            if ((ci & o.cm) != o.cv) continue;
            for (int j0 = 0; j0 < 4; ++j0) {
              if (j0 & (1 << o.target)) continue;
              if (((uint32_t)j0 & o.lm) != o.lv) continue;
              pair(v[lane][j0], v[lane][j0 | (1 << o.target)], o.op, o.cd, o.sd);
            }
          }
        } else {
          const uint32_t lm = 1u << (o.target - 2);
          for (uint32_t lane = 0; lane < 32; ++lane) {
            if (lane & lm) continue;
            const uint32_t ci = (tile << 5) | lane;
            if ((ci & o.cm) != o.cv) continue;
            for (int j = 0; j < 4; ++j)
              if (((uint32_t)j & o.lm) == o.lv) pair(v[lane][j], v[lane | lm][j], o.op, o.cd, o.sd);
          }
        }
      }
      for (uint32_t lane = 0; lane < 32; ++lane) {
        const uint32_t ci = (tile << 5) | lane;
        for (int j = 0; j < 4; ++j) {
          dst[2 * (((size_t)ci << 2) + j)] = v[lane][j][0];
          dst[2 * (((size_t)ci << 2) + j) + 1] = v[lane][j][1];
        }
      }
    }
    if (gather) std::swap(cur, nxt);
  }
  if (cur != amps) *amps = *cur;
}

}  // namespace csim
