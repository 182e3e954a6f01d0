// The fuser: groups consecutive elementary gates into sweeps, each one HBM pass.
//
// A sweep combines a permutation and tile-local gates:
//  * permutation: a maximal run of multi-controlled X gates whose target is a
//    qubit >= 2 and whose controls avoid qubits 0-1.  Such a run maps every
//    4-amplitude chunk (qubits 0-1) to another chunk.  The run is cut into
//    segments whose support (chunk-index bits read or written) has at most
//    kMaxSupport bits; each segment becomes a lookup table over its support.
//  * tile-local gates: any gate whose target is one of the 7 lowest qubits
//    (the 128-amplitude warp tile); controls may sit anywhere.  Runs of RY
//    gates on the same in-thread qubit (0 or 1) commute and become
//    multiplexed rotations (a few chunk-index bits select a bucket of
//    candidate gates, each checked in full).  A window of gates acting only
//    inside the tile whose 128 x 128 matrix is I (x) A + J (x) B over lane
//    bits becomes one averaging block (a warp reduction).
// Gather form: [permutation as a gather][tile gates].  Scatter form: [tile
// gates][permutation as a scatter].  A gate fitting neither class (e.g. H on
// a high qubit) becomes its own single-gate step.  Sweeps whose descriptors
// exceed the kernel parameter block are split.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "fuse.h"

namespace csim {

namespace {

// Key bits of a permutation or multiplexer table (CSIM_KEY_BITS overrides):
// wider keys mean fewer chained lookups but tables that spill out of L1.
int max_key_bits() {
  static const int v = [] {
    const char* e = std::getenv("CSIM_KEY_BITS");
    const int k = e ? std::atoi(e) : 0;
    return (k >= 8 && k <= 16) ? k : 14;
  }();
  return v;
}
// Key bits of a multiplexer bucket table (CSIM_MUX_KEY_BITS overrides).  The
// bucket word is prefetched before the permutation chain, so a table that
// lives in L2 rather than L1 costs little, while a wider key leaves fewer
// lanes with candidate lists (warp-divergent loops).
int mux_key_bits() {
  static const int v = [] {
    const char* e = std::getenv("CSIM_MUX_KEY_BITS");
    const int k = e ? std::atoi(e) : 0;
    return (k >= 8 && k <= 18) ? k : 16;
  }();
  return v;
}
constexpr int kMuxMinGates = 4;   // shorter RY runs stay individual gates

// Tiles over which the tile-order model counts shared 128-byte lines
// (CSIM_ORDER_WINDOW overrides; a power of two).
uint32_t order_window() {
  static const uint32_t v = [] {
    const char* e = std::getenv("CSIM_ORDER_WINDOW");
    const long k = e ? std::atol(e) : 0;
    return (k >= 64 && k <= 65536 && (k & (k - 1)) == 0) ? (uint32_t)k : 256u;
  }();
  return v;
}

// A permutation run followed by its inverse becomes one in-place sweep
// (CSIM_CONJUGATE=0 disables).
bool conjugation_enabled() {
  static const bool v = [] {
    const char* e = std::getenv("CSIM_CONJUGATE");
    return !(e && e[0] == '0');
  }();
  return v;
}

// Sibling-aware tile order for gather sweeps (CSIM_TILE_ORDER=0 disables).
bool tile_order_enabled() {
  static const bool v = [] {
    const char* e = std::getenv("CSIM_TILE_ORDER");
    return !(e && e[0] == '0');
  }();
  return v;
}

// Fast tile bits of the in-place conjugated sweeps, replacing the model's
// choice (CSIM_CONJ_FAST_BITS="b0,b1,..."; tile-index bits, most useful
// first).  Empty when unset.
const std::vector<int>& conj_fast_override() {
  static const std::vector<int> v = [] {
    std::vector<int> r;
    const char* e = std::getenv("CSIM_CONJ_FAST_BITS");
    if (!e) return r;
    for (const char* q = e; *q;) {
      char* end = nullptr;
      const long b = std::strtol(q, &end, 10);
      if (end == q) break;
      if (b >= 0 && b < 32 && (int)r.size() < kMaxFast) r.push_back((int)b);
      q = (*end == ',') ? end + 1 : end;
    }
    return r;
  }();
  return v;
}

// High qubits a sweep may stage in registers (CSIM_STAGE=0..3; default 3):
// gates on up to this many qubits above the warp tile join the sweep, which
// then runs 2^k tiles per warp iteration.
int stage_limit() {
  static const int v = [] {
    const char* e = std::getenv("CSIM_STAGE");
    const int k = e ? std::atoi(e) : kMaxStage;
    return (k >= 0 && k <= kMaxStage) ? k : kMaxStage;
  }();
  return v;
}

bool perm_eligible(const csim_gate& g) {
  return g.op == OP_X && g.target >= 2 && (g.cmask & 3ull) == 0;
}
// Tile-local: any gate on state bits 0-6, and a diagonal phase on any qubit
// (it needs no partner amplitude, only the index bit).
bool local_eligible(const csim_gate& g) { return g.target <= 6 || g.op == OP_ZPHASE; }

// Whether the permutation gate p (an X with controls) commutes with the
// tile-local gate l, so that p can move ahead of l inside one sweep: p must
// not flip a qubit l reads or acts on, and l must not change a qubit p reads
// (a diagonal l changes none).
bool commutes(const csim_gate& p, const csim_gate& l) {
  const uint64_t supp_l = l.cmask | (1ull << l.target);
  if ((supp_l >> p.target) & 1ull) return false;
  if (l.op == OP_ZPHASE) return true;
  return ((p.cmask >> l.target) & 1ull) == 0;
}

// Cover the set bits of `mask` with at most two windows of total width <=
// limit (one window when it fits).  Returns false if impossible.
bool cover2(uint32_t mask, int limit, KeyWin* w) {
  *w = KeyWin{0, 0, 0, 0};
  if (!mask) return true;
  const int lo = __builtin_ctz(mask), hi = 31 - __builtin_clz(mask);
  if (hi - lo + 1 <= limit) {
    *w = KeyWin{(uint8_t)lo, (uint8_t)(hi - lo + 1), 0, 0};
    return true;
  }
  // split at the largest gap between consecutive set bits
  int best_gap = 0, cut = -1, prev = lo;
  for (int b = lo + 1; b <= hi; ++b) {
    if (!((mask >> b) & 1u)) continue;
    if (b - prev - 1 > best_gap) {
      best_gap = b - prev - 1;
      cut = prev;
    }
    prev = b;
  }
  if (cut < 0) return false;
  int next = cut + 1;
  while (!((mask >> next) & 1u)) ++next;
  const int w0 = cut - lo + 1, w1 = hi - next + 1;
  if (w0 + w1 > limit) return false;
  *w = KeyWin{(uint8_t)lo, (uint8_t)w0, (uint8_t)next, (uint8_t)w1};
  return true;
}

uint32_t win_mask(const KeyWin& w) {
  return (((1u << w.w0) - 1u) << w.lo0) | (((1u << w.w1) - 1u) << w.lo1);
}
uint32_t win_key(uint32_t x, const KeyWin& w) {
  return ((x >> w.lo0) & ((1u << w.w0) - 1u)) | (((x >> w.lo1) & ((1u << w.w1) - 1u)) << w.w0);
}
uint32_t win_put(uint32_t x, uint32_t v, const KeyWin& w) {
  const uint32_t m0 = (1u << w.w0) - 1u, m1 = (1u << w.w1) - 1u;
  x &= ~((m0 << w.lo0) | (m1 << w.lo1));
  return x | ((v & m0) << w.lo0) | (((v >> w.w0) & m1) << w.lo1);
}

struct ChunkGate {
  uint32_t m, v, t;
};

ChunkGate chunk_gate(const csim_gate& g) {
  return {(uint32_t)(g.cmask >> 2), (uint32_t)(g.cval >> 2), 1u << (g.target - 2)};
}

// One permutation step before table compilation.
struct PermItem {
  bool add = false;       // controlled +-1 on a contiguous register
  uint32_t m = 0, v = 0;  // controls
  uint32_t t = 0;         // gate: target bit mask
  int base = 0, width = 0, neg = 0;
};

// Recognise controlled increment / decrement cascades of a contiguous
// register: gates X(r[j] | C, r[0..j-1] all 1 (or all 0)) for j = w-1..0.
// Off by default (CSIM_PERM_ADD=1 enables): measured slower than tables on
// the QSVT circuit because the arithmetic steps cost more issue slots than the
// table lookups they replace.
bool recognise_adds() {
  static const bool v = [] {
    const char* e = std::getenv("CSIM_PERM_ADD");
    return e && e[0] == '1';
  }();
  return v;
}

std::vector<PermItem> perm_items(const std::vector<csim_gate>& run) {
  std::vector<PermItem> out;
  size_t i = 0;
  while (i < run.size()) {
    if (!recognise_adds()) {
      const ChunkGate g = chunk_gate(run[i++]);
      PermItem it;
      it.m = g.m;
      it.v = g.v;
      it.t = g.t;
      out.push_back(it);
      continue;
    }
    const ChunkGate g0 = chunk_gate(run[i]);
    uint32_t ctl = g0.m, val = g0.v;
    std::vector<int> tgts = {__builtin_ctz(g0.t)};
    int sense = -1;  // 1: INC (controls 1), 0: DEC (controls 0)
    size_t j = i + 1;
    while (j < run.size()) {
      const ChunkGate g = chunk_gate(run[j]);
      const uint32_t tb = g.t;
      if (!(ctl & tb)) break;
      const int bv = (val & tb) ? 1 : 0;
      if (sense >= 0 && bv != sense) break;
      if (g.m != (ctl & ~tb) || g.v != (val & ~tb)) break;
      sense = bv;
      ctl = g.m;
      val = g.v;
      tgts.push_back(__builtin_ctz(tb));
      ++j;
    }
    // register bits r[0..w-1] are the targets in reverse order; need contiguous
    const int w = (int)tgts.size();
    bool ok = w >= 2;
    for (int k = 0; ok && k < w; ++k) ok = tgts[w - 1 - k] == tgts[w - 1] + k;
    if (ok) {
      PermItem it;
      it.add = true;
      it.m = ctl;
      it.v = val;
      it.base = tgts[w - 1];
      it.width = w;
      it.neg = sense == 0 ? 1 : 0;
      out.push_back(it);
      i = j;
      continue;
    }
    PermItem it;
    it.m = g0.m;
    it.v = g0.v;
    it.t = g0.t;
    out.push_back(it);
    ++i;
  }
  return out;
}

// Compiled steps of a run of X gates.  forward: time order, each step mapping
// an index to its image (scatter).  Otherwise reverse order with inverted
// steps, each mapping an index to its preimage (gather).
std::vector<PermSeg> compile_perm(const std::vector<csim_gate>& run, bool forward, Program* p) {
  std::vector<PermSeg> out;
  std::vector<PermItem> items = perm_items(run);
  if (!forward) {
    std::reverse(items.begin(), items.end());
    for (PermItem& it : items) it.neg ^= (int)it.add;
  }
  size_t i = 0;
  while (i < items.size()) {
    if (items[i].add) {
      PermSeg ps{};
      ps.kind = 2;
      ps.base = (uint8_t)items[i].base;
      ps.width = (uint8_t)items[i].width;
      ps.neg = (uint8_t)items[i].neg;
      ps.m = items[i].m;
      ps.v = items[i].v;
      out.push_back(ps);
      p->stats.segments++;
      ++i;
      continue;
    }
    std::vector<ChunkGate> seg;
    uint32_t sup = 0;
    KeyWin win{};
    while (i < items.size() && !items[i].add) {
      const uint32_t ns = sup | items[i].m | items[i].t;
      KeyWin nw;
      if (!cover2(ns, max_key_bits(), &nw)) break;
      sup = ns;
      win = nw;
      seg.push_back(ChunkGate{items[i].m, items[i].v, items[i].t});
      ++i;
    }
    if (seg.empty()) {  // this gate alone exceeds a table key: apply it directly
      PermSeg ps{};
      ps.kind = 1;
      ps.m = items[i].m;
      ps.v = items[i].v;
      ps.t = items[i].t;
      out.push_back(ps);
      p->stats.segments++;
      ++i;
      continue;
    }
    if (seg.size() == 1) {  // a single gate is cheaper applied directly
      PermSeg ps{};
      ps.kind = 1;
      ps.m = seg[0].m;
      ps.v = seg[0].v;
      ps.t = seg[0].t;
      out.push_back(ps);
      p->stats.segments++;
      continue;
    }
    const int w = win.w0 + win.w1;
    PermSeg ps{};
    ps.kind = 0;
    ps.win = win;
    std::string key(reinterpret_cast<const char*>(&win), sizeof(win));
    key.append(reinterpret_cast<const char*>(seg.data()), seg.size() * sizeof(ChunkGate));
    const auto hit = p->lut_cache.find(key);
    if (hit != p->lut_cache.end()) {
      ps.t = hit->second;
    } else {
      ps.t = (uint32_t)p->lut.size();
      p->lut_cache.emplace(std::move(key), ps.t);
      for (uint32_t k = 0; k < (1u << w); ++k) {
        uint32_t x = win_put(0u, k, win);
        for (const ChunkGate& cg : seg)
          if ((x & cg.m) == cg.v) x ^= cg.t;
        p->lut.push_back((uint16_t)win_key(x, win));
      }
    }
    out.push_back(ps);
    p->stats.segments++;
    p->stats.max_support = std::max<int64_t>(p->stats.max_support, w);
  }
  p->stats.perm_gates += (int64_t)run.size();
  return out;
}

LocalOp local_op(const csim_gate& g) {
  LocalOp o{};
  o.cm = (uint32_t)(g.cmask >> 2);
  o.cv = (uint32_t)(g.cval >> 2);
  o.lm = (uint8_t)(g.cmask & 3ull);
  o.lv = (uint8_t)(g.cval & 3ull);
  o.op = g.op;
  o.target = g.target;
  if (g.op == OP_ZPHASE && g.target >= 7) {
    o.op = 6;
    o.target = (uint8_t)(g.target - 2);
  }
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

// A tile-local op before it is placed into a sweep's parameter block.
struct OpItem {
  LocalOp op;
  MuxDesc mux;
  ReflectDesc refl;
  int mux_id = -1;  // index into Program::mux_descs (op 4)
};

// Order-free content of a multiplexer's gates, angles optionally negated.
std::string mux_signature(const std::vector<csim_gate>& grp, bool negate) {
  std::vector<std::array<uint64_t, 4>> v;
  for (const csim_gate& g : grp) {
    double a = negate ? -g.angle : g.angle;
    if (a == 0.0) a = 0.0;  // one zero
    uint64_t ab;
    std::memcpy(&ab, &a, sizeof(ab));
    v.push_back({(uint64_t)g.target, g.cmask, g.cval, ab});
  }
  std::sort(v.begin(), v.end());
  return std::string(reinterpret_cast<const char*>(v.data()), v.size() * sizeof(v[0]));
}

OpItem out_item_of(const Program* p, uint32_t mux_index) {
  OpItem it{};
  it.mux_id = (int)mux_index;
  it.mux = p->mux_descs[mux_index];
  it.op.op = 4;
  it.op.target = it.mux.target;
  return it;
}

void compile_mux_group(const std::vector<csim_gate>& grp, Program* p, std::vector<OpItem>* out) {
  std::string ckey(reinterpret_cast<const char*>(grp.data()), grp.size() * sizeof(csim_gate));
  const auto hit = p->mux_cache.find(ckey);
  if (hit != p->mux_cache.end()) {
    OpItem it = out_item_of(p, hit->second);
    out->push_back(it);
    p->stats.mux++;
    p->stats.mux_gates += (int64_t)grp.size();
    return;
  }
  // key windows: grow by the chunk bits constrained by the most gates
  int freq[32] = {0};
  for (const csim_gate& g : grp) {
    const uint32_t m = (uint32_t)(g.cmask >> 2);
    for (int b = 0; b < 32; ++b) freq[b] += (m >> b) & 1u;
  }
  std::vector<int> order;
  for (int b = 0; b < 32; ++b)
    if (freq[b] > 0) order.push_back(b);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return freq[a] > freq[b]; });
  uint32_t keybits = 0;
  KeyWin win{};
  for (int b : order) {
    KeyWin nw;
    if (cover2(keybits | (1u << b), mux_key_bits(), &nw)) {
      keybits |= 1u << b;
      win = nw;
    }
  }
  const uint32_t wmask = win_mask(win);
  const int w = win.w0 + win.w1;
  std::vector<std::vector<int>> bucket((size_t)1 << w);
  for (size_t gi = 0; gi < grp.size(); ++gi) {
    const uint32_t m = (uint32_t)(grp[gi].cmask >> 2) & wmask;
    const uint32_t v = (uint32_t)(grp[gi].cval >> 2) & wmask;
    const uint32_t fm = win_key(m, win), fv = win_key(v, win);
    for (uint32_t key = 0; key < (1u << w); ++key)
      if ((key & fm) == fv) bucket[key].push_back((int)gi);
  }
  OpItem it{};
  it.mux.win = win;
  it.mux.tab_off = (uint32_t)p->mtab.size();
  it.mux.target = grp[0].target;
  it.mux.lm = (uint8_t)(grp[0].cmask & 3ull);
  it.mux.lv = (uint8_t)(grp[0].cval & 3ull);
  for (uint32_t key = 0; key < (1u << w); ++key) {
    const std::vector<int>& bk = bucket[key];
    if (bk.empty()) {
      p->mtab.push_back(0u);
      continue;
    }
    bool pure = true;
    for (int gi : bk) pure = pure && (((uint32_t)(grp[gi].cmask >> 2) & ~wmask) == 0);
    if (pure) {
      double th = 0.0;
      for (int gi : bk) th += grp[gi].angle;
      p->angd.push_back(make_double2(std::cos(th / 2.0), std::sin(th / 2.0)));
      p->angf.push_back(make_float2((float)std::cos(th / 2.0), (float)std::sin(th / 2.0)));
      p->mtab.push_back(0x80000000u | (uint32_t)(p->angd.size() - 1));
      p->stats.max_bucket = std::max<int64_t>(p->stats.max_bucket, 1);
      continue;
    }
    if (bk.size() > 255 || p->mentf.size() >= (1u << 23)) {
      std::fprintf(stderr, "csim fuser: multiplexer bucket overflow\n");
      std::abort();
    }
    p->mtab.push_back(((uint32_t)p->mentf.size() << 8) | (uint32_t)bk.size());
    p->stats.max_bucket = std::max<int64_t>(p->stats.max_bucket, (int64_t)bk.size());
    for (int gi : bk) {
      const LocalOp o = local_op(grp[gi]);
      p->mentf.push_back(MuxEntryF{o.cm, o.cv, o.cf, o.sf});
      p->mentd.push_back(MuxEntryD{o.cm, o.cv, 0u, 0u, o.cd, o.sd});
    }
  }
  it.op.op = 4;
  it.op.target = grp[0].target;
  const uint32_t id = (uint32_t)p->mux_descs.size();
  it.mux_id = (int)id;
  p->mux_cache.emplace(std::move(ckey), id);
  p->mux_descs.push_back(it.mux);
  p->mux_inv.push_back(-1);
  p->mux_sig.emplace(mux_signature(grp, false), id);
  const auto inv = p->mux_sig.find(mux_signature(grp, true));
  if (inv != p->mux_sig.end() && inv->second != id) {
    const MuxDesc& o = p->mux_descs[inv->second];
    if (o.target == it.mux.target && o.lm == it.mux.lm && o.lv == it.mux.lv) {
      p->mux_inv[id] = (int)inv->second;
      p->mux_inv[inv->second] = (int)id;
    }
  }
  out->push_back(it);
  p->stats.mux++;
  p->stats.mux_gates += (int64_t)grp.size();
  p->stats.mux_entries = (int64_t)p->mentf.size();
  if (const char* dbg = std::getenv("CSIM_FUSE_STATS")) {
    if (dbg[0] == '2' && p->n >= 12) {
      // warp view: the candidate loop runs max-over-lanes iterations
      uint64_t rs = 0x9e3779b97f4a7c15ull;
      double loops = 0, warps_looping = 0, lanes_cand = 0;
      const int samples = 4096;
      const uint32_t tmask = (p->n - 7 >= 32) ? 0xffffffffu : ((1u << (p->n - 7)) - 1u);
      for (int k = 0; k < samples; ++k) {
        rs ^= rs << 13;
        rs ^= rs >> 7;
        rs ^= rs << 17;
        const uint32_t tile = (uint32_t)rs & tmask;
        uint32_t mx = 0;
        for (uint32_t lane = 0; lane < 32; ++lane) {
          const uint32_t w = p->mtab[it.mux.tab_off + win_key((tile << 5) | lane, win)];
          if (w != 0u && !(w & 0x80000000u)) {
            mx = std::max(mx, w & 255u);
            lanes_cand += 1;
          }
        }
        loops += mx;
        warps_looping += mx > 0;
      }
      std::fprintf(stderr,
                   "[csim fuse] mux %zu: key bits %d, lanes with candidates %.2f%%, warps looping "
                   "%.1f%%, mean warp trip count %.2f\n",
                   p->mux_descs.size() - 1, w, 100.0 * lanes_cand / (32.0 * samples),
                   100.0 * warps_looping / samples, loops / samples);
    }
  }
}

// RY gates on one in-thread qubit commute: split the run by its controls on
// state bits 0-1 and multiplex each part.
void compile_mux(const std::vector<csim_gate>& grp, Program* p, std::vector<OpItem>* out) {
  std::vector<std::vector<csim_gate>> parts;
  std::vector<uint32_t> keys;
  for (const csim_gate& g : grp) {
    const uint32_t k = (uint32_t)((g.cmask & 3ull) | ((g.cval & 3ull) << 2));
    size_t j = 0;
    while (j < keys.size() && keys[j] != k) ++j;
    if (j == keys.size()) {
      keys.push_back(k);
      parts.emplace_back();
    }
    parts[j].push_back(g);
  }
  for (const auto& part : parts) compile_mux_group(part, p, out);
}

using cplx = std::complex<double>;

bool in_tile(const csim_gate& g) { return g.target <= 6 && (g.cmask >> 7) == 0; }

// Dense 128 x 128 matrix (column by column) of a window of tile-only gates.
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
        const cplx a0 = v[x], a1 = v[x | tb];
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

// If the window's matrix is I (x) A + J (x) B over the lane bits in `lanes`,
// fill the descriptor and return true.
bool reflect_form(const std::vector<cplx>& U, uint32_t lanes, ReflectDesc* d) {
  auto at = [&](int row, int col) { return U[(size_t)col * 128 + row]; };
  const int cls = 1 << __builtin_popcount(lanes);
  int l1 = 0;
  for (int b = 0; b < 5; ++b)
    if ((lanes >> b) & 1u) {
      l1 = 1 << b;
      break;
    }
  cplx A[4][4], B[4][4];
  for (int y = 0; y < 4; ++y)
    for (int yp = 0; yp < 4; ++yp) {
      B[y][yp] = at(y, (l1 << 2) | yp) * (double)cls;
      A[y][yp] = at(y, yp) - B[y][yp] / (double)cls;
    }
  for (int l = 0; l < 32; ++l)
    for (int lp = 0; lp < 32; ++lp) {
      const bool same_class = ((l ^ lp) & ~lanes & 31) == 0;
      for (int y = 0; y < 4; ++y)
        for (int yp = 0; yp < 4; ++yp) {
          const cplx model =
              (l == lp ? A[y][yp] : 0.0) + (same_class ? B[y][yp] / (double)cls : 0.0);
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

bool is_lane_h(const csim_gate& g) { return g.op == OP_H && g.target >= 2 && g.cmask == 0; }

// Longest window starting at i (an H on a lane bit) with the averaging form.
size_t try_reflect(const std::vector<csim_gate>& run, size_t i, Program* p,
                   std::vector<OpItem>* out) {
  if (!is_lane_h(run[i])) return 0;
  size_t end = i;
  while (end < run.size() && in_tile(run[end])) ++end;
  for (size_t j = end; j > i + 1; --j) {
    if (!is_lane_h(run[j - 1])) continue;
    uint32_t lanes = 0;
    for (size_t k = i; k < j; ++k)
      if (run[k].op == OP_H && run[k].target >= 2) lanes |= 1u << (run[k].target - 2);
    OpItem it{};
    if (!reflect_form(tile_matrix(run, i, j), lanes, &it.refl)) continue;
    it.op.op = 5;
    out->push_back(it);
    p->stats.reflect++;
    return j - i;
  }
  return 0;
}

std::vector<OpItem> compile_local(const std::vector<csim_gate>& run, Program* p) {
  std::vector<OpItem> out;
  size_t i = 0;
  while (i < run.size()) {
    if (const size_t w = try_reflect(run, i, p, &out)) {
      i += w;
      continue;
    }
    const csim_gate& g = run[i];
    if (g.op == OP_RY && g.target < 2) {
      size_t j = i;
      while (j < run.size() && run[j].op == OP_RY && run[j].target == g.target) ++j;
      if ((int)(j - i) >= kMuxMinGates) {
        compile_mux(std::vector<csim_gate>(run.begin() + i, run.begin() + j), p, &out);
        i = j;
        continue;
      }
    }
    // uncontrolled H gates on distinct lane bits: one Walsh-Hadamard op
    if (g.op == OP_H && g.target >= 2 && g.target < 7 && g.cmask == 0) {
      uint32_t lanes = 0;
      size_t j = i;
      while (j < run.size() && run[j].op == OP_H && run[j].target >= 2 && run[j].target < 7 &&
             run[j].cmask == 0 && !((lanes >> (run[j].target - 2)) & 1u)) {
        lanes |= 1u << (run[j].target - 2);
        ++j;
      }
      if (j - i >= 2) {
        OpItem it{};
        it.op.op = 8;
        it.op.cm = lanes;
        const double sc = std::ldexp(1.0, -(int)(j - i) / 2) *
                          (((j - i) & 1) ? 0.70710678118654752440 : 1.0);
        it.op.cd = sc;
        it.op.cf = (float)sc;
        out.push_back(it);
        p->stats.wht++;
        i = j;
        continue;
      }
    }
    OpItem it{};
    it.op = local_op(g);
    out.push_back(it);
    ++i;
  }
  p->stats.local_gates += (int64_t)run.size();
  return out;
}

// Split an op list into chunks that fit one parameter block.
std::vector<std::vector<OpItem>> chunk_ops(const std::vector<OpItem>& ops) {
  std::vector<std::vector<OpItem>> out;
  std::vector<OpItem> cur;
  int nmux = 0, nrefl = 0;
  for (const OpItem& it : ops) {
    const bool m = it.op.op == 4, r = it.op.op == 5;
    if ((int)cur.size() + 1 > kMaxOps || (m && nmux + 1 > kMaxMux) || (r && nrefl + 1 > kMaxRefl)) {
      out.push_back(cur);
      cur.clear();
      nmux = nrefl = 0;
    }
    cur.push_back(it);
    nmux += m;
    nrefl += r;
  }
  if (!cur.empty()) out.push_back(cur);
  return out;
}

void emit_sweep(Program* p, const std::vector<PermSeg>& segs, const std::vector<OpItem>& ops) {
  SweepParams sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.scatter = p->scatter ? 1 : 0;
  sp.nseg = (int)segs.size();
  for (size_t k = 0; k < segs.size(); ++k) sp.segs[k] = segs[k];
  int nmux = 0, nrefl = 0;
  int last_mux = -1;  // the sweep's latest multiplexer (op 4), by mux_descs index
  for (const OpItem& it : ops) {
    LocalOp o = it.op;
    if (o.op == 4 && it.mux_id >= 0 && last_mux >= 0 && p->mux_inv[(size_t)it.mux_id] == last_mux) {
      // the inverse of the latest multiplexer: the kernel reuses its rotation
      o.op = 7;
      o.target = it.mux.target;
      o.lm = it.mux.lm;
      o.lv = it.mux.lv;
      o.cm = o.cv = 0;
      last_mux = -1;
      p->stats.mux_inverse++;
    } else if (o.op == 4) {
      sp.mux[nmux] = it.mux;
      o.cm = (uint32_t)nmux++;
      last_mux = it.mux_id;
    } else if (o.op == 5) {
      sp.refl[nrefl] = it.refl;
      o.cm = (uint32_t)nrefl++;
    }
    sp.ops[sp.nops++] = o;
  }
  sp.nmux = nmux;
  Step st;
  st.kind = 0;
  st.param = (int)p->params.size();
  st.gather = !segs.empty();
  p->params.push_back(sp);
  p->steps.push_back(st);
  p->stats.sweeps++;
}

uint32_t emu_permute(const Program& p, const SweepParams& sp, uint32_t x);

// Fraction of DRAM lines fetched per line used by a gather sweep when the
// tiles of `win` consecutive counters (deposited through the fast bits `fb`)
// are in flight together: distinct 128-byte source lines x 4 chunks over the
// chunks read.  Measured reads of the sweep kernel match a window of about 256
// tiles (the L2 does not keep a line much longer).
double line_fetch_ratio(const Program& p, const SweepParams& sp, const std::vector<int>& fb,
                        int tb, uint32_t win, int nwin) {
  uint32_t fm = 0;
  for (int b : fb) fm |= 1u << b;
  const uint32_t ntiles = 1u << tb;
  std::vector<uint32_t> lines;
  lines.reserve((size_t)win * 32);
  double used = 0, fetched = 0;
  for (int w = 0; w < nwin; ++w) {
    uint32_t c0 = (uint32_t)(((uint64_t)(2 * w + 1) * 0x9E3779B1u) % ntiles);
    c0 -= c0 % win;
    lines.clear();
    for (uint32_t c = c0; c < c0 + win; ++c) {
      uint32_t t = 0;
      for (size_t j = 0; j < fb.size(); ++j) t |= ((c >> j) & 1u) << fb[j];
      uint32_t hv = c >> fb.size();
      for (int b = 0; b < 32 && hv; ++b) {
        if ((fm >> b) & 1u) continue;
        t |= (hv & 1u) << b;
        hv >>= 1;
      }
      for (uint32_t l = 0; l < 32; ++l) lines.push_back(emu_permute(p, sp, (t << 5) | l) >> 2);
    }
    std::sort(lines.begin(), lines.end());
    fetched += 4.0 * (double)(std::unique(lines.begin(), lines.end()) - lines.begin());
    used += 32.0 * win;
  }
  return fetched / used;
}

// Fast tile bits for one gather sweep (kernel side: the lowest tile-counter
// bits go to these tile bits).  A lane of destination chunk x reads the
// source chunk y = P^-1(x); the other three 32-byte chunks of y's 128-byte
// line are read by destinations P(y ^ j), j = 1..3.  Candidates are the tile
// bits in which those destinations differ from x (sampled from the gate run,
// bits seen in >= 2% of the pairs); greedy selection then keeps each candidate
// that lowers line_fetch_ratio over a 256-tile window.  States that fit in L2
// (n < 24) keep the natural order.
void choose_fast_bits(const std::vector<csim_gate>& perm, const Program& p, const SweepParams& sp,
                      uint8_t* fast, int* nfast) {
  *nfast = 0;
  const int n = p.n;
  const int tb = n - 7;
  if (perm.empty() || n < 24) return;
  std::vector<ChunkGate> cg;
  cg.reserve(perm.size());
  for (const csim_gate& g : perm) cg.push_back(chunk_gate(g));
  const uint32_t nch_mask = (n - 2 >= 32) ? 0xffffffffu : ((1u << (n - 2)) - 1u);
  auto fwd = [&](uint32_t x) {
    for (const ChunkGate& g : cg)
      if ((x & g.m) == g.v) x ^= g.t;
    return x;
  };
  auto inv = [&](uint32_t x) {
    for (size_t k = cg.size(); k-- > 0;)
      if ((x & cg[k].m) == cg[k].v) x ^= cg[k].t;
    return x;
  };
  std::vector<double> w(tb, 0.0);
  int npairs = 0;
  uint64_t rs = 0x9e3779b97f4a7c15ull;  // fixed-seed xorshift: deterministic programs
  for (int s = 0; s < 1024; ++s) {
    rs ^= rs << 13;
    rs ^= rs >> 7;
    rs ^= rs << 17;
    const uint32_t x = (uint32_t)rs & nch_mask;
    const uint32_t y = inv(x);
    for (uint32_t j = 1; j < 4; ++j) {
      const uint32_t d = (fwd(y ^ j) ^ x) >> 5;
      ++npairs;
      for (int b = 0; b < tb; ++b)
        if ((d >> b) & 1u) w[b] += 1.0;
    }
  }
  std::vector<int> cand;
  for (int b = 0; b < tb; ++b)
    if (w[b] >= 0.02 * npairs) cand.push_back(b);
  std::sort(cand.begin(), cand.end(), [&](int x, int y) { return w[x] > w[y]; });
  if (cand.size() > 12) cand.resize(12);
  if (const char* dbg = std::getenv("CSIM_FUSE_STATS")) {
    if (dbg[0] == '2') {
      std::string cs;
      for (int b : cand) cs += std::to_string(b) + ":" + std::to_string(w[b] / npairs).substr(0, 5) + " ";
      std::fprintf(stderr, "[csim fuse] tile-order candidates %s\n", cs.c_str());
    }
  }
  const uint32_t win = std::min<uint32_t>(order_window(), 1u << (tb - 1));
  std::vector<int> fb;
  double cur = line_fetch_ratio(p, sp, fb, tb, win, 2);
  while ((int)fb.size() < kMaxFast) {
    int best = -1;
    double bv = cur - 0.005;
    for (int b : cand) {
      if (std::find(fb.begin(), fb.end(), b) != fb.end()) continue;
      std::vector<int> t = fb;
      t.push_back(b);
      const double v = line_fetch_ratio(p, sp, t, tb, win, 2);
      if (v < bv) {
        bv = v;
        best = b;
      }
    }
    if (best < 0) break;
    fb.push_back(best);
    cur = bv;
  }
  for (int b : fb) fast[(*nfast)++] = (uint8_t)b;
}

// Place one [permutation run, tile-local run] group into sweeps.
// Emit one [permutation run, tile-local run] group.  With conj (gather form),
// the group is followed by the inverse permutation, which the caller drops:
// when the group fits one sweep it becomes one in-place sweep that gathers
// through P^-1, applies the ops and stores back to the gathered addresses
// (P^-1 . ops . P); returns whether it did.
bool emit_group(Program* p, const std::vector<csim_gate>& perm, const std::vector<csim_gate>& local,
                bool conj = false, const std::vector<int>& stage = {}) {
  const std::vector<PermSeg> segs = compile_perm(perm, p->scatter, p);
  const size_t first_param = p->params.size();
  std::vector<std::vector<PermSeg>> sc;
  for (size_t k = 0; k < segs.size(); k += kMaxSeg)
    sc.emplace_back(segs.begin() + k, segs.begin() + std::min(segs.size(), k + kMaxSeg));
  std::vector<OpItem> ops = compile_local(local, p);
  // gates on staged qubits (above the tile, not diagonal): ops 9-11 on the
  // qubit's index in `stage`
  for (OpItem& it : ops) {
    LocalOp& o = it.op;
    if (o.op > 2 || o.target < 7) continue;
    const auto f = std::find(stage.begin(), stage.end(), (int)o.target);
    o.op = (uint8_t)(9 + o.op);
    o.target = (uint8_t)(f - stage.begin());
    p->stats.staged_gates++;
  }
  std::vector<std::vector<OpItem>> oc = chunk_ops(ops);
  conj = conj && !p->scatter && sc.size() == 1 && oc.size() <= 1;
  if (conj) {
    emit_sweep(p, sc[0], oc.empty() ? std::vector<OpItem>() : oc[0]);
    p->steps.back().inplace = true;
    p->params.back().inplace = 1;
    p->stats.conjugated++;
  } else if (!p->scatter) {
    // gather: segment chunks are in evaluation (reverse time) order, so the
    // last chunk holds the earliest gates and runs first
    for (size_t k = sc.size(); k > 1; --k) emit_sweep(p, sc[k - 1], {});
    emit_sweep(p, sc.empty() ? std::vector<PermSeg>() : sc[0],
               oc.empty() ? std::vector<OpItem>() : oc[0]);
    for (size_t k = 1; k < oc.size(); ++k) emit_sweep(p, {}, oc[k]);
  } else {
    // scatter: ops first (in place), the last op chunk with the first segments
    for (size_t k = 0; k + 1 < oc.size(); ++k) emit_sweep(p, {}, oc[k]);
    emit_sweep(p, sc.empty() ? std::vector<PermSeg>() : sc[0],
               oc.empty() ? std::vector<OpItem>() : oc.back());
    for (size_t k = 1; k < sc.size(); ++k) emit_sweep(p, sc[k], {});
  }
  if (!stage.empty()) {
    // every sweep of the group stages the same qubits: they are its first
    // fast tile bits, and the gather's own order (below) follows them
    for (size_t k = first_param; k < p->params.size(); ++k) {
      SweepParams& sp = p->params[k];
      sp.nstage = (int)stage.size();
      sp.nfast = 0;
      for (int q : stage) sp.fast[sp.nfast++] = (uint8_t)(q - 7);
      p->stats.staged_sweeps++;
    }
  }
  if (p->scatter || !tile_order_enabled()) return conj;
  for (size_t k = first_param; k < p->params.size(); ++k) {
    SweepParams& sp = p->params[k];
    if (sp.nseg == 0) continue;  // in place: no gather, natural order
    std::string key(reinterpret_cast<const char*>(sp.segs), sp.nseg * sizeof(PermSeg));
    auto hit = p->order_cache.find(key);
    if (hit == p->order_cache.end()) {
      uint8_t fast[kMaxFast] = {0};
      int nfast = 0;
      choose_fast_bits(perm, *p, sp, fast, &nfast);
      hit = p->order_cache.emplace(std::move(key), std::string(reinterpret_cast<char*>(fast), nfast))
                .first;
    }
    if (sp.nstage > 0) {
      // staged qubits first, then the gather's fast bits that are not staged
      for (char b : hit->second) {
        if (sp.nfast >= kMaxFast) break;
        bool dup = false;
        for (int j = 0; j < sp.nstage; ++j) dup = dup || sp.fast[j] == (uint8_t)b;
        if (!dup) sp.fast[sp.nfast++] = (uint8_t)b;
      }
      continue;
    }
    sp.nfast = (int)hit->second.size();
    std::memcpy(sp.fast, hit->second.data(), hit->second.size());
    if (sp.inplace && !conj_fast_override().empty()) {
      const std::vector<int>& ov = conj_fast_override();
      sp.nfast = 0;
      for (int b : ov)
        if (b < p->n - 7) sp.fast[sp.nfast++] = (uint8_t)b;
    }
    if (const char* dbg = std::getenv("CSIM_FUSE_STATS")) {
      if (dbg[0] == '2' && p->n >= 24) {
        std::vector<int> fb(sp.fast, sp.fast + sp.nfast), none;
        std::string bits;
        for (int b : fb) bits += std::to_string(b) + " ";
        std::fprintf(stderr, "[csim fuse] sweep %zu tile order: fast bits %s; line ratio %.3f (natural %.3f)\n",
                     p->params.size() - 1, bits.c_str(),
                     line_fetch_ratio(*p, sp, fb, p->n - 7, order_window(), 2),
                     line_fetch_ratio(*p, sp, none, p->n - 7, order_window(), 2));
      }
    }
  }
  return conj;
}

}  // namespace

void pair_op(double* a, double* b, int op, double c, double s);  // host executor (below)

// Fused steps of one run of gates, appended to the program.
void build_segment(const std::vector<csim_gate>& gates, Program* p) {
  const int n = p->n;
  std::vector<csim_gate> perm, local;
  std::vector<int> stage;  // staged qubits of the open group
  const int kstage = (n - 7 >= 1) ? std::min(p->stage_k, n - 7) : 0;
  bool open = false;
  const double sweep_cost = std::ldexp(1.0, n);
  // groups and lone gates in circuit order; emitted after the scan so that a
  // group can see whether the next one undoes its permutation
  struct Item {
    bool group = false;
    std::vector<csim_gate> perm, local;
    std::vector<int> stage;
    csim_gate g{};
  };
  std::vector<Item> items;
  auto single = [&](const csim_gate& g) {
    Item it;
    it.g = g;
    items.push_back(std::move(it));
  };
  auto close = [&]() {
    if (!open) return;
    Item it;
    it.group = true;
    it.perm = perm;
    it.local = local;
    it.stage = stage;
    items.push_back(std::move(it));
    perm.clear();
    local.clear();
    stage.clear();
    open = false;
  };
  // a non-diagonal gate above the tile joins the group as a staged-qubit gate
  // when its target is staged already or a staging slot is free (gather
  // form).  A permutation gate that cannot join the gather starts the next
  // group's gather instead unless the group stages qubits already: that keeps
  // the permutation runs of the QSVT circuit whole, so that a run and its
  // inverse still meet in one conjugated sweep.
  auto stageable = [&](const csim_gate& g) {
    if (p->scatter || g.target < 7 || g.op == OP_ZPHASE) return false;
    if (perm_eligible(g) && stage.empty()) return false;
    return std::find(stage.begin(), stage.end(), (int)g.target) != stage.end() ||
           (int)stage.size() < kstage;
  };
  auto add_staged = [&](const csim_gate& g) {
    if (std::find(stage.begin(), stage.end(), (int)g.target) == stage.end())
      stage.push_back((int)g.target);
    local.push_back(g);
  };
  auto commutes_all = [&](const csim_gate& g) {
    for (const csim_gate& l : local)
      if (!commutes(g, l)) return false;
    return true;
  };
  for (const csim_gate& g : gates) {
    const bool pe = perm_eligible(g), le = local_eligible(g);
    if (!p->scatter) {  // gather form: [perm][local]
      if (open && pe && (local.empty() || commutes_all(g))) {
        perm.push_back(g);
        continue;
      }
      if (open && le) {
        local.push_back(g);
        continue;
      }
      if (open && stageable(g)) {
        add_staged(g);
        continue;
      }
    } else {  // scatter form: [local][perm]
      if (open && perm.empty() && le) {
        local.push_back(g);
        continue;
      }
      if (open && pe) {
        perm.push_back(g);
        continue;
      }
    }
    close();
    if (pe || le) {
      open = true;
      if (!p->scatter)
        (pe ? perm : local).push_back(g);
      else
        (le ? local : perm).push_back(g);
    } else if (stageable(g)) {
      open = true;
      add_staged(g);
    } else {
      single(g);
    }
  }
  close();
  auto emit_single = [&](const csim_gate& g) {
    Step s;
    s.kind = 1;
    s.g = g;
    p->steps.push_back(s);
    p->stats.single++;
  };
  auto reversed_equal = [](const std::vector<csim_gate>& a, const std::vector<csim_gate>& b) {
    if (a.size() != b.size()) return false;
    for (size_t i = 0; i < a.size(); ++i)
      if (std::memcmp(&a[i], &b[b.size() - 1 - i], sizeof(csim_gate)) != 0) return false;
    return true;
  };
  for (size_t k = 0; k < items.size(); ++k) {
    Item& it = items[k];
    if (!it.group) {
      emit_single(it.g);
      continue;
    }
    // a group whose gates change fewer amplitudes in total than one sweep
    // moves (e.g. a few multi-controlled X) runs cheaper as single gates
    double cost = 0.0;
    for (const csim_gate& g : it.perm) cost += gate_amp_updates(g, n);
    for (const csim_gate& g : it.local) cost += gate_amp_updates(g, n);
    if (cost < sweep_cost) {
      for (const csim_gate& g : it.perm) emit_single(g);
      for (const csim_gate& g : it.local) emit_single(g);
      continue;
    }
    // P^-1, ops, P (every multi-controlled X is its own inverse): one in-place sweep
    const bool conj = conjugation_enabled() && !p->scatter && !it.perm.empty() &&
                      k + 1 < items.size() && items[k + 1].group &&
                      reversed_equal(it.perm, items[k + 1].perm);
    if (emit_group(p, it.perm, it.local, conj, it.stage) && conj) items[k + 1].perm.clear();
  }
}

// Dense blocks (CSIM_DENSE=0 disables them; CSIM_DENSE_MIN sets the least
// number of gates a block must hold, default 10).
bool dense_enabled() {
  static const bool v = [] {
    const char* e = std::getenv("CSIM_DENSE");
    return !(e && e[0] == '0');
  }();
  return v;
}
// CSIM_DENSE=2 also turns runs that stay inside the warp tile into dense
// blocks (for measurements: the sweep fuser applies those without a pass
// of their own).
bool dense_inside_tile() {
  static const bool v = [] {
    const char* e = std::getenv("CSIM_DENSE");
    return e && e[0] == '2';
  }();
  return v;
}
// A run earns a pass of its own only when it mixes amplitudes across the
// warp tile: an H or RY on a qubit above it.  Tile gates, phases and
// multi-controlled X (the gather's permutations) the sweeps apply for free.
bool run_leaves_tile(const std::vector<csim_gate>& run, bool force) {
  if (force) return true;
  for (const csim_gate& g : run)
    if (g.target >= 7 && (g.op == OP_H || g.op == OP_RY)) return true;
  return false;
}
int dense_min_gates() {
  static const int v = [] {
    const char* e = std::getenv("CSIM_DENSE_MIN");
    const int k = e ? std::atoi(e) : 10;
    return k >= 2 ? k : 10;
  }();
  return v;
}
int dense_engine_default() {
  const char* e = std::getenv("CSIM_DENSE_ENGINE");
  return (e && std::strcmp(e, "fp32") == 0) ? DENSE_FP32 : DENSE_TC;
}

uint64_t gate_support(const csim_gate& g) { return g.cmask | (1ull << g.target); }

// The 2^k x 2^k unitary of a run of gates on the qubits q[0..k-1] (the run
// touches no other qubit; local bit j is qubit q[j]), composed column by
// column in FP64.  M[r][c] is at 2 * (dim * r + c).
std::vector<double> compose_run(const std::vector<csim_gate>& run, const std::vector<int>& q) {
  const int k = (int)q.size();
  const uint32_t dim = 1u << k;
  auto local = [&](uint64_t mask) {
    uint32_t m = 0;
    for (int j = 0; j < k; ++j)
      if ((mask >> q[j]) & 1ull) m |= 1u << j;
    return m;
  };
  std::vector<double> M(2 * (size_t)dim * dim, 0.0);
  for (uint32_t c = 0; c < dim; ++c) M[2 * (dim * c + c)] = 1.0;
  for (const csim_gate& g : run) {
    int t = 0;
    while (q[t] != g.target) ++t;
    const uint32_t cm = local(g.cmask), cv = local(g.cval), tb = 1u << t;
    double c = 0.0, sn = 0.0;
    if (g.op == OP_RY) {
      c = std::cos(g.angle / 2.0);
      sn = std::sin(g.angle / 2.0);
    } else if (g.op == OP_ZPHASE) {
      c = std::cos(g.angle);
      sn = std::sin(g.angle);
    }
    for (uint32_t col = 0; col < dim; ++col)
      for (uint32_t r = 0; r < dim; ++r) {
        if ((r & tb) || (r & cm) != cv) continue;
        pair_op(&M[2 * (dim * r + col)], &M[2 * (dim * (r | tb) + col)], g.op, c, sn);
      }
  }
  return M;
}

std::vector<int> bits_of(uint64_t m) {
  std::vector<int> v;
  for (int b = 0; b < 64; ++b)
    if ((m >> b) & 1ull) v.push_back(b);
  return v;
}

void push_dense(DenseBlock&& b, size_t ngates, Program* p) {
  make_dense_block(&b);
  Step st;
  st.kind = 2;
  st.param = (int)p->dense.size();
  p->dense.push_back(std::move(b));
  p->steps.push_back(st);
  p->stats.dense_blocks++;
  p->stats.dense_gates += (int64_t)ngates;
}

// A run on at most five qubits: one 32 x 32 block (padded with other qubits
// when it touches fewer).
void emit_dense(const std::vector<csim_gate>& run, uint64_t support, Program* p) {
  DenseBlock b;
  int j = 0;
  for (int bit = 0; bit < p->n && j < 5; ++bit)
    if ((support >> bit) & 1ull) b.q[j++] = (uint8_t)bit;
  for (int bit = 0; j < 5; ++bit)  // fewer than five qubits: pad with others
    if (!((support >> bit) & 1ull)) {
      b.q[j++] = (uint8_t)bit;
      support |= 1ull << bit;
    }
  std::sort(b.q, b.q + 5);
  b.u = compose_run(run, std::vector<int>(b.q, b.q + 5));
  push_dense(std::move(b), run.size(), p);
}

// A run on six or seven qubits whose matrix never mixes the values of one or
// two of them (the selectors): one 32 x 32 block per selector value on the
// other five.  Returns false when no such pair or single qubit exists.
bool emit_dense_selected(const std::vector<csim_gate>& run, uint64_t support, Program* p) {
  const std::vector<int> q = bits_of(support);
  const int k = (int)q.size(), nsel = k - 5;
  if (nsel < 1 || nsel > 2) return false;
  const std::vector<double> M = compose_run(run, q);
  const uint32_t dim = 1u << k;
  for (int a = 0; a < k; ++a)
    for (int b2 = (nsel == 2 ? a + 1 : a); b2 < (nsel == 2 ? k : a + 1); ++b2) {
      const uint32_t smask = (1u << a) | (1u << b2);
      bool diag = true;  // no entry between different selector values
      for (uint32_t r = 0; r < dim && diag; ++r)
        for (uint32_t c = 0; c < dim; ++c) {
          if (((r ^ c) & smask) == 0) continue;
          if (std::abs(M[2 * (dim * r + c)]) + std::abs(M[2 * (dim * r + c) + 1]) > 1e-13) {
            diag = false;
            break;
          }
        }
      if (!diag) continue;
      DenseBlock blk;
      std::vector<int> rest;  // local indices of the five block qubits
      for (int j = 0; j < k; ++j)
        if (!((smask >> j) & 1u)) rest.push_back(j);
      for (int j = 0; j < 5; ++j) blk.q[j] = (uint8_t)q[rest[j]];
      blk.nsel = (uint8_t)nsel;
      blk.sel[0] = (uint8_t)q[a];
      if (nsel == 2) blk.sel[1] = (uint8_t)q[b2];
      blk.u.assign((size_t)(2 << nsel) * 1024, 0.0);
      for (int y = 0; y < (1 << nsel); ++y) {
        uint32_t ybits = (y & 1) ? (1u << a) : 0u;
        if (nsel == 2 && (y & 2)) ybits |= 1u << b2;
        for (uint32_t r = 0; r < 32; ++r)
          for (uint32_t c = 0; c < 32; ++c) {
            uint32_t R = ybits, Cc = ybits;
            for (int j = 0; j < 5; ++j) {
              R |= ((r >> j) & 1u) << rest[j];
              Cc |= ((c >> j) & 1u) << rest[j];
            }
            double* dst = blk.u.data() + (size_t)y * 2048 + 2 * (32 * r + c);
            dst[0] = M[2 * (dim * R + Cc)];
            dst[1] = M[2 * (dim * R + Cc) + 1];
          }
      }
      push_dense(std::move(blk), run.size(), p);
      return true;
    }
  return false;
}

void build_program(const std::vector<csim_gate>& gates, int n, csim_exec mode, Program* p,
                   bool allow_dense, int stage_k, int dense_mode) {
  *p = Program();
  p->n = n;
  p->mode = mode;
  p->stage_k = (stage_k >= 0 && stage_k <= kMaxStage) ? stage_k : stage_limit();
  const char* form = std::getenv("CSIM_SWEEP_FORM");
  p->scatter = form && std::strcmp(form, "scatter") == 0;
  p->dense_engine = dense_engine_default();
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
    p->pass_amps = p->amp_updates;
    return;
  }
  // dense_mode: -1 the switches (CSIM_DENSE), 0 off, 1 runs that leave the
  // tile, 2 runs inside the tile too
  const bool dense_wanted = dense_mode < 0 ? dense_enabled() : dense_mode > 0;
  const bool force_tile = dense_mode < 0 ? dense_inside_tile() : dense_mode == 2;
  p->dense_on = allow_dense && dense_wanted && n >= 12 && !p->scatter;
  if (p->dense_on) {
    // runs of consecutive gates on at most five qubits (targets and
    // controls), or on six or seven of which one or two only select the
    // matrix; the long ones become dense blocks, the rest go to the sweep
    // fuser in order
    std::vector<csim_gate> pending;
    size_t i = 0;
    const size_t N = gates.size();
    while (i < N) {
      uint64_t sup = 0, sup5 = 0;
      size_t j = i, p5 = i;  // the run is gates[i, j); gates[i, p5) stay on <= 5 qubits
      while (j < N && __builtin_popcountll(sup | gate_support(gates[j])) <= 7) {
        sup |= gate_support(gates[j]);
        ++j;
        if (__builtin_popcountll(sup) <= 5) {
          p5 = j;
          sup5 = sup;
        }
      }
      const std::vector<csim_gate> run(gates.begin() + i, gates.begin() + j);
      const int minimum = dense_min_gates();
      auto flush = [&]() {
        if (!pending.empty()) build_segment(pending, p);
        pending.clear();
      };
      const bool leaves = run_leaves_tile(run, force_tile);
      if ((int)run.size() >= minimum && leaves && __builtin_popcountll(sup) <= 5) {
        flush();
        emit_dense(run, sup, p);
        i = j;
        continue;
      }
      if ((int)run.size() >= minimum && leaves) {
        // try the selector form without disturbing the program when it fails
        Program trial;
        trial.n = p->n;
        if (emit_dense_selected(run, sup, &trial)) {
          flush();
          emit_dense_selected(run, sup, p);
          i = j;
          continue;
        }
      }
      if ((int)(p5 - i) >= minimum &&
          run_leaves_tile(std::vector<csim_gate>(gates.begin() + i, gates.begin() + p5),
                          force_tile)) {
        flush();
        emit_dense(std::vector<csim_gate>(gates.begin() + i, gates.begin() + p5), sup5, p);
        i = p5;  // the rest of the run is scanned again
        continue;
      }
      pending.push_back(gates[i]);
      ++i;
    }
    if (!pending.empty()) build_segment(pending, p);
  } else {
    build_segment(gates, p);
  }
  p->passes = (int64_t)p->steps.size();
  for (const Step& s : p->steps)
    p->pass_amps += s.kind != 1 ? std::ldexp(1.0, n) : gate_amp_updates(s.g, n);
  for (const Step& s : p->steps)
    if (s.kind == 0 && s.gather && !s.inplace) p->pingpong = true;
  p->stats.lut_entries = (int64_t)p->lut.size();
  if (std::getenv("CSIM_FUSE_STATS")) {
    const FuseStats& f = p->stats;
    std::fprintf(stderr,
                 "[csim fuse] n=%d form=%s sweeps=%lld single=%lld perm_gates=%lld segments=%lld "
                 "max_support=%lld lut=%lld local=%lld mux=%lld mux_gates=%lld entries=%lld "
                 "max_bucket=%lld reflect=%lld\n",
                 n, p->scatter ? "scatter" : "gather", (long long)f.sweeps, (long long)f.single,
                 (long long)f.perm_gates, (long long)f.segments, (long long)f.max_support,
                 (long long)f.lut_entries, (long long)f.local_gates, (long long)f.mux,
                 (long long)f.mux_gates, (long long)f.mux_entries, (long long)f.max_bucket,
                 (long long)f.reflect);
    if (std::getenv("CSIM_FUSE_STATS")[0] == '2') {
      // one line per fused sweep: segments by kind, then the local ops
      for (size_t k = 0; k < p->steps.size(); ++k) {
        const Step& st = p->steps[k];
        if (st.kind == 2) {
          const DenseBlock& b = p->dense[(size_t)st.param];
          std::fprintf(stderr, "[csim fuse] step %zu: dense block on qubits %d %d %d %d %d\n", k,
                       b.q[0], b.q[1], b.q[2], b.q[3], b.q[4]);
          continue;
        }
        if (st.kind != 0) {
          std::fprintf(stderr, "[csim fuse] step %zu: single gate op %d target %d\n", k,
                       (int)st.g.op, (int)st.g.target);
          continue;
        }
        const SweepParams& sp = p->params[(size_t)st.param];
        std::string segs, ops;
        for (int i = 0; i < sp.nseg; ++i) segs += "TGI"[sp.segs[i].kind];
        for (int i = 0; i < sp.nops; ++i) {
          ops += "XHRZMAPIW"[sp.ops[i].op];
          if (sp.ops[i].op < 4 || sp.ops[i].op == 6)
            ops += std::to_string(sp.ops[i].target) + "/" + std::to_string(sp.ops[i].cm) + ":" +
                   std::to_string(sp.ops[i].lm) + " ";
        }
        std::fprintf(stderr, "[csim fuse] step %zu: segs %s ops %s mux %d\n", k, segs.c_str(),
                     ops.c_str(), sp.nmux);
        for (int r = 0; r < sp.nops; ++r) {
          if (sp.ops[r].op != 5) continue;
          const ReflectDesc& rd = sp.refl[sp.ops[r].cm];
          std::string av;
          for (int y = 0; y < 4; ++y) {
            const int q = y * 5;
            char buf[160];
            std::snprintf(buf, sizeof(buf), " y%d A=(%.4f,%.4f) B=(%.4f,%.4f)", y, rd.ad[q].x,
                          rd.ad[q].y, rd.bd[q].x, rd.bd[q].y);
            av += buf;
          }
          std::fprintf(stderr, "[csim fuse]   block lanes %u nzA %x nzB %x%s\n", rd.lanemask, rd.nzA,
                       rd.nzB, av.c_str());
        }
      }
    }
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
  cudaError_t e = up(&p->d_lut, p->lut, st);
  if (e == cudaSuccess) e = up(&p->d_mtab, p->mtab, st);
  if (e == cudaSuccess) e = up(&p->d_mentf, p->mentf, st);
  if (e == cudaSuccess) e = up(&p->d_mentd, p->mentd, st);
  if (e == cudaSuccess) e = up(&p->d_angf, p->angf, st);
  if (e == cudaSuccess) e = up(&p->d_angd, p->angd, st);
  for (DenseBlock& b : p->dense)
    if (e == cudaSuccess) e = upload_dense(&b, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_program(p);
    return e;
  }
  for (SweepParams& sp : p->params) {
    sp.lut = p->d_lut;
    sp.mtab = p->d_mtab;
    sp.mentf = p->d_mentf;
    sp.mentd = p->d_mentd;
    sp.angf = p->d_angf;
    sp.angd = p->d_angd;
  }
  p->uploaded = true;
  return cudaSuccess;
}

namespace {
bool src_index_enabled() {
  static const bool v = [] {
    const char* e = std::getenv("CSIM_SRC_INDEX");
    return !(e && e[0] == '0');
  }();
  return v;
}
// Source indices loaded one loop iteration ahead (CSIM_SRC_PREFETCH=0 disables).
bool src_prefetch_enabled() {
  static const bool v = [] {
    const char* e = std::getenv("CSIM_SRC_PREFETCH");
    return !(e && e[0] == '0');
  }();
  return v;
}
std::string chain_key(const SweepParams& sp) {
  std::string k;
  for (int i = 0; i < sp.nseg; ++i) {
    const PermSeg& g = sp.segs[i];
    const uint32_t w[8] = {g.win.lo0, g.win.w0, g.win.lo1, g.win.w1,
                           (uint32_t)g.kind | (uint32_t)g.base << 8 | (uint32_t)g.width << 16 |
                               (uint32_t)g.neg << 24,
                           g.m, g.v, g.t};
    k.append(reinterpret_cast<const char*>(w), sizeof(w));
  }
  return k;
}
}  // namespace

int plan_src_index(Program* p, int max_tables) {
  if (!p->src_planned) {
    p->src_planned = true;
    p->src_tab.assign(p->params.size(), -1);
    p->src_first.clear();
    if (src_index_enabled() && p->n >= 7) {
      std::unordered_map<std::string, int> tab_of_key;
      for (const Step& s : p->steps) {
        if (s.kind != 0 || !s.gather) continue;  // sweeps that move data, in either form
        const SweepParams& sp = p->params[(size_t)s.param];
        if (sp.nseg == 0) continue;
        auto it = tab_of_key.emplace(chain_key(sp), (int)p->src_first.size());
        if (it.second) p->src_first.push_back(s.param);
        p->src_tab[(size_t)s.param] = it.first->second;
      }
    }
  }
  const int ntab = (int)p->src_first.size();
  return ntab <= max_tables ? ntab : 0;
}

cudaError_t launch_src_tables(const Program& p, uint32_t* const* tables, cudaStream_t st) {
  for (size_t t = 0; t < p.src_first.size(); ++t) {
    const cudaError_t e = launch_perm_index(tables[t], p.n, p.params[(size_t)p.src_first[t]], st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t build_src_index(Program* p, cudaStream_t st, int max_tables) {
  if (p->src_tried || !p->uploaded) return cudaSuccess;
  p->src_tried = true;
  const int ntab = plan_src_index(p, max_tables);
  if (ntab == 0) return cudaSuccess;
  const uint64_t bytes = 1ull << p->n;  // 2^(n-2) chunks x 4 bytes
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return cudaSuccess;
  }
  if ((uint64_t)ntab * bytes > fr / 4) return cudaSuccess;
  std::vector<uint32_t*> tabs((size_t)ntab, nullptr);
  cudaError_t e = cudaSuccess;
  for (int t = 0; t < ntab && e == cudaSuccess; ++t) e = cudaMalloc((void**)&tabs[(size_t)t], bytes);
  if (e == cudaSuccess) e = launch_src_tables(*p, tabs.data(), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    for (uint32_t* q : tabs)
      if (q) cudaFree(q);
    return e;
  }
  for (size_t k = 0; k < p->params.size(); ++k)
    if (p->src_tab[k] >= 0) {
      p->params[k].src = tabs[(size_t)p->src_tab[k]];
      p->params[k].src_prefetch = src_prefetch_enabled() ? 1 : 0;
    }
  p->d_src = tabs;
  return cudaSuccess;
}

void free_program(Program* p) {
  void* ptrs[] = {p->d_lut, p->d_mtab, p->d_mentf, p->d_mentd, p->d_angf, p->d_angd};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (uint32_t* q : p->d_src)
    if (q) cudaFree(q);
  p->d_src.clear();
  for (DenseBlock& b : p->dense) free_dense(&b);
  p->src_tried = false;
  for (SweepParams& sp : p->params) {
    sp.src = nullptr;
    sp.src_prefetch = 0;
  }
  p->d_lut = nullptr;
  p->d_mtab = nullptr;
  p->d_mentf = nullptr;
  p->d_mentd = nullptr;
  p->d_angf = nullptr;
  p->d_angd = nullptr;
  p->uploaded = false;
}

cudaError_t run_program(const Program& p, void* buf[2], int* cur, int prec, cudaStream_t st,
                        const uint32_t* const* src_tables) {
  return run_program_steps(p, buf, cur, prec, st, 0, (int64_t)p.steps.size(), src_tables);
}

bool program_fuses_norm(const Program& p, int prec) {
  if (p.steps.empty()) return false;
  const Step& s = p.steps.back();
  return s.kind == 0 && sweep_fuses_norm(prec, p.n, p.params[(size_t)s.param]);
}

cudaError_t run_program_steps(const Program& p, void* buf[2], int* cur, int prec, cudaStream_t st,
                              int64_t first, int64_t last, const uint32_t* const* src_tables,
                              const uint32_t* zero_map, int zero_steps, double* norm_part) {
  const int64_t final_step = (int64_t)p.steps.size() - 1;
  for (int64_t k = first; k < last; ++k) {
    const Step& s = p.steps[(size_t)k];
    cudaError_t e;
    if (k == final_step && norm_part && program_fuses_norm(p, prec)) {
      // the last sweep, summing |a|^2 of the state it writes
      SweepParams a = p.params[(size_t)s.param];
      if (s.gather && src_tables && (size_t)s.param < p.src_tab.size() &&
          p.src_tab[(size_t)s.param] >= 0) {
        a.src = src_tables[p.src_tab[(size_t)s.param]];
        a.src_prefetch = src_prefetch_enabled() ? 1 : 0;
      }
      a.norm_part = norm_part;
      void* out = s.gather && !s.inplace ? buf[1 - *cur] : buf[*cur];
      e = launch_sweep(buf[*cur], out, prec, p.n, a, st);
      if (s.gather && !s.inplace) *cur = 1 - *cur;
      if (e != cudaSuccess) return e;
      continue;
    }
    if (s.kind == 1) {
      e = launch_gate(buf[*cur], prec, p.n, s.g, st);
    } else if (s.kind == 2) {
      e = prec == CSIM_C64 ? launch_dense(buf[*cur], p.n, p.dense[(size_t)s.param], p.dense_engine, st)
                           : cudaErrorInvalidValue;
    } else if (!s.gather) {
      if (k == 0 && zero_map && zero_steps >= 1) {
        SweepParams a = p.params[(size_t)s.param];
        a.zero_map = zero_map;
        a.zero_mode = zero_steps == 2 ? 2 : 1;
        e = launch_sweep(buf[*cur], buf[*cur], prec, p.n, a, st);
      } else {
        e = launch_sweep(buf[*cur], buf[*cur], prec, p.n, p.params[s.param], st);
      }
    } else {
      void* out = s.inplace ? buf[*cur] : buf[1 - *cur];
      SweepParams a = p.params[(size_t)s.param];
      if (src_tables && (size_t)s.param < p.src_tab.size() && p.src_tab[(size_t)s.param] >= 0) {
        a.src = src_tables[p.src_tab[(size_t)s.param]];
        a.src_prefetch = src_prefetch_enabled() ? 1 : 0;
      }
      if (k == 1 && zero_map && zero_steps == 2) {
        a.zero_map = zero_map;
        a.zero_mode = 3;
      }
      e = launch_sweep(buf[*cur], out, prec, p.n, a, st);
      if (!s.inplace) *cur = 1 - *cur;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------ host executor
void pair_op(double* a, double* b, int op, double c, double s) {
  const double h = 0.70710678118654752440;
  const double ar = a[0], ai = a[1], br = b[0], bi = b[1];
  switch (op) {
    case 0: a[0] = br; a[1] = bi; b[0] = ar; b[1] = ai; break;
    case 1: a[0] = (ar + br) * h; a[1] = (ai + bi) * h; b[0] = (ar - br) * h; b[1] = (ai - bi) * h; break;
    case 2: a[0] = c * ar - s * br; a[1] = c * ai - s * bi; b[0] = s * ar + c * br; b[1] = s * ai + c * bi; break;
    default: a[0] = ar * c - ai * s; a[1] = ar * s + ai * c; b[0] = br * c + bi * s; b[1] = -br * s + bi * c; break;
  }
}

namespace {

uint32_t emu_permute(const Program& p, const SweepParams& sp, uint32_t x) {
  for (int k = 0; k < sp.nseg; ++k) {
    const PermSeg& g = sp.segs[k];
    if (g.kind == 1) {
      if ((x & g.m) == g.v) x ^= g.t;
    } else if (g.kind == 2) {
      if ((x & g.m) == g.v) {
        const uint32_t rm = (1u << g.width) - 1u;
        const uint32_t r = (((x >> g.base) & rm) + (g.neg ? rm : 1u)) & rm;
        x = (x & ~(rm << g.base)) | (r << g.base);
      }
    } else {
      x = win_put(x, p.lut[g.t + win_key(x, g.win)], g.win);
    }
  }
  return x;
}

// Ops [k0, k1) of a sweep on one tile.  mc / ms: the latest multiplexer's
// rotation per lane (op 7 inverts it), carried across calls.
void emu_ops(const Program& p, const SweepParams& sp, uint32_t tile, double (&v)[32][4][2],
             int k0, int k1, double (&mc)[32], double (&ms)[32]) {
  auto rot_all = [&](uint32_t lane, int target, uint32_t lm, uint32_t lv, double c, double s) {
    for (int j0 = 0; j0 < 4; ++j0) {
      if (j0 & (1 << target)) continue;
      if (((uint32_t)j0 & lm) != lv) continue;
      pair_op(v[lane][j0], v[lane][j0 | (1 << target)], 2, c, s);
    }
  };
  for (int k = k0; k < k1; ++k) {
    const LocalOp& o = sp.ops[k];
    if (o.op == 4) {
      const MuxDesc& md = sp.mux[o.cm];
      for (uint32_t lane = 0; lane < 32; ++lane) {
        const uint32_t ci = (tile << 5) | lane;
        const uint32_t word = p.mtab[md.tab_off + win_key(ci, md.win)];
        double c = 1.0, s = 0.0;
        if (word & 0x80000000u) {
          const double2 cs = p.angd[word & 0x7fffffffu];
          c = cs.x;
          s = cs.y;
        } else if (word != 0u) {
          for (uint32_t e = word >> 8; e < (word >> 8) + (word & 255u); ++e) {
            const MuxEntryD& E = p.mentd[e];
            if ((ci & E.cm) == E.cv) {
              const double nc = c * E.c - s * E.s;
              s = s * E.c + c * E.s;
              c = nc;
            }
          }
        }
        mc[lane] = c;
        ms[lane] = s;
        if (word != 0u) rot_all(lane, md.target, md.lm, md.lv, c, s);
      }
      continue;
    }
    if (o.op == 7) {
      for (uint32_t lane = 0; lane < 32; ++lane)
        rot_all(lane, o.target, o.lm, o.lv, mc[lane], -ms[lane]);
      continue;
    }
    if (o.op == 8) {  // H on every lane bit of o.cm, then one scale
      for (int b = 0; b < 5; ++b) {
        if (!((o.cm >> b) & 1u)) continue;
        for (uint32_t lane = 0; lane < 32; ++lane) {
          if (lane & (1u << b)) continue;
          const uint32_t hi = lane | (1u << b);
          for (int y = 0; y < 4; ++y)
            for (int r = 0; r < 2; ++r) {
              const double x0 = v[lane][y][r], x1 = v[hi][y][r];
              v[lane][y][r] = x0 + x1;
              v[hi][y][r] = x0 - x1;
            }
        }
      }
      for (uint32_t lane = 0; lane < 32; ++lane)
        for (int y = 0; y < 4; ++y)
          for (int r = 0; r < 2; ++r) v[lane][y][r] *= o.cd;
      continue;
    }
    if (o.op == 5) {
      const ReflectDesc& rd = sp.refl[o.cm];
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
    if (o.op == 6) {  // e^{i phi Z} on chunk bit o.target
      for (uint32_t lane = 0; lane < 32; ++lane) {
        const uint32_t ci = (tile << 5) | lane;
        if ((ci & o.cm) != o.cv) continue;
        const double sg = ((ci >> o.target) & 1u) ? -o.sd : o.sd;
        for (int j = 0; j < 4; ++j) {
          if (((uint32_t)j & o.lm) != o.lv) continue;
          const double re = v[lane][j][0], im = v[lane][j][1];
          v[lane][j][0] = re * o.cd - im * sg;
          v[lane][j][1] = re * sg + im * o.cd;
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
          pair_op(v[lane][j0], v[lane][j0 | (1 << o.target)], o.op, o.cd, o.sd);
        }
      }
    } else {
      const uint32_t lm = 1u << (o.target - 2);
      for (uint32_t lane = 0; lane < 32; ++lane) {
        if (lane & lm) continue;
        const uint32_t ci = (tile << 5) | lane;
        if ((ci & o.cm) != o.cv) continue;
        for (int j = 0; j < 4; ++j)
          if (((uint32_t)j & o.lm) == o.lv) pair_op(v[lane][j], v[lane | lm][j], o.op, o.cd, o.sd);
      }
    }
  }
}

}  // namespace

void emulate_program(const Program& p, std::vector<double>* amps) {
  const size_t N = (size_t)1 << p.n;
  std::vector<double> other(2 * N);
  std::vector<double>* cur = amps;
  std::vector<double>* nxt = &other;
  for (const Step& st : p.steps) {
    if (st.kind == 2) {  // y = U x on every group of the block's qubits, FP64
      const DenseBlock& b = p.dense[(size_t)st.param];
      uint64_t qm = 0;
      for (int j = 0; j < 5; ++j) qm |= 1ull << b.q[j];
      std::vector<double> x(64), y(64);
      for (uint64_t i = 0; i < N; ++i) {
        if (i & qm) continue;
        int ysel = 0;  // the matrix the selector bits of this group pick
        for (int j = 0; j < b.nsel; ++j) ysel |= (int)((i >> b.sel[j]) & 1ull) << j;
        const double* um = b.u.data() + (size_t)ysel * 2048;
        auto at = [&](int e) {
          uint64_t a = i;
          for (int j = 0; j < 5; ++j)
            if ((e >> j) & 1) a |= 1ull << b.q[j];
          return a;
        };
        for (int e = 0; e < 32; ++e) {
          x[2 * e] = (*cur)[2 * at(e)];
          x[2 * e + 1] = (*cur)[2 * at(e) + 1];
        }
        for (int r = 0; r < 32; ++r) {
          double re = 0.0, im = 0.0;
          for (int c = 0; c < 32; ++c) {
            const double ur = um[2 * (32 * r + c)], ui = um[2 * (32 * r + c) + 1];
            re += ur * x[2 * c] - ui * x[2 * c + 1];
            im += ur * x[2 * c + 1] + ui * x[2 * c];
          }
          y[2 * r] = re;
          y[2 * r + 1] = im;
        }
        for (int e = 0; e < 32; ++e) {
          (*cur)[2 * at(e)] = y[2 * e];
          (*cur)[2 * at(e) + 1] = y[2 * e + 1];
        }
      }
      continue;
    }
    if (st.kind == 1) {
      const csim_gate& g = st.g;
      double c = 0, s = 0;
      if (g.op == OP_RY) {
        c = std::cos(g.angle / 2);
        s = std::sin(g.angle / 2);
      }
      if (g.op == OP_ZPHASE) {
        c = std::cos(g.angle);
        s = std::sin(g.angle);
      }
      const uint64_t tb = 1ull << g.target;
      for (uint64_t i = 0; i < N; ++i)
        if (!(i & tb) && (i & g.cmask) == g.cval)
          pair_op(&(*cur)[2 * i], &(*cur)[2 * (i | tb)], g.op, c, s);
      continue;
    }
    const SweepParams& sp = p.params[st.param];
    std::vector<double>& dst = (st.gather && !st.inplace) ? *nxt : *cur;
    const uint32_t ntiles = (uint32_t)(N >> 7);
    // the 2^nstage tiles that differ in the staged qubits go together (one
    // group of one tile without staging)
    const int U = 1 << sp.nstage;
    uint32_t smask = 0;
    for (int j = 0; j < sp.nstage; ++j) smask |= 1u << sp.fast[j];
    std::vector<std::array<std::array<std::array<double, 2>, 4>, 32>> vg((size_t)U);
    std::vector<std::array<uint32_t, 32>> where((size_t)U);
    std::vector<uint32_t> tiles((size_t)U);
    std::vector<std::array<double, 32>> mcs((size_t)U), mss((size_t)U);
    for (uint32_t base = 0; base < ntiles; ++base) {
      if (base & smask) continue;
      for (int u = 0; u < U; ++u) {
        uint32_t t = base;
        for (int j = 0; j < sp.nstage; ++j)
          if ((u >> j) & 1) t |= 1u << sp.fast[j];
        tiles[(size_t)u] = t;
        for (uint32_t lane = 0; lane < 32; ++lane) {
          const uint32_t ci = (t << 5) | lane;
          const uint32_t src = sp.scatter ? ci : emu_permute(p, sp, ci);
          where[(size_t)u][lane] = sp.scatter ? emu_permute(p, sp, ci) : (st.inplace ? src : ci);
          for (int j = 0; j < 4; ++j) {
            vg[(size_t)u][lane][j][0] = (*cur)[2 * (((size_t)src << 2) + j)];
            vg[(size_t)u][lane][j][1] = (*cur)[2 * (((size_t)src << 2) + j) + 1];
          }
        }
        mcs[(size_t)u].fill(1.0);
        mss[(size_t)u].fill(0.0);
      }
      auto tile_v = [&](int u) -> double(&)[32][4][2] {
        return *reinterpret_cast<double(*)[32][4][2]>(vg[(size_t)u].data());
      };
      auto tile_m = [&](std::vector<std::array<double, 32>>& m, int u) -> double(&)[32] {
        return *reinterpret_cast<double(*)[32]>(m[(size_t)u].data());
      };
      for (int k = 0; k < sp.nops; ++k) {
        const LocalOp& o = sp.ops[k];
        if (o.op >= 9) {  // a gate on staged qubit o.target: pairs tiles u, u | bit
          const int bit = 1 << o.target;
          for (int u = 0; u < U; ++u) {
            if (u & bit) continue;
            for (uint32_t lane = 0; lane < 32; ++lane) {
              const uint32_t ci = (tiles[(size_t)u] << 5) | lane;
              if ((ci & o.cm) != o.cv) continue;
              for (int j = 0; j < 4; ++j)
                if (((uint32_t)j & o.lm) == o.lv)
                  pair_op(vg[(size_t)u][lane][j].data(), vg[(size_t)(u | bit)][lane][j].data(),
                          o.op - 9, o.cd, o.sd);
            }
          }
          continue;
        }
        for (int u = 0; u < U; ++u)
          emu_ops(p, sp, tiles[(size_t)u], tile_v(u), k, k + 1, tile_m(mcs, u), tile_m(mss, u));
      }
      for (int u = 0; u < U; ++u)
        for (uint32_t lane = 0; lane < 32; ++lane)
          for (int j = 0; j < 4; ++j) {
            dst[2 * (((size_t)where[(size_t)u][lane] << 2) + j)] = vg[(size_t)u][lane][j][0];
            dst[2 * (((size_t)where[(size_t)u][lane] << 2) + j) + 1] = vg[(size_t)u][lane][j][1];
          }
    }
    if (st.gather && !st.inplace) std::swap(cur, nxt);
  }
  if (cur != amps) *amps = *cur;
}

}  // namespace csim
