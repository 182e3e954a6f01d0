// Request pool: many circuit runs on one GPU (batching and serving).
//
//  * Admission.  Each request needs device memory for its two state buffers
//    (ping-pong), the compacted postselected block and the staging of b.  The
//    pool owns one arena of `hbm_budget` bytes carved by a buddy allocator
//    (every state is a power of two bytes), and admits queued requests in
//    arrival order while a stream slot is free and the head request's blocks
//    fit (first come, first served; the head is never overtaken).
//  * Execution.  An admitted request runs on its slot's CUDA stream:
//    H2D of b, init kernel, the fused program, FP64 norms, compaction and D2H
//    of the results into the slot's pinned buffers.  With use_graphs, all
//    requests admitted in one admission pass are captured into one CUDA graph
//    (one branch per request) and launched once.
//  * Completion.  csim_pool_poll retires finished requests (event queries),
//    releases their blocks and admits more: continuous batching.
//  * Planner.  csim_pool_plan runs the same arena and admission policy on a
//    discrete-event clock with given durations (no GPU) for capacity planning
//    and for testing the policy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "handles.h"
#include "kernels.h"

namespace csim {
void record_last_error(const std::string& msg);
}

namespace {

csim_status pfail(csim_status s, const std::string& msg) {
  csim::record_last_error(msg);
  return s;
}
csim_status pcuda(cudaError_t e, const char* where) {
  return pfail(CSIM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Buddy allocator over byte offsets [0, capacity).  The capacity is split
// into power-of-two regions (largest first); blocks are min_block << order.
class BuddyArena {
 public:
  void init(uint64_t bytes, uint64_t min_block) {
    min_ = min_block;
    regions_.clear();
    free_.assign(64, {});
    live_.clear();
    in_use_ = 0;
    uint64_t units = bytes / min_block, base = 0;
    for (int k = 63; k >= 0; --k) {
      if (!((units >> k) & 1ull)) continue;
      regions_.push_back({base, k});
      free_[k].insert(base);
      base += min_block << k;
    }
    cap_ = base;
  }
  static int order_for(uint64_t bytes, uint64_t min_block) {
    int k = 0;
    while ((min_block << k) < bytes) ++k;
    return k;
  }
  bool alloc(uint64_t bytes, uint64_t* off) {
    const int j = order_for(bytes, min_);
    int k = j;
    while (k < 64 && free_[k].empty()) ++k;
    if (k >= 64) return false;
    uint64_t o = *free_[k].begin();
    free_[k].erase(free_[k].begin());
    while (k > j) {
      --k;
      free_[k].insert(o + (min_ << k));
    }
    live_[o] = j;
    in_use_ += min_ << j;
    *off = o;
    return true;
  }
  void release(uint64_t off) {
    auto it = live_.find(off);
    if (it == live_.end()) return;
    int j = it->second;
    live_.erase(it);
    in_use_ -= min_ << j;
    const Region& r = region_of(off);
    while (j < r.order) {
      const uint64_t buddy = r.base + ((off - r.base) ^ (min_ << j));
      auto f = free_[j].find(buddy);
      if (f == free_[j].end()) break;
      free_[j].erase(f);
      off = std::min(off, buddy);
      ++j;
    }
    free_[j].insert(off);
  }
  uint64_t in_use() const { return in_use_; }
  uint64_t capacity() const { return cap_; }
  uint64_t min_block() const { return min_; }

 private:
  struct Region {
    uint64_t base;
    int order;
  };
  const Region& region_of(uint64_t off) const {
    for (const Region& r : regions_)
      if (off >= r.base && off < r.base + (min_ << r.order)) return r;
    return regions_.front();
  }
  uint64_t min_ = 1, cap_ = 0, in_use_ = 0;
  std::vector<Region> regions_;
  std::vector<std::set<uint64_t>> free_;
  std::map<uint64_t, int> live_;
};

// Blocks of a request: state 0, state 1, compacted block, staging of b, and
// the source-index tables of its program (two at most).  The planner's
// requests have the first four.
constexpr int kAllocs = 6, kPlanAllocs = 4, kTabBlock = 4, kMaxPoolTables = 2;

// Whether every block of one request fits an empty arena of this capacity.
bool fits_empty(uint64_t capacity, uint64_t min_block, const uint64_t* sizes, int n) {
  BuddyArena a;
  a.init(capacity, min_block);
  uint64_t off;
  for (int k = 0; k < n; ++k)
    if (sizes[k] && !a.alloc(sizes[k], &off)) return false;
  return true;
}

// All-or-nothing allocation of a request's blocks.
bool alloc_all(BuddyArena* a, const uint64_t* sizes, uint64_t* offs, int n) {
  for (int k = 0; k < n; ++k) {
    offs[k] = ~0ull;
    if (!sizes[k]) continue;
    if (!a->alloc(sizes[k], &offs[k])) {
      for (int j = 0; j < k; ++j)
        if (offs[j] != ~0ull) a->release(offs[j]);
      return false;
    }
  }
  return true;
}
void release_all(BuddyArena* a, const uint64_t* offs, int n) {
  for (int k = 0; k < n; ++k)
    if (offs[k] != ~0ull) a->release(offs[k]);
}

enum class RState { Queued, Running, Done };

struct Request {
  int64_t id = 0;
  csim_circuit* c = nullptr;
  int prec = 0;
  std::vector<uint64_t> idx;
  std::vector<double> val;
  uint64_t sizes[kAllocs] = {0, 0, 0, 0, 0, 0};
  uint64_t offs[kAllocs] = {~0ull, ~0ull, ~0ull, ~0ull, ~0ull, ~0ull};
  int ntab = 0;  // source-index tables built into blocks kTabBlock.. for this run
  RState st = RState::Queued;
  int slot = -1;
  uint64_t count = 0;  // compacted amplitudes
  int wave = -1;       // index into csim_pool::waves when launched in a graph
  double t_submit = 0, t_start = 0, t_done = 0;
  double p = 0, tot = 0, dev_ms = 0;
  double dev_t0 = -1, dev_t1 = -1;  // device start / end after the pool's epoch (stream mode)
  std::vector<double> amps;
  csim_status err = CSIM_OK;  // a request that failed on the host before its device work
  std::string err_msg;
  bool cancelled = false;     // discarded at retirement
  bool batched = false;       // ran in a persistent launch (its slot's flag holds the error)
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  uint64_t* d_pat = nullptr;
  double* d_partial = nullptr;
  double* d_out = nullptr;
  double* d_npart = nullptr;  // the last sweep's |a|^2 partials (kNormPartCap doubles)
  void* h_stage = nullptr;  // pinned: patterns, then idx, then val
  size_t h_stage_cap = 0;
  double* h_out = nullptr;  // pinned: 2 doubles
  double* h_amps = nullptr;  // pinned: compacted block
  size_t h_amps_cap = 0;
  uint32_t* h_flag = nullptr;  // pinned: the persistent launch's error word
  int64_t req = -1;
};

constexpr int kMaxPatterns = 64;

}  // namespace

struct csim_pool {
  csim_pool_opts o{};
  void* d_arena = nullptr;
  BuddyArena arena;
  std::vector<Slot> slots;
  cudaStream_t origin = nullptr;  // graph capture origin
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, Request> reqs;
  std::vector<int64_t> done_unreported;
  // One graph launch per admission pass.  Completion is taken from an event
  // recorded on the origin stream after the launch: an event-record node
  // inside the graph keeps its previous (completed) state until the node
  // runs, so it cannot tell whether this launch has finished.
  struct Wave {
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    int pending = 0;
  };
  std::vector<Wave> waves;
  int64_t next_id = 1;
  csim_pool_stats_t stats{};
  cudaEvent_t epoch = nullptr;  // recorded on the origin stream at creation
  cudaStream_t upload = nullptr;  // program uploads of submitted circuits
  // host-side fault injection (csim_pool_inject): request id -> what fails
  std::unordered_map<int64_t, int> inject;
};

namespace {

void request_sizes(const csim_circuit* c, int prec, size_t nnz, int ntab, uint64_t* sizes,
                   uint64_t* count) {
  const uint64_t S = ((uint64_t)1 << c->L.n) * (prec == CSIM_C64 ? 8 : 16);
  const csim::CompactGeom g = csim::compact_geom(c);
  sizes[0] = S;
  sizes[1] = (c->prog_built && !c->prog.pingpong) ? 0 : S;
  sizes[2] = std::max<uint64_t>(g.count * 16, 256);
  sizes[3] = std::max<uint64_t>(nnz * 16, 256);
  for (int t = 0; t < kMaxPoolTables; ++t)
    sizes[kTabBlock + t] = t < ntab ? std::max<uint64_t>((uint64_t)1 << c->L.n, 256) : 0;
  *count = g.count;
}

cudaError_t grow_pinned(Slot* s, size_t stage_bytes, size_t amp_bytes) {
  cudaError_t e = cudaSuccess;
  if (s->h_stage_cap < stage_bytes) {
    if (s->h_stage) cudaFreeHost(s->h_stage);
    s->h_stage = nullptr;
    s->h_stage_cap = 0;
    e = cudaMallocHost(&s->h_stage, stage_bytes);
    if (e != cudaSuccess) return e;
    s->h_stage_cap = stage_bytes;
  }
  if (s->h_amps_cap < amp_bytes) {
    if (s->h_amps) cudaFreeHost(s->h_amps);
    s->h_amps = nullptr;
    s->h_amps_cap = 0;
    e = cudaMallocHost((void**)&s->h_amps, amp_bytes);
    if (e != cudaSuccess) return e;
    s->h_amps_cap = amp_bytes;
  }
  return cudaSuccess;
}

// Enqueue one request's whole run on stream st (the slot's stream, possibly
// under capture).
cudaError_t enqueue_request(csim_pool* P, Request& r, Slot& s, bool in_graph, const char** where) {
  csim_circuit* c = r.c;
  char* base = static_cast<char*>(P->d_arena);
  void* buf[2] = {base + r.offs[0], r.offs[1] != ~0ull ? base + r.offs[1] : nullptr};
  double* d_compact = reinterpret_cast<double*>(base + r.offs[2]);
  char* d_stage = base + r.offs[3];
  const size_t nnz = r.idx.size();
  const int npat = (int)c->pm.size();
  // host staging (pinned): patterns (masks, values), idx, val
  char* hs = static_cast<char*>(s.h_stage);
  std::memcpy(hs, c->pm.data(), npat * 8);
  std::memcpy(hs + npat * 8, c->pv.data(), npat * 8);
  const size_t pat_bytes = 16 * (size_t)npat;
  std::memcpy(hs + pat_bytes, r.idx.data(), nnz * 8);
  std::memcpy(hs + pat_bytes + nnz * 8, r.val.data(), nnz * 8);
  cudaStream_t st = s.st;
  // per-request timing events on the stream path only: events recorded inside
  // a graph do not time (the wave is timed around the launch instead)
  *where = "start event";
  cudaError_t e = in_graph ? cudaSuccess : cudaEventRecord(s.ev0, st);
  if (e == cudaSuccess) {
    *where = "pattern copy";
    e = cudaMemcpyAsync(s.d_pat, hs, pat_bytes, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) {
    *where = "b copy";
    e = cudaMemcpyAsync(d_stage, hs + pat_bytes, nnz * 16, cudaMemcpyHostToDevice, st);
  }
  // sparse init: write the tiles of b only and leave the zeros to the
  // program's leading sweeps.  The tile map sits at the start of the second
  // state buffer, which those (in-place) sweeps do not write.
  const int zsteps =
      buf[1] && csim::sparse_init_enabled() ? csim::zero_fill_steps(c, r.prec) : 0;
  uint32_t* zmap = zsteps > 0 ? static_cast<uint32_t*>(buf[1]) : nullptr;
  if (e == cudaSuccess) *where = "init";
  if (e == cudaSuccess) {
    const uint64_t* d_idx = reinterpret_cast<const uint64_t*>(d_stage);
    const double* d_val = reinterpret_cast<const double*>(d_stage + nnz * 8);
    e = zmap ? csim::launch_init_sparse(buf[0], r.prec, c->L.n, d_idx, d_val, (int64_t)nnz, zmap, st)
             : csim::launch_init(buf[0], r.prec, (uint64_t)1 << c->L.n, d_idx, d_val,
                                 (int64_t)nnz, st);
  }
  uint32_t* tabs[kMaxPoolTables] = {nullptr, nullptr};
  for (int t = 0; t < r.ntab; ++t) tabs[t] = reinterpret_cast<uint32_t*>(base + r.offs[kTabBlock + t]);
  if (e == cudaSuccess && r.ntab > 0) {
    *where = "source-index tables";
    e = csim::launch_src_tables(c->prog, tabs, st);
  }
  int cur = 0;
  // the last sweep sums |a|^2 as csim_run's does, so the norms equal the run
  // alone bit for bit
  const bool fused = csim::program_fuses_norm(c->prog, r.prec);
  if (e == cudaSuccess) {
    *where = "program";
    e = csim::run_program_steps(c->prog, buf, &cur, r.prec, st, 0, (int64_t)c->prog.steps.size(),
                                r.ntab > 0 ? tabs : nullptr, zmap, zsteps,
                                fused ? s.d_npart : nullptr);
  }
  int lowk = 0;
  uint64_t lowv = 0;
  csim::mask_low_bits(c, &lowk, &lowv);
  if (e == cudaSuccess) *where = "norms";
  if (e == cudaSuccess)
    e = fused ? csim::launch_norms_fused(buf[cur], r.prec, c->L.n, s.d_pat, s.d_pat + npat, npat,
                                         lowk, lowv, s.d_npart, s.d_partial, s.d_out, st)
              : csim::launch_norms(buf[cur], r.prec, c->L.n, s.d_pat, s.d_pat + npat, npat, lowk,
                                   lowv, s.d_partial, s.d_out, st);
  const csim::CompactGeom g = csim::compact_geom(c);
  if (e == cudaSuccess) *where = "compaction";
  if (e == cudaSuccess && g.count)
    e = csim::launch_compact(buf[cur], r.prec, d_compact, g.count, g.free_shift, g.free_bits,
                             (uint64_t)c->L.Nt, g.m_shift, st);
  if (e == cudaSuccess) *where = "result copy";
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s.h_out, s.d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && g.count)
    e = cudaMemcpyAsync(s.h_amps, d_compact, g.count * 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && !in_graph) {
    *where = "end event";
    e = cudaEventRecord(s.ev1, st);
  }
  return e;
}

// Whether a request can run in a persistent launch: complex64, at least 12
// qubits, and a program of fused sweeps only (no staged high qubits).
bool batch_eligible(const Request& r) {
  if (r.prec != CSIM_C64 || r.c->L.n < 12) return false;
  const csim::Program& p = r.c->prog;
  for (const csim::Step& st : p.steps) {
    const csim::SweepParams& a = p.params[(size_t)st.param];
    if (st.kind != 0 || a.nstage != 0 || a.scatter) return false;
    // one of the four sweep op lists the kernel carries
    const int shape = csim::batch_shape(a);
    if (shape < 1 || shape > 4) return false;
    // a gather from its source-index table (built in the arena)
    if (st.gather && (r.ntab == 0 || (size_t)st.param >= p.src_tab.size() ||
                      p.src_tab[(size_t)st.param] < 0))
      return false;
    if (!st.gather && a.nseg != 0) return false;
  }
  return true;
}

bool batch_by_level() {
  static const bool v = [] {
    const char* e = std::getenv("CSIM_BATCH_ORDER");
    return e && std::strcmp(e, "level") == 0;
  }();
  return v;
}

// The persistent path of an admission pass (see csim.h): uploads and plain
// inits, the source-index tables, one launch over every request's sweeps
// (items queued level by level), then norms, compactions and result copies,
// all on the stream of the pass's first slot.  The slots of a pass are free
// when it is admitted, so consecutive passes run on different streams and
// the next one fills the GPU while the last levels of the previous one drain.
cudaError_t enqueue_batch(csim_pool* P, const std::vector<std::pair<int64_t, int>>& started,
                          const char** where) {
  cudaStream_t st = P->slots[started.front().second].st;
  char* base = static_cast<char*>(P->d_arena);
  std::vector<csim::SweepParams> sps;
  std::vector<csim::BatchStep> steps;
  std::vector<std::vector<int>> prog_steps(started.size());  // global step indices per request
  std::vector<int> final_cur(started.size(), 0);
  const uint32_t stride = csim::batch_stride();
  const uint32_t item_tiles = stride * 64;  // 1024 tiles (1 MiB of complex64) per item
  uint32_t drop = ~0u;
  cudaError_t e = cudaSuccess;
  csim_pool::Wave w;
  *where = "wave events";
  e = cudaEventCreate(&w.start);
  if (e == cudaSuccess) e = cudaEventCreate(&w.done);
  if (e == cudaSuccess) e = cudaEventRecord(w.start, st);
  // First, on the host only: each request's leading sweeps (those that
  // complete its sparse init) and its other sweeps as batch steps, with the
  // buffers each one reads and writes.  The tables are uploaded before any of
  // the pass's device work is queued: an upload from pageable memory waits
  // for the stream's earlier work.
  std::vector<int> lead(started.size(), 0);
  for (size_t q = 0; q < started.size(); ++q) {
    Request& r = P->reqs[started[q].first];
    csim_circuit* c = r.c;
    void* buf[2] = {base + r.offs[0], r.offs[1] != ~0ull ? base + r.offs[1] : nullptr};
    const int zsteps =
        buf[1] && csim::sparse_init_enabled() ? csim::zero_fill_steps(c, r.prec) : 0;
    lead[q] = zsteps;
    uint32_t* tabs[kMaxPoolTables] = {nullptr, nullptr};
    for (int t = 0; t < r.ntab; ++t) tabs[t] = reinterpret_cast<uint32_t*>(base + r.offs[kTabBlock + t]);
    int cur = 0, prev = -1;
    for (int j = 0; j < zsteps; ++j) {  // as run_program_steps moves the state
      const csim::Step& stp = c->prog.steps[(size_t)j];
      if (stp.kind == 0 && stp.gather && !stp.inplace) cur = 1 - cur;
    }
    const uint32_t ntiles = 1u << (c->L.n - 7);
    for (size_t j = (size_t)zsteps; j < c->prog.steps.size(); ++j) {
      const csim::Step& stp = c->prog.steps[j];
      csim::SweepParams a = c->prog.params[(size_t)stp.param];
      if (r.ntab > 0 && (size_t)stp.param < c->prog.src_tab.size() &&
          c->prog.src_tab[(size_t)stp.param] >= 0)
        a.src = tabs[c->prog.src_tab[(size_t)stp.param]];
      a.src_prefetch = 0;
      a.zero_map = nullptr;
      a.zero_mode = 0;
      csim::BatchStep bs{};
      bs.in = buf[cur];
      const bool moves = stp.gather && !stp.inplace;
      bs.out = moves ? buf[1 - cur] : buf[cur];
      if (moves) cur = 1 - cur;
      bs.nitems = (ntiles + item_tiles - 1) / item_tiles;
      bs.dep = prev;
      csim::batch_order(a, ntiles, &bs.nfe, &bs.fmask, &bs.hstep, &bs.li);
      bs.shape = csim::batch_shape(a);
      prev = (int)steps.size();
      prog_steps[q].push_back(prev);
      sps.push_back(a);
      steps.push_back(bs);
    }
    // the request's last sweep sums |a|^2 of the final state for its norms
    if (!prog_steps[q].empty() && (size_t)prog_steps[q].back() + 1 == steps.size() &&
        steps.back().shape == 4)
      steps.back().norm_part = P->slots[started[q].second].d_npart;
    final_cur[q] = cur;
    const auto inj = P->inject.find(r.id);
    if (inj != P->inject.end() && inj->second == CSIM_INJECT_BATCH_SIGNAL &&
        prog_steps[q].size() > 2)
      drop = (uint32_t)prog_steps[q][1];  // resolved to an item index below
    r.batched = true;
  }
  // The queue order of the steps.  Every step comes after the previous step
  // of its request, which is all the kernel's progress needs.  By progress
  // (default): step k of a request with L steps at key (k + 1) / L, so that
  // every request advances at the same relative pace and finishes near the
  // end of the pass; a request's consecutive steps are then separated by the
  // other requests' items, and the pass does not end on one small request's
  // last steps run alone.  By level (CSIM_BATCH_ORDER=level): step k of every
  // request before step k + 1 of any.  Ties: the larger request first.
  struct Entry {
    double key;
    int n;
    size_t q, k;
  };
  std::vector<Entry> order;
  for (size_t q = 0; q < prog_steps.size(); ++q) {
    const size_t L = prog_steps[q].size();
    for (size_t k = 0; k < L; ++k)
      order.push_back(Entry{batch_by_level() ? (double)k : (double)(k + 1) / (double)L,
                            P->reqs[started[q].first].c->L.n, q, k});
  }
  std::stable_sort(order.begin(), order.end(), [](const Entry& x, const Entry& y) {
    if (x.key != y.key) return x.key < y.key;
    return x.n > y.n;
  });
  std::vector<csim::BatchItem> items;
  uint32_t drop_item = ~0u;
  for (const Entry& en : order) {
    const int gs = prog_steps[en.q][en.k];
    const uint32_t ntiles = 1u << (en.n - 7);
    for (uint32_t c0 = 0; c0 < ntiles; c0 += item_tiles) {
      if ((uint32_t)gs == drop && drop_item == ~0u) drop_item = (uint32_t)items.size();
      items.push_back(csim::BatchItem{(uint32_t)gs, c0, std::min(ntiles, c0 + item_tiles)});
    }
  }
  // the tables in one stream-ordered allocation, freed after the launch
  const size_t o_steps = 0;
  const size_t o_sps = (o_steps + steps.size() * sizeof(csim::BatchStep) + 255) & ~(size_t)255;
  const size_t o_items = (o_sps + sps.size() * sizeof(csim::SweepParams) + 255) & ~(size_t)255;
  const size_t o_done = (o_items + items.size() * sizeof(csim::BatchItem) + 255) & ~(size_t)255;
  const size_t o_ctl = (o_done + steps.size() * 4 + 255) & ~(size_t)255;
  const size_t total = o_ctl + sizeof(csim::BatchCtl);
  char* d = nullptr;
  if (e == cudaSuccess) {
    *where = "table allocation";
    e = cudaMallocAsync(reinterpret_cast<void**>(&d), total, st);
  }
  if (e == cudaSuccess) {
    for (size_t i = 0; i < steps.size(); ++i)
      steps[i].sp = reinterpret_cast<const csim::SweepParams*>(d + o_sps) + i;
    const csim::BatchCtl ctl{0u, 0u, drop_item, 0u};
    if (drop_item != ~0u) P->stats.batch_dropped_signals++;
    *where = "table upload";
    e = cudaMemcpyAsync(d + o_steps, steps.data(), steps.size() * sizeof(csim::BatchStep),
                        cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d + o_sps, sps.data(), sps.size() * sizeof(csim::SweepParams),
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d + o_items, items.data(), items.size() * sizeof(csim::BatchItem),
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d + o_done, 0, steps.size() * 4, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d + o_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, st);
  }
  // each request's uploads, init, source-index tables and leading sweeps
  for (size_t q = 0; q < started.size() && e == cudaSuccess; ++q) {
    Request& r = P->reqs[started[q].first];
    Slot& sl = P->slots[started[q].second];
    csim_circuit* c = r.c;
    void* buf[2] = {base + r.offs[0], r.offs[1] != ~0ull ? base + r.offs[1] : nullptr};
    char* d_stage = base + r.offs[3];
    const size_t nnz = r.idx.size();
    const int npat = (int)c->pm.size();
    char* hs = static_cast<char*>(sl.h_stage);
    std::memcpy(hs, c->pm.data(), npat * 8);
    std::memcpy(hs + npat * 8, c->pv.data(), npat * 8);
    const size_t pat_bytes = 16 * (size_t)npat;
    std::memcpy(hs + pat_bytes, r.idx.data(), nnz * 8);
    std::memcpy(hs + pat_bytes + nnz * 8, r.val.data(), nnz * 8);
    *where = "uploads";
    e = cudaMemcpyAsync(sl.d_pat, hs, pat_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_stage, hs + pat_bytes, nnz * 16, cudaMemcpyHostToDevice, st);
    // sparse init, as on the stream path: the tiles of b only, the zeros
    // left to the program's leading sweeps (the tile map at the start of the
    // second buffer)
    const int zsteps = lead[q];
    uint32_t* zmap = zsteps > 0 ? static_cast<uint32_t*>(buf[1]) : nullptr;
    if (e == cudaSuccess) {
      *where = "init";
      const uint64_t* d_idx = reinterpret_cast<const uint64_t*>(d_stage);
      const double* d_val = reinterpret_cast<const double*>(d_stage + nnz * 8);
      e = zmap ? csim::launch_init_sparse(buf[0], r.prec, c->L.n, d_idx, d_val, (int64_t)nnz, zmap,
                                          st)
               : csim::launch_init(buf[0], r.prec, (uint64_t)1 << c->L.n, d_idx, d_val,
                                   (int64_t)nnz, st);
    }
    uint32_t* tabs[kMaxPoolTables] = {nullptr, nullptr};
    for (int t = 0; t < r.ntab; ++t) tabs[t] = reinterpret_cast<uint32_t*>(base + r.offs[kTabBlock + t]);
    if (e == cudaSuccess && r.ntab > 0) {
      *where = "source-index tables";
      e = csim::launch_src_tables(c->prog, tabs, st);
    }
    // the sweeps that complete the sparse init, with the sweep kernels (their
    // zero handling)
    if (e == cudaSuccess && zsteps > 0) {
      *where = "leading sweeps";
      int cur = 0;
      e = csim::run_program_steps(c->prog, buf, &cur, r.prec, st, 0, zsteps,
                                  r.ntab > 0 ? tabs : nullptr, zmap, zsteps);
    }
  }
  if (e == cudaSuccess) {
    *where = "persistent launch";
    e = csim::launch_batch(reinterpret_cast<const csim::BatchStep*>(d + o_steps),
                           reinterpret_cast<const csim::BatchItem*>(d + o_items),
                           (uint32_t)items.size(), reinterpret_cast<uint32_t*>(d + o_done),
                           reinterpret_cast<csim::BatchCtl*>(d + o_ctl), st);
  }
  // norms, compactions and result copies of every request
  for (size_t q = 0; q < started.size() && e == cudaSuccess; ++q) {
    Request& r = P->reqs[started[q].first];
    Slot& sl = P->slots[started[q].second];
    csim_circuit* c = r.c;
    void* fin = base + r.offs[final_cur[q] == 0 ? 0 : 1];
    double* d_compact = reinterpret_cast<double*>(base + r.offs[2]);
    const int npat = (int)c->pm.size();
    int lowk = 0;
    uint64_t lowv = 0;
    csim::mask_low_bits(c, &lowk, &lowv);
    *where = "norms";
    const bool fused = !prog_steps[q].empty() && steps[(size_t)prog_steps[q].back()].norm_part;
    e = fused ? csim::launch_norms_fused(fin, r.prec, c->L.n, sl.d_pat, sl.d_pat + npat, npat,
                                         lowk, lowv, sl.d_npart, sl.d_partial, sl.d_out, st)
              : csim::launch_norms(fin, r.prec, c->L.n, sl.d_pat, sl.d_pat + npat, npat, lowk,
                                   lowv, sl.d_partial, sl.d_out, st);
    const csim::CompactGeom g = csim::compact_geom(c);
    if (e == cudaSuccess && g.count) {
      *where = "compaction";
      e = csim::launch_compact(fin, r.prec, d_compact, g.count, g.free_shift, g.free_bits,
                               (uint64_t)c->L.Nt, g.m_shift, st);
    }
    if (e == cudaSuccess) {
      *where = "result copy";
      e = cudaMemcpyAsync(sl.h_out, sl.d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess && g.count)
      e = cudaMemcpyAsync(sl.h_amps, d_compact, g.count * 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && d)
      e = cudaMemcpyAsync(sl.h_flag, d + o_ctl + offsetof(csim::BatchCtl, error), 4,
                          cudaMemcpyDeviceToHost, st);
  }
  if (d) {
    const cudaError_t fe = cudaFreeAsync(d, st);
    if (e == cudaSuccess) e = fe;
  }
  if (e == cudaSuccess) e = cudaEventRecord(w.done, st);
  w.pending = (int)started.size();
  const int wi = (int)P->waves.size();
  P->waves.push_back(w);
  for (auto& [id, k] : started) P->reqs[id].wave = wi;
  if (e == cudaSuccess) {
    P->stats.batch_launches++;
    P->stats.batch_requests += (int64_t)started.size();
  }
  return e;
}

// A request that fails before any of its device work is enqueued: it leaves
// the queue with its error, holds no memory, and is reported by the next
// poll like a finished one; the pool keeps serving the others.
void fail_request(csim_pool* P, Request& r, csim_status err, const std::string& msg) {
  release_all(&P->arena, r.offs, kAllocs);
  for (uint64_t& o : r.offs) o = ~0ull;
  r.err = err;
  r.err_msg = msg;
  r.st = RState::Done;
  r.t_start = r.t_done = now_s();
  P->stats.failed++;
  if (!r.cancelled) P->done_unreported.push_back(r.id);
}

// Admit queued requests (FIFO) into free slots while their blocks fit, at
// most `cap` of them, as one admission pass; *n_started receives how many
// were admitted.
csim_status admit_pass(csim_pool* P, size_t cap, size_t* n_started) {
  std::vector<std::pair<int64_t, int>> started;
  *n_started = 0;
  while (!P->queue.empty() && started.size() < cap) {
    int free_slot = -1;
    for (int k = 0; k < (int)P->slots.size(); ++k)
      if (P->slots[k].req < 0) {
        free_slot = k;
        break;
      }
    if (free_slot < 0) break;
    Request& r = P->reqs[P->queue.front()];
    const auto inj = P->inject.find(r.id);
    const int fault = inj == P->inject.end() ? 0 : inj->second;
    if (fault == CSIM_INJECT_ARENA) {  // as if the arena refused the request's blocks
      P->queue.pop_front();
      fail_request(P, r, CSIM_ERR_OOM, "csim_pool: arena allocation refused (injected)");
      continue;
    }
    if (!alloc_all(&P->arena, r.sizes, r.offs, kAllocs)) break;
    Slot& s = P->slots[free_slot];
    cudaError_t e = fault == CSIM_INJECT_PINNED
                        ? cudaErrorMemoryAllocation
                        : grow_pinned(&s, 16 * kMaxPatterns + r.idx.size() * 16, r.count * 16 + 16);
    if (e != cudaSuccess) {
      cudaGetLastError();
      P->queue.pop_front();
      fail_request(P, r, CSIM_ERR_OOM,
                   std::string("csim_pool: pinned staging: ") + cudaGetErrorString(e) +
                       (fault == CSIM_INJECT_PINNED ? " (injected)" : ""));
      continue;
    }
    s.req = r.id;
    r.slot = free_slot;
    r.st = RState::Running;
    r.t_start = now_s();
    P->queue.pop_front();
    P->stats.admitted++;
    P->stats.src_tables += r.ntab;
    if (r.offs[1] != ~0ull && csim::sparse_init_enabled()) {
      const int z = csim::zero_fill_steps(r.c, r.prec);
      P->stats.sparse_saved_bytes += (uint64_t)(z == 2 ? 3 : z) * r.sizes[0];
    }
    P->stats.bytes_in_use = P->arena.in_use();
    P->stats.peak_bytes = std::max(P->stats.peak_bytes, P->arena.in_use());
    started.emplace_back(r.id, free_slot);
  }
  *n_started = started.size();
  if (started.empty()) return CSIM_OK;
  cudaError_t e = cudaSuccess;
  if (P->o.persistent) {
    // the eligible requests of the pass in one persistent launch, the others
    // on their own streams
    std::vector<std::pair<int64_t, int>> batch, rest;
    for (auto& pr : started) (batch_eligible(P->reqs[pr.first]) ? batch : rest).push_back(pr);
    if (!batch.empty()) {
      const char* where = "";
      e = enqueue_batch(P, batch, &where);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return pfail(CSIM_ERR_CUDA, std::string("csim_pool: persistent pass, ") + where + ": " +
                                        cudaGetErrorString(e));
      }
    }
    started.swap(rest);
    if (started.empty()) return CSIM_OK;
  }
  if (!P->o.use_graphs || P->o.persistent) {
    for (auto& [id, k] : started) {
      const char* step = "";
      e = enqueue_request(P, P->reqs[id], P->slots[k], false, &step);
      if (e != cudaSuccess)
        return pfail(CSIM_ERR_CUDA, std::string("csim_pool: enqueue, ") + step + ": " +
                                        cudaGetErrorString(e));
    }
    return CSIM_OK;
  }
  // one graph for the whole admission pass: fork from the origin stream into
  // each request's slot stream, join back, launch once
  const char* where = "event create";
  cudaEvent_t fork = nullptr;
  e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  std::vector<cudaEvent_t> joins(started.size(), nullptr);
  for (size_t k = 0; k < started.size() && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&joins[k], cudaEventDisableTiming);
  cudaGetLastError();  // a stale non-sticky error must not be read as a capture failure
  if (e == cudaSuccess) {
    where = "begin capture";
    e = cudaStreamBeginCapture(P->origin, cudaStreamCaptureModeThreadLocal);
  }
  if (e == cudaSuccess) {
    where = "fork record";
    e = cudaEventRecord(fork, P->origin);
  }
  std::string detail;
  for (size_t k = 0; k < started.size() && e == cudaSuccess; ++k) {
    Slot& s = P->slots[started[k].second];
    const cudaError_t stale = cudaPeekAtLastError();
    if (stale != cudaSuccess) {
      detail = std::string(" (pending error before request ") + std::to_string(k) + ": " +
               cudaGetErrorString(stale) + ")";
      cudaGetLastError();
    }
    where = "fork wait";
    e = cudaStreamWaitEvent(s.st, fork, 0);
    if (e == cudaSuccess) {
      const char* step = "";
      e = enqueue_request(P, P->reqs[started[k].first], s, true, &step);
      if (e != cudaSuccess) {
        where = step;
        detail += " (request " + std::to_string(k) + " of " + std::to_string(started.size()) +
                  ", " + std::to_string(P->reqs[started[k].first].c->L.n) + " qubits)";
      }
    }
    if (e == cudaSuccess) {
      where = "join record";
      e = cudaEventRecord(joins[k], s.st);
    }
    if (e == cudaSuccess) {
      where = "join wait";
      e = cudaStreamWaitEvent(P->origin, joins[k], 0);
    }
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(P->origin, &graph);
  if (e == cudaSuccess && ee != cudaSuccess) {
    where = "end capture";
    e = ee;
  }
  csim_pool::Wave w;
  if (e == cudaSuccess) {
    where = "instantiate";
    e = cudaGraphInstantiate(&w.exec, graph, 0);
  }
  if (e == cudaSuccess) {
    where = "wave event";
    e = cudaEventCreate(&w.done);
  }
  if (e == cudaSuccess) e = cudaEventCreate(&w.start);
  if (e == cudaSuccess) e = cudaEventRecord(w.start, P->origin);
  if (e == cudaSuccess) {
    where = "launch";
    e = cudaGraphLaunch(w.exec, P->origin);
  }
  if (e == cudaSuccess) e = cudaEventRecord(w.done, P->origin);
  if (graph) cudaGraphDestroy(graph);
  if (fork) cudaEventDestroy(fork);
  for (cudaEvent_t j : joins)
    if (j) cudaEventDestroy(j);
  w.pending = (int)started.size();
  const int wi = (int)P->waves.size();
  P->waves.push_back(w);
  for (auto& [id, k] : started) P->reqs[id].wave = wi;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return pfail(CSIM_ERR_CUDA, std::string("csim_pool: graph ") + where + ": " +
                                    cudaGetErrorString(e) + detail);
  }
  P->stats.graph_launches++;
  return CSIM_OK;
}

// Admission.  In persistent mode a pass takes at most half of the slots, so
// that the next pass is admitted while it runs and fills the GPU as its last
// levels drain; passes are formed until nothing more fits.
csim_status admit(csim_pool* P) {
  if (!P->o.persistent) {
    size_t n = 0;
    return admit_pass(P, P->slots.size(), &n);
  }
  const size_t cap = std::max<size_t>(1, P->slots.size() / 2);
  for (;;) {
    size_t n = 0;
    const csim_status s = admit_pass(P, cap, &n);
    if (s != CSIM_OK || n == 0) return s;
  }
}

// Retire every running request whose completion event has fired.
csim_status retire(csim_pool* P, int* n_retired) {
  *n_retired = 0;
  for (Slot& s : P->slots) {
    if (s.req < 0) continue;
    Request& r = P->reqs[s.req];
    const cudaError_t q = cudaEventQuery(r.wave >= 0 ? P->waves[r.wave].done : s.ev1);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return pcuda(q, "csim_pool: request failed");
    if (r.wave >= 0) P->waves[r.wave].pending--;
    r.tot = s.h_out[0];
    r.p = s.h_out[1];
    r.amps.assign(s.h_amps, s.h_amps + 2 * r.count);
    float ms = 0.f;
    const cudaError_t te = r.wave >= 0
                               ? cudaEventElapsedTime(&ms, P->waves[r.wave].start, P->waves[r.wave].done)
                               : cudaEventElapsedTime(&ms, s.ev0, s.ev1);
    if (te == cudaSuccess)
      r.dev_ms = ms;
    else
      cudaGetLastError();  // a failed timing query must not linger as the last error
    if (r.wave < 0 && P->epoch) {  // the request's device interval on the pool's clock
      float a = 0.f, b = 0.f;
      if (cudaEventElapsedTime(&a, P->epoch, s.ev0) == cudaSuccess &&
          cudaEventElapsedTime(&b, P->epoch, s.ev1) == cudaSuccess) {
        r.dev_t0 = a * 1e-3;
        r.dev_t1 = b * 1e-3;
      } else {
        cudaGetLastError();
      }
    }
    r.t_done = now_s();
    r.st = RState::Done;
    if (r.batched && *s.h_flag != 0u) {  // a dependency wait of the launch ran out
      r.err = CSIM_ERR_TIMEOUT;
      r.err_msg = "csim_pool: the persistent launch's dependency wait ran out; results invalid";
      P->stats.failed++;
      *s.h_flag = 0u;
    }
    release_all(&P->arena, r.offs, kAllocs);
    s.req = -1;
    P->stats.completed++;
    ++*n_retired;
    if (r.cancelled) {  // cancelled while running: its result is dropped
      P->reqs.erase(r.id);
      continue;
    }
    P->done_unreported.push_back(r.id);
  }
  P->stats.bytes_in_use = P->arena.in_use();
  bool busy = false;
  for (const Slot& s : P->slots) busy = busy || s.req >= 0;
  if (!busy) {  // every admission pass has finished: drop its graph and event
    for (csim_pool::Wave& w : P->waves) {
      if (w.exec) cudaGraphExecDestroy(w.exec);
      if (w.done) cudaEventDestroy(w.done);
      if (w.start) cudaEventDestroy(w.start);
    }
    P->waves.clear();
  }
  return CSIM_OK;
}

void destroy_pool(csim_pool* P) {
  for (Slot& s : P->slots) {
    if (s.st) cudaStreamSynchronize(s.st);
  }
  if (P->origin) cudaStreamSynchronize(P->origin);
  for (csim_pool::Wave& w : P->waves) {
    if (w.exec) cudaGraphExecDestroy(w.exec);
    if (w.done) cudaEventDestroy(w.done);
    if (w.start) cudaEventDestroy(w.start);
  }
  for (Slot& s : P->slots) {
    if (s.ev0) cudaEventDestroy(s.ev0);
    if (s.ev1) cudaEventDestroy(s.ev1);
    if (s.d_pat) cudaFree(s.d_pat);
    if (s.d_partial) cudaFree(s.d_partial);
    if (s.d_out) cudaFree(s.d_out);
    if (s.d_npart) cudaFree(s.d_npart);
    if (s.h_stage) cudaFreeHost(s.h_stage);
    if (s.h_out) cudaFreeHost(s.h_out);
    if (s.h_amps) cudaFreeHost(s.h_amps);
    if (s.h_flag) cudaFreeHost(s.h_flag);
    if (s.st) cudaStreamDestroy(s.st);
  }
  if (P->epoch) cudaEventDestroy(P->epoch);
  if (P->upload) {
    cudaStreamSynchronize(P->upload);
    cudaStreamDestroy(P->upload);
  }
  if (P->origin) cudaStreamDestroy(P->origin);
  if (P->d_arena) cudaFree(P->d_arena);
  delete P;
}

}  // namespace

extern "C" {

csim_status csim_pool_create(const csim_pool_opts* opts, csim_pool** out) {
  if (!out) return pfail(CSIM_ERR_ARG, "null argument");
  *out = nullptr;
  csim_pool* P = new (std::nothrow) csim_pool();
  if (!P) return pfail(CSIM_ERR_OOM, "host allocation");
  if (opts) P->o = *opts;
  if (P->o.n_streams <= 0) P->o.n_streams = 4;
  if (P->o.n_streams > 64) P->o.n_streams = 64;
  if (P->o.max_qubits <= 0) P->o.max_qubits = 32;
  if (P->o.min_block == 0) P->o.min_block = 1u << 20;
  if (P->o.min_block % 256u != 0) {
    delete P;
    return pfail(CSIM_ERR_ARG, "min_block must be a multiple of 256 bytes");
  }
  cudaError_t e = cudaSuccess;
  if (P->o.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
      delete P;
      return pcuda(e, "csim_pool_create");
    }
    P->o.hbm_budget = (uint64_t)(0.9 * (double)fr);
  }
  const uint64_t cap = P->o.hbm_budget / P->o.min_block * P->o.min_block;
  e = cudaMalloc(&P->d_arena, cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete P;
    return pfail(CSIM_ERR_OOM, "csim_pool_create: arena of " + std::to_string(cap) + " bytes");
  }
  P->arena.init(cap, P->o.min_block);
  P->stats.budget = P->arena.capacity();
  P->slots.resize(P->o.n_streams);
  for (Slot& s : P->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&s.ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&s.ev1);
    if (e == cudaSuccess) e = cudaMalloc(&s.d_pat, 2 * kMaxPatterns * sizeof(uint64_t));
    if (e == cudaSuccess)
      e = cudaMalloc(&s.d_partial, 2 * csim::norm_partials_needed() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s.d_out, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s.d_npart, csim::kNormPartCap * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_out, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_flag, sizeof(uint32_t));
    if (e == cudaSuccess) *s.h_flag = 0;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->origin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->upload, cudaStreamNonBlocking);
  // pinned staging for typical requests now: growing it later (a pinned
  // allocation) would stall the device work of the requests in flight
  for (Slot& s : P->slots)
    if (e == cudaSuccess) e = grow_pinned(&s, 256u << 10, 2u << 20);
  if (e == cudaSuccess) e = cudaEventCreate(&P->epoch);
  if (e == cudaSuccess) e = cudaEventRecord(P->epoch, P->origin);
  // load every kernel and fill the launch-configuration caches now: a lazy
  // module load must not happen inside a graph capture
  if (e == cudaSuccess) e = csim::warm_kernels();
  if (e == cudaSuccess && P->o.persistent) e = csim::warm_batch();
  if (e != cudaSuccess) {
    cudaGetLastError();
    destroy_pool(P);
    return pcuda(e, "csim_pool_create");
  }
  *out = P;
  return CSIM_OK;
}

csim_status csim_pool_submit(csim_pool* P, csim_circuit* c, const double* f0, csim_precision prec,
                             int64_t* id) {
  if (!P || !c || !f0 || !id) return pfail(CSIM_ERR_ARG, "null argument");
  if (prec != CSIM_C64 && prec != CSIM_C128) return pfail(CSIM_ERR_ARG, "bad precision");
  *id = 0;
  P->stats.submitted++;
  if (c->L.n > P->o.max_qubits) {
    P->stats.rejected++;
    return pfail(CSIM_ERR_TOO_LARGE, "csim_pool_submit: " + std::to_string(c->L.n) +
                                         " qubits exceed the pool's cap of " +
                                         std::to_string(P->o.max_qubits));
  }
  if ((int)c->pm.size() > kMaxPatterns) return pfail(CSIM_ERR_ARG, "too many mask patterns");
  std::string err;
  // a stream of its own for program uploads: the upload waits for itself,
  // not for the requests already running on the slots
  if (!csim::ensure_program(c, P->upload, &err)) return pfail(CSIM_ERR_CUDA, err);
  Request r;
  if (!csim::circuit_rhs(c, f0, &r.idx, &r.val, &err)) return pfail(CSIM_ERR_ARG, err);
  r.c = c;
  r.prec = prec;
  // source-index tables from the arena, unless the program has its own (from a
  // csim_run) or the request only fits without them
  r.ntab = c->prog.d_src.empty() ? csim::plan_src_index(&c->prog, kMaxPoolTables) : 0;
  request_sizes(c, prec, r.idx.size(), r.ntab, r.sizes, &r.count);
  if (r.ntab > 0 && !fits_empty(P->arena.capacity(), P->arena.min_block(), r.sizes, kAllocs)) {
    r.ntab = 0;
    request_sizes(c, prec, r.idx.size(), 0, r.sizes, &r.count);
  }
  if (!fits_empty(P->arena.capacity(), P->arena.min_block(), r.sizes, kAllocs)) {
    P->stats.rejected++;
    return pfail(CSIM_ERR_TOO_LARGE, "csim_pool_submit: the request's device memory exceeds "
                                     "the pool's budget");
  }
  r.id = P->next_id++;
  r.t_submit = now_s();
  *id = r.id;
  P->queue.push_back(r.id);
  P->reqs.emplace(r.id, std::move(r));
  int n = 0;
  csim_status s = retire(P, &n);
  // persistent mode admits at the next poll, so that a burst of submissions
  // forms one pass
  if (s == CSIM_OK && !P->o.persistent) s = admit(P);
  P->stats.queued = (int64_t)P->queue.size();
  return s;
}

csim_status csim_pool_poll(csim_pool* P, int32_t wait_ms, int64_t* done, size_t cap,
                           size_t* n_done) {
  if (!P) return pfail(CSIM_ERR_ARG, "null argument");
  const double t_end = now_s() + (wait_ms > 0 ? wait_ms * 1e-3 : 0.0);
  for (;;) {
    int n = 0;
    csim_status s = retire(P, &n);
    if (s == CSIM_OK) s = admit(P);
    if (s != CSIM_OK) return s;
    bool running = false;
    for (const Slot& sl : P->slots) running = running || sl.req >= 0;
    if (!P->done_unreported.empty() || !running || now_s() >= t_end) break;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  const size_t k = std::min(cap, P->done_unreported.size());
  if (done && k) std::memcpy(done, P->done_unreported.data(), k * sizeof(int64_t));
  P->done_unreported.erase(P->done_unreported.begin(), P->done_unreported.begin() + (done ? k : 0));
  if (n_done) *n_done = done ? k : 0;
  int64_t running = 0;
  for (const Slot& sl : P->slots) running += sl.req >= 0;
  P->stats.running = running;
  P->stats.queued = (int64_t)P->queue.size();
  return CSIM_OK;
}

csim_status csim_pool_result(csim_pool* P, int64_t id, double* p_success, double* norm_total,
                             double* out_amps, size_t cap, size_t* len, double* times) {
  if (!P) return pfail(CSIM_ERR_ARG, "null argument");
  auto it = P->reqs.find(id);
  if (it == P->reqs.end()) return pfail(CSIM_ERR_ARG, "unknown request id");
  Request& r = it->second;
  if (r.st != RState::Done) return pfail(CSIM_ERR_STATE, "request not finished");
  if (r.err != CSIM_OK) {  // failed before its device work: report and release
    const csim_status err = r.err;
    const std::string msg = r.err_msg;
    P->reqs.erase(it);
    return pfail(err, msg);
  }
  if (len) *len = r.count;
  if (out_amps) {
    if (cap < r.count) return pfail(CSIM_ERR_ARG, "out_amps too small");
    std::memcpy(out_amps, r.amps.data(), r.count * 16);
  }
  if (p_success) *p_success = r.p;
  if (norm_total) *norm_total = r.tot;
  if (times) {
    times[0] = r.t_start - r.t_submit;  // queueing
    times[1] = r.t_done - r.t_submit;   // submit to retirement
    times[2] = r.dev_ms * 1e-3;         // device time of the request's stream work
    times[3] = r.dev_t0;                // device start and end after the pool's epoch,
    times[4] = r.dev_t1;                // -1 for requests run inside a graph
  }
  P->reqs.erase(it);
  return CSIM_OK;
}

csim_status csim_pool_cancel(csim_pool* P, int64_t id) {
  if (!P) return pfail(CSIM_ERR_ARG, "null argument");
  auto it = P->reqs.find(id);
  if (it == P->reqs.end() || it->second.cancelled) return pfail(CSIM_ERR_ARG, "unknown request id");
  Request& r = it->second;
  P->stats.cancelled++;
  if (r.st == RState::Queued) {
    P->queue.erase(std::find(P->queue.begin(), P->queue.end(), id));
    P->stats.queued = (int64_t)P->queue.size();
    P->reqs.erase(it);
  } else if (r.st == RState::Running) {
    r.cancelled = true;  // its device work finishes; retirement frees it and drops the result
  } else {
    P->done_unreported.erase(std::remove(P->done_unreported.begin(), P->done_unreported.end(), id),
                             P->done_unreported.end());
    P->reqs.erase(it);
  }
  // memory or a slot may have been freed: admit what now fits
  int n = 0;
  csim_status s = retire(P, &n);
  if (s == CSIM_OK) s = admit(P);
  return s;
}

csim_status csim_pool_inject(csim_pool* P, int32_t what, int64_t id) {
  if (!P) return pfail(CSIM_ERR_ARG, "null argument");
  if (what != CSIM_INJECT_NONE && what != CSIM_INJECT_PINNED && what != CSIM_INJECT_ARENA &&
      what != CSIM_INJECT_BATCH_SIGNAL)
    return pfail(CSIM_ERR_ARG, "unknown fault kind");
  if (what == CSIM_INJECT_NONE)
    P->inject.erase(id);
  else
    P->inject[id] = what;
  return CSIM_OK;
}

csim_status csim_pool_stats(const csim_pool* P, csim_pool_stats_t* out) {
  if (!P || !out) return pfail(CSIM_ERR_ARG, "null argument");
  *out = P->stats;
  return CSIM_OK;
}

csim_status csim_pool_free(csim_pool* P) {
  if (!P) return CSIM_OK;
  destroy_pool(P);
  return CSIM_OK;
}

csim_status csim_pool_plan(uint64_t budget, uint64_t min_block, int32_t n_streams, size_t count,
                           const uint64_t* alloc_bytes, const double* arrival,
                           const double* duration, double* start, double* finish,
                           uint64_t* peak_bytes) {
  if (!alloc_bytes || !duration || !start || !finish || n_streams <= 0)
    return pfail(CSIM_ERR_ARG, "bad argument");
  if (min_block == 0) min_block = 1u << 20;
  BuddyArena a;
  a.init(budget / min_block * min_block, min_block);
  struct Run {
    double t_end;
    size_t i;
    uint64_t offs[kPlanAllocs];
  };
  std::vector<Run> running;
  std::deque<size_t> queue;
  std::vector<size_t> order(count);
  for (size_t i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
    return (arrival ? arrival[x] : 0.0) < (arrival ? arrival[y] : 0.0);
  });
  size_t next = 0;
  double t = 0.0;
  uint64_t peak = 0;
  for (size_t i = 0; i < count; ++i) start[i] = finish[i] = -1.0;
  for (;;) {
    // arrivals up to t
    while (next < count && (arrival ? arrival[order[next]] : 0.0) <= t) {
      const size_t i = order[next++];
      if (fits_empty(a.capacity(), min_block, alloc_bytes + kPlanAllocs * i, kPlanAllocs))
        queue.push_back(i);
    }
    // admit FIFO
    while (!queue.empty() && (int)running.size() < n_streams) {
      Run r{};
      r.i = queue.front();
      if (!alloc_all(&a, alloc_bytes + kPlanAllocs * r.i, r.offs, kPlanAllocs)) break;
      queue.pop_front();
      start[r.i] = t;
      r.t_end = t + duration[r.i];
      running.push_back(r);
      peak = std::max(peak, a.in_use());
    }
    // next event: a completion or an arrival
    double tn = 1e300;
    for (const Run& r : running) tn = std::min(tn, r.t_end);
    if (next < count) tn = std::min(tn, arrival ? arrival[order[next]] : 0.0);
    if (tn >= 1e300) break;
    t = std::max(t, tn);
    for (size_t k = 0; k < running.size();) {
      if (running[k].t_end <= t) {
        finish[running[k].i] = running[k].t_end;
        release_all(&a, running[k].offs, kPlanAllocs);
        running[k] = running.back();
        running.pop_back();
      } else {
        ++k;
      }
    }
  }
  if (peak_bytes) *peak_bytes = peak;
  return CSIM_OK;
}

}  // extern "C"
