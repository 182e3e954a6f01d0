// C ABI of include/csim.h: handle management, argument checking, device
// allocation and the run/postselect sequence.  No exception crosses the ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fuse.h"
#include "handles.h"
#include "internal.h"
#include "kernels.h"

using csim::Gate;
using csim::Layout;
using csim::Program;

namespace {
thread_local std::string g_err;

// Distinct gather chains that get a source-index table: a QSVT circuit has
// one or two (U_L^dag, and U_L when it is not fused into a conjugated sweep);
// a gate stream with more keeps the lookup chains.
constexpr int kSrcIndexTables = 2;

csim_status fail(csim_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
csim_status cuda_fail(cudaError_t e, const char* where) {
  return fail(CSIM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
}  // namespace

namespace csim {
// Lets entry points defined in other translation units set the message that
// csim_last_error returns on this thread.
void record_last_error(const std::string& msg) { g_err = msg; }
}  // namespace csim

namespace {


// Upload b (idx, val) and write the state: the whole state (memset and
// scatter), or with map the tiles of b only (launch_init_sparse).
cudaError_t write_initial_state(csim_circuit* c, const std::vector<uint64_t>& idx,
                                const std::vector<double>& val, uint32_t* map) {
  uint64_t* d_idx = nullptr;
  double* d_val = nullptr;
  cudaError_t e = cudaMallocAsync(&d_idx, idx.size() * sizeof(uint64_t), c->stream);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_val, val.size() * sizeof(double), c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_idx, idx.data(), idx.size() * sizeof(uint64_t), cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_val, val.data(), val.size() * sizeof(double), cudaMemcpyHostToDevice,
                        c->stream);
  c->cur = 0;
  if (e == cudaSuccess)
    e = map ? csim::launch_init_sparse(c->buf[0], c->prec, c->L.n, d_idx, d_val,
                                       (int64_t)idx.size(), map, c->stream)
            : csim::launch_init(c->buf[0], c->prec, (uint64_t)1 << c->L.n, d_idx, d_val,
                                (int64_t)idx.size(), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (d_idx) cudaFreeAsync(d_idx, c->stream);
  if (d_val) cudaFreeAsync(d_val, c->stream);
  return e;
}

// Before the state is read (or handed out) while a sparse init's zero fill is
// incomplete: zero the unmarked tiles.  The leading sweeps map those tiles to
// themselves and zero to zero, so this gives the state at any step before
// the fill completes.
cudaError_t materialize(csim_circuit* c) {
  if (!c->zero_fill) return cudaSuccess;
  c->zero_fill = false;
  cudaError_t e = csim::launch_zero_unmarked(c->buf[c->cur], c->prec, c->L.n, c->d_zmap, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e;
}

// The zero map for the run from the next step, and how many leading steps
// take it: those of a sparse init while the program still starts with the
// same sweeps.  Otherwise (the execution mode changed since csim_init, say)
// the state is completed first.
cudaError_t zero_map_for_run(csim_circuit* c, const uint32_t** zmap, int* zsteps) {
  *zmap = nullptr;
  *zsteps = 0;
  if (!c->zero_fill) return cudaSuccess;
  if (c->next_step < c->zero_steps && csim::zero_fill_steps(c, c->prec) == c->zero_steps) {
    *zmap = c->d_zmap;
    *zsteps = c->zero_steps;
    return cudaSuccess;
  }
  return materialize(c);
}

void free_device(csim_circuit* c) {
  for (void*& b : c->buf) {
    if (b) cudaFree(b);
    b = nullptr;
  }
  if (c->d_zmap) cudaFree(c->d_zmap);
  c->d_zmap = nullptr;
  c->zero_fill = false;
  c->zero_steps = 0;
  if (c->d_pat) cudaFree(c->d_pat);
  if (c->d_partial) cudaFree(c->d_partial);
  if (c->d_out) cudaFree(c->d_out);
  if (c->d_compact) cudaFree(c->d_compact);
  if (c->d_npart) cudaFree(c->d_npart);
  c->d_npart = nullptr;
  c->norm_fused = false;
  c->d_pat = nullptr;
  c->d_partial = nullptr;
  c->d_out = nullptr;
  c->d_compact = nullptr;
  c->compact_cap = 0;
  c->bytes = 0;
  c->prec = -1;
  csim::free_program(&c->prog);
  c->prog_built = false;
}


// State buffers (two for the fused path's ping-pong) and the reduction
// work buffers, reused when the precision and size are unchanged.
csim_status alloc_state(csim_circuit* c, csim_precision prec) {
  const Layout& L = c->L;
  const size_t esz = prec == CSIM_C64 ? 8 : 16;
  const size_t bytes = ((size_t)1 << L.n) * esz;
  const int nbuf = c->exec == CSIM_EXEC_FUSED ? 2 : 1;
  if (c->prec != (int)prec || c->bytes != bytes || (nbuf == 2 && !c->buf[1])) {
    for (void*& b : c->buf) {
      if (b) cudaFree(b);
      b = nullptr;
    }
    c->bytes = 0;
    c->prec = -1;
    for (int k = 0; k < nbuf; ++k) {
      cudaError_t e = cudaMalloc(&c->buf[k], bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        for (void*& b : c->buf) {
          if (b) cudaFree(b);
          b = nullptr;
        }
        return fail(CSIM_ERR_OOM, "state allocation of " + std::to_string(bytes) + " bytes: " +
                                      cudaGetErrorString(e));
      }
    }
    c->bytes = bytes;
    c->prec = prec;
  }
  if (!c->d_pat) {
    cudaError_t e = cudaMalloc(&c->d_pat, 2 * 64 * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_partial, 2 * csim::norm_partials_needed() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_out, 2 * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_device(c);
      return fail(CSIM_ERR_OOM, "work buffers");
    }
  }
  return CSIM_OK;
}

}  // namespace

namespace csim {

uint64_t place_bits(const std::vector<int>& bits, uint64_t v) {
  uint64_t idx = 0;
  for (size_t j = 0; j < bits.size(); ++j) idx |= ((v >> j) & 1ull) << bits[j];
  return idx;
}

void ensure_built(csim_circuit* c) {
  if (c->prog_built && c->prog.mode == c->exec) return;
  csim::free_program(&c->prog);
  std::vector<Gate> all = csim::build_qsvt(c->L, c->UL, c->phases);
  csim::build_program(all, c->L.n, c->exec, &c->prog);
  c->prog_built = true;
}

// Sparse initialisation (csim_init and pool requests) unless
// CSIM_SPARSE_INIT=0.
bool sparse_init_enabled() {
  static const bool v = [] {
    const char* e = std::getenv("CSIM_SPARSE_INIT");
    return !(e && e[0] == '0');
  }();
  return v;
}

// Sweeps at the start of the program that complete a sparse init's zero
// fill (launch_init_sparse) for a state of precision prec: 2 when the first
// is an in-place tile sweep and the second an in-place gather sweep whose
// kernels take the zero map (modes 2 and 3), 1 when only the first does
// (mode 1), else 0.  Neither leading sweep writes the second state buffer.
int zero_fill_steps(const csim_circuit* c, int prec) {
  const Program& P = c->prog;
  if (P.mode != CSIM_EXEC_FUSED || P.steps.empty() || c->L.n < 12) return 0;
  const Step& s0 = P.steps[0];
  if (s0.kind != 0 || s0.gather || sweep_zero_kind(prec, c->L.n, P.params[(size_t)s0.param]) != 1)
    return 0;
  if (P.steps.size() > 1) {
    const Step& s1 = P.steps[1];
    if (s1.kind == 0 && s1.gather && s1.inplace &&
        sweep_zero_kind(prec, c->L.n, P.params[(size_t)s1.param]) == 3)
      return 2;
  }
  return 1;
}

bool ensure_program(csim_circuit* c, cudaStream_t st, std::string* err) {
  ensure_built(c);
  if (c->prog.uploaded) return true;
  cudaError_t e = csim::upload_program(&c->prog, st);
  if (e != cudaSuccess) {
    *err = std::string("program upload: ") + cudaGetErrorString(e);
    csim::free_program(&c->prog);
    return false;
  }
  return true;
}

bool circuit_rhs(const csim_circuit* c, const double* f0, std::vector<uint64_t>* idx,
                 std::vector<double>* val, std::string* err) {
  const Layout& L = c->L;
  const size_t nf = (size_t)L.Nx * 3;
  for (size_t i = 0; i < nf; ++i)
    if (!std::isfinite(f0[i])) {
      *err = "f0 has a non-finite entry";
      return false;
    }
  idx->clear();
  val->clear();
  double nrm2 = 0.0;
  for (int a = 0; a < L.Nx; ++a)
    for (int q = 0; q < 3; ++q) {
      const double v = f0[a * 3 + q];
      nrm2 += v * v;
      if (v != 0.0) {
        idx->push_back(place_bits(L.a1, a) | place_bits(L.q1, q));
        val->push_back(v);
      }
    }
  if (L.NC == 2) {
    for (int a1 = 0; a1 < L.Nx; ++a1)
      for (int q1 = 0; q1 < 3; ++q1)
        for (int a2 = 0; a2 < L.Nx; ++a2)
          for (int q2 = 0; q2 < 3; ++q2) {
            const double v = f0[a1 * 3 + q1] * f0[a2 * 3 + q2];
            nrm2 += v * v;
            if (v != 0.0) {
              idx->push_back(place_bits(L.a1, a1) | place_bits(L.q1, q1) | place_bits(L.a2, a2) |
                             place_bits(L.q2, q2) | place_bits(L.ord, 1));
              val->push_back(v);
            }
          }
  }
  if (!(nrm2 > 0)) {
    *err = "f0 is zero";
    return false;
  }
  const double inv = 1.0 / std::sqrt(nrm2);
  for (double& v : *val) v *= inv;
  return true;
}

void mask_low_bits(const csim_circuit* c, int* lowk, uint64_t* lowv) {
  const int npat = (int)c->pm.size();
  int k = 0;
  uint64_t v = 0;
  while (npat > 0 && k < c->L.n) {
    const uint64_t b = 1ull << k;
    bool all = true;
    for (int j = 0; j < npat; ++j)
      all = all && (c->pm[j] & b) && ((c->pv[j] & b) == (c->pv[0] & b));
    if (!all) break;
    v |= c->pv[0] & b;
    ++k;
  }
  *lowk = k;
  *lowv = v;
}

CompactGeom compact_geom(const csim_circuit* c) {
  const Layout& L = c->L;
  CompactGeom g;
  g.free_shift = 2 + L.niL;
  g.m_shift = L.m[0];
  g.free_bits = g.m_shift - g.free_shift;
  g.count = (((uint64_t)1 << L.nm) - (uint64_t)L.Nt) << g.free_bits;
  return g;
}

}  // namespace csim

extern "C" {

const char* csim_last_error(void) { return g_err.c_str(); }

csim_status csim_build_ex(const csim_build_opts* o, csim_circuit** out) {
  if (!o || !out) return fail(CSIM_ERR_ARG, "null argument");
  *out = nullptr;
  if (!(o->tau > 0) || !(o->dt > 0) || !std::isfinite(o->tau) || !std::isfinite(o->dt))
    return fail(CSIM_ERR_ARG, "tau and dt must be positive and finite");
  if (o->bc != CSIM_BC_PERIODIC && o->bc != CSIM_BC_BOUNCEBACK)
    return fail(CSIM_ERR_ARG, "bc must be CSIM_BC_PERIODIC or CSIM_BC_BOUNCEBACK");
  Layout L;
  std::string err;
  if (!csim::make_layout(o->Nx, o->N_C, o->K, o->Nt, &L, &err)) return fail(CSIM_ERR_ARG, err);
  L.bc = o->bc;
  const int maxq = o->max_qubits > 0 ? o->max_qubits : 34;
  if (L.n > maxq || L.n > 62)
    return fail(CSIM_ERR_TOO_LARGE, "circuit needs " + std::to_string(L.n) + " qubits > limit " +
                                        std::to_string(maxq));
  csim_circuit* c = new (std::nothrow) csim_circuit();
  if (!c) return fail(CSIM_ERR_OOM, "host allocation");
  c->L = L;
  c->tau = o->tau;
  c->dt = o->dt;
  c->max_qubits = maxq;
  c->eps = o->eps > 0 ? o->eps : 1e-3;
  c->Lmax = csim::lmax_value(o->tau, o->N_C, o->dt, o->bc);
  c->lambda = std::ldexp(1.0, L.niL) * c->Lmax;
  try {
    c->UL = csim::build_UL(L, o->tau, o->dt);
  } catch (const std::exception& ex) {
    delete c;
    return fail(CSIM_ERR_ARG, ex.what());
  }
  csim::postselect_patterns(L, &c->pm, &c->pv);
  if (o->phases) {
    if (o->n_phases < 2 || o->n_phases % 2 != 0) {
      delete c;
      return fail(CSIM_ERR_ARG, "n_phases must be d+1 with d odd");
    }
    c->phases.assign(o->phases, o->phases + o->n_phases);
    c->d = o->n_phases - 1;
    c->kappa = o->kappa_qsvt;
    c->scale = 0.0;
  } else {
    c->kappa = o->kappa_qsvt;
    if (!(c->kappa > 0)) {
      c->kappa = csim::kappa_of_L(L, o->tau, o->dt, &err);
      if (!(c->kappa > 0)) {
        delete c;
        return fail(CSIM_ERR_NUMERIC, err);
      }
    }
    if (!(c->kappa > 1.0)) {
      delete c;
      return fail(CSIM_ERR_ARG, "kappa_qsvt must exceed 1");
    }
    c->d = o->d > 0 ? o->d : csim::degree_from_kappa(c->kappa, c->eps);
    if (c->d % 2 == 0) {
      delete c;
      return fail(CSIM_ERR_ARG, "d must be odd");
    }
    if (!csim::solve_phases(c->kappa, c->d, &c->phases, &c->scale, &err)) {
      delete c;
      return fail(CSIM_ERR_NUMERIC, err);
    }
  }
  *out = c;
  return CSIM_OK;
}

csim_status csim_build(int32_t Nx, double tau, int32_t N_C, int32_t K, double dt, int32_t Nt,
                       csim_circuit** out) {
  csim_build_opts o;
  std::memset(&o, 0, sizeof(o));
  o.Nx = Nx;
  o.tau = tau;
  o.N_C = N_C;
  o.K = K;
  o.dt = dt;
  o.Nt = Nt;
  o.bc = CSIM_BC_PERIODIC;
  return csim_build_ex(&o, out);
}

csim_status csim_info(const csim_circuit* c, csim_info_t* out) {
  if (!c || !out) return fail(CSIM_ERR_ARG, "null argument");
  std::memset(out, 0, sizeof(*out));
  out->n_qubits = c->L.n;
  out->d = c->d;
  out->n_a = c->L.na;
  out->n_k = c->L.nk;
  out->n_m = c->L.nm;
  out->n_iL = c->L.niL;
  out->lambda_L = c->lambda;
  out->L_max = c->Lmax;
  out->kappa_qsvt = c->kappa;
  out->poly_scale = c->scale;
  out->n_gates_UL = (int64_t)c->UL.size();
  out->n_gates_total = (int64_t)c->d * ((int64_t)c->UL.size() + 3) + 5;
  out->amp_updates_run = 0.0;
  for (const Gate& g : c->UL) out->amp_updates_run += c->d * csim::gate_amp_updates(g, c->L.n);
  for (const Gate& g : csim::phase_gates(c->L, 0.0))
    out->amp_updates_run += (c->d + 1) * csim::gate_amp_updates(g, c->L.n);
  out->amp_updates_run += 2.0 * std::ldexp(1.0, c->L.n);
  out->n_sweeps_run = c->prog_built ? c->prog.passes : 0;
  out->state_bytes = c->bytes;
  out->n_src_tables = (int32_t)c->prog.d_src.size();
  out->sparse_init = c->sparse_init;
  return CSIM_OK;
}

csim_status csim_export_gates(const csim_circuit* c, int32_t which, csim_gate* buf, size_t cap,
                              size_t* len) {
  if (!c || !len) return fail(CSIM_ERR_ARG, "null argument");
  std::vector<Gate> all;
  const std::vector<Gate>* src = &c->UL;
  if (which == 1) {
    all = csim::build_qsvt(c->L, c->UL, c->phases);
    src = &all;
  } else if (which != 0) {
    return fail(CSIM_ERR_ARG, "which must be 0 (U_L) or 1 (QSVT)");
  }
  *len = src->size();
  if (buf) {
    if (cap < src->size()) return fail(CSIM_ERR_ARG, "buffer too small");
    std::memcpy(buf, src->data(), src->size() * sizeof(Gate));
  }
  return CSIM_OK;
}

csim_status csim_export_phases(const csim_circuit* c, double* buf, size_t cap, size_t* len) {
  if (!c || !len) return fail(CSIM_ERR_ARG, "null argument");
  *len = c->phases.size();
  if (buf) {
    if (cap < c->phases.size()) return fail(CSIM_ERR_ARG, "buffer too small");
    std::memcpy(buf, c->phases.data(), c->phases.size() * sizeof(double));
  }
  return CSIM_OK;
}

csim_status csim_export_mask(const csim_circuit* c, uint64_t* masks, uint64_t* vals, size_t cap,
                             size_t* len) {
  if (!c || !len) return fail(CSIM_ERR_ARG, "null argument");
  *len = c->pm.size();
  if (masks || vals) {
    if (!masks || !vals || cap < c->pm.size()) return fail(CSIM_ERR_ARG, "buffer too small");
    std::memcpy(masks, c->pm.data(), c->pm.size() * sizeof(uint64_t));
    std::memcpy(vals, c->pv.data(), c->pv.size() * sizeof(uint64_t));
  }
  return CSIM_OK;
}

csim_status csim_init(csim_circuit* c, const double* f0, csim_precision prec, void* stream) {
  if (!c || !f0) return fail(CSIM_ERR_ARG, "null argument");
  if (prec != CSIM_C64 && prec != CSIM_C128) return fail(CSIM_ERR_ARG, "bad precision");
  const Layout& L = c->L;
  // host: b = (f, f (x) f) normalised, in register coordinates
  std::vector<uint64_t> idx;
  std::vector<double> val;
  {
    std::string err;
    if (!csim::circuit_rhs(c, f0, &idx, &val, &err)) return fail(CSIM_ERR_ARG, err);
  }

  c->stream = (cudaStream_t)stream;
  {
    const csim_status st = alloc_state(c, prec);
    if (st != CSIM_OK) return st;
  }
  // sparse when the program's leading sweeps can write the zeros of the
  // tiles that b does not touch
  int zsteps = 0;
  if (csim::sparse_init_enabled() && c->exec == CSIM_EXEC_FUSED && L.n >= 12) {
    std::string err;
    if (csim::ensure_program(c, c->stream, &err)) zsteps = csim::zero_fill_steps(c, prec);
    if (zsteps > 0 && !c->d_zmap) {
      if (cudaMalloc(&c->d_zmap, ((size_t)1 << (L.n - 12)) * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        c->d_zmap = nullptr;
        zsteps = 0;
      }
    }
  }
  c->zero_fill = false;
  const cudaError_t e = write_initial_state(c, idx, val, zsteps > 0 ? c->d_zmap : nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "csim_init");
  c->zero_fill = zsteps > 0;
  c->zero_steps = zsteps;
  c->sparse_init = zsteps;
  c->loaded = true;
  c->ran = false;
  c->next_step = 0;
  c->norm_fused = false;
  return CSIM_OK;
}

csim_status csim_compile(csim_circuit* c) {
  if (!c) return fail(CSIM_ERR_ARG, "null argument");
  csim::ensure_built(c);
  return CSIM_OK;
}

csim_status csim_set_launch_shape(csim_precision prec, int32_t n_qubits, int32_t u, int32_t minb,
                                  int32_t waves) {
  if (prec != CSIM_C64 && prec != CSIM_C128) return fail(CSIM_ERR_ARG, "bad precision");
  if (n_qubits < 7 || n_qubits >= 64) return fail(CSIM_ERR_ARG, "qubit count out of range");
  if (u == 0) {
    csim::set_launch_shape(prec, n_qubits, nullptr);
    return CSIM_OK;
  }
  const csim::LaunchShape sh{u, minb, waves};
  if (!csim::valid_launch_shape(prec, sh)) return fail(CSIM_ERR_ARG, "unsupported launch shape");
  csim::set_launch_shape(prec, n_qubits, &sh);
  return CSIM_OK;
}

csim_status csim_tune_launch(csim_circuit* c, csim_precision prec, int32_t max_steps,
                             int32_t reps, csim_launch_tune_t* out) {
  if (!c || !out) return fail(CSIM_ERR_ARG, "null argument");
  if (prec != CSIM_C64 && prec != CSIM_C128) return fail(CSIM_ERR_ARG, "bad precision");
  if (max_steps < 1 || reps < 1) return fail(CSIM_ERR_ARG, "max_steps and reps must be positive");
  if (c->exec != CSIM_EXEC_FUSED) return fail(CSIM_ERR_ARG, "the launch tuner needs fused mode");
  *out = csim_launch_tune_t{};
  const int n = c->L.n;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "csim_tune_launch: stream");
  std::string err;
  if (!csim::ensure_program(c, st, &err)) {
    cudaStreamDestroy(st);
    return fail(CSIM_ERR_CUDA, err);
  }
  e = csim::build_src_index(&c->prog, st, kSrcIndexTables);
  const size_t bytes = ((size_t)1 << n) * (prec == CSIM_C64 ? 8 : 16);
  void* buf[2] = {nullptr, nullptr};
  if (e == cudaSuccess) e = cudaMalloc(&buf[0], bytes);
  if (e == cudaSuccess && c->prog.pingpong) e = cudaMalloc(&buf[1], bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    if (buf[0]) cudaFree(buf[0]);
    cudaStreamDestroy(st);
    return fail(CSIM_ERR_OOM, "csim_tune_launch: scratch state");
  }
  // finite amplitudes of about 0.01: every trial does real arithmetic
  if (e == cudaSuccess) e = cudaMemsetAsync(buf[0], 0x3c, bytes, st);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const int64_t last = std::min<int64_t>((int64_t)c->prog.steps.size(), max_steps);
  // candidates: the default first, then the other kernel variants and grids
  const csim::LaunchShape def = csim::default_launch_shape(prec);
  std::vector<csim::LaunchShape> cand{def};
  const int uvals[] = {1, 2, 4}, mvals[] = {1, 2, 4}, wvals[] = {1, 2, 4, 8};
  for (int u : uvals)
    for (int m : mvals) {
      if (u == 4 && m == 4) continue;  // no such kernel (launch_sweep runs it as 1, 4)
      for (int w : wvals) {
        const csim::LaunchShape x{u, m, w};
        if (x.u == def.u && x.minb == def.minb && x.waves == def.waves) continue;
        // the default kernel at other grids, and other kernels at the default grid
        if (!(x.u == def.u && x.minb == def.minb) && x.waves != def.waves) continue;
        cand.push_back(x);
      }
    }
  csim::LaunchShape saved;
  const bool had = csim::launch_shape_for(prec, n, &saved);
  double best = 1e300;
  csim::LaunchShape pick = def;
  for (const csim::LaunchShape& x : cand) {
    if (e != cudaSuccess) break;
    csim::set_launch_shape(prec, n, &x);
    int cur = 0;
    e = csim::run_program_steps(c->prog, buf, &cur, prec, st, 0, last);  // untimed
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r)
      e = csim::run_program_steps(c->prog, buf, &cur, prec, st, 0, last);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) break;
    const double per = (double)ms / reps;
    if (out->n_trials < 32) {
      const int k = out->n_trials++;
      out->trial_u[k] = x.u;
      out->trial_minb[k] = x.minb;
      out->trial_waves[k] = x.waves;
      out->trial_ms[k] = per;
    }
    if (&x == &cand.front()) out->ms_default = per;
    if (per < best) {
      best = per;
      pick = x;
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  for (void* q : buf)
    if (q) cudaFree(q);
  cudaStreamDestroy(st);
  if (e != cudaSuccess) {
    if (had)
      csim::set_launch_shape(prec, n, &saved);
    else
      csim::set_launch_shape(prec, n, nullptr);
    return cuda_fail(e, "csim_tune_launch");
  }
  csim::set_launch_shape(prec, n, &pick);
  out->u = pick.u;
  out->minb = pick.minb;
  out->waves = pick.waves;
  out->ms = best;
  out->steps = (int32_t)last;
  return CSIM_OK;
}

csim_status csim_set_exec(csim_circuit* c, csim_exec mode) {
  if (!c) return fail(CSIM_ERR_ARG, "null argument");
  if (mode != CSIM_EXEC_FUSED && mode != CSIM_EXEC_GATE) return fail(CSIM_ERR_ARG, "bad mode");
  c->exec = mode;
  return CSIM_OK;
}

// The fused-norm buffer of a run that reaches the program's last sweep, when
// that sweep can sum |a|^2 (nullptr otherwise, or when it cannot be
// allocated: the norms are then read separately).
double* fused_norm_buffer(csim_circuit* c) {
  if (!csim::program_fuses_norm(c->prog, c->prec)) return nullptr;
  if (!c->d_npart && cudaMalloc(&c->d_npart, csim::kNormPartCap * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    c->d_npart = nullptr;
  }
  return c->d_npart;
}

csim_status csim_run(csim_circuit* c) {
  if (!c) return fail(CSIM_ERR_ARG, "null argument");
  if (!c->loaded) return fail(CSIM_ERR_STATE, "csim_run needs a fresh csim_init");
  std::string err;
  if (!csim::ensure_program(c, c->stream, &err)) return fail(CSIM_ERR_CUDA, err);
  if (c->prog.pingpong && !c->buf[1]) {
    cudaError_t e = cudaMalloc(&c->buf[1], c->bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->buf[1] = nullptr;
      return fail(CSIM_ERR_OOM, "second state buffer");
    }
  }
  cudaError_t e = csim::build_src_index(&c->prog, c->stream, kSrcIndexTables);
  if (e != cudaSuccess) return cuda_fail(e, "csim_run: source index");
  const uint32_t* zmap = nullptr;
  int zsteps = 0;
  e = zero_map_for_run(c, &zmap, &zsteps);
  if (e != cudaSuccess) return cuda_fail(e, "csim_run: initial state");
  double* npart = fused_norm_buffer(c);
  c->norm_fused = false;
  e = csim::run_program_steps(c->prog, c->buf, &c->cur, c->prec, c->stream, c->next_step,
                              (int64_t)c->prog.steps.size(), nullptr, zmap, zsteps, npart);
  c->zero_fill = false;
  if (e != cudaSuccess) return cuda_fail(e, "csim_run");
  c->norm_fused = npart != nullptr && !c->prog.steps.empty();
  c->next_step = (int64_t)c->prog.steps.size();
  c->loaded = false;
  c->ran = true;
  return CSIM_OK;
}

csim_status csim_run_steps(csim_circuit* c, int64_t n_steps, int64_t* next_step) {
  if (!c || n_steps < 0) return fail(CSIM_ERR_ARG, "bad argument");
  if (!c->loaded) return fail(CSIM_ERR_STATE, "csim_run_steps needs csim_init or csim_restore");
  std::string err;
  if (!csim::ensure_program(c, c->stream, &err)) return fail(CSIM_ERR_CUDA, err);
  if (c->prog.pingpong && !c->buf[1]) {
    cudaError_t e = cudaMalloc(&c->buf[1], c->bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->buf[1] = nullptr;
      return fail(CSIM_ERR_OOM, "second state buffer");
    }
  }
  const int64_t total = (int64_t)c->prog.steps.size();
  const int64_t last = std::min(total, c->next_step + n_steps);
  cudaError_t e = csim::build_src_index(&c->prog, c->stream, kSrcIndexTables);
  if (e != cudaSuccess) return cuda_fail(e, "csim_run_steps: source index");
  const uint32_t* zmap = nullptr;
  int zsteps = 0;
  if (last > c->next_step) {
    e = zero_map_for_run(c, &zmap, &zsteps);
    if (e != cudaSuccess) return cuda_fail(e, "csim_run_steps: initial state");
  }
  double* npart = last == total && last > c->next_step ? fused_norm_buffer(c) : nullptr;
  if (last > c->next_step) c->norm_fused = false;
  e = csim::run_program_steps(c->prog, c->buf, &c->cur, c->prec, c->stream, c->next_step, last,
                              nullptr, zmap, zsteps, npart);
  if (last >= c->zero_steps) c->zero_fill = false;
  if (e != cudaSuccess) return cuda_fail(e, "csim_run_steps");
  if (npart) c->norm_fused = true;
  c->next_step = last;
  if (last == total) {
    c->loaded = false;
    c->ran = true;
  }
  if (next_step) *next_step = last;
  return CSIM_OK;
}

csim_status csim_checkpoint(csim_circuit* c, double* out, size_t cap_amps, int64_t* next_step) {
  if (!c || !out || !next_step) return fail(CSIM_ERR_ARG, "null argument");
  const csim_status s = csim_read_state(c, out, cap_amps);
  if (s != CSIM_OK) return s;
  *next_step = c->next_step;
  return CSIM_OK;
}

csim_status csim_restore(csim_circuit* c, const double* amps, size_t n_amps, csim_precision prec,
                         int64_t next_step, void* stream) {
  if (!c || !amps) return fail(CSIM_ERR_ARG, "null argument");
  if (prec != CSIM_C64 && prec != CSIM_C128) return fail(CSIM_ERR_ARG, "bad precision");
  const size_t N = (size_t)1 << c->L.n;
  if (n_amps != N) return fail(CSIM_ERR_ARG, "n_amps must be 2^n");
  csim::ensure_built(c);
  const int64_t total = (int64_t)c->prog.steps.size();
  if (next_step < 0 || next_step > total) return fail(CSIM_ERR_ARG, "next_step out of range");
  c->stream = (cudaStream_t)stream;
  {
    const csim_status st = alloc_state(c, prec);
    if (st != CSIM_OK) return st;
  }
  c->zero_fill = false;
  c->sparse_init = 0;
  c->norm_fused = false;
  cudaError_t e;
  c->cur = 0;
  if (prec == CSIM_C128) {
    e = cudaMemcpyAsync(c->buf[0], amps, N * 16, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  } else {
    std::vector<float> tmp(2 * N);
    for (size_t i = 0; i < 2 * N; ++i) tmp[i] = (float)amps[i];
    e = cudaMemcpyAsync(c->buf[0], tmp.data(), N * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "csim_restore");
  c->next_step = next_step;
  c->loaded = next_step < total;
  c->ran = !c->loaded;
  return CSIM_OK;
}

csim_status csim_sync(csim_circuit* c) {
  if (!c) return fail(CSIM_ERR_ARG, "null argument");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "csim_sync");
  return CSIM_OK;
}

csim_status csim_postselect(csim_circuit* c, double* out_amps, size_t cap, size_t* len,
                            double* p_success, double* norm_total) {
  if (!c) return fail(CSIM_ERR_ARG, "null argument");
  if (!c->buf[c->cur] || c->prec < 0) return fail(CSIM_ERR_STATE, "no state");
  {
    const cudaError_t e0 = materialize(c);
    if (e0 != cudaSuccess) return cuda_fail(e0, "csim_postselect");
  }
  const Layout& L = c->L;
  const int npat = (int)c->pm.size();
  std::vector<uint64_t> pat(c->pm);
  pat.insert(pat.end(), c->pv.begin(), c->pv.end());
  cudaError_t e = cudaMemcpyAsync(c->d_pat, pat.data(), pat.size() * sizeof(uint64_t),
                                  cudaMemcpyHostToDevice, c->stream);
  // low index bits fixed (to the same value) by every pattern
  int lowk = 0;
  uint64_t lowv = 0;
  csim::mask_low_bits(c, &lowk, &lowv);
  if (e == cudaSuccess)
    e = c->norm_fused
            ? csim::launch_norms_fused(c->buf[c->cur], c->prec, L.n, c->d_pat, c->d_pat + npat,
                                       npat, lowk, lowv, c->d_npart, c->d_partial, c->d_out,
                                       c->stream)
            : csim::launch_norms(c->buf[c->cur], c->prec, L.n, c->d_pat, c->d_pat + npat, npat,
                                 lowk, lowv, c->d_partial, c->d_out, c->stream);
  double h[2] = {0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h, c->d_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  const csim::CompactGeom cg = csim::compact_geom(c);
  const int free_shift = cg.free_shift, m_shift = cg.m_shift, free_bits = cg.free_bits;
  const uint64_t count = cg.count;
  if (len) *len = count;
  if (e == cudaSuccess && out_amps) {
    if (cap < count) return fail(CSIM_ERR_ARG, "out_amps too small");
    if (c->compact_cap < count) {
      if (c->d_compact) cudaFree(c->d_compact);
      c->d_compact = nullptr;
      c->compact_cap = 0;
      e = cudaMalloc(&c->d_compact, count * 2 * sizeof(double));
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CSIM_ERR_OOM, "postselect buffer");
      }
      c->compact_cap = count;
    }
    e = csim::launch_compact(c->buf[c->cur], c->prec, c->d_compact, count, free_shift, free_bits,
                             (uint64_t)L.Nt, m_shift, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out_amps, c->d_compact, count * 2 * sizeof(double),
                          cudaMemcpyDeviceToHost, c->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "csim_postselect");
  if (norm_total) *norm_total = h[0];
  if (p_success) *p_success = h[1];
  return CSIM_OK;
}

csim_status csim_final_distribution(const csim_circuit* c, const double* f0, const double* amps,
                                    size_t len, double* f_out) {
  if (!c || !f0 || !amps || !f_out) return fail(CSIM_ERR_ARG, "null argument");
  const Layout& L = c->L;
  const csim::CompactGeom g = csim::compact_geom(c);
  if (len < g.count) return fail(CSIM_ERR_ARG, "amps is shorter than the postselected block");
  // |v0|: the norm of the Carleman vector (f0, f0 (x) f0) that csim_init normalised
  double nrm2 = 0.0, n1 = 0.0;
  for (int i = 0; i < L.Nx * 3; ++i) n1 += f0[i] * f0[i];
  nrm2 = n1;
  if (L.NC == 2) nrm2 += n1 * n1;  // |f0 (x) f0|^2 = |f0|^4
  if (!(nrm2 > 0) || !std::isfinite(nrm2)) return fail(CSIM_ERR_ARG, "f0 is zero or not finite");
  const double factor = std::sqrt(nrm2) / (c->scale * c->lambda);
  const uint64_t fmask = ((uint64_t)1 << g.free_bits) - 1u;
  for (int a = 0; a < L.Nx; ++a)
    for (int q = 0; q < 3; ++q) {
      const uint64_t I = csim::place_bits(L.m, (uint64_t)L.Nt) | csim::place_bits(L.a1, (uint64_t)a) |
                         csim::place_bits(L.q1, (uint64_t)q);
      const uint64_t pos = (((I >> g.m_shift) - (uint64_t)L.Nt) << g.free_bits) |
                           ((I >> g.free_shift) & fmask);
      f_out[a * 3 + q] = amps[2 * pos] * factor;
    }
  return CSIM_OK;
}

csim_status csim_state_device(const csim_circuit* c, void** d_state, int32_t* n,
                              csim_precision* prec) {
  if (!c || !d_state) return fail(CSIM_ERR_ARG, "null argument");
  if (!c->buf[c->cur] || c->prec < 0) return fail(CSIM_ERR_STATE, "no state");
  {  // the handed-out state must be whole (a sparse init writes it now)
    const cudaError_t e = materialize(const_cast<csim_circuit*>(c));
    if (e != cudaSuccess) return cuda_fail(e, "csim_state_device");
  }
  *d_state = c->buf[c->cur];
  if (n) *n = c->L.n;
  if (prec) *prec = (csim_precision)c->prec;
  return CSIM_OK;
}

csim_status csim_read_state(csim_circuit* c, double* out, size_t cap_amps) {
  if (!c || !out) return fail(CSIM_ERR_ARG, "null argument");
  if (!c->buf[c->cur] || c->prec < 0) return fail(CSIM_ERR_STATE, "no state");
  const size_t N = (size_t)1 << c->L.n;
  if (cap_amps < N) return fail(CSIM_ERR_ARG, "buffer too small");
  cudaError_t e = materialize(c);
  if (e != cudaSuccess) return cuda_fail(e, "csim_read_state");
  if (c->prec == CSIM_C128) {
    e = cudaMemcpyAsync(out, c->buf[c->cur], N * 16, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  } else {
    std::vector<float> tmp(2 * N);
    e = cudaMemcpyAsync(tmp.data(), c->buf[c->cur], N * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    for (size_t i = 0; i < 2 * N; ++i) out[i] = tmp[i];
  }
  if (e != cudaSuccess) return cuda_fail(e, "csim_read_state");
  return CSIM_OK;
}

csim_status csim_free(csim_circuit* c) {
  if (!c) return CSIM_OK;
  if (c->stream || c->buf[0]) cudaStreamSynchronize(c->stream);
  free_device(c);
  delete c;
  return CSIM_OK;
}

// ------------------------------------------------------------ raw states
namespace {
csim_status sv_compile(csim_sv* s, const std::vector<Gate>& gl, csim_exec mode, bool allow_dense,
                       int stage_k, int dense_mode = -1);
}

csim_status csim_sv_create(int32_t n, csim_precision prec, void* stream, csim_sv** out) {
  if (!out) return fail(CSIM_ERR_ARG, "null argument");
  *out = nullptr;
  if (n < 1 || n > 34) return fail(CSIM_ERR_TOO_LARGE, "n must be in [1, 34]");
  if (prec != CSIM_C64 && prec != CSIM_C128) return fail(CSIM_ERR_ARG, "bad precision");
  csim_sv* s = new (std::nothrow) csim_sv();
  if (!s) return fail(CSIM_ERR_OOM, "host allocation");
  s->n = n;
  s->prec = prec;
  s->stream = (cudaStream_t)stream;
  s->bytes = ((size_t)1 << n) * (prec == CSIM_C64 ? 8 : 16);
  cudaError_t e = cudaMalloc(&s->buf[0], s->bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->buf[0], 0, s->bytes, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (s->buf[0]) cudaFree(s->buf[0]);
    delete s;
    return fail(CSIM_ERR_OOM, std::string("state allocation: ") + cudaGetErrorString(e));
  }
  if (csim::dense_timeouts(&s->timeouts_seen) != cudaSuccess) cudaGetLastError();
  *out = s;
  return CSIM_OK;
}

csim_status csim_sv_load(csim_sv* s, const double* amps, size_t n_amps) {
  if (!s || !amps) return fail(CSIM_ERR_ARG, "null argument");
  const size_t N = (size_t)1 << s->n;
  if (n_amps != N) return fail(CSIM_ERR_ARG, "n_amps must be 2^n");
  cudaError_t e;
  s->cur = 0;
  if (s->prec == CSIM_C128) {
    e = cudaMemcpyAsync(s->buf[0], amps, N * 16, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  } else {
    std::vector<float> tmp(2 * N);
    for (size_t i = 0; i < 2 * N; ++i) tmp[i] = (float)amps[i];
    e = cudaMemcpyAsync(s->buf[0], tmp.data(), N * 8, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "csim_sv_load");
  return CSIM_OK;
}

csim_status csim_sv_compile(csim_sv* s, const csim_gate* gates, size_t n_gates, csim_exec mode) {
  if (!s || (!gates && n_gates)) return fail(CSIM_ERR_ARG, "null argument");
  for (size_t i = 0; i < n_gates; ++i) {
    const csim_gate& g = gates[i];
    if (g.op > 3 || g.target >= s->n || ((g.cmask >> g.target) & 1ull) || (g.cval & ~g.cmask) ||
        (s->n < 64 && (g.cmask >> s->n)))
      return fail(CSIM_ERR_ARG, "invalid gate record " + std::to_string(i));
  }
  std::vector<Gate> gl(gates, gates + n_gates);
  return sv_compile(s, gl, mode, s->prec == CSIM_C64 && s->tune_dense != 0, s->tune_stage);
}

namespace {
csim_status sv_compile(csim_sv* s, const std::vector<Gate>& gl, csim_exec mode, bool allow_dense,
                       int stage_k, int dense_mode) {
  s->compiled = false;
  csim::free_program(&s->prog);
  csim::build_program(gl, s->n, mode, &s->prog, allow_dense, stage_k, dense_mode);
  cudaError_t e = csim::upload_program(&s->prog, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "csim_sv_compile");
  if (s->prog.pingpong && !s->buf[1]) {
    e = cudaMalloc(&s->buf[1], s->bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      s->buf[1] = nullptr;
      return fail(CSIM_ERR_OOM, "second state buffer");
    }
  }
  e = csim::build_src_index(&s->prog, s->stream, kSrcIndexTables);
  if (e != cudaSuccess) return cuda_fail(e, "csim_sv_compile: source index");
  s->compiled = true;
  return CSIM_OK;
}
}  // namespace

csim_status csim_sv_compile_opts(csim_sv* s, const csim_gate* gates, size_t n_gates,
                                 csim_exec mode, int32_t stage, int32_t dense) {
  if (!s || (!gates && n_gates)) return fail(CSIM_ERR_ARG, "null argument");
  if (stage < -1 || stage > csim::kMaxStage || dense < -1 || dense > 2)
    return fail(CSIM_ERR_ARG, "stage must be in [-1, 3] and dense in [-1, 2]");
  for (size_t i = 0; i < n_gates; ++i) {
    const csim_gate& g = gates[i];
    if (g.op > 3 || g.target >= s->n || ((g.cmask >> g.target) & 1ull) || (g.cval & ~g.cmask) ||
        (s->n < 64 && (g.cmask >> s->n)))
      return fail(CSIM_ERR_ARG, "invalid gate record " + std::to_string(i));
  }
  std::vector<Gate> gl(gates, gates + n_gates);
  return sv_compile(s, gl, mode, s->prec == CSIM_C64 && dense != 0, stage, dense);
}

csim_status csim_sv_autotune(csim_sv* s, const csim_gate* gates, size_t n_gates, int32_t reps,
                             csim_tune_t* out) {
  if (!s || !out || (!gates && n_gates)) return fail(CSIM_ERR_ARG, "null argument");
  if (reps < 1) return fail(CSIM_ERR_ARG, "reps must be at least 1");
  *out = csim_tune_t{};
  // validate through the plain compile first (and keep its program if the
  // trials fail)
  s->tune_stage = s->tune_dense = -1;
  csim_status st = csim_sv_compile(s, gates, n_gates, CSIM_EXEC_FUSED);
  if (st != CSIM_OK) return st;
  std::vector<Gate> gl(gates, gates + n_gates);
  void* saved = nullptr;
  cudaError_t e = cudaMalloc(&saved, s->bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(CSIM_ERR_OOM, "csim_sv_autotune: copy of the state");
  }
  e = cudaMemcpyAsync(saved, s->buf[s->cur], s->bytes, cudaMemcpyDeviceToDevice, s->stream);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  double best = 1e300;
  int best_k = 0, best_d = 0;
  const bool dense_ok = s->prec == CSIM_C64 && s->n >= 12;
  for (int d = 0; d <= (dense_ok ? 1 : 0) && e == cudaSuccess; ++d) {
    for (int k = 0; k <= csim::kMaxStage && e == cudaSuccess; ++k) {
      st = sv_compile(s, gl, CSIM_EXEC_FUSED, d == 1, k);
      if (st != CSIM_OK) break;
      if (d == 1 && !s->prog.dense_on) break;
      if (d == 1 && s->prog.stats.dense_blocks == 0) break;  // the same programs as without
      e = csim::run_program(s->prog, s->buf, &s->cur, s->prec, s->stream);  // untimed
      if (e == cudaSuccess) e = cudaEventRecord(a, s->stream);
      for (int r = 0; r < reps && e == cudaSuccess; ++r)
        e = csim::run_program(s->prog, s->buf, &s->cur, s->prec, s->stream);
      if (e == cudaSuccess) e = cudaEventRecord(b, s->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e != cudaSuccess) break;
      const double per = (double)ms / reps;
      if (out->n_trials < 8) {
        out->trial_stage[out->n_trials] = k;
        out->trial_dense[out->n_trials] = d;
        out->trial_ms[out->n_trials] = per;
        out->n_trials++;
      }
      if (per < best) {
        best = per;
        best_k = k;
        best_d = d;
      }
    }
  }
  // the state the caller loaded, then the fastest program
  if (e == cudaSuccess) {
    s->cur = 0;
    e = cudaMemcpyAsync(s->buf[0], saved, s->bytes, cudaMemcpyDeviceToDevice, s->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(saved);
  if (e != cudaSuccess) return cuda_fail(e, "csim_sv_autotune");
  if (st != CSIM_OK) return st;
  st = sv_compile(s, gl, CSIM_EXEC_FUSED, best_d == 1, best_k);
  if (st != CSIM_OK) return st;
  s->tune_stage = best_k;
  s->tune_dense = best_d;
  out->stage = best_k;
  out->dense = best_d;
  out->ms = best;
  return CSIM_OK;
}

csim_status csim_sv_run(csim_sv* s, int32_t reps) {
  if (!s) return fail(CSIM_ERR_ARG, "null argument");
  if (!s->compiled) return fail(CSIM_ERR_STATE, "compile a gate list first");
  for (int r = 0; r < reps; ++r) {
    cudaError_t e = csim::run_program(s->prog, s->buf, &s->cur, s->prec, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "csim_sv_run");
  }
  return CSIM_OK;
}

csim_status csim_sv_read(csim_sv* s, double* out, size_t n_amps) {
  if (!s || !out) return fail(CSIM_ERR_ARG, "null argument");
  const size_t N = (size_t)1 << s->n;
  if (n_amps < N) return fail(CSIM_ERR_ARG, "buffer too small");
  cudaError_t e;
  if (s->prec == CSIM_C128) {
    e = cudaMemcpyAsync(out, s->buf[s->cur], N * 16, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  } else {
    std::vector<float> tmp(2 * N);
    e = cudaMemcpyAsync(tmp.data(), s->buf[s->cur], N * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    for (size_t i = 0; i < 2 * N; ++i) out[i] = tmp[i];
  }
  if (e != cudaSuccess) return cuda_fail(e, "csim_sv_read");
  unsigned int to = 0;
  if (csim::dense_timeouts(&to) == cudaSuccess && to != s->timeouts_seen) {
    s->timeouts_seen = to;
    return fail(CSIM_ERR_TIMEOUT, "csim_sv_read: a dense block's wait for its tensor-core "
                                  "products ran out; the state is not valid");
  }
  return CSIM_OK;
}

csim_status csim_sv_apply_dense(csim_sv* s, const int32_t* qubits, const double* u,
                                int32_t engine) {
  if (!s || !qubits || !u) return fail(CSIM_ERR_ARG, "null argument");
  if (s->prec != CSIM_C64) return fail(CSIM_ERR_ARG, "dense blocks need a complex64 state");
  if (engine != csim::DENSE_TC && engine != csim::DENSE_FP32)
    return fail(CSIM_ERR_ARG, "unknown engine");
  if (s->n < (engine == csim::DENSE_TC ? 12 : 5))
    return fail(CSIM_ERR_ARG, "too few qubits for this engine");
  int order[5];
  for (int j = 0; j < 5; ++j) {
    if (qubits[j] < 0 || qubits[j] >= s->n) return fail(CSIM_ERR_ARG, "qubit out of range");
    for (int k = 0; k < j; ++k)
      if (qubits[k] == qubits[j]) return fail(CSIM_ERR_ARG, "repeated qubit");
    order[j] = j;
  }
  std::sort(order, order + 5, [&](int a, int b) { return qubits[a] < qubits[b]; });
  // element bit j of the caller's U is qubits[j]; the kernels take the
  // qubits ascending, so U's rows and columns are relabelled to that order
  auto relabel = [&](int x) {
    int y = 0;
    for (int j = 0; j < 5; ++j)
      if ((x >> order[j]) & 1) y |= 1 << j;
    return y;
  };
  csim::DenseBlock& b = s->dense;
  b.nsel = 0;
  for (int j = 0; j < 5; ++j) b.q[j] = (uint8_t)qubits[order[j]];
  b.u.assign(2 * 1024, 0.0);
  for (int r = 0; r < 32; ++r)
    for (int c = 0; c < 32; ++c) {
      const int r2 = relabel(r), c2 = relabel(c);
      b.u[2 * (32 * r2 + c2)] = u[2 * (32 * r + c)];
      b.u[2 * (32 * r2 + c2) + 1] = u[2 * (32 * r + c) + 1];
    }
  csim::make_dense_block(&b);
  // the previous block's device copy may still be read by queued work
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess) e = csim::upload_dense(&b, s->stream);
  if (e == cudaSuccess) e = csim::launch_dense(s->buf[s->cur], s->n, b, engine, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "csim_sv_apply_dense");
  return CSIM_OK;
}

csim_status csim_sv_info(const csim_sv* s, int64_t* n_sweeps, double* amp_updates,
                         uint64_t* state_bytes) {
  if (!s) return fail(CSIM_ERR_ARG, "null argument");
  if (n_sweeps) *n_sweeps = s->compiled ? s->prog.passes : 0;
  if (amp_updates) *amp_updates = s->compiled ? s->prog.amp_updates : 0.0;
  if (state_bytes) *state_bytes = s->bytes;
  return CSIM_OK;
}

csim_status csim_sv_stats(const csim_sv* s, csim_sv_stats_t* out) {
  if (!s || !out) return fail(CSIM_ERR_ARG, "null argument");
  *out = csim_sv_stats_t{};
  out->state_bytes = s->bytes;
  if (!s->compiled) return CSIM_OK;
  out->passes = s->prog.passes;
  out->sweeps = s->prog.stats.sweeps;
  out->single = s->prog.stats.single;
  out->amp_updates = s->prog.amp_updates;
  out->pass_amps = s->prog.pass_amps;
  out->dense_blocks = s->prog.stats.dense_blocks;
  out->staged_sweeps = s->prog.stats.staged_sweeps;
  return CSIM_OK;
}

csim_status csim_sv_load_device(csim_sv* s, const void* d_amps, size_t n_amps) {
  if (!s || !d_amps) return fail(CSIM_ERR_ARG, "null argument");
  if (n_amps != ((size_t)1 << s->n)) return fail(CSIM_ERR_ARG, "n_amps must be 2^n");
  s->cur = 0;
  cudaError_t e = cudaMemcpyAsync(s->buf[0], d_amps, s->bytes, cudaMemcpyDeviceToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "csim_sv_load_device");
  return CSIM_OK;
}

csim_status csim_sv_device(const csim_sv* s, void** d_state) {
  if (!s || !d_state) return fail(CSIM_ERR_ARG, "null argument");
  *d_state = s->buf[s->cur];
  return CSIM_OK;
}

csim_status csim_sv_free(csim_sv* s) {
  if (!s) return CSIM_OK;
  cudaStreamSynchronize(s->stream);
  for (void*& b : s->buf) {
    if (b) cudaFree(b);
    b = nullptr;
  }
  csim::free_program(&s->prog);
  csim::free_dense(&s->dense);
  delete s;
  return CSIM_OK;
}

csim_status csim_emulate_fused(const csim_gate* gates, size_t n_gates, int32_t n, double* amps,
                               int64_t* stats) {
  if (!gates && n_gates) return fail(CSIM_ERR_ARG, "null argument");
  if (n < 7 || n > (amps ? 24 : 34)) return fail(CSIM_ERR_ARG, "n out of range");
  for (size_t i = 0; i < n_gates; ++i) {
    const csim_gate& g = gates[i];
    if (g.op > 3 || g.target >= n || ((g.cmask >> g.target) & 1ull) || (g.cval & ~g.cmask) ||
        (g.cmask >> n))
      return fail(CSIM_ERR_ARG, "invalid gate record " + std::to_string(i));
  }
  Program p;
  std::vector<Gate> gl(gates, gates + n_gates);
  csim::build_program(gl, n, CSIM_EXEC_FUSED, &p, true);
  if (amps) {
    const size_t N = (size_t)1 << n;
    std::vector<double> st(amps, amps + 2 * N);
    csim::emulate_program(p, &st);
    std::memcpy(amps, st.data(), 2 * N * sizeof(double));
  }
  if (stats) {
    const csim::FuseStats& f = p.stats;
    const int64_t v[20] = {f.sweeps,      f.single,      f.perm_gates,  f.segments, f.local_gates,
                           f.mux,         f.mux_gates,   f.mux_entries, f.max_bucket,
                           f.lut_entries, f.max_support, p.passes,      f.reflect,  f.mux_inverse,
                           f.wht,         f.conjugated,  f.staged_sweeps, f.staged_gates,
                           f.dense_blocks, f.dense_gates};
    std::memcpy(stats, v, sizeof(v));
  }
  return CSIM_OK;
}

}  // extern "C"
