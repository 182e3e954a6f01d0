// The fuser: groups consecutive elementary gates into sweeps, each one HBM pass.
//
// A sweep is  [permutation]  then  [tile-local gates]:
//  * permutation: a maximal run of multi-controlled X gates whose target is a
//    qubit >= 2 and whose controls avoid qubits 0-1.  Such a run maps every
//    4-amplitude chunk (qubits 0-1) to another chunk, so the kernel gathers
//    each destination chunk from the source index obtained by applying the
//    run's X gates in reverse order to the destination index;
//  * tile-local gates: any gate whose target is one of the 7 lowest qubits
//    (the 128-amplitude warp tile); controls may sit anywhere.
// A gate fitting neither class (e.g. H on a high qubit) becomes its own
// single-gate step.
#include <cmath>

#include "fuse.h"

namespace csim {

namespace {

bool perm_eligible(const csim_gate& g) {
  return g.op == OP_X && g.target >= 2 && (g.cmask & 3ull) == 0;
}
bool local_eligible(const csim_gate& g) { return g.target <= 6; }

LocalOp to_local(const csim_gate& g) {
  LocalOp o;
  o.cmask = g.cmask;
  o.cval = g.cval;
  o.op = g.op;
  o.target = g.target;
  if (g.op == OP_RY) {
    o.c = std::cos(g.angle / 2.0);
    o.s = std::sin(g.angle / 2.0);
  } else if (g.op == OP_ZPHASE) {
    o.c = std::cos(g.angle);
    o.s = std::sin(g.angle);
  } else {
    o.c = o.s = 0.0;
  }
  return o;
}

PermOp to_perm(const csim_gate& g) {
  PermOp p;
  p.mask = g.cmask >> 2;
  p.val = g.cval >> 2;
  p.tbit = 1ull << (g.target - 2);
  return p;
}

}  // namespace

void build_program(const std::vector<csim_gate>& gates, int n, csim_exec mode, Program* p) {
  *p = Program();
  p->n = n;
  p->mode = mode;
  for (const csim_gate& g : gates) p->amp_updates += gate_amp_updates(g, n);
  if (mode == CSIM_EXEC_GATE || n < 7) {
    for (const csim_gate& g : gates) {
      Step s;
      s.kind = 1;
      s.g = g;
      p->steps.push_back(s);
    }
    p->passes = (int64_t)p->steps.size();
    return;
  }
  bool open = false, in_local = false;
  Step cur;
  auto close = [&]() {
    if (open) p->steps.push_back(cur);
    open = false;
    in_local = false;
  };
  for (const csim_gate& g : gates) {
    const bool pe = perm_eligible(g), le = local_eligible(g);
    if (open && !in_local && pe) {
      p->perm.push_back(to_perm(g));
      ++cur.perm_cnt;
      continue;
    }
    if (open && le) {
      p->ops.push_back(to_local(g));
      ++cur.op_cnt;
      in_local = true;
      continue;
    }
    close();
    if (pe || le) {
      cur = Step();
      cur.kind = 0;
      cur.perm_off = (int)p->perm.size();
      cur.op_off = (int)p->ops.size();
      open = true;
      if (pe) {
        p->perm.push_back(to_perm(g));
        cur.perm_cnt = 1;
      } else {
        p->ops.push_back(to_local(g));
        cur.op_cnt = 1;
        in_local = true;
      }
    } else {
      Step s;
      s.kind = 1;
      s.g = g;
      p->steps.push_back(s);
    }
  }
  close();
  p->passes = (int64_t)p->steps.size();
  for (const Step& s : p->steps)
    if (s.kind == 0 && s.perm_cnt > 0) p->pingpong = true;
}

cudaError_t upload_program(Program* p, cudaStream_t st) {
  if (p->uploaded) return cudaSuccess;
  cudaError_t e;
  if (!p->perm.empty()) {
    e = cudaMalloc(&p->d_perm, p->perm.size() * sizeof(PermOp));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(p->d_perm, p->perm.data(), p->perm.size() * sizeof(PermOp),
                        cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
  }
  if (!p->ops.empty()) {
    e = cudaMalloc(&p->d_ops, p->ops.size() * sizeof(LocalOp));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(p->d_ops, p->ops.data(), p->ops.size() * sizeof(LocalOp),
                        cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  p->uploaded = true;
  return cudaSuccess;
}

void free_program(Program* p) {
  if (p->d_perm) cudaFree(p->d_perm);
  if (p->d_ops) cudaFree(p->d_ops);
  p->d_perm = nullptr;
  p->d_ops = nullptr;
  p->uploaded = false;
}

cudaError_t run_program(const Program& p, void* buf[2], int* cur, int prec, cudaStream_t st) {
  for (const Step& s : p.steps) {
    cudaError_t e;
    if (s.kind == 1) {
      e = launch_gate(buf[*cur], prec, p.n, s.g, st);
    } else if (s.perm_cnt == 0) {
      e = launch_sweep(buf[*cur], buf[*cur], prec, p.n, nullptr, 0, p.d_ops + s.op_off, s.op_cnt,
                       st);
    } else {
      e = launch_sweep(buf[*cur], buf[1 - *cur], prec, p.n, p.d_perm + s.perm_off, s.perm_cnt,
                       p.d_ops + s.op_off, s.op_cnt, st);
      *cur = 1 - *cur;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace csim
