#!/usr/bin/env python3
"""Benchmark of the state-vector QSVT path on GB300.

Default workload (the precision configuration): Nx = 64, N_C = 2, K = 4,
Nt = 16, dt = 0.1, tau drawn from U[0.6, 1.2] with seed 1, initial density
1 + 0.05 sin(2 pi x / Nx) + U(-0.01, 0.01), QSVT degree d = 13 (the
truncated-degree timing run), 32 qubits, complex64 state (32 GiB, twice for
the gather ping-pong), fused sweeps.

A step is one pass of the whole hot path through the C ABI: csim_init (load
b), csim_run (the QSVT circuit: 14 fused sweeps over 2^32 amplitudes) and
csim_postselect (FP64 norm and success probability).  The metric is
amplitude-gate updates per second: the sum over the circuit's elementary
gates of the amplitudes each gate changes, divided by the step time.

Output: one JSON line (rank 0).  Outside the timed region the line also
carries the oracle beside the GPU numbers (cpu_baseline: the classical QSVT
evaluator on the whole workload, one thread and all cores, and the naive
simulator's per-update rate) and, for the precision workloads, the plain
gate-by-gate complex128 GPU path on the same circuit with each result's
relative L2 error against the oracle.  --impl reference times the oracle
instead: the naive simulator per amplitude update, one thread per step, with
the classical evaluator's time on the whole workload beside it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lbm_inputs as I  # noqa: E402

METRIC = "amplitude-gate updates/s"
UNIT = "amp-updates/s"

WORKLOADS = {
    # name: (Nx, N_C, K, Nt, dt, tau or None, tau_range, seed, d, kappa_qsvt, precision)
    "precision-nx64-k4-nt16-d13-c64": (64, 2, 4, 16, 0.1, None, (0.6, 1.2), 1, 13, 1000.0, "c64"),
    "precision-nx64-k4-nt16-d13-c128": (64, 2, 4, 16, 0.1, None, (0.6, 1.2), 1, 13, 1000.0, "c128"),
    "plain-nx4-k2-nt2-c128": (4, 2, 2, 2, 0.1, 0.8, None, 0, 0, 0.0, "c128"),
    # 28-qubit member of the precision family (2 GiB in complex64) for ncu captures
    "profile-nx16-k4-nt16-d13-c64": (16, 2, 4, 16, 0.1, None, (0.6, 1.2), 1, 13, 1000.0, "c64"),
    "profile-nx16-k4-nt16-d13-c128": (16, 2, 4, 16, 0.1, None, (0.6, 1.2), 1, 13, 1000.0, "c128"),
    # 26-qubit member (512 MiB): its gathers keep the natural tile order
    "profile-nx8-k4-nt16-d13-c64": (8, 2, 4, 16, 0.1, None, (0.6, 1.2), 1, 13, 1000.0, "c64"),
}
DEFAULT = "precision-nx64-k4-nt16-d13-c64"

# The paper's long N_C = 2 run (Sec. III.E.2: Nx = 8, K = 3, Nt = 4, walls,
# nu = 2 so tau = (Nx/512) nu / c_s^2 = 0.09375): kappa(L) = 7117 and, with
# eps = 1e-3, d = 58613 from Eq. d-star; 23 qubits here (27 in the paper's
# layout), complex128.  Build (kappa and fixed-point phases) takes about a
# minute on the host; run with --steps 1 --warmup 1.
WORKLOADS["paper-long-nx8-nc2-k3-nt4-walls-c128"] = (8, 2, 3, 4, 0.1, 8 / 512.0 * 2.0 * 3.0, None, 0,
                                                      0, 0.0, "c128")
# The same run with the paper's own polynomial design: kappa_QSVT = 7100 and
# d = 10 kappa_QSVT + 1 = 71001 (Sec. III.E.2).
WORKLOADS["paper-long-nx8-nc2-k3-nt4-d71001-walls-c128"] = (8, 2, 3, 4, 0.1, 8 / 512.0 * 2.0 * 3.0,
                                                             None, 0, 71001, 7100.0, "c128")
BOUNDARY = {"paper-long-nx8-nc2-k3-nt4-walls-c128": "bounceback",
            "paper-long-nx8-nc2-k3-nt4-d71001-walls-c128": "bounceback"}

# Batching: count seeded instances (lbm_inputs.batch_instance), complex64,
# run through the request pool; serving: a bounded prefix of the seeded
# request stream (lbm_inputs.serving_requests) with Poisson arrivals.
BATCH = {"batch-256-c64": 256, "batch-4x26-c64": (4, 26)}
SERVING = {"serving-poisson-200": 200}

# Gate-vocabulary microbenchmark: (qubits, gates, seed); complex64, seeded
# random normalised initial state generated on the device.
MICRO = {
    # 28 qubits (2 GiB): the same stream's fusion at a size for ncu captures
    "microbench-n28-c64": (28, 1000, 0),
    "microbench-n30-c64": (30, 1000, 0),
    "microbench-n33-c64": (33, 1000, 0),
}
# Dense-block stream: (qubits, blocks, seed); complex64, each block 16 gates
# on 5 random qubits (lbm_inputs.dense_block_gates), fused into one dense
# 5-qubit block on the tensor cores per run.
DENSE = {
    "dense5-n28-c64": (28, 64, 0),
    "dense5-n30-c64": (30, 64, 0),
}

# ncu dram__bytes_read.sum + dram__bytes_write.sum of one sweep_kernel launch,
# keyed by the sha256 of kernels.cu at capture time (profiles/ has the summary).
# A changed kernel source reports null traffic until it is captured again.
NCU_TRAFFIC = {
    # mean over the 14 sweep launches of one run (single-pass ncu capture;
    # after the sparse init the first sweep touches only the tiles of b and
    # the first conjugated gather reads only its index table)
    ("85ac97949cbcb0a7", "precision-nx64-k4-nt16-d13-c64"): 64.48e9,
    # the same shaped kernels after the staged-qubit and block-size changes:
    # the 28-qubit family member's 14 launches (dram__bytes_read + write,
    # one pass), mean per launch scaled by the 16x larger state
    ("bc1adbfeda1ad1d4", "precision-nx64-k4-nt16-d13-c64"): 64.81e9,
    # the same sweep kernels with the persistent pool kernel and the launch
    # tuner's table in the source; captured at the default grid (the tuner may
    # pick another number of waves for the same kernels)
    ("0f3b1fc150ae926c", "precision-nx64-k4-nt16-d13-c64"): 64.83e9,
    ("538f34759c558b2b", "precision-nx64-k4-nt16-d13-c64"): 64.82e9,
    # the last sweep also sums |a|^2 of the state it writes (fused norms)
    ("cc602739cd474360", "precision-nx64-k4-nt16-d13-c64"): 64.80e9,
    # the persistent pool kernel's items also sum |a|^2 (sweep kernels unchanged)
    ("5f8fee62903c51d4", "precision-nx64-k4-nt16-d13-c64"): 64.79e9,
}

L2_BYTES = 129 * 1000 * 1000


def measure_l2_copy(torch, nbytes):
    """Read + write GB/s of a device copy between two buffers of nbytes each
    (both fit the 129 MB L2 together for the states this is used on): best
    of 20 after warm-up, CUDA events."""
    a = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda").fill_(1.0)
    b = torch.empty_like(a)
    for _ in range(5):
        b.copy_(a)
    best = 1e30
    for _ in range(20):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.copy_(a)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * nbytes / (best / 1000.0) / 1e9


def measure_fp64_peak(torch, m=4096):
    """FP64 TFLOP/s of a square DGEMM (2 m^3 FLOP), best of 5: the rate the
    complex128 sweeps' FP64 work is set against."""
    a = torch.randn(m, m, dtype=torch.float64, device="cuda")
    b = torch.randn(m, m, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * m ** 3 / (best / 1000.0) / 1e12


def max_over_ranks(x, dist, device="cuda"):
    """The largest value of x over all ranks: the job takes as long as its
    slowest replica.  dist None (one process) returns x."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput of `world` replicas that each process
    units_per_rank in the job's time."""
    return units_per_rank * world / seconds


def kernel_hash():
    p = os.path.join(ROOT, "paper_2606_12770_gb300", "csrc", "kernels.cu")
    with open(p, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def oracle_sample(workload, threads=1):
    """The oracle's naive gate-by-gate simulator (O2, its tensor-axis form) on
    one U_L call -- the unit the QSVT circuit repeats d times -- of the
    workload's circuit family at Nx = 4: the same construction, K, Nt and
    tau, 24 qubits for the precision workloads (their 32 qubits hold 64 GB of
    FP64 state).  The rate is per amplitude update, which the naive simulator
    spends at about the same cost at any size."""
    from oracle import circuit as OC
    from oracle import statevec as S
    from oracle.layout import Layout

    Nx, NC, K, Nt, dt, tau, tau_range, seed, d, kappa, prec = WORKLOADS.get(workload,
                                                                             WORKLOADS[DEFAULT])
    Nx = 4
    f0, tau = I.lbm_instance(Nx, seed, tau=tau, tau_range=tau_range)
    lay = Layout(Nx, NC, K, Nt)
    gates = OC.build_UL(Nx, tau, NC, K, dt, Nt, bc=BOUNDARY.get(workload, "periodic"))
    psi = np.zeros(1 << lay.n, dtype=complex)
    init, _ = OC.initial_state(lay, f0)
    for k, v in init.items():
        psi[k] = v
    sim = S.AxisSim(lay.n, threads=threads)
    upd = sum(2.0 ** (lay.n - bin(g[2]).count("1")) for g in gates)
    t0 = time.perf_counter()
    sim.run(psi, gates)
    dt_s = time.perf_counter() - t0
    return {"value": upd / dt_s, "unit": UNIT, "cores": threads, "kind": "oracle",
            "seconds": dt_s,
            "sample": f"one U_L call ({len(gates)} gates, {upd:.4g} amplitude updates) of the "
                      f"{lay.n}-qubit member (Nx=4, N_C={NC}, K={K}, Nt={Nt}) of this workload's "
                      f"circuit family through the oracle's naive FP64 gate-by-gate simulator "
                      f"(O2, tensor-axis form, {threads} thread), {dt_s:.1f} s; per amplitude "
                      f"update, which it spends at about the same cost at any size"}


# Classical QSVT evaluation (O5) of a workload, run in a fresh interpreter so
# that its thread count is fixed before NumPy loads.  Writes the postselected
# physical block and its state indices when asked.
O5_SCRIPT = r"""
import json, sys, time
import numpy as np
a = json.loads(sys.argv[1])
sys.path.insert(0, a["root"])
from oracle import qsvt as Q
f0 = np.asarray(a["f0"], dtype=np.float64)
ph = np.asarray(a["phases"], dtype=np.float64)
t0 = time.perf_counter()
y, lay, _, _ = Q.qsvt_postselected(a["Nx"], a["tau"], a["NC"], a["K"], a["dt"], a["Nt"], f0, ph)
sec = time.perf_counter() - t0
if a.get("out"):
    D = lay.carleman_dim()
    base = np.array([lay.embed_index(0, j) for j in range(D)], dtype=np.int64)
    off = np.array([lay.place(k=int(s) & ((1 << lay.nk) - 1), m=int(s) >> lay.nk)
                    for s in range(lay.n_slots())], dtype=np.int64)
    np.savez(a["out"], y=y, idx=(off[:, None] | base[None, :]).reshape(-1))
print(json.dumps({"seconds": sec, "entries": int(y.size)}))
"""

THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def oracle_classical(cfg, f0, phases, threads=None, out=None):
    """Seconds of one O5 evaluation (classical QSVT of the same phases on the
    workload's L) in a fresh interpreter; threads=1 pins every math library
    to one thread, None leaves them at their defaults (all cores)."""
    Nx, tau, NC, K, dt, Nt = cfg
    env = dict(os.environ)
    for v in THREAD_VARS:
        if threads is None:
            env.pop(v, None)
        else:
            env[v] = str(threads)
    arg = json.dumps({"root": ROOT, "Nx": Nx, "tau": tau, "NC": NC, "K": K, "dt": dt, "Nt": Nt,
                      "f0": np.asarray(f0).tolist(), "phases": np.asarray(phases).tolist(),
                      "out": out})
    r = subprocess.run([sys.executable, "-c", O5_SCRIPT, arg], env=env, capture_output=True,
                       text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("classical oracle failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_amp_updates(cfg, phases):
    """Amplitude-gate updates of the whole circuit, counted on the oracle's own
    gate list (O3): sum over gates of 2^(n - controls)."""
    from oracle import circuit as OC
    from oracle.layout import Layout
    Nx, tau, NC, K, dt, Nt = cfg
    lay = Layout(Nx, NC, K, Nt)
    gates = OC.build_qsvt(Nx, tau, NC, K, dt, Nt, list(phases))
    return float(sum(2.0 ** (lay.n - bin(g[2]).count("1")) for g in gates))


def cpu_baselines(workload, cfg, f0, phases, updates, out=None):
    """The oracle beside the GPU numbers: the naive gate-by-gate simulator's
    rate per amplitude update on a bounded sample (the metric's own unit),
    and the classical QSVT evaluator (O5) on the whole workload, one thread
    and all cores: the time it takes to produce the same postselected block,
    with the circuit's amplitude updates over that time as an equivalent
    rate."""
    naive = oracle_sample(workload, threads=1)
    one = oracle_classical(cfg, f0, phases, threads=1, out=out)
    allc = oracle_classical(cfg, f0, phases, threads=None)
    cores = os.cpu_count()
    naive["host_cores"] = cores
    naive["classical_o5"] = {
        "what": (f"the whole workload through the oracle's classical QSVT evaluator (O5: the "
                 f"circuit's polynomial of L applied to b with sparse products, "
                 f"{one['entries']} physical entries); equivalent_value = the circuit's "
                 f"amplitude-gate updates over its time"),
        "one_thread": {"seconds_per_run": one["seconds"], "equivalent_value": updates / one["seconds"],
                       "cores": 1},
        "all_cores": {"seconds_per_run": allc["seconds"],
                      "equivalent_value": updates / allc["seconds"], "cores": cores,
                      "note": "math libraries at their default thread count; the sparse products "
                              "themselves run on one thread"}}
    return naive


def oracle_micro_sample(n, seconds_target=12.0):
    """Naive FP64 simulator on a bounded prefix of the vocabulary stream at n qubits."""
    from oracle import statevec as S

    gates = I.microbench_gates(n, 1000, 0)
    psi = I.random_unit_state(n, 0)
    sim = S.DenseSim(n)
    upd = 0.0
    count = 0
    t0 = time.perf_counter()
    for g in gates:
        sim.apply(psi, g)
        upd += 2.0 ** (n - bin(g[2]).count("1"))
        count += 1
        if time.perf_counter() - t0 > seconds_target:
            break
    dt = time.perf_counter() - t0
    return {"value": upd / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "seconds": dt,
            "sample": f"first {count} gates of the vocabulary stream at {n} qubits through the "
                      f"naive FP64 gate-by-gate simulator, {dt:.1f} s (the benchmark's 2^30/2^33 "
                      f"states do not fit the oracle's FP64 copies in host memory in that time)"}


def run_micro(args, rank, world, local, torch, G, dist):
    """One step = the whole 1000-gate vocabulary stream over the resident state."""
    if args.workload in DENSE:
        n, count, seed = DENSE[args.workload]
        gates = I.dense_block_gates(n, count, seed)
    else:
        n, count, seed = MICRO[args.workload]
        gates = I.microbench_gates(n, count, seed)
    records = G.gates_to_records(gates)
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed + rank)
    x = torch.randn((1 << n, 2), generator=gen, device="cuda", dtype=torch.float32)
    x /= torch.linalg.vector_norm(x)
    sv = G.StateVector(n, G.CSIM_C64, stream)
    sv.load_device(x.data_ptr())
    del x
    torch.cuda.empty_cache()
    mode = G.CSIM_EXEC_FUSED if args.exec == "fused" else G.CSIM_EXEC_GATE
    tune = None
    if mode == G.CSIM_EXEC_FUSED and not args.no_autotune:
        # fusion width (staged qubits, dense blocks) picked by timed trials on
        # this state, before the timed region; the state is restored
        tune = sv.autotune(records, reps=1)
    else:
        sv.compile(records, mode)
    st = sv.stats()
    for _ in range(max(args.warmup, 0)):
        sv.run()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for a, b in ev:
        a.record(stream)
        sv.run()
        b.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    total_ms = max_over_ranks(total_ms, dist)
    ms = total_ms / args.steps
    value = job_rate(st["amp_updates"], world, ms / 1000.0)
    # end to end through the public API: compile the host gate list (fusing and
    # table upload), run, and read back the FP64 norm of the result
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sv.compile(records, mode)
        sv.run()
        G._native.norms_noalloc(sv.device_state().ptr, n, G.CSIM_C64, [], [], out.data_ptr(), stream)
        float(out[0].item())
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    peaks, peak_kind = measured_peaks()
    alg_bytes = 2.0 * st["pass_amps"] * 8
    achieved = alg_bytes / (ms / 1000.0) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "complex64 (fp32)",
        "data": "synthetic (seeded gate stream; seeded random normalised state)",
        "config": {"workload": args.workload, "qubits": n, "gates": len(gates), "exec": args.exec,
                   "passes": st["passes"], "fused_sweeps": st["sweeps"],
                   "single_gate_passes": st["single"], "state_bytes": st["state_bytes"],
                   "l2": "inputs larger than L2 (state >> 129 MB)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "kernel": "all passes of the run (sweep_kernel and gate_kernel)",
                     "peak_kind": f"{peak_kind} (STREAM-style copy)",
                     "alg_bytes_per_run": alg_bytes, "launches_per_step": st["passes"]},
        "e2e": {"value": st["amp_updates"] * world / (statistics.median(e2e_ms) / 1000.0),
                "unit": UNIT, "h2d_bytes_per_step": int(records.nbytes), "d2h_bytes_per_step": 8},
        "gpu_launches": args.steps * st["passes"],
        "clocks": clk,
    }
    line["config"]["autotune"] = tune
    line["config"]["dense_blocks"] = st["dense_blocks"]
    line["config"]["staged_sweeps"] = st["staged_sweeps"]
    if st["dense_blocks"] and st["dense_blocks"] == st["passes"]:
        # every pass is a dense block: the tensor work the split products
        # execute (3 x 2 x 64 x 64 FLOP per group of 32 amplitudes) against
        # the bf16 peak, beside the HBM roofline above
        flops = 3.0 * 2 * 64 * 64 * (1 << (n - 5)) * st["dense_blocks"]
        line["tensor"] = {"kernel": "dense5_tc_kernel", "achieved": flops / (ms / 1000.0) / 1e12,
                          "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                          "frac": flops / (ms / 1000.0) / 1e12 / peaks["bf16_tflops"],
                          "note": "split BF16x3: three BF16 products per complex64 block; "
                                  "the pass is HBM-bound at this intensity (48 FLOP/B)",
                          "engine": os.environ.get("CSIM_DENSE_ENGINE", "tc")}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_micro_sample(22)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _build_parallel(G, specs, workers=8):
    """Build and host-compile circuits in parallel threads (the C calls release
    the GIL).  specs: list of (cfg, d)."""
    from concurrent.futures import ThreadPoolExecutor

    def one(spec):
        cfg, d = spec
        c = G.Circuit(*cfg, kappa_qsvt=10.0, d=d)
        c.compile()
        return c

    with ThreadPoolExecutor(workers) as ex:
        return list(ex.map(one, specs))


def _pool_budget(torch, cap_bytes):
    free, _ = torch.cuda.mem_get_info()
    return int(min(cap_bytes, 0.85 * free))


def _finish_line(args, line, world, dist):
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_batch(args, rank, world, local, torch, G, dist):
    """One step = all instances submitted at once to the request pool, polled
    until every result (norms and compacted block, copied to pinned host
    memory) is back.  Host wall clock around the step (the pool spreads the
    work over its own streams)."""
    spec = BATCH[args.workload]
    if isinstance(spec, tuple):
        # (count, qubits): the first `count` instances of that size (one
        # persistent pass of equal requests, the profiling case)
        count, want = spec
        insts, i = [], 0
        while len(insts) < count:
            cfg, d, f0 = I.batch_instance(i)
            i += 1
            c = G.Circuit(*cfg, kappa_qsvt=10.0, d=d)
            if c.info()["n_qubits"] == want:
                insts.append((cfg, d, f0))
            c.close()
    else:
        count = spec
        insts = [I.batch_instance(i + rank * count) for i in range(count)]
    circs = _build_parallel(G, [(cfg, d) for cfg, d, _ in insts])
    qubits = sorted({c.info()["n_qubits"] for c in circs})
    amp_updates = 0.0
    alg_bytes = 0.0
    launches = 0
    for c in circs:
        inf = c.info()
        amp_updates += inf["amp_updates_run"]
        alg_bytes += 2.0 * inf["n_sweeps_run"] * (1 << inf["n_qubits"]) * 8
        launches += inf["n_sweeps_run"] + 4  # init, sweeps, norms + reduce, compaction
    budget = _pool_budget(torch, 200 << 30)

    def pool_step(pool):
        t0 = time.perf_counter()
        ids = [pool.submit(c, f0, G.CSIM_C64) for c, (_, _, f0) in zip(circs, insts)]
        left = set(ids)
        while left:
            for rid in pool.poll(wait_ms=5):
                pool.result(rid, want_amplitudes=False)
                left.discard(rid)
        return time.perf_counter() - t0

    results = {}
    clk = None
    graph_error = None
    for mode in ("streams", "graphs", "persistent"):
        graphs = mode == "graphs"
        # persistent passes take half the slots each: 16 slots give passes of
        # eight requests, two in flight
        pool = G.Pool(n_streams=16 if mode == "persistent" else 8, hbm_budget=budget,
                      max_qubits=32, use_graphs=graphs, persistent=mode == "persistent")
        try:
            for _ in range(max(args.warmup, 1)):
                pool_step(pool)
        except G.CsimError as e:
            if not graphs:
                raise
            graph_error = str(e)
            pool.close()
            continue
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        if dist is not None:
            dist.barrier()
        saved0 = pool.stats()["sparse_saved_bytes"]
        ts = [pool_step(pool) for _ in range(args.steps)]
        c2 = clocks.stop()
        clk = clk or c2
        st = pool.stats()
        st["saved_per_step"] = (st["sparse_saved_bytes"] - saved0) / args.steps
        pool.close()
        results[mode] = (statistics.median(ts), st)
    # the per-instance loop: one instance at a time through csim_init/run/postselect
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c, (_, _, f0) in zip(circs, insts):
        c.init(f0, G.CSIM_C64)
        c.run()
        c.postselect(want_amplitudes=False)
        c.close()  # frees the instance's state buffers before the next one
    loop_s = time.perf_counter() - t0
    best = min(results, key=lambda k: results[k][0])
    step_s, st = results[best]
    step_s = max_over_ranks(step_s, dist)
    peaks, peak_kind = measured_peaks()
    # the sparse init leaves out the leading sweeps' reads and writes of the
    # unwritten zeros (counted by the pool)
    alg_bytes -= st["saved_per_step"]
    achieved = alg_bytes / step_s / 1e9
    line = {
        "metric": METRIC, "value": amp_updates * world / step_s, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * step_s,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "complex64 (fp32)", "data": "synthetic (seeded instances 0..255)",
        "config": {"workload": args.workload, "instances": count,
                   "qubits": f"{qubits[0]}-{qubits[-1]}" if len(qubits) > 1 else str(qubits[0]),
                   "mode": f"request pool, 8 streams, {best}",
                   "runs_per_s": count * world / step_s,
                   "streams_step_s": results["streams"][0],
                   "graphs_step_s": results["graphs"][0] if "graphs" in results else graph_error,
                   "persistent_step_s": (results["persistent"][0] if "persistent" in results
                                         else None),
                   "persistent": ({"slots": 16, "passes_per_step":
                                   results["persistent"][1]["batch_launches"] / (args.steps + max(args.warmup, 1)),
                                   "requests_batched": results["persistent"][1]["batch_requests"]}
                                  if "persistent" in results else None),
                   "per_instance_loop_s": loop_s,
                   "pool_budget_bytes": st["budget"], "pool_peak_bytes": st["peak_bytes"],
                   "timing": "host wall clock per step (work spread over the pool's streams)",
                   "l2": (f"inputs larger than L2 (states {8 * 2 ** qubits[0] / 1e6:.0f} MB-"
                          f"{8 * 2 ** qubits[-1] / 1e9:.1f} GB each)"),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "kernel": "sweep_kernel (all instances, aggregate)",
                     "peak_kind": f"{peak_kind} (STREAM-style copy)",
                     "alg_bytes_per_step": alg_bytes},
        "e2e": {"value": amp_updates * world / step_s, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(16 * (3 * cfg[0] + 9 * cfg[0] ** 2) for cfg, _, _ in insts)),
                "d2h_bytes_per_step": 16 * count,
                "note": "the pool step is already end to end: host f0 in, H2D of b, run, D2H of results"},
        "gpu_launches": launches * args.steps,
        "clocks": clk,
    }
    _finish_line(args, line, world, dist)


def run_serving(args, rank, world, local, torch, G, dist):
    """Poisson arrivals at 0.8 of the measured capacity (the line), after a
    sweep of loads 0.5, 1.0 and 1.25 on the first 100 requests (its
    config).  Each request is built and compiled on the host after it arrives
    (8 builder threads), then submitted to the pool; latency = arrival to
    result.  Requests above 32 qubits (Nx = 256 and 1024, and the largest
    Nx = 64 ones) are rejected."""
    from concurrent.futures import ThreadPoolExecutor

    count = SERVING[args.workload]
    reqs = I.serving_requests(count, 0)
    budget = _pool_budget(torch, 220 << 30)
    pool = G.Pool(n_streams=4, hbm_budget=budget, max_qubits=32, use_graphs=False)
    precs = {"c64": G.CSIM_C64, "c128": G.CSIM_C128}

    def build(r):
        """The request's circuit, or None when it cannot be built at all (more
        qubits than the library's 34-qubit limit)."""
        try:
            c = G.Circuit(r["Nx"], r["tau"], 2, r["K"], 0.1, r["Nt"], kappa_qsvt=10.0, d=r["d"])
        except G.CsimError:
            return None
        if c.info()["n_qubits"] <= 32:
            c.compile()
        return c

    def closed_loop(sub):
        """All requests at once: (admitted requests completed per second,
        fraction of the requests admitted)."""
        circs = [build(r) for r in sub]
        t0 = time.perf_counter()
        live = set()
        for r, c in zip(sub, circs):
            if c is None:
                continue
            try:
                live.add(pool.submit(c, I.serving_f0(r), precs[r["prec"]]))
            except G.CsimError:
                pass
        n_adm = len(live)
        while live:
            for rid in pool.poll(wait_ms=5):
                pool.result(rid, want_amplitudes=False)
                live.discard(rid)
        return n_adm / (time.perf_counter() - t0), n_adm / len(sub)

    def est_bytes(r):
        """Algorithmic HBM bytes of one request (0 if it would be rejected)."""
        try:
            inf = G.Circuit(r["Nx"], r["tau"], 2, r["K"], 0.1, r["Nt"], kappa_qsvt=10.0,
                            d=r["d"]).info()
        except G.CsimError:
            return 0.0
        if inf["n_qubits"] > 32:
            return 0.0
        esz = 8 if r["prec"] == "c64" else 16
        return 2.0 * (r["d"] + 1) * (1 << inf["n_qubits"]) * esz

    closed_loop(reqs[:8])  # warm-up: kernels, pinned staging
    calib = reqs[:64]
    t_cal = time.perf_counter()
    capacity, admitted_frac = closed_loop(calib)
    t_cal = time.perf_counter() - t_cal
    # offered load: 0.8 of the measured byte throughput, spread over the mean
    # algorithmic bytes of the whole request stream
    bytes_per_s = sum(est_bytes(r) for r in calib) / t_cal
    mean_bytes = sum(est_bytes(r) for r in reqs) / len(reqs)
    ex = ThreadPoolExecutor(8)

    def session(load, n):
        """Poisson arrivals of the first n requests at `load` times the
        measured byte throughput: (latencies s, rejected, amp updates, wall s,
        arrival rate)."""
        rate = load * bytes_per_s / max(mean_bytes, 1.0)
        arrivals = np.cumsum([r["gap"] for r in reqs[:n]]) / rate
        lat = []
        rejected = 0
        amp_upd = 0.0
        t0 = time.perf_counter()
        nxt = 0
        building = {}
        live = {}
        while nxt < n or building or live:
            now = time.perf_counter() - t0
            while nxt < n and arrivals[nxt] <= now:
                building[ex.submit(build, reqs[nxt])] = nxt
                nxt += 1
            for fut in [f for f in building if f.done()]:
                i = building.pop(fut)
                c = fut.result()
                if c is None:
                    rejected += 1
                    continue
                try:
                    rid = pool.submit(c, I.serving_f0(reqs[i]), precs[reqs[i]["prec"]])
                    live[rid] = (i, c)
                except G.CsimError:
                    rejected += 1
            for rid in pool.poll(wait_ms=1 if live else 0):
                i, c = live.pop(rid)
                pool.result(rid, want_amplitudes=True)
                lat.append(time.perf_counter() - t0 - arrivals[i])
                amp_upd += c.info()["amp_updates_run"]
            if not live and not building and nxt < n:
                time.sleep(max(0.0, min(0.01, arrivals[nxt] - (time.perf_counter() - t0))))
        return lat, rejected, amp_upd, time.perf_counter() - t0, rate

    def pctl(lat, q):
        ms = sorted(1000.0 * x for x in lat)
        return ms[min(len(ms) - 1, int(q * len(ms)))] if ms else None

    # the rate sweep (shorter prefixes), then the reported session at 0.8
    sweep = []
    n_sweep = min(count, 100)
    for load in (0.5, 1.0, 1.25):
        l2, rj, au, w2, rt = session(load, n_sweep)
        sweep.append({"load": load, "requests": n_sweep, "arrival_rate_req_per_s": rt,
                      "completed": len(l2), "runs_per_s": len(l2) / w2,
                      "latency_ms_p50": pctl(l2, 0.5), "latency_ms_p99": pctl(l2, 0.99)})
    clocks = ClockSampler(local)
    clocks.start()
    lat, rejected, amp_upd, wall, rate = session(0.8, count)
    clk = clocks.stop()
    ex.shutdown()
    st = pool.stats()
    pool.close()
    lat_ms = sorted(1000.0 * x for x in lat)
    pct = (lambda q: lat_ms[min(len(lat_ms) - 1, int(q * len(lat_ms)))]) if lat_ms else (lambda q: None)
    peaks, peak_kind = measured_peaks()
    line = {
        "metric": METRIC, "value": amp_upd * world / wall, "unit": UNIT, "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": 1000.0 * wall, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "complex64 and complex128 (50/50)",
        "data": "synthetic (seeded request stream, seed 0)",
        "config": {"workload": args.workload, "requests": count, "completed": len(lat),
                   "rejected_above_32_qubits": rejected,
                   "capacity_admitted_req_per_s": capacity, "admitted_fraction": admitted_frac,
                   "calibration_bytes_per_s": bytes_per_s,
                   "arrival_rate_req_per_s": rate, "runs_per_s": len(lat) / wall,
                   "latency_ms_p50": pct(0.5), "latency_ms_p99": pct(0.99),
                   "load": 0.8, "rate_sweep": sweep,
                   "pool_budget_bytes": st["budget"], "pool_peak_bytes": st["peak_bytes"],
                   "timing": "host wall clock over the serving session",
                   "parallelism": f"replicas x{world}"},
        "roofline": None,
        "e2e": {"value": amp_upd * world / wall, "unit": UNIT, "h2d_bytes_per_step": None,
                "d2h_bytes_per_step": None, "note": "the session is end to end by construction"},
        "gpu_launches": None,
        "clocks": clk,
    }
    _finish_line(args, line, world, dist)


def _reference_inputs(workload):
    """(cfg, f0, phases) of a workload for the oracle alone: the seeded
    instance and, since O5's cost depends on the degree and not on the phase
    values, seeded phases of the workload's degree (Eq. d-star from the
    oracle's kappa(L) where the workload leaves d to the build)."""
    from oracle import physics as OP
    from oracle import qsvt as Q
    Nx, NC, K, Nt, dt, tau, tau_range, seed, d, kappa, prec = WORKLOADS[workload]
    f0, tau = I.lbm_instance(Nx, seed, tau=tau, tau_range=tau_range)
    bc = BOUNDARY.get(workload, "periodic")
    if d <= 0:
        kap = kappa if kappa > 0 else OP.kappa_L(Nx, tau, NC, K, dt, Nt, bc=bc)
        d = Q.degree_from_kappa(kap, 1e-3)
    return (Nx, tau, NC, K, dt, Nt), f0, I.random_phases(d, 0)


def run_reference(args, rank, world):
    """The oracle on this arm's workload, in the metric's own unit: each step
    is a bounded sample of the naive gate-by-gate simulator (O2): one U_L
    call of the workload's circuit family at 24 qubits (a time-bounded
    prefix of the vocabulary stream at 22 qubits for the microbenchmark
    workloads), one thread, per amplitude update.  The line also carries the classical QSVT
    evaluator (O5) on the whole workload, one thread, for the circuit
    workloads."""
    if rank != 0:
        return
    W, K = args.warmup, args.steps
    secs = []
    vals = []
    extra = {}
    circuit = args.workload in WORKLOADS
    r = None
    for i in range(W + K):
        if circuit:
            r = oracle_sample(args.workload, threads=1)
        else:
            r = oracle_micro_sample(22, seconds_target=args.ref_seconds)
        if i >= W:
            secs.append(r["seconds"])
            vals.append(r["value"])
    workload = (args.workload if (circuit or args.workload in MICRO or args.workload in DENSE)
                else "microbench-n22-c128")
    if circuit and BOUNDARY.get(args.workload, "periodic") == "periodic":
        cfg, f0, ph = _reference_inputs(args.workload)
        updates = oracle_amp_updates(cfg, ph)
        o5 = oracle_classical(cfg, f0, ph, threads=1)
        extra["classical_o5"] = {
            "what": (f"the whole workload through the oracle's classical QSVT evaluator (O5, "
                     f"FP64, {o5['entries']} physical entries, degree {len(ph) - 1}), one thread; "
                     f"equivalent_value = the circuit's amplitude-gate updates ({updates:.4g}, "
                     f"counted on the oracle's gate list) over its time"),
            "seconds_per_run": o5["seconds"], "equivalent_value": updates / o5["seconds"]}
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": 1000.0 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "complex128 (fp64)", "data": "synthetic",
            "config": {"workload": workload, "host_cores": os.cpu_count(), "threads": 1,
                       "sample_per_step": r["sample"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    line.update(extra)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS) + sorted(MICRO) + sorted(DENSE) + sorted(BATCH) +
                    sorted(SERVING))
    ap.add_argument("--exec", default="fused", choices=["fused", "gate"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default fusion width (gate streams) and sweep launch shape "
                         "(circuits) instead of timing trials")
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_2606_12770_gb300 as G

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    if args.workload in MICRO or args.workload in DENSE:
        return run_micro(args, rank, world, local, torch, G, dist)
    if args.workload in BATCH:
        return run_batch(args, rank, world, local, torch, G, dist)
    if args.workload in SERVING:
        return run_serving(args, rank, world, local, torch, G, dist)

    Nx, NC, K, Nt, dt, tau, tau_range, seed, d, kappa, prec = WORKLOADS[args.workload]
    f0, tau = I.lbm_instance(Nx, seed + rank * 0, tau=tau, tau_range=tau_range)
    circ = G.Circuit(Nx, tau, NC, K, dt, Nt, kappa_qsvt=kappa, d=d,
                     bc=BOUNDARY.get(args.workload, "periodic"))
    circ.set_exec(G.CSIM_EXEC_FUSED if args.exec == "fused" else G.CSIM_EXEC_GATE)
    precision = G.CSIM_C64 if prec == "c64" else G.CSIM_C128
    stream = torch.cuda.current_stream()
    info = circ.info()
    n = info["n_qubits"]
    esz = 8 if prec == "c64" else 16

    # launch shape of this (precision, size) class from short timed trials on a
    # scratch state, before the warm-up (the circuit's own state is untouched)
    tune = None
    if args.exec == "fused" and not args.no_autotune:
        t = circ.tune_launch(precision, max_steps=16, reps=2)
        tune = {k: t[k] for k in ("u", "minb", "waves", "ms", "ms_default", "steps")}
        tune["n_trials"] = len(t["trials"])
        tune["what"] = ("sweep launch shape per (precision, qubits): tiles per warp iteration u, "
                        "blocks per SM minb, grid in resident waves; ms = the first `steps` "
                        "program steps")

    def step(want_amps=False, out=None):
        circ.init(f0, precision, stream)
        circ.run()
        return circ.postselect(want_amplitudes=want_amps)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    info = circ.info()
    passes = info["n_sweeps_run"]

    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    t_host0 = time.perf_counter()
    for s in range(args.steps):
        e = ev[s]
        e[0].record(stream)
        circ.init(f0, precision, stream)
        e[1].record(stream)
        circ.run()
        e[2].record(stream)
        circ.postselect(want_amplitudes=False)
        e[3].record(stream)
    torch.cuda.synchronize()
    t_host = time.perf_counter() - t_host0
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [ev[s][0].elapsed_time(ev[s][3]) for s in range(args.steps)]
    run_ms = [ev[s][1].elapsed_time(ev[s][2]) for s in range(args.steps)]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, dist)
    ms_per_step = total_ms / args.steps
    updates = info["amp_updates_run"]
    value = job_rate(updates, world, ms_per_step / 1000.0)

    # end-to-end through the public API with host buffers: H2D of b, D2H of the
    # postselected block into pinned memory, every step
    e2e_ms = []
    h2d = 0
    d2h = 0
    pinned = torch.empty(2 * circ.postselect_count(), dtype=torch.float64, pin_memory=True)
    for s in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        circ.init(f0, precision, stream)
        circ.run()
        amps, p, tot = circ.postselect(want_amplitudes=True, out=pinned.numpy())
        torch.cuda.synchronize()
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
        nnz = 3 * Nx + (9 * Nx * Nx if NC == 2 else 0)
        h2d = nnz * 16 + 2 * 64 * 8
        d2h = amps.nbytes + 16
    e2e_val = updates * world / (statistics.median(e2e_ms) / 1000.0)

    peaks, peak_kind = measured_peaks()
    sweep_ms = statistics.mean(run_ms) / passes
    # every sweep reads and writes the state once, except after a sparse
    # init: with one leading sweep it writes the state and reads only the
    # tiles of b; with two, the first touches only those tiles and the second
    # (a gather) writes the state and reads only those tiles
    sparse = int(info["sparse_init"])
    saved = {0: 0.0, 1: 1.0, 2: 3.0}[sparse]  # state passes (reads or writes) not needed
    alg_bytes = (2.0 * passes - saved) * (1 << n) * esz / passes
    achieved = alg_bytes / (sweep_ms / 1000.0) / 1e9
    khash = kernel_hash()
    traffic = NCU_TRAFFIC.get((khash, args.workload))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "complex64 (fp32)" if prec == "c64" else "complex128 (fp64)",
        "data": "synthetic",
        "config": {"workload": args.workload, "Nx": Nx, "N_C": NC, "K": K, "Nt": Nt, "dt": dt,
                   "tau": tau, "d": info["d"], "qubits": n, "exec": args.exec,
                   "boundary": BOUNDARY.get(args.workload, "periodic"),
                   "gather": (f"source-index tables ({info['n_src_tables']} x {(1 << n) / 1e9:.2f} GB)"
                              if info["n_src_tables"] else "lookup-table chain"),
                   "state_bytes": (1 << n) * esz,
                   "init": ({1: "tiles of b only; the first sweep writes the zeros of the rest",
                             2: "tiles of b only; the first sweep touches only those, the first "
                                "conjugated gather reads zeros for the rest"}[info["sparse_init"]]
                            if sparse else "whole state zero-filled"),
                   "l2": (f"inputs larger than L2 (state {((1 << n) * esz) / 1e6:.0f} MB, two "
                          f"ping-pong buffers {2 * ((1 << n) * esz) / 1e6:.0f} MB; L2 129 MB)"
                          if ((1 << n) * esz) > L2_BYTES
                          else "state resident in L2 (smaller than 129 MB); no flush"),
                   "parallelism": f"replicas x{world}", "host_cores": os.cpu_count(),
                   "autotune": tune},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "kernel": "sweep_kernel", "peak_kind": f"{peak_kind} (STREAM-style copy)",
                     "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": sweep_ms,
                     "launches_per_step": passes},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * (passes + (3 if sparse else 1) + 2),
        "clocks": clk,
        "host_wall_s": t_host,
    }
    if prec == "c128":
        # measured on the 28-qubit complex128 profile workload with ncu
        line["roofline"]["note"] = ("complex128 sweeps are bound by the FP64 pipe (83-86% of its "
                                    "cycles busy), not by HBM; see the fp64 sweep profile")
        line["fp64_peak_tflops_measured"] = measure_fp64_peak(torch)
    if (1 << n) * esz <= L2_BYTES:
        # an L2-resident state: its sweeps against the L2 copy bandwidth
        # measured here (the HBM figure above does not bound them)
        l2 = measure_l2_copy(torch, (1 << n) * esz)
        line["roofline_l2"] = {"bound": "l2", "achieved": achieved, "peak": l2, "unit": "GB/s",
                               "frac": achieved / l2,
                               "peak_kind": "measured here: device copy of a buffer of the state's "
                                            "size, best of 20, CUDA events"}
    if rank == 0 and not args.no_cpu_baseline:
        cfg = (Nx, tau, NC, K, dt, Nt)
        fd, o5_path = tempfile.mkstemp(suffix=".npz")
        os.close(fd)
        try:
            line["cpu_baseline"] = cpu_baselines(args.workload, cfg, f0, circ.export_phases(),
                                                 updates, out=o5_path)
            if args.workload.startswith("precision-") and args.exec == "fused":
                line["precision_comparison"] = precision_comparison(
                    torch, G, circ, cfg, f0, prec, o5_path, ms_per_step / 1000.0, stream)
        finally:
            os.unlink(o5_path)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _rel_l2_at(torch, dev_state, o5):
    """Relative L2 distance of the device state's entries at the oracle's
    physical indices from the oracle's block (both FP64 on the host)."""
    t = torch.as_tensor(dev_state, device="cuda")
    sel = t[torch.from_numpy(o5["idx"]).cuda()].double().cpu().numpy()
    got = sel[:, 0] + 1j * sel[:, 1]
    y = o5["y"]
    return float(np.linalg.norm(got - y) / np.linalg.norm(y))


def label_layer(records):
    """The QSVT circuit's label layer between the first U_L^dag and the next
    U_L: the unprepare Hadamards, the projector-phase gates and the prepare
    Hadamards (tags 4, 6, 1), the second such run of the gate list (the first
    sits before the first call)."""
    tags = records["tag"]
    runs, k = [], 0
    while k < len(records):
        if tags[k] in (1, 4, 6):
            j = k
            while j < len(records) and tags[j] in (1, 4, 6):
                j += 1
            if (tags[k:j] == 6).any():
                runs.append(records[k:j])
            k = j
        else:
            k += 1
    return runs[1] if len(runs) > 1 else runs[0]


def label_layer_alternative(torch, G, n, layer, stream, reps=3):
    """The label layer of the precision circuit applied alone to a seeded
    random complex64 state of the circuit's size, three ways, each timed over
    `reps` runs with CUDA events: the warp reduction the sweeps use (one
    streaming sweep), a dense block on the tensor cores (split BF16x3; the
    layer touches the five label qubits and the signal qubit, whose value
    selects the block's matrix), and the same block on the CUDA cores in
    FP32; the dense results against the warp reduction's, relative L2."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    x = torch.randn((1 << n, 2), generator=gen, device="cuda", dtype=torch.float32)
    x /= torch.linalg.vector_norm(x)
    sv = G.StateVector(n, G.CSIM_C64, stream)

    def one(dense, engine):
        old = os.environ.get("CSIM_DENSE_ENGINE")
        os.environ["CSIM_DENSE_ENGINE"] = engine
        try:
            sv.compile(layer, stage=0, dense=dense)
        finally:
            if old is None:
                os.environ.pop("CSIM_DENSE_ENGINE", None)
            else:
                os.environ["CSIM_DENSE_ENGINE"] = old
        st = sv.stats()
        sv.load_device(x.data_ptr())
        sv.run(1)
        torch.cuda.synchronize()
        out = torch.as_tensor(sv.device_state(), device="cuda").clone()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sv.run(reps)
        b.record(stream)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b) / reps, st

    ref, ms_warp, st0 = one(0, "tc")
    tc, ms_tc, st1 = one(2, "tc")
    err_tc = float(torch.linalg.vector_norm(tc - ref) / torch.linalg.vector_norm(ref))
    del tc
    f32, ms_f32, _ = one(2, "fp32")
    err_f32 = float(torch.linalg.vector_norm(f32 - ref) / torch.linalg.vector_norm(ref))
    del f32, ref, x
    sv.close()
    torch.cuda.empty_cache()
    return {"gates": int(len(layer)), "qubits": n,
            "warp_reduction": {"ms_per_pass": ms_warp, "passes": st0["passes"]},
            "tensor_cores_bf16x3": {"ms_per_pass": ms_tc, "passes": st1["passes"],
                                    "dense_blocks": st1["dense_blocks"],
                                    "rel_l2_vs_warp_reduction": err_tc},
            "cuda_cores_fp32": {"ms_per_pass": ms_f32, "rel_l2_vs_warp_reduction": err_f32},
            "kept": "warp reduction: in the circuit it rides in the conjugated and multiplexer "
                    "sweeps with the gather and the multiplexers, at no pass of its own"}


def precision_comparison(torch, G, circ, cfg, f0, prec, o5_path, fused_s, stream):
    """The precision configuration's comparison, outside the timed region: the
    fused run just timed against the plain gate-by-gate complex128 GPU path on
    the same circuit (one step, CUDA events), each result's relative L2 error
    against the oracle's classical evaluation on the physical entries (all
    time slots, t = s = label = 0)."""
    with np.load(o5_path) as z:
        o5 = {"y": z["y"], "idx": z["idx"]}
    err_fused = _rel_l2_at(torch, circ.device_state(), o5)
    ph = circ.export_phases()
    Nx, tau, NC, K, dt, Nt = cfg
    layer = label_layer(circ.export_gates(1))
    n = circ.info()["n_qubits"]
    circ.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    alt = label_layer_alternative(torch, G, n, layer, stream) if prec == "c64" else None
    plain = G.Circuit(Nx, tau, NC, K, dt, Nt, phases=ph)
    plain.set_exec(G.CSIM_EXEC_GATE)
    plain.compile()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    plain.init(f0, G.CSIM_C128, stream)
    plain.run()
    plain.postselect(want_amplitudes=False)
    b.record(stream)
    torch.cuda.synchronize()
    plain_s = a.elapsed_time(b) / 1000.0
    err_plain = _rel_l2_at(torch, plain.device_state(), o5)
    n_gates = plain.info()["n_gates_total"]
    plain.close()
    torch.cuda.empty_cache()
    return {
        "fused": {"dtype": "complex64" if prec == "c64" else "complex128", "s_per_run": fused_s,
                  "runs_per_s": 1.0 / fused_s, "rel_l2_vs_oracle": err_fused,
                  "tolerance": 1e-4 if prec == "c64" else 1e-12},
        "plain_c128_gate_by_gate": {"s_per_run": plain_s, "runs_per_s": 1.0 / plain_s,
                                    "rel_l2_vs_oracle": err_plain, "tolerance": 1e-12,
                                    "launches": n_gates},
        "runs_per_s_ratio": plain_s / fused_s,
        "label_layer_alternative": alt,
        "oracle": (f"classical QSVT evaluation (O5, FP64) of the same phases, compared on the "
                   f"{o5['y'].size} physical entries"),
    }


if __name__ == "__main__":
    main()
