/*
 * csim.h -- C ABI of the GB300 state-vector simulator for the Carleman-linearised
 * D1Q3 lattice-Boltzmann QSVT circuit (Kanno et al., "Explicit Quantum Circuit
 * Simulation of Nonlinear 1-Dimensional Fluid with Carleman-linearized Boltzmann
 * Method").
 *
 * The calls follow the paper's statement of the problem:
 *   csim_build      -- register layout, gate list and QSP phases (Sec. II.D; Fig. L;
 *                      Fig. circuit-qsvt; Eq. d-star), host only, FP64.
 *   csim_init       -- load f(0) as the right-hand side b (Sec. II.D.5).
 *   csim_run        -- apply the QSVT circuit on the GPU.
 *   csim_postselect -- final-time block (ancillas 0, signal 0, m >= Nt) and its
 *                      success probability (Sec. II.D.4-5).
 *
 * Conventions for every entry point:
 *   - Every call returns a csim_status; nothing throws across the ABI.
 *     csim_last_error() returns a thread-local message for the last failure.
 *   - The library owns the handle and all device memory it allocates.  The
 *     caller owns every host buffer it passes and keeps it valid for the call.
 *   - Device work is asynchronous on the CUDA stream given to csim_init
 *     (NULL = the legacy default stream).  csim_sync waits for it.
 *   - One handle must not be used by two threads at the same time.  Handles
 *     may share a stream.
 *   - Complex amplitudes cross the ABI as interleaved (re, im) doubles.
 *   - Qubit indices are bit positions in the state index (bit 0 least
 *     significant).  Registers are little-endian and allocated from bit 0 up:
 *       t    1 bit   value-encoding target of the RY branches
 *       s    1 bit   QSVT signal qubit
 *       iL   n_iL    row label of U_L (n_iL = max(1 + n_iA, 2 + n_k), n_iA = 2
 *                    for N_C = 1 and 4 for N_C = 2); iL[0..1] is the A11
 *                    output-velocity label, iL[2..3] the N_C = 2 case label
 *       q1   2 bits  velocity 0 (e = +1), 1 (e = -1), 2 (e = 0); 3 unused
 *       a1   n_a     lattice site (n_a = log2 Nx)
 *       q2, a2, ord  (N_C = 2 only) second velocity, second site, Carleman
 *                    order (0: f^(1), 1: f^(1) (x) f^(1))
 *       k    n_k     Taylor index (n_k = bit length of K)
 *       m    n_m     time step (n_m = bit length of Nt - 1, plus 1)
 *     A basis state is physical when t, s and iL are 0, every velocity is at
 *     most 2 and, for N_C = 2 and ord = 0, q2 = a2 = 0.  csim_info reports n;
 *     csim_export_mask gives the postselected patterns in these bit positions.
 */
#ifndef CSIM_H
#define CSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct csim_circuit csim_circuit; /* opaque, library-owned */
typedef struct csim_sv csim_sv;           /* opaque raw state vector, library-owned */

typedef enum {
  CSIM_OK = 0,
  CSIM_ERR_ARG = -1,       /* invalid argument or buffer too small */
  CSIM_ERR_TOO_LARGE = -2, /* qubit count above the limit */
  CSIM_ERR_OOM = -3,       /* device or host allocation failed; nothing kept */
  CSIM_ERR_CUDA = -4,      /* a CUDA call failed (message in csim_last_error) */
  CSIM_ERR_STATE = -5,     /* call out of order (e.g. run before init) */
  CSIM_ERR_TIMEOUT = -6,   /* a bounded device wait expired */
  CSIM_ERR_NUMERIC = -7    /* phase solver or norm check failed */
} csim_status;

typedef enum { CSIM_C64 = 0, CSIM_C128 = 1 } csim_precision;
typedef enum { CSIM_BC_PERIODIC = 0, CSIM_BC_BOUNCEBACK = 1 } csim_bc;

/* How csim_run applies the gate list.
 *   CSIM_EXEC_FUSED: the fuser groups gates into sweeps (one HBM pass each).
 *   CSIM_EXEC_GATE:  one kernel launch per elementary gate (the plain path). */
typedef enum { CSIM_EXEC_FUSED = 0, CSIM_EXEC_GATE = 1 } csim_exec;

/* Gate record: 32 bytes.  op 0 = X, 1 = H, 2 = RY(angle), 3 = ZPHASE(angle) =
 * e^{i angle Z}.  The gate acts on `target` for every basis index with
 * (index & cmask) == cval.  tag: 1/4 label H layers, 2 permutation, 3 value
 * encoding, 5 target X, 6 projector phase, 7 signal H (0 for user gates). */
typedef struct {
  uint8_t op;
  uint8_t target;
  uint16_t tag;
  uint32_t reserved; /* 0 */
  uint64_t cmask;
  uint64_t cval;
  double angle;
} csim_gate;

/* Build options.  Zero or negative numeric fields select the defaults. */
typedef struct {
  int32_t Nx;          /* grid size, power of two >= 2 */
  double tau;          /* BGK relaxation time > 0 */
  int32_t N_C;         /* Carleman order, 1 or 2 */
  int32_t K;           /* Taylor order >= 1 */
  double dt;           /* time step > 0 */
  int32_t Nt;          /* number of time steps >= 1 */
  int32_t bc;          /* csim_bc: periodic, or bounce-back walls (a population
                          leaving the lattice returns to its site with the
                          opposite velocity) */
  double kappa_qsvt;   /* <= 0: kappa(L) = lambda_L / sigma_min(L), computed */
  int32_t d;           /* <= 0: Eq. d-star, odd ceil(kappa ln(2 kappa/eps)/2) */
  double eps;          /* <= 0: 1e-3 */
  int32_t max_qubits;  /* <= 0: 34 */
  const double* phases; /* NULL: computed; else n_phases = d+1 phases (copied) */
  int32_t n_phases;
} csim_build_opts;

typedef struct {
  int32_t n_qubits;
  int32_t d;              /* QSVT degree (odd) = number of U_L / U_L^dag calls */
  int32_t n_a, n_k, n_m, n_iL;
  double lambda_L;        /* 2^{n_iL} L_max (Sec. II.D.4) */
  double L_max;
  double kappa_qsvt;      /* design parameter of the 1/x polynomial */
  double poly_scale;      /* target polynomial = poly_scale * p(x), p ~ 1/x */
  int64_t n_gates_UL;     /* gates of one U_L */
  int64_t n_gates_total;  /* gates of the whole QSVT circuit */
  int64_t n_sweeps_run;   /* fused sweeps (HBM passes) per csim_run = program steps;
                             0 until csim_init (fused mode), csim_run or
                             csim_run_steps fuses the program
                             (csim_run_steps(c, 0, ...) fuses only) */
  double amp_updates_run; /* sum over gates of amplitudes the gate changes */
  uint64_t state_bytes;   /* bytes of the current state (0 before csim_init) */
  int32_t n_src_tables;   /* source-index tables the gather sweeps load (2^n bytes
                             each; 0: the sweeps walk the lookup-table chain) */
  int32_t sparse_init;    /* > 0: the last csim_init wrote the tiles of b only and
                             left the zeros to the first sparse_init sweeps
                             (csim_init); 0: it wrote the whole state */
} csim_info_t;

/* --- building (host only; no GPU needed) -------------------------------- */

/* Compile the circuit for the D1Q3 Carleman system of order N_C with Taylor
 * order K, step dt and Nt steps (Sec. II.B-D), periodic or with the bounce-back
 * walls of Sec. II.A (csim_build_ex).  Defaults: periodic, eps
 * 1e-3, kappa_qsvt = kappa(L), d from Eq. d-star, phases by Newton iteration.
 * Errors: CSIM_ERR_ARG for invalid parameters (Nx not a power of two >= 2,
 * tau/dt <= 0, N_C not 1/2, K < 1, Nt < 1), CSIM_ERR_TOO_LARGE above
 * max_qubits, CSIM_ERR_NUMERIC if the phase solver does not converge.
 * On success *out receives a new handle (free with csim_free). */
csim_status csim_build(int32_t Nx, double tau, int32_t N_C, int32_t K, double dt,
                       int32_t Nt, csim_circuit** out);
csim_status csim_build_ex(const csim_build_opts* opts, csim_circuit** out);

csim_status csim_info(const csim_circuit* c, csim_info_t* out);

/* Canonical gate list.  which = 0: one U_L; which = 1: the whole QSVT circuit
 * (H_s, PHI(phi_0), d alternating calls U_L^dag, U_L, U_L^dag, ... each followed by
 * PHI, H_s; starting with U_L^dag makes the 1/x polynomial act as lambda_L L^{-1}).
 * Writes min(cap, total) records to buf (may be NULL when cap = 0) and the
 * total count to *len.  Returns CSIM_ERR_ARG if cap < total and buf != NULL. */
csim_status csim_export_gates(const csim_circuit* c, int32_t which, csim_gate* buf,
                              size_t cap, size_t* len);

/* QSP phases phi_0..phi_d (reflection convention of Fig. circuit-qsvt). */
csim_status csim_export_phases(const csim_circuit* c, double* buf, size_t cap, size_t* len);

/* Postselection mask as a union of (mask, value) patterns over the state index:
 * s = 0, t = 0, label = 0, m >= Nt. */
csim_status csim_export_mask(const csim_circuit* c, uint64_t* masks, uint64_t* vals,
                             size_t cap, size_t* len);

/* --- device path ---------------------------------------------------------- */

/* Allocate the 2^n-amplitude state (complex64 or complex128) on the current
 * CUDA device and load b: f0 is [Nx][3] doubles in the paper's velocity order
 * (e = +1, -1, 0); the Carleman vector (f0, f0 (x) f0) is normalised and
 * placed in slot (m, k) = (0, 0) with all ancillas 0 (Sec. II.D.5).  A second
 * call reuses the allocation when the precision is unchanged.
 * In the fused mode at n >= 12, when the program's first step is an in-place
 * sweep (the circuit's opening Walsh-Hadamard and multiplexer), csim_init
 * fuses the program, writes only the 128-amplitude tiles that hold b and
 * marks them in a 2^(n-12)-word bitmap.  The leading sweeps write the zeros
 * of the unmarked tiles instead of a memset: the first sweep itself
 * (csim_info().sparse_init = 1), or, when the second is a conjugated gather,
 * that gather, which reads zeros for chunks in unmarked tiles while the first
 * sweep touches only the marked ones (sparse_init = 2).  CSIM_SPARSE_INIT=0 in
 * the environment always writes the whole state.  Every call that reads the
 * state before those sweeps have run (csim_read_state, csim_checkpoint,
 * csim_state_device, csim_postselect) zeroes the unmarked tiles first, so the
 * difference is not observable.  Errors: CSIM_ERR_OOM (nothing kept),
 * CSIM_ERR_CUDA. */
csim_status csim_init(csim_circuit* c, const double* f0, csim_precision prec,
                      void* cuda_stream);

csim_status csim_set_exec(csim_circuit* c, csim_exec mode);

/* Launch-shape autotuner of the fused sweeps, per (precision, qubit count)
 * class.  Times the circuit's first max_steps program steps on a scratch
 * state of its size (two buffers when the program moves data; filled with
 * finite values; CSIM_ERR_OOM when they cannot be allocated) for each
 * candidate launch shape: the default kernel variant (tiles per warp
 * iteration u, minimum resident blocks per SM minb) at grids of 1, 2, 4 and
 * 8 resident waves, and every other variant at the default grid.  Each
 * candidate runs once untimed, then `reps` times between CUDA events.  The
 * fastest becomes the process-wide shape of the class: every later sweep of a
 * fused program on a state of this precision and size uses it, except the
 * sweeps that complete a sparse csim_init (their zero handling exists in the
 * default variant only).  The circuit's own state is not touched.  Results do
 * not depend on the shape beyond rounding: variants other than the default
 * run the general op interpreter instead of the shaped op lists.  Needs the
 * fused exec mode. */
typedef struct {
  int32_t u, minb, waves;  /* chosen shape */
  double ms;               /* time of the steps with it */
  double ms_default;       /* time of the steps with the default shape */
  int32_t steps;           /* program steps timed */
  int32_t n_trials;
  int32_t trial_u[32], trial_minb[32], trial_waves[32];
  double trial_ms[32];
} csim_launch_tune_t;
csim_status csim_tune_launch(csim_circuit* c, csim_precision prec, int32_t max_steps,
                             int32_t reps, csim_launch_tune_t* out);
/* Set the launch shape of a class directly (u = 0 clears it; the default
 * shape is then used).  u in {1, 2, 4}, minb in {1, 2, 4} (not 4 with 4),
 * waves in 1..64; CSIM_ERR_ARG otherwise. */
csim_status csim_set_launch_shape(csim_precision prec, int32_t n_qubits, int32_t u, int32_t minb,
                                  int32_t waves);

/* Compile the circuit's program for the current exec mode on the host (the
 * fusing that the first csim_run or pool submission would otherwise do); no
 * GPU work.  Calls on different handles may run in parallel threads. */
csim_status csim_compile(csim_circuit* c);

/* Enqueue the whole QSVT circuit on the stream.  CSIM_ERR_STATE unless a
 * csim_init has loaded the state since the last run.  When the program's
 * last sweep is the shaped last-sweep kernel of the default variant, it also
 * sums |a|^2 of the state it writes (FP64 per-block partials; complex64
 * amplitudes squared and added in FP32 four at a time), which the next
 * csim_postselect takes as the total instead of reading the state again
 * (csim_run_steps does the same when it runs the last sweep). */
csim_status csim_run(csim_circuit* c);
csim_status csim_sync(csim_circuit* c);

/* Synchronises, then reduces in FP64 on the device: *norm_total = sum |a|^2
 * over the whole state and *p_success = sum |a|^2 over the postselection mask.
 * out_amps (caller-owned, may be NULL) receives the masked amplitudes with
 * s = t = label = 0 and m >= Nt, ordered by state index, as interleaved
 * doubles; cap counts complex amplitudes, *len receives the total. */
csim_status csim_postselect(csim_circuit* c, double* out_amps, size_t cap, size_t* len,
                            double* p_success, double* norm_total);

/* The final-time distribution f(T)[alpha][q] (alpha = 0..Nx-1, q in the order
 * e = +1, -1, 0), read from the compacted block that csim_postselect returned
 * (amps: len complex amplitudes, interleaved).  It is the f^(1) part (ord = 0,
 * second site and velocity 0 at N_C = 2) of the first postselected slot
 * (m = Nt, k = 0; Sec. II.D.4), rescaled to physical units: the block
 * approximates poly_scale * lambda_L * L^{-1} b with b = v0 / |v0| and v0 the
 * Carleman vector of f0 (Sec. II.D.5), so f(T) = Re(block) |v0| /
 * (poly_scale lambda_L).  f0 is the initial distribution passed to csim_init
 * (3 Nx doubles); f_out receives 3 Nx doubles.  Host arithmetic only.
 * CSIM_ERR_ARG for a short block or a zero f0. */
csim_status csim_final_distribution(const csim_circuit* c, const double* f0, const double* amps,
                                    size_t len, double* f_out);

/* Copy the whole state to the host as interleaved doubles (2 * 2^n values). */
csim_status csim_read_state(csim_circuit* c, double* out, size_t cap_amps);

/* Checkpointed runs, for circuits of large degree (Sec. III.E.2: d ~ 7e4 calls).
 * The QSVT circuit is executed as a fixed sequence of program steps (fused
 * sweeps or single gates; csim_info().n_sweeps_run of them).
 *   csim_run_steps: after csim_init or csim_restore, enqueue the next n_steps
 *     steps (fewer at the end); *next_step (may be NULL) receives the index of
 *     the next step.  When the last step has run, the run is complete, as after
 *     csim_run.  csim_run finishes a run that csim_run_steps started.  With
 *     n_steps = 0 it fuses the program and runs nothing, after which
 *     csim_info().n_sweeps_run holds the step count.
 *   csim_checkpoint: synchronise, copy the state to the host (2 * 2^n doubles,
 *     as csim_read_state) and return the next step index.
 *   csim_restore: load such a state (in either precision) and the step index
 *     into this or another handle of the same circuit, allocating like
 *     csim_init, so that csim_run_steps / csim_run continue from there.
 * A run split at any step boundary, with or without a checkpoint round trip,
 * gives the same state as csim_run (complex128 round trips are exact).
 * Errors: CSIM_ERR_STATE without a loaded state, CSIM_ERR_ARG for a bad size
 * or step index, CSIM_ERR_OOM, CSIM_ERR_CUDA. */
csim_status csim_run_steps(csim_circuit* c, int64_t n_steps, int64_t* next_step);
csim_status csim_checkpoint(csim_circuit* c, double* out, size_t cap_amps, int64_t* next_step);
csim_status csim_restore(csim_circuit* c, const double* amps, size_t n_amps, csim_precision prec,
                         int64_t next_step, void* cuda_stream);

/* Borrowed device pointer to the circuit's current state: 2^n amplitudes,
 * float2 (complex64) or double2 (complex128) per *prec, index bit b = qubit b.
 * Valid until the next csim_init, csim_run or csim_free of this handle; the
 * library keeps ownership.  For reading sampled amplitudes on the device
 * without a 2^n host copy.  CSIM_ERR_STATE when no state is loaded. */
csim_status csim_state_device(const csim_circuit* c, void** d_state, int32_t* n,
                              csim_precision* prec);

csim_status csim_free(csim_circuit* c);

/* --- raw state vectors (microbenchmark and parity tests) ---------------- */

/* A 2^n-amplitude state on the current device (n <= 34), zero-initialised. */
csim_status csim_sv_create(int32_t n, csim_precision prec, void* cuda_stream, csim_sv** out);
/* Host -> device copy of 2^n interleaved complex values. */
csim_status csim_sv_load(csim_sv* sv, const double* amps, size_t n_amps);
/* Compile (fuse) a gate list for this state; the program is kept in the handle. */
csim_status csim_sv_compile(csim_sv* sv, const csim_gate* gates, size_t n_gates, csim_exec mode);
/* Enqueue the compiled program `reps` times. */
csim_status csim_sv_run(csim_sv* sv, int32_t reps);
csim_status csim_sv_read(csim_sv* sv, double* out, size_t n_amps);
/* Device -> device copy of 2^n amplitudes already in the state's precision
 * (float2 or double2), e.g. a seeded random state generated on the GPU. */
csim_status csim_sv_load_device(csim_sv* sv, const void* d_amps, size_t n_amps);
/* Borrowed device pointer to the current state (valid until the next
 * csim_sv_run, csim_sv_load* or csim_sv_free). */
csim_status csim_sv_device(const csim_sv* sv, void** d_state);
csim_status csim_sv_info(const csim_sv* sv, int64_t* n_sweeps, double* amp_updates,
                         uint64_t* state_bytes);
/* Program statistics of the compiled gate list (zeros before a compile).
 * pass_amps: amplitudes the passes must read and write at minimum, 2^n per
 * fused sweep and the changed amplitudes per single-gate pass, so that
 * 2 * pass_amps * (8 or 16 bytes) is the algorithmic HBM traffic of one run. */
typedef struct {
  int64_t passes;       /* kernel launches (HBM passes) per run */
  int64_t sweeps;       /* of which fused sweeps */
  int64_t single;       /* of which single-gate passes */
  double amp_updates;   /* sum over gates of the amplitudes each gate changes */
  double pass_amps;
  uint64_t state_bytes;
  int64_t dense_blocks;  /* of the passes, dense 5-qubit blocks */
  int64_t staged_sweeps; /* of the fused sweeps, those that stage qubits above the tile */
} csim_sv_stats_t;
csim_status csim_sv_stats(const csim_sv* sv, csim_sv_stats_t* out);
csim_status csim_sv_free(csim_sv* sv);

/* csim_sv_compile with the fuser's choices fixed: stage = how many qubits
 * above the warp tile a sweep may stage (0-3; -1 the default), dense = 0 no
 * dense blocks, 1 dense blocks for runs on at most five qubits (plus up to
 * two selector qubits) that mix amplitudes across the warp tile, 2 for every
 * such run of at least the minimum length, inside the tile too (-1 the
 * default).  Dense blocks need a complex64 state of at least 12 qubits. */
csim_status csim_sv_compile_opts(csim_sv* sv, const csim_gate* gates, size_t n_gates,
                                 csim_exec mode, int32_t stage, int32_t dense);

/* Autotuner of a gate stream's fusion width.  Compiles the gate list (fused)
 * with every staging width k = 0..3 (how many qubits above the warp tile a
 * sweep may hold in registers) and, for complex64 states of at least 12
 * qubits whose stream has runs on at most five qubits, with and without
 * dense blocks; times `reps` runs of each on this state after one untimed run
 * (CUDA events on the state's stream), and leaves the fastest program
 * compiled, as csim_sv_compile would.  The state is restored afterwards: the
 * call takes a device copy of it for the duration (CSIM_ERR_OOM when that
 * copy cannot be allocated).  out receives the choice, its time per run and
 * up to 8 trials.  Later csim_sv_compile calls on this state use the chosen
 * width and dense-block setting. */
typedef struct {
  int32_t stage;        /* chosen staging width */
  int32_t dense;        /* 1: dense blocks chosen */
  double ms;            /* time per run of the chosen program */
  int32_t n_trials;
  int32_t trial_stage[8];
  int32_t trial_dense[8];
  double trial_ms[8];
} csim_tune_t;
csim_status csim_sv_autotune(csim_sv* sv, const csim_gate* gates, size_t n_gates, int32_t reps,
                             csim_tune_t* out);

/* A dense 5-qubit block: apply the 32 x 32 complex matrix u (row-major,
 * interleaved re/im doubles; element bit j of its row and column index is
 * qubit qubits[j]) to the complex64 state, for every group of 32 amplitudes
 * that differ only in those five distinct qubits.  Enqueued on the state's
 * stream; the fuser emits the same operation for long runs of gates on at
 * most five qubits.  engine 0: the tensor cores (tcgen05 MMA into TMEM, split
 * BF16x3 with FP32 accumulation: each factor is a sum of two BF16 values,
 * three of the four cross products are kept, relative error about 2^-17 per
 * product; n >= 12); engine 1: the CUDA cores in FP32 (n >= 5).  The
 * tensor-core kernel waits for its products with an iteration limit; when it
 * runs out the kernel gives up on the state and the next csim_sv_read
 * returns CSIM_ERR_TIMEOUT.  CSIM_ERR_ARG for a complex128 state, repeated or
 * out-of-range qubits, too few qubits or an unknown engine. */
csim_status csim_sv_apply_dense(csim_sv* sv, const int32_t* qubits, const double* u,
                                int32_t engine);

/* Host-only reference executor of the fused-program format: compiles the gate
 * list with the same fuser as CSIM_EXEC_FUSED and executes the resulting
 * sweeps (lookup-table permutations, multiplexed rotations, warp-tile gates)
 * on the host in FP64 with the kernel's semantics.  amps: 2^n interleaved
 * complex values, updated in place (n in [7, 24]), or NULL to compile only and
 * report the statistics (n in [7, 34]).  For testing the fuser without a GPU.
 * If stats is non-NULL it receives 20 counters: sweeps, single-gate steps,
 * permutation gates, lookup tables, local gates, multiplexers, multiplexed
 * gates, multiplexer entries, largest bucket, table entries, largest table
 * support, HBM passes, averaging blocks, multiplexers run as the inverse of
 * the sweep's previous multiplexer, Walsh-Hadamard ops (H on several lane
 * bits fused), in-place conjugated sweeps (a permutation, tile ops and the
 * inverse permutation), sweeps that stage qubits above the warp tile in
 * registers, gates on those staged qubits, dense 5-qubit blocks, and the
 * gates those blocks hold. */
csim_status csim_emulate_fused(const csim_gate* gates, size_t n_gates, int32_t n, double* amps,
                               int64_t* stats);

/* --- request pool: batching and serving ----------------------------------- */

/* Many independent runs (instances or serving requests) on one GPU.  The pool
 * owns an arena of hbm_budget bytes (a buddy allocator over power-of-two
 * blocks: each request takes its two state buffers, the compacted block and
 * the staging of b) and n_streams CUDA streams.  Queued requests are admitted
 * in submission order whenever a stream is free and the head request's blocks
 * fit; finished requests release their blocks at the next csim_pool_poll, so
 * new work is admitted continuously.  With use_graphs, the requests admitted in
 * one pass are captured into one CUDA graph (a branch per request) and
 * launched once.  A pool is used from one thread at a time.  A circuit stays
 * borrowed while it has requests in the pool: do not csim_free it or change
 * its exec mode until their results are taken. */
typedef struct csim_pool csim_pool;
typedef struct {
  int32_t n_streams;    /* concurrent requests; <= 0: 4 (max 64) */
  int32_t max_qubits;   /* larger circuits are rejected; <= 0: 32 */
  uint64_t hbm_budget;  /* arena bytes; 0: 90% of the free device memory */
  int32_t use_graphs;   /* 1: one CUDA graph launch per admission pass */
  uint32_t min_block;   /* smallest arena block in bytes, a multiple of 256; 0: 1 MiB */
  int32_t persistent;   /* 1: the sweeps of the complex64 requests admitted in one pass
                           run in one persistent launch (see below) */
} csim_pool_opts;
typedef struct {
  int64_t submitted, admitted, completed, rejected, queued, running;
  uint64_t bytes_in_use, peak_bytes, budget;
  int64_t graph_launches; /* admission passes launched as one CUDA graph */
  int64_t src_tables;     /* source-index tables built in the arena for admitted requests */
  uint64_t sparse_saved_bytes; /* state reads and writes that admitted requests'
                                  sparse inits left out: one state's bytes per
                                  request with one leading sweep, three with two */
  int64_t failed;         /* requests that failed: refused pinned or arena allocations,
                             and every request of a persistent pass whose wait ran out */
  int64_t cancelled;      /* csim_pool_cancel calls that took effect */
  int64_t batch_launches; /* admission passes run as one persistent launch */
  int64_t batch_dropped_signals; /* persistent passes launched with an injected missing signal */
  int64_t batch_requests; /* requests whose sweeps ran in a persistent launch */
} csim_pool_stats_t;

csim_status csim_pool_create(const csim_pool_opts* opts, csim_pool** out);
/* Queue one run of circuit c (QSVT circuit on b from f0, as csim_init +
 * csim_run + csim_postselect) and try to admit (in persistent mode, admission
 * waits for the next csim_pool_poll).  f0 is copied.  *id receives
 * the request id.  Besides its state buffers, a request takes the source-index
 * tables of its sweeps from the arena (2^n bytes per distinct permutation
 * chain, one for a QSVT circuit; built on the request's stream before its
 * sweeps), unless the circuit already holds its own from a csim_run or the
 * request fits the arena only without them.  CSIM_ERR_TOO_LARGE (counted as
 * rejected) when the circuit exceeds max_qubits or its blocks cannot fit the
 * arena. */
csim_status csim_pool_submit(csim_pool* p, csim_circuit* c, const double* f0,
                             csim_precision prec, int64_t* id);
/* Retire finished requests and admit queued ones.  wait_ms > 0 blocks until a
 * request finishes or the time passes.  Writes up to cap ids of requests
 * finished since the last poll to done (NULL: keep them for later). */
csim_status csim_pool_poll(csim_pool* p, int32_t wait_ms, int64_t* done, size_t cap,
                           size_t* n_done);
/* Results of a finished request, as csim_postselect; times (may be NULL)
 * receives 5 doubles in seconds: queueing (submit to admission), submit to
 * retirement, device time of the request, and its device start and end on
 * the pool's clock (after an event recorded when the pool was created; -1
 * for requests run inside a graph, whose events do not time).  Releases the
 * request record.  A request that failed before its device work (see
 * failures below) returns that error here, with its message, and is released
 * too. */
csim_status csim_pool_result(csim_pool* p, int64_t id, double* p_success, double* norm_total,
                             double* out_amps, size_t cap, size_t* len, double* times);
/* Cancel a request.  A queued request leaves the queue at once; a running one
 * cannot be stopped on the device, so its work finishes and its blocks are
 * freed at retirement with the result dropped; a finished one is released.
 * Either way the id is no longer reported or accepted, and whatever memory or
 * slot this frees goes to the next queued requests.  CSIM_ERR_ARG for an
 * unknown id.
 *
 * Failures of single requests: when a request's pinned staging (or, through
 * csim_pool_inject, its arena blocks) cannot be allocated at admission, that
 * request alone fails: it leaves the queue holding no memory, poll reports it,
 * csim_pool_result returns CSIM_ERR_OOM, and the other requests proceed. */
csim_status csim_pool_cancel(csim_pool* p, int64_t id);
/* Host-side fault injection for tests: make an allocation of request `id`
 * fail at its admission as if the host or the arena refused it
 * (CSIM_INJECT_PINNED: the pinned staging; CSIM_INJECT_ARENA: the arena
 * blocks; CSIM_INJECT_NONE clears), or, in persistent mode, keep one work
 * item of the second sweep the launch runs for the request from signalling
 * its completion
 * (CSIM_INJECT_BATCH_SIGNAL): the items that depend on it wait out their
 * time limit and the whole pass reports CSIM_ERR_TIMEOUT.  Nothing is faulted
 * on the device.
 *
 * Persistent mode (csim_pool_opts.persistent): submissions only queue, and
 * the next csim_pool_poll admits them, so a burst of submissions forms
 * admission passes of at most half of n_streams requests each (the next pass
 * is admitted while one runs).  A pass's complex64 requests of at least 12
 * qubits whose steps are all sweeps with one of the four op lists of the QSVT
 * circuits' sweeps (gathers from source-index tables) run as: their uploads,
 * inits, tables and the sweeps that complete a sparse init (with the sweep
 * kernels); one launch of a persistent kernel over all their other sweeps;
 * their norms, compactions and result copies; all on the stream of the
 * pass's first slot.  The pass's other requests run on their own streams as
 * in stream mode (use_graphs is not combined with it).  The kernel's CTAs
 * take work items (64 warp iterations of one sweep of one request) from a
 * queue in device memory, ordered by each request's relative progress, and
 * wait, with a 2 s limit per wait, for the previous sweep of the same
 * request; at the end of the queue, CTAs beyond the items left leave, so
 * consecutive passes (on different streams) overlap.  The kernel runs the
 * sweep kernels' op bodies: the amplitudes equal the run alone; each
 * request's last sweep also sums |a|^2 per work item for its norms, which
 * agree with the run alone up to the order of the FP64 summation. */
enum { CSIM_INJECT_NONE = 0, CSIM_INJECT_PINNED = 1, CSIM_INJECT_ARENA = 2,
       CSIM_INJECT_BATCH_SIGNAL = 3 };
csim_status csim_pool_inject(csim_pool* p, int32_t what, int64_t id);
csim_status csim_pool_stats(const csim_pool* p, csim_pool_stats_t* out);
/* Waits for running work, then frees everything (pending results are lost). */
csim_status csim_pool_free(csim_pool* p);

/* The pool's admission policy on a simulated clock (host only, no GPU):
 * request i arrives at arrival[i] (NULL: all at 0), needs the 4 blocks
 * alloc_bytes[4i..4i+3] (0 = none) and runs for duration[i].  Writes start[i]
 * and finish[i] (-1 for a request that cannot fit an empty arena) and the
 * peak arena bytes in use.  For capacity planning and for testing the policy. */
csim_status csim_pool_plan(uint64_t budget, uint64_t min_block, int32_t n_streams, size_t count,
                           const uint64_t* alloc_bytes, const double* arrival,
                           const double* duration, double* start, double* finish,
                           uint64_t* peak_bytes);

/* --- reduction for callers that cannot allocate -------------------------- */

/* csim_norms_noalloc has no counterpart in the paper.  It is the FP64
 * reduction of csim_postselect, offered to callers that cannot call cudaMalloc:
 * code inside another framework's memory pool that forbids side allocations,
 * or a host that keeps its device footprint fixed after start-up.  The call
 * allocates nothing.  Its per-block partial sums live in a fixed library array
 * of 2048 (total, masked) pairs, 32 KiB, which every GPU that loads the library
 * holds until the process exits.
 *
 * d_state: 2^n amplitudes on the current device, complex64 (float2) or
 * complex128 (double2) as `prec` says, 16-byte aligned; n in [1, 34].
 * pm, pv: host arrays of npat masks and values (0 <= npat <= 16); an index i
 * is selected when (i & pm[k]) == pv[k] for some k (csim_export_mask gives the
 * circuit's postselection patterns).
 * d_out: device memory for 2 doubles, 8-byte aligned, receiving sum |a|^2 over
 * the whole state and over the selected indices (each |a|^2 formed and summed
 * in FP64, complex64 amplitudes widened first).
 * The work is enqueued on cuda_stream (NULL = the legacy default stream); the
 * call does not synchronise.  The caller owns d_state, d_out and the host
 * arrays, which only need to stay valid for the call itself.
 *
 * Errors: CSIM_ERR_TOO_LARGE for n > 34 or more than 16 patterns; CSIM_ERR_ARG
 * for null or misaligned pointers (d_state not 16-byte, d_out not 8-byte
 * aligned), n < 1, a value outside its mask, or a mask with bits at or above
 * n; CSIM_ERR_CUDA when the launch or the set-up fails (a failed set-up is
 * retried by the next call).
 *
 * The first call on each device looks up the array's device address with that
 * device current.  That lookup can load the library's module, so make the
 * first call on each device before any stream capture begins.  Every call
 * shares the one array per device and leaves its partial sums there.  Nothing
 * in it has to start at zero, but calls that overlap on the GPU (on different
 * streams of one device) race on it. */
csim_status csim_norms_noalloc(const void* d_state, int32_t n, csim_precision prec,
                               const uint64_t* pm, const uint64_t* pv, int32_t npat,
                               double* d_out, void* cuda_stream);

const char* csim_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CSIM_H */
