"""ctypes binding of include/csim.h (argument marshalling only).

Every function here forwards to the C ABI of ``_lib/libcsim.so``; all
computation happens in the library (host compiler in C++, state-vector work
in the CUDA kernels).  There is no Python fallback: if the library or a GPU
is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcsim.so")

CSIM_OK, CSIM_ERR_ARG, CSIM_ERR_TOO_LARGE, CSIM_ERR_OOM = 0, -1, -2, -3
CSIM_ERR_CUDA, CSIM_ERR_STATE, CSIM_ERR_TIMEOUT, CSIM_ERR_NUMERIC = -4, -5, -6, -7
CSIM_C64, CSIM_C128 = 0, 1
CSIM_EXEC_FUSED, CSIM_EXEC_GATE = 0, 1
CSIM_INJECT_NONE, CSIM_INJECT_PINNED, CSIM_INJECT_ARENA, CSIM_INJECT_BATCH_SIGNAL = 0, 1, 2, 3
_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_TOO_LARGE", -3: "ERR_OOM", -4: "ERR_CUDA",
          -5: "ERR_STATE", -6: "ERR_TIMEOUT", -7: "ERR_NUMERIC"}

# Every symbol declared in include/csim.h.
EXPORTED = [
    "csim_build", "csim_build_ex", "csim_info", "csim_export_gates", "csim_export_phases",
    "csim_export_mask", "csim_init", "csim_set_exec", "csim_run", "csim_sync",
    "csim_postselect", "csim_read_state", "csim_free", "csim_sv_create", "csim_sv_load",
    "csim_sv_compile", "csim_sv_run", "csim_sv_read", "csim_sv_info", "csim_sv_free",
    "csim_emulate_fused", "csim_last_error", "csim_norms_noalloc", "csim_state_device",
    "csim_sv_load_device", "csim_sv_device", "csim_sv_stats", "csim_pool_create",
    "csim_pool_submit", "csim_pool_poll", "csim_pool_result", "csim_pool_stats", "csim_pool_free",
    "csim_pool_plan", "csim_compile", "csim_run_steps", "csim_checkpoint", "csim_restore",
    "csim_final_distribution", "csim_pool_cancel", "csim_pool_inject", "csim_sv_apply_dense",
    "csim_sv_autotune", "csim_sv_compile_opts", "csim_tune_launch", "csim_set_launch_shape",
]


class CsimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"csim {_NAMES.get(status, status)}: {msg}")
        self.status = status


class Gate(C.Structure):
    _fields_ = [("op", C.c_uint8), ("target", C.c_uint8), ("tag", C.c_uint16),
                ("reserved", C.c_uint32), ("cmask", C.c_uint64), ("cval", C.c_uint64),
                ("angle", C.c_double)]


GATE_DTYPE = np.dtype([("op", "u1"), ("target", "u1"), ("tag", "<u2"), ("reserved", "<u4"),
                       ("cmask", "<u8"), ("cval", "<u8"), ("angle", "<f8")])
assert GATE_DTYPE.itemsize == C.sizeof(Gate) == 32


class BuildOpts(C.Structure):
    _fields_ = [("Nx", C.c_int32), ("tau", C.c_double), ("N_C", C.c_int32), ("K", C.c_int32),
                ("dt", C.c_double), ("Nt", C.c_int32), ("bc", C.c_int32),
                ("kappa_qsvt", C.c_double), ("d", C.c_int32), ("eps", C.c_double),
                ("max_qubits", C.c_int32), ("phases", C.POINTER(C.c_double)),
                ("n_phases", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("d", C.c_int32), ("n_a", C.c_int32),
                ("n_k", C.c_int32), ("n_m", C.c_int32), ("n_iL", C.c_int32),
                ("lambda_L", C.c_double), ("L_max", C.c_double), ("kappa_qsvt", C.c_double),
                ("poly_scale", C.c_double), ("n_gates_UL", C.c_int64),
                ("n_gates_total", C.c_int64), ("n_sweeps_run", C.c_int64),
                ("amp_updates_run", C.c_double), ("state_bytes", C.c_uint64),
                ("n_src_tables", C.c_int32), ("sparse_init", C.c_int32)]


_lib = None


def load():
    """Load the library (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    _build.build()
    lib = C.CDLL(LIB_PATH)
    P, VP, SZ, SZP = C.POINTER, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)
    D, DP = C.c_double, C.POINTER(C.c_double)
    sig = {
        "csim_build": ([C.c_int32, D, C.c_int32, C.c_int32, D, C.c_int32, P(VP)], C.c_int),
        "csim_build_ex": ([P(BuildOpts), P(VP)], C.c_int),
        "csim_info": ([VP, P(Info)], C.c_int),
        "csim_export_gates": ([VP, C.c_int32, VP, SZ, SZP], C.c_int),
        "csim_export_phases": ([VP, DP, SZ, SZP], C.c_int),
        "csim_export_mask": ([VP, P(C.c_uint64), P(C.c_uint64), SZ, SZP], C.c_int),
        "csim_init": ([VP, DP, C.c_int, VP], C.c_int),
        "csim_set_exec": ([VP, C.c_int], C.c_int),
        "csim_compile": ([VP], C.c_int),
        "csim_run_steps": ([VP, C.c_int64, P(C.c_int64)], C.c_int),
        "csim_final_distribution": ([VP, P(C.c_double), P(C.c_double), C.c_size_t,
                                     P(C.c_double)], C.c_int),
        "csim_checkpoint": ([VP, DP, SZ, P(C.c_int64)], C.c_int),
        "csim_restore": ([VP, DP, SZ, C.c_int, C.c_int64, VP], C.c_int),
        "csim_run": ([VP], C.c_int),
        "csim_sync": ([VP], C.c_int),
        "csim_postselect": ([VP, DP, SZ, SZP, DP, DP], C.c_int),
        "csim_read_state": ([VP, DP, SZ], C.c_int),
        "csim_free": ([VP], C.c_int),
        "csim_sv_create": ([C.c_int32, C.c_int, VP, P(VP)], C.c_int),
        "csim_sv_load": ([VP, DP, SZ], C.c_int),
        "csim_sv_compile": ([VP, VP, SZ, C.c_int], C.c_int),
        "csim_sv_run": ([VP, C.c_int32], C.c_int),
        "csim_sv_read": ([VP, DP, SZ], C.c_int),
        "csim_sv_info": ([VP, P(C.c_int64), DP, P(C.c_uint64)], C.c_int),
        "csim_sv_free": ([VP], C.c_int),
        "csim_emulate_fused": ([VP, SZ, C.c_int32, DP, P(C.c_int64)], C.c_int),
        "csim_last_error": ([], C.c_char_p),
        "csim_state_device": ([VP, P(VP), P(C.c_int32), P(C.c_int)], C.c_int),
        "csim_sv_load_device": ([VP, VP, SZ], C.c_int),
        "csim_sv_device": ([VP, P(VP)], C.c_int),
        "csim_sv_stats": ([VP, VP], C.c_int),
        "csim_pool_create": ([VP, P(VP)], C.c_int),
        "csim_pool_submit": ([VP, VP, DP, C.c_int, P(C.c_int64)], C.c_int),
        "csim_pool_poll": ([VP, C.c_int32, P(C.c_int64), SZ, SZP], C.c_int),
        "csim_pool_result": ([VP, C.c_int64, DP, DP, DP, SZ, SZP, DP], C.c_int),
        "csim_pool_stats": ([VP, VP], C.c_int),
        "csim_pool_free": ([VP], C.c_int),
        "csim_pool_cancel": ([VP, C.c_int64], C.c_int),
        "csim_sv_apply_dense": ([VP, P(C.c_int32), DP, C.c_int32], C.c_int),
        "csim_sv_autotune": ([VP, VP, SZ, C.c_int32, VP], C.c_int),
        "csim_sv_compile_opts": ([VP, VP, SZ, C.c_int, C.c_int32, C.c_int32], C.c_int),
        "csim_tune_launch": ([VP, C.c_int, C.c_int32, C.c_int32, VP], C.c_int),
        "csim_set_launch_shape": ([C.c_int, C.c_int32, C.c_int32, C.c_int32, C.c_int32], C.c_int),
        "csim_pool_inject": ([VP, C.c_int32, C.c_int64], C.c_int),
        "csim_pool_plan": ([C.c_uint64, C.c_uint64, C.c_int32, SZ, P(C.c_uint64), DP, DP, DP, DP,
                            P(C.c_uint64)], C.c_int),
        "csim_norms_noalloc": ([VP, C.c_int32, C.c_int, P(C.c_uint64), P(C.c_uint64), C.c_int32,
                                DP, VP], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(status):
    if status != CSIM_OK:
        raise CsimError(status, _lib.csim_last_error().decode(errors="replace"))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_handle(stream):
    """Accept None, an int handle, or a torch.cuda.Stream-like object."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


class Circuit:
    """Handle of ``csim_circuit`` (csim_build / csim_init / csim_run / csim_postselect)."""

    def __init__(self, Nx, tau, N_C, K, dt, Nt, kappa_qsvt=0.0, d=0, eps=0.0,
                 max_qubits=0, phases=None, bc="periodic"):
        lib = load()
        o = BuildOpts()
        o.Nx, o.tau, o.N_C, o.K, o.dt, o.Nt = int(Nx), float(tau), int(N_C), int(K), float(dt), int(Nt)
        if bc not in ("periodic", "bounceback"):
            raise ValueError("bc must be 'periodic' or 'bounceback'")
        o.bc = 0 if bc == "periodic" else 1
        o.kappa_qsvt, o.d, o.eps, o.max_qubits = float(kappa_qsvt), int(d), float(eps), int(max_qubits)
        self._phases_keep = None
        if phases is not None:
            ph = np.ascontiguousarray(phases, dtype=np.float64)
            self._phases_keep = ph
            o.phases = _dp(ph)
            o.n_phases = int(ph.shape[0])
        h = C.c_void_p()
        _check(lib.csim_build_ex(C.byref(o), C.byref(h)))
        self._h = h
        self._Nt = int(Nt)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.csim_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        inf = Info()
        _check(_lib.csim_info(self._h, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in Info._fields_}

    def export_gates(self, which: int = 0) -> np.ndarray:
        n = C.c_size_t()
        _check(_lib.csim_export_gates(self._h, which, None, 0, C.byref(n)))
        out = np.zeros(n.value, dtype=GATE_DTYPE)
        _check(_lib.csim_export_gates(self._h, which, out.ctypes.data_as(C.c_void_p), n.value,
                                      C.byref(n)))
        return out

    def export_phases(self) -> np.ndarray:
        n = C.c_size_t()
        _check(_lib.csim_export_phases(self._h, None, 0, C.byref(n)))
        out = np.zeros(n.value)
        _check(_lib.csim_export_phases(self._h, _dp(out), n.value, C.byref(n)))
        return out

    def export_mask(self):
        n = C.c_size_t()
        _check(_lib.csim_export_mask(self._h, None, None, 0, C.byref(n)))
        m = np.zeros(n.value, dtype=np.uint64)
        v = np.zeros(n.value, dtype=np.uint64)
        P = C.POINTER(C.c_uint64)
        _check(_lib.csim_export_mask(self._h, m.ctypes.data_as(P), v.ctypes.data_as(P), n.value,
                                     C.byref(n)))
        return m, v

    def init(self, f0, precision=CSIM_C128, stream=None):
        f = np.ascontiguousarray(f0, dtype=np.float64)
        _check(_lib.csim_init(self._h, _dp(f), int(precision), _stream_handle(stream)))

    def compile(self):
        """Fuse the circuit's program on the host now (releases the GIL)."""
        _check(_lib.csim_compile(self._h))

    def set_exec(self, mode):
        _check(_lib.csim_set_exec(self._h, int(mode)))

    def tune_launch(self, precision, max_steps=32, reps=2):
        """csim_tune_launch: time the first max_steps program steps on a scratch
        state under each candidate launch shape and keep the fastest for this
        (precision, qubit count) class; returns the choice and the trials."""
        r = LaunchTuneResult()
        _check(_lib.csim_tune_launch(self._h, int(precision), int(max_steps), int(reps),
                                     C.cast(C.byref(r), C.c_void_p)))
        trials = [{"u": r.trial_u[i], "minb": r.trial_minb[i], "waves": r.trial_waves[i],
                   "ms": r.trial_ms[i]} for i in range(r.n_trials)]
        return {"u": r.u, "minb": r.minb, "waves": r.waves, "ms": r.ms,
                "ms_default": r.ms_default, "steps": r.steps, "trials": trials}

    def run(self):
        _check(_lib.csim_run(self._h))

    def sync(self):
        _check(_lib.csim_sync(self._h))

    def postselect(self, want_amplitudes=True, out=None):
        """Return (amplitudes or None, p_success, norm_total).

        out (optional): a caller-owned float64 array of at least
        2 * postselect_count() values (for example a view of pinned memory),
        which receives the block; otherwise a new array is allocated."""
        n = C.c_size_t()
        p = C.c_double()
        t = C.c_double()
        if not want_amplitudes:
            _check(_lib.csim_postselect(self._h, None, 0, C.byref(n), C.byref(p), C.byref(t)))
            return None, p.value, t.value
        count = self.postselect_count()
        if out is None:
            out = np.zeros(2 * count)
        elif out.dtype != np.float64 or not out.flags.c_contiguous or out.size < 2 * count:
            raise ValueError("out must be a contiguous float64 array of 2 * postselect_count() values")
        _check(_lib.csim_postselect(self._h, _dp(out), count, C.byref(n), C.byref(p), C.byref(t)))
        return out[:2 * count].view(np.complex128), p.value, t.value

    def device_state(self):
        """Borrowed view of the current device state (see DeviceState)."""
        p = C.c_void_p()
        n = C.c_int32()
        pr = C.c_int()
        _check(_lib.csim_state_device(self._h, C.byref(p), C.byref(n), C.byref(pr)))
        return DeviceState(p.value, n.value, pr.value, self)

    def final_distribution(self, f0, amps) -> np.ndarray:
        """f(T) as an (Nx, 3) array from the compacted block of postselect()
        (complex amplitudes) and the f0 given to init (csim_final_distribution)."""
        f = np.ascontiguousarray(np.asarray(f0, dtype=np.float64).reshape(-1))
        a = np.ascontiguousarray(np.asarray(amps, dtype=np.complex128)).view(np.float64)
        out = np.zeros(f.shape[0], dtype=np.float64)
        _check(_lib.csim_final_distribution(self._h, _dp(f), _dp(a), a.shape[0] // 2, _dp(out)))
        return out.reshape(-1, 3)

    def postselect_count(self) -> int:
        """Number of amplitudes in the compacted postselected block."""
        inf = self.info()
        free_bits = (self._m_shift() - (2 + inf["n_iL"]))
        return ((1 << inf["n_m"]) - self._Nt) << free_bits

    def _m_shift(self):
        inf = self.info()
        return inf["n_qubits"] - inf["n_m"]

    def run_steps(self, n_steps):
        """Enqueue the next n_steps program steps; returns the next step index."""
        nxt = C.c_int64()
        _check(_lib.csim_run_steps(self._h, int(n_steps), C.byref(nxt)))
        return nxt.value

    def checkpoint(self):
        """(state as complex128 array, next step index)."""
        N = 1 << self.info()["n_qubits"]
        out = np.zeros(2 * N)
        nxt = C.c_int64()
        _check(_lib.csim_checkpoint(self._h, _dp(out), N, C.byref(nxt)))
        return out.view(np.complex128), nxt.value

    def restore(self, amps, next_step, precision=CSIM_C128, stream=None):
        a = np.ascontiguousarray(amps, dtype=np.complex128)
        _check(_lib.csim_restore(self._h, _dp(a.view(np.float64)), a.shape[0], int(precision),
                                 int(next_step), _stream_handle(stream)))

    def read_state(self) -> np.ndarray:
        N = 1 << self.info()["n_qubits"]
        out = np.zeros(2 * N)
        _check(_lib.csim_read_state(self._h, _dp(out), N))
        return out.view(np.complex128)


class SvStats(C.Structure):
    _fields_ = [("passes", C.c_int64), ("sweeps", C.c_int64), ("single", C.c_int64),
                ("amp_updates", C.c_double), ("pass_amps", C.c_double), ("state_bytes", C.c_uint64),
                ("dense_blocks", C.c_int64), ("staged_sweeps", C.c_int64)]


class LaunchTuneResult(C.Structure):
    _fields_ = [("u", C.c_int32), ("minb", C.c_int32), ("waves", C.c_int32), ("ms", C.c_double),
                ("ms_default", C.c_double), ("steps", C.c_int32), ("n_trials", C.c_int32),
                ("trial_u", C.c_int32 * 32), ("trial_minb", C.c_int32 * 32),
                ("trial_waves", C.c_int32 * 32), ("trial_ms", C.c_double * 32)]


def set_launch_shape(precision, n_qubits, u=0, minb=0, waves=0):
    """csim_set_launch_shape: fix (u, minb, waves) for a class; u = 0 clears."""
    _check(_lib.csim_set_launch_shape(int(precision), int(n_qubits), int(u), int(minb), int(waves)))


class TuneResult(C.Structure):
    _fields_ = [("stage", C.c_int32), ("dense", C.c_int32), ("ms", C.c_double),
                ("n_trials", C.c_int32), ("trial_stage", C.c_int32 * 8),
                ("trial_dense", C.c_int32 * 8), ("trial_ms", C.c_double * 8)]


class DeviceState:
    """A borrowed device state exposed through ``__cuda_array_interface__`` as
    a (2^n, 2) array of float32 (complex64 state) or float64 (complex128 state)
    (re, im) pairs, so ``torch.as_tensor(ds, device="cuda")`` views it without
    a copy.  Valid until the owner's next init/run/load/free."""

    def __init__(self, ptr, n, precision, owner):
        self.ptr, self.n, self.precision, self._owner = int(ptr), int(n), int(precision), owner

    @property
    def __cuda_array_interface__(self):
        return {"shape": (1 << self.n, 2), "typestr": "<f4" if self.precision == CSIM_C64 else "<f8",
                "data": (self.ptr, False), "version": 3, "strides": None}


class StateVector:
    """Handle of ``csim_sv``: a raw 2^n state plus a compiled gate program."""

    def __init__(self, n, precision=CSIM_C64, stream=None):
        lib = load()
        h = C.c_void_p()
        _check(lib.csim_sv_create(int(n), int(precision), _stream_handle(stream), C.byref(h)))
        self._h = h
        self.n = int(n)
        self.precision = int(precision)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.csim_sv_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, amps):
        a = np.ascontiguousarray(amps, dtype=np.complex128)
        _check(_lib.csim_sv_load(self._h, _dp(a.view(np.float64)), a.shape[0]))

    def load_device(self, ptr):
        """Copy 2^n amplitudes in this state's precision from device memory at ptr."""
        _check(_lib.csim_sv_load_device(self._h, C.c_void_p(int(ptr)), 1 << self.n))

    def device_state(self):
        p = C.c_void_p()
        _check(_lib.csim_sv_device(self._h, C.byref(p)))
        return DeviceState(p.value, self.n, self.precision, self)

    def compile(self, gates, mode=CSIM_EXEC_FUSED, stage=None, dense=None):
        """csim_sv_compile, or csim_sv_compile_opts when stage (0-3) or dense
        (0 off, 1 runs mixing across the warp tile, 2 every long run) is given."""
        g = gates_to_records(gates)
        if stage is None and dense is None:
            _check(_lib.csim_sv_compile(self._h, g.ctypes.data_as(C.c_void_p), g.shape[0],
                                        int(mode)))
        else:
            _check(_lib.csim_sv_compile_opts(self._h, g.ctypes.data_as(C.c_void_p), g.shape[0],
                                             int(mode), -1 if stage is None else int(stage),
                                             -1 if dense is None else int(dense)))

    def run(self, reps=1):
        _check(_lib.csim_sv_run(self._h, int(reps)))

    def read(self) -> np.ndarray:
        N = 1 << self.n
        out = np.zeros(2 * N)
        _check(_lib.csim_sv_read(self._h, _dp(out), N))
        return out.view(np.complex128)

    def info(self):
        ns = C.c_int64()
        au = C.c_double()
        sb = C.c_uint64()
        _check(_lib.csim_sv_info(self._h, C.byref(ns), C.byref(au), C.byref(sb)))
        return {"n_sweeps": ns.value, "amp_updates": au.value, "state_bytes": sb.value}

    def autotune(self, gates, reps=1):
        """csim_sv_autotune: time every staging width (and dense blocks where
        they apply), keep the fastest compiled; returns the choice and trials."""
        g = gates if isinstance(gates, np.ndarray) else gates_to_records(gates)
        g = np.ascontiguousarray(g)
        r = TuneResult()
        _check(_lib.csim_sv_autotune(self._h, g.ctypes.data_as(C.c_void_p), g.shape[0], int(reps),
                                     C.cast(C.byref(r), C.c_void_p)))
        trials = [{"stage": r.trial_stage[i], "dense": r.trial_dense[i], "ms": r.trial_ms[i]}
                  for i in range(r.n_trials)]
        return {"stage": r.stage, "dense": r.dense, "ms": r.ms, "trials": trials}

    def apply_dense(self, qubits, u, engine=0):
        """csim_sv_apply_dense: the 32 x 32 matrix u (element bit j = qubits[j])
        on five qubits; engine 0 tensor cores (split BF16x3), 1 CUDA cores FP32."""
        q = np.ascontiguousarray(qubits, dtype=np.int32)
        if q.shape != (5,):
            raise ValueError("five qubits")
        m = np.ascontiguousarray(u, dtype=np.complex128)
        if m.shape != (32, 32):
            raise ValueError("u must be 32 x 32")
        _check(_lib.csim_sv_apply_dense(self._h, q.ctypes.data_as(C.POINTER(C.c_int32)),
                                        _dp(m.view(np.float64)), int(engine)))

    def stats(self):
        st = SvStats()
        _check(_lib.csim_sv_stats(self._h, C.cast(C.byref(st), C.c_void_p)))
        return {k: getattr(st, k) for k, _ in SvStats._fields_}


FUSE_STAT_NAMES = ["sweeps", "single", "perm_gates", "segments", "local_gates", "mux",
                   "mux_gates", "mux_entries", "max_bucket", "lut_entries", "max_support", "passes",
                   "reflect", "mux_inverse", "wht", "conjugated", "staged_sweeps", "staged_gates",
                   "dense_blocks", "dense_gates"]


def emulate_fused(gates, n, amps):
    """Host executor of the fused program (testing aid); returns (state, stats dict).

    amps=None compiles only and returns (None, stats)."""
    lib = load()
    g = gates_to_records(gates)
    st = np.zeros(len(FUSE_STAT_NAMES), dtype=np.int64)
    a = None if amps is None else np.ascontiguousarray(amps, dtype=np.complex128).copy()
    _check(lib.csim_emulate_fused(g.ctypes.data_as(C.c_void_p), g.shape[0], int(n),
                                  None if a is None else _dp(a.view(np.float64)),
                                  st.ctypes.data_as(C.POINTER(C.c_int64))))
    return a, dict(zip(FUSE_STAT_NAMES, (int(x) for x in st)))


def gates_to_records(gates) -> np.ndarray:
    """Gate tuples (op, target, cmask, cval, angle, tag) or a record array -> records."""
    if isinstance(gates, np.ndarray) and gates.dtype == GATE_DTYPE:
        return np.ascontiguousarray(gates)
    out = np.zeros(len(gates), dtype=GATE_DTYPE)
    for i, g in enumerate(gates):
        out[i] = (g[0], g[1], g[5] if len(g) > 5 else 0, 0, g[2], g[3], g[4])
    return out


def norms_noalloc(state_ptr, n, prec, pm, pv, out_ptr, stream=None):
    """csim_norms_noalloc: FP64 (total, masked) norms of a caller-owned device
    state into the caller's 2-double device buffer `out_ptr`, with no device
    allocation by the library (for callers that cannot allocate)."""
    lib = load()
    m = np.ascontiguousarray(pm, dtype=np.uint64)
    v = np.ascontiguousarray(pv, dtype=np.uint64)
    if m.shape != v.shape:
        raise ValueError("pm and pv differ in length")
    _check(lib.csim_norms_noalloc(C.c_void_p(int(state_ptr)), int(n), int(prec),
                                  m.ctypes.data_as(C.POINTER(C.c_uint64)),
                                  v.ctypes.data_as(C.POINTER(C.c_uint64)), int(m.shape[0]),
                                  C.cast(C.c_void_p(int(out_ptr)), C.POINTER(C.c_double)),
                                  _stream_handle(stream)))


class PoolOpts(C.Structure):
    _fields_ = [("n_streams", C.c_int32), ("max_qubits", C.c_int32), ("hbm_budget", C.c_uint64),
                ("use_graphs", C.c_int32), ("min_block", C.c_uint32), ("persistent", C.c_int32)]


class PoolStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("rejected", C.c_int64), ("queued", C.c_int64), ("running", C.c_int64),
                ("bytes_in_use", C.c_uint64), ("peak_bytes", C.c_uint64), ("budget", C.c_uint64),
                ("graph_launches", C.c_int64), ("src_tables", C.c_int64),
                ("sparse_saved_bytes", C.c_uint64), ("failed", C.c_int64),
                ("cancelled", C.c_int64), ("batch_launches", C.c_int64),
                ("batch_dropped_signals", C.c_int64), ("batch_requests", C.c_int64)]


class Pool:
    """Handle of ``csim_pool``: admission under an HBM budget, concurrent streams,
    optional CUDA-graph admission waves (batching and serving)."""

    def __init__(self, n_streams=4, hbm_budget=0, max_qubits=32, use_graphs=False, min_block=0,
                 persistent=False):
        lib = load()
        o = PoolOpts()
        o.n_streams, o.hbm_budget, o.max_qubits = int(n_streams), int(hbm_budget), int(max_qubits)
        o.use_graphs, o.min_block = int(bool(use_graphs)), int(min_block)
        o.persistent = int(bool(persistent))
        h = C.c_void_p()
        _check(lib.csim_pool_create(C.cast(C.byref(o), C.c_void_p), C.byref(h)))
        self._h = h
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.csim_pool_free(self._h)
            self._h = None
            self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, circuit, f0, precision=CSIM_C64):
        """Queue one run; returns the request id (raises CsimError when rejected)."""
        f = np.ascontiguousarray(f0, dtype=np.float64)
        rid = C.c_int64()
        _check(_lib.csim_pool_submit(self._h, circuit._h, _dp(f), int(precision), C.byref(rid)))
        self._keep[rid.value] = circuit
        return rid.value

    def poll(self, wait_ms=0, cap=4096):
        ids = np.zeros(cap, dtype=np.int64)
        n = C.c_size_t()
        _check(_lib.csim_pool_poll(self._h, int(wait_ms), ids.ctypes.data_as(C.POINTER(C.c_int64)),
                                   cap, C.byref(n)))
        return [int(x) for x in ids[:n.value]]

    def result(self, rid, want_amplitudes=True):
        """(amplitudes or None, p_success, norm_total, times) of a finished request."""
        p = C.c_double()
        t = C.c_double()
        n = C.c_size_t()
        times = np.zeros(5)
        out = None
        if want_amplitudes:
            # the count is known from the circuit's geometry: ask with cap 0 first is not
            # possible after release, so size from the circuit's mask geometry
            cnt = self._keep[rid].postselect_count()
            out = np.zeros(2 * cnt)
            _check(_lib.csim_pool_result(self._h, int(rid), C.byref(p), C.byref(t), _dp(out), cnt,
                                         C.byref(n), _dp(times)))
            out = out.view(np.complex128)
        else:
            _check(_lib.csim_pool_result(self._h, int(rid), C.byref(p), C.byref(t), None, 0,
                                         C.byref(n), _dp(times)))
        self._keep.pop(rid, None)
        return out, p.value, t.value, {"queue_s": times[0], "latency_s": times[1],
                                       "device_s": times[2], "device_start_s": times[3],
                                       "device_end_s": times[4]}

    def cancel(self, rid):
        """csim_pool_cancel: drop a queued, running or finished request."""
        _check(_lib.csim_pool_cancel(self._h, int(rid)))
        self._keep.pop(rid, None)

    def inject(self, what, rid):
        """csim_pool_inject: host-side allocation failure of request rid at its
        admission (CSIM_INJECT_PINNED or CSIM_INJECT_ARENA; NONE clears)."""
        _check(_lib.csim_pool_inject(self._h, int(what), int(rid)))

    def stats(self):
        st = PoolStats()
        _check(_lib.csim_pool_stats(self._h, C.cast(C.byref(st), C.c_void_p)))
        return {k: getattr(st, k) for k, _ in PoolStats._fields_}


def pool_plan(budget, n_streams, alloc_bytes, duration, arrival=None, min_block=0):
    """csim_pool_plan: (start, finish, peak_bytes) of the admission policy."""
    lib = load()
    a = np.ascontiguousarray(alloc_bytes, dtype=np.uint64).reshape(-1, 4)
    d = np.ascontiguousarray(duration, dtype=np.float64)
    count = a.shape[0]
    arr = None if arrival is None else np.ascontiguousarray(arrival, dtype=np.float64)
    start = np.zeros(count)
    finish = np.zeros(count)
    peak = C.c_uint64()
    _check(lib.csim_pool_plan(int(budget), int(min_block), int(n_streams), count,
                              a.ctypes.data_as(C.POINTER(C.c_uint64)),
                              None if arr is None else _dp(arr), _dp(d), _dp(start), _dp(finish),
                              C.byref(peak)))
    return start, finish, int(peak.value)
