"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the simulated method.  It only draws
numbers (with ``numpy.random.default_rng``) and lays them out:

* the initial density profile of the Carleman-LBM workloads:
  rho(x) = 1 + A sin(2 pi x / Nx) + U(-0.01, 0.01), drawn for x = 0..Nx-1,
  at zero velocity.  The initial distribution is the zero-velocity
  equilibrium of Eq. feq, which reduces to f_q = w_q rho with the D1Q3
  weights (1/6, 1/6, 2/3) in the paper's velocity order (e=+1, -1, 0);
* the step profile of the paper's QSVT runs (left half 1 + drho/2, right
  half 1 - drho/2), at zero velocity;
* relaxation times drawn uniformly from a range;
* random QSP phase lists for parity tests;
* the random gate stream of the gate-vocabulary microbenchmark, emitted as
  canonical gate records (op, target, cmask, cval, angle, tag).
"""
from __future__ import annotations

import math

import numpy as np

D1Q3_WEIGHTS = (1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0)


def density_profile(Nx: int, rng: np.random.Generator, amplitude: float = 0.05,
                    noise: float = 0.01) -> np.ndarray:
    x = np.arange(Nx, dtype=np.float64)
    return 1.0 + amplitude * np.sin(2.0 * np.pi * x / Nx) + rng.uniform(-noise, noise, Nx)


def equilibrium_at_rest(rho: np.ndarray) -> np.ndarray:
    """f0[alpha][q] = w_q rho(alpha), shape (Nx, 3)."""
    return np.outer(rho, np.asarray(D1Q3_WEIGHTS))


def lbm_instance(Nx: int, seed: int, tau=None, tau_range=None, amplitude: float = 0.05):
    """One synthetic Carleman-LBM instance.

    If ``tau`` is None it is drawn first from U(tau_range); the density noise
    is drawn next.  Returns (f0 of shape (Nx, 3), tau).
    """
    rng = np.random.default_rng(seed)
    if tau is None:
        lo, hi = tau_range
        tau = float(rng.uniform(lo, hi))
    rho = density_profile(Nx, rng, amplitude)
    return equilibrium_at_rest(rho), float(tau)


def step_instance(Nx: int, drho: float) -> np.ndarray:
    """The step initial condition of the paper's QSVT runs (Sec. III.E): density
    1 + drho/2 on the left half of the sites and 1 - drho/2 on the right half
    (the symmetric range [1 - drho/2, 1 + drho/2]), at zero velocity.  Returns
    f0 of shape (Nx, 3)."""
    rho = np.where(np.arange(Nx) < Nx // 2, 1.0 + 0.5 * drho, 1.0 - 0.5 * drho)
    return equilibrium_at_rest(rho)


def random_phases(d: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(-math.pi, math.pi, d + 1)


def random_unit_state(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def microbench_gates(n: int, count: int, seed: int):
    """Gate stream of the vocabulary microbenchmark (canonical records, tag 0).

    40% single-qubit RY or RZ (50/50, angle U[0, 2pi), uniform target);
    30% CNOT (distinct random control and target); 20% multi-controlled X
    with U{2..8} distinct controls; 10% controlled +1 on a random 6-qubit
    register (LSB first) with one random control outside it, emitted as its
    MCX cascade.  RZ(theta) = diag(e^{-i theta/2}, e^{i theta/2}) is emitted as
    the ZPHASE record with angle -theta/2.
    """
    rng = np.random.default_rng(seed)
    out = []
    X, RY, ZP = 0, 2, 3
    for _ in range(count):
        u = rng.uniform()
        if u < 0.4:
            tgt = int(rng.integers(n))
            ang = float(rng.uniform(0.0, 2.0 * math.pi))
            if rng.uniform() < 0.5:
                out.append((RY, tgt, 0, 0, ang, 0))
            else:
                out.append((ZP, tgt, 0, 0, -ang / 2.0, 0))
        elif u < 0.7:
            c, t = (int(v) for v in rng.choice(n, 2, replace=False))
            out.append((X, t, 1 << c, 1 << c, 0.0, 0))
        elif u < 0.9:
            nc = int(rng.integers(2, 9))
            qs = [int(v) for v in rng.choice(n, nc + 1, replace=False)]
            t, cs = qs[0], qs[1:]
            m = sum(1 << c for c in cs)
            out.append((X, t, m, m, 0.0, 0))
        else:
            qs = [int(v) for v in rng.choice(n, 7, replace=False)]
            reg, c = qs[:6], qs[6]
            for j in range(5, -1, -1):
                m = (1 << c) | sum(1 << b for b in reg[:j])
                out.append((X, reg[j], m, m, 0.0, 0))
    return out


def dense_block_gates(n: int, blocks: int, seed: int):
    """Gate stream of dense 5-qubit blocks (canonical records, tag 0): each
    block picks 5 distinct random qubits and applies RY on each (angles
    U[0, 2pi)), a CNOT chain along them, RY on each again and H on two of
    them: 16 gates whose targets and controls stay inside the block."""
    rng = np.random.default_rng(seed)
    X, H, RY = 0, 1, 2
    out = []
    for _ in range(blocks):
        q = [int(v) for v in rng.choice(n, 5, replace=False)]
        for t in q:
            out.append((RY, t, 0, 0, float(rng.uniform(0.0, 2.0 * math.pi)), 0))
        for a, b in zip(q, q[1:]):
            out.append((X, b, 1 << a, 1 << a, 0.0, 0))
        for t in q:
            out.append((RY, t, 0, 0, float(rng.uniform(0.0, 2.0 * math.pi)), 0))
        for t in rng.choice(q, 2, replace=False):
            out.append((H, int(t), 0, 0, 0.0, 0))
    return out


def batch_instance(i: int):
    """Instance i of the 256-instance batching workload (seed i).

    Draw order: Nx from {8, 16, 32}, K from {2, 3, 4}, Nt from {4, 8},
    tau ~ U[0.55, 1.5], the QSVT degree d from the odd numbers 3..31, then the
    density noise of the initial condition.  N_C = 2, dt = 0.1.  Returns
    ((Nx, tau, 2, K, 0.1, Nt), d, f0).
    """
    rng = np.random.default_rng(i)
    Nx = int(rng.choice([8, 16, 32]))
    K = int(rng.choice([2, 3, 4]))
    Nt = int(rng.choice([4, 8]))
    tau = float(rng.uniform(0.55, 1.5))
    d = int(rng.choice(np.arange(3, 32, 2)))
    rho = density_profile(Nx, rng)
    return (Nx, tau, 2, K, 0.1, Nt), d, equilibrium_at_rest(rho)


def serving_requests(count: int, seed: int = 0):
    """The serving request stream (seed 0): for each request, in order, a
    unit-rate exponential inter-arrival gap (scaled by the caller's arrival
    rate), Nx from {16, 64, 256, 1024}, K from 2..6, Nt from 4..64, tau ~
    U[0.55, 1.5], d from the odd numbers 3..31, complex64 or complex128 with
    probability 1/2, and a per-request seed for the initial density.
    Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        gap = float(rng.exponential(1.0))
        Nx = int(rng.choice([16, 64, 256, 1024]))
        K = int(rng.integers(2, 7))
        Nt = int(rng.integers(4, 65))
        tau = float(rng.uniform(0.55, 1.5))
        d = int(rng.choice(np.arange(3, 32, 2)))
        prec = "c64" if rng.uniform() < 0.5 else "c128"
        out.append({"gap": gap, "Nx": Nx, "K": K, "Nt": Nt, "tau": tau, "d": d, "prec": prec,
                    "seed": 1000 + r})
    return out


def serving_f0(req: dict) -> np.ndarray:
    rng = np.random.default_rng(req["seed"])
    return equilibrium_at_rest(density_profile(req["Nx"], rng))
