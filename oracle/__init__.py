"""FP64 CPU oracle for the Carleman-linearised D1Q3 lattice-Boltzmann QSVT circuit.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the C-ABI library, its
Python binding, or the benchmark's GPU arm) may import, call, link or execute
anything in this package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle shares no code with the CUDA path.  It restates the paper
(Kanno et al., "Explicit Quantum Circuit Simulation of Nonlinear
1-Dimensional Fluid with Carleman-linearized Boltzmann Method") in plain,
slow, obviously-checkable FP64 Python:

* ``physics``   -- O1: D1Q3 BGK (Sec. II.A), Carleman blocks A11/A12/A22
                   (Eqs. A11-elements, A12-elements, A12-kernel,
                   carleman-second, carleman-system), the Taylor recurrence
                   (Eqs. taylor-recurrence, step-transition), the L matrix
                   (Fig. L, Berry et al. Def. 1) and kappa(L).
* ``layout``    -- the register layout and the embedding of the Carleman /
                   Taylor-slot index into the qubit register.
* ``circuit``   -- O3: an independent gate compiler for U_A, U_L (Sec. II.D)
                   and the QSVT wrapper (Fig. circuit-qsvt).
* ``statevec``  -- O2: naive gate-by-gate state-vector simulator and a dense
                   unitary brute force for <= 10 qubits.
* ``blockenc``  -- O4: block-encoding extraction by basis sweep (App. B).
* ``qsvt``      -- O5: QSP evaluation of a phase sequence, its Chebyshev
                   coefficients, and the singular-value Chebyshev recurrence
                   that applies the transformed matrix classically.

Functions whose result has no independent pin say "parity unpinned" in their
docstring.  Every other function is pinned by a ``-m "not gpu"`` test against
values the paper prints, closed forms, invariants or brute force.
"""
