"""O4 -- block-encoding extraction by sweeping computational-basis inputs (App. B).

Test infrastructure only.  For every basis input |x>|0>_anc of the system
register, the gate list is applied exactly (``statevec.SparseColumns``), the
|0>_anc projection of the output is read, and the result is multiplied by the
encoder normalisation lambda.  The extracted matrix is then compared, block by
block, with L assembled from the paper's equations (``physics.l_matrix``).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import circuit as C
from . import physics as P
from .layout import Layout
from .statevec import SparseColumns


def system_inputs(lay: Layout) -> np.ndarray:
    """Every basis index with t = s = iL = 0 (all system-register values)."""
    sysb = lay.system_bits()
    N = 1 << len(sysb)
    ar = np.arange(N, dtype=np.int64)
    idx = np.zeros(N, dtype=np.int64)
    for j, b in enumerate(sysb):
        idx |= ((ar >> j) & 1) << b
    return idx


def extract_UL(Nx, tau, NC, K, dt, Nt, bc="periodic"):
    """Return (M_scaled, inputs, lam): M_scaled[r, c] = lambda_L <inputs[r]|U_L|inputs[c]>."""
    lay = Layout(Nx, NC, K, Nt)
    gates = C.build_UL(Nx, tau, NC, K, dt, Nt, bc)
    inputs = system_inputs(lay)
    sim = SparseColumns(lay.n, inputs).run(gates)
    anc = 0
    for b in lay.regs["t"] + lay.regs["s"] + lay.regs["iL"]:
        anc |= 1 << b
    keep = (sim.key & anc) == 0
    pos = {int(v): i for i, v in enumerate(inputs)}
    rows = np.array([pos[int(k)] for k in sim.key[keep]], dtype=np.int64)
    cols = sim.col[keep]
    lam = float(1 << lay.niL) * C.lmax_value(tau, NC, dt, bc)
    N = inputs.shape[0]
    M = sp.csr_matrix((sim.amp[keep] * lam, (rows, cols)), shape=(N, N))
    return M, inputs, lam, lay


def compare_with_L(Nx, tau, NC, K, dt, Nt, bc="periodic"):
    """Max |M_phys - L| and max |cross terms|, with M extracted from the circuit."""
    M, inputs, lam, lay = extract_UL(Nx, tau, NC, K, dt, Nt, bc)
    A = P.carleman_A(Nx, tau, NC, bc)
    L = P.l_matrix(A, dt, K, Nt).toarray()
    phys = lay.physical_indices()
    pos = {int(v): i for i, v in enumerate(inputs)}
    pidx = np.array([pos[int(v)] for v in phys], dtype=np.int64)
    Md = M.toarray()
    Mp = Md[np.ix_(pidx, pidx)]
    err_phys = float(np.max(np.abs(Mp - L)))
    np_mask = np.ones(inputs.shape[0], dtype=bool)
    np_mask[pidx] = False
    cross = 0.0
    if np_mask.any():
        cross = max(float(np.max(np.abs(Md[np.ix_(np_mask, pidx)]))),
                    float(np.max(np.abs(Md[np.ix_(pidx, np_mask)]))))
    return err_phys, cross, lam
