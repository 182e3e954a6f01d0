"""csim_norms_noalloc (the reduction for callers that cannot allocate device
memory) against csim_postselect, through the C ABI, on two calls in a row.

The first call reduces a 20-qubit complex128 state, the second a smaller
complex64 state with a smaller grid, so a stale partial sum left in the shared
scratch array by the first call would show up in the second.  Tolerances:
complex128, both paths accumulate in FP64 and differ only in summation order,
1e-12 relative; complex64, csim_postselect adds eight FP32 products in FP32
before its FP64 accumulation (relative error below 8 * 2^-24 = 5e-7), 1e-6,
while this entry point forms every product in FP64, so against the host sum
of the same values it is held to 1e-12 as well.
"""
import numpy as np
import pytest

import lbm_inputs as I
import paper_2606_12770_gb300 as G
from paper_2606_12770_gb300 import _native as N

pytestmark = pytest.mark.gpu

TOL = 1e-12
TOL_C64 = 1e-6


def _close(a, b, tol=TOL):
    return abs(a - b) <= tol * max(abs(b), 1e-300)


def _run_circuit(cfg, d, prec, stream):
    f0, _ = I.lbm_instance(cfg[0], 3, tau=cfg[1])
    c = G.Circuit(*cfg, phases=I.random_phases(d, 7))
    c.init(f0, prec, stream)
    c.run()
    _, p, tot = c.postselect(want_amplitudes=False)
    return c, p, tot


def _masked_norm_host(psi, pm, pv):
    idx = np.arange(psi.shape[0], dtype=np.uint64)
    hit = np.zeros(psi.shape[0], dtype=bool)
    for m, v in zip(pm, pv):
        hit |= (idx & np.uint64(m)) == np.uint64(v)
    return float(np.sum(np.abs(psi[hit]) ** 2)), float(np.sum(np.abs(psi) ** 2))


def test_noalloc_norms_match_postselect_twice():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    stream = torch.cuda.current_stream()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")

    # call 1: C1 circuit (20 qubits), complex128
    c1, p1, t1 = _run_circuit((4, 0.8, 2, 2, 0.1, 2), 5, G.CSIM_C128, stream)
    n1 = c1.info()["n_qubits"]
    psi1 = c1.read_state()
    dev1 = torch.from_numpy(psi1.view(np.float64).copy()).cuda()
    pm1, pv1 = c1.export_mask()
    N.norms_noalloc(dev1.data_ptr(), n1, G.CSIM_C128, pm1, pv1, out.data_ptr(), stream)
    torch.cuda.synchronize()
    tot1, sel1 = out.cpu().tolist()
    assert _close(tot1, t1) and _close(sel1, p1), (tot1, t1, sel1, p1)
    hs, ht = _masked_norm_host(psi1, pm1, pv1)
    assert _close(sel1, hs) and _close(tot1, ht)

    # call 2: a smaller N_C = 1 circuit, complex64, same output buffer
    out.fill_(float("nan"))
    c2, p2, t2 = _run_circuit((8, 0.7, 1, 3, 0.2, 3), 3, G.CSIM_C64, stream)
    n2 = c2.info()["n_qubits"]
    assert n2 < n1
    psi2 = c2.read_state().astype(np.complex64)  # exact: the state is complex64 on the device
    dev2 = torch.from_numpy(psi2.view(np.float32).copy()).cuda()
    pm2, pv2 = c2.export_mask()
    N.norms_noalloc(dev2.data_ptr(), n2, G.CSIM_C64, pm2, pv2, out.data_ptr(), stream)
    torch.cuda.synchronize()
    tot2, sel2 = out.cpu().tolist()
    assert _close(tot2, t2, TOL_C64) and _close(sel2, p2), (tot2, t2, sel2, p2)
    # against the host sum of the same complex64 values, widened: both sides
    # form every product in FP64, so only the summation order differs
    hs2, ht2 = _masked_norm_host(psi2.astype(np.complex128), pm2, pv2)
    assert _close(tot2, ht2) and _close(sel2, hs2), (tot2, ht2, sel2, hs2)
    assert sel2 != sel1


@pytest.mark.parametrize("prec", [G.CSIM_C128, G.CSIM_C64])
def test_noalloc_edge_patterns(prec):
    """Edge paths of the candidate enumeration on an 8-qubit random state: no
    pattern (the masked sum is exactly 0), one pattern that fixes every index
    bit (a single candidate), and two full patterns that share only their low
    bits; each against the host sum."""
    torch = pytest.importorskip("torch")
    n = 8
    rng = np.random.default_rng(11)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    if prec == G.CSIM_C64:
        psi = psi.astype(np.complex64)
        dev = torch.from_numpy(psi.view(np.float32).copy()).cuda()
    else:
        dev = torch.from_numpy(psi.view(np.float64).copy()).cuda()
    wide = psi.astype(np.complex128)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    full = (1 << n) - 1
    cases = [([], []), ([full], [0x5A]), ([full, full], [0x13, 0xF3])]
    for pm, pv in cases:
        out.fill_(float("nan"))
        N.norms_noalloc(dev.data_ptr(), n, prec, np.array(pm, dtype=np.uint64),
                        np.array(pv, dtype=np.uint64), out.data_ptr(), stream)
        torch.cuda.synchronize()
        tot, sel = out.cpu().tolist()
        hs, ht = _masked_norm_host(wide, pm, pv)
        assert _close(tot, ht) and _close(sel, hs), (pm, pv, tot, ht, sel, hs)
        if not pm:
            assert sel == 0.0
        if len(pm) == 1:
            assert sel == pytest.approx(abs(wide[pv[0]]) ** 2, rel=1e-15)


def test_noalloc_rejects_misaligned_output():
    torch = pytest.importorskip("torch")
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(G.CsimError) as e:
        N.norms_noalloc(buf.data_ptr(), 4, G.CSIM_C128, [], [], buf.data_ptr() + 4)
    assert e.value.status == -1


def test_noalloc_rejects_sizes_beyond_its_limits():
    torch = pytest.importorskip("torch")
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(G.CsimError) as e:
        N.norms_noalloc(buf.data_ptr(), 35, G.CSIM_C128, [], [], buf.data_ptr())
    assert e.value.status == -2
    many = np.ones(17, dtype=np.uint64)
    with pytest.raises(G.CsimError) as e:
        N.norms_noalloc(buf.data_ptr(), 4, G.CSIM_C128, many, many, buf.data_ptr())
    assert e.value.status == -2
