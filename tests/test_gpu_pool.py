"""The request pool on the GPU: every request's results equal the same
circuit run alone through csim_init / csim_run / csim_postselect (bit for bit:
the kernels are deterministic, a request's work does not depend on what runs
beside it, and its source-index tables built in the arena hold the same
indices as the circuit's own), with and without CUDA-graph admission waves,
under a budget small enough to force several admission waves."""
import numpy as np
import pytest

import lbm_inputs as I
import paper_2606_12770_gb300 as G

pytestmark = pytest.mark.gpu

MIX = [  # (Nx, tau, N_C, K, dt, Nt), d, precision
    ((4, 0.8, 2, 2, 0.1, 2), 5, G.CSIM_C64),
    ((4, 0.8, 2, 2, 0.1, 2), 5, G.CSIM_C128),
    ((8, 0.7, 1, 3, 0.2, 3), 7, G.CSIM_C64),
    ((2, 1.1, 2, 3, 0.1, 2), 9, G.CSIM_C128),
    ((4, 0.6, 2, 1, 0.15, 3), 3, G.CSIM_C64),
    ((8, 0.9, 2, 2, 0.1, 2), 11, G.CSIM_C64),
    ((2, 0.55, 2, 4, 0.1, 5), 13, G.CSIM_C128),
    ((16, 1.2, 1, 2, 0.1, 8), 5, G.CSIM_C64),
]


def _instances():
    out = []
    for k, (cfg, d, prec) in enumerate(MIX):
        f0, _ = I.lbm_instance(cfg[0], 10 + k, tau=cfg[1])
        c = G.Circuit(*cfg, kappa_qsvt=10.0, d=d)
        out.append((c, f0, prec))
    return out


def _alone(inst):
    res = []
    for c, f0, prec in inst:
        c.init(f0, prec)
        c.run()
        res.append(c.postselect())
    return res


@pytest.mark.parametrize("graphs", [False, True])
def test_pool_mix_equals_alone(graphs):
    # separate handles: the pool's circuits have not run alone, so their
    # source-index tables come from the arena
    alone = _alone(_instances())
    inst = _instances()
    # budget: room for about two of the largest requests at once
    pool = G.Pool(n_streams=3, hbm_budget=160 << 20, max_qubits=30, use_graphs=graphs)
    ids = [pool.submit(c, f0, prec) for c, f0, prec in inst]
    done = set()
    for _ in range(20000):
        done.update(pool.poll(wait_ms=20))
        if len(done) == len(ids):
            break
    assert len(done) == len(ids)
    st = pool.stats()
    assert st["completed"] == len(ids) and st["rejected"] == 0
    assert 0 < st["peak_bytes"] <= st["budget"]
    assert (st["graph_launches"] > 0) == graphs
    # one chain per request: U_L^dag's (each U_L permutation undoes the one
    # before it, so those pairs run as in-place conjugated sweeps)
    assert st["src_tables"] == len(ids)
    for rid, (amps0, p0, t0) in zip(ids, alone):
        amps, p, t, times = pool.result(rid)
        assert np.array_equal(amps, amps0)
        assert p == p0 and t == t0
        assert times["latency_s"] >= times["queue_s"] >= 0.0
    pool.close()


def test_pool_rejects_above_the_qubit_cap():
    pool = G.Pool(n_streams=2, hbm_budget=64 << 20, max_qubits=18)
    c = G.Circuit(4, 0.8, 2, 2, 0.1, 2, kappa_qsvt=10.0, d=3)  # 20 qubits
    f0, _ = I.lbm_instance(4, 0, tau=0.8)
    with pytest.raises(G.CsimError) as e:
        pool.submit(c, f0, G.CSIM_C64)
    assert e.value.status == -2
    assert pool.stats()["rejected"] == 1
    pool.close()


def test_pool_rejects_requests_larger_than_the_budget():
    pool = G.Pool(n_streams=2, hbm_budget=8 << 20, max_qubits=30)
    c = G.Circuit(4, 0.8, 2, 2, 0.1, 2, kappa_qsvt=10.0, d=3)  # 2 x 16 MiB in complex128
    f0, _ = I.lbm_instance(4, 0, tau=0.8)
    with pytest.raises(G.CsimError) as e:
        pool.submit(c, f0, G.CSIM_C128)
    assert e.value.status == -2
    pool.close()


def _drain(pool, n, polls=20000):
    done = []
    for _ in range(polls):
        done += pool.poll(wait_ms=20)
        if len(done) >= n:
            break
    return done


def test_pool_requests_overlap_on_device():
    """Continuous batching runs requests side by side: in stream mode each
    request's device interval (its first and last event on its stream, on the
    pool's clock) is reported, and at least two admitted requests' intervals
    intersect.  The requests are 26-27-qubit runs of d = 21 (several ms of
    device work each), fused on the host before they are submitted, so that
    one still runs when the next is admitted."""
    specs = [((16, 0.7, 2, 4, 0.1, 8), 21), ((16, 0.9, 2, 3, 0.1, 8), 21),
             ((16, 1.1, 2, 4, 0.1, 4), 21), ((8, 0.6, 2, 4, 0.1, 16), 21)]
    inst = []
    for k, (cfg, d) in enumerate(specs):
        f0, _ = I.lbm_instance(cfg[0], 40 + k, tau=cfg[1])
        c = G.Circuit(*cfg, kappa_qsvt=10.0, d=d)
        c.compile()
        inst.append((c, f0))
    pool = G.Pool(n_streams=4, max_qubits=30)
    ids = [pool.submit(c, f0, G.CSIM_C64) for c, f0 in inst]
    assert len(_drain(pool, len(ids))) == len(ids)
    iv = []
    for rid in ids:
        _, _, _, times = pool.result(rid, want_amplitudes=False)
        assert 0.0 <= times["device_start_s"] < times["device_end_s"]
        iv.append((times["device_start_s"], times["device_end_s"]))
    overlaps = sum(1 for i in range(len(iv)) for j in range(i + 1, len(iv))
                   if iv[i][0] < iv[j][1] and iv[j][0] < iv[i][1])
    print("device intervals (s):", [(round(a, 4), round(b, 4)) for a, b in iv],
          "overlapping pairs:", overlaps)
    assert overlaps >= 1
    pool.close()


@pytest.mark.parametrize("graphs", [False, True])
def test_pool_failures_and_cancellation_leave_the_rest_intact(graphs):
    """Host-side failures and cancellation inside a busy pool: request 3's
    pinned staging and request 5's arena blocks are refused at admission
    (injected on the host; nothing faults on the device), request 7 is
    cancelled while queued and request 2 while it may be running.  The
    failed requests report CSIM_ERR_OOM and hold no memory, the cancelled ones
    are never reported, every other request equals its run alone bit for bit,
    and the arena is empty at the end."""
    alone = _alone(_instances())
    inst = _instances()
    pool = G.Pool(n_streams=2, hbm_budget=160 << 20, max_qubits=30, use_graphs=graphs)
    # ids are assigned in submission order from 1: inject before submitting
    pool.inject(G._native.CSIM_INJECT_PINNED, 3)
    pool.inject(G._native.CSIM_INJECT_ARENA, 5)
    ids = [pool.submit(c, f0, prec) for c, f0, prec in inst]
    assert ids == list(range(1, len(inst) + 1))
    pool.cancel(7)  # two slots: request 7 is still queued
    pool.cancel(2)
    with pytest.raises(G.CsimError):
        pool.cancel(7)
    expect = [i for i in ids if i not in (2, 7)]
    done = _drain(pool, len(expect))
    assert sorted(done) == expect
    st = pool.stats()
    assert st["failed"] == 2 and st["cancelled"] == 2
    for rid in expect:
        if rid in (3, 5):
            with pytest.raises(G.CsimError) as e:
                pool.result(rid)
            assert e.value.status == -3
            continue
        amps0, p0, t0 = alone[rid - 1]
        amps, p, t, _ = pool.result(rid)
        assert np.array_equal(amps, amps0) and p == p0 and t == t0
    pool.poll(wait_ms=100)
    assert pool.stats()["bytes_in_use"] == 0
    pool.close()


MIX64 = [(cfg, d, G.CSIM_C64) for cfg, d, _ in MIX]


def _instances64():
    out = []
    for k, (cfg, d, prec) in enumerate(MIX64):
        f0, _ = I.lbm_instance(cfg[0], 10 + k, tau=cfg[1])
        out.append((G.Circuit(*cfg, kappa_qsvt=10.0, d=d), f0, prec))
    return out


def test_persistent_pass_equals_alone():
    """Persistent mode: every admission pass runs the sweeps of all its
    requests in one launch whose CTAs take work items from a device queue and
    wait (with a time limit) for each request's previous sweep.  Each result
    equals the circuit run alone within complex64 rounding (the launch runs
    the sweep kernels' op bodies, with another number of tiles per warp):
    1e-5 relative on the block, 1e-6 on the norms."""
    alone = _alone(_instances64())
    inst = _instances64()
    pool = G.Pool(n_streams=4, hbm_budget=160 << 20, max_qubits=30, persistent=True)
    ids = [pool.submit(c, f0, prec) for c, f0, prec in inst]
    assert len(_drain(pool, len(ids))) == len(ids)
    st = pool.stats()
    assert st["batch_launches"] >= 2 and st["completed"] == len(ids) and st["failed"] == 0
    print(f"persistent pass: {st['batch_requests']} of {len(ids)} requests in "
          f"{st['batch_launches']} launches")
    assert st["batch_requests"] >= len(ids) // 2
    errs = []
    for rid, (amps0, p0, t0) in zip(ids, alone):
        amps, p, t, _ = pool.result(rid)
        err = float(np.linalg.norm(amps - amps0) / max(np.linalg.norm(amps0), 1e-300))
        errs.append(err)
        assert err < 1e-5, (rid, err)
        assert abs(t - t0) < 1e-6 and abs(p - p0) <= 1e-5 * max(p0, 1e-30) + 1e-12
    print(f"persistent pass vs alone: max rel L2 {max(errs):.3e}, "
          f"{sum(e == 0.0 for e in errs)} of {len(errs)} bit-identical")
    pool.close()


def test_persistent_wait_times_out_and_pool_recovers():
    """A work item that never signals (injected on the host: the first item of
    one request's second sweep keeps its completion count back) makes the
    items that depend on it wait out their 2 s limit; the launch stops, every
    request of that pass reports CSIM_ERR_TIMEOUT, and the next pass runs
    normally.  Nothing faults or hangs on the device."""
    inst = _instances64()[:2]
    pool = G.Pool(n_streams=2, max_qubits=30, persistent=True)
    pool.inject(G._native.CSIM_INJECT_BATCH_SIGNAL, 1)
    ids = [pool.submit(c, f0, prec) for c, f0, prec in inst]
    assert sorted(_drain(pool, 2)) == ids
    st = pool.stats()
    print("persistent timeout test stats:", st)
    assert st["batch_dropped_signals"] == 1
    # the injected request fails with the timeout (and so does any request
    # that shared its pass)
    with pytest.raises(G.CsimError) as e:
        pool.result(ids[0])
    assert e.value.status == -6
    try:
        pool.result(ids[1])
    except G.CsimError as e2:
        assert e2.status == -6
    assert pool.stats()["failed"] >= 1
    alone = _alone(_instances64()[:2])
    ids2 = [pool.submit(c, f0, prec) for c, f0, prec in _instances64()[:2]]
    assert sorted(_drain(pool, 2)) == ids2
    for rid, (amps0, p0, t0) in zip(ids2, alone):
        amps, p, t, _ = pool.result(rid)
        assert float(np.linalg.norm(amps - amps0) / max(np.linalg.norm(amps0), 1e-300)) < 1e-5
    pool.close()


def test_persistent_mixed_precisions():
    """A persistent pool given complex64 and complex128 requests together:
    the complex64 ones of a pass share one persistent launch, the complex128
    ones run on their own streams in the same pass; every result equals the
    circuit run alone (bit for bit in complex128, within complex64 rounding
    otherwise)."""
    inst = [(c, f0, G.CSIM_C128 if k % 2 else prec) for k, (c, f0, prec) in enumerate(_instances64())]
    alone = _alone(inst)
    inst = [(c, f0, G.CSIM_C128 if k % 2 else prec) for k, (c, f0, prec) in enumerate(_instances64())]
    pool = G.Pool(n_streams=8, max_qubits=30, persistent=True)
    ids = [pool.submit(c, f0, prec) for c, f0, prec in inst]
    assert sorted(_drain(pool, len(ids))) == ids
    st = pool.stats()
    assert st["batch_launches"] >= 1 and st["failed"] == 0
    for rid, (amps0, p0, t0), (_, _, prec) in zip(ids, alone, inst):
        amps, p, t, _ = pool.result(rid)
        if prec == G.CSIM_C128:
            assert np.array_equal(amps, amps0) and p == p0 and t == t0
        else:
            err = float(np.linalg.norm(amps - amps0) / max(np.linalg.norm(amps0), 1e-300))
            assert err < 1e-5, (rid, err)
    pool.close()
