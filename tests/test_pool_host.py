"""The request pool's admission policy on the simulated clock (csim_pool_plan,
host only): the buddy arena never exceeds its budget, at most n_streams run at
once, requests start in arrival order, requests that cannot fit are rejected,
and freed blocks coalesce so that a full-size request runs after the rest."""
import numpy as np
import pytest

from paper_2606_12770_gb300 import _native as N

MiB = 1 << 20


def _blocks(*sizes):
    row = list(sizes) + [0] * (4 - len(sizes))
    return row


def _pow2_blocks(row, min_block=MiB):
    tot = 0
    for b in row:
        if b:
            k = 0
            while (min_block << k) < b:
                k += 1
            tot += min_block << k
    return tot


def test_two_streams_equal_requests():
    a = [_blocks(MiB, MiB)] * 4
    s, f, peak = N.pool_plan(64 * MiB, 2, a, [1.0] * 4)
    assert list(s) == [0, 0, 1, 1] and list(f) == [1, 1, 2, 2]
    assert peak == 4 * MiB


def test_budget_limits_concurrency():
    a = [_blocks(MiB, MiB)] * 6
    s, f, peak = N.pool_plan(4 * MiB, 8, a, [1.0] * 6)
    assert list(s) == [0, 0, 1, 1, 2, 2]
    assert peak <= 4 * MiB


def test_head_of_line_is_not_overtaken():
    # request 1 needs the whole arena; request 2 is small but waits behind it
    a = [_blocks(2 * MiB), _blocks(4 * MiB), _blocks(MiB)]
    s, f, _ = N.pool_plan(4 * MiB, 4, a, [1.0, 1.0, 1.0])
    assert list(s) == [0, 1, 2]


def test_oversize_request_rejected():
    a = [_blocks(MiB), _blocks(8 * MiB), _blocks(MiB)]
    s, f, _ = N.pool_plan(4 * MiB, 4, a, [1.0, 1.0, 1.0])
    assert s[1] == -1 and f[1] == -1
    assert s[0] == 0 and s[2] == 0


def test_coalescing_after_fragmented_use():
    # many small blocks in a 16 MiB arena, then one request of the whole arena
    a = [_blocks(MiB)] * 12 + [_blocks(16 * MiB)]
    d = list(np.linspace(1.0, 3.0, 12)) + [1.0]
    s, f, peak = N.pool_plan(16 * MiB, 16, a, d)
    assert s[12] == pytest.approx(max(f[:12]))
    assert peak == 16 * MiB


def test_non_power_of_two_budget_and_rounding():
    # 24 MiB = 16 + 8 MiB regions; a 9 MiB block rounds up to 16 MiB
    a = [_blocks(9 * MiB), _blocks(8 * MiB), _blocks(8 * MiB)]
    s, f, peak = N.pool_plan(24 * MiB, 4, a, [2.0, 1.0, 1.0])
    assert list(s) == [0, 0, 1]
    assert peak == 24 * MiB


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_random_streams_invariants(seed):
    rng = np.random.default_rng(seed)
    n, streams, budget = 200, 4, 64 * MiB
    sizes = rng.choice([MiB, 2 * MiB, 4 * MiB, 8 * MiB, 16 * MiB], size=(n, 2))
    a = np.zeros((n, 4), dtype=np.uint64)
    a[:, 0] = sizes[:, 0]
    a[:, 1] = sizes[:, 0]
    a[:, 2] = sizes[:, 1] // 4
    a[:, 3] = MiB // 2
    arrival = np.cumsum(rng.exponential(0.3, n))
    dur = rng.uniform(0.1, 2.0, n)
    s, f, peak = N.pool_plan(budget, streams, a, dur, arrival=arrival)
    ok = s >= 0
    assert ok.all()
    assert np.all(s >= arrival - 1e-12)
    assert np.allclose(f - s, dur)
    # first come, first served: start times follow arrival order
    order = np.argsort(arrival, kind="stable")
    assert np.all(np.diff(s[order]) >= -1e-12)
    # at every start: running requests <= streams and rounded bytes <= budget
    need = np.array([_pow2_blocks(row) for row in a.astype(np.int64)])
    for t in s:
        live = (s <= t) & (f > t)
        assert live.sum() <= streams
        assert need[live].sum() <= budget
    assert peak <= budget
