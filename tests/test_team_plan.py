"""Host logic of the batched solver: the team plan (nlsp_plan_teams runs on
the host, no GPU needed).  Checked against its definition: team sizes by the
documented formula, windows inside the CTA range, no CTA holding two teams at
once under the documented duration model, and an execution of the per-CTA
task lists in (start, instance) order that never waits forever, whatever the
real durations are."""
import heapq
import math
import os

import numpy as np
import pytest

from paper_2601_20174_gb300 import _lib as L

pytestmark = pytest.mark.skipif(not os.path.exists(L.LIB_PATH), reason="libnlsp.so not built")


def _plan(n, G, tpc):
    from paper_2601_20174_gb300 import api
    return api.plan_teams(list(n), G, tpc)


def _model(n, s):
    tiles = -(-n // 128)
    share = -(-tiles // s)
    return math.sqrt(n) * (share + (1.5 if s > 1 else 0.0))


def _batch(count, seed):
    rng = np.random.default_rng(seed)
    sides = rng.choice([64, 128, 192, 256, 384, 512], size=count)
    return [int(s) * int(s) for s in sides]


@pytest.mark.parametrize("G,tpc,count", [(152, 0, 256), (152, 4, 64), (152, 1000, 300), (7, 16, 40), (1, 3, 5)])
def test_plan_sizes_windows_and_no_overlap(G, tpc, count):
    n = _batch(count, seed=G + count)
    first, size, start = _plan(n, G, tpc)
    t = tpc or 16
    for i in range(count):
        tiles = -(-n[i] // 128)
        assert size[i] == max(1, min(G, tiles, -(-tiles // t)))
        assert 0 <= first[i] and first[i] + size[i] <= G
        assert start[i] >= 0.0
    # per CTA, the planned intervals [start, start + duration) are disjoint
    for c in range(G):
        iv = sorted((start[i], start[i] + _model(n[i], size[i])) for i in range(count)
                    if first[i] <= c < first[i] + size[i])
        for (a0, a1), (b0, b1) in zip(iv, iv[1:]):
            assert b0 >= a1 - 1e-9 * max(1.0, a1)
    # the makespan stays within twice the area bound plus the longest task
    area = sum(_model(n[i], size[i]) * size[i] for i in range(count)) / G
    longest = max(_model(n[i], size[i]) for i in range(count))
    makespan = max(start[i] + _model(n[i], size[i]) for i in range(count))
    assert makespan <= 2.0 * area + longest


def _simulate(n, first, size, start, G, rng):
    """Runs every CTA's task list in (start, instance) order with random true
    durations; a team starts when all its CTAs have reached it.  Returns the
    number of finished instances (all of them unless the order deadlocks)."""
    count = len(n)
    lists = [sorted((start[i], i) for i in range(count) if first[i] <= c < first[i] + size[i]) for c in range(G)]
    pos = [0] * G
    arrived = [0] * count
    free_t = [0.0] * G
    done = 0
    events = []  # (finish time, instance)
    def arrive(c, now):
        if pos[c] < len(lists[c]):
            i = lists[c][pos[c]][1]
            arrived[i] += 1
            if arrived[i] == size[i]:
                heapq.heappush(events, (now + rng.uniform(0.1, 10.0), i))
    for c in range(G):
        arrive(c, 0.0)
    while events:
        t, i = heapq.heappop(events)
        done += 1
        for c in range(first[i], first[i] + size[i]):
            pos[c] += 1
            free_t[c] = t
            arrive(c, t)
    return done


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_task_order_never_deadlocks(seed):
    G = 19
    rng = np.random.default_rng(seed)
    n = [int(x) for x in rng.integers(1, 40 * 128, size=60)]
    first, size, start = _plan(n, G, 2)
    assert _simulate(n, first, size, start, G, rng) == len(n)


def test_plan_rejects_bad_arguments():
    from paper_2601_20174_gb300 import api
    with pytest.raises(L.NlspError):
        api.plan_teams([100, 0], 4)
    with pytest.raises(L.NlspError):
        api.plan_teams([100], 0)
    assert api.plan_teams([], 4) == ([], [], [])
