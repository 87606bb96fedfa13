"""Host logic: the schedule of the persistent tensor-core batch launch.

The kernel (tc_kernel with PIPE) deals the output tiles of all stages
round-robin over its CTAs.  A tile of stage g loads the state planes of
blocks l-1 and l+1 (buffer g mod 2) once every row tile of those blocks
(same pulse columns) has finished stage g-1, updates its own state once
every row tile of block l has finished stage g-1, and writes the planes of
stage g+1 into buffer (g+1) mod 2.  Two buffers suffice: the tiles that read
block l's planes from that buffer (stage g-1, blocks l-1 and l+1) are the
very tiles a writer of block l has waited for.  This event simulation
replays the protocol with random durations and a producer that runs ahead
of the products, and checks that it never deadlocks, never loads planes
before they are written or overwrites planes still being read, and updates
every tile's state in stage order.  Dropping one of the waits makes the
checks fail, which shows they can."""
import heapq
import itertools

import numpy as np
import pytest


def simulate(lmax, mt, nt, G, nst, nbuf, seed, ahead=2, wait_right=True, wait_own=True):
    """Returns (finished, violations): violations lists overwrites of planes
    still being read and out-of-order state updates."""
    rng = np.random.default_rng(seed)
    ntiles = (lmax + 1) * mt * nt
    items = {b: [w for w in range(b, nst * ntiles, G)] for b in range(G)}

    def tile(w):
        g, t = divmod(w, ntiles)
        l, rem = divmod(t, mt * nt)
        return g, l, rem // nt, rem % nt          # stage, block, row tile, column tile

    done = {}                                   # (g, l, p) -> row tiles finished
    readers = {}                                # (buf, l, p) -> set of items reading it
    last_state = {}                             # (l, i, p) -> last stage updated
    violations = []
    # per CTA: index of the next item to load, and items loaded but not finished
    nxt = {b: 0 for b in range(G)}
    inflight = {b: [] for b in range(G)}
    clock = 0.0
    events = []                                 # (time, seq, kind, cta, item)
    seq = itertools.count()

    def ready_to_load(w):
        g, l, i, p = tile(w)
        if g == 0:
            return True
        need = (l - 1, l + 1) if wait_right else (l - 1,)
        return all(done.get((g - 1, lb, p), 0) == mt for lb in need if 0 <= lb <= lmax)

    def ready_to_update(w):
        g, l, i, p = tile(w)
        return g == 0 or not wait_own or done.get((g - 1, l, p), 0) == mt

    def try_load(b):
        # the producer issues the next item's loads once its inputs are ready,
        # at most `ahead` items beyond the one whose products and update run
        while nxt[b] < len(items[b]) and len(inflight[b]) < ahead and ready_to_load(items[b][nxt[b]]):
            w = items[b][nxt[b]]
            g, l, i, p = tile(w)
            for lb in (l - 1, l + 1):
                if 0 <= lb <= lmax:
                    if g > 0 and done.get((g - 1, lb, p), 0) != mt:
                        violations.append(("stale planes", g, lb, p))
                    readers.setdefault((g % nbuf, lb, p), set()).add(w)
            inflight[b].append(w)
            nxt[b] += 1
            if len(inflight[b]) == 1:
                heapq.heappush(events, (clock + rng.uniform(1, 3), next(seq), "mma", b, w))

    for b in range(G):
        try_load(b)
    finished = 0
    waiting = {}                                # cta -> item whose update waits for block counts
    while events:
        clock, _, kind, b, w = heapq.heappop(events)
        g, l, i, p = tile(w)
        if kind == "mma":
            # products done: the item's plane reads are over
            for lb in (l - 1, l + 1):
                if 0 <= lb <= lmax:
                    readers[(g % nbuf, lb, p)].discard(w)
            if ready_to_update(w):
                heapq.heappush(events, (clock + rng.uniform(0.5, 2), next(seq), "upd", b, w))
            else:
                waiting[b] = w
        else:
            # the update writes the tile's state and its planes of stage g + 1
            if last_state.get((l, i, p), -1) != g - 1:
                violations.append(("state order", g, l, i, p))
            last_state[(l, i, p)] = g
            if readers.get(((g + 1) % nbuf, l, p)):
                violations.append(("overwrite", g, l, p, sorted(readers[((g + 1) % nbuf, l, p)])))
            done[(g, l, p)] = done.get((g, l, p), 0) + 1
            finished += 1
            inflight[b].pop(0)
            if inflight[b]:
                heapq.heappush(events, (clock + rng.uniform(1, 3), next(seq), "mma", b, inflight[b][0]))
            # counts changed: retry every CTA's waiting update and loads
            for c in list(waiting):
                if ready_to_update(waiting[c]):
                    heapq.heappush(events, (clock + rng.uniform(0.5, 2), next(seq), "upd", c, waiting.pop(c)))
            for c in range(G):
                try_load(c)
    return finished == nst * (lmax + 1) * mt * nt, violations


@pytest.mark.parametrize("lmax,mt,nt,G", [(3, 2, 2, 5), (5, 3, 1, 7), (15, 8, 4, 152), (0, 2, 2, 3), (1, 1, 1, 1)])
def test_two_buffers_finish_without_stale_or_overwritten_planes(lmax, mt, nt, G):
    nst = 9
    for seed in range(6 if G < 100 else 2):
        finished, violations = simulate(lmax, mt, nt, G, nst, 2, seed)
        assert finished, (lmax, mt, nt, G, seed)
        assert not violations, violations[:3]


def test_dropping_a_wait_is_caught():
    kinds = set()
    for seed in range(20):
        _, v = simulate(5, 3, 1, 7, 9, 2, seed, wait_right=False)
        kinds |= {x[0] for x in v}
        _, v = simulate(5, 3, 1, 7, 9, 2, seed, wait_own=False)
        kinds |= {x[0] for x in v}
    assert "stale planes" in kinds and "state order" in kinds, kinds
