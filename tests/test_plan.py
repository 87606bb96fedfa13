"""Host logic: the work-balanced row partition of the block mat-vec
(paper Sec. 4.1 work split), compiled from the library's own planner source."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1201_6062_gb300", "csrc")


@pytest.fixture(scope="module")
def planlib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("plan") / "libplan.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-I", CSRC, "-o", out,
                           os.path.join(CSRC, "plan.cpp"), os.path.join(ROOT, "tests", "helpers", "plan_capi.cpp")])
    lib = ctypes.CDLL(out)
    lib.plan_run.restype = ctypes.c_int
    return lib


def run(lib, G, lmax, n, ovh=32, seg_rows=0):
    lmax = np.asarray(lmax, np.int32)
    n = np.asarray(n, np.int32)
    maxs = int(lmax.sum()) + 4 * G + 16
    segs = np.zeros((maxs, 5), np.int32)
    off = np.zeros(G + 1, np.int32)
    sb = np.zeros(int((lmax + 1).sum()), np.int32)
    P = ctypes.POINTER(ctypes.c_int)
    k = lib.plan_run(G, len(lmax), lmax.ctypes.data_as(P), n.ctypes.data_as(P), ovh, seg_rows, segs.ctypes.data_as(P), maxs,
                     off.ctypes.data_as(P), sb.ctypes.data_as(P))
    assert k >= 0
    return segs[:k], off, sb


CASES = [
    (152, [31], [2000]), (304, [31], [2000]), (152, [3], [50]), (152, [1], [1]), (7, [2], [3]),
    (152, [0], [10]), (152, [15], [1000]), (5, [4, 0, 2], [7, 3, 9]),
    (304, [20, 5, 32, 4], [1500, 200, 800, 1333]),
]


@pytest.mark.parametrize("seg_rows", [0, 8])
@pytest.mark.parametrize("G,lmax,n", CASES)
def test_plan_covers_every_row_once_and_balances(planlib, G, lmax, n, seg_rows):
    segs, off, sb = run(planlib, G, lmax, n, seg_rows=seg_rows)
    assert off[0] == 0 and off[-1] == len(segs) and np.all(np.diff(off) >= 0)
    # every row of every stored block exactly once, in order
    cover = {}
    for s, l, i0, i1, slot in segs:
        assert 0 <= s < len(lmax) and 0 <= l < lmax[s] and 0 <= i0 < i1 <= n[s]
        cover.setdefault((s, l), []).append((i0, i1, slot))
    for s in range(len(lmax)):
        for l in range(lmax[s]):
            iv = cover[(s, l)]
            assert iv[0][0] == 0 and iv[-1][1] == n[s]
            assert all(iv[k][1] == iv[k + 1][0] for k in range(len(iv) - 1))
    # slots: per system consecutive, block l owns sb[l]..sb[l+1]-1
    q = 0
    for s in range(len(lmax)):
        sbs = sb[q:q + lmax[s] + 1]
        q += lmax[s] + 1
        slots = [seg[4] for seg in segs if seg[0] == s]
        assert slots == list(range(len(slots)))
        for l in range(lmax[s]):
            mine = [seg[4] for seg in segs if seg[0] == s and seg[1] == l]
            assert mine == list(range(sbs[l], sbs[l + 1]))
    # balance: each CTA's cost (rows, plus seg_rows rows for each block it
    # starts) is within one row, with its block-start share, of the mean
    cost = np.zeros(G)
    for b in range(G):
        for s, l, i0, i1, _ in segs[off[b]:off[b + 1]]:
            cost[b] += (i1 - i0 + (seg_rows if i0 == 0 else 0)) * (n[s] + 32)
    total = sum(lmax[s] * (n[s] + seg_rows) * (n[s] + 32) for s in range(len(lmax)))
    assert abs(cost.sum() - total) < 1e-9
    if total > 0:
        wmax = max(n[s] + 32 for s in range(len(lmax)) if lmax[s] > 0)
        assert cost.max() <= total / G + (1 + seg_rows) * wmax + 1e-9


def test_plan_is_sorted_by_cta(planlib):
    segs, off, _ = run(planlib, 152, [31], [2000])
    rows = [(s, l, i0) for s, l, i0, _, _ in segs]
    assert rows == sorted(rows)


def test_block_start_cost_moves_rows_off_the_ctas_that_cross_a_block(planlib):
    # lmax=15, n=500 over 152 CTAs: about 49 rows each; 14 CTAs straddle a
    # block boundary.  With 8 rows charged per block start they take about
    # 8 rows fewer than the others; without, the same count within one row.
    for seg_rows, gap in ((0, 0), (8, 8)):
        segs, off, _ = run(planlib, 152, [15], [500], seg_rows=seg_rows)
        rows = np.array([sum(i1 - i0 for _, _, i0, i1, _ in segs[off[b]:off[b + 1]]) for b in range(152)])
        two = np.array([off[b + 1] - off[b] == 2 for b in range(152)])
        assert two.sum() >= 10
        d = rows[~two].mean() - rows[two].mean()
        assert abs(d - gap) <= 1.5, (seg_rows, d)
