"""The query kernels' early-stopping walk, modelled on the CPU and checked
against the oracle's Alg. 3 (no GPU).

The kernels do not run Alg. 3 literally. They walk repetition-0 cells in
groups of count levels and skip cells whose level is below the admission
bound's score. They hold candidates in a buffer that is cut to the k best
whenever it fills (the bound becomes the k-th key), and they stop once the
k-th best candidate scores at least the last completed level. This model
takes those steps in the same order, with every order the kernels leave
open drawn at random:
- cell order within a level;
- member order within a group;
- the group size;
- how full the buffer gets before it is cut (tiny buffers force many
  mid-group cuts).

Its output must equal Alg. 3's on every input. That pins the stop rule and
the pruning as a design, on far more cases than the GPU parity tests reach.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_11565_gb300 import workloads as WL


def kernel_walk(cnt, gid, B, L, kq, t_min, gcells, cap_fill, rng):
    """The kernels' decode order, with their free choices drawn from rng.
    Keys are (-score, last cell, id): the kernels' 64-bit key in tuple form."""
    N, R = gid.shape
    if kq == 0:
        return [], []
    members = {b: rng.permutation(np.nonzero(gid[:, 0] == b)[0]).tolist() for b in range(B)}
    levels = {t: rng.permutation([b for b in range(B) if cnt[b] == t]).tolist() for t in range(t_min, L + 1)}

    def key_of(x):
        score, last = 1 << 30, 0
        for r in range(R):                       # repetition order, as in the kernels
            c = r * B + int(gid[x, r])
            if cnt[c] <= score:
                score, last = int(cnt[c]), c
        return (-score, last, int(x))

    buf, bound, bscore = [], None, 0
    have_k, kth = False, 0
    t = L
    while t >= t_min:
        nc, t_end = len(levels[t]), t
        while t_end > t_min and nc + len(levels[t_end - 1]) <= gcells:
            t_end -= 1
            nc += len(levels[t_end])
        cells = [b for lv in range(t, t_end - 1, -1) for b in levels[lv]]
        pos = 0
        while pos < len(cells):                  # chunks of the group's cells
            chunk = cells[pos:pos + int(rng.integers(1, len(cells) - pos + 1))]
            pos += len(chunk)
            # cells below the bound's score are skipped when the chunk is set up
            mem = [x for b in chunk if cnt[b] >= bscore for x in members[b]]
            for x in rng.permutation(mem).tolist() if mem else []:
                k = key_of(x)
                if -k[0] >= max(t_min, bscore) and (bound is None or k <= bound):
                    buf.append(k)
                if len(buf) > cap_fill:          # the buffer is cut to the k best
                    buf = sorted(buf)[:kq]
                    bound = buf[-1]
                    bscore = -bound[0]
        if nc > 0 and len(buf) >= kq:            # end of a group: cut and check
            buf = sorted(buf)[:kq]
            bound = buf[-1]
            kth = bscore = -bound[0]
            have_k = True
        if have_k and kth >= t_end:              # every point of score >= t_end is seen
            break
        t = t_end - 1
    out = sorted(buf)[:kq]
    return [x for _, _, x in out], [-s for s, _, _ in out]


@pytest.mark.parametrize("seed", range(300))
def test_kernel_walk_equals_alg3(seed):
    rng = np.random.default_rng(seed)
    N = int(rng.integers(1, 90))
    R = int(rng.integers(1, 5))
    B = int(rng.integers(1, N + 3))
    L = int(rng.integers(1, 13))
    t_min = int(rng.integers(1, min(L, 3) + 1))
    if seed % 3 == 0:
        gid = O.groups(WL.group_permutations(seed, R, N), B)          # Alg. 1's design
    else:
        gid = O.design_groups(WL.random_design(seed, R, N, B), B)     # a design given outright
    moff, mem = O.members(gid, B)
    # counts with many ties (few distinct levels) and with spread
    hi = L if seed % 2 else min(L, 3)
    cnt = rng.integers(0, hi + 1, size=B * R).astype(np.uint16)
    for kq in (1, 2, 5, N, N + 3):
        gcells = int(rng.integers(1, B + 2))
        cap_fill = kq + int(rng.integers(1, 9))
        ids, sc, n = O.alg3(cnt, moff, mem, N, R, B, k=kq, t_min=t_min)
        w_ids, w_sc = kernel_walk(cnt, gid, B, L, kq, t_min, gcells, cap_fill, rng)
        assert w_ids == ids[:n].tolist() and w_sc == sc[:n].tolist(), (kq, gcells, cap_fill)


def group_extent_linear(lvl_n, t, t_min, gcells):
    """The group rule as stated: level t, then the levels below it while the
    group holds at most gcells cells."""
    nc, t_end = lvl_n[t], t
    while t_end > t_min and nc + lvl_n[t_end - 1] <= gcells:
        t_end -= 1
        nc += lvl_n[t_end]
    return t_end, nc


def group_extent_bsearch(lvl_n, t, t_min, gcells):
    """The kernels' form: ge[v] = cells at levels >= v (the level placement's
    end cursors), first = ge[t] - lvl_n[t], then a binary search for the lowest
    t_end with ge[t_end] <= first + gcells (level t always belongs)."""
    L = len(lvl_n) - 1
    ge = [0] * (L + 2)
    for v in range(L, -1, -1):
        ge[v] = ge[v + 1] + lvl_n[v]
    first = ge[t] - lvl_n[t]
    lim = first + gcells
    t_end = t
    if ge[t] <= lim:
        lo, hi = t_min, t
        while lo < hi:
            mid = (lo + hi) >> 1
            if ge[mid] <= lim:
                hi = mid
            else:
                lo = mid + 1
        t_end = lo
    return t_end, ge[t_end] - first


@pytest.mark.parametrize("seed", range(200))
def test_group_extent_binary_search_equals_walk(seed):
    rng = np.random.default_rng(1000 + seed)
    L = int(rng.integers(1, 600))
    t_min = int(rng.integers(1, min(L, 4) + 1))
    # mostly empty levels with a few crowded ones, as at high table counts
    lvl_n = np.zeros(L + 1, np.int64)
    busy = rng.choice(np.arange(t_min, L + 1), size=int(rng.integers(0, min(L - t_min + 1, 40) + 1)),
                      replace=False)
    lvl_n[busy] = rng.integers(1, 400, size=len(busy))
    lvl_n = lvl_n.tolist()
    for gcells in (1, 7, int(rng.integers(1, 500)), 10 ** 6):
        t = L
        while t >= t_min:
            a = group_extent_linear(lvl_n, t, t_min, gcells)
            b = group_extent_bsearch(lvl_n, t, t_min, gcells)
            assert a == b, (t, gcells)
            t = a[0] - 1
