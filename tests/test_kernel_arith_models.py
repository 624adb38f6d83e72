"""CPU models of three pieces of the query kernels' arithmetic, checked against
their plain definitions (no GPU).

* Heavy-bucket counts (Sec. 5: a cell's count is the number of tables whose
  bucket holds it). For a heavy bucket the kernels add the cell bitmaps of
  all heavy tables in bit-sliced form: a carry-save adder tree over eight
  bitmap words, the weight-8 carry rippled into higher planes, a pass per
  248 tables, then the planes spread into packed 8- or 16-bit counters. The
  model must give each cell's number of set bits, for any table count.
* The contiguous-slice walk over flattened lists. Each warp takes a slice of
  the entries; a lane finds its list by a forward search from its previous
  one (four steps, then a binary search), ended by the prefix sums past the
  last list and a sentinel at NT. The model must visit every entry exactly
  once, in its own list, with empty lists anywhere.
* The decode's member walk: a warp-uniform cursor holds the cell of the
  step's first member, and one pass over the cell boundaries inside the step
  maps every lane to its cell. The model must visit every member exactly
  once, in its own cell, with empty cells anywhere.
* The radix select that cuts a buffer of more than 256 candidates to the k
  best: the (prefix, mask) it returns must keep exactly the k smallest keys,
  for 8- and 16-bit score fields and long runs of equal leading digits.
"""
import numpy as np
import pytest

M32 = 0xFFFFFFFF


def csa(a, b, c):
    u = a ^ b
    return (a & b) | (u & c), u ^ c            # carry, sum


def bitsliced_counts(words, cw):
    """words: (nh, nw) uint32 bitmaps. Returns the packed counter words the
    kernels add: cw = 1 -> 8 words of 4 byte counts per bitmap word, cw = 2
    -> 16 words of 2 half-word counts."""
    nh, nw = words.shape
    k_per = 8 if cw == 1 else 16
    k_cells = 32 // k_per
    out = np.zeros(nw * k_per, np.uint64)
    for w in range(nw):
        for i1 in range(0, nh, 248):
            i2 = min(nh, i1 + 248)
            pl = [0] * 8
            for i0 in range(i1, i2, 8):
                x = [int(words[i0 + v, w]) if i0 + v < i2 else 0 for v in range(8)]
                t0, pl[0] = csa(pl[0], x[0], x[1])
                t1, pl[0] = csa(pl[0], x[2], x[3])
                f0, pl[1] = csa(pl[1], t0, t1)
                t0, pl[0] = csa(pl[0], x[4], x[5])
                t1, pl[0] = csa(pl[0], x[6], x[7])
                f1, pl[1] = csa(pl[1], t0, t1)
                e, pl[2] = csa(pl[2], f0, f1)
                for p in range(3, 8):
                    c = pl[p] & e
                    pl[p] ^= e
                    e = c
                assert e == 0                      # at most 247 per pass: 8 planes suffice
            np_ = (i2 - i1).bit_length()
            for j in range(k_per):
                acc = 0
                for p in range(np_):
                    bits = (pl[p] >> (k_cells * j)) & ((1 << k_cells) - 1)
                    if cw == 1:
                        acc += ((bits * 0x00204081) & 0x01010101) << p
                    else:
                        acc += ((bits * 0x8001) & 0x10001) << p
                out[w * k_per + j] += acc & M32
    return out


@pytest.mark.parametrize("nh", [1, 2, 7, 8, 9, 63, 247, 248, 249, 255, 500, 1000])
@pytest.mark.parametrize("cw", [1, 2])
def test_bitsliced_heavy_counts_equal_popcounts(nh, cw):
    if cw == 1 and nh > 255:
        pytest.skip("8-bit counters hold at most 255 tables")
    rng = np.random.default_rng([nh, cw])
    nw = 3
    words = rng.integers(0, 1 << 32, size=(nh, nw), dtype=np.uint64).astype(np.uint32)
    if nh > 5:
        words[:, 0] = M32                      # every table holds the first word's cells
        words[: nh // 2, 1] = 0
    got = bitsliced_counts(words, cw)
    k_per = 8 if cw == 1 else 16
    k_cells = 32 // k_per
    width = 8 if cw == 1 else 16
    for w in range(nw):
        for cell in range(32):
            want = int(((words[:, w].astype(np.uint64) >> cell) & 1).sum())
            j, i = divmod(cell, k_cells)
            field = (int(got[w * k_per + j]) >> (width * i)) & ((1 << width) - 1)
            assert field == want, (w, cell)


def find_seg(pre, n, j, lo=0):
    hi = n
    while hi - lo > 1:
        mid = (lo + hi) >> 1
        if pre[mid] <= j:
            lo = mid
        else:
            hi = mid
    return lo


def slice_walk(lens, NT, U):
    """Entries visited by the kernels' contiguous-slice walk: (entry, list)."""
    n = len(lens)
    assert n <= NT
    pre = np.zeros(NT + 1, np.int64)
    total = int(sum(lens))
    run = 0
    for t in range(NT):
        pre[t] = run
        run += lens[t] if t < n else 0
    pre[NT] = M32                               # the sentinel
    seen = []
    nwarps = NT // 32
    per = ((total + nwarps - 1) // nwarps + 31) & ~31
    for w in range(nwarps):
        eb0 = min(w * per, total)
        ee = min(eb0 + per, total)
        for lane in range(32):
            hint = [find_seg(pre, n, eb0 + u * 32 + lane) if eb0 + u * 32 + lane < ee else 0 for u in range(U)]
            for eb in range(eb0, ee, 32 * U):
                for u in range(U):
                    e = eb + u * 32 + lane
                    if e >= ee:
                        continue
                    t = hint[u]
                    step = 0
                    while pre[t + 1] <= e:
                        if step == 4:
                            t = find_seg(pre, n, e, t + 1)
                            break
                        t += 1
                        step += 1
                    hint[u] = t
                    seen.append((e, t))
    return seen, pre


@pytest.mark.parametrize("seed", range(40))
def test_slice_walk_visits_every_entry_once_in_its_list(seed):
    rng = np.random.default_rng(seed)
    NT = int(rng.choice([128, 256, 512]))
    U = int(rng.choice([1, 4]))
    n = int(rng.integers(1, NT + 1))
    lens = rng.choice([0, 0, 1, 3, 17, 40, 200, 1000], size=n).tolist()
    seen, pre = slice_walk(lens, NT, U)
    total = int(sum(lens))
    assert sorted(e for e, _ in seen) == list(range(total))
    for e, t in seen:
        assert pre[t] <= e < pre[t] + lens[t] and lens[t] > 0


def cursor_walk(lens, NT, U):
    """Members visited by the decode's walk: each warp takes a contiguous slice;
    a warp-uniform cursor (the cell holding the step's first member) and one
    pass over the cell boundaries inside each step map lanes to cells. Returns
    (member, cell) pairs, and the number of boundary reads per step."""
    n = len(lens)
    assert n <= NT
    pre = np.zeros(NT + 1, np.int64)
    total = int(sum(lens))
    run = 0
    for t in range(NT):
        pre[t] = run
        run += lens[t] if t < n else 0
    pre[NT] = M32                               # the sentinel
    seen, reads = [], []
    nwarps = NT // 32
    per = ((total + nwarps - 1) // nwarps + 31) & ~31
    for w in range(nwarps):
        jb = min(w * per, total)
        je = min(jb + per, total)
        cur = find_seg(pre, n, jb) if jb < je else 0
        while jb < je:
            last_j = min(jb + 32 * U, je) - 1
            my = [[cur] * 32 for _ in range(U)]
            k = cur + 1
            bnd = pre[k]
            nread = 1
            while bnd <= last_j:
                for u in range(U):
                    for lane in range(32):
                        if jb + u * 32 + lane >= bnd:
                            my[u][lane] = k
                k += 1
                bnd = pre[k]
                nread += 1
            reads.append(nread)
            for u in range(U):
                for lane in range(32):
                    j = jb + u * 32 + lane
                    if j < je:
                        seen.append((j, my[u][lane]))
            jb += 32 * U
            cur = k - 1
    return seen, pre, reads


@pytest.mark.parametrize("seed", range(60))
def test_cursor_walk_visits_every_member_once_in_its_cell(seed):
    rng = np.random.default_rng(500 + seed)
    NT = int(rng.choice([128, 256, 512]))
    U = int(rng.choice([1, 4]))
    n = int(rng.integers(1, NT + 1))
    # empty cells anywhere (skipped cells have no members), runs of tiny ones
    lens = rng.choice([0, 0, 0, 1, 2, 24, 25, 100, 500], size=n).tolist()
    seen, pre, reads = cursor_walk(lens, NT, U)
    total = int(sum(lens))
    assert sorted(j for j, _ in seen) == list(range(total))
    for j, c in seen:
        assert pre[c] <= j < pre[c] + lens[c] and lens[c] > 0
    # the pass reads one boundary per cell it crosses, plus one
    if reads:
        assert max(reads) <= 32 * U + NT


# ---------------------------------------------------------------- radix select
#
# Buffers of more than 256 candidates are cut to the k best by a radix select
# over the 64-bit keys (-score as kScoreMax - score, last cell, id): from the
# top digit down, a histogram of the keys that match the prefix chosen so far
# picks the digit holding the k-th key; it stops early once that digit's
# bucket is taken whole. The kept keys are those with (key & mask) <= prefix.

def block_select(keys, kk, top_shift):
    prefix = mask = 0
    rem = kk
    for shift in range(top_shift, -1, -8):
        hist = [0] * 256
        for v in keys:
            if (v & mask) == prefix:
                hist[(v >> shift) & 0xFF] += 1
        run, d = 0, 0
        for d in range(256):
            if run + hist[d] >= rem:
                break
            run += hist[d]
        hd = hist[d]
        rem -= run
        prefix |= d << shift
        mask |= 0xFF << shift
        if hd == rem:
            break
    return prefix, mask


@pytest.mark.parametrize("seed", range(60))
def test_radix_select_keeps_exactly_the_k_smallest(seed):
    rng = np.random.default_rng(seed)
    wide = seed % 2 == 1                        # 16-bit counts: a 12-bit score field
    kmax_score = 4095 if wide else 255
    top_shift = 56 if wide else 48
    n = int(rng.integers(257, 3000))
    # few distinct scores and cells, so long runs of equal top digits
    score = rng.integers(0, rng.choice([2, 5, kmax_score + 1]), size=n)
    last = rng.integers(0, rng.choice([3, 60000]), size=n)
    ids = rng.permutation(1 << 20)[:n]          # distinct ids: distinct keys
    keys = [((kmax_score - int(s)) << 48) | (int(c) << 32) | int(x) for s, c, x in zip(score, last, ids)]
    for kk in {1, 2, 10, 100, 256, n - 1, n, int(rng.integers(1, n + 1))}:
        prefix, mask = block_select(keys, kk, top_shift)
        kept = sorted(v for v in keys if (v & mask) <= prefix)
        assert kept == sorted(keys)[:kk], kk


# ---------------------------------------------------------------- build: small-slot sort
#
# The build sorts and deduplicates each slot of at most sixteen cells in one
# thread's registers with a fixed compare-exchange network (Batcher's odd-even
# merge sort for sixteen inputs, 63 comparators; its first nineteen sort the
# first eight inputs alone), padded with 0xFFFFFFFF. By the 0-1 principle a
# network that sorts all binary inputs sorts every input; the dedupe then
# keeps the first of each run. The network is read from the kernel's source.


def net_sort(vals):
    net = kernel_network()
    n = 8 if len(vals) <= 8 else 16
    v = list(vals) + [M32] * (n - len(vals))
    for i, j in (net[:19] if n == 8 else net):
        if v[i] > v[j]:
            v[i], v[j] = v[j], v[i]
    return v


@pytest.mark.parametrize("seed", range(20))
def test_small_slot_sort_and_dedupe(seed):
    rng = np.random.default_rng(900 + seed)
    for _ in range(200):
        n = int(rng.integers(0, 17))
        vals = rng.integers(0, int(rng.choice([3, 20, 65536])), size=n).tolist()
        v = net_sort(vals)
        out = [x for i, x in enumerate(v) if x != M32 and (i == 0 or x != v[i - 1])]
        assert out == sorted(set(vals))


def kernel_network():
    """The compare-exchange pairs of k_slot_unique_small, read from the source."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_2106_11565_gb300", "csrc", "build.cu")).read()
    body = src[src.index("kNet16[63][2] = {"):]
    body = body[:body.index("};")]
    return [(int(a), int(b)) for a, b in re.findall(r"\{(\d+), (\d+)\}", body)]


def test_kernel_network_sorts_16_and_its_prefix_sorts_8():
    net = kernel_network()
    assert len(net) == 63
    # 0-1 principle, vectorised over all 2^16 binary inputs
    m = np.arange(1 << 16, dtype=np.uint32)
    v = ((m[:, None] >> np.arange(16, dtype=np.uint32)[None, :]) & 1).astype(np.uint8)
    for i, j in net:
        lo = np.minimum(v[:, i], v[:, j])
        hi = np.maximum(v[:, i], v[:, j])
        v[:, i], v[:, j] = lo, hi
    assert np.all(np.diff(v.astype(np.int8), axis=1) >= 0)
    # the first nineteen comparators touch only the first eight inputs and sort them
    pre = net[:19]
    assert all(i < 8 and j < 8 for i, j in pre)
    m = np.arange(1 << 8, dtype=np.uint32)
    v = ((m[:, None] >> np.arange(8, dtype=np.uint32)[None, :]) & 1).astype(np.uint8)
    for i, j in pre:
        lo = np.minimum(v[:, i], v[:, j])
        hi = np.maximum(v[:, i], v[:, j])
        v[:, i], v[:, j] = lo, hi
    assert np.all(np.diff(v.astype(np.int8), axis=1) >= 0)
