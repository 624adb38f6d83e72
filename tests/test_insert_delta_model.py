"""The touched-slot insert's index arithmetic, modelled on the CPU step by step
as the kernels take it, against a plain rebuild of the union (the oracle's
CSR of all points):

- per table, the batch's (bucket, cell) keys sorted and deduplicated, less
  the cells the slot's old list holds; the touched slots and their first
  added cell;
- flattened in slot order: gslot, gdbeg (added cells before touched slot j),
  gbeg / gend (old extent), with the sentinels past the end;
- the offsets pass in chunks: the chunk's first touched slot precomputed,
  then four slots per vector with one search and the in-vector step rule;
- the cell pass in chunks: each thread loads its entries (pairs of words)
  and walks the runs between touched slots with its own cursor from the
  chunk's precomputed run;
- the merge of each touched slot by ranks in the other list.

Chunks are a few entries long so that every boundary case occurs: touched
slots at chunk edges, empty old lists, runs spanning chunks, untouched
tables."""
import bisect

import numpy as np
import pytest

from oracle import oracle as O

NONE = 0xFFFFFFFF


def model_insert(off, cells, L, W, R, B, nbuck, ngid, chunk_slots=8, threads=4, words=2):
    nslot = L << W
    n = nbuck.shape[0]
    cells = list(int(c) for c in cells)
    off = [int(o) for o in off]
    # step 1: per table
    rcell, rt = [], []
    for l in range(L):
        keys = sorted({(int(nbuck[x, l]) << 16) | (r * B + int(ngid[x, r])) for x in range(n) for r in range(R)})
        kept = []
        for k in keys:
            s = (l << W) | (k >> 16)
            old = cells[off[s]:off[s + 1]]
            if (k & 0xFFFF) not in old:
                kept.append(k)
        rcell.append([k & 0xFFFF for k in kept])
        rt.append([(k >> 16, i) for i, k in enumerate(kept) if i == 0 or (k >> 16) != (kept[i - 1] >> 16)])
    # step 2: flatten in slot order
    gslot, gdbeg, gbeg, gend, gdcell = [], [], [], [], []
    a0 = 0
    for l in range(L):
        for b, first in rt[l]:
            s = (l << W) | b
            gslot.append(s)
            gdbeg.append(a0 + first)
            gbeg.append(off[s])
            gend.append(off[s + 1])
        gdcell += rcell[l]
        a0 += len(rcell[l])
    Tt, added = len(gslot), a0
    gslot.append(NONE)
    gdbeg.append(added)
    gbeg.append(NONE)
    gend.append(NONE)
    n_cells = len(cells)
    # step 3: offsets, chunk by chunk, four slots per vector
    noff = [None] * (nslot + 1)
    nc_off = (nslot + 1 + chunk_slots - 1) // chunk_slots
    off_j = [bisect.bisect_left(gslot, c * chunk_slots, 0, Tt) if c * chunk_slots <= nslot else Tt
             for c in range(nc_off + 1)]
    for c in range(nc_off):
        s0, s1 = c * chunk_slots, min(c * chunk_slots + chunk_slots, nslot + 1)
        j0, nj = off_j[c], off_j[c + 1] - off_j[c]
        assert nj <= s1 - s0
        sgs, sgd = gslot[j0:j0 + nj + 1], gdbeg[j0:j0 + nj + 1]

        def first_at(s):
            return bisect.bisect_left(sgs, s, 0, nj)
        nv = (s1 - s0) // 4
        for v in range(nv):
            s = s0 + 4 * v
            t = first_at(s)
            sh = sgd[t]
            out = [off[s] + sh]
            for q in range(3):
                if t < nj and sgs[t] == s + q:
                    t += 1
                    sh = sgd[t]
                out.append(off[s + q + 1] + sh)
            noff[s:s + 4] = out
        for s in range(s0 + 4 * nv, s1):
            noff[s] = off[s] + sgd[first_at(s)]
    # step 4: the untouched runs, per chunk and thread
    ncells = [None] * (n_cells + added)
    chunk = 2 * threads * words
    nc_mov = (n_cells + chunk - 1) // chunk
    for c in range(nc_mov):
        i0 = c * chunk
        mov_lo = bisect.bisect_right(gend, i0, 0, Tt)
        for th in range(threads):
            j = mov_lo
            e, b, sh = gend[j], gbeg[j], gdbeg[j]
            for k in range(2 * words):
                i = i0 + 2 * ((k >> 1) * threads + th) + (k & 1)
                if i >= n_cells:
                    break
                while i >= e:
                    j += 1
                    e, b, sh = gend[j], gbeg[j], gdbeg[j]
                if i < b:
                    assert ncells[i + sh] is None
                    ncells[i + sh] = cells[i]
    # step 5: the touched slots' unions by ranks
    for j in range(Tt):
        s = gslot[j]
        old = cells[off[s]:off[s + 1]]
        add = gdcell[gdbeg[j]:gdbeg[j + 1]]
        dst = off[s] + gdbeg[j]
        for i, cval in enumerate(old):
            ncells[dst + i + bisect.bisect_left(add, cval)] = cval
        for i, cval in enumerate(add):
            ncells[dst + i + bisect.bisect_left(old, cval)] = cval
    return np.array(noff, np.uint32), np.array(ncells, np.uint16), Tt


@pytest.mark.parametrize("seed", range(60))
def test_model_equals_rebuild_of_the_union(seed):
    rng = np.random.default_rng(4000 + seed)
    L, W, R = int(rng.integers(1, 5)), int(rng.integers(1, 6)), int(rng.integers(1, 4))
    B = int(rng.integers(1, 7))
    N0, n = int(rng.integers(1, 40)), int(rng.integers(1, 12))
    nb_max = 1 << W if seed % 3 else min(2, 1 << W)       # some cases crowd a few buckets
    ob = rng.integers(0, nb_max, size=(N0, L)).astype(np.uint32)
    og = rng.integers(0, B, size=(N0, R)).astype(np.uint16)
    nb = rng.integers(0, nb_max, size=(n, L)).astype(np.uint32)
    ng = rng.integers(0, B, size=(n, R)).astype(np.uint16)
    if seed % 5 == 0:                                      # repeat indexed points
        nb[: min(n, N0)] = ob[: min(n, N0)]
        ng[: min(n, N0)] = og[: min(n, N0)]
    off, cells = O.build_csr(ob, og, B, W)
    noff, ncells, _ = model_insert(off, cells, L, W, R, B, nb, ng,
                                   chunk_slots=int(rng.choice([4, 8, 12])),
                                   threads=int(rng.integers(1, 4)), words=int(rng.integers(1, 3)))
    roff, rcells = O.build_csr(np.concatenate([ob, nb]), np.concatenate([og, ng]), B, W)
    assert np.array_equal(noff, roff)
    assert np.array_equal(ncells, rcells)


def test_model_catches_a_shift_off_by_one():
    """The in-vector step rule matters: compare with the slot itself instead
    of the slot before and the model no longer matches the rebuild."""
    rng = np.random.default_rng(7)
    bad = 0
    for _ in range(40):
        L, W, R, B = 2, 3, 2, 3
        ob = rng.integers(0, 8, size=(10, L)).astype(np.uint32)
        og = rng.integers(0, B, size=(10, R)).astype(np.uint16)
        nb = rng.integers(0, 8, size=(4, L)).astype(np.uint32)
        ng = rng.integers(0, B, size=(4, R)).astype(np.uint16)
        off, cells = O.build_csr(ob, og, B, W)
        noff, _, _ = model_insert(off, cells, L, W, R, B, nb, ng, chunk_slots=8)
        roff, _ = O.build_csr(np.concatenate([ob, nb]), np.concatenate([og, ng]), B, W)
        # the wrong rule: every slot of a vector takes the vector's first shift
        wrong = noff.copy()
        for s in range(0, (L << W) + 1 - 3, 4):
            wrong[s + 1:s + 4] = off[s + 1:s + 4] + (noff[s] - off[s])
        bad += not np.array_equal(wrong, roff)
        assert np.array_equal(noff, roff)
    assert bad > 0
