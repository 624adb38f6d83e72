// Insert of a small batch into a built index (the reverse index of Sec. 5;
// the batch's groups, Alg. 1, are already in gid). Only the slots that gain
// cells are merged. Every other list keeps its content and moves by the
// number of cells added to the slots before it, so the offsets and the cell
// array each take one streaming pass, and no work runs per slot of the whole
// index (L * 2^W slots, most of them untouched by a batch).
//
//  1. k_delta_table, one CTA per table: the batch's (bucket, cell) entries of
//     table l (n * R of them) sorted in shared memory, deduplicated (a filter
//     bit is set once, Sec. 3.3), and stripped of the cells the slot's list
//     already holds; what remains is "added". The table's touched slots
//     (those with added cells) and their first added cell.
//  2. Prefix sums of the per-table totals; k_delta_flatten lays the touched
//     slots of all tables out in slot order: gslot[j], gdbeg[j] (added cells
//     before touched slot j, over the whole index), gbeg[j] / gend[j] (the old
//     extent of its list), and the added cells gdcell in the same order.
//  3. new off[s] = off[s] + gdbeg[first touched slot >= s], and
//  4. the untouched lists between two touched slots, a run of old entries,
//     move together by the cells added before them: both passes in one
//     launch, k_delta_stream, their chunks interleaved.
//  5. k_delta_merge, a warp per touched slot, on a second stream beside 3-4
//     (it writes only the touched slots' lists): the union of its old and
//     added cells (disjoint, both sorted) written at its new offset, each
//     element at its own index plus its rank in the other list; cell bitmaps
//     of heavy slots get the added cells; slots that become heavy are listed.
//  6. New bitmaps for the listed slots (the host grows the bitmap array first).
#include <algorithm>
#include <utility>

#include "internal.cuh"

namespace flinng {
namespace {

constexpr int kDeltaThreads = 1024;
constexpr int kWarps = 8;                 // warps per CTA of the warp-per-slot kernels
constexpr uint32_t kChunk = 4096;         // slots / entries per CTA of the streaming passes

// Exclusive prefix of v over the CTA (thread order); total in *total.
// wsum: 32 words of shared memory. Contains __syncthreads.
__device__ uint32_t cta_excl_scan(uint32_t v, uint32_t *wsum, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    const uint32_t before = warp > 0 ? wsum[warp - 1] : 0u;
    *total = wsum[nw - 1];
    __syncthreads();
    return before + x - v;
}

// First index in a[lo, hi) with a[index] >= v (hi if none).
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *a, uint32_t lo, uint32_t hi, uint32_t v)
{
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// First index in a[lo, hi) with a[index] > v (hi if none).
__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t *a, uint32_t lo, uint32_t hi, uint32_t v)
{
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Number of entries of the sorted list a[0, n) smaller than v.
__device__ __forceinline__ uint32_t rank_u16(const uint16_t *a, uint32_t n, uint32_t v)
{
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (uint32_t(a[mid]) < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Step 1. Keys are (bucket << CB) | cell (CB bits hold a cell id), 32-bit
// when W + CB <= 31; P2 (a power of two, 32 .. 32 E blockDim, >= n R) of
// them in shared memory, E = max(1, P2 / blockDim) per thread.
template <class KT, int E>
__global__ void __launch_bounds__(kDeltaThreads)
k_delta_table(const uint32_t *__restrict__ buckets, const uint16_t *__restrict__ gid, uint64_t n_old, uint32_t n,
              uint32_t L, uint32_t W, uint32_t R, uint32_t B, uint32_t rp, uint32_t P2, uint32_t CB,
              const uint32_t *__restrict__ off, const uint16_t *__restrict__ cells, uint16_t *__restrict__ rcell,
              uint2 *__restrict__ rt, uint32_t *__restrict__ A, uint32_t *__restrict__ T)
{
    constexpr KT kNone = ~KT(0);
    extern __shared__ __align__(16) unsigned char dsm[];
    KT *key = reinterpret_cast<KT *>(dsm);
    uint32_t *wsum = reinterpret_cast<uint32_t *>(key + P2);
    const uint32_t l = blockIdx.x, nR = n * R, tid = threadIdx.x, nt = blockDim.x;
    const KT cmask = (KT(1) << CB) - 1;
    for (uint32_t i = tid; i < P2; i += nt) {
        KT k = kNone;
        if (i < nR) {
            const uint32_t x = i / R, r = i - x * R;
            const uint32_t b = buckets[uint64_t(x) * L + l];
            const uint32_t c = r * B + gid[(n_old + x) * rp + r];
            k = (KT(b) << CB) | KT(c);
        }
        key[i] = k;
    }
    __syncthreads();
    // Bitonic sort. Warp w holds keys w 32 E .. (w + 1) 32 E - 1, lane-major
    // (key e 32 + lane of its block in register e): compare-exchanges at
    // distance < 32 are warp shuffles, at distance < 32 E between registers,
    // and only the longer ones go through shared memory.
    const uint32_t warp = tid >> 5, lane = tid & 31;
    const bool active = warp * 32 * E < P2;
    const uint32_t base = warp * 32 * E;
    KT v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = active ? key[base + e * 32 + lane] : kNone;
    for (uint32_t k2 = 2; k2 <= P2; k2 <<= 1) {
        uint32_t j = k2 >> 1;
        if (j >= 32u * E) {
            if (active) {
#pragma unroll
                for (int e = 0; e < E; ++e) key[base + e * 32 + lane] = v[e];
            }
            __syncthreads();
            for (; j >= 32u * E; j >>= 1) {
                for (uint32_t i = tid; i < P2; i += nt) {
                    const uint32_t p = i ^ j;
                    if (p > i) {
                        const KT x = key[i], y = key[p];
                        if ((x > y) == ((i & k2) == 0)) {
                            key[i] = y;
                            key[p] = x;
                        }
                    }
                }
                __syncthreads();
            }
            if (active) {
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = key[base + e * 32 + lane];
            }
        }
        if (!active) continue;
#pragma unroll
        for (int jj = E / 2; jj >= 1; jj >>= 1) {      // distance 32 jj: registers e and e ^ jj
            if (j != 32u * jj) continue;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int p = e ^ jj;
                if (p > e) {
                    const uint32_t i = base + e * 32 + lane;
                    const KT x = v[e], y = v[p];
                    if ((x > y) == ((i & k2) == 0)) {
                        v[e] = y;
                        v[p] = x;
                    }
                }
            }
            j >>= 1;
        }
        for (; j > 0; j >>= 1) {                       // distance < 32: lanes
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const uint32_t i = base + e * 32 + lane;
                const KT o = __shfl_xor_sync(0xffffffffu, v[e], j);
                const bool up = (i & k2) == 0, lower = (lane & j) == 0;
                v[e] = (lower == up) ? (v[e] < o ? v[e] : o) : (v[e] < o ? o : v[e]);
            }
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int e = 0; e < E; ++e) key[base + e * 32 + lane] = v[e];
    }
    __syncthreads();
    // keep the first of equal keys whose cell the slot's old list lacks; each
    // thread now takes E consecutive keys
    const uint32_t i0 = tid * E;
    KT mine[8];
    uint32_t keepm = 0, cnt = 0;
#pragma unroll
    for (uint32_t e = 0; e < 8; ++e) {
        mine[e] = kNone;
        if (e >= E) break;
        const uint32_t i = i0 + e;
        if (i >= P2) break;
        const KT k = key[i];
        mine[e] = k;
        if (k == kNone || (i > 0 && key[i - 1] == k)) continue;
        const uint64_t slot = (uint64_t(l) << W) | uint64_t(k >> CB);
        const uint32_t o0 = off[slot], o1 = off[slot + 1];
        const uint32_t c = uint32_t(k & cmask);
        const uint32_t rk = rank_u16(cells + o0, o1 - o0, c);
        if (o0 + rk < o1 && cells[o0 + rk] == c) continue;
        keepm |= 1u << e;
        ++cnt;
    }
    uint32_t total;
    uint32_t pos = cta_excl_scan(cnt, wsum, &total);      // every read of key[] is above this barrier
#pragma unroll
    for (uint32_t e = 0; e < 8; ++e)
        if ((keepm >> e) & 1u) key[pos++] = mine[e];
    __syncthreads();
    // touched slots: the first kept key of each bucket
    const uint32_t nA = total;
    uint32_t tcnt = 0, tm = 0;
#pragma unroll
    for (uint32_t e = 0; e < 8; ++e) {
        if (e >= E) break;
        const uint32_t i = i0 + e;
        if (i >= nA) break;
        rcell[uint64_t(l) * nR + i] = uint16_t(key[i] & cmask);
        if (i == 0 || (key[i] >> CB) != (key[i - 1] >> CB)) {
            tm |= 1u << e;
            ++tcnt;
        }
    }
    uint32_t nT;
    uint32_t tp = cta_excl_scan(tcnt, wsum, &nT);
#pragma unroll
    for (uint32_t e = 0; e < 8; ++e)
        if ((tm >> e) & 1u) rt[uint64_t(l) * nR + tp++] = make_uint2(uint32_t(key[i0 + e] >> CB), i0 + e);
    if (tid == 0) {
        A[l] = nA;
        T[l] = nT;
    }
}

// Step 2. Apre, Tpre: exclusive prefixes of A, T over the tables (L + 1
// entries, totals last). Sentinels close gslot / gdbeg / gend.
__global__ void k_delta_flatten(const uint32_t *__restrict__ Apre, const uint32_t *__restrict__ Tpre, uint32_t L,
                                uint32_t W, uint32_t nR, const uint16_t *__restrict__ rcell,
                                const uint2 *__restrict__ rt, const uint32_t *__restrict__ off,
                                uint32_t *__restrict__ gslot, uint32_t *__restrict__ gdbeg,
                                uint32_t *__restrict__ gbeg, uint32_t *__restrict__ gend,
                                uint16_t *__restrict__ gdcell)
{
    const uint32_t l = blockIdx.x;
    const uint32_t a0 = Apre[l], na = Apre[l + 1] - a0, t0 = Tpre[l], ntt = Tpre[l + 1] - t0;
    for (uint32_t i = threadIdx.x; i < na; i += blockDim.x) gdcell[a0 + i] = rcell[uint64_t(l) * nR + i];
    for (uint32_t j = threadIdx.x; j < ntt; j += blockDim.x) {
        const uint2 t = rt[uint64_t(l) * nR + j];
        const uint32_t slot = (l << W) | t.x;
        gslot[t0 + j] = slot;
        gdbeg[t0 + j] = a0 + t.y;
        gbeg[t0 + j] = off[slot];
        gend[t0 + j] = off[slot + 1];
    }
    if (l == 0 && threadIdx.x == 0) {
        const uint32_t Tt = Tpre[L];
        gslot[Tt] = kEmpty32;
        gdbeg[Tt] = Apre[L];
        gbeg[Tt] = kEmpty32;
        gend[Tt] = kEmpty32;
    }
}

// The touched slots each chunk of the streaming passes meets, found by one
// thread per chunk, so that no CTA of a pass starts with a long dependent
// search. Offsets pass: off_j[c] = first j with gslot[j] >= c kChunk (Tt past
// the last slot). Move pass: mov_lo[c] = the number of touched lists ending at
// or before entry c kChunk, the run holding that entry.
__global__ void k_delta_chunks(const uint32_t *__restrict__ gslot, const uint32_t *__restrict__ gend,
                               const uint32_t *__restrict__ Tpre, uint32_t L, uint64_t nslot, uint64_t n_cells,
                               uint32_t nc_off, uint32_t nc_mov, uint32_t *__restrict__ off_j,
                               uint32_t *__restrict__ mov_lo)
{
    const uint32_t Tt = Tpre[L];
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= nc_off) {
        const uint64_t s = uint64_t(t) * kChunk;
        off_j[t] = s > nslot ? Tt : lower_bound_u32(gslot, 0, Tt, uint32_t(s));
    }
    if (t < nc_mov) mov_lo[t] = upper_bound_u32(gend, 0, Tt, uint32_t(uint64_t(t) * kChunk));
}

// Step 3, over slots 0 .. nslot (the offsets' nslot + 1 entries), four
// slots per 16-byte access. Chunk c's slots [s0, s1) meet the touched slots
// j0 .. j1 - 1, which it stages in shared memory with gdbeg[j1] (when fewer
// than kStage; else it searches them in place).
constexpr uint32_t kStage = 1024;     // touched slots a chunk stages in shared memory

__device__ void delta_offsets(uint32_t c, uint32_t *sgs, uint32_t *sgd, const uint32_t *__restrict__ off,
                              uint64_t nslot, const uint32_t *__restrict__ gslot, const uint32_t *__restrict__ gdbeg,
                              const uint32_t *__restrict__ off_j, uint32_t *__restrict__ noff)
{
    const uint64_t s0 = uint64_t(c) * kChunk;
    const uint64_t s1 = s0 + kChunk < nslot + 1 ? s0 + kChunk : nslot + 1;
    // off_j[c + 1] is the first touched slot >= s1 (the total past the last chunk)
    const uint32_t j0 = off_j[c], nj = off_j[c + 1] - j0;   // nj <= s1 - s0
    const bool staged = nj < kStage;
    if (staged) {
        for (uint32_t t = threadIdx.x; t <= nj; t += blockDim.x) {
            sgs[t] = gslot[j0 + t];
            sgd[t] = gdbeg[j0 + t];
        }
    }
    __syncthreads();
    // first touched index >= j0 (relative) with gslot >= s, and the shift there
    auto first_at = [&](uint32_t s) {
        uint32_t lo = 0, hi = nj;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if ((staged ? sgs[mid] : gslot[j0 + mid]) < s) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    auto slot_at = [&](uint32_t t) { return staged ? sgs[t] : gslot[j0 + t]; };   // t <= nj: sentinel past the end
    auto shift_at = [&](uint32_t t) { return staged ? sgd[t] : gdbeg[j0 + t]; };
    const uint32_t nv = uint32_t((s1 - s0) / 4);
    for (uint32_t v = threadIdx.x; v < nv; v += blockDim.x) {
        const uint64_t s = s0 + uint64_t(v) * 4;
        uint4 x = *reinterpret_cast<const uint4 *>(off + s);
        uint32_t t = first_at(uint32_t(s));
        // slots s .. s + 3 share the shift unless a touched slot lies among s .. s + 2
        uint32_t sh = shift_at(t);
        x.x += sh;
        if (t < nj && slot_at(t) == uint32_t(s)) sh = shift_at(++t);
        x.y += sh;
        if (t < nj && slot_at(t) == uint32_t(s + 1)) sh = shift_at(++t);
        x.z += sh;
        if (t < nj && slot_at(t) == uint32_t(s + 2)) sh = shift_at(++t);
        x.w += sh;
        *reinterpret_cast<uint4 *>(noff + s) = x;
    }
    for (uint64_t s = s0 + uint64_t(nv) * 4 + threadIdx.x; s < s1; s += blockDim.x)
        noff[s] = off[s] + shift_at(first_at(uint32_t(s)));
}

// Step 4, over the old entries, kChunk per CTA. Between touched slots j - 1
// and j lies a run of untouched lists, old entries [gend[j-1], gbeg[j]) (0
// and n_cells at the ends), that moves by gdbeg[j]; the touched slots' own
// entries are left to the merge. A thread loads all its entries first (one
// memory latency; pairs of entries as 32-bit words), then walks the runs from
// mov_lo[c] with a cursor, its entries being in increasing order.
constexpr int kMoveWords = kChunk / 512;     // 32-bit words (two entries) per thread

__device__ void delta_move(uint32_t c, const uint16_t *__restrict__ cells, uint64_t n_cells,
                           const uint32_t *__restrict__ gbeg, const uint32_t *__restrict__ gend,
                           const uint32_t *__restrict__ gdbeg, const uint32_t *__restrict__ mov_lo,
                           uint16_t *__restrict__ out)
{
    const uint64_t i0 = uint64_t(c) * kChunk;      // even: words are 4-byte aligned
    const uint32_t *cw = reinterpret_cast<const uint32_t *>(cells + i0);
    uint32_t v[kMoveWords];
#pragma unroll
    for (int k = 0; k < kMoveWords; ++k) {
        const uint64_t i = i0 + 2 * (uint64_t(k) * 256 + threadIdx.x);
        v[k] = 0u;
        if (i + 1 < n_cells) v[k] = cw[uint64_t(k) * 256 + threadIdx.x];
        else if (i < n_cells) v[k] = cells[i];
    }
    uint32_t j = mov_lo[c];
    uint32_t e = gend[j], b = gbeg[j], sh = gdbeg[j];      // kEmpty32 past the last touched slot
#pragma unroll
    for (int k = 0; k < 2 * kMoveWords; ++k) {
        const uint64_t i = i0 + 2 * (uint64_t(k >> 1) * 256 + threadIdx.x) + (k & 1);
        if (i >= n_cells) break;
        while (i >= e) {                     // past touched slot j: the next run
            ++j;
            e = gend[j];
            b = gbeg[j];
            sh = gdbeg[j];
        }
        if (i < b) out[i + sh] = uint16_t(v[k >> 1] >> (16 * (k & 1)));
    }
}

// Steps 3 and 4 in one launch, their chunks interleaved in proportion so that
// both streams run side by side: block b is an offsets chunk when
// floor((b + 1) nc_off / nb) > floor(b nc_off / nb), its index then
// floor(b nc_off / nb); else a move chunk of index b - floor((b + 1) nc_off / nb).
__global__ void __launch_bounds__(256)
k_delta_stream(uint32_t nc_off, uint32_t nc_mov, const uint32_t *__restrict__ off, uint64_t nslot,
               const uint32_t *__restrict__ gslot, const uint32_t *__restrict__ gdbeg,
               const uint32_t *__restrict__ off_j, uint32_t *__restrict__ noff, const uint16_t *__restrict__ cells,
               uint64_t n_cells, const uint32_t *__restrict__ gbeg, const uint32_t *__restrict__ gend,
               const uint32_t *__restrict__ mov_lo, uint16_t *__restrict__ out)
{
    __shared__ uint32_t sgs[kStage], sgd[kStage];
    const uint64_t nb = uint64_t(nc_off) + nc_mov, b = blockIdx.x;
    const uint64_t before = b * nc_off / nb, upto = (b + 1) * nc_off / nb;
    if (upto > before)
        delta_offsets(uint32_t(before), sgs, sgd, off, nslot, gslot, gdbeg, off_j, noff);
    else
        delta_move(uint32_t(b - upto), cells, n_cells, gbeg, gend, gdbeg, mov_lo, out);
}

// Step 5, a warp per touched slot.
__global__ void __launch_bounds__(kWarps * 32)
k_delta_merge(const uint32_t *__restrict__ off, const uint16_t *__restrict__ cells, const uint32_t *__restrict__ gslot,
              const uint32_t *__restrict__ gdbeg, const uint16_t *__restrict__ gdcell,
              const uint32_t *__restrict__ Tpre, uint32_t L, uint32_t heavy_min, const uint32_t *__restrict__ hidx,
              uint32_t *__restrict__ hbm, uint32_t BRw, uint16_t *__restrict__ out, uint32_t *__restrict__ newh,
              uint32_t *__restrict__ n_newh)
{
    const int lane = threadIdx.x & 31;
    const uint32_t Tt = Tpre[L];
    const uint64_t gw = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t j = gw; j < Tt; j += nw) {
        const uint32_t s = gslot[j];
        const uint32_t o0 = off[s], na = off[s + 1] - o0;
        const uint32_t a0 = gdbeg[j], nb = gdbeg[j + 1] - a0;
        const uint32_t dst = o0 + a0;
        const uint16_t *old = cells + o0, *add = gdcell + a0;
        for (uint32_t i = lane; i < na; i += 32) {
            const uint32_t c = old[i];
            out[dst + i + rank_u16(add, nb, c)] = uint16_t(c);
        }
        for (uint32_t i = lane; i < nb; i += 32) {
            const uint32_t c = add[i];
            out[dst + i + rank_u16(old, na, c)] = uint16_t(c);
        }
        if (na + nb >= heavy_min) {
            if (na >= heavy_min) {
                uint32_t *bm = hbm + uint64_t(hidx[s]) * BRw;
                for (uint32_t i = lane; i < nb; i += 32) {
                    const uint32_t c = add[i];
                    atomicOr(&bm[c >> 5], 1u << (c & 31));
                }
            } else if (lane == 0) {
                newh[atomicAdd(n_newh, 1u)] = s;
            }
        }
    }
}

// Step 6, a warp per slot that became heavy: bitmap row first + i.
__global__ void __launch_bounds__(kWarps * 32)
k_delta_heavy_new(const uint32_t *__restrict__ noff, const uint16_t *__restrict__ ncells,
                  const uint32_t *__restrict__ newh, uint32_t nh, uint32_t first, uint32_t BRw,
                  uint32_t *__restrict__ hidx, uint32_t *__restrict__ hbm)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t i = gw; i < nh; i += nw) {
        const uint32_t s = newh[i];
        uint32_t *bm = hbm + (uint64_t(first) + i) * BRw;
        for (uint32_t w = lane; w < BRw; w += 32) bm[w] = 0u;
        __syncwarp();
        for (uint32_t t = noff[s] + lane; t < noff[s + 1]; t += 32) {
            const uint32_t c = ncells[t];
            atomicOr(&bm[c >> 5], 1u << (c & 31));
        }
        if (lane == 0) hidx[s] = first + uint32_t(i);
        __syncwarp();
    }
}

inline uint32_t pow2_ceil(uint32_t v)
{
    uint32_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

inline unsigned blocks_of(uint64_t items, uint64_t per)
{
    const uint64_t b = (items + per - 1) / per;
    return unsigned(b ? b : 1);
}

template <class KT, int E, class... Args>
int launch_table_e(uint32_t grid, uint32_t P2, cudaStream_t st, Args... args)
{
    const size_t smem = size_t(P2) * sizeof(KT) + 32 * 4;
    FL_TRY(ensure_dyn_smem((const void *)k_delta_table<KT, E>, smem));
    k_delta_table<KT, E><<<grid, kDeltaThreads, smem, st>>>(args...);
    return FLINNG_OK;
}

template <class KT, class... Args>
int launch_table(int E, uint32_t grid, uint32_t P2, cudaStream_t st, Args... args)
{
    switch (E) {
    case 8: return launch_table_e<KT, 8>(grid, P2, st, args...);
    case 4: return launch_table_e<KT, 4>(grid, P2, st, args...);
    case 2: return launch_table_e<KT, 2>(grid, P2, st, args...);
    default: return launch_table_e<KT, 1>(grid, P2, st, args...);
    }
}

}  // namespace

bool delta_insert_applies(const flinng_index *ix, uint64_t n)
{
    return ix->n_cells > 0 && n > 0 && n * ix->cfg.R <= kDeltaMaxKeys;
}

size_t delta_workspace_bytes(const flinng_index *ix, uint64_t n)
{
    const uint64_t L = ix->cfg.L, nR = n * ix->cfg.R, D = L * nR;
    return carve_bytes<uint16_t>(D) + carve_bytes<uint2>(D) + 4 * carve_bytes<uint32_t>(L + 1) +
           4 * carve_bytes<uint32_t>(D + 1) + carve_bytes<uint16_t>(D) + carve_bytes<uint32_t>(D + 1) +
           carve_bytes<uint32_t>(4) + scan_workspace_bytes(L + 1) +
           2 * carve_bytes<uint32_t>(std::max(ix->nslot + 1, ix->n_cells + n * L * ix->cfg.R) / kChunk + 3);
}

int insert_delta(flinng_index *ix, const uint32_t *buckets, uint64_t n, void *ws)
{
    const cudaStream_t st = ix->stream;
    const uint32_t R = ix->cfg.R, B = ix->cfg.B, L = ix->cfg.L, W = ix->cfg.range_bits;
    const uint64_t n_old = ix->n_points, nslot = ix->nslot, n_cells = ix->n_cells;
    const uint32_t nR = uint32_t(n * R);
    const uint64_t D = uint64_t(L) * nR;
    if (!delta_insert_applies(ix, n))
        return set_error(FLINNG_ERR_INVALID_ARG, "internal: delta insert of %llu points", (unsigned long long)n);
    Carver c(ws, ~size_t(0));
    uint16_t *rcell = c.take<uint16_t>(D);
    uint2 *rt = c.take<uint2>(D);
    uint32_t *A = c.take<uint32_t>(L + 1), *T = c.take<uint32_t>(L + 1);
    uint32_t *Apre = c.take<uint32_t>(L + 1), *Tpre = c.take<uint32_t>(L + 1);
    uint32_t *gslot = c.take<uint32_t>(D + 1), *gdbeg = c.take<uint32_t>(D + 1);
    uint32_t *gbeg = c.take<uint32_t>(D + 1), *gend = c.take<uint32_t>(D + 1);
    uint16_t *gdcell = c.take<uint16_t>(D);
    uint32_t *newh = c.take<uint32_t>(D + 1);
    const uint64_t nchunk = std::max(nslot + 1, n_cells) / kChunk + 2;
    uint32_t *off_j = c.take<uint32_t>(nchunk + 1), *mov_lo = c.take<uint32_t>(nchunk);
    uint32_t *cnt = c.take<uint32_t>(4);
    void *scan_ws = c.base + ((c.used + 255) & ~size_t(255));

    const uint32_t P2 = pow2_ceil(nR < 32 ? 32u : nR);
    uint32_t CB = 1;
    while ((1u << CB) < ix->BR) ++CB;
    const int E = P2 >= 8192 ? 8 : P2 >= 4096 ? 4 : P2 >= 2048 ? 2 : 1;
    if (W + CB <= 31)        // all-ones marks padding: real keys stay below it
        FL_TRY(launch_table<uint32_t>(E, L, P2, st, buckets, ix->gid, n_old, uint32_t(n), L, W, R, B, ix->rp, P2,
                                      CB, ix->off, ix->cells, rcell, rt, A, T));
    else
        FL_TRY(launch_table<uint64_t>(E, L, P2, st, buckets, ix->gid, n_old, uint32_t(n), L, W, R, B, ix->rp, P2,
                                      CB, ix->off, ix->cells, rcell, rt, A, T));
    count_launch();
    FL_CUDA(cudaGetLastError());
    FL_TRY(scan_exclusive(A, Apre, L, scan_ws, st));
    FL_TRY(scan_exclusive(T, Tpre, L, scan_ws, st));
    k_delta_flatten<<<L, 256, 0, st>>>(Apre, Tpre, L, W, nR, rcell, rt, ix->off, gslot, gdbeg, gbeg, gend, gdcell);
    count_launch();
    FL_CUDA(cudaGetLastError());
    uint32_t *noff = ix->slot_b;
    const unsigned nc_off = blocks_of(nslot + 1, kChunk), nc_mov = blocks_of(n_cells, kChunk);
    k_delta_chunks<<<blocks_of(uint64_t(nc_off > nc_mov ? nc_off : nc_mov) + 1, 256), 256, 0, st>>>(
        gslot, gend, Tpre, L, nslot, n_cells, nc_off, nc_mov, off_j, mov_lo);
    count_launch();
    FL_CUDA(cudaGetLastError());
    // the merge writes only the touched slots' new lists, the streaming passes
    // only the other lists and the offsets: the merge runs beside them
    FL_CUDA(cudaMemsetAsync(cnt, 0, 4 * sizeof(uint32_t), st));
    if (!ix->side) {
        FL_CUDA(cudaStreamCreateWithFlags(&ix->side, cudaStreamNonBlocking));
        FL_CUDA(cudaEventCreateWithFlags(&ix->ev_fork, cudaEventDisableTiming));
        FL_CUDA(cudaEventCreateWithFlags(&ix->ev_join, cudaEventDisableTiming));
    }
    FL_CUDA(cudaEventRecord(ix->ev_fork, st));
    FL_CUDA(cudaStreamWaitEvent(ix->side, ix->ev_fork, 0));
    k_delta_merge<<<152 * 16, kWarps * 32, 0, ix->side>>>(ix->off, ix->cells, gslot, gdbeg, gdcell, Tpre, L,
                                                         ix->heavy_min, ix->hidx, ix->hbm, ix->BRw, ix->cells_tmp,
                                                         newh, cnt);
    count_launch();
    FL_CUDA(cudaGetLastError());
    FL_CUDA(cudaEventRecord(ix->ev_join, ix->side));
    k_delta_stream<<<nc_off + nc_mov, 256, 0, st>>>(nc_off, nc_mov, ix->off, nslot, gslot, gdbeg, off_j, noff,
                                                     ix->cells, n_cells, gbeg, gend, mov_lo, ix->cells_tmp);
    count_launch();
    FL_CUDA(cudaGetLastError());
    FL_CUDA(cudaStreamWaitEvent(st, ix->ev_join, 0));
    // added cells and slots that became heavy
    FL_CUDA(cudaMemcpyAsync(ix->h_flag, Apre + L, 4, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaMemcpyAsync(ix->h_flag + 1, cnt, 4, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    const uint64_t added = ix->h_flag[0];
    const uint32_t nh_new = ix->h_flag[1];
    if (nh_new > 0) {
        const uint64_t words = (uint64_t(ix->n_heavy) + nh_new) * ix->BRw;
        if (words > ix->hbm_words) {
            // a larger bitmap array, the existing rows copied over (stream-ordered)
            const uint64_t want = words + words / 8 + ix->BRw;
            uint32_t *nb = nullptr;
            FL_CUDA(cudaMallocAsync(&nb, want * 4, st));
            if (ix->hbm && ix->n_heavy)
                FL_CUDA(cudaMemcpyAsync(nb, ix->hbm, uint64_t(ix->n_heavy) * ix->BRw * 4, cudaMemcpyDeviceToDevice,
                                        st));
            if (ix->hbm) {
                FL_CUDA(cudaFreeAsync(ix->hbm, st));
                ix->device_bytes -= ix->hbm_words * 4;
            }
            ix->hbm = nb;
            ix->hbm_words = want;
            ix->device_bytes += want * 4;
        }
        k_delta_heavy_new<<<blocks_of(nh_new, kWarps), kWarps * 32, 0, st>>>(noff, ix->cells_tmp, newh, nh_new,
                                                                             ix->n_heavy, ix->BRw, ix->hidx, ix->hbm);
        count_launch();
        FL_CUDA(cudaGetLastError());
    }
    std::swap(ix->off, ix->slot_b);
    std::swap(ix->cells, ix->cells_tmp);
    ix->n_cells = n_cells + added;
    ix->n_heavy += nh_new;
    ix->n_points = n_old + n;
    return FLINNG_OK;
}

}  // namespace flinng
