// Index construction (Alg. 1 and the reverse index of Sec. 5) in one pass
// over the new points' buckets.
//
// Group assignment (Alg. 1): position i of repetition r's random permutation
// holds point n_old + perm[r][i], whose group is (n_old + i) mod B.
//
// Member lists: the points of cell c = r*B + b, a counting sort of all points
// by cell (histogram, scan, scatter).
//
// Reverse index: every (point, table l) contributes the R cells r*B + gid_r to
// the list of slot (l, bucket). A counting sort on the slot - a one-digit
// radix sort whose digit is the whole (table, bucket) key - places old lists
// and new entries in one array; each slot is then sorted and deduplicated (a
// Bloom-filter bit is set once, Sec. 3.3) and the slots are compacted into
// the final CSR.
#include <algorithm>
#include <utility>

#include "internal.cuh"
#include "trace.h"

namespace flinng {

namespace {

constexpr int kWarpsPerBlock = 8;

inline unsigned warp_blocks(uint64_t items)
{
    uint64_t b = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (b > 152ull * 128) b = 152ull * 128;
    return (unsigned)(b ? b : 1);
}

inline unsigned thread_blocks(uint64_t items, int threads = 256)
{
    uint64_t b = (items + threads - 1) / threads;
    if (b > 152ull * 256) b = 152ull * 256;
    return (unsigned)(b ? b : 1);
}

__global__ void k_perm_check(const uint32_t *__restrict__ perm, uint32_t R, uint64_t n,
                             uint32_t *__restrict__ seen, uint32_t *__restrict__ flag)
{
    const uint64_t nw = (n + 31) / 32;
    const uint64_t total = uint64_t(R) * n;
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t r = t / n;
        const uint32_t x = perm[t];
        if (x >= n) {
            atomicOr(flag, 1u);
            continue;
        }
        const uint32_t bit = 1u << (x & 31);
        const uint32_t old = atomicOr(&seen[r * nw + x / 32], bit);
        if (old & bit) atomicOr(flag, 2u);
    }
}

__global__ void k_groups(const uint32_t *__restrict__ perm, uint32_t R, uint64_t n,
                         uint64_t n_old, uint32_t B, uint32_t rp, uint16_t *__restrict__ gid)
{
    const uint64_t total = uint64_t(R) * n;
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t r = t / n, i = t % n;
        const uint32_t x = perm[t];
        if (x < n) gid[(n_old + x) * rp + r] = uint16_t((n_old + i) % B);
    }
}

// Groups given outright (any non-adaptive design with one test per point and
// repetition, Sec. 3.1): row r of groups (R x n) holds the new points' groups
// in repetition r. Flag bit 8: a group id >= B (nothing is written then by
// the caller, which checks first).
__global__ void k_check_groups(const uint16_t *__restrict__ groups, uint64_t total, uint32_t B,
                               uint32_t *__restrict__ flag)
{
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += uint64_t(gridDim.x) * blockDim.x)
        if (groups[t] >= B) atomicOr(flag, 8u);
}

__global__ void k_groups_given(const uint16_t *__restrict__ groups, uint32_t R, uint64_t n,
                               uint64_t n_old, uint32_t rp, uint16_t *__restrict__ gid)
{
    const uint64_t total = uint64_t(R) * n;
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t r = t / n, i = t % n;
        gid[(n_old + i) * rp + r] = groups[t];
    }
}

__global__ void k_member_hist(const uint16_t *__restrict__ gid, uint64_t N, uint32_t R,
                              uint32_t B, uint32_t rp, uint32_t *__restrict__ cnt)
{
    const uint64_t total = N * R;
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t x = t / R;
        const uint32_t r = uint32_t(t % R);
        atomicAdd(&cnt[r * B + gid[x * rp + r]], 1u);
    }
}

__global__ void k_member_scatter(const uint16_t *__restrict__ gid, uint64_t N, uint32_t R,
                                 uint32_t B, uint32_t rp, uint32_t *__restrict__ cursor,
                                 uint32_t *__restrict__ mem)
{
    const uint64_t total = N * R;
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t x = t / R;
        const uint32_t r = uint32_t(t % R);
        const uint32_t pos = atomicAdd(&cursor[r * B + gid[x * rp + r]], 1u);
        mem[pos] = uint32_t(x);
    }
}

// Repetition-0 member records, in member-list order: word 0 = point id,
// words 1.. = group ids of repetitions 1..R-1, two per word (low half first).
__global__ void k_member_records(const uint32_t *__restrict__ mem, const uint16_t *__restrict__ gid,
                                 uint64_t N, uint32_t R, uint32_t rp, uint32_t rw,
                                 uint32_t *__restrict__ rec)
{
    for (uint64_t m = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; m < N;
         m += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t x = mem[m];
        const uint16_t *g = gid + uint64_t(x) * rp;
        rec[m * rw] = x;
        for (uint32_t w = 1; w < rw; ++w) {
            const uint32_t r = 2 * (w - 1) + 1;
            const uint32_t lo = r < R ? g[r] : 0u;
            const uint32_t hi = r + 1 < R ? g[r + 1] : 0u;
            rec[m * rw + w] = lo | (hi << 16);
        }
    }
}

// The (point, table) entries are taken table-major (t = l n + x): the threads
// in flight then touch the slots and lists of a few tables at a time, which
// stay in L2, instead of random slots of the whole index.
__global__ void k_slot_hist(const uint32_t *__restrict__ buckets, uint64_t n, uint32_t L,
                            uint32_t W, uint32_t R, uint32_t *__restrict__ hist)
{
    const uint64_t total = n * L;
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t l = uint32_t(t / n);
        const uint64_t x = t % n;
        atomicAdd(&hist[(uint64_t(l) << W) | buckets[x * L + l]], R);
    }
}

__global__ void k_slot_scatter_new(const uint32_t *__restrict__ buckets, const uint16_t *__restrict__ gid,
                                   uint64_t n_old, uint64_t n, uint32_t L, uint32_t W, uint32_t R,
                                   uint32_t B, uint32_t rp, uint32_t *__restrict__ cursor,
                                   uint16_t *__restrict__ tmp)
{
    const uint64_t total = n * L;
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t l = uint32_t(t / n);               // table-major, as k_slot_hist
        const uint64_t x = t % n;
        const uint32_t pos = atomicAdd(&cursor[(uint64_t(l) << W) | buckets[x * L + l]], R);
        const uint16_t *g = gid + (n_old + x) * rp;
        for (uint32_t r = 0; r < R; ++r) tmp[pos + r] = uint16_t(r * B + g[r]);
    }
}

__device__ __forceinline__ void cex(uint32_t &a, uint32_t &b)
{
    const uint32_t lo = min(a, b);
    b = max(a, b);
    a = lo;
}

// Append value to list for every lane that wants to, one atomic per warp.
// All 32 lanes must call it together.
__device__ __forceinline__ void warp_append(bool want, uint32_t value, uint32_t *__restrict__ list,
                                            uint32_t *__restrict__ count)
{
    const uint32_t m = __ballot_sync(0xffffffffu, want);
    if (!m) return;
    const int lane = threadIdx.x & 31, lead = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == lead) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, lead);
    if (want) list[base + __popc(m & ((1u << lane) - 1u))] = value;
}

// Thread per slot: the new cells of a slot holding at most kSmallSlot of them
// are sorted in registers by Batcher's odd-even merge network for sixteen
// inputs (its first nineteen comparators alone sort the first eight, which
// is all a slot of up to eight cells needs) and deduplicated in place (a
// Bloom-filter bit is set once, Sec. 3.3); ulen[s] = distinct cells. Larger
// slots go to a worklist. The loop runs warp-uniformly (the worklist append
// is warp-aggregated), so lanes past nslot idle in the last round.
constexpr uint32_t kSmallSlot = 16;

__global__ void k_slot_unique_small(const uint32_t *__restrict__ toff, uint64_t nslot, uint16_t *__restrict__ tmp,
                                    uint32_t *__restrict__ ulen, uint32_t *__restrict__ big,
                                    uint32_t *__restrict__ nbig)
{
    // kNet16: (i, j) compare-exchanges
    constexpr unsigned char kNet16[63][2] = {
        {0, 1}, {2, 3}, {0, 2}, {1, 3}, {1, 2}, {4, 5}, {6, 7}, {4, 6}, {5, 7}, {5, 6}, {0, 4}, {2, 6},
        {2, 4}, {1, 5}, {3, 7}, {3, 5}, {1, 2}, {3, 4}, {5, 6}, {8, 9}, {10, 11}, {8, 10}, {9, 11},
        {9, 10}, {12, 13}, {14, 15}, {12, 14}, {13, 15}, {13, 14}, {8, 12}, {10, 14}, {10, 12}, {9, 13},
        {11, 15}, {11, 13}, {9, 10}, {11, 12}, {13, 14}, {0, 8}, {4, 12}, {4, 8}, {2, 10}, {6, 14},
        {6, 10}, {2, 4}, {6, 8}, {10, 12}, {1, 9}, {5, 13}, {5, 9}, {3, 11}, {7, 15}, {7, 11}, {3, 5},
        {7, 9}, {11, 13}, {1, 2}, {3, 4}, {5, 6}, {7, 8}, {9, 10}, {11, 12}, {13, 14}};
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t s = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; s - lane < nslot; s += stride) {
        const bool valid = s < nslot;
        uint32_t beg = 0, len = 0;
        if (valid) {
            beg = toff[s];
            len = toff[s + 1] - beg;
        }
        warp_append(len > kSmallSlot, uint32_t(s), big, nbig);
        if (!valid || len > kSmallSlot) continue;
        if (len <= 1) {
            ulen[s] = len;
            continue;
        }
        uint32_t v[16];
#pragma unroll
        for (uint32_t i = 0; i < 16; ++i) v[i] = i < len ? uint32_t(tmp[beg + i]) : 0xFFFFFFFFu;
        if (len <= 8) {
#pragma unroll
            for (int c = 0; c < 19; ++c) cex(v[kNet16[c][0]], v[kNet16[c][1]]);
        } else {
#pragma unroll
            for (int c = 0; c < 63; ++c) cex(v[kNet16[c][0]], v[kNet16[c][1]]);
        }
        uint32_t cnt = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const bool keep = v[i] != 0xFFFFFFFFu && (i == 0 || v[i] != v[i > 0 ? i - 1 : 0]);
            if (keep) tmp[beg + cnt++] = uint16_t(v[i]);
        }
        ulen[s] = cnt;
    }
}

// Warp per worklist slot: sort and deduplicate in place. <= 32 cells: warp
// bitonic sort in registers; more: a bitmap over the B*R cells in shared
// memory, read back in cell order.
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_slot_unique_big(const uint32_t *__restrict__ toff, const uint32_t *__restrict__ big,
                  const uint32_t *__restrict__ nbig, uint32_t BR, uint16_t *__restrict__ tmp,
                  uint32_t *__restrict__ ulen)
{
    extern __shared__ uint32_t bm_all[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nwords = (BR + 31) / 32;
    uint32_t *bm = bm_all + warp * nwords;
    const uint32_t nb = *nbig;
    for (uint32_t i = blockIdx.x * kWarpsPerBlock + warp; i < nb; i += gridDim.x * kWarpsPerBlock) {
        const uint32_t s = big[i];
        const uint32_t beg = toff[s], len = toff[s + 1] - beg;
        if (len <= 32) {
            uint32_t v = lane < len ? uint32_t(tmp[beg + lane]) : 0xFFFFFFFFu;
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                for (int j = k >> 1; j > 0; j >>= 1) {
                    const uint32_t o = __shfl_xor_sync(0xffffffffu, v, j);
                    const bool up = ((lane & k) == 0);
                    const bool lower = ((lane & j) == 0);
                    v = (lower == up) ? min(v, o) : max(v, o);
                }
            }
            const uint32_t prev = __shfl_up_sync(0xffffffffu, v, 1);
            const bool keep = lane < (int)len && (lane == 0 || v != prev);
            const uint32_t m = __ballot_sync(0xffffffffu, keep);
            __syncwarp();
            if (keep) tmp[beg + __popc(m & ((1u << lane) - 1u))] = uint16_t(v);
            if (lane == 0) ulen[s] = __popc(m);
            __syncwarp();
            continue;
        }
        for (uint32_t w = lane; w < nwords; w += 32) bm[w] = 0u;
        __syncwarp();
        for (uint32_t t = lane; t < len; t += 32) {
            const uint32_t c = tmp[beg + t];
            atomicOr(&bm[c >> 5], 1u << (c & 31));
        }
        __syncwarp();
        uint32_t written = 0;
        for (uint32_t w0 = 0; w0 < nwords; w0 += 32) {
            const uint32_t w = w0 + lane;
            uint32_t bits = w < nwords ? bm[w] : 0u;
            const uint32_t cnt = __popc(bits);
            uint32_t incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            uint32_t pos = written + incl - cnt;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                tmp[beg + pos++] = uint16_t(w * 32 + b);
            }
            written += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) ulen[s] = written;
        __syncwarp();
    }
}

// Merge of each slot's old list (sorted, distinct) with its new cells (sorted,
// distinct, from k_slot_unique_*). A slot whose two lists together hold at
// most kThreadMerge cells is handled by one thread (two-pointer merge);
// larger ones go to a worklist for a warp. off == nullptr: no old lists.
constexpr uint32_t kThreadMerge = 64;

__global__ void k_merge_count(const uint32_t *__restrict__ off, const uint16_t *__restrict__ cells,
                              const uint32_t *__restrict__ dtoff, const uint32_t *__restrict__ dlen,
                              const uint16_t *__restrict__ dbuf, uint64_t nslot, uint32_t *__restrict__ mlen,
                              uint32_t *__restrict__ big, uint32_t *__restrict__ nbig)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t s = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; s - lane < nslot; s += stride) {
        const bool valid = s < nslot;
        uint32_t oa = 0, na = 0, db = 0, nb = 0;
        if (valid) {
            oa = off ? off[s] : 0u;
            na = off ? off[s + 1] - oa : 0u;
            db = dtoff[s];
            nb = dlen[s];
        }
        warp_append(na + nb > kThreadMerge, uint32_t(s), big, nbig);
        if (!valid) continue;
        if (na == 0 || nb == 0) {
            mlen[s] = na + nb;
            continue;
        }
        if (na + nb > kThreadMerge) continue;           // counted by the warp kernel
        uint32_t i = 0, j = 0, cnt = 0;
        uint32_t a = cells[oa], b = dbuf[db];
        while (i < na && j < nb) {
            ++cnt;
            if (a <= b) {
                if (a == b) {
                    ++j;
                    b = j < nb ? dbuf[db + j] : 0u;
                }
                ++i;
                a = i < na ? cells[oa + i] : 0u;
            } else {
                ++j;
                b = j < nb ? dbuf[db + j] : 0u;
            }
        }
        mlen[s] = cnt + (na - i) + (nb - j);
    }
}

// Thread per slot (at most kThreadMerge cells in its two lists): the merged,
// distinct, sorted list written at noff[s].
__global__ void k_merge_write(const uint32_t *__restrict__ off, const uint16_t *__restrict__ cells,
                              const uint32_t *__restrict__ dtoff, const uint32_t *__restrict__ dlen,
                              const uint16_t *__restrict__ dbuf, uint64_t nslot, const uint32_t *__restrict__ noff,
                              uint16_t *__restrict__ out)
{
    for (uint64_t s = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < nslot;
         s += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t oa = off ? off[s] : 0u, na = off ? off[s + 1] - oa : 0u;
        const uint32_t db = dtoff[s], nb = dlen[s];
        if (na + nb == 0 || na + nb > kThreadMerge) continue;
        uint32_t dst = noff[s];
        uint32_t i = 0, j = 0;
        while (i < na || j < nb) {
            const uint32_t a = i < na ? uint32_t(cells[oa + i]) : 0xFFFFFFFFu;
            const uint32_t b = j < nb ? uint32_t(dbuf[db + j]) : 0xFFFFFFFFu;
            const uint32_t m = min(a, b);
            i += (a == m) ? 1u : 0u;
            j += (b == m) ? 1u : 0u;
            out[dst++] = uint16_t(m);
        }
    }
}

// Warp per worklist slot: one list empty -> a coalesced copy of the other;
// else the union through a bitmap over the B*R cells in shared memory
// (count pass: mlen; write pass: the cells in order at noff[s]).
template <bool WRITE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_merge_big(const uint32_t *__restrict__ off, const uint16_t *__restrict__ cells, const uint32_t *__restrict__ dtoff,
            const uint32_t *__restrict__ dlen, const uint16_t *__restrict__ dbuf, const uint32_t *__restrict__ big,
            const uint32_t *__restrict__ nbig, uint32_t BR, uint32_t *__restrict__ mlen,
            const uint32_t *__restrict__ noff, uint16_t *__restrict__ out)
{
    extern __shared__ uint32_t bm_all[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nwords = (BR + 31) / 32;
    uint32_t *bm = bm_all + warp * nwords;
    const uint32_t nbg = *nbig;
    for (uint32_t i = blockIdx.x * kWarpsPerBlock + warp; i < nbg; i += gridDim.x * kWarpsPerBlock) {
        const uint32_t s = big[i];
        const uint32_t oa = off ? off[s] : 0u, na = off ? off[s + 1] - oa : 0u;
        const uint32_t db = dtoff[s], nb = dlen[s];
        if (na == 0 || nb == 0) {
            if (WRITE) {
                const uint16_t *src = na ? cells + oa : dbuf + db;
                const uint32_t len = na + nb, dst = noff[s];
                for (uint32_t t = lane; t < len; t += 32) out[dst + t] = src[t];
            }
            continue;
        }
        for (uint32_t w = lane; w < nwords; w += 32) bm[w] = 0u;
        __syncwarp();
        for (uint32_t t = lane; t < na; t += 32) {
            const uint32_t c = cells[oa + t];
            atomicOr(&bm[c >> 5], 1u << (c & 31));
        }
        for (uint32_t t = lane; t < nb; t += 32) {
            const uint32_t c = dbuf[db + t];
            atomicOr(&bm[c >> 5], 1u << (c & 31));
        }
        __syncwarp();
        uint32_t written = 0;
        const uint32_t dst = WRITE ? noff[s] : 0u;
        for (uint32_t w0 = 0; w0 < nwords; w0 += 32) {
            const uint32_t w = w0 + lane;
            uint32_t bits = w < nwords ? bm[w] : 0u;
            const uint32_t cnt = __popc(bits);
            uint32_t incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            if (WRITE) {
                uint32_t pos = dst + written + incl - cnt;
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    out[pos++] = uint16_t(w * 32 + b);
                }
            }
            written += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (!WRITE && lane == 0) mlen[s] = written;
        __syncwarp();
    }
}

// One pass over the slots, four per thread (16-byte accesses): hidx[s] = the
// bitmap row of heavy slot s (a list of at least heavy_min cells) or
// kEmpty32; the heavy slots appended to list (warp-aggregated; row order is
// the append order, which no result depends on), their number in *nh.
__global__ void k_heavy_collect(const uint32_t *__restrict__ off, uint64_t nslot, uint32_t heavy_min,
                                uint32_t *__restrict__ hidx, uint32_t *__restrict__ list, uint32_t *__restrict__ nh)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t nv = (nslot + 3) / 4;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t v = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; v - lane < nv; v += stride) {
        const uint64_t s0 = v * 4;
        uint32_t o[5] = {0u, 0u, 0u, 0u, 0u};
        if (v < nv) {
            if (s0 + 4 <= nslot) {
                const uint4 a = *reinterpret_cast<const uint4 *>(off + s0);
                o[0] = a.x;
                o[1] = a.y;
                o[2] = a.z;
                o[3] = a.w;
                o[4] = off[s0 + 4];
            } else {
                for (uint32_t t = 0; t < 5; ++t) o[t] = s0 + t <= nslot ? off[s0 + t] : 0u;
            }
        }
        uint32_t h[4];
#pragma unroll
        for (uint32_t t = 0; t < 4; ++t) {
            const bool heavy = v < nv && s0 + t < nslot && o[t + 1] - o[t] >= heavy_min;
            const uint32_t m = __ballot_sync(0xffffffffu, heavy);
            uint32_t base = 0;
            if (m) {
                const uint32_t lead = __ffs(m) - 1;
                if (lane == lead) base = atomicAdd(nh, __popc(m));
                base = __shfl_sync(0xffffffffu, base, lead);
            }
            h[t] = kEmpty32;
            if (heavy) {
                h[t] = base + __popc(m & ((1u << lane) - 1u));
                list[h[t]] = uint32_t(s0 + t);
            }
        }
        if (v < nv) {
            if (s0 + 4 <= nslot) {
                *reinterpret_cast<uint4 *>(hidx + s0) = make_uint4(h[0], h[1], h[2], h[3]);
            } else {
                for (uint32_t t = 0; t < 4; ++t)
                    if (s0 + t < nslot) hidx[s0 + t] = h[t];
            }
        }
    }
}

// Warp per heavy slot: its cell bitmap.
__global__ void k_heavy_fill(const uint32_t *__restrict__ off, const uint16_t *__restrict__ cells,
                             const uint32_t *__restrict__ list, uint32_t nh, uint32_t BRw,
                             uint32_t *__restrict__ hbm)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t i = gw; i < nh; i += nw) {
        const uint32_t s = list[i];
        uint32_t *bm = hbm + i * BRw;
        for (uint32_t w = lane; w < BRw; w += 32) bm[w] = 0u;
        __syncwarp();
        const uint32_t beg = off[s], end = off[s + 1];
        for (uint32_t t = beg + lane; t < end; t += 32) {
            const uint32_t c = cells[t];
            atomicOr(&bm[c >> 5], 1u << (c & 31));
        }
        __syncwarp();
    }
}

}  // namespace

// Cell bitmaps of the heavy slots (those whose list has >= heavy_min cells).
// Uses a word of the build scratch slot_a and a worklist of at least
// n_cells / heavy_min + 1 entries; grows the bitmap array if needed.
int build_heavy(flinng_index *ix, void *scan_ws, uint32_t *list)
{
    (void)scan_ws;
    const cudaStream_t st = ix->stream;
    const uint64_t nslot = ix->nslot;
    uint32_t *count = ix->slot_a;        // build scratch, free at this point
    FL_CUDA(cudaMemsetAsync(count, 0, sizeof(uint32_t), st));
    k_heavy_collect<<<thread_blocks((nslot + 3) / 4), 256, 0, st>>>(ix->off, nslot, ix->heavy_min, ix->hidx, list,
                                                                    count);
    count_launch();
    FL_CUDA(cudaGetLastError());
    FL_CUDA(cudaMemcpyAsync(ix->h_flag, count, 4, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    const uint32_t nh = *ix->h_flag;
    if (ix->BRw * 32 < ix->BR || ix->BRw == 0)
        return set_error(FLINNG_ERR_INVALID_ARG, "internal: cell bitmap width %u for B*R=%u", ix->BRw, ix->BR);
    const uint64_t words = uint64_t(nh) * ix->BRw;
    if (words > ix->hbm_words) {
        if (ix->hbm) {
            FL_CUDA(cudaFreeAsync(ix->hbm, st));     // stream-ordered, as the workspace
            ix->device_bytes -= ix->hbm_words * 4;
            ix->hbm = nullptr;
            ix->hbm_words = 0;
        }
        const uint64_t want = words + words / 8 + ix->BRw;
        FL_CUDA(cudaMallocAsync(&ix->hbm, want * 4, st));
        ix->hbm_words = want;
        ix->device_bytes += want * 4;
    }
    if (nh > 0 && (!ix->hbm || ix->hbm_words < words))
        return set_error(FLINNG_ERR_OOM, "internal: no storage for %u cell bitmaps", nh);
    if (nh > 0) {
        k_heavy_fill<<<warp_blocks(nh), kWarpsPerBlock * 32, 0, st>>>(ix->off, ix->cells, list, nh, ix->BRw,
                                                                     ix->hbm);
        count_launch();
        FL_CUDA(cudaGetLastError());
    }
    ix->n_heavy = nh;
    return FLINNG_OK;
}

size_t perm_check_workspace_bytes(uint32_t R, uint64_t n)
{
    return carve_bytes<uint32_t>(uint64_t(R) * ((n + 31) / 32) + 1);
}

int check_perm(flinng_index *ix, const uint32_t *perm, uint64_t n, void *ws)
{
    const cudaStream_t st = ix->stream;
    const uint32_t R = ix->cfg.R;
    if (n == 0) return FLINNG_OK;
    Carver c(ws, ~size_t(0));
    uint32_t *seen = c.take<uint32_t>(uint64_t(R) * ((n + 31) / 32) + 1);
    FL_CUDA(cudaMemsetAsync(seen, 0, uint64_t(R) * ((n + 31) / 32) * 4 + 4, st));
    k_perm_check<<<thread_blocks(uint64_t(R) * n), 256, 0, st>>>(perm, R, n, seen, ix->flag);
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}

namespace {

// Entries of the one worklist the reverse-index stage uses in turn: slots of
// more than kSmallSlot new cells, slots whose merge holds more than
// kThreadMerge cells, heavy slots.
uint64_t worklist_entries(const flinng_index *ix, uint64_t n, bool reset)
{
    const uint64_t D = n * ix->cfg.L * ix->cfg.R;
    const uint64_t old = reset ? 0 : ix->n_cells;
    uint64_t w = D / (kSmallSlot + 1);
    w = std::max<uint64_t>(w, (old + D) / (kThreadMerge + 1));
    w = std::max<uint64_t>(w, (old + D) / ix->heavy_min);
    return std::min<uint64_t>(w, ix->nslot) + 2;
}

}  // namespace

size_t insert_workspace_bytes(const flinng_index *ix, uint64_t n, bool reset)
{
    if (!reset && delta_insert_applies(ix, n))
        return carve_bytes<uint32_t>(ix->BR + 1) +
               std::max(delta_workspace_bytes(ix, n), scan_workspace_bytes(size_t(ix->BR) + 1)) + 256;
    const size_t ns = ix->nslot + 1;
    const size_t big = ns > size_t(ix->BR) + 1 ? ns : size_t(ix->BR) + 1;
    const uint64_t D = n * ix->cfg.L * ix->cfg.R;
    return 2 * carve_bytes<uint32_t>(ns) + carve_bytes<uint32_t>(ix->BR + 1) +
           carve_bytes<uint32_t>(worklist_entries(ix, n, reset)) + carve_bytes<uint32_t>(4) +
           (reset ? 0 : carve_bytes<uint16_t>(D)) + scan_workspace_bytes(big);
}

int check_groups(flinng_index *ix, const uint16_t *groups, uint64_t n)
{
    const cudaStream_t st = ix->stream;
    if (n == 0) return FLINNG_OK;
    k_check_groups<<<thread_blocks(uint64_t(ix->cfg.R) * n), 256, 0, st>>>(groups, uint64_t(ix->cfg.R) * n,
                                                                         ix->cfg.B, ix->flag);
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}

int check_result(flinng_index *ix)
{
    FL_CUDA(cudaMemcpyAsync(ix->h_flag, ix->flag, 4, cudaMemcpyDeviceToHost, ix->stream));
    FL_CUDA(cudaStreamSynchronize(ix->stream));
    const uint32_t f = *ix->h_flag;
    if (f & 1u) return set_error(FLINNG_ERR_INVALID_ARG, "perm: entry out of range [0, n)");
    if (f & 2u) return set_error(FLINNG_ERR_INVALID_ARG, "perm: a row repeats an index");
    if (f & 8u) return set_error(FLINNG_ERR_INVALID_ARG, "groups: a group id is >= B");
    if (f & 4u) return set_error(FLINNG_ERR_INVALID_ARG, "build_buckets: a bucket is >= 2^W");
    return FLINNG_OK;
}

namespace {

// Groups of the n new points (Alg. 1 from the permutations, or given
// outright) and the member lists and records of all cells.
int member_stage(flinng_index *ix, const uint32_t *perm, const uint16_t *groups, uint64_t n, uint32_t *mcur,
                 void *scan_ws)
{
    TraceRange trace_("groups and member lists");
    const cudaStream_t st = ix->stream;
    const uint32_t R = ix->cfg.R, B = ix->cfg.B, BR = ix->BR, rp = ix->rp;
    const uint64_t n_old = ix->n_points, N = n_old + n;
    if (n > 0) {
        if (groups)
            k_groups_given<<<thread_blocks(uint64_t(R) * n), 256, 0, st>>>(groups, R, n, n_old, rp, ix->gid);
        else
            k_groups<<<thread_blocks(uint64_t(R) * n), 256, 0, st>>>(perm, R, n, n_old, B, rp, ix->gid);
        count_launch();
        FL_CUDA(cudaGetLastError());
    }
    // member lists of all cells
    FL_CUDA(cudaMemsetAsync(ix->cell_cnt, 0, (BR + 1) * sizeof(uint32_t), st));
    if (N > 0) {
        k_member_hist<<<thread_blocks(N * R), 256, 0, st>>>(ix->gid, N, R, B, rp, ix->cell_cnt);
        count_launch();
        FL_CUDA(cudaGetLastError());
    }
    FL_TRY(scan_exclusive(ix->cell_cnt, ix->moff, BR, scan_ws, st));
    FL_CUDA(cudaMemcpyAsync(mcur, ix->moff, BR * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    if (N > 0) {
        k_member_scatter<<<thread_blocks(N * R), 256, 0, st>>>(ix->gid, N, R, B, rp, mcur, ix->mem);
        count_launch();
        FL_CUDA(cudaGetLastError());
        k_member_records<<<thread_blocks(N), 256, 0, st>>>(ix->mem, ix->gid, N, R, rp, ix->rw, ix->mrec);
        count_launch();
        FL_CUDA(cudaGetLastError());
    }
    return FLINNG_OK;
}

}  // namespace

int insert_hashed(flinng_index *ix, const uint32_t *buckets, const uint32_t *perm, const uint16_t *groups,
                  uint64_t n, void *ws)
{
    const cudaStream_t st = ix->stream;
    const uint32_t R = ix->cfg.R, B = ix->cfg.B, L = ix->cfg.L, W = ix->cfg.range_bits;
    const uint32_t BR = ix->BR, rp = ix->rp;
    const uint64_t n_old = ix->n_points, N = n_old + n, nslot = ix->nslot;
    const bool have_old = ix->n_cells > 0;
    const uint64_t D = n * L * R;   // new (table, cell) entries before deduplication
    const bool delta = delta_insert_applies(ix, n);
    Carver c(ws, ~size_t(0));
    uint32_t *mcur = c.take<uint32_t>(BR + 1);
    if (delta) {
        // a small batch: only the slots that gain cells are merged
        void *dws = c.base + ((c.used + 255) & ~size_t(255));
        FL_TRY(member_stage(ix, perm, groups, n, mcur, dws));
        TraceRange stage2("reverse index (delta)");
        return insert_delta(ix, buckets, n, dws);
    }
    uint32_t *dtoff = c.take<uint32_t>(nslot + 1);     // new entries of slot s start here
    uint32_t *cursor = c.take<uint32_t>(nslot + 1);    // scatter cursors, then merged lengths
    uint32_t *work = c.take<uint32_t>(worklist_entries(ix, n, !have_old));
    uint32_t *cnt = c.take<uint32_t>(4);
    // the new entries: in the build scratch for a build from scratch, in the
    // workspace for an insert (the scratch then receives the merged lists)
    uint16_t *dbuf = have_old ? c.take<uint16_t>(D) : ix->cells_tmp;
    void *scan_ws = c.base + ((c.used + 255) & ~size_t(255));

    FL_TRY(member_stage(ix, perm, groups, n, mcur, scan_ws));

    TraceRange stage2("reverse index");    // 1. the new entries by slot: counting sort (histogram, scan, scatter)
    uint32_t *hist = ix->slot_a;
    FL_CUDA(cudaMemsetAsync(hist, 0, (nslot + 1) * sizeof(uint32_t), st));
    FL_CUDA(cudaMemsetAsync(cnt, 0, 4 * sizeof(uint32_t), st));
    if (n > 0) {
        k_slot_hist<<<thread_blocks(n * L), 256, 0, st>>>(buckets, n, L, W, R, hist);
        count_launch();
        FL_CUDA(cudaGetLastError());
    }
    FL_TRY(scan_exclusive(hist, dtoff, nslot, scan_ws, st));
    if (n > 0) {
        FL_CUDA(cudaMemcpyAsync(cursor, dtoff, nslot * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        k_slot_scatter_new<<<thread_blocks(n * L), 256, 0, st>>>(buckets, ix->gid, n_old, n, L, W, R, B, rp, cursor,
                                                                 dbuf);
        count_launch();
        FL_CUDA(cudaGetLastError());
    }
    // 2. each slot's new cells sorted and deduplicated (dlen reuses the histogram)
    uint32_t *dlen = hist;
    const size_t smem = size_t(kWarpsPerBlock) * ((BR + 31) / 32) * sizeof(uint32_t);
    k_slot_unique_small<<<thread_blocks(nslot), 256, 0, st>>>(dtoff, nslot, dbuf, dlen, work, cnt + 0);
    count_launch();
    FL_CUDA(cudaGetLastError());
    FL_TRY(ensure_dyn_smem((const void *)k_slot_unique_big, smem));
    k_slot_unique_big<<<152 * 8, kWarpsPerBlock * 32, smem, st>>>(dtoff, work, cnt + 0, BR, dbuf, dlen);
    count_launch();
    FL_CUDA(cudaGetLastError());
    // 3. merged lengths |old u new| (cursor now holds them), new offsets by a scan
    const uint32_t *old_off = have_old ? ix->off : nullptr;
    uint32_t *mlen = cursor;
    k_merge_count<<<thread_blocks(nslot), 256, 0, st>>>(old_off, ix->cells, dtoff, dlen, dbuf, nslot, mlen, work,
                                                        cnt + 1);
    count_launch();
    FL_CUDA(cudaGetLastError());
    FL_TRY(ensure_dyn_smem((const void *)k_merge_big<false>, smem));
    FL_TRY(ensure_dyn_smem((const void *)k_merge_big<true>, smem));
    if (have_old) {
        k_merge_big<false><<<152 * 8, kWarpsPerBlock * 32, smem, st>>>(old_off, ix->cells, dtoff, dlen, dbuf, work,
                                                                       cnt + 1, BR, mlen, nullptr, nullptr);
        count_launch();
        FL_CUDA(cudaGetLastError());
    }
    uint32_t *noff = ix->slot_b;
    FL_TRY(scan_exclusive(mlen, noff, nslot, scan_ws, st));
    // 4. the merged lists written once, in slot order (an insert writes the
    //    build scratch, then the scratch and the list array trade places)
    uint16_t *out = have_old ? ix->cells_tmp : ix->cells;
    k_merge_write<<<thread_blocks(nslot), 256, 0, st>>>(old_off, ix->cells, dtoff, dlen, dbuf, nslot, noff, out);
    count_launch();
    FL_CUDA(cudaGetLastError());
    k_merge_big<true><<<152 * 8, kWarpsPerBlock * 32, smem, st>>>(old_off, ix->cells, dtoff, dlen, dbuf, work,
                                                                  cnt + 1, BR, nullptr, noff, out);
    count_launch();
    FL_CUDA(cudaGetLastError());
    std::swap(ix->off, ix->slot_b);
    if (have_old) std::swap(ix->cells, ix->cells_tmp);
    // the cell total arrives with the heavy-slot count (one wait, in build_heavy)
    FL_CUDA(cudaMemcpyAsync(ix->h_flag + 1, ix->off + nslot, 4, cudaMemcpyDeviceToHost, st));
    stage2.end();
    TraceRange stage3("heavy bitmaps");
    const int rc = build_heavy(ix, scan_ws, work);
    if (rc != FLINNG_OK) cudaStreamSynchronize(st);    // the lists are in place either way
    ix->n_cells = ix->h_flag[1];
    ix->n_points = N;
    return rc;
}

}  // namespace flinng
