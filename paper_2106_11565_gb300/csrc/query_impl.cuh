// Batched query: collision counts, group tests, AND-over-R decode and top-k
// (Sec. 5, Alg. 2 and Alg. 3). One CTA of 256 threads per query.
//
// Alg. 3 walks cells by count (descending, ties by cell id) and emits a point
// when the last of its R cells is reached. That order is the ascending order
// of the key (-score, lastcell, id) with score = the least count among the
// point's R cells and lastcell = the largest cell id among those cells with
// that count; points with score < t_min are never emitted. The kernel
// computes the k smallest keys without the per-point counter array:
//
//  1. counts: cnt[c] += 1 for every cell c in the query's list of each table,
//     in shared memory: bytes when L <= 255, 16-bit words up to L = 4095
//     (count width CW). Tables are taken NT at a time; their lists are
//     flattened over the whole CTA.
//  2. group tests at decreasing thresholds: the cells of repetition 0 are
//     bucketed by count; level t holds those with count exactly t.
//  3. decode: walk levels t = L, L-1, ..., t_min. A point of score >= t has
//     all R cells at count >= t, in particular its repetition-0 cell, so after
//     level t every point with score >= t has been seen. The members of a
//     level's cells are flattened over the CTA (coalesced member reads, no
//     per-cell imbalance); each member's key comes from its R group ids (the
//     AND over R). Stop once >= k points of score >= t were seen: no unseen
//     point can precede them.
//  4. top-k: candidates go to one shared buffer; when it would overflow, a
//     radix select over the keys (56 bits for CW = 1, 60 for CW = 2) keeps
//     the k best and tightens the admission cutoff. At the end a radix select
//     cuts the buffer to k keys, which a small bitonic sort orders.
//
// The kernels are templates on the count width; query.cu instantiates CW = 1
// and query_c16.cu CW = 2, each in its own translation unit.
#pragma once
#include "internal.cuh"

namespace flinng {

constexpr int kQTmax = 256;              // CTA size of the counts kernel
constexpr int kPlainUnroll = 4;          // plain kernel: loads in flight per thread
constexpr uint32_t kRankSelectMax = 256; // compactions of at most this many keys rank them directly

// key = (score_max - score) << 48 | lastcell << 32 | id
template <int CW> struct CountWidth;
template <> struct CountWidth<1> {
    static constexpr uint32_t kScoreMax = 255;
    static constexpr int kTopShift = 48;          // highest 8-bit radix digit
    static constexpr uint64_t kKeyBits = (1ull << 56) - 1;
};
template <> struct CountWidth<2> {
    static constexpr uint32_t kScoreMax = 4095;
    static constexpr int kTopShift = 56;
    static constexpr uint64_t kKeyBits = (1ull << 60) - 1;
};

struct QArgs {
    const uint32_t *qb;
    const uint16_t *cnt_in;   // per-cell counts given by the caller (nq x BR), or null: gather them
    uint32_t nq;
    const uint32_t *k;
    uint32_t k_max;
    const uint32_t *off;
    const uint16_t *cells;
    const uint32_t *moff;
    const uint32_t *mrec;     // repetition-0 member records (RW words each)
    const uint32_t *hidx;     // per slot: heavy bitmap index or kEmpty32
    const uint32_t *hbm;      // heavy slots' cell bitmaps, BRw words each
    uint32_t L, W, R, B, BR, BRw, t_min;
    uint32_t heavy_min; // a slot is heavy (has a cell bitmap) iff its list holds >= heavy_min cells
    uint32_t gcells;   // cells per level group of the decode (at least 1)
    uint32_t avg_cell; // members per repetition-0 cell, rounded up (host side, sizes gcells)
    uint32_t cap;      // candidate buffer entries (power of two)
    uint32_t kp;       // final sort width: power of two >= k_max
    uint32_t *out_ids;
    uint16_t *out_scores;
    const uint32_t *out_row;  // per query: its row of the outputs, or null (row = query index)
    uint16_t *out_counts;
};

struct QSmem {
    uint64_t *buf;       // cap candidate keys
    uint64_t *keep;      // kp keys (selection output, final sort)
    uint32_t *u;         // 8 scalars: nbuf, nkeep, digit, rank, whole, heavy tables, bound (u[6..7])
    uint32_t *lvl_n;     // nlev: repetition-0 cells per count
    uint32_t *lvl_cur;   // nlev
    uint32_t *rhist;     // 256: radix histogram
    uint32_t *c_pre;     // NT + 4: exclusive prefix of member (list) lengths; c_pre[NT] = ~0
    uint2 *c_rec;        // NT: per cell of a chunk {record base, cell | level << 16}
    uint32_t *c_start;   // NT: per table of a chunk, list base (gather; shares c_rec's space)
    uint32_t *g_hl;      // NT: bitmap indices of the heavy tables of a chunk of tables (the last
                         // NT words of buf: the gather runs before any candidate is kept)
    uint32_t *wsum;      // NT / 32: block-scan scratch
    uint32_t *cntw;      // count words: 4 byte counts (CW = 1) or 2 16-bit counts (CW = 2) each
    uint16_t *lvl_cells; // B
};

// count levels 0..L, rounded up to a multiple of 4
__host__ __device__ inline uint32_t q_nlev(uint32_t L) { return (L + 4) & ~3u; }
__host__ __device__ inline uint32_t q_count_words(uint32_t BR, int cw) { return cw == 1 ? (BR + 3) / 4 : (BR + 1) / 2; }

__host__ __device__ inline size_t qsmem_bytes(uint32_t cap, uint32_t kp, uint32_t BR, uint32_t B, int NT, uint32_t L,
                                              int cw)
{
    size_t b = size_t(cap) * 8 + size_t(kp) * 8 + 8 * 4 + 2 * size_t(q_nlev(L)) * 4 + 256 * 4 +
               (NT + 4) * 4 + 2 * NT * 4 + (NT / 32) * 4;
    b = (b + 15) & ~size_t(15);
    b += size_t(q_count_words(BR, cw)) * 4;
    b += size_t(B) * 2;
    return (b + 15) & ~size_t(15);
}

template <int NT, int CW>
__device__ inline QSmem carve_q(unsigned char *sm, uint32_t cap, uint32_t kp, uint32_t BR, uint32_t L)
{
    QSmem s;
    const uint32_t nlev = q_nlev(L);
    s.buf = (uint64_t *)sm;
    s.keep = s.buf + cap;
    s.u = (uint32_t *)(s.keep + kp);
    s.lvl_n = s.u + 8;
    s.lvl_cur = s.lvl_n + nlev;
    s.rhist = s.lvl_cur + nlev;
    s.c_pre = s.rhist + 256;
    s.c_rec = reinterpret_cast<uint2 *>(s.c_pre + NT + 4);   // 8-byte aligned: offsets are even
    s.c_start = reinterpret_cast<uint32_t *>(s.c_rec);
    s.g_hl = reinterpret_cast<uint32_t *>(s.buf + cap) - NT;   // needs 2 cap >= NT
    s.wsum = reinterpret_cast<uint32_t *>(s.c_rec + NT);
    size_t o = (size_t)((unsigned char *)(s.wsum + NT / 32) - sm);
    o = (o + 15) & ~size_t(15);
    s.cntw = (uint32_t *)(sm + o);
    s.lvl_cells = (uint16_t *)(s.cntw + q_count_words(BR, CW));
    return s;
}

template <int CW>
__device__ __forceinline__ uint32_t cnt_at(const QSmem &s, uint32_t c)
{
    if constexpr (CW == 1) return reinterpret_cast<const uint8_t *>(s.cntw)[c];
    else return reinterpret_cast<const uint16_t *>(s.cntw)[c];
}

namespace {

// Member record of repetition 0: word 0 = point id, words 1.. = the group
// ids of repetitions 1..R-1, two 16-bit ids per word.
template <int RW>
__device__ inline void load_record(const uint32_t *__restrict__ rec, uint32_t m, uint32_t w[RW])
{
    if constexpr (RW == 1) {
        w[0] = __ldg(rec + m);
    } else if constexpr (RW == 2) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(rec) + m);
        w[0] = v.x; w[1] = v.y;
    } else if constexpr (RW == 4) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(rec) + m);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(rec) + 2 * size_t(m));
        const uint4 u = __ldg(reinterpret_cast<const uint4 *>(rec) + 2 * size_t(m) + 1);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
        w[4] = u.x; w[5] = u.y; w[6] = u.z; w[7] = u.w;
    }
}

// Exclusive block scan of one value per thread; returns the prefix and
// writes the total to *total (all threads). Contains __syncthreads.
template <int NT>
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t *wsum, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        const uint32_t t = wsum[w];
        before += (w < warp) ? t : 0u;
        all += t;
    }
    __syncthreads();
    *total = all;
    return before + x - v;
}

// Largest i in [lo, n) with pre[i] <= j (pre ascending, pre[lo] <= j).
__device__ inline uint32_t find_seg(const uint32_t *pre, uint32_t n, uint32_t j, uint32_t lo = 0)
{
    uint32_t hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Radix select over keys[0..n): returns (prefix, mask) such that exactly kk
// keys satisfy (key & mask) <= prefix (keys are unique, kk <= n).
template <int NT, int CW>
__device__ void block_select(const uint64_t *keys, uint32_t n, uint32_t kk, const QSmem &s,
                             uint64_t &prefix_out, uint64_t &mask_out)
{
    const int tid = threadIdx.x, lane = tid & 31;
    uint64_t prefix = 0, mask = 0;
    uint32_t rem = kk;
    for (int shift = CountWidth<CW>::kTopShift; shift >= 0; shift -= 8) {
        for (int i = tid; i < 256; i += NT) s.rhist[i] = 0u;
        __syncthreads();
        // keys share their leading digits: aggregate per warp before the
        // shared-memory atomic (one per distinct digit per warp)
        for (uint32_t ib = tid & ~31u; ib < n; ib += NT) {
            const uint32_t i = ib + lane;
            bool in = false;
            uint32_t dg = 256;
            if (i < n) {
                const uint64_t v = keys[i];
                in = (v & mask) == prefix;
                dg = in ? uint32_t((v >> shift) & 0xFF) : 256u;
            }
            const uint32_t grp = __match_any_sync(0xffffffffu, dg);
            if (in && lane == __ffs(grp) - 1) atomicAdd(&s.rhist[dg], __popc(grp));
        }
        __syncthreads();
        if (tid < 32) {
            uint32_t h[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                h[j] = s.rhist[lane * 8 + j];
                sum += h[j];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            uint32_t run = incl - sum;
            if (run < rem && rem <= incl) {       // exactly one lane holds the digit
                uint32_t d = 0, hd = 0;
                bool found = false;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (!found) {
                        if (run + h[j] >= rem) {
                            d = lane * 8 + j;
                            hd = h[j];
                            found = true;
                        } else {
                            run += h[j];
                        }
                    }
                }
                s.u[2] = d;
                s.u[3] = rem - run;               // rank inside the digit's bucket
                s.u[4] = (hd == rem - run) ? 1u : 0u;   // the bucket is taken whole
            }
        }
        __syncthreads();
        const uint32_t d = s.u[2];
        rem = s.u[3];
        const bool whole = s.u[4] != 0;
        __syncthreads();
        prefix |= uint64_t(d) << shift;
        mask |= uint64_t(0xFF) << shift;
        if (whole) break;
    }
    prefix_out = prefix;
    mask_out = mask;
}

// Keep the kk best of buf[0..nbuf) in buf[0..kk); returns the new admission
// bound: the largest kept key (later keys above it can never enter the top kk).
template <int NT, int CW>
__device__ uint64_t block_compact(const QSmem &s, uint32_t nbuf, uint32_t kk)
{
    const int lane = threadIdx.x & 31;
    if (nbuf <= kRankSelectMax) {
        // few keys (the common case once the admission bound is tight): a
        // key's rank is its count of smaller keys (keys are distinct); the
        // kk lowest ranks land in order, and the bound is the last of them
        for (uint32_t i = threadIdx.x; i < nbuf; i += NT) {
            const uint64_t x = s.buf[i];
            uint32_t r = 0;
            for (uint32_t j = 0; j < nbuf; ++j) r += s.buf[j] < x ? 1u : 0u;
            if (r < kk) s.keep[r] = x;
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < kk; i += NT) s.buf[i] = s.keep[i];
        const uint64_t top = s.keep[kk - 1];
        if (threadIdx.x == 0) s.u[0] = kk;
        __syncthreads();
        return top;
    }
    uint64_t prefix, mask;
    block_select<NT, CW>(s.buf, nbuf, kk, s, prefix, mask);
    if (threadIdx.x == 0) s.u[1] = 0u;
    __syncthreads();
    for (uint32_t ib = threadIdx.x & ~31u; ib < nbuf; ib += NT) {
        const uint32_t i = ib + lane;
        const uint64_t v = i < nbuf ? s.buf[i] : kKeyNone;
        const bool take = i < nbuf && (v & mask) <= prefix;
        const uint32_t wm = __ballot_sync(0xffffffffu, take);
        if (wm) {
            uint32_t base = 0;
            if (lane == __ffs(wm) - 1) base = atomicAdd(&s.u[1], __popc(wm));
            base = __shfl_sync(0xffffffffu, base, __ffs(wm) - 1);
            if (take) s.keep[base + __popc(wm & ((1u << lane) - 1u))] = v;
        }
    }
    __syncthreads();
    uint64_t mx = 0;
    for (uint32_t i = threadIdx.x; i < kk; i += NT) {
        const uint64_t v = s.keep[i];
        s.buf[i] = v;
        mx = v > mx ? v : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t y = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    // u[6..7]: one 64-bit word (8-byte aligned: u follows the 64-bit keep array)
    if (threadIdx.x == 0) {
        s.u[0] = kk;
        s.u[6] = 0u;
        s.u[7] = 0u;
    }
    __syncthreads();
    if (lane == 0 && mx) {
        atomicMax(reinterpret_cast<unsigned long long *>(&s.u[6]), (unsigned long long)mx);
    }
    __syncthreads();
    const uint64_t bound = *reinterpret_cast<const unsigned long long *>(&s.u[6]);
    __syncthreads();
    return bound;
}

// Carry-save adder on 32 bit lanes: a + b + c = sum + 2 carry in every lane.
__device__ __forceinline__ void csa(uint32_t &carry, uint32_t &sum, uint32_t a, uint32_t b, uint32_t c)
{
    const uint32_t u = a ^ b;
    sum = u ^ c;
    carry = (a & b) | (u & c);
}

// Per-cell collision counts of one query (Sec. 5), NT tables at a time.
// Tables whose bucket is heavy contribute their cell bitmap: each thread owns
// one bitmap word position (32 cells) and sums it over the heavy tables in
// bit-sliced form, then adds the sums to its counter words without atomics. The
// other tables' lists are flattened over the CTA and counted with shared-memory
// atomics, U cell loads in flight per thread. Expects s.u[5] == 0 (the heavy
// table count, zeroed with the query state) and leaves it 0. Contains
// __syncthreads.
template <int NT, int CW, int U = 1>
__device__ void gather_counts(const QArgs &a, const QSmem &s, const uint32_t *qb)
{
    const int tid = threadIdx.x;
    const uint32_t nwords = q_count_words(a.BR, CW);
    for (uint32_t l0 = 0; l0 < a.L; l0 += NT) {
        const uint32_t l = l0 + tid;
        uint32_t beg = 0, len = 0;
        if (l < a.L) {
            const uint64_t slot = (uint64_t(l) << a.W) | qb[l];
            // the list's length decides whether the slot is heavy, so the
            // bitmap index (another random DRAM access) is read for heavy
            // slots only
            const uint32_t o0 = a.off[slot], o1 = a.off[slot + 1];
            if (o1 - o0 >= a.heavy_min) {
                s.g_hl[atomicAdd(&s.u[5], 1u)] = a.hidx[slot];
            } else {
                beg = o0;
                len = o1 - o0;
            }
        }
        if (tid == 0) s.c_pre[NT] = ~0u;   // ends every forward search of c_pre
        uint32_t total;
        const uint32_t pre = block_excl_scan<NT>(len, s.wsum, &total);
        s.c_start[tid] = beg - pre;   // entry e of the flattened lists sits at c_start + e
        s.c_pre[tid] = pre;
        __syncthreads();
        const uint32_t nh = s.u[5];
        if (nh > 0) {
            constexpr int kPer = CW == 1 ? 8 : 16;        // counter words per bitmap word
            constexpr uint32_t kCells = 32 / kPer;        // cells per counter word
            constexpr uint32_t kSub = 248;                // tables per pass: counts below 256, 8 bit planes
            for (uint32_t w = tid; w < a.BRw; w += NT) {
                for (uint32_t i1 = 0; i1 < nh; i1 += kSub) {
                    const uint32_t i2 = min(nh, i1 + kSub);
                    // bit-sliced counters of the word's 32 cells: pl[p] holds bit p
                    // of every cell's count. Eight bitmap words at a time (loaded
                    // together) go through a carry-save adder tree into planes 0..2;
                    // the weight-8 carry ripples into the planes above.
                    uint32_t pl[8];
#pragma unroll
                    for (int p = 0; p < 8; ++p) pl[p] = 0u;
                    for (uint32_t i0 = i1; i0 < i2; i0 += 8) {
                        uint32_t x[8];
#pragma unroll
                        for (int v = 0; v < 8; ++v)
                            x[v] = i0 + v < i2 ? __ldg(a.hbm + size_t(s.g_hl[i0 + v]) * a.BRw + w) : 0u;
                        uint32_t t0, t1, f0, f1, e;
                        csa(t0, pl[0], pl[0], x[0], x[1]);
                        csa(t1, pl[0], pl[0], x[2], x[3]);
                        csa(f0, pl[1], pl[1], t0, t1);
                        csa(t0, pl[0], pl[0], x[4], x[5]);
                        csa(t1, pl[0], pl[0], x[6], x[7]);
                        csa(f1, pl[1], pl[1], t0, t1);
                        csa(e, pl[2], pl[2], f0, f1);
#pragma unroll
                        for (int p = 3; p < 8; ++p) {
                            const uint32_t c = pl[p] & e;
                            pl[p] ^= e;
                            e = c;
                        }
                    }
                    // back to packed counters: bit p of cell i goes to bit p of its
                    // byte (CW = 1) or half word (CW = 2); a pass adds at most 247
                    const uint32_t np = 32u - __clz(i2 - i1);
#pragma unroll
                    for (int j = 0; j < kPer; ++j) {
                        uint32_t acc = 0u;
#pragma unroll
                        for (int p = 0; p < 8; ++p) {
                            if (uint32_t(p) >= np) break;
                            const uint32_t bits = (pl[p] >> (kCells * j)) & ((1u << kCells) - 1u);
                            if constexpr (CW == 1) acc += (bits * 0x00204081u & 0x01010101u) << p;
                            else acc += (bits * 0x8001u & 0x10001u) << p;
                        }
                        if (w * kPer + j < nwords) s.cntw[w * kPer + j] += acc;
                    }
                }
            }
            __syncthreads();
        }
        const uint32_t nl = min(uint32_t(NT), a.L - l0);
        // each warp counts a contiguous slice of the flattened lists, so a lane's
        // table index moves forward by at most a table per step (c_pre is total
        // past the last table and ~0 at NT, which ends the search)
        const uint32_t per = ((total + NT / 32 - 1) / (NT / 32) + 31) & ~31u;
        const uint32_t eb0 = min(uint32_t(tid >> 5) * per, total);
        const uint32_t ee = min(eb0 + per, total);
        uint32_t hint[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t e = eb0 + uint32_t(u) * 32 + (tid & 31);
            hint[u] = e < ee ? find_seg(s.c_pre, nl, e) : 0u;
        }
        for (uint32_t eb = eb0; eb < ee; eb += 32 * U) {
            uint32_t c[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t e = eb + uint32_t(u) * 32 + (tid & 31);
                c[u] = kEmpty32;
                if (e < ee) {
                    uint32_t t = hint[u];
                    for (int step = 0; s.c_pre[t + 1] <= e; ++step) {
                        if (step == 4) {
                            t = find_seg(s.c_pre, nl, e, t + 1);
                            break;
                        }
                        ++t;
                    }
                    hint[u] = t;
                    c[u] = a.cells[s.c_start[t] + e];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (c[u] == kEmpty32) continue;
                if constexpr (CW == 1) atomicAdd(&s.cntw[c[u] >> 2], 1u << ((c[u] & 3) * 8));
                else atomicAdd(&s.cntw[c[u] >> 1], 1u << ((c[u] & 1) * 16));
            }
        }
        // every thread read nh before the heavy section's barrier (or nh was 0)
        if (tid == 0) s.u[5] = 0u;
        __syncthreads();
    }
}

// Per-cell counts given by the caller (e.g. the sum of table shards' counts)
// packed into the shared counters; values above L (here the caller's total
// table count) are clamped to L. Contains __syncthreads.
template <int NT, int CW>
__device__ void load_counts(const QArgs &a, const QSmem &s, const uint16_t *cnt)
{
    constexpr uint32_t kPer = CW == 1 ? 4u : 2u;
    const uint32_t nwords = q_count_words(a.BR, CW);
    for (uint32_t i = threadIdx.x; i < nwords; i += NT) {
        uint32_t wv = 0;
#pragma unroll
        for (uint32_t j = 0; j < kPer; ++j) {
            const uint32_t c = i * kPer + j;
            const uint32_t v = c < a.BR ? min(uint32_t(cnt[c]), a.L) : 0u;
            wv |= v << (j * (CW == 1 ? 8u : 16u));
        }
        s.cntw[i] = wv;
    }
    __syncthreads();
}

template <int NT, int CW>
__device__ inline void zero_query_state(const QArgs &a, const QSmem &s)
{
    const int tid = threadIdx.x;
    const uint32_t nwords = q_count_words(a.BR, CW);
    for (uint32_t i = tid; i < nwords; i += NT) s.cntw[i] = 0u;
    const uint32_t nlev = q_nlev(a.L);
    for (uint32_t i = tid; i < nlev; i += NT) {
        s.lvl_n[i] = 0u;
    }
    if (tid < 8) s.u[tid] = 0u;
}

// Group tests, AND-over-R decode and top-k of query q, from the counts in
// shared memory; writes row q of the outputs.
template <int NT, int RW, int CW, int U = 1>
__device__ void decode_topk(const QArgs &a, const QSmem &s, uint32_t q, uint32_t kq)
{
    constexpr uint32_t kScoreMax = CountWidth<CW>::kScoreMax;
    uint16_t *lvl_cells = s.lvl_cells;
    const int tid = threadIdx.x, lane = tid & 31;
    if (kq > 0) {
        // group tests of repetition 0, bucketed by count level
        for (uint32_t b = tid; b < a.B; b += NT) {
            const uint32_t v = cnt_at<CW>(s, b);
            if (v >= a.t_min) atomicAdd(&s.lvl_n[v], 1u);
        }
        __syncthreads();
        if (tid < 32) {
            // start of each level in descending level order, by one warp: lane
            // i takes the i-th run of consecutive levels from L down to t_min
            const uint32_t nl = a.L - a.t_min + 1;
            const uint32_t per = (nl + 31) / 32;
            uint32_t local = 0;
            for (uint32_t i = 0; i < per; ++i) {
                const uint32_t pos = uint32_t(lane) * per + i;
                if (pos < nl) local += s.lvl_n[a.L - pos];
            }
            uint32_t incl = local;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            uint32_t run = incl - local;
            for (uint32_t i = 0; i < per; ++i) {
                const uint32_t pos = uint32_t(lane) * per + i;
                if (pos < nl) {
                    s.lvl_cur[a.L - pos] = run;
                    run += s.lvl_n[a.L - pos];
                }
            }
        }
        __syncthreads();
        for (uint32_t b = tid; b < a.B; b += NT) {
            const uint32_t v = cnt_at<CW>(s, b);
            if (v >= a.t_min) lvl_cells[atomicAdd(&s.lvl_cur[v], 1u)] = uint16_t(b);
        }
        __syncthreads();
        // decode, level by level. After level t every point of score >= t has
        // been seen (its repetition-0 cell has count >= t), so the walk stops
        // once the kq-th best candidate scores >= t: no later point can enter.
        uint64_t bound = CountWidth<CW>::kKeyBits;   // admission: key <= bound
        uint32_t bscore = 0;                 // the bound's score: lower scores cannot enter
        bool have_k = false;                 // kq candidates held at the last check
        uint32_t kth_score = 0;              // score of the kq-th best candidate then
        // Levels are taken in groups: level t and the levels below it while the
        // group holds at most a.gcells cells (about 4,096 members). A group's
        // cells are contiguous in lvl_cells (levels descending).
        // After the placement above, lvl_cur[v] is the number of cells at levels
        // >= v (non-increasing in v), so a group's extent is a binary search,
        // not a walk over the (mostly empty) levels.
        int t = int(a.L);
        while (t >= int(a.t_min)) {
            const uint32_t first = s.lvl_cur[t] - s.lvl_n[t];   // cells at levels above t
            const uint32_t lim = first + a.gcells;
            int t_end = t;
            if (s.lvl_cur[t] <= lim) {
                // the lowest t_end in [t_min, t] whose levels [t_end, t] hold <= gcells cells
                int lo = int(a.t_min), hi = t;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (s.lvl_cur[mid] <= lim) hi = mid;
                    else lo = mid + 1;
                }
                t_end = lo;
            }
            const uint32_t nc = s.lvl_cur[t_end] - first;
            for (uint32_t c0 = 0; c0 < nc; c0 += NT) {
                const uint32_t ci = c0 + tid;
                uint32_t ms = 0, sz = 0, b = 0, lev = 0;
                if (ci < nc) {
                    b = lvl_cells[first + ci];
                    lev = cnt_at<CW>(s, b);
                    // a member's score is at most its repetition-0 cell's level:
                    // members of cells below the bound's score cannot enter
                    if (lev >= bscore) {
                        ms = a.moff[b];
                        sz = a.moff[b + 1] - ms;
                    }
                }
                if (tid == 0) s.c_pre[NT] = ~0u;   // ends every forward search of c_pre
                uint32_t M;
                const uint32_t pre = block_excl_scan<NT>(sz, s.wsum, &M);
                s.c_pre[tid] = pre;
                // member j of this cell: record c_rec.x + j; the cell and its count (its level)
                s.c_rec[tid] = make_uint2(ms - pre, b | (lev << 16));
                const uint32_t ncc = min(uint32_t(NT), nc - c0);
                __syncthreads();
                // Each warp walks its own contiguous slice of the member indices,
                // 32 U at a time, so a lane's cell index moves forward by a cell or
                // less per step (cells hold tens to hundreds of members).
                const uint32_t per = ((M + NT / 32 - 1) / (NT / 32) + 31) & ~31u;
                uint32_t jb = min(uint32_t(tid >> 5) * per, M);   // this warp's cursor (warp-uniform)
                const uint32_t je = min(jb + per, M);
                // the cell holding member jb (warp-uniform; the largest such index
                // is never an empty cell)
                uint32_t cur = jb < je ? find_seg(s.c_pre, ncc, jb) : 0u;
                // Members are decoded without per-round reservations: a warp about
                // to append reads the buffer fill first and appends only while it
                // is at or below hwm. Above it the warp pauses; once every warp has
                // paused or finished, the block compacts and the warps resume from
                // their own cursors. Once the fill passes hwm every warp appends at
                // most once more (the step it read the fill in, 32 U keys), so the
                // buffer cannot overflow: hwm = cap - (NT + 32) U.
                const uint32_t hwm = a.cap - uint32_t(NT + 32) * U;
                for (;;) {
                    const uint32_t smin = max(a.t_min, bscore);   // lower scores cannot enter
                    while (jb < je) {
                        // lanes to cells: one warp-uniform pass over the cell
                        // boundaries inside this step (a cell or two for 32 members);
                        // c_pre is M at the chunk's end and ~0 at NT, so the pass
                        // stops at the step's last member
                        const uint32_t last_j = min(jb + 32u * U, je) - 1u;
                        uint32_t my[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) my[u] = cur;
                        uint32_t k = cur + 1, bnd = s.c_pre[k];
                        while (bnd <= last_j) {
#pragma unroll
                            for (int u = 0; u < U; ++u)
                                if (jb + uint32_t(u) * 32 + lane >= bnd) my[u] = k;
                            bnd = s.c_pre[++k];
                        }
                        uint32_t w[U][RW];
                        uint32_t cell[U];
                        bool in[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const uint32_t j = jb + uint32_t(u) * 32 + lane;
                            in[u] = j < je;
                            cell[u] = 0;
                            if (in[u]) {
                                const uint2 cr = s.c_rec[my[u]];
                                cell[u] = cr.y;
                                load_record<RW>(a.mrec, cr.x + j, w[u]);
                            }
                        }
                        uint64_t key[U];
                        uint32_t wm[U], any = 0u;
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            bool want = false;
                            key[u] = 0;
                            if (in[u]) {
                                // repetition 0: the cell itself, at its level
                                uint32_t score = cell[u] >> 16, last = cell[u] & 0xFFFFu;
#pragma unroll
                                for (int r = 1; r < 2 * RW - 1; ++r) {
                                    if (r >= int(a.R)) break;
                                    const uint32_t g = (w[u][1 + (r - 1) / 2] >> (16 * ((r - 1) & 1))) & 0xFFFFu;
                                    const uint32_t c = uint32_t(r) * a.B + g;
                                    const uint32_t v = cnt_at<CW>(s, c);
                                    if (v <= score) {
                                        last = c;
                                        score = v;
                                    }
                                }
                                if (score >= smin) {
                                    key[u] = (uint64_t(kScoreMax - score) << 48) | (uint64_t(last) << 32) | w[u][0];
                                    want = key[u] <= bound;
                                }
                            }
                            wm[u] = __ballot_sync(0xffffffffu, want);
                            any |= wm[u];
                        }
                        if (any) {
                            // the fill, read once per warp (lane 0) so the decision is
                            // warp-uniform; above hwm the warp pauses and redoes this
                            // step after the compaction
                            uint32_t fill = lane == 0 ? *reinterpret_cast<volatile uint32_t *>(&s.u[0]) : 0u;
                            fill = __shfl_sync(0xffffffffu, fill, 0);
                            if (fill > hwm) break;
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                if (!wm[u]) continue;
                                uint32_t base = 0;
                                if (lane == __ffs(wm[u]) - 1) base = atomicAdd(&s.u[0], __popc(wm[u]));
                                base = __shfl_sync(0xffffffffu, base, __ffs(wm[u]) - 1);
                                if ((wm[u] >> lane) & 1u) s.buf[base + __popc(wm[u] & ((1u << lane) - 1u))] = key[u];
                            }
                        }
                        jb += 32 * U;
                        cur = k - 1;   // the cell holding member last_j
                    }
                    __syncthreads();
                    const uint32_t nb0 = s.u[0];   // same value in every thread (read after the barrier)
                    if (nb0 <= hwm) break;          // no warp paused: every cursor is at its end
                    bound = block_compact<NT, CW>(s, nb0, kq);
                    bscore = kScoreMax - uint32_t(bound >> 48);
                }
            }
            if (nc > 0) {
                // the buffer fill is final after the last round's barrier; the
                // compaction's own barriers order its writes after every read
                const uint32_t nb = s.u[0];
                if (nb >= kq) {
                    bound = block_compact<NT, CW>(s, nb, kq);
                    kth_score = kScoreMax - uint32_t(bound >> 48);
                    bscore = kth_score;
                    have_k = true;
                }
            }
            // every level >= t_end is complete: points of score >= t_end are all seen
            if (have_k && kth_score >= uint32_t(t_end)) break;
            t = t_end - 1;
        }
    }
    __syncthreads();
    // final top-k: cut to kq keys, order them, write
    const uint32_t nbuf = s.u[0];
    const uint32_t nk = nbuf < kq ? nbuf : kq;
    if (nbuf > kq) block_compact<NT, CW>(s, nbuf, kq);
    if (nk <= 256) {
        // rank sort: the keys are distinct, so a key's rank is the number of
        // smaller keys; one barrier instead of a sorting network
        for (uint32_t i = tid; i < nk; i += NT) {
            const uint64_t x = s.buf[i];
            uint32_t r = 0;
            for (uint32_t j = 0; j < nk; ++j) r += s.buf[j] < x ? 1u : 0u;
            s.keep[r] = x;
        }
        __syncthreads();
    } else {
        for (uint32_t i = tid; i < a.kp; i += NT) s.keep[i] = (i < nk) ? s.buf[i] : kKeyNone;
        __syncthreads();
        for (uint32_t k2 = 2; k2 <= a.kp; k2 <<= 1) {
            for (uint32_t j = k2 >> 1; j > 0; j >>= 1) {
                for (uint32_t i = tid; i < a.kp; i += NT) {
                    const uint32_t l = i ^ j;
                    if (l > i) {
                        const uint64_t x = s.keep[i], y = s.keep[l];
                        const bool up = (i & k2) == 0;
                        if ((x > y) == up) {
                            s.keep[i] = y;
                            s.keep[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
    }
    const size_t row = a.out_row ? size_t(a.out_row[q]) : size_t(q);
    for (uint32_t i = tid; i < a.k_max; i += NT) {
        const uint64_t key = (i < nk) ? s.keep[i] : kKeyNone;
        const bool ok = key != kKeyNone;
        a.out_ids[row * a.k_max + i] = ok ? uint32_t(key & 0xFFFFFFFFu) : 0xFFFFFFFFu;
        if (a.out_scores)
            a.out_scores[row * a.k_max + i] = ok ? uint16_t(kScoreMax - uint32_t(key >> 48)) : uint16_t(0);
    }
    __syncthreads();
}

template <int NT, int RW, int CW>
__global__ void __launch_bounds__(NT, 1024 / NT)
k_query(QArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const QSmem s = carve_q<NT, CW>(sm, a.cap, a.kp, a.BR, a.L);
    for (uint32_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
        uint32_t kq = a.k ? a.k[q] : a.k_max;
        if (kq > a.k_max) kq = a.k_max;
        zero_query_state<NT, CW>(a, s);
        __syncthreads();
        if (kq > 0) {
            if (a.cnt_in) load_counts<NT, CW>(a, s, a.cnt_in + size_t(q) * a.BR);
            else gather_counts<NT, CW, kPlainUnroll>(a, s, a.qb + size_t(q) * a.L);
        }
        decode_topk<NT, RW, CW, kPlainUnroll>(a, s, q, kq);
    }
}

// ---------------------------------------------------------------- fused form
//
// One launch for the whole batch: each CTA hashes its query in shared memory
// (DOPH over the query's set, or the L*K sign projections of its vector),
// then runs the same gather / decode / top-k. The grid is persistent: CTAs
// loop over queries. The hashing follows the same definitions as the hash
// kernels (hash.cu), the bucket results are identical.

struct HArgs {
    // Jaccard
    const uint64_t *q_off;
    const uint32_t *q_el;
    uint32_t nb, da, db;
    uint64_t seed;
    const uint64_t *ba;
    const uint64_t *bc;
    // cosine
    const float *x;
    uint64_t ldx;
    const float *w;
    uint32_t d;
    float gamma2, tiny;
    double gamma64;
    unsigned long long *stats;
    uint32_t *qnext;    // next query to hand out (zeroed before each launch)
    uint32_t K;
    size_t hash_off;    // byte offset of the hash region in shared memory (0: inside the
                        // candidate buffer, which is free until the decode)
};

__device__ __forceinline__ uint64_t splitmix64_q(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// DOPH of query q into qb[0..L) (shared memory). Contains __syncthreads.
template <int NT>
__device__ void cta_doph(const QArgs &a, const HArgs &h, uint32_t q, uint32_t *qb, uint32_t *val)
{
    const int tid = threadIdx.x;
    const uint32_t nb = h.nb;
    uint32_t *occ = val + nb;
    for (uint32_t k = tid; k < nb; k += NT) val[k] = kEmpty32;
    for (uint32_t k = tid; k < (nb + 31) / 32; k += NT) occ[k] = 0u;
    __syncthreads();
    const uint64_t beg = h.q_off[q], end = h.q_off[q + 1];
    for (uint64_t t = beg + tid; t < end; t += NT) {
        const uint32_t pe = h.da * __ldg(h.q_el + t) + h.db;
        const uint32_t bin = __umulhi(pe, nb);
        atomicMin(&val[bin], pe);
        atomicOr(&occ[bin >> 5], 1u << (bin & 31));
    }
    __syncthreads();
    if (end > beg) {
        const bool pow2 = (nb & (nb - 1u)) == 0u;     // z mod nb is a mask then
        for (uint32_t k = tid; k < nb; k += NT) {
            if ((occ[k >> 5] >> (k & 31)) & 1u) continue;
            bool found = false;
            for (uint32_t att = 1; att <= kDophMaxAttempts; ++att) {
                const uint64_t z = splitmix64_q(h.seed ^ ((uint64_t(k) << 32) | att));
                const uint32_t j = pow2 ? uint32_t(z) & (nb - 1u) : uint32_t(z % nb);
                if ((occ[j >> 5] >> (j & 31)) & 1u) {
                    val[k] = val[j];
                    found = true;
                    break;
                }
            }
            if (!found) {
                for (uint32_t s2 = 1; s2 <= nb; ++s2) {
                    const uint32_t j = (k + s2) % nb;
                    if ((occ[j >> 5] >> (j & 31)) & 1u) {
                        val[k] = val[j];
                        break;
                    }
                }
            }
        }
    }
    __syncthreads();
    for (uint32_t l = tid; l < a.L; l += NT) {
        uint64_t hh = h.bc[l];
        for (uint32_t j = 0; j < h.K; ++j) hh += h.ba[l * h.K + j] * uint64_t(val[l * h.K + j]);
        qb[l] = uint32_t(hh >> (64 - a.W));
    }
    __syncthreads();
}

// Exact sign of sum_t a_t b_t for fp32 inputs, by one warp: fixed-point
// digits of 32 bits from 2^-384 upward, summed over lanes in int64.
__device__ int warp_exact_sign(const float *xa, const float *wb, uint32_t d, int lane)
{
    constexpr int kLimbs = 24;
    long long acc[kLimbs + 2];
    for (int i = 0; i < kLimbs + 2; ++i) acc[i] = 0;
    for (uint32_t t = lane; t < d; t += 32) {
        const double v = double(xa[t]) * double(wb[t]);
        const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
        const int ex = int((bits >> 52) & 0x7FF);
        unsigned long long man = bits & ((1ull << 52) - 1);
        if (ex == 0 && man == 0) continue;
        int lsb;
        if (ex == 0) {
            lsb = 1 - 1075;
        } else {
            man |= 1ull << 52;
            lsb = ex - 1075;
        }
        const int pos = lsb + 384;
        const int qd = pos >> 5, r = pos & 31;
        const unsigned long long d0 = (man << r) & 0xffffffffull;
        const unsigned long long d1 = (r == 0 ? (man >> 32) : (man >> (32 - r))) & 0xffffffffull;
        const unsigned long long d2 = (r == 0) ? 0ull : (man >> (64 - r));
        const long long sg = (bits >> 63) ? -1 : 1;
        acc[qd] += sg * (long long)d0;
        acc[qd + 1] += sg * (long long)d1;
        acc[qd + 2] += sg * (long long)d2;
    }
    for (int i = 0; i < kLimbs + 2; ++i) {
        long long v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[i] = v;
    }
    acc[kLimbs - 1] += acc[kLimbs] * 4294967296ll;
    for (int i = 0; i < kLimbs - 1; ++i) {
        const long long c = acc[i] >> 32;
        acc[i] -= c * 4294967296ll;
        acc[i + 1] += c;
    }
    if (acc[kLimbs - 1] != 0) return acc[kLimbs - 1] > 0 ? 1 : -1;
    for (int i = kLimbs - 2; i >= 0; --i)
        if (acc[i] != 0) return 1;
    return 0;
}

// SRP codes of query q into qb[0..L): one warp per projection, fp32 with a
// rigorous error bound, fp64 re-check, exact accumulator last. Contains
// __syncthreads.
template <int NT>
__device__ void cta_srp(const QArgs &a, const HArgs &h, uint32_t q, uint32_t *qb, float *xs)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float *xq = h.x + size_t(q) * h.ldx;
    for (uint32_t t = tid; t < h.d; t += NT) xs[t] = xq[t];
    for (uint32_t l = tid; l < a.L; l += NT) qb[l] = 0u;
    __syncthreads();
    const uint32_t P = a.L * h.K;
    for (uint32_t j = warp; j < P; j += (NT / 32)) {
        const float *wj = h.w + size_t(j) * h.d;
        float p = 0.f, sa = 0.f;
        for (uint32_t t = lane; t < h.d; t += 32) {
            const float wv = __ldg(wj + t), xv = xs[t];
            p = fmaf(wv, xv, p);
            sa = fmaf(fabsf(wv), fabsf(xv), sa);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            p += __shfl_xor_sync(0xffffffffu, p, o);
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
        }
        p = __shfl_sync(0xffffffffu, p, 0);
        sa = __shfl_sync(0xffffffffu, sa, 0);
        bool positive;
        if (fabsf(p) > fmaf(h.gamma2, sa, h.tiny)) {
            positive = p > 0.f;
        } else {
            double p64 = 0.0, s64 = 0.0;
            for (uint32_t t = lane; t < h.d; t += 32) {
                const double prod = double(wj[t]) * double(xs[t]);
                p64 += prod;
                s64 += fabs(prod);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                p64 += __shfl_xor_sync(0xffffffffu, p64, o);
                s64 += __shfl_xor_sync(0xffffffffu, s64, o);
            }
            p64 = __shfl_sync(0xffffffffu, p64, 0);
            s64 = __shfl_sync(0xffffffffu, s64, 0);
            if (fabs(p64) > h.gamma64 * s64) {
                positive = p64 > 0.0;
            } else {
                positive = warp_exact_sign(xs, wj, h.d, lane) > 0;
                if (lane == 0) atomicAdd(&h.stats[1], 1ull);
            }
            if (lane == 0) {
                atomicAdd(&h.stats[0], 1ull);
                atomicAdd(&h.stats[2], 1ull);
                if (positive != (p > 0.f)) atomicAdd(&h.stats[4], 1ull);
            }
        }
        if (lane == 0 && positive) atomicOr(&qb[j / h.K], 1u << (j % h.K));
    }
    __syncthreads();
}

template <int NT, int RW, int HASH, int CW>
__global__ void __launch_bounds__(NT, (HASH == 2 ? 1024 : 2048) / NT)
k_query_fused(QArgs a, HArgs h)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const QSmem s = carve_q<NT, CW>(sm, a.cap, a.kp, a.BR, a.L);
    uint32_t *qb = reinterpret_cast<uint32_t *>(sm + h.hash_off);
    uint32_t *qslot = qb + ((a.L + 3) & ~3u);
    uint32_t *hs = qslot + 4;
    // queries are handed out one at a time from a counter (zeroed before the
    // launch), so CTAs that drew cheap queries take more of them
    for (;;) {
        if (threadIdx.x == 0) qslot[0] = atomicAdd(h.qnext, 1u);
        __syncthreads();
        const uint32_t q = qslot[0];
        if (q >= a.nq) break;
        uint32_t kq = a.k ? a.k[q] : a.k_max;
        if (kq > a.k_max) kq = a.k_max;
        zero_query_state<NT, CW>(a, s);
        if (kq > 0) {
            if constexpr (HASH == 1) cta_doph<NT>(a, h, q, qb, hs);
            else cta_srp<NT>(a, h, q, qb, reinterpret_cast<float *>(hs));
            gather_counts<NT, CW>(a, s, qb);
        } else {
            __syncthreads();
        }
        decode_topk<NT, RW, CW>(a, s, q, kq);
    }
}

template <int CW>
__global__ void __launch_bounds__(kQTmax)
k_counts(QArgs a)
{
    constexpr int NT = kQTmax;
    extern __shared__ __align__(16) unsigned char sm[];
    const QSmem s = carve_q<NT, CW>(sm, a.cap, a.kp, a.BR, a.L);
    const int tid = threadIdx.x;
    const uint32_t nwords = q_count_words(a.BR, CW);
    for (uint32_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
        for (uint32_t i = tid; i < nwords; i += NT) s.cntw[i] = 0u;
        if (tid < 8) s.u[tid] = 0u;
        __syncthreads();
        gather_counts<NT, CW>(a, s, a.qb + size_t(q) * a.L);
        for (uint32_t c = tid; c < a.BR; c += NT) a.out_counts[size_t(q) * a.BR + c] = uint16_t(cnt_at<CW>(s, c));
        __syncthreads();
    }
}

// Kernel entry points of one count width, by CTA size and record width.
template <int CW>
const void *plain_kernel_t(int NT, uint32_t rw)
{
#define FL_PLAIN(N) \
    switch (rw) { \
    case 1: return (const void *)k_query<N, 1, CW>; \
    case 2: return (const void *)k_query<N, 2, CW>; \
    case 4: return (const void *)k_query<N, 4, CW>; \
    default: return (const void *)k_query<N, 8, CW>; \
    }
    if (NT == 1024) { FL_PLAIN(1024) }
    if (NT == 512) { FL_PLAIN(512) }
    FL_PLAIN(256)
#undef FL_PLAIN
}

template <int CW>
const void *fused_kernel_t(int NT, uint32_t rw, bool srp)
{
#define FL_FUSED(N) \
    switch ((srp ? 10 : 0) + rw) { \
    case 1: return (const void *)k_query_fused<N, 1, 1, CW>; \
    case 2: return (const void *)k_query_fused<N, 2, 1, CW>; \
    case 4: return (const void *)k_query_fused<N, 4, 1, CW>; \
    case 8: return (const void *)k_query_fused<N, 8, 1, CW>; \
    case 11: return (const void *)k_query_fused<N, 1, 2, CW>; \
    case 12: return (const void *)k_query_fused<N, 2, 2, CW>; \
    case 14: return (const void *)k_query_fused<N, 4, 2, CW>; \
    default: return (const void *)k_query_fused<N, 8, 2, CW>; \
    }
    if (NT == 128) { FL_FUSED(128) }
    if (NT == 512) { FL_FUSED(512) }
    FL_FUSED(256)
#undef FL_FUSED
}

}  // namespace

// Per count width: the plain, fused and counts kernels (query.cu: CW = 1,
// query_c16.cu: CW = 2).
const void *plain_kernel_c1(int NT, uint32_t rw);
const void *fused_kernel_c1(int NT, uint32_t rw, bool srp);
const void *counts_kernel_c1();
const void *plain_kernel_c2(int NT, uint32_t rw);
const void *fused_kernel_c2(int NT, uint32_t rw, bool srp);
const void *counts_kernel_c2();

}  // namespace flinng
