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
//  1. counts: cnt[c] += 1 for every cell c in the query's list of each table
//     (bytes in shared memory, L <= 255). The L lists are flattened over the
//     whole CTA.
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
//     radix select over the 56-bit keys keeps the k best and tightens the
//     admission cutoff. At the end a radix select cuts the buffer to k keys,
//     which a small bitonic sort orders.
#include "internal.cuh"

namespace flinng {

namespace {

constexpr int kQT = 256;                 // threads per query CTA
constexpr int kQW = kQT / 32;
constexpr uint64_t kKeyBits = (1ull << 56) - 1;

struct QArgs {
    const uint32_t *qb;
    uint32_t nq;
    const uint32_t *k;
    uint32_t k_max;
    const uint32_t *off;
    const uint16_t *cells;
    const uint16_t *gid;
    const uint32_t *moff;
    const uint32_t *mem;
    uint32_t L, W, R, B, BR, t_min;
    uint32_t cap;      // candidate buffer entries (power of two)
    uint32_t kp;       // final sort width: power of two >= k_max
    uint32_t *out_ids;
    uint8_t *out_scores;
    uint8_t *out_counts;
};

struct QSmem {
    uint64_t *buf;       // cap candidate keys
    uint64_t *keep;      // kp keys (selection output, final sort)
    uint32_t *u;         // 8 scalars: nbuf, nkeep, sel digit, sel rem, ...
    uint32_t *hist_s;    // 256: points seen, by score
    uint32_t *lvl_n;     // 256: repetition-0 cells per count
    uint32_t *lvl_cur;   // 256
    uint32_t *rhist;     // 256: radix histogram
    uint32_t *c_start;   // kQT: member start of each cell of a chunk / list start
    uint32_t *c_pre;     // kQT + 1: exclusive prefix of member counts
    uint32_t *wsum;      // kQW: block-scan scratch
    uint32_t *cntw;      // (BR + 3) / 4 words of byte counts
    uint16_t *lvl_cells; // B
};

__host__ __device__ inline size_t qsmem_bytes(uint32_t cap, uint32_t kp, uint32_t BR, uint32_t B)
{
    size_t b = size_t(cap) * 8 + size_t(kp) * 8 + 8 * 4 + 4 * 256 * 4 + kQT * 4 + (kQT + 1) * 4 + kQW * 4;
    b = (b + 15) & ~size_t(15);
    b += size_t((BR + 3) / 4) * 4;
    b += size_t(B) * 2;
    return (b + 15) & ~size_t(15);
}

__device__ inline QSmem carve_q(unsigned char *sm, uint32_t cap, uint32_t kp)
{
    QSmem s;
    s.buf = (uint64_t *)sm;
    s.keep = s.buf + cap;
    s.u = (uint32_t *)(s.keep + kp);
    s.hist_s = s.u + 8;
    s.lvl_n = s.hist_s + 256;
    s.lvl_cur = s.lvl_n + 256;
    s.rhist = s.lvl_cur + 256;
    s.c_start = s.rhist + 256;
    s.c_pre = s.c_start + kQT;
    s.wsum = s.c_pre + kQT + 1;
    size_t o = (size_t)((unsigned char *)(s.wsum + kQW) - sm);
    o = (o + 15) & ~size_t(15);
    s.cntw = (uint32_t *)(sm + o);
    return s;
}

__device__ inline uint16_t *lvl_cells_ptr(const QSmem &s, uint32_t BR)
{
    return (uint16_t *)(s.cntw + (BR + 3) / 4);
}

template <int RP>
__device__ inline void load_gid(const uint16_t *__restrict__ gid, uint32_t x, uint32_t g[RP])
{
    if constexpr (RP == 1) {
        g[0] = gid[x];
    } else if constexpr (RP == 2) {
        const uint32_t v = __ldg(reinterpret_cast<const uint32_t *>(gid) + x);
        g[0] = v & 0xFFFFu;
        g[1] = v >> 16;
    } else if constexpr (RP == 4) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(gid) + x);
        g[0] = v.x & 0xFFFFu; g[1] = v.x >> 16; g[2] = v.y & 0xFFFFu; g[3] = v.y >> 16;
    } else {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(gid) + x);
        g[0] = v.x & 0xFFFFu; g[1] = v.x >> 16; g[2] = v.y & 0xFFFFu; g[3] = v.y >> 16;
        g[4] = v.z & 0xFFFFu; g[5] = v.z >> 16; g[6] = v.w & 0xFFFFu; g[7] = v.w >> 16;
    }
}

// Exclusive block scan of one value per thread; returns the prefix and
// writes the total to *total (all threads). Contains __syncthreads.
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
    for (int w = 0; w < kQW; ++w) {
        const uint32_t t = wsum[w];
        before += (w < warp) ? t : 0u;
        all += t;
    }
    __syncthreads();
    *total = all;
    return before + x - v;
}

// Largest i in [0, n) with pre[i] <= j (pre ascending, pre[0] = 0 <= j).
__device__ inline uint32_t find_seg(const uint32_t *pre, uint32_t n, uint32_t j)
{
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Radix select over keys[0..n): returns (prefix, mask) such that exactly kk
// keys satisfy (key & mask) <= prefix (keys are unique, kk <= n).
__device__ void block_select(const uint64_t *keys, uint32_t n, uint32_t kk, const QSmem &s,
                             uint64_t &prefix_out, uint64_t &mask_out)
{
    const int tid = threadIdx.x, lane = tid & 31;
    uint64_t prefix = 0, mask = 0;
    uint32_t rem = kk;
    for (int shift = 48; shift >= 0; shift -= 8) {
        s.rhist[tid] = 0u;                      // kQT == 256 bins
        __syncthreads();
        for (uint32_t i = tid; i < n; i += kQT) {
            const uint64_t v = keys[i];
            if ((v & mask) == prefix) atomicAdd(&s.rhist[(v >> shift) & 0xFF], 1u);
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
// bound (keys above it can never enter the top kk).
__device__ uint64_t block_compact(const QSmem &s, uint32_t nbuf, uint32_t kk)
{
    uint64_t prefix, mask;
    block_select(s.buf, nbuf, kk, s, prefix, mask);
    if (threadIdx.x == 0) s.u[1] = 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nbuf; i += kQT) {
        const uint64_t v = s.buf[i];
        if ((v & mask) <= prefix) s.keep[atomicAdd(&s.u[1], 1u)] = v;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kk; i += kQT) s.buf[i] = s.keep[i];
    if (threadIdx.x == 0) s.u[0] = kk;
    __syncthreads();
    return prefix | (~mask & kKeyBits);
}

__device__ void gather_counts(const QArgs &a, const QSmem &s, uint32_t q)
{
    const int tid = threadIdx.x;
    // one thread per table: its list's start and length
    uint32_t len = 0;
    for (uint32_t l0 = 0; l0 < a.L; l0 += kQT) {
        const uint32_t l = l0 + tid;
        uint32_t beg = 0;
        len = 0;
        if (l < a.L) {
            const uint64_t slot = (uint64_t(l) << a.W) | a.qb[size_t(q) * a.L + l];
            beg = a.off[slot];
            len = a.off[slot + 1] - beg;
        }
        uint32_t total;
        const uint32_t pre = block_excl_scan(len, s.wsum, &total);
        s.c_start[tid] = beg;
        s.c_pre[tid] = pre;
        __syncthreads();
        const uint32_t nl = min(uint32_t(kQT), a.L - l0);
        for (uint32_t e = tid; e < total; e += kQT) {
            const uint32_t t = find_seg(s.c_pre, nl, e);
            const uint32_t c = a.cells[s.c_start[t] + (e - s.c_pre[t])];
            atomicAdd(&s.cntw[c >> 2], 1u << ((c & 3) * 8));
        }
        __syncthreads();
    }
}

template <int RP>
__global__ void __launch_bounds__(kQT)
k_query(QArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const QSmem s = carve_q(sm, a.cap, a.kp);
    uint16_t *lvl_cells = lvl_cells_ptr(s, a.BR);
    const uint8_t *cnt8 = reinterpret_cast<const uint8_t *>(s.cntw);
    const int tid = threadIdx.x;
    const uint32_t nwords = (a.BR + 3) / 4;

    for (uint32_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
        uint32_t kq = a.k ? a.k[q] : a.k_max;
        if (kq > a.k_max) kq = a.k_max;
        for (uint32_t i = tid; i < nwords; i += kQT) s.cntw[i] = 0u;
        s.hist_s[tid] = 0u;
        s.lvl_n[tid] = 0u;
        if (tid < 8) s.u[tid] = 0u;
        __syncthreads();
        if (kq > 0) {
            gather_counts(a, s, q);
            // group tests of repetition 0, bucketed by count level
            for (uint32_t b = tid; b < a.B; b += kQT) {
                const uint32_t v = cnt8[b];
                if (v >= a.t_min) atomicAdd(&s.lvl_n[v], 1u);
            }
            __syncthreads();
            if (tid == 0) {
                uint32_t run = 0;
                for (int t = int(a.L); t >= int(a.t_min); --t) {
                    s.lvl_cur[t] = run;
                    run += s.lvl_n[t];
                }
            }
            __syncthreads();
            for (uint32_t b = tid; b < a.B; b += kQT) {
                const uint32_t v = cnt8[b];
                if (v >= a.t_min) lvl_cells[atomicAdd(&s.lvl_cur[v], 1u)] = uint16_t(b);
            }
            __syncthreads();
            // decode, level by level
            uint64_t bound = kKeyBits;           // admission: key <= bound
            uint32_t seen = 0;                   // points with score >= current level
            const uint32_t sub = a.cap - a.kp;   // members per round (room after a compaction)
            for (int t = int(a.L); t >= int(a.t_min); --t) {
                const uint32_t nc = s.lvl_n[t];
                const uint32_t first = s.lvl_cur[t] - nc;
                for (uint32_t c0 = 0; c0 < nc; c0 += kQT) {
                    const uint32_t ci = c0 + tid;
                    uint32_t ms = 0, sz = 0;
                    if (ci < nc) {
                        const uint32_t b = lvl_cells[first + ci];
                        ms = a.moff[b];
                        sz = a.moff[b + 1] - ms;
                    }
                    uint32_t M;
                    const uint32_t pre = block_excl_scan(sz, s.wsum, &M);
                    s.c_start[tid] = ms;
                    s.c_pre[tid] = pre;
                    const uint32_t ncc = min(uint32_t(kQT), nc - c0);
                    __syncthreads();
                    for (uint32_t j0 = 0; j0 < M; j0 += sub) {
                        const uint32_t jn = min(M, j0 + sub);
                        if (s.u[0] + (jn - j0) > a.cap) bound = block_compact(s, s.u[0], kq);
                        for (uint32_t j = j0 + tid; j < jn; j += kQT) {
                            const uint32_t cs = find_seg(s.c_pre, ncc, j);
                            const uint32_t x = __ldg(a.mem + s.c_start[cs] + (j - s.c_pre[cs]));
                            uint32_t g[RP];
                            load_gid<RP>(a.gid, x, g);
                            uint32_t score = 256, last = 0;
#pragma unroll
                            for (int r = 0; r < RP; ++r) {
                                if (r < int(a.R)) {
                                    const uint32_t c = uint32_t(r) * a.B + g[r];
                                    const uint32_t v = cnt8[c];
                                    if (v < score) {
                                        score = v;
                                        last = c;
                                    } else if (v == score) {
                                        last = c;
                                    }
                                }
                            }
                            if (score >= a.t_min) {
                                atomicAdd(&s.hist_s[score], 1u);
                                const uint64_t key = (uint64_t(255u - score) << 48) | (uint64_t(last) << 32) | x;
                                if (key <= bound) s.buf[atomicAdd(&s.u[0], 1u)] = key;
                            }
                        }
                        __syncthreads();
                    }
                }
                seen += s.hist_s[t];             // final: later levels only add scores < t
                if (seen >= kq) break;
            }
        }
        __syncthreads();
        // final top-k: cut to kq keys, sort, write
        const uint32_t nbuf = s.u[0];
        const uint32_t nk = nbuf < kq ? nbuf : kq;
        if (nbuf > kq) {
            block_compact(s, nbuf, kq);
        }
        for (uint32_t i = tid; i < a.kp; i += kQT) s.keep[i] = (i < nk) ? s.buf[i] : kKeyNone;
        __syncthreads();
        for (uint32_t k2 = 2; k2 <= a.kp; k2 <<= 1) {
            for (uint32_t j = k2 >> 1; j > 0; j >>= 1) {
                for (uint32_t i = tid; i < a.kp; i += kQT) {
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
        for (uint32_t i = tid; i < a.k_max; i += kQT) {
            const uint64_t key = (i < nk) ? s.keep[i] : kKeyNone;
            const bool ok = key != kKeyNone;
            a.out_ids[size_t(q) * a.k_max + i] = ok ? uint32_t(key & 0xFFFFFFFFu) : 0xFFFFFFFFu;
            if (a.out_scores)
                a.out_scores[size_t(q) * a.k_max + i] = ok ? uint8_t(255u - uint32_t(key >> 48)) : uint8_t(0);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kQT)
k_counts(QArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const QSmem s = carve_q(sm, a.cap, a.kp);
    const uint8_t *cnt8 = reinterpret_cast<const uint8_t *>(s.cntw);
    const int tid = threadIdx.x;
    const uint32_t nwords = (a.BR + 3) / 4;
    for (uint32_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
        for (uint32_t i = tid; i < nwords; i += kQT) s.cntw[i] = 0u;
        __syncthreads();
        gather_counts(a, s, q);
        for (uint32_t c = tid; c < a.BR; c += kQT) a.out_counts[size_t(q) * a.BR + c] = cnt8[c];
        __syncthreads();
    }
}

inline uint32_t pow2_at_least(uint32_t v)
{
    uint32_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

QArgs make_args(flinng_index *ix, const uint32_t *qb, uint32_t nq)
{
    QArgs a{};
    a.qb = qb;
    a.nq = nq;
    a.off = ix->off;
    a.cells = ix->cells;
    a.gid = ix->gid;
    a.moff = ix->moff;
    a.mem = ix->mem;
    a.L = ix->cfg.L;
    a.W = ix->cfg.range_bits;
    a.R = ix->cfg.R;
    a.B = ix->cfg.B;
    a.BR = ix->BR;
    a.t_min = ix->cfg.min_threshold;
    return a;
}

template <int RP>
int launch_query_rp(const QArgs &a, size_t smem, cudaStream_t st)
{
    if (smem > 48 * 1024)
        FL_CUDA(cudaFuncSetAttribute(k_query<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_query<RP><<<a.nq, kQT, smem, st>>>(a);
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}

}  // namespace

int query_launch(flinng_index *ix, const uint32_t *qbuckets, uint32_t nq,
                 const uint32_t *k, uint32_t k_max, uint32_t *out_ids,
                 uint8_t *out_scores)
{
    if (nq == 0) return FLINNG_OK;
    QArgs a = make_args(ix, qbuckets, nq);
    a.k = k;
    a.k_max = k_max;
    a.kp = pow2_at_least(k_max > 1 ? k_max : 2);
    // room for one full round of members after a compaction to k keys
    a.cap = pow2_at_least(a.kp + 2 * kQT > 2048 ? a.kp + 2 * kQT : 2048);
    a.out_ids = out_ids;
    a.out_scores = out_scores;
    size_t smem = qsmem_bytes(a.cap, a.kp, a.BR, a.B);
    while (smem > 227 * 1024 && a.cap > a.kp + kQT) {       // large B*R: trade buffer for room
        a.cap >>= 1;
        smem = qsmem_bytes(a.cap, a.kp, a.BR, a.B);
    }
    if (smem > 227 * 1024 || a.cap < a.kp + kQT)
        return set_error(FLINNG_ERR_INVALID_ARG,
                         "query: k_max=%u with B*R=%u needs %zu bytes of shared memory (> 227 KB)",
                         k_max, a.BR, smem);
    switch (ix->rp) {
    case 1: return launch_query_rp<1>(a, smem, ix->stream);
    case 2: return launch_query_rp<2>(a, smem, ix->stream);
    case 4: return launch_query_rp<4>(a, smem, ix->stream);
    default: return launch_query_rp<8>(a, smem, ix->stream);
    }
}

int counts_launch(flinng_index *ix, const uint32_t *qbuckets, uint32_t nq,
                  uint8_t *out_counts)
{
    if (nq == 0) return FLINNG_OK;
    QArgs a = make_args(ix, qbuckets, nq);
    a.cap = 2;
    a.kp = 2;
    a.out_counts = out_counts;
    const size_t smem = qsmem_bytes(a.cap, a.kp, a.BR, a.B);
    if (smem > 48 * 1024)
        FL_CUDA(cudaFuncSetAttribute(k_counts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_counts<<<nq, kQT, smem, ix->stream>>>(a);
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}

}  // namespace flinng
