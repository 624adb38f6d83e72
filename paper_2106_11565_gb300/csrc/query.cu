// Batched query: collision counts, group tests, AND-over-R decode and top-k
// (Sec. 5, Alg. 2 and Alg. 3). One CTA per query.
//
// Alg. 3 walks cells by count (descending, ties by cell id) and emits a point
// when the last of its R cells is reached. That order is the ascending order
// of the key (-score, lastcell, id) with score = the least count among the
// point's R cells and lastcell = the largest cell id among those cells with
// that count; points with score < t_min are never emitted. The kernel
// computes the k smallest keys without the per-point counter array:
//
//  1. counts: cnt[c] += 1 for every cell c in the query's list of each table
//     (bytes in shared memory, L <= 255).
//  2. group tests at decreasing thresholds: the cells of repetition 0 are
//     bucketed by count; level t holds those with count exactly t.
//  3. decode: walk levels t = L, L-1, ..., t_min. A point of score >= t has
//     all R cells at count >= t, in particular its repetition-0 cell, so after
//     level t every point with score >= t has been seen. Each member of a
//     level-t cell gets its key from its R group ids (the AND over R);
//     stop once >= k points of score >= t were seen - no unseen point can
//     precede them.
//  4. top-k: each warp keeps its own buffer of candidate keys below its
//     running cutoff, sorted and cut to k when full; the warp buffers are
//     merged by one block-wide bitonic sort.
#include "internal.cuh"

namespace flinng {

namespace {

constexpr int kQW = 8;   // warps per query CTA

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
    uint32_t L, W, R, B, BR, t_min, cw;
    uint32_t *out_ids;
    uint8_t *out_scores;
    uint8_t *out_counts;
};

struct QSmem {
    uint64_t *buf;     // kQW * cw keys
    uint64_t *wcut;    // kQW
    uint32_t *wn;      // kQW
    uint32_t *hist_s;  // 256: points seen, by score
    uint32_t *lvl_n;   // 256: repetition-0 cells per count
    uint32_t *lvl_cur; // 256
    uint32_t *cntw;    // (BR + 3) / 4 words of byte counts
    uint16_t *lvl_cells;   // B
};

__host__ __device__ inline size_t qsmem_bytes(uint32_t cw, uint32_t BR, uint32_t B)
{
    size_t b = size_t(kQW) * cw * 8 + kQW * 8 + kQW * 4 + 3 * 256 * 4;
    b += size_t((BR + 3) / 4) * 4;
    b += size_t(B) * 2;
    return (b + 15) & ~size_t(15);
}

__device__ inline QSmem carve_q(unsigned char *sm, uint32_t cw, uint32_t BR)
{
    QSmem s;
    s.buf = (uint64_t *)sm;
    s.wcut = s.buf + size_t(kQW) * cw;
    s.wn = (uint32_t *)(s.wcut + kQW);
    s.hist_s = s.wn + kQW;
    s.lvl_n = s.hist_s + 256;
    s.lvl_cur = s.lvl_n + 256;
    s.cntw = s.lvl_cur + 256;
    s.lvl_cells = (uint16_t *)(s.cntw + (BR + 3) / 4);
    return s;
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

// Sort wb[0..cw) ascending with one warp after padding entries >= n.
__device__ void warp_sort(uint64_t *wb, uint32_t n, uint32_t cw, int lane)
{
    for (uint32_t i = lane; i < cw; i += 32)
        if (i >= n) wb[i] = kKeyNone;
    __syncwarp();
    for (uint32_t k = 2; k <= cw; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = lane; i < cw; i += 32) {
                const uint32_t l = i ^ j;
                if (l > i) {
                    const uint64_t a = wb[i], b = wb[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        wb[i] = b;
                        wb[l] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Warp-cooperative insertion of one key per lane into the warp's buffer.
__device__ void warp_insert(uint64_t key, bool has, uint64_t *wb, uint32_t *wn,
                            uint64_t *wcut, uint32_t kq, uint32_t cw, int lane)
{
    uint64_t cut = *wcut;
    bool want = has && key < cut;
    uint32_t m = __ballot_sync(0xffffffffu, want);
    if (m == 0) return;
    uint32_t n = *wn;
    if (n + __popc(m) > cw) {
        warp_sort(wb, n, cw, lane);
        if (n > kq) n = kq;
        if (n == kq) cut = wb[kq - 1];
        want = has && key < cut;
        m = __ballot_sync(0xffffffffu, want);
    }
    if (want) wb[n + __popc(m & ((1u << lane) - 1u))] = key;
    __syncwarp();
    if (lane == 0) {
        *wn = n + __popc(m);
        *wcut = cut;
    }
    __syncwarp();
}

__device__ void gather_counts(const QArgs &a, const QSmem &s, uint32_t q, int lane, int warp)
{
    const uint32_t *qb = a.qb + size_t(q) * a.L;
    for (uint32_t l = warp; l < a.L; l += kQW) {
        const uint64_t slot = (uint64_t(l) << a.W) | qb[l];
        const uint32_t beg = a.off[slot], end = a.off[slot + 1];
        for (uint32_t t = beg + lane; t < end; t += 32) {
            const uint32_t c = a.cells[t];
            atomicAdd(&s.cntw[c >> 2], 1u << ((c & 3) * 8));
        }
    }
}

template <int RP>
__global__ void __launch_bounds__(kQW * 32)
k_query(QArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const QSmem s = carve_q(sm, a.cw, a.BR);
    const uint8_t *cnt8 = reinterpret_cast<const uint8_t *>(s.cntw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = kQW * 32;
    const uint32_t nwords = (a.BR + 3) / 4;

    for (uint32_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
        uint32_t kq = a.k ? a.k[q] : a.k_max;
        if (kq > a.k_max) kq = a.k_max;
        for (uint32_t i = tid; i < nwords; i += nthr) s.cntw[i] = 0u;
        for (uint32_t i = tid; i < 256; i += nthr) {
            s.hist_s[i] = 0u;
            s.lvl_n[i] = 0u;
        }
        if (lane == 0) {
            s.wn[warp] = 0u;
            s.wcut[warp] = kKeyNone;
        }
        __syncthreads();
        if (kq > 0) {
            gather_counts(a, s, q, lane, warp);
            __syncthreads();
            for (uint32_t b = tid; b < a.B; b += nthr) {
                const uint32_t v = cnt8[b];
                if (v >= a.t_min) atomicAdd(&s.lvl_n[v], 1u);
            }
            __syncthreads();
            if (tid == 0) {
                uint32_t run = 0;
                for (int t = int(a.L); t >= int(a.t_min); --t) {
                    run += s.lvl_n[t];
                    s.lvl_cur[t] = run - s.lvl_n[t];
                }
            }
            __syncthreads();
            for (uint32_t b = tid; b < a.B; b += nthr) {
                const uint32_t v = cnt8[b];
                if (v >= a.t_min) s.lvl_cells[atomicAdd(&s.lvl_cur[v], 1u)] = uint16_t(b);
            }
            __syncthreads();
            uint64_t *wb = s.buf + size_t(warp) * a.cw;
            for (int t = int(a.L); t >= int(a.t_min); --t) {
                const uint32_t nc = s.lvl_n[t];
                const uint32_t start = s.lvl_cur[t] - nc;
                for (uint32_t ci = warp; ci < nc; ci += kQW) {
                    const uint32_t b = s.lvl_cells[start + ci];
                    const uint32_t mb = a.moff[b], me = a.moff[b + 1];
                    for (uint32_t m0 = mb; m0 < me; m0 += 32) {
                        const uint32_t m = m0 + lane;
                        bool has = false;
                        uint64_t key = kKeyNone;
                        if (m < me) {
                            const uint32_t x = __ldg(a.mem + m);
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
                                has = true;
                                key = (uint64_t(255u - score) << 48) | (uint64_t(last) << 32) | x;
                                atomicAdd(&s.hist_s[score], 1u);
                            }
                        }
                        warp_insert(key, has, wb, &s.wn[warp], &s.wcut[warp], kq, a.cw, lane);
                    }
                }
                __syncthreads();
                uint32_t total = 0;
                for (uint32_t sc = uint32_t(t); sc <= a.L; ++sc) total += s.hist_s[sc];
                if (total >= kq) break;
            }
        }
        __syncthreads();
        const uint32_t T = kQW * a.cw;
        for (uint32_t i = tid; i < T; i += nthr)
            if ((i % a.cw) >= s.wn[i / a.cw]) s.buf[i] = kKeyNone;
        __syncthreads();
        for (uint32_t k = 2; k <= T; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t i = tid; i < T; i += nthr) {
                    const uint32_t l = i ^ j;
                    if (l > i) {
                        const uint64_t x = s.buf[i], y = s.buf[l];
                        const bool up = (i & k) == 0;
                        if ((x > y) == up) {
                            s.buf[i] = y;
                            s.buf[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (uint32_t i = tid; i < a.k_max; i += nthr) {
            const uint64_t key = (i < kq) ? s.buf[i] : kKeyNone;
            const bool ok = key != kKeyNone;
            a.out_ids[size_t(q) * a.k_max + i] = ok ? uint32_t(key & 0xFFFFFFFFu) : 0xFFFFFFFFu;
            if (a.out_scores)
                a.out_scores[size_t(q) * a.k_max + i] = ok ? uint8_t(255u - uint32_t(key >> 48)) : uint8_t(0);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kQW * 32)
k_counts(QArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const QSmem s = carve_q(sm, a.cw, a.BR);
    const uint8_t *cnt8 = reinterpret_cast<const uint8_t *>(s.cntw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nwords = (a.BR + 3) / 4;
    for (uint32_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
        for (uint32_t i = tid; i < nwords; i += kQW * 32) s.cntw[i] = 0u;
        __syncthreads();
        gather_counts(a, s, q, lane, warp);
        __syncthreads();
        for (uint32_t c = tid; c < a.BR; c += kQW * 32) a.out_counts[size_t(q) * a.BR + c] = cnt8[c];
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
    k_query<RP><<<a.nq, kQW * 32, smem, st>>>(a);
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
    a.cw = pow2_at_least(k_max + 32 > 64 ? k_max + 32 : 64);
    a.out_ids = out_ids;
    a.out_scores = out_scores;
    const size_t smem = qsmem_bytes(a.cw, a.BR, a.B);
    if (smem > 227 * 1024)
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
    a.cw = 1;
    a.out_counts = out_counts;
    const size_t smem = qsmem_bytes(a.cw, a.BR, a.B);
    if (smem > 48 * 1024)
        FL_CUDA(cudaFuncSetAttribute(k_counts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_counts<<<nq, kQW * 32, smem, ix->stream>>>(a);
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}

}  // namespace flinng
