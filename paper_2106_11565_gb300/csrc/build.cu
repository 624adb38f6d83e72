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

__global__ void k_slot_hist(const uint32_t *__restrict__ buckets, uint64_t n, uint32_t L,
                            uint32_t W, uint32_t R, uint32_t *__restrict__ hist)
{
    const uint64_t total = n * L;
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t l = uint32_t(t % L);
        atomicAdd(&hist[(uint64_t(l) << W) | buckets[t]], R);
    }
}

__global__ void k_slot_add_old(const uint32_t *__restrict__ off, uint64_t nslot,
                               uint32_t *__restrict__ hist)
{
    for (uint64_t s = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < nslot;
         s += uint64_t(gridDim.x) * blockDim.x)
        hist[s] += off[s + 1] - off[s];
}

// cursor[s] = toff[s] + old length; old list copied to the head of the slot.
__global__ void k_slot_copy_old(const uint32_t *__restrict__ off, const uint16_t *__restrict__ cells,
                                const uint32_t *__restrict__ toff, uint64_t nslot, int have_old,
                                uint32_t *__restrict__ cursor, uint16_t *__restrict__ tmp)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t s = gw; s < nslot; s += nw) {
        const uint32_t dst = toff[s];
        uint32_t len = 0;
        if (have_old) {
            const uint32_t beg = off[s];
            len = off[s + 1] - beg;
            for (uint32_t t = lane; t < len; t += 32) tmp[dst + t] = cells[beg + t];
        }
        if (lane == 0) cursor[s] = dst + len;
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
        const uint64_t x = t / L;
        const uint32_t l = uint32_t(t % L);
        const uint32_t pos = atomicAdd(&cursor[(uint64_t(l) << W) | buckets[t]], R);
        const uint16_t *g = gid + (n_old + x) * rp;
        for (uint32_t r = 0; r < R; ++r) tmp[pos + r] = uint16_t(r * B + g[r]);
    }
}

// Sort and deduplicate each slot in place; ulen[s] = distinct cells.
// <= 32 entries: warp bitonic sort in registers. More: a bitmap over all
// B*R cells in shared memory, read back in cell order.
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_slot_unique(const uint32_t *__restrict__ toff, uint64_t nslot, uint32_t BR,
              uint16_t *__restrict__ tmp, uint32_t *__restrict__ ulen)
{
    extern __shared__ uint32_t bm_all[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nwords = (BR + 31) / 32;
    uint32_t *bm = bm_all + warp * nwords;
    const uint64_t gw = uint64_t(blockIdx.x) * kWarpsPerBlock + warp;
    const uint64_t nw = uint64_t(gridDim.x) * kWarpsPerBlock;
    for (uint64_t s = gw; s < nslot; s += nw) {
        const uint32_t beg = toff[s], len = toff[s + 1] - beg;
        if (len == 0) {
            if (lane == 0) ulen[s] = 0;
            continue;
        }
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

__global__ void k_slot_compact(const uint32_t *__restrict__ toff, const uint32_t *__restrict__ off,
                               uint64_t nslot, const uint16_t *__restrict__ tmp,
                               uint16_t *__restrict__ cells)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t s = gw; s < nslot; s += nw) {
        const uint32_t src = toff[s], dst = off[s], len = off[s + 1] - dst;
        for (uint32_t t = lane; t < len; t += 32) cells[dst + t] = tmp[src + t];
    }
}

__global__ void k_heavy_flag(const uint32_t *__restrict__ off, uint64_t nslot, uint32_t heavy_min,
                             uint32_t *__restrict__ flag)
{
    for (uint64_t s = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < nslot;
         s += uint64_t(gridDim.x) * blockDim.x)
        flag[s] = (off[s + 1] - off[s]) >= heavy_min ? 1u : 0u;
}

// hidx[s] = bitmap index of heavy slot s (exclusive prefix of the flags) or
// kEmpty32; each heavy slot's bitmap is written by one warp.
__global__ void k_heavy_fill(const uint32_t *__restrict__ off, const uint16_t *__restrict__ cells,
                             const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pre,
                             uint64_t nslot, uint32_t BRw, uint32_t *__restrict__ hidx,
                             uint32_t *__restrict__ hbm)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t s = gw; s < nslot; s += nw) {
        const bool heavy = flag[s] != 0u;
        if (lane == 0) hidx[s] = heavy ? pre[s] : kEmpty32;
        if (!heavy) continue;
        uint32_t *bm = hbm + uint64_t(pre[s]) * BRw;
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
// Uses the build scratch slot_a / slot_b; grows the bitmap array if needed.
int build_heavy(flinng_index *ix, void *scan_ws)
{
    const cudaStream_t st = ix->stream;
    const uint64_t nslot = ix->nslot;
    k_heavy_flag<<<thread_blocks(nslot), 256, 0, st>>>(ix->off, nslot, ix->heavy_min, ix->slot_a);
    count_launch();
    FL_CUDA(cudaGetLastError());
    FL_TRY(scan_exclusive(ix->slot_a, ix->slot_b, nslot, scan_ws, st));
    FL_CUDA(cudaMemcpyAsync(ix->h_flag, ix->slot_b + nslot, 4, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    const uint32_t nh = *ix->h_flag;
    if (ix->BRw * 32 < ix->BR || ix->BRw == 0)
        return set_error(FLINNG_ERR_INVALID_ARG, "internal: cell bitmap width %u for B*R=%u", ix->BRw, ix->BR);
    const uint64_t words = uint64_t(nh) * ix->BRw;
    if (words > ix->hbm_words) {
        if (ix->hbm) {
            cudaFree(ix->hbm);
            ix->device_bytes -= ix->hbm_words * 4;
            ix->hbm = nullptr;
            ix->hbm_words = 0;
        }
        const uint64_t want = words + words / 8 + ix->BRw;
        FL_CUDA(cudaMalloc(&ix->hbm, want * 4));
        ix->hbm_words = want;
        ix->device_bytes += want * 4;
    }
    if (nh > 0 && (!ix->hbm || ix->hbm_words < words))
        return set_error(FLINNG_ERR_OOM, "internal: no storage for %u cell bitmaps", nh);
    k_heavy_fill<<<warp_blocks(nslot), kWarpsPerBlock * 32, 0, st>>>(ix->off, ix->cells, ix->slot_a, ix->slot_b,
                                                                    nslot, ix->BRw, ix->hidx, ix->hbm);
    count_launch();
    FL_CUDA(cudaGetLastError());
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
    FL_CUDA(cudaMemsetAsync(ix->flag, 0, 4, st));
    k_perm_check<<<thread_blocks(uint64_t(R) * n), 256, 0, st>>>(perm, R, n, seen, ix->flag);
    count_launch();
    FL_CUDA(cudaGetLastError());
    FL_CUDA(cudaMemcpyAsync(ix->h_flag, ix->flag, 4, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    if (*ix->h_flag & 1u) return set_error(FLINNG_ERR_INVALID_ARG, "perm: entry out of range [0, n)");
    if (*ix->h_flag & 2u) return set_error(FLINNG_ERR_INVALID_ARG, "perm: a row repeats an index");
    return FLINNG_OK;
}

size_t insert_workspace_bytes(const flinng_index *ix)
{
    const size_t ns = ix->nslot + 1;
    const size_t big = ns > size_t(ix->BR) + 1 ? ns : size_t(ix->BR) + 1;
    return carve_bytes<uint32_t>(ns) + carve_bytes<uint32_t>(ix->BR + 1) + scan_workspace_bytes(big);
}

int check_groups(flinng_index *ix, const uint16_t *groups, uint64_t n)
{
    const cudaStream_t st = ix->stream;
    if (n == 0) return FLINNG_OK;
    FL_CUDA(cudaMemsetAsync(ix->flag, 0, 4, st));
    k_check_groups<<<thread_blocks(uint64_t(ix->cfg.R) * n), 256, 0, st>>>(groups, uint64_t(ix->cfg.R) * n,
                                                                         ix->cfg.B, ix->flag);
    count_launch();
    FL_CUDA(cudaGetLastError());
    FL_CUDA(cudaMemcpyAsync(ix->h_flag, ix->flag, 4, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    if (*ix->h_flag & 8u) return set_error(FLINNG_ERR_INVALID_ARG, "groups: a group id is >= B");
    return FLINNG_OK;
}

int insert_hashed(flinng_index *ix, const uint32_t *buckets, const uint32_t *perm, const uint16_t *groups,
                  uint64_t n, void *ws)
{
    const cudaStream_t st = ix->stream;
    const uint32_t R = ix->cfg.R, B = ix->cfg.B, L = ix->cfg.L, W = ix->cfg.range_bits;
    const uint32_t BR = ix->BR, rp = ix->rp;
    const uint64_t n_old = ix->n_points, N = n_old + n, nslot = ix->nslot;
    Carver c(ws, ~size_t(0));
    uint32_t *cursor = c.take<uint32_t>(nslot + 1);
    uint32_t *mcur = c.take<uint32_t>(BR + 1);
    void *scan_ws = c.base + ((c.used + 255) & ~size_t(255));

    // groups of the new points: Alg. 1 from the permutations, or given outright
    TraceRange stage1("groups and member lists");
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

    stage1.end();
    TraceRange stage2("reverse index");
    // reverse index: histogram of old lists + new entries per slot
    uint32_t *hist = ix->slot_a, *toff = ix->slot_b;
    const int have_old = (n_old > 0 && ix->n_cells > 0) ? 1 : 0;
    FL_CUDA(cudaMemsetAsync(hist, 0, (nslot + 1) * sizeof(uint32_t), st));
    if (n > 0) {
        k_slot_hist<<<thread_blocks(n * L), 256, 0, st>>>(buckets, n, L, W, R, hist);
        count_launch();
        FL_CUDA(cudaGetLastError());
    }
    if (have_old) {
        k_slot_add_old<<<thread_blocks(nslot), 256, 0, st>>>(ix->off, nslot, hist);
        count_launch();
        FL_CUDA(cudaGetLastError());
    }
    FL_TRY(scan_exclusive(hist, toff, nslot, scan_ws, st));
    k_slot_copy_old<<<warp_blocks(nslot), kWarpsPerBlock * 32, 0, st>>>(
        ix->off, ix->cells, toff, nslot, have_old, cursor, ix->cells_tmp);
    count_launch();
    FL_CUDA(cudaGetLastError());
    if (n > 0) {
        k_slot_scatter_new<<<thread_blocks(n * L), 256, 0, st>>>(buckets, ix->gid, n_old, n, L, W, R, B,
                                                                 rp, cursor, ix->cells_tmp);
        count_launch();
        FL_CUDA(cudaGetLastError());
    }
    // sort + dedupe each slot; ulen reuses the histogram buffer
    uint32_t *ulen = hist;
    const size_t smem = size_t(kWarpsPerBlock) * ((BR + 31) / 32) * sizeof(uint32_t);
    FL_TRY(ensure_dyn_smem((const void *)k_slot_unique, smem));
    k_slot_unique<<<warp_blocks(nslot), kWarpsPerBlock * 32, smem, st>>>(toff, nslot, BR, ix->cells_tmp, ulen);
    count_launch();
    FL_CUDA(cudaGetLastError());
    FL_TRY(scan_exclusive(ulen, ix->off, nslot, scan_ws, st));
    k_slot_compact<<<warp_blocks(nslot), kWarpsPerBlock * 32, 0, st>>>(toff, ix->off, nslot,
                                                                       ix->cells_tmp, ix->cells);
    count_launch();
    FL_CUDA(cudaGetLastError());
    FL_CUDA(cudaMemcpyAsync(ix->h_flag, ix->off + nslot, 4, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    ix->n_cells = *ix->h_flag;
    ix->n_points = N;
    stage2.end();
    TraceRange stage3("heavy bitmaps");
    FL_TRY(build_heavy(ix, scan_ws));
    return FLINNG_OK;
}

}  // namespace flinng
