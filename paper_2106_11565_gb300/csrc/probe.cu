// Multi-probe per-cell counts (an option of cosine / SRP indices; the related
// work's multi-probe LSH as a recall lever). In table l the query probes its
// own bucket and the P - 1 buckets that differ from it in exactly one of the
// code's bits 0 .. P-2 (the sign of projection l*K + j flipped). A cell
// counts table l once if any probed bucket's list holds it, so counts stay in
// [0, L] and Alg. 3 decodes them unchanged (query_launch_counts).
//
// One CTA per query, one warp per table at a time: the warp ORs the P probed
// lists (or heavy bitmaps) of its table into a bitmap over the B*R cells in
// shared memory, then adds the bitmap's set bits to the query's 16-bit
// counters (shared-memory atomics).
#include "internal.cuh"

namespace flinng {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeWarps = kProbeThreads / 32;

struct ProbeArgs {
    const uint32_t *qb;        // nq x L query buckets
    uint32_t nq, L, W, BR, BRw, P, heavy_min;
    const uint32_t *off;
    const uint16_t *cells;
    const uint32_t *hidx;
    const uint32_t *hbm;
    uint16_t *out;             // nq x BR counts
};

__global__ void __launch_bounds__(kProbeThreads)
k_counts_probe(ProbeArgs a)
{
    extern __shared__ __align__(16) uint32_t psm[];
    const uint32_t nwords = (a.BR + 1) / 2;            // two 16-bit counters per word
    uint32_t *cntw = psm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *bm = psm + ((nwords + 3) & ~3u) + warp * a.BRw;
    for (uint32_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
        for (uint32_t i = tid; i < nwords; i += kProbeThreads) cntw[i] = 0u;
        __syncthreads();
        for (uint32_t l = warp; l < a.L; l += kProbeWarps) {
            for (uint32_t w = lane; w < a.BRw; w += 32) bm[w] = 0u;
            __syncwarp();
            const uint32_t b = a.qb[uint64_t(q) * a.L + l];
            for (uint32_t i = 0; i < a.P; ++i) {
                const uint64_t slot = (uint64_t(l) << a.W) | (i == 0 ? b : (b ^ (1u << (i - 1))));
                const uint32_t o0 = a.off[slot], o1 = a.off[slot + 1];
                if (o1 - o0 >= a.heavy_min) {
                    const uint32_t *hb = a.hbm + uint64_t(a.hidx[slot]) * a.BRw;
                    for (uint32_t w = lane; w < a.BRw; w += 32) bm[w] |= hb[w];   // each lane owns its words
                } else {
                    for (uint32_t t = o0 + lane; t < o1; t += 32) {
                        const uint32_t c = a.cells[t];
                        atomicOr(&bm[c >> 5], 1u << (c & 31));
                    }
                }
                __syncwarp();
            }
            for (uint32_t w = lane; w < a.BRw; w += 32) {
                uint32_t bits = bm[w];
                while (bits) {
                    const uint32_t c = w * 32 + uint32_t(__ffs(bits) - 1);
                    bits &= bits - 1;
                    atomicAdd(&cntw[c >> 1], 1u << ((c & 1) * 16));
                }
            }
            __syncwarp();
        }
        __syncthreads();
        const uint16_t *c16 = reinterpret_cast<const uint16_t *>(cntw);
        for (uint32_t c = tid; c < a.BR; c += kProbeThreads) a.out[uint64_t(q) * a.BR + c] = c16[c];
        __syncthreads();
    }
}

}  // namespace

size_t probe_smem_bytes(uint32_t BR)
{
    const uint32_t nwords = (BR + 1) / 2, BRw = (BR + 31) / 32;
    return (size_t((nwords + 3) & ~3u) + size_t(kProbeWarps) * BRw) * sizeof(uint32_t);
}

int probe_counts_launch(flinng_index *ix, const uint32_t *qb, uint32_t nq, uint32_t P, uint16_t *out_counts)
{
    if (nq == 0) return FLINNG_OK;
    ProbeArgs a{};
    a.qb = qb;
    a.nq = nq;
    a.L = ix->cfg.L;
    a.W = ix->cfg.range_bits;
    a.BR = ix->BR;
    a.BRw = ix->BRw;
    a.P = P;
    a.heavy_min = ix->heavy_min;
    a.off = ix->off;
    a.cells = ix->cells;
    a.hidx = ix->hidx;
    a.hbm = ix->hbm;
    a.out = out_counts;
    const size_t smem = probe_smem_bytes(ix->BR);
    if (smem > 227 * 1024)
        return set_error(FLINNG_ERR_INVALID_ARG, "multi-probe counts: B*R=%u needs %zu bytes of shared memory",
                         ix->BR, smem);
    FL_TRY(ensure_dyn_smem((const void *)k_counts_probe, smem));
    if (!ix->sms) FL_CUDA(cudaDeviceGetAttribute(&ix->sms, cudaDevAttrMultiProcessorCount, ix->device));
    int per_sm = 0;
    FL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_counts_probe, kProbeThreads, smem));
    uint64_t grid = uint64_t(ix->sms) * (per_sm > 0 ? per_sm : 1);
    if (grid > nq) grid = nq;
    k_counts_probe<<<unsigned(grid), kProbeThreads, smem, ix->stream>>>(a);
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}

}  // namespace flinng
