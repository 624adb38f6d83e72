// Host side of the batched query: launch shapes, shared-memory budgets,
// the fused form's graphs and the autotuned shapes, and the count-width
// dispatch. The kernels are in query_impl.cuh.
#include "query_impl.cuh"

namespace flinng {
namespace {

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
    a.moff = ix->moff;
    a.mrec = ix->mrec;
    a.hidx = ix->hidx;
    a.hbm = ix->hbm;
    a.BRw = ix->BRw;
    a.heavy_min = ix->heavy_min;
    a.L = ix->cfg.L;
    a.W = ix->cfg.range_bits;
    a.R = ix->cfg.R;
    a.B = ix->cfg.B;
    a.BR = ix->BR;
    a.t_min = ix->cfg.min_threshold;
    a.avg_cell = uint32_t((ix->n_points + ix->cfg.B - 1) / ix->cfg.B);
    a.gcells = 1;
    return a;
}

// Candidate buffer: room for one full round of members after a compaction
// to k keys; tune->cap overrides the default when large enough.
void pick_buffer(QArgs &a, int NT, const QueryTuning *tune, size_t extra, size_t *smem_out, int cw, int unroll)
{
    a.kp = pow2_at_least(a.k_max > 1 ? a.k_max : 2);
    // the decode appends freely up to cap - (NT + 32) * unroll, then compacts:
    // that mark must stay above the kp keys a compaction keeps
    const uint32_t cap_min = pow2_at_least(a.kp + uint32_t(NT + 32) * unroll + 1);
    uint32_t cap = (tune && tune->cap) ? pow2_at_least(tune->cap) : 2048;
    if (cap < cap_min) cap = cap_min;
    a.cap = cap;
    size_t smem = qsmem_bytes(a.cap, a.kp, a.BR, a.B, NT, a.L, cw);
    while (smem + extra > 227 * 1024 && a.cap > cap_min) {
        a.cap >>= 1;
        smem = qsmem_bytes(a.cap, a.kp, a.BR, a.B, NT, a.L, cw);
    }
    *smem_out = smem;
    // a level group holds about 4,096 members: one stop check per group
    const uint32_t per = a.avg_cell ? a.avg_cell : 1u;
    uint32_t g = 4096u / per;
    a.gcells = g < 1 ? 1u : (g > uint32_t(NT) ? uint32_t(NT) : g);
}

}  // namespace

int query_launch(flinng_index *ix, const uint32_t *qbuckets, uint32_t nq,
                 const uint32_t *k, uint32_t k_max, uint32_t *out_ids,
                 uint16_t *out_scores, const uint32_t *out_row)
{
    return query_launch_counts(ix, qbuckets, nullptr, 0, nq, k, k_max, out_ids, out_scores, out_row);
}

int query_launch_counts(flinng_index *ix, const uint32_t *qbuckets, const uint16_t *counts, uint32_t max_count,
                        uint32_t nq, const uint32_t *k, uint32_t k_max, uint32_t *out_ids, uint16_t *out_scores,
                        const uint32_t *out_row)
{
    if (nq == 0) return FLINNG_OK;
    QArgs a = make_args(ix, qbuckets, nq);
    int cw = int(ix->cw);
    if (counts) {
        // decode from given counts: levels run to the caller's table total
        a.cnt_in = counts;
        a.L = max_count;
        cw = max_count <= 255 ? 1 : 2;
    }
    a.k = k;
    a.k_max = k_max;
    a.out_ids = out_ids;
    a.out_scores = out_scores;
    a.out_row = out_row;
    // CTA size: when shared memory admits only one or two CTAs per SM (large
    // B*R), wider CTAs keep about 1,024 threads per SM decoding
    int NT = 256;
    size_t smem;
    pick_buffer(a, NT, nullptr, 0, &smem, cw, kPlainUnroll);
    const size_t fit = (228 * 1024) / (smem + 1024);
    if (fit < 4) {
        NT = fit < 2 ? 1024 : 512;
        pick_buffer(a, NT, nullptr, 0, &smem, cw, kPlainUnroll);
    }
    if (smem > 227 * 1024)
        return set_error(FLINNG_ERR_INVALID_ARG,
                         "query: k_max=%u with B*R=%u needs %zu bytes of shared memory (> 227 KB)",
                         k_max, a.BR, smem);
    const void *fn = cw == 1 ? plain_kernel_c1(NT, ix->rw) : plain_kernel_c2(NT, ix->rw);
    FL_TRY(ensure_dyn_smem(fn, smem));
    void *args[] = {&a};
    FL_CUDA(cudaLaunchKernel(fn, dim3(nq), dim3(NT), args, smem, ix->stream));   // one CTA per query
    count_launch();
    return FLINNG_OK;
}

// Everything one fused launch needs: kernel, shape, shared memory and the
// argument blocks (kept in this struct so that a graph node can point at them).
struct FusedPlan {
    QArgs a;
    HArgs h;
    const void *fn;
    int threads;
    size_t smem;
    uint32_t grid;
    void *args[2];
};

static int fused_prepare(flinng_index *ix, const FusedQuery &fq, const uint32_t *k, uint32_t k_max,
                         uint32_t *out_ids, uint16_t *out_scores, const QueryTuning *tune,
                         uint32_t grid_for, FusedPlan *P)
{
    const uint32_t nq = fq.nq;
    const int NT = (tune && (tune->threads == 128 || tune->threads == 512)) ? int(tune->threads) : 256;
    QArgs &a = P->a;
    HArgs &h = P->h;
    a = make_args(ix, nullptr, nq);
    a.k = k;
    a.k_max = k_max;
    a.out_ids = out_ids;
    a.out_scores = out_scores;
    a.out_row = fq.out_row;
    h = HArgs{};
    const bool srp = ix->cfg.metric == FLINNG_COSINE_SRP;
    h.K = ix->cfg.K;
    h.qnext = ix->qnext;
    size_t hash_bytes = size_t((ix->cfg.L + 3) & ~3u) * 4 + 16;
    if (srp) {
        h.x = fq.x;
        h.ldx = fq.ldx;
        h.w = ix->srp_w;
        h.d = ix->cfg.dim;
        h.gamma2 = ix->srp_margin_gamma;
        h.tiny = float(h.d) * ldexpf(1.0f, -146);
        h.gamma64 = ix->srp_gamma64;
        h.stats = ix->stats;
        hash_bytes += size_t(h.d) * 4;
    } else {
        h.q_off = fq.off;
        h.q_el = fq.elems;
        h.nb = ix->P;
        h.da = ix->doph_a;
        h.db = ix->doph_b;
        h.seed = ix->doph_seed;
        h.ba = ix->bucket_a;
        h.bc = ix->bucket_c;
        hash_bytes += size_t(h.nb + (h.nb + 31) / 32) * 4;
    }
    hash_bytes = (hash_bytes + 15) & ~size_t(15);
    // The hash region (query buckets, hash scratch, the query slot) is live
    // only before the decode keeps candidates, so it shares the candidate
    // buffer with the gather's heavy-table list (the buffer's last NT words)
    // when both fit; otherwise it follows the query state.
    size_t qbytes;
    pick_buffer(a, NT, tune, 0, &qbytes, int(ix->cw), 1);
    if (hash_bytes + size_t(NT) * 4 <= size_t(a.cap) * 8) {
        h.hash_off = 0;
        P->smem = qbytes;
    } else {
        pick_buffer(a, NT, tune, hash_bytes, &qbytes, int(ix->cw), 1);
        h.hash_off = qbytes;
        P->smem = qbytes + hash_bytes;
    }
    if (P->smem > 227 * 1024)
        return set_error(FLINNG_ERR_INVALID_ARG, "fused query: %zu bytes of shared memory needed (> 227 KB)", P->smem);
    P->fn = ix->cw == 1 ? fused_kernel_c1(NT, ix->rw, srp) : fused_kernel_c2(NT, ix->rw, srp);
    P->threads = NT;
    FL_TRY(ensure_dyn_smem(P->fn, P->smem));
    int per_sm = 0;
    for (uint32_t i = 0; i < ix->n_occ; ++i) {
        const OccEntry &e = ix->occ[i];
        if (e.fn == P->fn && e.threads == NT && e.smem == P->smem) per_sm = e.per_sm;
    }
    if (!per_sm) {
        FL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, P->fn, NT, P->smem));
        if (per_sm < 1) per_sm = 1;
        const uint32_t slot = ix->n_occ < 8 ? ix->n_occ++ : 7;
        ix->occ[slot] = OccEntry{P->fn, NT, P->smem, per_sm};
    }
    if (!ix->sms) FL_CUDA(cudaDeviceGetAttribute(&ix->sms, cudaDevAttrMultiProcessorCount, ix->device));
    const int sms = ix->sms;
    uint32_t want = (tune && tune->ctas_per_sm) ? tune->ctas_per_sm : uint32_t(per_sm);
    if (want > uint32_t(per_sm)) want = per_sm;
    uint64_t grid = uint64_t(sms) * want;
    if (grid > grid_for) grid = grid_for;
    P->grid = uint32_t(grid ? grid : 1);
    P->args[0] = &P->a;
    P->args[1] = &P->h;
    return FLINNG_OK;
}

int query_fused_launch(flinng_index *ix, const FusedQuery &fq, const uint32_t *k, uint32_t k_max,
                       uint32_t *out_ids, uint16_t *out_scores, const QueryTuning *tune)
{
    if (fq.nq == 0) return FLINNG_OK;
    FusedPlan P;
    FL_TRY(fused_prepare(ix, fq, k, k_max, out_ids, out_scores, tune, fq.nq, &P));
    if (ix->cfg.metric == FLINNG_COSINE_SRP)
        FL_CUDA(cudaMemsetAsync(ix->stats, 0, kStats * sizeof(unsigned long long), ix->stream));
    FL_CUDA(cudaMemsetAsync(ix->qnext, 0, sizeof(uint32_t), ix->stream));
    FL_CUDA(cudaLaunchKernel(P.fn, dim3(P.grid), dim3(P.threads), P.args, P.smem, ix->stream));
    count_launch();
    return FLINNG_OK;
}

// Graph form: one CUDA graph per batch-size class (nq rounded up to a power
// of two) and per result width, built once and replayed; each call only
// rewrites the kernel node's arguments (query and output pointers, nq).
int query_graph_launch(flinng_index *ix, const FusedQuery &fq, const uint32_t *k, uint32_t k_max,
                       uint32_t *out_ids, uint16_t *out_scores, const QueryTuning *tune)
{
    const uint32_t nq = fq.nq;
    if (nq == 0) return FLINNG_OK;
    uint32_t bucket = 0;
    while ((1u << bucket) < nq) ++bucket;
    FusedPlan P;
    FL_TRY(fused_prepare(ix, fq, k, k_max, out_ids, out_scores, tune, 1u << bucket, &P));
    QueryGraph &g = ix->graphs[bucket];
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void *>(P.fn);
    kp.gridDim = dim3(P.grid);
    kp.blockDim = dim3(P.threads);
    kp.sharedMemBytes = (unsigned)P.smem;
    kp.kernelParams = P.args;
    const bool srp = ix->cfg.metric == FLINNG_COSINE_SRP;
    if (!g.exec || g.fn != P.fn || g.smem != P.smem || g.grid != P.grid) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        g = QueryGraph{};
        FL_CUDA(cudaGraphCreate(&g.graph, 0));
        cudaGraphNode_t deps[2];
        int ndep = 0;
        cudaMemsetParams mp{};
        mp.dst = ix->qnext;      // query counter
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = 1;
        mp.height = 1;
        FL_CUDA(cudaGraphAddMemsetNode(&deps[ndep++], g.graph, nullptr, 0, &mp));
        if (srp) {
            mp.dst = ix->stats;
            mp.width = 2 * kStats;   // 64-bit counters
            FL_CUDA(cudaGraphAddMemsetNode(&deps[ndep++], g.graph, nullptr, 0, &mp));
        }
        FL_CUDA(cudaGraphAddKernelNode(&g.node, g.graph, deps, ndep, &kp));
        FL_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
        g.fn = P.fn;
        g.smem = P.smem;
        g.grid = P.grid;
    } else {
        FL_CUDA(cudaGraphExecKernelNodeSetParams(g.exec, g.node, &kp));
    }
    FL_CUDA(cudaGraphLaunch(g.exec, ix->stream));
    count_launch();
    return FLINNG_OK;
}

void destroy_graphs(flinng_index *ix)
{
    for (QueryGraph &g : ix->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        g = QueryGraph{};
    }
}

int counts_launch(flinng_index *ix, const uint32_t *qbuckets, uint32_t nq,
                  uint16_t *out_counts)
{
    if (nq == 0) return FLINNG_OK;
    QArgs a = make_args(ix, qbuckets, nq);
    a.cap = kQTmax / 2;      // the heavy-table list takes the buffer's last kQTmax words
    a.kp = 2;
    a.out_counts = out_counts;
    const size_t smem = qsmem_bytes(a.cap, a.kp, a.BR, a.B, kQTmax, a.L, int(ix->cw));
    const void *fn = ix->cw == 1 ? counts_kernel_c1() : counts_kernel_c2();
    FL_TRY(ensure_dyn_smem(fn, smem));
    void *args[] = {&a};
    FL_CUDA(cudaLaunchKernel(fn, dim3(nq), dim3(kQTmax), args, smem, ix->stream));
    count_launch();
    return FLINNG_OK;
}

const void *plain_kernel_c1(int NT, uint32_t rw) { return plain_kernel_t<1>(NT, rw); }
const void *fused_kernel_c1(int NT, uint32_t rw, bool srp) { return fused_kernel_t<1>(NT, rw, srp); }
const void *counts_kernel_c1() { return (const void *)k_counts<1>; }

}  // namespace flinng
