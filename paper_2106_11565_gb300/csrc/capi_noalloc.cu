// flinng_query_noalloc: the batched query for callers that must not allocate
// device memory (declared in include/flinng.h).
//
// flinng_query keeps its intermediate query buckets (and, for cosine indices,
// the list of projections whose sign needs the fp64 re-check) in a workspace
// that it grows with cudaMalloc when a batch is larger than any before. This
// variant puts that scratch in one fixed array in this file instead, so a
// call makes no cudaMalloc, no cudaFree and no allocating library call.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kScratchBytes) until the process exits. Host code cannot
// use the variable's name as a device address; the address is looked up by
// cudaGetSymbolAddress, with the device current, on the first call made in
// each CUDA context of a device, and cached under that context's unique id.
// A context torn down and made again (cudaDeviceReset, then any call) gets a
// new id and a new module load, so the next call looks the address up again
// instead of reusing a stale one.
#include <cuda.h>

#include <mutex>

#include "internal.cuh"

namespace flinng {
namespace {

constexpr size_t kBucketBytes = size_t(1) << 20;   // query buckets: nq * L uint32
constexpr size_t kHashBytes = size_t(5) << 20;     // SRP re-check counter + list
constexpr size_t kScratchBytes = kBucketBytes + kHashBytes;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_query_scratch[kScratchBytes];

std::mutex g_scratch_mu;
struct ScratchAddr {
    unsigned long long ctx_id;   // unique id of the context the address belongs to (0: none yet)
    void *ptr;
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique id of the current context (ids are never reused within a process).
int current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        FL_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa));
        FL_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb));
        if (!a || !b || qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess)
            return set_error(FLINNG_ERR_CUDA, "query_noalloc: cuCtxGetCurrent / cuCtxGetId not available");
        get_current = reinterpret_cast<CtxGetCurrentFn>(a);
        get_id = reinterpret_cast<CtxGetIdFn>(b);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx)
        return set_error(FLINNG_ERR_CUDA, "query_noalloc: no current CUDA context");
    if (get_id(ctx, id) != CUDA_SUCCESS) return set_error(FLINNG_ERR_CUDA, "query_noalloc: cuCtxGetId failed");
    return FLINNG_OK;
}

// Device address of the scratch array in the current context of `device`
// (which must be the current device).
int scratch_address(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices)
        return set_error(FLINNG_ERR_INVALID_ARG, "query_noalloc: device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    unsigned long long id = 0;
    FL_TRY(current_context_id(&id));
    ScratchAddr &a = g_scratch_addr[device];
    if (a.ctx_id != id || !a.ptr) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_query_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(query scratch)");
        a.ctx_id = id;
        a.ptr = p;
    }
    *out = a.ptr;
    return FLINNG_OK;
}

}  // namespace
}  // namespace flinng

using namespace flinng;

extern "C" int flinng_query_noalloc(flinng_index *idx, const flinng_points *q, uint32_t nq,
                                    const uint32_t *k, uint32_t k_max, uint32_t *out_ids,
                                    uint16_t *out_scores)
{
    if (!idx) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    if (k_max > kMaxKMax) return set_error(FLINNG_ERR_INVALID_ARG, "query_noalloc: k_max > %u", kMaxKMax);
    if (nq == 0) return FLINNG_OK;
    if (!q || !out_ids) return set_error(FLINNG_ERR_INVALID_ARG, "query_noalloc: null q or out_ids");
    if (idx->probes > 1) return set_error(FLINNG_ERR_INVALID_ARG, "query_noalloc: multi-probe counting needs a workspace");
    const bool srp = idx->cfg.metric == FLINNG_COSINE_SRP;
    if (srp ? (!q->x || q->ld < idx->cfg.dim) : (!q->off || !q->elems))
        return set_error(FLINNG_ERR_INVALID_ARG, "query_noalloc: bad points");
    const uint64_t bucket_bytes = uint64_t(nq) * idx->cfg.L * sizeof(uint32_t);
    if (bucket_bytes > kBucketBytes)
        return set_error(FLINNG_ERR_INVALID_ARG,
                         "query_noalloc: nq * L = %llu exceeds the limit of %llu (fixed scratch)",
                         (unsigned long long)(uint64_t(nq) * idx->cfg.L),
                         (unsigned long long)(kBucketBytes / sizeof(uint32_t)));
    if (srp && idx->cfg.precision != FLINNG_PREC_FP32 && srp_workspace_bytes(idx, nq) > kHashBytes)
        return set_error(FLINNG_ERR_INVALID_ARG,
                         "query_noalloc: batch of %u needs %zu bytes of tensor-core scratch (limit %zu)", nq,
                         srp_workspace_bytes(idx, nq), kHashBytes);
    if (srp && 512 + uint64_t(nq) * idx->P * 8 > kHashBytes)
        return set_error(FLINNG_ERR_INVALID_ARG,
                         "query_noalloc: nq * L * K = %llu exceeds the cosine limit of %llu (fixed scratch)",
                         (unsigned long long)(uint64_t(nq) * idx->P),
                         (unsigned long long)((kHashBytes - 512) / 8));
    int dev = -1;
    FL_CUDA(cudaGetDevice(&dev));
    if (dev != idx->device)
        return set_error(FLINNG_ERR_INVALID_ARG, "query_noalloc: the index's device (%d) must be current (%d)",
                         idx->device, dev);
    void *scratch = nullptr;
    FL_TRY(scratch_address(dev, &scratch));
    uint32_t *qb = static_cast<uint32_t *>(scratch);
    void *hws = static_cast<char *>(scratch) + kBucketBytes;
    // buckets are fully written by the hash kernels (SRP clears them first);
    // the re-check counter is cleared by srp_hash before use
    if (srp) {
        FL_TRY(srp_hash(idx, q->x, q->ld, nq, qb, nullptr, hws, kHashBytes));
    } else {
        // the same counters as flinng_query leaves (zero for MinHash)
        FL_CUDA(cudaMemsetAsync(idx->stats, 0, kStats * sizeof(unsigned long long), idx->stream));
        FL_TRY(doph_hash(idx, q->off, q->elems, nq, qb, nullptr));
    }
    return query_launch(idx, qb, nq, k, k_max, out_ids, out_scores);
}
