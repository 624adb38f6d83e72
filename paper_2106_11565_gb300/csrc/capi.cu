// extern "C" entry points of libflinng.so (declared in include/flinng.h):
// argument checks, device memory of the index, host<->device staging, and
// the order of the kernel stages.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"
#include "trace.h"

namespace flinng {

static thread_local char g_err[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void count_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_error(cudaError_t e, const char *what)
{
    const int code = (e == cudaErrorMemoryAllocation) ? FLINNG_ERR_OOM : FLINNG_ERR_CUDA;
    cudaGetLastError();   // clear a non-sticky error
    return set_error(code, "%s: %s", what, cudaGetErrorString(e));
}

int ensure_dyn_smem(const void *fn, size_t smem)
{
    if (smem <= 48 * 1024) return FLINNG_OK;
    struct Limit {
        const void *fn;
        int device;
        size_t smem;
    };
    static std::mutex mu;
    static std::vector<Limit> set;     // per kernel and device: the limit set so far
    std::lock_guard<std::mutex> lock(mu);
    int dev = 0;
    FL_CUDA(cudaGetDevice(&dev));
    for (Limit &e : set)
        if (e.fn == fn && e.device == dev) {
            if (e.smem < smem) {
                FL_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                e.smem = smem;
            }
            return FLINNG_OK;
        }
    FL_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    set.push_back(Limit{fn, dev, smem});
    return FLINNG_OK;
}

int ws_reserve(flinng_index *ix, size_t bytes)
{
    if (bytes <= ix->ws.bytes) return FLINNG_OK;
    // stream-ordered: the old workspace is released after the work already
    // queued on the index's stream and the new one is ready for the next;
    // unlike cudaFree this waits for no other stream (other indices, batches
    // served on other streams)
    if (ix->ws.ptr) {
        FL_CUDA(cudaFreeAsync(ix->ws.ptr, ix->stream));
        ix->device_bytes -= ix->ws.bytes;
        ix->ws.ptr = nullptr;
        ix->ws.bytes = 0;
    }
    const size_t want = bytes + (bytes >> 3);
    FL_CUDA(cudaMallocAsync(&ix->ws.ptr, want, ix->stream));
    ix->ws.bytes = want;
    ix->device_bytes += want;
    return FLINNG_OK;
}

namespace {

template <class T>
int dalloc(flinng_index *ix, T **p, size_t n)
{
    const size_t b = (n ? n : 1) * sizeof(T);
    FL_CUDA(cudaMalloc((void **)p, b));
    ix->device_bytes += b;
    return FLINNG_OK;
}

void free_index(flinng_index *ix)
{
    if (!ix) return;
    destroy_graphs(ix);
    void *ptrs[] = {ix->srp_w, ix->bucket_a, ix->bucket_c, ix->gid, ix->moff, ix->mem, ix->mrec, ix->off,
                    ix->hidx, ix->hbm,
                    ix->cells, ix->cells_tmp, ix->slot_a, ix->slot_b, ix->cell_cnt, ix->flag, ix->qnext,
                    ix->stats, ix->ws.ptr, ix->w_split, ix->w_norm, ix->w_aux, ix->tc_err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (ix->h_flag) cudaFreeHost(ix->h_flag);
    if (ix->ev_fork) cudaEventDestroy(ix->ev_fork);
    if (ix->ev_join) cudaEventDestroy(ix->ev_join);
    if (ix->side) cudaStreamDestroy(ix->side);
    delete ix;
}

int check_config(const flinng_config *c, const flinng_params *p)
{
    if (!c || !p) return set_error(FLINNG_ERR_INVALID_ARG, "create: null config or params");
    if (c->metric != FLINNG_COSINE_SRP && c->metric != FLINNG_JACCARD_DOPH)
        return set_error(FLINNG_ERR_INVALID_ARG, "create: unknown metric %u", c->metric);
    if (c->R < 1 || c->R > 8) return set_error(FLINNG_ERR_INVALID_ARG, "create: R must be in 1..8");
    if (c->B < 1 || uint64_t(c->B) * c->R > 65536)
        return set_error(FLINNG_ERR_INVALID_ARG, "create: need 1 <= B and B*R <= 65536");
    if (c->L < 1 || c->L > kMaxL) return set_error(FLINNG_ERR_INVALID_ARG, "create: L must be in 1..%u", kMaxL);
    if (c->K < 1) return set_error(FLINNG_ERR_INVALID_ARG, "create: K must be >= 1");
    if (c->range_bits < 1 || c->range_bits > 30 || (uint64_t(c->L) << c->range_bits) >= (1ull << 31))
        return set_error(FLINNG_ERR_INVALID_ARG, "create: need 1 <= W <= 30 and L*2^W < 2^31");
    if (c->min_threshold < 1 || c->min_threshold > c->L)
        return set_error(FLINNG_ERR_INVALID_ARG, "create: min_threshold must be in 1..L");
    if (c->precision > FLINNG_PREC_FP8)
        return set_error(FLINNG_ERR_INVALID_ARG, "create: unsupported precision %u", c->precision);
    if (c->precision != FLINNG_PREC_FP32 && c->metric != FLINNG_COSINE_SRP)
        return set_error(FLINNG_ERR_INVALID_ARG, "create: the tensor-core precisions are for cosine indices");
    if ((c->precision == FLINNG_PREC_BF16X2 || c->precision == FLINNG_PREC_BF16) && c->dim % 8 != 0)
        return set_error(FLINNG_ERR_INVALID_ARG, "create: the BF16 tensor-core precisions need dim % 8 == 0");
    if (c->precision == FLINNG_PREC_FP8 && c->dim % 16 != 0)
        return set_error(FLINNG_ERR_INVALID_ARG, "create: the FP8 tensor-core precision needs dim % 16 == 0");
    if (c->capacity < 1 || uint64_t(c->L) * c->R * c->capacity >= (1ull << 32))
        return set_error(FLINNG_ERR_INVALID_ARG, "create: need capacity >= 1 and L*R*capacity < 2^32");
    if (c->metric == FLINNG_COSINE_SRP) {
        if (c->dim < 1 || c->dim > 65536) return set_error(FLINNG_ERR_INVALID_ARG, "create: dim must be in 1..65536");
        if (c->K > 30) return set_error(FLINNG_ERR_INVALID_ARG, "create: SRP needs K <= 30");
        if (c->range_bits != c->K) return set_error(FLINNG_ERR_INVALID_ARG, "create: SRP needs range_bits == K");
        if (!p->srp_w) return set_error(FLINNG_ERR_INVALID_ARG, "create: srp_w is null");
    } else {
        if (uint64_t(c->L) * c->K > 4096) return set_error(FLINNG_ERR_INVALID_ARG, "create: MinHash needs L*K <= 4096");
        if (!p->bucket_a || !p->bucket_c) return set_error(FLINNG_ERR_INVALID_ARG, "create: bucket_a/bucket_c null");
        if ((p->doph_a & 1u) == 0) return set_error(FLINNG_ERR_INVALID_ARG, "create: doph_a must be odd");
    }
    return FLINNG_OK;
}

struct Staged {
    const float *x = nullptr;
    uint64_t ld = 0;
    const uint64_t *off = nullptr;
    const uint32_t *elems = nullptr;
};

// Workspace bytes to stage a host batch of points (0 when on device).
size_t stage_bytes(const flinng_index *ix, const flinng_points *pts, uint64_t n, int on_device)
{
    if (on_device || n == 0) return 0;
    if (ix->cfg.metric == FLINNG_COSINE_SRP) return carve_bytes<float>(n * ix->cfg.dim);
    return carve_bytes<uint64_t>(n + 1) + carve_bytes<uint32_t>(pts->off[n] - pts->off[0]);
}

int check_points(const flinng_index *ix, const flinng_points *pts, uint64_t n, int on_device)
{
    if (n == 0) return FLINNG_OK;
    if (!pts) return set_error(FLINNG_ERR_INVALID_ARG, "points: null");
    if (ix->cfg.metric == FLINNG_COSINE_SRP) {
        if (!pts->x) return set_error(FLINNG_ERR_INVALID_ARG, "points: x is null");
        if (pts->ld < ix->cfg.dim) return set_error(FLINNG_ERR_INVALID_ARG, "points: ld < dim");
    } else {
        if (!pts->off) return set_error(FLINNG_ERR_INVALID_ARG, "points: off is null");
        if (!on_device) {
            if (pts->off[0] != 0) return set_error(FLINNG_ERR_INVALID_ARG, "points: off[0] must be 0");
            for (uint64_t i = 0; i < n; ++i)
                if (pts->off[i + 1] < pts->off[i])
                    return set_error(FLINNG_ERR_INVALID_ARG, "points: off must be non-decreasing");
            if (pts->off[n] > 0 && !pts->elems) return set_error(FLINNG_ERR_INVALID_ARG, "points: elems is null");
        } else if (!pts->elems) {
            return set_error(FLINNG_ERR_INVALID_ARG, "points: elems is null");
        }
    }
    return FLINNG_OK;
}

int stage_points(flinng_index *ix, const flinng_points *pts, uint64_t n, int on_device, Carver &c, Staged &s)
{
    const cudaStream_t st = ix->stream;
    if (ix->cfg.metric == FLINNG_COSINE_SRP) {
        if (on_device || n == 0) {
            s.x = pts ? pts->x : nullptr;
            s.ld = pts ? pts->ld : ix->cfg.dim;
            return FLINNG_OK;
        }
        float *d = c.take<float>(n * ix->cfg.dim);
        FL_CUDA(cudaMemcpy2DAsync(d, ix->cfg.dim * sizeof(float), pts->x, pts->ld * sizeof(float),
                                  ix->cfg.dim * sizeof(float), n, cudaMemcpyHostToDevice, st));
        s.x = d;
        s.ld = ix->cfg.dim;
        return FLINNG_OK;
    }
    if (on_device || n == 0) {
        s.off = pts ? pts->off : nullptr;
        s.elems = pts ? pts->elems : nullptr;
        return FLINNG_OK;
    }
    const uint64_t ne = pts->off[n] - pts->off[0];
    uint64_t *doff = c.take<uint64_t>(n + 1);
    uint32_t *del = c.take<uint32_t>(ne);
    FL_CUDA(cudaMemcpyAsync(doff, pts->off, (n + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    if (ne) FL_CUDA(cudaMemcpyAsync(del, pts->elems, ne * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    s.off = doff;
    s.elems = del;
    return FLINNG_OK;
}

// Device address of a host buffer of the given size when all of it is
// page-locked memory known to CUDA (cudaHostAlloc, cudaHostRegister): kernels
// can then read or write it in place over the host link. nullptr otherwise
// (pageable memory, or a range that leaves the allocation).
template <class T>
T *pinned_view(T *p, size_t bytes)
{
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes a0{}, a1{};
    const char *first = reinterpret_cast<const char *>(p);
    if (cudaPointerGetAttributes(&a0, first) != cudaSuccess ||
        cudaPointerGetAttributes(&a1, first + bytes - 1) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
        return nullptr;
    const char *d0 = static_cast<const char *>(a0.devicePointer), *d1 = static_cast<const char *>(a1.devicePointer);
    if (d1 - d0 != ptrdiff_t(bytes - 1)) return nullptr;
    return reinterpret_cast<T *>(const_cast<char *>(d0));
}

// A host batch read in place by kernels that load each element once (the
// fused query's per-CTA hashing, DOPH hashing): true when its buffers are
// page-locked, with s set to their device addresses; no staging copy.
bool pinned_points(const flinng_index *ix, const flinng_points *pts, uint64_t n, Staged &s)
{
    if (n == 0) return false;
    if (ix->cfg.metric == FLINNG_COSINE_SRP) {
        const float *x = pinned_view(pts->x, ((n - 1) * pts->ld + ix->cfg.dim) * sizeof(float));
        if (!x) return false;
        s.x = x;
        s.ld = pts->ld;
        return true;
    }
    const uint64_t ne = pts->off[n];
    const uint64_t *off = pinned_view(pts->off, (n + 1) * sizeof(uint64_t));
    const uint32_t *el = ne ? pinned_view(pts->elems, ne * sizeof(uint32_t)) : nullptr;
    if (!off || (ne && !el)) return false;
    s.off = off;
    s.elems = el;
    return true;
}

int hash_staged(flinng_index *ix, const Staged &s, uint64_t n, uint32_t *buckets, uint32_t *values,
                float *proj, void *hws, size_t hws_bytes)
{
    if (ix->cfg.metric == FLINNG_COSINE_SRP) return srp_hash(ix, s.x, s.ld, n, buckets, proj, hws, hws_bytes);
    FL_CUDA(cudaMemsetAsync(ix->stats, 0, kStats * sizeof(unsigned long long), ix->stream));
    return doph_hash(ix, s.off, s.elems, n, buckets, values);
}

size_t hash_ws_bytes(const flinng_index *ix, uint64_t n)
{
    return ix->cfg.metric == FLINNG_COSINE_SRP ? srp_workspace_bytes(ix, n) : 0;
}

// Checks buckets < 2^W on the device (sets ix->flag bit 4 otherwise).
__global__ void k_check_buckets(const uint32_t *__restrict__ b, uint64_t n, uint32_t W, uint32_t *flag)
{
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
         t += uint64_t(gridDim.x) * blockDim.x)
        if (b[t] >> W) atomicOr(flag, 4u);
}

int insert_common(flinng_index *ix, const flinng_points *pts, uint64_t n, const uint32_t *perm,
                  int on_device, bool reset, const uint32_t *given_buckets = nullptr,
                  const uint16_t *groups = nullptr)
{
    if (!ix) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    const uint64_t base = reset ? 0 : ix->n_points;
    if (n > ix->cfg.capacity - base)
        return set_error(FLINNG_ERR_CAPACITY, "insert: %llu + %llu points exceed capacity %llu",
                         (unsigned long long)base, (unsigned long long)n,
                         (unsigned long long)ix->cfg.capacity);
    if (!given_buckets) FL_TRY(check_points(ix, pts, n, on_device));
    if (n > 0 && !perm && !groups) return set_error(FLINNG_ERR_INVALID_ARG, "insert: perm is null");
    const cudaStream_t st = ix->stream;
    const uint32_t R = ix->cfg.R, L = ix->cfg.L;
    const size_t need = (given_buckets ? 0 : stage_bytes(ix, pts, n, on_device)) + carve_bytes<uint32_t>(uint64_t(R) * n) +
                        carve_bytes<uint16_t>(uint64_t(R) * n) +
                        carve_bytes<uint32_t>(n * L) + perm_check_workspace_bytes(R, n) +
                        hash_ws_bytes(ix, n) + insert_workspace_bytes(ix, n, reset) + 4096;
    FL_TRY(ws_reserve(ix, need));
    Carver c(ix->ws.ptr, ix->ws.bytes);
    Staged s;
    if (!given_buckets) FL_TRY(stage_points(ix, pts, n, on_device, c, s));
    const uint32_t *dperm = groups ? nullptr : perm;
    const uint16_t *dgroups = groups;
    if (!on_device && n > 0) {
        if (groups) {
            uint16_t *g = c.take<uint16_t>(uint64_t(R) * n);
            FL_CUDA(cudaMemcpyAsync(g, groups, uint64_t(R) * n * sizeof(uint16_t), cudaMemcpyHostToDevice, st));
            dgroups = g;
        } else {
            uint32_t *p = c.take<uint32_t>(uint64_t(R) * n);
            FL_CUDA(cudaMemcpyAsync(p, perm, uint64_t(R) * n * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
            dperm = p;
        }
    }
    uint32_t *buckets = c.take<uint32_t>(n * L);
    void *pws = c.take<char>(perm_check_workspace_bytes(R, n));
    const size_t hb = hash_ws_bytes(ix, n);
    void *hws = c.take<char>(hb);
    void *iws = c.take<char>(insert_workspace_bytes(ix, n, reset));
    // the device checks of the inputs run ahead of the hash (which writes only
    // the workspace); one wait for all of them before the index changes
    FL_CUDA(cudaMemsetAsync(ix->flag, 0, 4, st));
    if (groups) FL_TRY(check_groups(ix, dgroups, n));
    else FL_TRY(check_perm(ix, dperm, n, pws));
    if (given_buckets) {
        if (on_device) {
            FL_CUDA(cudaMemcpyAsync(buckets, given_buckets, n * L * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        } else if (n) {
            FL_CUDA(cudaMemcpyAsync(buckets, given_buckets, n * L * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        }
        if (n) {
            k_check_buckets<<<1024, 256, 0, st>>>(buckets, n * L, ix->cfg.range_bits, ix->flag);
            count_launch();
            FL_CUDA(cudaGetLastError());
        }
    } else {
        FL_TRY(hash_staged(ix, s, n, buckets, nullptr, nullptr, hws, hb));
    }
    FL_TRY(check_result(ix));
    if (reset) {
        ix->n_points = 0;
        ix->n_cells = 0;
    }
    FL_TRY(insert_hashed(ix, buckets, dperm, dgroups, n, iws));
    return FLINNG_OK;
}

}  // namespace
}  // namespace flinng

using namespace flinng;

extern "C" {

const char *flinng_last_error(void) { return g_err; }

uint64_t flinng_kernel_launches(void) { return g_launches.load(); }

int flinng_create(const flinng_config *cfg, const flinng_params *params, void *stream,
                  flinng_index **out)
{
    TraceRange trace_("flinng_create");
    if (!out) return set_error(FLINNG_ERR_INVALID_ARG, "create: out is null");
    *out = nullptr;
    FL_TRY(check_config(cfg, params));
    flinng_index *ix = new flinng_index();   // value-initialised: null pointers, zero counters
    ix->cfg = *cfg;
    ix->stream = (cudaStream_t)stream;
    cudaGetDevice(&ix->device);
    const uint32_t L = cfg->L, K = cfg->K, R = cfg->R;
    ix->P = L * K;
    ix->rp = R == 1 ? 1 : R == 2 ? 2 : R <= 4 ? 4 : 8;
    ix->rw = R == 1 ? 1 : R <= 3 ? 2 : R <= 7 ? 4 : 8;
    ix->cw = cfg->L <= 255 ? 1 : 2;
    ix->BR = cfg->B * R;
    ix->BRw = (ix->BR + 31) / 32;
    // a heavy slot's bitmap (B*R bits) is no larger than its list (2 bytes a cell)
    ix->heavy_min = ix->BR / 16 > 32 ? ix->BR / 16 : 32;
    ix->nslot = uint64_t(L) << cfg->range_bits;
    ix->entries_cap = uint64_t(L) * R * cfg->capacity;
    ix->query_mode = FLINNG_QUERY_FUSED;
    int rc = FLINNG_OK;
#define ALLOC(ptr, n)                                      \
    if (rc == FLINNG_OK) rc = dalloc(ix, &ix->ptr, (n));
    if (cfg->metric == FLINNG_COSINE_SRP) {
        ALLOC(srp_w, size_t(ix->P) * cfg->dim);
    } else {
        ALLOC(bucket_a, size_t(ix->P));
        ALLOC(bucket_c, size_t(L));
    }
    ALLOC(gid, size_t(cfg->capacity) * ix->rp);
    ALLOC(moff, size_t(ix->BR) + 1);
    ALLOC(mem, size_t(R) * cfg->capacity);
    ALLOC(mrec, size_t(ix->rw) * cfg->capacity);
    ALLOC(off, ix->nslot + 1);
    ALLOC(hidx, ix->nslot + 1);
    ALLOC(cells, ix->entries_cap);
    ALLOC(cells_tmp, ix->entries_cap);
    ALLOC(slot_a, ix->nslot + 1);
    ALLOC(slot_b, ix->nslot + 1);
    ALLOC(cell_cnt, size_t(ix->BR) + 1);
    ALLOC(flag, 4);
    ALLOC(qnext, 4);
    ALLOC(stats, kStats);
    ALLOC(tc_err, 4);
#undef ALLOC
    if (rc == FLINNG_OK) {
        cudaError_t e = cudaMallocHost((void **)&ix->h_flag, 16);
        if (e != cudaSuccess) rc = cuda_error(e, "cudaMallocHost");
        else std::memset(ix->h_flag, 0, 16);
    }
    const cudaStream_t st = ix->stream;
    auto chk = [&](cudaError_t e, const char *w) {
        if (rc == FLINNG_OK && e != cudaSuccess) rc = cuda_error(e, w);
    };
    if (rc == FLINNG_OK) {
        if (cfg->metric == FLINNG_COSINE_SRP) {
            chk(cudaMemcpyAsync(ix->srp_w, params->srp_w, size_t(ix->P) * cfg->dim * sizeof(float),
                                cudaMemcpyHostToDevice, st), "copy srp_w");
            const double d = cfg->dim;
            const double g32 = d * std::ldexp(1.0, -24) / (1.0 - d * std::ldexp(1.0, -24));
            ix->srp_margin_gamma = std::nextafter(float(2.0 * g32), INFINITY);
            const double g64 = d * std::ldexp(1.0, -53) / (1.0 - d * std::ldexp(1.0, -53));
            ix->srp_gamma64 = 2.0 * g64;
        } else {
            chk(cudaMemcpyAsync(ix->bucket_a, params->bucket_a, size_t(ix->P) * sizeof(uint64_t),
                                cudaMemcpyHostToDevice, st), "copy bucket_a");
            chk(cudaMemcpyAsync(ix->bucket_c, params->bucket_c, size_t(L) * sizeof(uint64_t),
                                cudaMemcpyHostToDevice, st), "copy bucket_c");
            ix->doph_a = params->doph_a;
            ix->doph_b = params->doph_b;
            ix->doph_seed = params->doph_seed;
        }
        chk(cudaMemsetAsync(ix->off, 0, (ix->nslot + 1) * sizeof(uint32_t), st), "zero off");
        chk(cudaMemsetAsync(ix->hidx, 0xFF, (ix->nslot + 1) * sizeof(uint32_t), st), "clear hidx");
        chk(cudaMemsetAsync(ix->moff, 0, (size_t(ix->BR) + 1) * sizeof(uint32_t), st), "zero moff");
        chk(cudaMemsetAsync(ix->stats, 0, kStats * sizeof(unsigned long long), st), "zero stats");
        chk(cudaMemsetAsync(ix->tc_err, 0, 4, st), "zero tensor-core flag");
        // the insert's second stream and its fork / join events
        chk(cudaStreamCreateWithFlags(&ix->side, cudaStreamNonBlocking), "create side stream");
        chk(cudaEventCreateWithFlags(&ix->ev_fork, cudaEventDisableTiming), "create event");
        chk(cudaEventCreateWithFlags(&ix->ev_join, cudaEventDisableTiming), "create event");
        if (rc == FLINNG_OK && cfg->precision != FLINNG_PREC_FP32) rc = srp_tc_prepare_weights(ix);
        chk(cudaStreamSynchronize(st), "create sync");
    }
    if (rc != FLINNG_OK) {
        free_index(ix);
        return rc;
    }
    *out = ix;
    return FLINNG_OK;
}

int flinng_destroy(flinng_index *idx)
{
    if (!idx) return FLINNG_OK;
    cudaStreamSynchronize(idx->stream);
    free_index(idx);
    return FLINNG_OK;
}

uint64_t flinng_size(const flinng_index *idx) { return idx ? idx->n_points : 0; }

uint64_t flinng_device_bytes(const flinng_index *idx) { return idx ? idx->device_bytes : 0; }

int flinng_set_stream(flinng_index *idx, void *stream)
{
    if (!idx) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    FL_CUDA(cudaStreamSynchronize(idx->stream));
    idx->stream = (cudaStream_t)stream;
    return FLINNG_OK;
}

int flinng_set_tc_wait(flinng_index *idx, uint64_t limit_ns)
{
    if (!idx) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    idx->tc_wait_ns = limit_ns + 1;     // 0 (the overflow of UINT64_MAX) keeps the default
    return FLINNG_OK;
}

int flinng_set_probes(flinng_index *idx, uint32_t probes)
{
    if (!idx) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    if (probes > 1 && idx->cfg.metric != FLINNG_COSINE_SRP)
        return set_error(FLINNG_ERR_INVALID_ARG, "set_probes: multi-probe counting is defined for SRP codes only");
    if (probes > idx->cfg.K + 1)
        return set_error(FLINNG_ERR_INVALID_ARG, "set_probes: %u probes > K + 1 = %u", probes, idx->cfg.K + 1);
    idx->probes = probes;
    return FLINNG_OK;
}

int flinng_set_query_mode(flinng_index *idx, uint32_t mode)
{
    if (!idx) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    if (mode != FLINNG_QUERY_PLAIN && mode != FLINNG_QUERY_FUSED && mode != FLINNG_QUERY_GRAPH)
        return set_error(FLINNG_ERR_INVALID_ARG, "unknown query mode %u", mode);
    idx->query_mode = mode;
    return FLINNG_OK;
}

int flinng_tune_query(flinng_index *idx, const flinng_points *q, uint32_t nq, uint32_t k_max,
                      int on_device, uint32_t *chosen)
{
    TraceRange trace_("flinng_tune_query");
    if (!idx) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    if (nq == 0) return set_error(FLINNG_ERR_INVALID_ARG, "tune: empty batch");
    if (idx->cfg.metric == FLINNG_COSINE_SRP && uint64_t(idx->P) * idx->cfg.dim > (1ull << 18)) {
        // batches of this index are hashed by the GEMM, not by the fused kernel
        if (chosen) chosen[0] = chosen[1] = chosen[2] = 0;
        return FLINNG_OK;
    }
    if (k_max > kMaxKMax) return set_error(FLINNG_ERR_INVALID_ARG, "tune: k_max > %u", kMaxKMax);
    FL_TRY(check_points(idx, q, nq, on_device));
    const cudaStream_t st = idx->stream;
    const size_t need = 4096 + stage_bytes(idx, q, nq, on_device) + carve_bytes<uint32_t>(uint64_t(nq) * k_max) +
                        carve_bytes<uint16_t>(uint64_t(nq) * k_max);
    FL_TRY(ws_reserve(idx, need));
    Carver c(idx->ws.ptr, idx->ws.bytes);
    Staged fs;
    FL_TRY(stage_points(idx, q, nq, on_device, c, fs));
    uint32_t *ids = c.take<uint32_t>(uint64_t(nq) * k_max);
    uint16_t *sc = c.take<uint16_t>(uint64_t(nq) * k_max);
    FusedQuery fq{nq, fs.x, fs.ld, fs.off, fs.elems};
    cudaEvent_t e0, e1;
    FL_CUDA(cudaEventCreate(&e0));
    FL_CUDA(cudaEventCreate(&e1));
    QueryTuning best{};
    float best_ms = 1e30f;
    const uint32_t threads[] = {256, 128, 512};
    const uint32_t cps[] = {0, 4, 2};
    const uint32_t caps[] = {0, 4096, 1024};
    int rc = FLINNG_OK;
    for (uint32_t th : threads)
        for (uint32_t cp : cps)
            for (uint32_t cap : caps) {
                if (rc != FLINNG_OK) break;
                QueryTuning t{th, cp, cap, 1};
                rc = query_fused_launch(idx, fq, nullptr, k_max, ids, sc, &t);
                if (rc != FLINNG_OK) break;
                float ms_min = 1e30f;
                for (int rep = 0; rep < 3 && rc == FLINNG_OK; ++rep) {
                    cudaEventRecord(e0, st);
                    rc = query_fused_launch(idx, fq, nullptr, k_max, ids, sc, &t);
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess) rc = cuda_error(cudaGetLastError(), "tune sync");
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < ms_min) ms_min = ms;
                }
                if (ms_min < best_ms) {
                    best_ms = ms_min;
                    best = t;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != FLINNG_OK) return rc;
    uint32_t bucket = 0;
    while ((1u << bucket) < nq) ++bucket;
    idx->tuning[bucket] = best;
    if (chosen) {
        chosen[0] = best.threads;
        chosen[1] = best.ctas_per_sm;
        chosen[2] = best.cap;
    }
    return FLINNG_OK;
}

int flinng_set_tuning(flinng_index *idx, uint32_t nq, uint32_t threads, uint32_t ctas_per_sm, uint32_t cap)
{
    if (!idx) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    if (nq == 0) return set_error(FLINNG_ERR_INVALID_ARG, "set_tuning: nq is 0");
    if (threads != 128 && threads != 256 && threads != 512)
        return set_error(FLINNG_ERR_INVALID_ARG, "set_tuning: threads must be 128, 256 or 512");
    if (ctas_per_sm > 16) return set_error(FLINNG_ERR_INVALID_ARG, "set_tuning: ctas_per_sm > 16");
    if (cap != 0 && (cap < 64 || cap > 8192 || (cap & (cap - 1)) != 0))
        return set_error(FLINNG_ERR_INVALID_ARG, "set_tuning: cap must be 0 or a power of two in [64, 8192]");
    uint32_t bucket = 0;
    while ((1u << bucket) < nq) ++bucket;
    idx->tuning[bucket] = QueryTuning{threads, ctas_per_sm, cap, 1};
    return FLINNG_OK;
}

int flinng_build(flinng_index *idx, const flinng_points *pts, uint64_t n, const uint32_t *perm,
                 int on_device)
{
    TraceRange trace_("flinng_build");
    return insert_common(idx, pts, n, perm, on_device, true);
}

int flinng_build_buckets(flinng_index *idx, const uint32_t *buckets, uint64_t n, const uint32_t *perm,
                         int on_device)
{
    TraceRange trace_("flinng_build_buckets");
    if (n > 0 && !buckets) return set_error(FLINNG_ERR_INVALID_ARG, "build_buckets: buckets is null");
    return insert_common(idx, nullptr, n, perm, on_device, true, buckets);
}

int flinng_insert(flinng_index *idx, const flinng_points *pts, uint64_t n, const uint32_t *perm,
                  int on_device)
{
    TraceRange trace_("flinng_insert");
    return insert_common(idx, pts, n, perm, on_device, false);
}

int flinng_build_groups(flinng_index *idx, const flinng_points *pts, uint64_t n, const uint16_t *groups,
                        int on_device)
{
    TraceRange trace_("flinng_build_groups");
    if (n > 0 && !groups) return set_error(FLINNG_ERR_INVALID_ARG, "build_groups: groups is null");
    return insert_common(idx, pts, n, nullptr, on_device, true, nullptr, groups);
}

int flinng_insert_groups(flinng_index *idx, const flinng_points *pts, uint64_t n, const uint16_t *groups,
                         int on_device)
{
    TraceRange trace_("flinng_insert_groups");
    if (n > 0 && !groups) return set_error(FLINNG_ERR_INVALID_ARG, "insert_groups: groups is null");
    return insert_common(idx, pts, n, nullptr, on_device, false, nullptr, groups);
}

int flinng_hash(flinng_index *idx, const flinng_points *pts, uint64_t n, uint32_t *out_buckets,
                uint32_t *out_values, float *out_proj, int on_device)
{
    TraceRange trace_("flinng_hash");
    if (!idx) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    if (n > 0 && !out_buckets) return set_error(FLINNG_ERR_INVALID_ARG, "hash: out_buckets is null");
    FL_TRY(check_points(idx, pts, n, on_device));
    const cudaStream_t st = idx->stream;
    const uint32_t L = idx->cfg.L, P = idx->P;
    const bool srp = idx->cfg.metric == FLINNG_COSINE_SRP;
    if (!srp) out_proj = nullptr;
    if (srp) out_values = nullptr;
    size_t need = stage_bytes(idx, pts, n, on_device) + hash_ws_bytes(idx, n) + 4096;
    if (!on_device)
        need += carve_bytes<uint32_t>(n * L) + carve_bytes<uint32_t>(out_values ? n * P : 0) +
                carve_bytes<float>(out_proj ? n * P : 0);
    FL_TRY(ws_reserve(idx, need));
    Carver c(idx->ws.ptr, idx->ws.bytes);
    Staged s;
    FL_TRY(stage_points(idx, pts, n, on_device, c, s));
    uint32_t *b = out_buckets, *v = out_values;
    float *pr = out_proj;
    if (!on_device) {
        b = c.take<uint32_t>(n * L);
        v = out_values ? c.take<uint32_t>(n * P) : nullptr;
        pr = out_proj ? c.take<float>(n * P) : nullptr;
    }
    const size_t hb = hash_ws_bytes(idx, n);
    void *hws = c.take<char>(hb);
    FL_TRY(hash_staged(idx, s, n, b, v, pr, hws, hb));
    if (!on_device && n > 0) {
        FL_CUDA(cudaMemcpyAsync(out_buckets, b, n * L * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        if (out_values) FL_CUDA(cudaMemcpyAsync(out_values, v, n * P * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        if (out_proj) FL_CUDA(cudaMemcpyAsync(out_proj, pr, n * P * sizeof(float), cudaMemcpyDeviceToHost, st));
        FL_CUDA(cudaStreamSynchronize(st));
        // the tensor-core pipeline's timeout flag has landed by now
        if (srp && idx->h_flag[3]) return set_error(FLINNG_ERR_TIMEOUT, "tensor-core SRP: a pipeline wait timed out");
    }
    return FLINNG_OK;
}

static int query_common(flinng_index *idx, const flinng_points *q, const uint32_t *qbuckets,
                        uint32_t nq, const uint32_t *k, uint32_t k_max, uint32_t *out_ids,
                        uint16_t *out_scores, int on_device)
{
    if (!idx) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    if (k_max > kMaxKMax) return set_error(FLINNG_ERR_INVALID_ARG, "query: k_max > %u", kMaxKMax);
    if (nq == 0) return FLINNG_OK;
    if (!out_ids) return set_error(FLINNG_ERR_INVALID_ARG, "query: out_ids is null");
    if (!q && !qbuckets) return set_error(FLINNG_ERR_INVALID_ARG, "query: no queries");
    if (q) FL_TRY(check_points(idx, q, nq, on_device));
    if (k && !on_device)
        for (uint32_t i = 0; i < nq; ++i)
            if (k[i] > k_max) return set_error(FLINNG_ERR_INVALID_ARG, "query: k[%u] = %u > k_max", i, k[i]);
    const cudaStream_t st = idx->stream;
    const uint32_t L = idx->cfg.L;
    const bool probe = idx->probes > 1;
    size_t need = 4096 + carve_bytes<uint32_t>(uint64_t(nq) * L);
    if (probe) need += carve_bytes<uint16_t>(uint64_t(nq) * idx->BR);
    if (q) need += stage_bytes(idx, q, nq, on_device) + hash_ws_bytes(idx, nq);
    if (!on_device)
        need += carve_bytes<uint32_t>(nq) + carve_bytes<uint32_t>(uint64_t(nq) * k_max) +
                carve_bytes<uint16_t>(uint64_t(nq) * k_max);
    FL_TRY(ws_reserve(idx, need));
    Carver c(idx->ws.ptr, idx->ws.bytes);
    uint32_t *qb = nullptr;
    // Per-CTA hashing reads all L*K projection rows for every query: for a
    // large projection matrix the batched GEMM (plain form) hashes far better.
    const bool big_srp = idx->cfg.metric == FLINNG_COSINE_SRP && uint64_t(idx->P) * idx->cfg.dim > (1ull << 18);
    const bool fused = q && !big_srp && !probe &&
                       (idx->query_mode == FLINNG_QUERY_FUSED || idx->query_mode == FLINNG_QUERY_GRAPH);
    Staged fs;
    if (fused) {
        if (on_device || !pinned_points(idx, q, nq, fs)) FL_TRY(stage_points(idx, q, nq, on_device, c, fs));
    } else if (q) {
        Staged s;
        const bool in_place = !on_device && idx->cfg.metric == FLINNG_JACCARD_DOPH && pinned_points(idx, q, nq, s);
        if (!in_place) FL_TRY(stage_points(idx, q, nq, on_device, c, s));
        qb = c.take<uint32_t>(uint64_t(nq) * L);
        const size_t hb = hash_ws_bytes(idx, nq);
        void *hws = c.take<char>(hb);
        FL_TRY(hash_staged(idx, s, nq, qb, nullptr, nullptr, hws, hb));
    } else if (on_device) {
        qb = const_cast<uint32_t *>(qbuckets);
    } else {
        qb = c.take<uint32_t>(uint64_t(nq) * L);
        FL_CUDA(cudaMemcpyAsync(qb, qbuckets, uint64_t(nq) * L * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    }
    const uint32_t *dk = k;
    uint32_t *dids = out_ids;
    uint16_t *dsc = out_scores;
    bool out_in_place = false;
    if (!on_device) {
        if (k) {
            uint32_t *t = c.take<uint32_t>(nq);
            FL_CUDA(cudaMemcpyAsync(t, k, nq * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
            dk = t;
        }
        // page-locked outputs are written in place by the query kernel
        uint32_t *pid = pinned_view(out_ids, size_t(nq) * k_max * sizeof(uint32_t));
        uint16_t *psc = out_scores ? pinned_view(out_scores, size_t(nq) * k_max * sizeof(uint16_t)) : nullptr;
        out_in_place = pid && (!out_scores || psc);
        if (out_in_place) {
            dids = pid;
            dsc = psc;
        } else {
            dids = c.take<uint32_t>(uint64_t(nq) * k_max);
            dsc = out_scores ? c.take<uint16_t>(uint64_t(nq) * k_max) : nullptr;
        }
    }
    if (fused) {
        FusedQuery fq{nq, fs.x, fs.ld, fs.off, fs.elems};
        const QueryTuning *tune = nullptr;
        uint32_t bucket = 0;
        while ((1u << bucket) < nq) ++bucket;
        if (idx->tuning[bucket].valid) tune = &idx->tuning[bucket];
        if (idx->query_mode == FLINNG_QUERY_GRAPH)
            FL_TRY(query_graph_launch(idx, fq, dk, k_max, dids, dsc, tune));
        else
            FL_TRY(query_fused_launch(idx, fq, dk, k_max, dids, dsc, tune));
    } else if (probe) {
        uint16_t *cnt = c.take<uint16_t>(uint64_t(nq) * idx->BR);
        FL_TRY(probe_counts_launch(idx, qb, nq, idx->probes, cnt));
        FL_TRY(query_launch_counts(idx, nullptr, cnt, L, nq, dk, k_max, dids, dsc));
    } else {
        FL_TRY(query_launch(idx, qb, nq, dk, k_max, dids, dsc));
    }
    if (!on_device) {
        if (k_max && !out_in_place) {
            FL_CUDA(cudaMemcpyAsync(out_ids, dids, uint64_t(nq) * k_max * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            if (out_scores)
                FL_CUDA(cudaMemcpyAsync(out_scores, dsc, uint64_t(nq) * k_max * sizeof(uint16_t),
                                        cudaMemcpyDeviceToHost, st));
        }
        FL_CUDA(cudaStreamSynchronize(st));
        if (idx->h_flag[3]) return set_error(FLINNG_ERR_TIMEOUT, "tensor-core SRP: a pipeline wait timed out");
    }
    return FLINNG_OK;
}

int flinng_query(flinng_index *idx, const flinng_points *q, uint32_t nq, const uint32_t *k,
                 uint32_t k_max, uint32_t *out_ids, uint16_t *out_scores, int on_device)
{
    TraceRange trace_("flinng_query");
    if (nq > 0 && !q) return set_error(FLINNG_ERR_INVALID_ARG, "query: q is null");
    return query_common(idx, q, nullptr, nq, k, k_max, out_ids, out_scores, on_device);
}

// Host buckets are checked against 2^W before any copy (the kernels index the
// table's slots with them); device buckets are the caller's to keep in range.
static int check_host_buckets(const flinng_index *idx, const uint32_t *qb, uint64_t n, const char *what)
{
    const uint32_t W = idx->cfg.range_bits;
    for (uint64_t i = 0; i < n; ++i)
        if (qb[i] >> W) return set_error(FLINNG_ERR_INVALID_ARG, "%s: a bucket is >= 2^W", what);
    return FLINNG_OK;
}

int flinng_query_buckets(flinng_index *idx, const uint32_t *qbuckets, uint32_t nq, const uint32_t *k,
                         uint32_t k_max, uint32_t *out_ids, uint16_t *out_scores, int on_device)
{
    TraceRange trace_("flinng_query_buckets");
    if (nq > 0 && !qbuckets) return set_error(FLINNG_ERR_INVALID_ARG, "query: qbuckets is null");
    if (idx && nq > 0 && !on_device)
        FL_TRY(check_host_buckets(idx, qbuckets, uint64_t(nq) * idx->cfg.L, "query_buckets"));
    return query_common(idx, nullptr, qbuckets, nq, k, k_max, out_ids, out_scores, on_device);
}

int flinng_query_counts(flinng_index *idx, const uint16_t *counts, uint32_t nq, uint32_t max_count,
                        const uint32_t *k, uint32_t k_max, uint32_t *out_ids, uint16_t *out_scores, int on_device)
{
    TraceRange trace_("flinng_query_counts");
    if (!idx) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    if (k_max > kMaxKMax) return set_error(FLINNG_ERR_INVALID_ARG, "query_counts: k_max > %u", kMaxKMax);
    if (max_count < 1 || max_count > kMaxL)
        return set_error(FLINNG_ERR_INVALID_ARG, "query_counts: max_count must be in 1..%u", kMaxL);
    if (nq == 0) return FLINNG_OK;
    if (!counts || !out_ids) return set_error(FLINNG_ERR_INVALID_ARG, "query_counts: null counts or out_ids");
    if (k && !on_device)
        for (uint32_t i = 0; i < nq; ++i)
            if (k[i] > k_max) return set_error(FLINNG_ERR_INVALID_ARG, "query_counts: k[%u] = %u > k_max", i, k[i]);
    if (on_device)
        return query_launch_counts(idx, nullptr, counts, max_count, nq, k, k_max, out_ids, out_scores);
    const cudaStream_t st = idx->stream;
    const uint64_t BR = idx->BR;
    FL_TRY(ws_reserve(idx, 4096 + carve_bytes<uint16_t>(nq * BR) + carve_bytes<uint32_t>(nq) +
                               carve_bytes<uint32_t>(uint64_t(nq) * k_max) + carve_bytes<uint16_t>(uint64_t(nq) * k_max)));
    Carver c(idx->ws.ptr, idx->ws.bytes);
    uint16_t *dc = c.take<uint16_t>(nq * BR);
    FL_CUDA(cudaMemcpyAsync(dc, counts, nq * BR * sizeof(uint16_t), cudaMemcpyHostToDevice, st));
    const uint32_t *dk = nullptr;
    if (k) {
        uint32_t *t = c.take<uint32_t>(nq);
        FL_CUDA(cudaMemcpyAsync(t, k, nq * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        dk = t;
    }
    uint32_t *dids = c.take<uint32_t>(uint64_t(nq) * k_max);
    uint16_t *dsc = out_scores ? c.take<uint16_t>(uint64_t(nq) * k_max) : nullptr;
    FL_TRY(query_launch_counts(idx, nullptr, dc, max_count, nq, dk, k_max, dids, dsc));
    if (k_max) {
        FL_CUDA(cudaMemcpyAsync(out_ids, dids, uint64_t(nq) * k_max * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        if (out_scores)
            FL_CUDA(cudaMemcpyAsync(out_scores, dsc, uint64_t(nq) * k_max * sizeof(uint16_t),
                                    cudaMemcpyDeviceToHost, st));
    }
    FL_CUDA(cudaStreamSynchronize(st));
    return FLINNG_OK;
}

int flinng_counts(flinng_index *idx, const uint32_t *qbuckets, uint32_t nq, uint16_t *out_counts,
                  int on_device)
{
    TraceRange trace_("flinng_counts");
    if (!idx) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    if (nq == 0) return FLINNG_OK;
    if (!qbuckets || !out_counts) return set_error(FLINNG_ERR_INVALID_ARG, "counts: null buffer");
    const cudaStream_t st = idx->stream;
    const uint32_t L = idx->cfg.L, BR = idx->BR;
    const uint32_t P = idx->probes;
    if (on_device)
        return P > 1 ? probe_counts_launch(idx, qbuckets, nq, P, out_counts) : counts_launch(idx, qbuckets, nq, out_counts);
    FL_TRY(check_host_buckets(idx, qbuckets, uint64_t(nq) * L, "counts"));
    FL_TRY(ws_reserve(idx, carve_bytes<uint32_t>(uint64_t(nq) * L) + carve_bytes<uint16_t>(uint64_t(nq) * BR) + 1024));
    Carver c(idx->ws.ptr, idx->ws.bytes);
    uint32_t *qb = c.take<uint32_t>(uint64_t(nq) * L);
    uint16_t *oc = c.take<uint16_t>(uint64_t(nq) * BR);
    FL_CUDA(cudaMemcpyAsync(qb, qbuckets, uint64_t(nq) * L * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    FL_TRY(P > 1 ? probe_counts_launch(idx, qb, nq, P, oc) : counts_launch(idx, qb, nq, oc));
    FL_CUDA(cudaMemcpyAsync(out_counts, oc, uint64_t(nq) * BR * sizeof(uint16_t), cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    return FLINNG_OK;
}

int flinng_export(flinng_index *idx, uint32_t *off, uint16_t *cells, uint64_t cells_cap,
                  uint64_t *n_cells, uint16_t *gid)
{
    TraceRange trace_("flinng_export");
    if (!idx) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    const cudaStream_t st = idx->stream;
    FL_CUDA(cudaStreamSynchronize(st));
    if (n_cells) *n_cells = idx->n_cells;
    if (cells && idx->n_cells > cells_cap)
        return set_error(FLINNG_ERR_CAPACITY, "export: %llu cells do not fit in %llu",
                         (unsigned long long)idx->n_cells, (unsigned long long)cells_cap);
    if (off) FL_CUDA(cudaMemcpy(off, idx->off, (idx->nslot + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (cells && idx->n_cells)
        FL_CUDA(cudaMemcpy(cells, idx->cells, idx->n_cells * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    if (gid && idx->n_points) {
        const uint32_t R = idx->cfg.R, rp = idx->rp;
        if (rp == R) {
            FL_CUDA(cudaMemcpy(gid, idx->gid, idx->n_points * R * sizeof(uint16_t), cudaMemcpyDeviceToHost));
        } else {
            FL_CUDA(cudaMemcpy2D(gid, R * sizeof(uint16_t), idx->gid, rp * sizeof(uint16_t),
                                 R * sizeof(uint16_t), idx->n_points, cudaMemcpyDeviceToHost));
        }
    }
    return FLINNG_OK;
}

int flinng_hash_stats(const flinng_index *idx, uint64_t *n_recheck, uint64_t *n_exact)
{
    if (!idx) return set_error(FLINNG_ERR_INVALID_ARG, "index is null");
    unsigned long long h[2] = {0, 0};
    FL_CUDA(cudaStreamSynchronize(idx->stream));
    FL_CUDA(cudaMemcpy(h, idx->stats, sizeof h, cudaMemcpyDeviceToHost));   // [0] undecided, [1] exact
    if (n_recheck) *n_recheck = h[0];
    if (n_exact) *n_exact = h[1];
    return FLINNG_OK;
}

int flinng_hash_counters(const flinng_index *idx, uint64_t *out)
{
    if (!idx || !out) return set_error(FLINNG_ERR_INVALID_ARG, "hash_counters: null argument");
    unsigned long long h[kStats] = {};
    FL_CUDA(cudaStreamSynchronize(idx->stream));
    FL_CUDA(cudaMemcpy(h, idx->stats, sizeof h, cudaMemcpyDeviceToHost));
    for (int i = 0; i < kStats; ++i) out[i] = h[i];
    if (idx->h_flag && idx->h_flag[3])
        return set_error(FLINNG_ERR_TIMEOUT, "tensor-core SRP: a pipeline wait timed out");
    return FLINNG_OK;
}

}  // extern "C"
