// Serving runtime: continuous batching of queries and inserts over several
// device-resident indices (declared in include/flinng.h, flinng_server_*).
//
// The server replays a trace of requests, each admitted when the wall clock
// reaches its arrival time. Pending queries are grouped per index into
// batches (uneven k and set sizes in one launch: per-query k, CSR sets) and
// launched on one of several CUDA streams ("slots"), each with its own
// pinned staging buffers and device scratch, so batches of different indices
// - and further batches of the same index - overlap on the device while
// earlier ones run. A slot is reused as soon as its batch's event completes;
// its results are copied back and the requests marked done. An insert runs
// once every batch in flight on its index has finished, in arrival order
// with that index's queries (later queries see the new points), on a thread
// of its own so that the other indices keep being served.
// Admission is by HBM budget: an index is accepted only if its device
// memory plus the slots' scratch fits, an insert only if the index has
// capacity left and stays within the budget.
// Staging: where the GPU can read any host memory (pageable memory access,
// e.g. over NVLink-C2C on Grace systems), a batch's inputs are gathered by a
// kernel straight from the requests' own buffers, and the host only writes a
// small descriptor per request; the query kernel then writes each result row
// straight into the caller's output buffers too. Elsewhere the host copies
// the inputs into pinned staging first and the results back out of it.
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <vector>

#include "internal.cuh"
#include "trace.h"

namespace flinng {
namespace {

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t start = nullptr;   // recorded before the batch's first copy (timing)
    cudaEvent_t done = nullptr;    // recorded after its results reach the host staging (timing)
    bool busy = false;
    bool direct = false;           // the batch's results go straight to the caller's buffers
    uint32_t index = 0;
    std::vector<uint64_t> reqs;
    // device scratch
    void *dscratch = nullptr;
    size_t dbytes = 0;
    // pinned host staging
    void *hstage = nullptr;
    size_t hbytes = 0;
};

// An insert runs on a thread of its own (flinng_insert on the index's own
// stream) while the scheduling thread keeps serving the other indices; the
// index takes no batch until it is done.
struct InsertJob {
    std::thread th;
    std::atomic<bool> finished{false};
    bool active = false;
    int rc = FLINNG_OK;
    uint64_t req = 0;
};

struct ServerIndex {
    flinng_index *ix;
    uint32_t version = 0;      // inserts applied
    uint32_t inflight = 0;     // batches on the device
    std::deque<uint64_t> pending;
    std::unique_ptr<InsertJob> job{new InsertJob()};
};

// Per-slot layout (device and host mirror): counter + stats, the batch
// header (gather descriptors, input offsets, per-query k: one copy), query
// input (rows or CSR), query buckets, re-check list, outputs.
struct Layout {
    size_t hdr, in_el, qb, srp, ids, sc, total;
};

// Offsets inside the header region for a batch of nb queries: descriptors,
// then nb + 1 input offsets, then nb values of k; `bytes` is what one copy
// moves to the device.
struct HdrOff {
    size_t desc, in_off, k, row, bytes;
};

// One request's input for the device gather: 4-byte words from a host
// address to a word offset of the batch's input.
struct GatherDesc {
    uint64_t src;
    uint64_t dst;
    uint64_t n;
};

// A CTA per request; each thread issues all its loads from host memory (up to
// kGatherUnroll per pass) before storing, so a request of up to
// kGatherUnroll * blockDim elements costs one round trip over the link.
constexpr int kGatherUnroll = 4;

__global__ void k_gather_requests(const GatherDesc *__restrict__ desc, uint32_t nb, uint32_t *__restrict__ dst)
{
    for (uint32_t i = blockIdx.x; i < nb; i += gridDim.x) {
        const GatherDesc g = desc[i];
        const uint32_t *src = reinterpret_cast<const uint32_t *>(g.src);
        for (uint64_t t0 = threadIdx.x; t0 < g.n; t0 += uint64_t(kGatherUnroll) * blockDim.x) {
            uint32_t v[kGatherUnroll];
#pragma unroll
            for (int u = 0; u < kGatherUnroll; ++u) {
                const uint64_t t = t0 + uint64_t(u) * blockDim.x;
                v[u] = t < g.n ? src[t] : 0u;
            }
#pragma unroll
            for (int u = 0; u < kGatherUnroll; ++u) {
                const uint64_t t = t0 + uint64_t(u) * blockDim.x;
                if (t < g.n) dst[g.dst + t] = v[u];
            }
        }
    }
}

}  // namespace
}  // namespace flinng

struct flinng_server {
    flinng_server_config cfg;
    std::vector<flinng::ServerIndex> idx;
    std::vector<flinng::Slot> slots;
    uint64_t bytes_used = 0;
    // sizes the slots are laid out for (maximum over the indices)
    uint32_t max_L = 0, max_dim = 0;
    uint64_t max_P = 0;
    bool device_gather = false;   // the GPU reads requests' host buffers directly
    cudaEvent_t ref = nullptr;    // recorded when a replay begins: origin of the device times
};

namespace flinng {
namespace {

double now_s()
{
    using C = std::chrono::steady_clock;
    return std::chrono::duration<double>(C::now().time_since_epoch()).count();
}

HdrOff hdr_for(uint64_t nb)
{
    Carver c(nullptr, ~size_t(0));
    HdrOff h{};
    h.desc = (size_t)c.take<GatherDesc>(nb);
    h.in_off = (size_t)c.take<uint64_t>(nb + 1);
    h.k = (size_t)c.take<uint32_t>(nb);
    h.row = (size_t)c.take<uint32_t>(nb);
    h.bytes = c.used;
    return h;
}

Layout layout_for(const flinng_server *srv)
{
    const uint64_t nb = srv->cfg.max_batch, km = srv->cfg.k_max;
    Layout L{};
    Carver c(nullptr, ~size_t(0));
    c.take<unsigned long long>(8);                                  // query counter, 4 hash counters
    L.hdr = (size_t)c.take<char>(hdr_for(nb).bytes);
    const uint64_t in_floats = nb * uint64_t(srv->max_dim);
    const uint64_t in_elems = uint64_t(srv->cfg.max_batch_elems);
    L.in_el = (size_t)c.take<uint32_t>(in_floats > in_elems ? in_floats : in_elems);
    L.qb = (size_t)c.take<uint32_t>(nb * srv->max_L);
    // re-check lists (fp32 path) or the tensor-core split operands and lists
    L.srp = (size_t)c.take<unsigned long long>(2 * nb * srv->max_P + 64 + nb * srv->max_dim / 2 + 2 * nb + 1024);
    L.ids = (size_t)c.take<uint32_t>(nb * km);
    L.sc = (size_t)c.take<uint16_t>(nb * km);
    L.total = c.used + 256;
    return L;
}

int size_slots(flinng_server *srv, size_t dbytes, size_t hbytes)
{
    for (Slot &s : srv->slots) {
        if (s.dbytes < dbytes) {
            if (s.dscratch) cudaFree(s.dscratch);
            s.dscratch = nullptr;
            FL_CUDA(cudaMalloc(&s.dscratch, dbytes));
            s.dbytes = dbytes;
        }
        if (s.hbytes < hbytes) {
            if (s.hstage) cudaFreeHost(s.hstage);
            s.hstage = nullptr;
            FL_CUDA(cudaMallocHost(&s.hstage, hbytes));
            s.hbytes = hbytes;
        }
    }
    return FLINNG_OK;
}

// Launch the queries in slot.reqs against index si on the slot's stream.
// Where the device reads host memory directly, the query kernel writes each
// result row straight into the caller's out_ids / out_scores (row = request
// index); otherwise results come back through the slot's pinned staging.
int launch_batch(flinng_server *srv, Slot &slot, const flinng_request *reqs, uint32_t *out_ids,
                 uint16_t *out_scores)
{
    TraceRange trace_("server batch");
    ServerIndex &S = srv->idx[slot.index];
    flinng_index *ix = S.ix;
    const Layout Lo = layout_for(srv);
    const uint32_t nb = (uint32_t)slot.reqs.size();
    const uint32_t km = srv->cfg.k_max;
    const bool srp = ix->cfg.metric == FLINNG_COSINE_SRP;
    char *h = static_cast<char *>(slot.hstage);
    char *d = static_cast<char *>(slot.dscratch);
    const HdrOff ho_ = hdr_for(nb);
    char *hh = h + Lo.hdr;
    char *dh = d + Lo.hdr;
    uint32_t *hk = reinterpret_cast<uint32_t *>(hh + ho_.k);
    uint32_t *hr = reinterpret_cast<uint32_t *>(hh + ho_.row);
    uint64_t *ho = reinterpret_cast<uint64_t *>(hh + ho_.in_off);
    const bool big_srp = srp && uint64_t(ix->P) * ix->cfg.dim > (1ull << 18);
    slot.direct = srv->device_gather;
    FL_CUDA(cudaEventRecord(slot.start, slot.stream));
    ho[0] = 0;
    if (srv->device_gather) {
        // descriptors only: the gather kernel reads each request's buffer
        GatherDesc *hd = reinterpret_cast<GatherDesc *>(hh + ho_.desc);
        for (uint32_t i = 0; i < nb; ++i) {
            const flinng_request &r = reqs[slot.reqs[i]];
            hk[i] = r.k;
            hr[i] = uint32_t(slot.reqs[i]);
            const uint64_t n = srp ? uint64_t(ix->cfg.dim) : r.n;
            hd[i] = GatherDesc{reinterpret_cast<uint64_t>(r.data), ho[i], r.data ? n : 0};
            ho[i + 1] = ho[i] + n;
        }
        // header (descriptors, offsets, k) in one copy
        FL_CUDA(cudaMemcpyAsync(dh, hh, ho_.bytes, cudaMemcpyHostToDevice, slot.stream));
        const unsigned grid = nb < 152u * 8u ? nb : 152u * 8u;
        k_gather_requests<<<grid, 256, 0, slot.stream>>>(reinterpret_cast<const GatherDesc *>(dh + ho_.desc), nb,
                                                          reinterpret_cast<uint32_t *>(d + Lo.in_el));
        count_launch();
        FL_CUDA(cudaGetLastError());
    } else {
        size_t in_bytes;
        if (srp) {
            float *hx = reinterpret_cast<float *>(h + Lo.in_el);
            for (uint32_t i = 0; i < nb; ++i) {
                const flinng_request &r = reqs[slot.reqs[i]];
                hk[i] = r.k;
                std::memcpy(hx + size_t(i) * ix->cfg.dim, r.data, size_t(ix->cfg.dim) * sizeof(float));
            }
            in_bytes = size_t(nb) * ix->cfg.dim * sizeof(float);
        } else {
            uint32_t *he = reinterpret_cast<uint32_t *>(h + Lo.in_el);
            for (uint32_t i = 0; i < nb; ++i) {
                const flinng_request &r = reqs[slot.reqs[i]];
                hk[i] = r.k;
                std::memcpy(he + ho[i], r.data, size_t(r.n) * sizeof(uint32_t));
                ho[i + 1] = ho[i] + r.n;
            }
            in_bytes = size_t(ho[nb]) * sizeof(uint32_t);
        }
        FL_CUDA(cudaMemcpyAsync(dh, hh, ho_.bytes, cudaMemcpyHostToDevice, slot.stream));
        if (in_bytes)
            FL_CUDA(cudaMemcpyAsync(d + Lo.in_el, h + Lo.in_el, in_bytes, cudaMemcpyHostToDevice, slot.stream));
    }
    if (ix->probes > 1) return set_error(FLINNG_ERR_INVALID_ARG, "server: multi-probe indices are not served");
    // bind the slot's stream and scratch to the index for these launches
    const cudaStream_t s0 = ix->stream;
    uint32_t *qn0 = ix->qnext;
    unsigned long long *st0 = ix->stats;
    ix->stream = slot.stream;
    ix->qnext = reinterpret_cast<uint32_t *>(d);
    ix->stats = reinterpret_cast<unsigned long long *>(d) + 2;
    int rc = FLINNG_OK;
    const uint32_t *dk = reinterpret_cast<const uint32_t *>(dh + ho_.k);
    uint32_t *dids = reinterpret_cast<uint32_t *>(d + Lo.ids);
    uint16_t *dsc = reinterpret_cast<uint16_t *>(d + Lo.sc);
    if (big_srp) {
        uint32_t *qb = reinterpret_cast<uint32_t *>(d + Lo.qb);
        rc = srp_hash(ix, reinterpret_cast<const float *>(d + Lo.in_el), ix->cfg.dim, nb, qb, nullptr, d + Lo.srp,
                      (2 * size_t(nb) * ix->P + 64) * 8);
        if (slot.direct) {
            dids = out_ids;
            dsc = out_scores;
        }
        if (rc == FLINNG_OK)
            rc = query_launch(ix, qb, nb, dk, km, dids, dsc,
                              slot.direct ? reinterpret_cast<const uint32_t *>(dh + ho_.row) : nullptr);
    } else {
        FusedQuery fq{nb, reinterpret_cast<const float *>(d + Lo.in_el), ix->cfg.dim,
                      reinterpret_cast<const uint64_t *>(dh + ho_.in_off), reinterpret_cast<const uint32_t *>(d + Lo.in_el)};
        if (slot.direct) {
            fq.out_row = reinterpret_cast<const uint32_t *>(dh + ho_.row);
            dids = out_ids;
            dsc = out_scores;
        }
        uint32_t bucket = 0;
        while ((1u << bucket) < nb) ++bucket;
        const QueryTuning *tune = ix->tuning[bucket].valid ? &ix->tuning[bucket] : nullptr;
        rc = query_fused_launch(ix, fq, dk, km, dids, dsc, tune);
    }
    ix->stream = s0;
    ix->qnext = qn0;
    ix->stats = st0;
    FL_TRY(rc);
    if (!slot.direct) {
        FL_CUDA(cudaMemcpyAsync(h + Lo.ids, d + Lo.ids, size_t(nb) * km * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                slot.stream));
        FL_CUDA(cudaMemcpyAsync(h + Lo.sc, d + Lo.sc, size_t(nb) * km * sizeof(uint16_t), cudaMemcpyDeviceToHost,
                                slot.stream));
    }
    FL_CUDA(cudaEventRecord(slot.done, slot.stream));
    return FLINNG_OK;
}

}  // namespace
}  // namespace flinng

using namespace flinng;

extern "C" {

int flinng_server_create(const flinng_server_config *cfg, flinng_server **out)
{
    if (!cfg || !out) return set_error(FLINNG_ERR_INVALID_ARG, "server: null argument");
    *out = nullptr;
    if (cfg->n_slots < 1 || cfg->n_slots > 64 || cfg->max_batch < 1 || cfg->k_max < 1 || cfg->k_max > kMaxKMax)
        return set_error(FLINNG_ERR_INVALID_ARG, "server: need 1 <= n_slots <= 64, max_batch >= 1, 1 <= k_max <= %u",
                         kMaxKMax);
    flinng_server *srv = new flinng_server();
    srv->cfg = *cfg;
    {
        int dev = 0, pageable = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) == cudaSuccess)
            srv->device_gather = pageable != 0;
    }
    srv->slots.resize(cfg->n_slots);
    {
        const cudaError_t e = cudaEventCreate(&srv->ref);
        if (e != cudaSuccess) {
            flinng_server_destroy(srv);
            return cuda_error(e, "server events");
        }
    }
    for (Slot &s : srv->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&s.start);
        if (e == cudaSuccess) e = cudaEventCreate(&s.done);
        if (e != cudaSuccess) {
            flinng_server_destroy(srv);
            return cuda_error(e, "server streams");
        }
    }
    *out = srv;
    return FLINNG_OK;
}

int flinng_server_destroy(flinng_server *srv)
{
    if (!srv) return FLINNG_OK;
    for (Slot &s : srv->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.start) cudaEventDestroy(s.start);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.dscratch) cudaFree(s.dscratch);
        if (s.hstage) cudaFreeHost(s.hstage);
    }
    if (srv->ref) cudaEventDestroy(srv->ref);
    delete srv;
    return FLINNG_OK;
}

int flinng_server_add_index(flinng_server *srv, flinng_index *ix, uint32_t *index_id)
{
    if (!srv || !ix) return set_error(FLINNG_ERR_INVALID_ARG, "server: null argument");
    if (ix->probes > 1) return set_error(FLINNG_ERR_INVALID_ARG, "server: multi-probe indices are not served");
    const uint32_t L0 = srv->max_L, d0 = srv->max_dim;
    const uint64_t P0 = srv->max_P;
    if (ix->cfg.L > srv->max_L) srv->max_L = ix->cfg.L;
    if (ix->cfg.metric == FLINNG_COSINE_SRP) {
        if (ix->cfg.dim > srv->max_dim) srv->max_dim = ix->cfg.dim;
        if (ix->P > srv->max_P) srv->max_P = ix->P;
    }
    const Layout Lo = layout_for(srv);
    const uint64_t slots_bytes = uint64_t(Lo.total) * srv->slots.size();
    const uint64_t need = flinng_device_bytes(ix) + slots_bytes;
    uint64_t others = 0;
    for (const ServerIndex &S : srv->idx) others += flinng_device_bytes(S.ix);
    if (others + need > srv->cfg.hbm_budget) {
        srv->max_L = L0;
        srv->max_dim = d0;
        srv->max_P = P0;
        return set_error(FLINNG_ERR_OOM, "server: index needs %llu bytes, %llu of the %llu-byte budget are taken",
                         (unsigned long long)need, (unsigned long long)others,
                         (unsigned long long)srv->cfg.hbm_budget);
    }
    FL_TRY(size_slots(srv, Lo.total, Lo.total));
    srv->bytes_used = others + need;
    ServerIndex S;
    S.ix = ix;
    srv->idx.push_back(std::move(S));
    if (index_id) *index_id = uint32_t(srv->idx.size() - 1);
    return FLINNG_OK;
}

uint64_t flinng_server_device_bytes(const flinng_server *srv) { return srv ? srv->bytes_used : 0; }

int flinng_server_replay(flinng_server *srv, const flinng_request *reqs, uint64_t n, uint32_t *out_ids,
                         uint16_t *out_scores, flinng_request_result *res)
{
    TraceRange trace_("flinng_server_replay");
    if (!srv || (n && (!reqs || !out_ids || !res))) return set_error(FLINNG_ERR_INVALID_ARG, "replay: null argument");
    if (n > 0xFFFFFFFFull) return set_error(FLINNG_ERR_INVALID_ARG, "replay: more than 2^32 - 1 requests");
    const uint32_t km = srv->cfg.k_max;
    const Layout Lo = layout_for(srv);
    for (uint64_t i = 0; i < n; ++i) {
        const flinng_request &r = reqs[i];
        if (r.index >= srv->idx.size()) return set_error(FLINNG_ERR_INVALID_ARG, "replay: request %llu: bad index", (unsigned long long)i);
        if (i && r.arrival_s < reqs[i - 1].arrival_s)
            return set_error(FLINNG_ERR_INVALID_ARG, "replay: arrivals must be non-decreasing");
        if (r.kind == FLINNG_REQ_QUERY) {
            if (r.k > km) return set_error(FLINNG_ERR_INVALID_ARG, "replay: request %llu: k > k_max", (unsigned long long)i);
            const flinng_index *ix = srv->idx[r.index].ix;
            if (!r.data && (ix->cfg.metric == FLINNG_COSINE_SRP || r.n))
                return set_error(FLINNG_ERR_INVALID_ARG, "replay: request %llu: no data", (unsigned long long)i);
            if (ix->cfg.metric != FLINNG_COSINE_SRP && r.n > srv->cfg.max_batch_elems)
                return set_error(FLINNG_ERR_INVALID_ARG, "replay: request %llu: set larger than max_batch_elems",
                                 (unsigned long long)i);
        } else if (r.kind != FLINNG_REQ_INSERT) {
            return set_error(FLINNG_ERR_INVALID_ARG, "replay: request %llu: unknown kind", (unsigned long long)i);
        }
        std::memset(&res[i], 0, sizeof(res[i]));
    }
    for (ServerIndex &S : srv->idx) {
        S.pending.clear();
        S.inflight = 0;
        if (S.job->th.joinable()) S.job->th.join();
        S.job->active = false;
    }
    // an early return (a failed launch) still waits for running inserts
    struct JoinInserts {
        flinng_server *srv;
        ~JoinInserts()
        {
            for (ServerIndex &S : srv->idx)
                if (S.job->th.joinable()) S.job->th.join();
        }
    } join_inserts{srv};
    if (n) FL_CUDA(cudaEventRecord(srv->ref, srv->slots[0].stream));
    const double t0 = now_s();
    uint64_t next = 0, done = 0, batches = 0;
    size_t rr = 0;
    while (done < n) {
        double now = now_s() - t0;
        while (next < n && reqs[next].arrival_s <= now) {
            res[next].t_admit = now;
            srv->idx[reqs[next].index].pending.push_back(next);
            ++next;
        }
        bool progress = false;
        // harvest finished batches
        for (size_t si = 0; si < srv->slots.size(); ++si) {
            Slot &s = srv->slots[si];
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) return cuda_error(q, "replay: batch");
            const double t = now_s() - t0;
            // device times of the batch (both events and the origin have completed)
            float ms0 = -1.0f, ms1 = -1.0f;
            if (cudaEventElapsedTime(&ms0, srv->ref, s.start) != cudaSuccess ||
                cudaEventElapsedTime(&ms1, srv->ref, s.done) != cudaSuccess) {
                ms0 = ms1 = -1.0f;
                (void)cudaGetLastError();   // not sticky: clear it so later launch checks stay clean
            }
            const char *h = static_cast<const char *>(s.hstage);
            for (size_t i = 0; i < s.reqs.size(); ++i) {
                const uint64_t r = s.reqs[i];
                if (!s.direct) {
                    std::memcpy(out_ids + r * km, h + Lo.ids + i * km * sizeof(uint32_t), km * sizeof(uint32_t));
                    if (out_scores)
                        std::memcpy(out_scores + r * km, h + Lo.sc + i * km * sizeof(uint16_t),
                                    km * sizeof(uint16_t));
                }
                res[r].t_done = t;
                res[r].status = FLINNG_OK;
                res[r].slot = uint32_t(si);
                res[r].d_start = ms0 * 1e-3;
                res[r].d_done = ms1 * 1e-3;
            }
            done += s.reqs.size();
            srv->idx[s.index].inflight--;
            s.busy = false;
            s.reqs.clear();
            progress = true;
        }
        // inserts that finished on their threads
        for (ServerIndex &S : srv->idx) {
            InsertJob &J = *S.job;
            if (!J.active || !J.finished.load(std::memory_order_acquire)) continue;
            J.th.join();
            J.active = false;
            res[J.req].status = uint32_t(J.rc);
            res[J.req].t_done = now_s() - t0;
            if (J.rc == FLINNG_OK) {
                ++S.version;
                uint64_t total = 0;
                for (const ServerIndex &T : srv->idx) total += flinng_device_bytes(T.ix);
                srv->bytes_used = total + uint64_t(Lo.total) * srv->slots.size();
            }
            ++done;
            progress = true;
        }
        // an insert at the head of an idle index starts on its own thread
        for (ServerIndex &S : srv->idx) {
            InsertJob &J = *S.job;
            if (J.active || S.pending.empty() || reqs[S.pending.front()].kind != FLINNG_REQ_INSERT || S.inflight)
                continue;
            const uint64_t r = S.pending.front();
            S.pending.pop_front();
            const flinng_request &q = reqs[r];
            res[r].t_start = now_s() - t0;
            res[r].version = S.version;
            progress = true;
            if (S.ix->n_points + q.n > S.ix->cfg.capacity) {
                res[r].status = FLINNG_ERR_CAPACITY;
                res[r].t_done = now_s() - t0;
                ++done;
                continue;
            }
            J.active = true;
            J.req = r;
            J.rc = FLINNG_OK;
            J.finished.store(false, std::memory_order_relaxed);
            flinng_index *ix = S.ix;
            InsertJob *jp = &J;
            J.th = std::thread([ix, jp, &q]() {
                jp->rc = flinng_insert(ix, static_cast<const flinng_points *>(q.data), q.n, q.perm, (int)q.on_device);
                jp->finished.store(true, std::memory_order_release);
            });
        }
        // fill free slots with batches, indices in turn
        for (Slot &s : srv->slots) {
            if (s.busy) continue;
            bool launched = false;
            for (size_t tries = 0; tries < srv->idx.size() && !launched; ++tries) {
                const size_t ii = (rr + tries) % srv->idx.size();
                ServerIndex &S = srv->idx[ii];
                if (S.job->active || S.pending.empty() || reqs[S.pending.front()].kind != FLINNG_REQ_QUERY) continue;
                const bool sets = S.ix->cfg.metric != FLINNG_COSINE_SRP;
                uint64_t elems = 0;
                s.index = uint32_t(ii);
                const double t = now_s() - t0;
                while (!S.pending.empty() && s.reqs.size() < srv->cfg.max_batch) {
                    const uint64_t r = S.pending.front();
                    if (reqs[r].kind != FLINNG_REQ_QUERY) break;
                    if (sets && elems + reqs[r].n > srv->cfg.max_batch_elems) break;
                    elems += sets ? reqs[r].n : 0;
                    S.pending.pop_front();
                    s.reqs.push_back(r);
                    res[r].t_start = t;
                    res[r].version = S.version;
                    res[r].batch = uint32_t(batches);
                }
                FL_TRY(launch_batch(srv, s, reqs, out_ids, out_scores));
                s.busy = true;
                S.inflight++;
                ++batches;
                launched = true;
                progress = true;
                rr = ii + 1;
            }
        }
        if (!progress) {
            bool any_busy = false;
            for (const Slot &s : srv->slots) any_busy |= s.busy;
            for (const ServerIndex &S : srv->idx) any_busy |= S.job->active;
            if (!any_busy && next < n) {
                const double wait = reqs[next].arrival_s - (now_s() - t0);
                if (wait > 200e-6) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 100e-6));
            }
        }
    }
    return FLINNG_OK;
}

}  // extern "C"

extern "C" int flinng_server_staging(const flinng_server *srv)
{
    if (!srv) {
        set_error(FLINNG_ERR_INVALID_ARG, "server: null argument");
        return -FLINNG_ERR_INVALID_ARG;
    }
    return srv->device_gather ? 1 : 0;
}
