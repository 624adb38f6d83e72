// Internal declarations of the FLINNG CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "flinng.h"

namespace flinng {

constexpr uint32_t kEmpty32 = 0xFFFFFFFFu;
constexpr uint64_t kKeyNone = ~0ull;
constexpr uint32_t kMaxKMax = 1024;
constexpr uint32_t kMaxL = 4095;          // 12-bit scores in the query keys
constexpr uint32_t kDophMaxAttempts = 4096;
// hash counters: [0] undecided after the first pass, [1] exact accumulator,
// [2] fp64 re-checks, [3] compensated fp32 re-checks, [4] first-pass signs
// that a re-check reversed (flips)
constexpr int kStats = 5;
// re-check list entries: bit 63 the first pass's tentative sign (p > 0),
// bits 20..62 the row, bits 0..19 the projection
constexpr unsigned long long kEntSign = 1ull << 63;
__host__ __device__ inline uint64_t ent_row(unsigned long long e) { return (e >> 20) & ((1ull << 43) - 1); }
__host__ __device__ inline uint32_t ent_col(unsigned long long e) { return uint32_t(e & 0xFFFFF); }

// Error plumbing: every internal step returns an int status and leaves a
// message in the thread-local buffer.
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);

#define FL_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::flinng::cuda_error(e_, #call);  \
    } while (0)

#define FL_TRY(call)                      \
    do {                                  \
        int rc_ = (call);                 \
        if (rc_ != FLINNG_OK) return rc_; \
    } while (0)

// Grow-only device scratch region.
struct Workspace {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct QueryTuning {
    uint32_t threads;        // CTA size: 128, 256 or 512 (0: 256)
    uint32_t ctas_per_sm;    // 0: occupancy limit
    uint32_t cap;            // candidate buffer entries; 0: default
    uint32_t valid;
};

// Occupancy of one fused-kernel launch shape, kept per index so that a
// launch does not query it again.
struct OccEntry {
    const void *fn;
    int threads;
    size_t smem;
    int per_sm;
};

struct QueryGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node = nullptr;
    const void *fn = nullptr;
    size_t smem = 0;
    uint32_t grid = 0;
};

// Bump allocator over a workspace, 256-byte aligned slices.
struct Carver {
    char *base;
    size_t cap, used = 0;
    Carver(void *p, size_t c) : base((char *)p), cap(c) {}
    template <class T>
    T *take(size_t n) {
        size_t a = (used + 255) & ~size_t(255);
        used = a + n * sizeof(T);
        return (T *)(base + a);
    }
};

template <class T>
inline size_t carve_bytes(size_t n) { return ((n * sizeof(T) + 255) & ~size_t(255)) + 256; }

}  // namespace flinng

struct flinng_index {
    flinng_config cfg;
    cudaStream_t stream;
    int device;

    // hash parameters (device copies)
    float *srp_w;          // P x dim
    uint64_t *bucket_a;    // L x K
    uint64_t *bucket_c;    // L
    uint32_t doph_a, doph_b;
    uint64_t doph_seed;
    float srp_margin_gamma;   // 2 * gamma_d in fp32, rounded up
    double srp_gamma64;       // 2 * gamma_d for the fp64 recheck
    void *w_split;            // tensor-core precision: bf16 w1 then w2, P x dim each
    float *w_norm;            // upper bounds of ||w_j||
    float *w_aux;             // single-term tensor forms: P upper bounds of ||w_j - q(w_j)||, then P row scales
    uint32_t *tc_err;         // tensor-core pipeline timeout flag
    uint64_t tc_wait_ns;      // limit of the tensor-core pipeline's waits + 1 (0: the default)

    // shape
    uint32_t P;            // L * K projections / MinHash values per point
    uint32_t rp;           // gid row stride (R rounded up to 1, 2, 4 or 8)
    uint32_t rw;           // words per repetition-0 member record (1, 2, 4 or 8)
    uint32_t cw;           // bytes per per-cell count in the query kernels: 1 (L <= 255) or 2
    uint32_t BR;
    uint64_t nslot;        // L << W
    uint64_t entries_cap;  // L * R * capacity

    // index state
    uint64_t n_points;
    uint64_t n_cells;
    uint16_t *gid;         // capacity x rp
    uint32_t *moff;        // BR + 1: members of cell c are mem[moff[c] .. moff[c+1])
    uint32_t *mem;         // R * capacity point ids
    uint32_t *mrec;        // capacity * rw: repetition-0 members with their other group ids
    uint32_t *off;         // nslot + 1
    uint32_t *hidx;        // nslot: index of the slot's cell bitmap, or kEmpty32 (light slot)
    uint32_t *hbm;         // n_heavy x BRw words: bitmaps of the heavy slots' cell lists
    uint64_t hbm_words;    // allocated words of hbm
    uint32_t n_heavy;
    uint32_t heavy_min;    // a slot with at least this many cells also gets a bitmap
    uint32_t BRw;          // 32-bit words per cell bitmap
    uint16_t *cells;       // entries_cap
    uint16_t *cells_tmp;   // entries_cap (build scratch)
    uint32_t *slot_a;      // nslot + 1 (build scratch)
    uint32_t *slot_b;      // nslot + 1 (build scratch)
    uint32_t *cell_cnt;    // BR + 1 (build scratch)
    uint32_t *flag;        // device status word
    uint32_t *qnext;       // query counter of the fused kernel
    uint32_t *h_flag;      // pinned host copy
    unsigned long long *stats;   // [recheck, exact]
    uint64_t last_recheck, last_exact;

    flinng::Workspace ws;
    uint64_t device_bytes;
    uint32_t query_mode;   // FLINNG_QUERY_PLAIN, _FUSED or _GRAPH
    uint32_t probes;       // buckets probed per table (0 or 1: the query's own only)
    cudaStream_t side;     // second stream of the insert's concurrent passes (created on first use)
    cudaEvent_t ev_fork, ev_join;
    int sms;               // multiprocessors of the device (0: not looked up yet)
    flinng::OccEntry occ[8];          // occupancy of recent fused launch shapes
    uint32_t n_occ;
    flinng::QueryTuning tuning[33];   // per batch-size class (ceil log2 nq)
    flinng::QueryGraph graphs[33];
};

namespace flinng {

int ws_reserve(flinng_index *ix, size_t bytes);

// Raise a kernel's dynamic shared-memory limit to at least `smem` (never
// lowers it, so launches from other indices keep their headroom).
int ensure_dyn_smem(const void *fn, size_t smem);

// Process-wide count of kernel launches made by the library.
void count_launch(unsigned n = 1);

// ---- scan.cu
size_t scan_workspace_bytes(size_t n);
// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.
int scan_exclusive(const uint32_t *in, uint32_t *out, size_t n, void *ws,
                   cudaStream_t st);

// ---- hash.cu
// SRP: buckets n x L; proj (optional) n x P; rows of x with stride ld.
size_t srp_workspace_bytes(const flinng_index *ix, uint64_t n);
int srp_hash(flinng_index *ix, const float *x, uint64_t ld, uint64_t n,
             uint32_t *buckets, float *proj, void *ws, size_t ws_bytes);
// DOPH + bucket combine: buckets n x L; values (optional) n x P.
int doph_hash(flinng_index *ix, const uint64_t *off, const uint32_t *elems,
              uint64_t n, uint32_t *buckets, uint32_t *values);
// fp64 / exact re-check of listed (row << 20 | projection) entries
int srp_recheck_list(flinng_index *ix, const float *x, uint64_t ld, const unsigned long long *list,
                     const unsigned long long *count, uint32_t *codes);
int add_counter(unsigned long long *dst, const unsigned long long *src, cudaStream_t st);

// ---- srp_tc.cu (tensor-core precision form)
int srp_tc_prepare_weights(flinng_index *ix);
size_t srp_tc_workspace_bytes(const flinng_index *ix, uint64_t n);
int srp_hash_tc(flinng_index *ix, const float *x, uint64_t ld, uint64_t n, uint32_t *buckets, float *proj,
                void *ws);

// ---- build.cu
size_t perm_check_workspace_bytes(uint32_t R, uint64_t n);
// Input checks on the device: each ORs its error bits into ix->flag (zeroed by
// the caller first) without waiting; check_result waits for them all and
// turns the bits into an error.
int check_perm(flinng_index *ix, const uint32_t *perm, uint64_t n, void *ws);
int check_groups(flinng_index *ix, const uint16_t *groups, uint64_t n);
int check_result(flinng_index *ix);
// Workspace of insert_hashed for n new points (reset: a build from scratch).
size_t insert_workspace_bytes(const flinng_index *ix, uint64_t n, bool reset);
int insert_hashed(flinng_index *ix, const uint32_t *buckets, const uint32_t *perm, const uint16_t *groups,
                  uint64_t n, void *ws);
int build_heavy(flinng_index *ix, void *scan_ws, uint32_t *list);

// ---- query.cu
struct FusedQuery {
    uint32_t nq;
    const float *x;          // cosine: device rows
    uint64_t ldx;
    const uint64_t *off;     // Jaccard: device CSR
    const uint32_t *elems;
    const uint32_t *out_row = nullptr;   // per query: its output row, or null (row = query index)
};
int query_fused_launch(flinng_index *ix, const FusedQuery &fq, const uint32_t *k, uint32_t k_max,
                       uint32_t *out_ids, uint16_t *out_scores, const QueryTuning *tune);
int query_graph_launch(flinng_index *ix, const FusedQuery &fq, const uint32_t *k, uint32_t k_max,
                       uint32_t *out_ids, uint16_t *out_scores, const QueryTuning *tune);
void destroy_graphs(flinng_index *ix);
// Decode from caller-given per-cell counts (nq x B*R, each clamped to max_count)
// instead of gathering them; qbuckets unused then.
int query_launch_counts(flinng_index *ix, const uint32_t *qbuckets, const uint16_t *counts, uint32_t max_count,
                        uint32_t nq, const uint32_t *k, uint32_t k_max, uint32_t *out_ids, uint16_t *out_scores,
                        const uint32_t *out_row = nullptr);
// out_row (optional, device): per query, its row of out_ids / out_scores
int query_launch(flinng_index *ix, const uint32_t *qbuckets, uint32_t nq,
                 const uint32_t *k, uint32_t k_max, uint32_t *out_ids,
                 uint16_t *out_scores, const uint32_t *out_row = nullptr);
int counts_launch(flinng_index *ix, const uint32_t *qbuckets, uint32_t nq,
                  uint16_t *out_counts);

// ---- insert_delta.cu
// An insert of n points into a built index merges only the slots that gain
// cells when n * R <= kDeltaMaxKeys (the batch's entries of one table are
// sorted in shared memory); larger batches take the full merge of build.cu.
constexpr uint32_t kDeltaMaxKeys = 8192;
bool delta_insert_applies(const flinng_index *ix, uint64_t n);
size_t delta_workspace_bytes(const flinng_index *ix, uint64_t n);
// After insert_hashed's group and member-list stage: the reverse index.
int insert_delta(flinng_index *ix, const uint32_t *buckets, uint64_t n, void *ws);

// ---- probe.cu
// Multi-probe counts (probes P >= 1 per table): nq x B*R uint16, each <= L.
size_t probe_smem_bytes(uint32_t BR);
int probe_counts_launch(flinng_index *ix, const uint32_t *qbuckets, uint32_t nq, uint32_t P,
                        uint16_t *out_counts);

}  // namespace flinng
