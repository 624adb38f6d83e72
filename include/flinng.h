/*
 * flinng.h - C ABI of the GB300 FLINNG library (libflinng.so).
 *
 * FLINNG: Engels, Coleman, Shrivastava, "Practical Near Neighbor Search via
 * Group Testing" (arXiv 2106.11565). The index answers the randomized
 * nearest-neighbour problem of Def. 1: given a dataset D and a query y,
 * report points of D close to y. It is the B x R grid of group tests of
 * Sec. 4 (Alg. 1 builds it, Alg. 2 / Alg. 3 query it), each test a
 * distance-sensitive Bloom filter (Sec. 3.3) stored as a reverse index
 * (Sec. 5).
 *
 * Conventions for every entry point
 * ---------------------------------
 *  - Return value: FLINNG_OK (0) or one of the FLINNG_ERR_* codes below;
 *    flinng_last_error() then gives a message (thread-local, valid until the
 *    next call on the same thread). A failed call leaves the index as it was
 *    unless the message says otherwise.
 *  - Memory: the index owns all device memory it allocates (at create time,
 *    sized by flinng_config.capacity, plus a workspace that grows with the
 *    largest batch seen). The caller owns every input and output buffer.
 *    No caller pointer is kept after a call returns.
 *  - on_device: 1 means every caller buffer of the call is CUDA device memory
 *    of the current device; the call is then asynchronous on the index's
 *    stream (synchronise that stream before reading outputs or freeing
 *    inputs). 0 means every caller buffer is host memory; the call copies
 *    in, computes, copies out and returns after the stream is idle. In
 *    flinng_query, host buffers that are page-locked (cudaHostAlloc,
 *    cudaHostRegister) skip the copies: the query kernel writes the outputs
 *    in place, and reads the queries in place where it loads each element
 *    once (Jaccard queries; cosine queries hashed per CTA, see
 *    flinng_set_query_mode).
 *  - Threads: calls on one index must not overlap; the caller serialises
 *    them (an index owns one stream, one workspace and its CUDA graphs).
 *    Different indices may be used from different threads at once, except
 *    for flinng_query_noalloc, whose calls all share one scratch array.
 *  - Point ids are insertion order: the first build gives ids 0..n-1, each
 *    insert continues the numbering.
 *  - Cell ids are r * B + b for repetition r and group b; they are 16-bit
 *    (B * R <= 65536, the paper's "BR < 2^16", Sec. 5 and appendix).
 */
#ifndef FLINNG_H
#define FLINNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FLINNG_OK 0
#define FLINNG_ERR_INVALID_ARG 1 /* bad size, pointer, config or permutation */
#define FLINNG_ERR_OOM 2         /* device allocation failed */
#define FLINNG_ERR_CAPACITY 3    /* insert would exceed flinng_config.capacity */
#define FLINNG_ERR_CUDA 4        /* a CUDA call failed (message has the CUDA error) */
#define FLINNG_ERR_TIMEOUT 5     /* a bounded device-side wait gave up */

/* similarity / LSH family */
#define FLINNG_COSINE_SRP 0      /* dense fp32 vectors, sign random projections */
#define FLINNG_JACCARD_DOPH 1    /* sets of uint32, densified one-permutation MinHash */

/* arithmetic of the SRP projection (cosine only); the sign bits are exact in
 * every precision */
#define FLINNG_PREC_FP32 0     /* fp32 FMA tiles; fp64 / exact re-check below a rigorous margin */
#define FLINNG_PREC_BF16X2 1   /* tensor cores (tcgen05): each operand split into two bf16 parts,
                                  fp32 accumulation; compensated fp32, then fp64 / exact re-check of
                                  projections below a rigorous margin; needs dim % 8 == 0. Its
                                  pipeline waits are bounded: a wait that gave up (never expected)
                                  makes the index's next hash or query, and flinng_hash_counters,
                                  return FLINNG_ERR_TIMEOUT from then on */
#define FLINNG_PREC_BF16 2     /* tensor cores (tcgen05), one bf16 term per operand, fp32 accumulation;
                                  the margin is a-posteriori: it uses each row's own quantisation
                                  residual norm ||x - bf16(x)|| (and the same for every projection
                                  row), so it is rigorous yet follows the data; needs dim % 8 == 0 */
#define FLINNG_PREC_FP8 3      /* tensor cores (tcgen05 kind::f8f6f4), FP8 E4M3 operands with a
                                  power-of-two scale per row (values that would be E4M3 subnormals
                                  become 0), fp32 accumulation, the same a-posteriori margin; needs
                                  dim % 16 == 0. With every tensor-core form, projections inside the
                                  margin go to compensated fp32, then fp64 / exact re-checks, so the
                                  codes are those of FLINNG_PREC_FP32; the waits are bounded as
                                  for FLINNG_PREC_BF16X2 */

typedef struct flinng_config {
    uint32_t metric;        /* FLINNG_COSINE_SRP or FLINNG_JACCARD_DOPH */
    uint32_t dim;           /* cosine: vector length d (1..65536); ignored for sets */
    uint32_t R;             /* repetitions, 1..8 (Sec. 3.1) */
    uint32_t B;             /* groups per repetition, B * R <= 65536 (Sec. 3.1) */
    uint32_t L;             /* hash tables = Bloom-filter arrays, 1..4095 (paper: m) */
    uint32_t K;             /* hashes concatenated per table (paper: L, Sec. 3.2);
                               SRP: 1..30 (it is also W) */
    uint32_t range_bits;    /* W: buckets per table = 2^W; SRP requires W == K;
                               1..30 with L * 2^W < 2^31 */
    uint32_t min_threshold; /* t_min >= 1: cells with fewer collisions never test
                               positive (Sec. 5 threshold t, relaxed by Alg. 3) */
    uint32_t precision;     /* FLINNG_PREC_FP32, _BF16X2, _BF16 or _FP8 (cosine) */
    uint32_t reserved;
    uint64_t capacity;      /* maximum number of points, inserts included;
                               L * R * capacity < 2^32 */
} flinng_config;

/* Hash parameters: the LSH functions shared by all filters (Sec. 5), drawn by
 * the caller from its seed and passed as data. Host pointers, copied at
 * create time. */
typedef struct flinng_params {
    const float *srp_w;         /* cosine: (L*K) x dim row-major fp32 projection
                                   rows; row l*K + j gives bit j of table l */
    uint32_t doph_a;            /* Jaccard: pi(e) = doph_a * e + doph_b mod 2^32; odd */
    uint32_t doph_b;
    uint64_t doph_seed;         /* Jaccard: seed of the densification choices */
    const uint64_t *bucket_a;   /* Jaccard: L x K odd multipliers */
    const uint64_t *bucket_c;   /* Jaccard: L offsets */
} flinng_params;

/* A batch of points or queries. */
typedef struct flinng_points {
    const float *x;             /* cosine: n x dim fp32, row stride ld floats */
    uint64_t ld;                /* cosine: row stride (>= dim) */
    const uint64_t *off;        /* Jaccard: n + 1 offsets into elems (off[0] = 0,
                                   non-decreasing) */
    const uint32_t *elems;      /* Jaccard: set elements; duplicates allowed */
} flinng_points;

typedef struct flinng_index flinng_index;

/*
 * Create an empty index on the current CUDA device.
 * Allocates the index's device memory for cfg->capacity points.
 * stream: a cudaStream_t, or NULL for the legacy default stream.
 * Errors: INVALID_ARG (config out of range, missing params), OOM, CUDA.
 */
int flinng_create(const flinng_config *cfg, const flinng_params *params,
                  void *stream, flinng_index **out);

/*
 * Build the index from scratch over n points (Alg. 1 then Sec. 5): discards
 * the previous contents, hashes every point with the L shared LSH functions,
 * assigns point perm[r][i] to cell (r, i mod B) for each repetition r, and
 * writes the reverse index (per table: bucket -> sorted list of distinct cell
 * ids) in one pass.
 * perm: R x n uint32, row r a permutation of [0, n) (Alg. 1's random
 * permutation pi, drawn by the caller).
 * Errors: INVALID_ARG (a row of perm is not a permutation, n = 0 is allowed),
 * CAPACITY (n > capacity), CUDA.
 */
int flinng_build(flinng_index *idx, const flinng_points *pts, uint64_t n,
                 const uint32_t *perm, int on_device);

/*
 * flinng_build from precomputed buckets (n x L uint32, as flinng_hash
 * returns them) instead of points: Alg. 1 and the reverse index of Sec. 5
 * over points already hashed, e.g. hashed batch by batch by the caller so
 * that the points themselves are never held at once.
 * Errors: as flinng_build; INVALID_ARG also for a bucket >= 2^W.
 */
int flinng_build_buckets(flinng_index *idx, const uint32_t *buckets, uint64_t n,
                         const uint32_t *perm, int on_device);

/*
 * Add n points with ids size .. size+n-1. Alg. 1 applied to the batch with
 * positions continuing after the current size: position i of row r of perm
 * goes to cell (r, (size + i) mod B). The reverse index becomes that of the
 * union.
 * Errors: as flinng_build; CAPACITY leaves the index unchanged.
 */
int flinng_insert(flinng_index *idx, const flinng_points *pts, uint64_t n,
                  const uint32_t *perm, int on_device);

/*
 * Build (replacing the index) or insert with the group design given
 * outright instead of Alg. 1's permutations. The framework takes any
 * non-adaptive design (Sec. 3.1); with one test per point and repetition,
 * Alg. 2's AND over the R tests and Alg. 3's relaxed decode apply unchanged.
 * Groups may be of any size, some empty, e.g. each point's group drawn
 * independently per repetition.
 * groups: R x n uint16, row-major: groups[r * n + i] is the group (< B) of
 * point i of this batch in repetition r (its cell is r * B + group).
 * Errors: as flinng_build / flinng_insert; INVALID_ARG (index unchanged) if
 * a group id is >= B or groups is null with n > 0.
 */
int flinng_build_groups(flinng_index *idx, const flinng_points *pts, uint64_t n,
                        const uint16_t *groups, int on_device);
int flinng_insert_groups(flinng_index *idx, const flinng_points *pts, uint64_t n,
                         const uint16_t *groups, int on_device);

/*
 * Batched query (Sec. 5 with Alg. 3): hash each query once, count per cell
 * the tables whose bucket list holds the cell, and return the points in
 * Alg. 3's order - cells by count descending (ties: cell id ascending),
 * points as their last cell is reached, by id within a cell - keeping
 * only points whose R cells all have count >= min_threshold.
 * k: per-query result counts (nq entries, each <= k_max), or NULL for k_max
 * for every query. k_max <= 1024.
 * out_ids: nq x k_max point ids, padded with 0xFFFFFFFF.
 * out_scores: nq x k_max uint16, the score of each returned point (the least
 * count among its R cells, 0..L), padded with 0; may be NULL.
 * Errors: INVALID_ARG (k > k_max, k_max > 1024, null outputs), CUDA.
 */
int flinng_query(flinng_index *idx, const flinng_points *q, uint32_t nq,
                 const uint32_t *k, uint32_t k_max, uint32_t *out_ids,
                 uint16_t *out_scores, int on_device);

/* Destroy the index and free its device memory. NULL is a no-op. */
int flinng_destroy(flinng_index *idx);

/*
 * Save a built index to a file, and load it back onto the current device
 * (the index of Sec. 5 with its groups from Alg. 1). The file holds the
 * configuration, the hash parameters, the group ids, member lists and
 * records, each table's bucket-to-cell lists and the heavy buckets' cell
 * bitmaps. A loaded index answers every query exactly as the saved one
 * and takes inserts up to the same capacity. The format is this library's
 * own (little endian, versioned); it is not portable across byte orders.
 * flinng_save synchronises the index's stream; flinng_load allocates like
 * flinng_create and runs on `stream`.
 * Errors: INVALID_ARG (unreadable, wrong or truncated file; a file that
 * exceeds its stated capacity), OOM, CUDA.
 */
int flinng_save(flinng_index *idx, const char *path);
int flinng_load(const char *path, void *stream, flinng_index **out);

/* The configuration an index was created (or loaded) with. */
int flinng_get_config(const flinng_index *idx, flinng_config *out);

/* Message of the last failed call on this thread ("" if none). */
const char *flinng_last_error(void);

/* Number of points in the index. */
uint64_t flinng_size(const flinng_index *idx);

/* Device bytes held by the index (index arrays, scratch, workspace). */
uint64_t flinng_device_bytes(const flinng_index *idx);

/* Set the stream used by subsequent calls (cudaStream_t or NULL). */
int flinng_set_stream(flinng_index *idx, void *stream);

/* Limit of each wait in the tensor-core SRP pipeline of this index (default
 * 1,000,000,000 ns; 0 makes each wait a single try; UINT64_MAX restores the
 * default). The paper has no counterpart: this exercises the failure path
 * of the bounded waits. A wait that gives up makes the kernel stop issuing
 * work, wait (with the default limit) for the copies and MMAs it issued,
 * free its tensor memory and set the index's timeout flag, so the context
 * stays usable; calls that synchronise (host buffers) return
 * FLINNG_ERR_TIMEOUT at once, and every later hash or query of the index
 * does. Errors: INVALID_ARG for NULL. */
int flinng_set_tc_wait(flinng_index *idx, uint64_t limit_ns);

/* Multi-probe counting (cosine / SRP indices; the multi-probe LSH that the
 * related work of Sec. 2 cites, as an option the paper does not use): with
 * probes = P > 1, table l of a query probes its own bucket b_l and the P - 1
 * buckets b_l ^ (1 << j), j = 0 .. P-2 (the sign of projection l*K + j
 * flipped). A cell counts table l once if the list of any probed bucket of
 * that table holds it, so counts stay in 0..L and Alg. 3 decodes them as
 * usual; with P = 1 (the default; 0 means 1) every call is the paper's
 * single-probe method. flinng_query and flinng_query_buckets then count with
 * a separate kernel and decode from those counts (the fused and graph modes
 * are not used for such an index; nq x B*R x 2 bytes of workspace), and
 * flinng_counts returns the multi-probe counts. The server and
 * flinng_query_noalloc reject such an index (INVALID_ARG).
 * Errors: INVALID_ARG (NULL, a set index and P > 1, or P > K + 1). */
int flinng_set_probes(flinng_index *idx, uint32_t probes);

/* How flinng_query runs a batch (same results in every mode):
 * FLINNG_QUERY_PLAIN - a hash kernel for the batch, then one count / decode /
 *   top-k kernel (one CTA per query);
 * FLINNG_QUERY_FUSED - one persistent kernel that hashes each query in its
 *   CTA and goes straight on to count / decode / top-k (default);
 * FLINNG_QUERY_GRAPH - the fused kernel launched through a CUDA graph kept
 *   per batch-size class (nq rounded up to a power of two); each call
 *   rewrites the graph's kernel arguments and replays it.
 * Cosine indices whose projection matrix has more than 2^18 entries (L*K*dim)
 * hash every batch with the batched GEMM in all modes. */
#define FLINNG_QUERY_PLAIN 0
#define FLINNG_QUERY_FUSED 1
#define FLINNG_QUERY_GRAPH 2
int flinng_set_query_mode(flinng_index *idx, uint32_t mode);

/* Autotune the fused query on a sample batch: times CTA sizes (128, 256, 512),
 * CTAs per SM and candidate-buffer sizes on this batch (synchronously) and
 * keeps the fastest for batches of the same size class (power of two of
 * nq); later fused/graph calls of that class use it. Results never depend on
 * the tuning. chosen (optional, 3 entries): threads, CTAs per SM (0 = as many
 * as fit), buffer entries (0 = default); all 0 when the index's batches are
 * hashed by the GEMM (nothing to tune). */
int flinng_tune_query(flinng_index *idx, const flinng_points *q, uint32_t nq,
                      uint32_t k_max, int on_device, uint32_t *chosen);

/* Set the fused query's launch shape for batches of nq's size class (the
 * power of two at or above nq) instead of tuning it, e.g. to a shape tuned
 * offline or under other cache conditions. threads: 128, 256 or 512;
 * ctas_per_sm: 0 (as many as fit) to 16; cap: candidate buffer entries, 0
 * (default) or a power of two in [64, 8192] (raised to the decode's minimum
 * when smaller). Results never depend on the shape. FLINNG_ERR_INVALID_ARG on
 * any other value. */
int flinng_set_tuning(flinng_index *idx, uint32_t nq, uint32_t threads, uint32_t ctas_per_sm,
                      uint32_t cap);

/* ---------------------------------------------------------------------- */
/* Stage entry points, for parity checks of each step against a reference */
/* ---------------------------------------------------------------------- */

/*
 * Hash n points with the index's LSH functions (Sec. 3.2 concatenation,
 * Sec. 5 shared functions). Errors: INVALID_ARG (null buckets, malformed
 * points), TIMEOUT (tensor-core precision: a bounded wait gave up), CUDA.
 * out_buckets: n x L uint32 bucket per table (SRP: the K sign bits, bit j =
 *   (projection l*K + j > 0); Jaccard: the W-bit combination of the K MinHash
 *   values of table l).
 * out_values: Jaccard only, n x (L*K) uint32 MinHash values, or NULL.
 * out_proj: cosine only, n x (L*K) fp32 projections as computed before the
 *   sign decision, or NULL.
 */
int flinng_hash(flinng_index *idx, const flinng_points *pts, uint64_t n,
                uint32_t *out_buckets, uint32_t *out_values, float *out_proj,
                int on_device);

/*
 * Query from precomputed buckets (nq x L), skipping the hash step.
 * Same outputs as flinng_query. Every bucket must be < 2^W: host buffers are
 * checked (INVALID_ARG, nothing launched); device buffers are not checked,
 * and keeping them in range is the caller's part of the contract.
 * Errors: as flinng_query.
 */
int flinng_query_buckets(flinng_index *idx, const uint32_t *qbuckets,
                         uint32_t nq, const uint32_t *k, uint32_t k_max,
                         uint32_t *out_ids, uint16_t *out_scores,
                         int on_device);

/*
 * Per-cell collision counts of nq queries given their buckets (Sec. 5):
 * out_counts nq x (B*R) uint16 (each in 0..L; the multi-probe counts when the
 * index probes more than one bucket per table, see flinng_set_probes).
 * Buckets < 2^W, checked as in flinng_query_buckets. Errors: INVALID_ARG, CUDA.
 */
int flinng_counts(flinng_index *idx, const uint32_t *qbuckets, uint32_t nq,
                  uint16_t *out_counts, int on_device);

/*
 * Query from per-cell counts instead of query buckets: Alg. 3's group tests,
 * AND-over-R decode and top-k on counts the caller supplies (Sec. 5: the
 * count of a cell is the number of tables whose list for the query's bucket
 * holds it). This is the decode step of a table-sharded index: each shard
 * holds a disjoint subset of the tables over the same groups (same points and
 * permutation), flinng_counts gives its partial counts, their sum over shards
 * (an all-reduce) equals the counts of the whole index, and this call decodes
 * them on any one shard.
 * counts: nq x (B*R) uint16. max_count: the total number of tables (the
 * largest count possible, 1..4095); larger values are clamped to it.
 * Same k, k_max and outputs as flinng_query. Errors: INVALID_ARG, CUDA.
 */
int flinng_query_counts(flinng_index *idx, const uint16_t *counts, uint32_t nq,
                        uint32_t max_count, const uint32_t *k, uint32_t k_max,
                        uint32_t *out_ids, uint16_t *out_scores, int on_device);

/*
 * Copy the index out to HOST buffers (synchronous).
 * off: L * 2^W + 1 uint32 CSR offsets; cells: the cell lists (cells_cap
 * entries available; *n_cells receives the count); gid: size x R uint16
 * cell of each point per repetition (group b, not r*B+b). Any may be NULL.
 * Errors: CAPACITY if cells_cap is too small (nothing written to cells).
 */
int flinng_export(flinng_index *idx, uint32_t *off, uint16_t *cells,
                  uint64_t cells_cap, uint64_t *n_cells, uint16_t *gid);

/* Counters of the last hash call (cosine): projections the first pass (fp32
 * FMA or tensor cores) could not decide, and those that needed the exact
 * accumulator. A build or insert hashes its points while its permutation or
 * group checks run, so a call refused by those checks still leaves the
 * counters of its hash. */
int flinng_hash_stats(const flinng_index *idx, uint64_t *n_recheck,
                      uint64_t *n_exact);

/* All counters of the last cosine hash, or query (Sec. 3.2 signs), on this
 * index: out[0] projections the first pass (fp32 FMA or tensor cores) could
 * not decide; out[1] those decided by the exact accumulator; out[2] fp64
 * re-checks; out[3] compensated fp32 re-checks (tensor-core precision only);
 * out[4] flips: first-pass signs that a re-check reversed (the hash-bit flip
 * rate before re-check is out[4] / (n * L * K)). out: 5 HOST uint64, written
 * after the index's stream is synchronised. Errors: INVALID_ARG for NULL. */
int flinng_hash_counters(const flinng_index *idx, uint64_t *out);

/* Number of CUDA kernels this library has launched in this process (all
 * indices, all threads); memset/memcpy operations are not counted. */
uint64_t flinng_kernel_launches(void);

/*
 * flinng_query without any device allocation. The paper has no counterpart:
 * this is a deployment variant of the batched query.
 *
 * Who needs it: flinng_query keeps its intermediate query buckets (and, for
 * cosine indices, its sign re-check list) in a workspace that it grows with
 * cudaMalloc - after synchronising the stream and freeing the old one -
 * whenever a batch is larger than any before. Some callers cannot allow
 * that: a server whose HBM is handed out up front to resident indices and
 * request slots under a fixed budget, where an allocation at query time can
 * fail or breach the budget; a latency-critical loop that cannot absorb the
 * device-wide synchronisation of cudaFree; a host application whose device
 * memory must come from its own pool. This entry point allocates nothing:
 * its scratch is one fixed array inside the library (6 MiB per GPU that
 * loads the library, held until the process exits), the caller passes the
 * inputs and outputs.
 *
 * Arguments and results are those of flinng_query with on_device = 1: q, k,
 * out_ids and out_scores are device memory; the call is asynchronous on the
 * index's stream. The index's device must be the current device.
 * Limits: nq * L <= 262144, and for cosine indices nq * L * K <= 655296.
 * Cosine indices of a tensor-core precision also stage every query row's
 * quantised parts (at most 4 * dim bytes: FLINNG_PREC_BF16X2) and two
 * re-check lists in the same 5 MiB part of
 * the array: about nq * (4 * dim + 16 * L * K + 12) + 8192 <= 5242880 bytes
 * (the call computes the exact figure). Larger batches are rejected with
 * FLINNG_ERR_INVALID_ARG before anything runs (split them, or use
 * flinng_query).
 * The first call in a device's CUDA context looks up the scratch array's
 * device address (cudaGetSymbolAddress) and caches it under that context's
 * unique id; a context made again after cudaDeviceReset is looked up afresh.
 * Make that first call before any stream capture.
 * All calls share the one array and it keeps the last call's contents (each
 * call overwrites what it reads): calls whose GPU work overlaps - on
 * different streams, or different indices - race on it and must be
 * serialised by the caller.
 */
int flinng_query_noalloc(flinng_index *idx, const flinng_points *q, uint32_t nq,
                         const uint32_t *k, uint32_t k_max, uint32_t *out_ids,
                         uint16_t *out_scores);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching over several resident indices             */
/* ---------------------------------------------------------------------- */

/* The paper runs one query at a time on one core (Sec. 6); this runtime
 * serves a stream of requests against several device-resident indices:
 * queries that arrive are batched per index (uneven k and set sizes in one
 * launch) and run on one of n_slots CUDA streams, each with its own staging
 * and scratch, so batches overlap on the device; a slot takes the next batch
 * as soon as its previous one completes. An insert runs when every batch in
 * flight on its index has finished, in arrival order with that index's
 * queries (later queries see the inserted points), on a host thread of its
 * own: the other indices keep being served meanwhile, and its own index
 * takes no batch until the insert is done. Results equal those of
 * flinng_query on the index as it stood when the query ran. */
typedef struct flinng_server flinng_server;

typedef struct flinng_server_config {
    uint64_t hbm_budget;       /* device bytes the indices and the slots may hold */
    uint32_t n_slots;          /* batches in flight at once (1..64), one stream each */
    uint32_t max_batch;        /* queries per batch */
    uint32_t k_max;            /* result width of every query, 1..1024 */
    uint32_t max_batch_elems;  /* set elements staged per batch (Jaccard indices) */
} flinng_server_config;

#define FLINNG_REQ_QUERY 0
#define FLINNG_REQ_INSERT 1

typedef struct flinng_request {
    double arrival_s;          /* seconds after the start of the replay (non-decreasing) */
    uint32_t kind;             /* FLINNG_REQ_QUERY or FLINNG_REQ_INSERT */
    uint32_t index;            /* id from flinng_server_add_index */
    uint32_t k;                /* query: results wanted, <= k_max */
    uint32_t on_device;        /* insert: 1 if *data and perm are device memory */
    uint64_t n;                /* query: set size (Jaccard; ignored for cosine); insert: points */
    const void *data;          /* query: dim floats or n uint32 set elements, HOST memory;
                                  insert: a const flinng_points * */
    const uint32_t *perm;      /* insert: R x n permutation, as flinng_insert */
} flinng_request;

typedef struct flinng_request_result {
    double t_admit, t_start, t_done;   /* host clock, seconds after the start of the replay:
                                          admitted, batch launched (insert started), results
                                          in the caller's buffers (insert done) */
    uint32_t status;           /* FLINNG_OK or the insert's error (CAPACITY, ...) */
    uint32_t version;          /* inserts applied to the index when the request ran */
    uint32_t batch;            /* queries: sequence number of the batch it ran in */
    uint32_t slot;             /* queries: the stream slot (0..n_slots-1) the batch ran on */
    double d_start, d_done;    /* queries: device clock (CUDA events on the slot's stream),
                                  seconds after an event recorded when the replay began:
                                  the batch's first copy started, its results reached the
                                  host staging; 0 for inserts */
} flinng_request_result;

/* Create a server (streams and events; no index yet). */
int flinng_server_create(const flinng_server_config *cfg, flinng_server **out);

/* Register an index (created and built by the caller, not owned by the
 * server; its stream must not be used by anyone else while the server runs).
 * Admission by HBM budget: the index's device bytes plus the slots' scratch
 * must fit hbm_budget with the indices already registered, else
 * FLINNG_ERR_OOM and nothing changes. */
int flinng_server_add_index(flinng_server *srv, flinng_index *idx, uint32_t *index_id);

/* Device bytes held by the registered indices and the slots. */
uint64_t flinng_server_device_bytes(const flinng_server *srv);

/* How the server stages query inputs and results: 1 = a kernel gathers the
 * inputs straight from the requests' host buffers and the query kernel
 * writes each result row straight into the caller's out_ids / out_scores
 * (the device can read and write pageable host memory), 0 = the host copies
 * inputs into pinned staging first and results back out of it. Negative:
 * an error code (NULL server). */
int flinng_server_staging(const flinng_server *srv);

/* Serve n requests (n < 2^32), each admitted when the clock reaches its
 * arrival time; returns when all are done. out_ids / out_scores: n x k_max
 * (HOST), rows of queries written (padding as flinng_query), rows of inserts
 * untouched. With staging 1 (flinng_server_staging) the GPU writes the rows
 * itself: the buffers must stay valid for the whole call, and pages touched
 * beforehand avoid first-touch faults during the replay.
 * res: per-request times, status, index version and batch.
 * Errors: INVALID_ARG (bad request, checked before anything runs), CUDA. */
int flinng_server_replay(flinng_server *srv, const flinng_request *reqs, uint64_t n,
                         uint32_t *out_ids, uint16_t *out_scores, flinng_request_result *res);

/* Destroy the server (not its indices). NULL is a no-op. */
int flinng_server_destroy(flinng_server *srv);

/* ---------------------------------------------------------------------- */
/* Synthetic input (not part of FLINNG)                                    */
/* ---------------------------------------------------------------------- */

/* Embeddings streamed from a seed, shaped like the paper's YFCC100M
 * workload (Sec. 6, Table 1: 4096-dimensional neural activations, about half
 * zeros): ReLU of a Gaussian mixture with n_centers centres ~ N(0, I),
 * points = ReLU(centre + sigma * z), queries = ReLU(pre-ReLU value of a
 * random point + q_sigma * z), z from Philox4x32-10 counters through an
 * Irwin-Hall sum of four uniforms. Any row can be regenerated alone. */
typedef struct flinng_embed_spec {
    uint64_t seed;
    uint32_t dim;
    uint32_t n_centers;
    float sigma;
    float q_sigma;
    uint64_t n_points;      /* queries draw their source point from [0, n_points) */
} flinng_embed_spec;

/* Write rows first .. first+n-1 of the point stream (queries = 0) or of the
 * query stream (queries = 1) to out (DEVICE memory, n x spec->dim, row stride
 * ld floats), asynchronously on stream (cudaStream_t or NULL). Row indices
 * must stay below 2^32. Errors: INVALID_ARG, CUDA. */
int flinng_generate_embeddings(const flinng_embed_spec *spec, int queries, uint64_t first,
                               uint64_t n, float *out, uint64_t ld, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FLINNG_H */
