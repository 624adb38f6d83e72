/*
 * FLINNG oracle: a plain, slow, single-threaded CPU implementation of what the
 * GPU library computes. TEST INFRASTRUCTURE ONLY: tests, the smoke check and
 * the bench's CPU-baseline leg call it; the library never does. It shares no
 * code with the CUDA path.
 *
 * Paper: Engels, Coleman, Shrivastava, "Practical Near Neighbor Search via
 * Group Testing" (arXiv 2106.11565).
 *
 *   oracle_srp_codes        Sec. 3.2 (LSH, concatenation trick) + Sec. 5
 *                           (shared hash functions); sign random projections.
 *   oracle_doph             Sec. 6 (sets "compressed via MinHash"); densified
 *                           one-permutation MinHash (reading stated below).
 *   oracle_minhash_buckets  Sec. 3.2 concatenation trick: K MinHash values of
 *                           table l combined into one W-bit bucket.
 *   oracle_groups           Alg. 1: permute, cell of position i is i mod B.
 *   oracle_members          Alg. 1: member sets M_{r,b}.
 *   oracle_build_csr        Sec. 5: reverse index, per table, from hash value
 *                           to the cells whose filter holds that value.
 *   oracle_counts           Sec. 5: per-cell collision counts of a query.
 *   oracle_query            Alg. 3 (threshold relaxation), literally.
 *
 * Readings of the paper where it is silent (all restated in the design
 * notes): bit j of table l is projection l*K+j, least significant first;
 * bit = (p > 0); a bucket list holds a cell at most once (bit-array filter,
 * Sec. 3.3); cells are visited by (count desc, cell id asc), members of a
 * cell by id asc; cells whose count is below t_min are never positive.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* exact sign of a sum of fp32 x fp32 products (long accumulator)            */
/* ------------------------------------------------------------------------ */

/* A product of two fp32 values is exact in fp64 and its magnitude lies in
 * [2^-298, 2^256). Written as im * 2^(e-53) with |im| < 2^53, its lowest
 * bit sits at 2^-350 or above. The accumulator holds bits from 2^-LIMB_BIAS
 * upward in 32-bit digits kept in int64, so that up to 2^31 additions cannot
 * overflow a digit; NLIMB digits reach far above 2^(256+31). */
#define NLIMB 24
#define LIMB_BIAS 384

static void acc_add(int64_t *acc, double v)
{
    if (v == 0.0) return;
    int e;
    double m = frexp(v, &e);                  /* v = m * 2^e, 0.5 <= |m| < 1 */
    int64_t im = (int64_t)ldexp(m, 53);        /* exact: |im| < 2^53 */
    int pos = e - 53 + LIMB_BIAS;             /* bit position of im's LSB */
    int64_t sgn = im < 0 ? -1 : 1;
    uint64_t mag = (uint64_t)(im < 0 ? -im : im);
    int limb = pos / 32, sh = pos % 32;
    /* mag * 2^sh has at most 85 bits: three 32-bit digits */
    uint64_t d0 = (mag << sh) & 0xffffffffull;
    uint64_t d1 = (sh == 0 ? mag >> 32 : mag >> (32 - sh)) & 0xffffffffull;
    uint64_t d2 = sh == 0 ? 0 : mag >> (64 - sh);
    acc[limb] += sgn * (int64_t)d0;
    acc[limb + 1] += sgn * (int64_t)d1;
    acc[limb + 2] += sgn * (int64_t)d2;
}

/* returns +1, 0 or -1 */
static int acc_sign(int64_t *acc)
{
    for (int i = 0; i < NLIMB - 1; ++i) {
        int64_t c = acc[i] >> 32;             /* floor division by 2^32 */
        acc[i] -= c * ((int64_t)1 << 32);
        acc[i + 1] += c;
    }
    if (acc[NLIMB - 1] > 0) return 1;
    if (acc[NLIMB - 1] < 0) return -1;
    for (int i = NLIMB - 2; i >= 0; --i)
        if (acc[i] != 0) return 1;            /* lower digits are in [0, 2^32) */
    return 0;
}

int oracle_exact_dot_sign(const float *a, const float *b, uint32_t d)
{
    int64_t acc[NLIMB + 2];
    memset(acc, 0, sizeof acc);
    for (uint32_t i = 0; i < d; ++i) acc_add(acc, (double)a[i] * (double)b[i]);
    return acc_sign(acc);
}

/* ------------------------------------------------------------------------ */
/* A1: sign random projections                                               */
/* ------------------------------------------------------------------------ */

/*
 * For point i and projection j: p = sum_t w[j][t] * x[i][t], summed in fp64
 * in order t = 0..d-1 (each product exact). The fp64 sum is within
 * gamma_d * sum|w x| of the exact value, gamma_d = d u / (1 - d u),
 * u = 2^-53; when |p| is not larger than twice that bound the sign is taken
 * from the exact long accumulator instead. bit = (exact p > 0).
 * code[i][l] = sum_{j<K} bit(l*K + j) << j.
 *
 * proj (optional, n x L*K) receives the fp64 sums. Returns the number of
 * projections that needed the exact accumulator.
 */
uint64_t oracle_srp_codes(const float *x, uint64_t n, uint32_t d, uint64_t ldx,
                          const float *w, uint32_t L, uint32_t K,
                          uint32_t *codes, double *proj)
{
    const uint32_t P = L * K;
    const double u = ldexp(1.0, -53);
    const double gamma = (d * u) / (1.0 - d * u);
    uint64_t n_exact = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const float *xi = x + i * ldx;
        for (uint32_t l = 0; l < L; ++l) codes[i * L + l] = 0;
        for (uint32_t j = 0; j < P; ++j) {
            const float *wj = w + (uint64_t)j * d;
            double p = 0.0, s = 0.0;
            for (uint32_t t = 0; t < d; ++t) {
                double prod = (double)wj[t] * (double)xi[t];
                p += prod;
                s += fabs(prod);
            }
            if (proj) proj[i * P + j] = p;
            int positive;
            if (fabs(p) > 2.0 * gamma * s) {
                positive = p > 0.0;
            } else {
                ++n_exact;
                positive = oracle_exact_dot_sign(wj, xi, d) > 0;
            }
            if (positive) codes[i * L + j / K] |= 1u << (j % K);
        }
    }
    return n_exact;
}

/* ------------------------------------------------------------------------ */
/* A2: densified one-permutation MinHash                                    */
/* ------------------------------------------------------------------------ */

/* splitmix64 finaliser (Steele, Lea, Flood 2014), used as the random
 * hash that picks the bin an empty bin borrows from. */
uint64_t oracle_splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

#define DOPH_MAX_ATTEMPTS 4096u
#define DOPH_EMPTY 0xFFFFFFFFu

/*
 * One permutation pi(e) = a*e + b mod 2^32 (a odd: a bijection of uint32).
 * nb bins split the 32-bit range evenly: bin(e) = (pi(e) * nb) >> 32.
 * Value of a bin = the smallest pi(e) that falls in it.
 * Densification of an empty bin i: for attempt = 1, 2, ...: j =
 * splitmix64(seed ^ (i << 32 | attempt)) mod nb; the first j whose bin was
 * non-empty before densification gives its value. After DOPH_MAX_ATTEMPTS
 * failures the first originally non-empty bin after i (cyclically) is used.
 * An empty set yields DOPH_EMPTY in every bin.
 * out: n x nb.
 */
void oracle_doph(const uint64_t *off, const uint32_t *elems, uint64_t n,
                 uint32_t nb, uint32_t a, uint32_t b, uint64_t seed,
                 uint32_t *out)
{
    uint32_t *val = (uint32_t *)malloc(sizeof(uint32_t) * nb);
    uint8_t *full = (uint8_t *)malloc(nb);
    for (uint64_t i = 0; i < n; ++i) {
        for (uint32_t k = 0; k < nb; ++k) { val[k] = DOPH_EMPTY; full[k] = 0; }
        for (uint64_t t = off[i]; t < off[i + 1]; ++t) {
            uint32_t pe = a * elems[t] + b;
            uint32_t bin = (uint32_t)(((uint64_t)pe * nb) >> 32);
            if (!full[bin] || pe < val[bin]) val[bin] = pe;
            full[bin] = 1;
        }
        uint32_t *o = out + i * nb;
        int any = 0;
        for (uint32_t k = 0; k < nb; ++k) any |= full[k];
        for (uint32_t k = 0; k < nb; ++k) {
            if (full[k] || !any) { o[k] = val[k]; continue; }
            int found = 0;
            for (uint32_t att = 1; att <= DOPH_MAX_ATTEMPTS; ++att) {
                uint64_t h = oracle_splitmix64(seed ^ (((uint64_t)k << 32) | att));
                uint32_t j = (uint32_t)(h % nb);
                if (full[j]) { o[k] = val[j]; found = 1; break; }
            }
            if (!found) {
                for (uint32_t s = 1; s <= nb; ++s) {
                    uint32_t j = (k + s) % nb;
                    if (full[j]) { o[k] = val[j]; break; }
                }
            }
        }
    }
    free(val);
    free(full);
}

/* ------------------------------------------------------------------------ */
/* A3: buckets                                                               */
/* ------------------------------------------------------------------------ */

/* bucket[i][l] = ((sum_j ba[l][j] * v[i][l*K+j] + bc[l]) mod 2^64) >> (64-W) */
void oracle_minhash_buckets(const uint32_t *v, uint64_t n, uint32_t L,
                            uint32_t K, const uint64_t *ba, const uint64_t *bc,
                            uint32_t W, uint32_t *bucket)
{
    for (uint64_t i = 0; i < n; ++i)
        for (uint32_t l = 0; l < L; ++l) {
            uint64_t h = bc[l];
            for (uint32_t j = 0; j < K; ++j)
                h += ba[(uint64_t)l * K + j] * (uint64_t)v[i * (uint64_t)L * K + (uint64_t)l * K + j];
            bucket[i * L + l] = (uint32_t)(h >> (64 - W));
        }
}

/* ------------------------------------------------------------------------ */
/* A4: group assignment (Alg. 1)                                             */
/* ------------------------------------------------------------------------ */

/*
 * perm: R x n, a permutation of the batch's local indices per repetition.
 * Position i of repetition r holds point n_old + perm[r][i]; its cell is
 * (n_old + i) mod B (positions continue across insert batches).
 * gid: point-major, gid[x * R + r], rows n_old .. n_old+n-1 written.
 * Returns 0, or -1 if a perm row is not a permutation.
 */
int oracle_groups(const uint32_t *perm, uint32_t R, uint64_t n, uint64_t n_old,
                  uint32_t B, uint16_t *gid)
{
    uint8_t *seen = (uint8_t *)malloc(n ? n : 1);
    int rc = 0;
    for (uint32_t r = 0; r < R && rc == 0; ++r) {
        memset(seen, 0, n ? n : 1);
        for (uint64_t i = 0; i < n; ++i) {
            uint32_t x = perm[(uint64_t)r * n + i];
            if (x >= n || seen[x]) { rc = -1; break; }
            seen[x] = 1;
            gid[(n_old + x) * R + r] = (uint16_t)((n_old + i) % B);
        }
    }
    free(seen);
    return rc;
}

/* Members of cell (r, b) in ascending point id: moff[r*(B+1) + b] .. +1,
 * into mem[r * N + ...]. */
void oracle_members(const uint16_t *gid, uint64_t N, uint32_t R, uint32_t B,
                    uint64_t *moff, uint32_t *mem)
{
    for (uint32_t r = 0; r < R; ++r) {
        uint64_t *o = moff + (uint64_t)r * (B + 1);
        for (uint32_t b = 0; b <= B; ++b) o[b] = 0;
        for (uint64_t x = 0; x < N; ++x) o[gid[x * R + r] + 1]++;
        for (uint32_t b = 0; b < B; ++b) o[b + 1] += o[b];
        uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * (B ? B : 1));
        for (uint32_t b = 0; b < B; ++b) fill[b] = o[b];
        for (uint64_t x = 0; x < N; ++x) {
            uint16_t g = gid[x * R + r];
            mem[(uint64_t)r * N + fill[g]++] = (uint32_t)x;
        }
        free(fill);
    }
}

/* ------------------------------------------------------------------------ */
/* A5: reverse index                                                         */
/* ------------------------------------------------------------------------ */

static int cmp_u64(const void *p, const void *q)
{
    uint64_t a = *(const uint64_t *)p, b = *(const uint64_t *)q;
    return (a > b) - (a < b);
}

/*
 * For every point x, table l and repetition r the triple
 * (l, bucket[x][l], cell = r*B + gid[x][r]) is an entry; entries are sorted
 * and duplicates dropped (a filter's bit is set at most once).
 * CSR: the list of table l, bucket h is cells[off[l*2^W + h] .. off[...+1]).
 * off has L*2^W + 1 entries. Returns the number of cells written, or -1 if
 * they do not fit in cells_cap.
 */
int64_t oracle_build_csr(const uint32_t *bucket, const uint16_t *gid,
                         uint64_t N, uint32_t L, uint32_t R, uint32_t B,
                         uint32_t W, uint32_t *off, uint16_t *cells,
                         uint64_t cells_cap)
{
    uint64_t ne = N * L * R;
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (ne ? ne : 1));
    uint64_t e = 0;
    for (uint64_t x = 0; x < N; ++x)
        for (uint32_t l = 0; l < L; ++l)
            for (uint32_t r = 0; r < R; ++r) {
                uint64_t slot = ((uint64_t)l << W) | bucket[x * L + l];
                uint64_t cell = (uint64_t)r * B + gid[x * R + r];
                key[e++] = (slot << 16) | cell;
            }
    qsort(key, ne, sizeof(uint64_t), cmp_u64);
    uint64_t nslot = (uint64_t)L << W;
    for (uint64_t s = 0; s <= nslot; ++s) off[s] = 0;
    uint64_t nc = 0;
    for (uint64_t t = 0; t < ne; ++t) {
        if (t > 0 && key[t] == key[t - 1]) continue;
        if (nc >= cells_cap) { free(key); return -1; }
        cells[nc++] = (uint16_t)(key[t] & 0xffff);
        off[(key[t] >> 16) + 1]++;
    }
    for (uint64_t s = 0; s < nslot; ++s) off[s + 1] += off[s];
    free(key);
    return (int64_t)nc;
}

/* ------------------------------------------------------------------------ */
/* A6: per-cell collision counts                                             */
/* ------------------------------------------------------------------------ */

/* cnt[c] = number of tables l whose list for the query's bucket holds c. */
void oracle_counts(const uint32_t *off, const uint16_t *cells, uint32_t L,
                   uint32_t W, const uint32_t *qbucket, uint32_t BR,
                   uint16_t *cnt)
{
    for (uint32_t c = 0; c < BR; ++c) cnt[c] = 0;
    for (uint32_t l = 0; l < L; ++l) {
        uint64_t s = ((uint64_t)l << W) | qbucket[l];
        for (uint32_t t = off[s]; t < off[s + 1]; ++t) cnt[cells[t]]++;
    }
}

/* Counts straight from the definition, with no reverse index (Sec. 5: a
 * cell's count is the number of tables whose filter holds the query's
 * bucket, i.e. in which some member of the cell shares it):
 * cnt[r*B + gid[x][r]] counts table l once if some x has bucket[x][l] ==
 * qbucket[l]. For sampled queries on indices too large to rebuild here. */
void oracle_counts_direct(const uint32_t *bucket, const uint16_t *gid,
                          uint64_t N, uint32_t L, uint32_t R, uint32_t B,
                          const uint32_t *qbucket, uint16_t *cnt)
{
    const uint32_t BR = B * R;
    uint8_t *hit = (uint8_t *)malloc(BR ? BR : 1);
    for (uint32_t c = 0; c < BR; ++c) cnt[c] = 0;
    for (uint32_t l = 0; l < L; ++l) {
        memset(hit, 0, BR ? BR : 1);
        for (uint64_t x = 0; x < N; ++x)
            if (bucket[x * L + l] == qbucket[l])
                for (uint32_t r = 0; r < R; ++r) hit[r * B + gid[x * R + r]] = 1;
        for (uint32_t c = 0; c < BR; ++c) cnt[c] += hit[c];
    }
    free(hit);
}

/* Multi-probe counts (the multi-probe LSH idea the related work cites, as an
 * option): in table l the query probes its own bucket and the P - 1 buckets
 * that differ from it in exactly one of the code's bits 0 .. P-2 (SRP: the
 * sign of projection l*K + j flipped). A cell counts table l once if some
 * member's bucket in table l is one of those probes, so counts stay in
 * [0, L]. P = 1 is oracle_counts_direct. */
void oracle_counts_multiprobe(const uint32_t *bucket, const uint16_t *gid,
                              uint64_t N, uint32_t L, uint32_t R, uint32_t B,
                              const uint32_t *qbucket, uint32_t P, uint16_t *cnt)
{
    const uint32_t BR = B * R;
    uint8_t *hit = (uint8_t *)malloc(BR ? BR : 1);
    for (uint32_t c = 0; c < BR; ++c) cnt[c] = 0;
    for (uint32_t l = 0; l < L; ++l) {
        memset(hit, 0, BR ? BR : 1);
        for (uint64_t x = 0; x < N; ++x) {
            const uint32_t diff = bucket[x * L + l] ^ qbucket[l];
            int probed = diff == 0;
            for (uint32_t j = 0; j + 1 < P && !probed; ++j) probed = diff == (1u << j);
            if (probed)
                for (uint32_t r = 0; r < R; ++r) hit[r * B + gid[x * R + r]] = 1;
        }
        for (uint32_t c = 0; c < BR; ++c) cnt[c] += hit[c];
    }
    free(hit);
}

/* ------------------------------------------------------------------------ */
/* A7-A9: Alg. 3, threshold relaxation                                       */
/* ------------------------------------------------------------------------ */

static const uint16_t *g_sort_cnt;

static int cmp_cell(const void *p, const void *q)
{
    uint32_t a = *(const uint32_t *)p, b = *(const uint32_t *)q;
    if (g_sort_cnt[a] != g_sort_cnt[b]) return g_sort_cnt[a] > g_sort_cnt[b] ? -1 : 1;
    return (a > b) - (a < b);
}

/*
 * Alg. 3 for one query: A = all B*R cells sorted by count descending (ties:
 * cell id ascending). Walk the cells; a cell whose count is below t_min ends
 * the walk. For each member x (ascending id) increment Counts[x]; when it
 * reaches R, append x with score = the cell's count; stop at k results.
 * Unused output slots get id 0xFFFFFFFF and score 0. Returns #results.
 * counts_scratch: N bytes (R <= 255).
 */
static uint32_t alg3_one(const uint16_t *cnt, const uint64_t *moff,
                         const uint32_t *mem, uint64_t N, uint32_t R,
                         uint32_t B, uint32_t k, uint32_t t_min,
                         uint8_t *counts, uint32_t *order,
                         uint32_t *out_ids, uint16_t *out_scores, uint32_t k_max)
{
    const uint32_t BR = B * R;
    for (uint32_t i = 0; i < k_max; ++i) { out_ids[i] = 0xFFFFFFFFu; out_scores[i] = 0; }
    if (k == 0) return 0;
    for (uint32_t c = 0; c < BR; ++c) order[c] = c;
    g_sort_cnt = cnt;
    qsort(order, BR, sizeof(uint32_t), cmp_cell);
    memset(counts, 0, N);
    uint32_t nres = 0;
    for (uint32_t i = 0; i < BR; ++i) {
        uint32_t c = order[i];
        if (cnt[c] < t_min) break;
        uint32_t r = c / B, b = c % B;
        const uint64_t *o = moff + (uint64_t)r * (B + 1);
        for (uint64_t t = o[b]; t < o[b + 1]; ++t) {
            uint32_t x = mem[(uint64_t)r * N + t];
            if (++counts[x] == R) {
                out_ids[nres] = x;
                out_scores[nres] = cnt[c];
                if (++nres == k) return nres;
            }
        }
    }
    return nres;
}

/*
 * Full query for a batch: per query, counts from the reverse index (A6),
 * then Alg. 3. k: per-query k (NULL: k_max for all). Output nq x k_max.
 * Returns 0, or -1 if a k exceeds k_max.
 */
int oracle_query(const uint32_t *off, const uint16_t *cells, uint32_t L,
                 uint32_t W, const uint64_t *moff, const uint32_t *mem,
                 uint64_t N, uint32_t R, uint32_t B, uint32_t t_min,
                 const uint32_t *qbucket, uint64_t nq, const uint32_t *k,
                 uint32_t k_max, uint32_t *out_ids, uint16_t *out_scores)
{
    const uint32_t BR = B * R;
    uint16_t *cnt = (uint16_t *)malloc(sizeof(uint16_t) * (BR ? BR : 1));
    uint8_t *counts = (uint8_t *)malloc(N ? N : 1);
    uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * (BR ? BR : 1));
    int rc = 0;
    for (uint64_t q = 0; q < nq; ++q) {
        uint32_t kq = k ? k[q] : k_max;
        if (kq > k_max) { rc = -1; break; }
        oracle_counts(off, cells, L, W, qbucket + q * L, BR, cnt);
        alg3_one(cnt, moff, mem, N, R, B, kq, t_min, counts, order,
                 out_ids + q * k_max, out_scores + q * k_max, k_max);
    }
    free(cnt);
    free(counts);
    free(order);
    return rc;
}

/* Alg. 3 from given counts (used by tests to drive the decode directly). */
uint32_t oracle_alg3(const uint16_t *cnt, const uint64_t *moff,
                     const uint32_t *mem, uint64_t N, uint32_t R, uint32_t B,
                     uint32_t k, uint32_t t_min, uint32_t *out_ids,
                     uint16_t *out_scores, uint32_t k_max)
{
    uint8_t *counts = (uint8_t *)malloc(N ? N : 1);
    uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * ((B * R) != 0 ? (B * R) : 1));
    uint32_t n = alg3_one(cnt, moff, mem, N, R, B, k, t_min, counts, order,
                          out_ids, out_scores, k_max);
    free(counts);
    free(order);
    return n;
}
