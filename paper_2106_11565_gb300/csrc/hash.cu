// LSH hashing of points and queries (Sec. 3.2, Sec. 5: the L shared hash
// functions, each the concatenation of K base hashes).
//
// Cosine: sign random projections. bit j of table l = (w_{lK+j} . x > 0),
// table bucket = the K bits, bit j at position j. The sign is exact: an FP32
// tile GEMM computes p~ and a rigorous bound on |p~ - p|; the few
// projections whose |p~| does not clear the bound are recomputed in fp64
// (fp32 x fp32 products are exact in fp64) and, if still ambiguous, summed
// exactly in a fixed-point long accumulator.
//
// Jaccard: densified one-permutation MinHash. pi(e) = a e + b mod 2^32,
// nb = L*K bins of the 32-bit range, bin value = min pi(e) in the bin; an
// empty bin copies the value of the first originally non-empty bin among
// j = splitmix64(seed ^ (i << 32 | attempt)) mod nb, attempt = 1, 2, ...
// (4096 tries, then the next non-empty bin cyclically). Table l combines its
// K values as ((sum_j a_{l,j} v_{lK+j} + c_l) mod 2^64) >> (64 - W).
#include "internal.cuh"

namespace flinng {

namespace {

// ------------------------------------------------------------------ SRP

constexpr int kBM = 128, kBN = 64, kBK = 16, kSrpThreads = 256;   // 8 x 4 outputs per thread
constexpr int kSrpChunkRows = 1 << 14;

__global__ void __launch_bounds__(kSrpThreads)
k_srp_fp32(const float *__restrict__ X, uint64_t ldx, uint64_t n,
           const float *__restrict__ Wm, uint32_t P, uint32_t d, uint32_t L,
           uint32_t K, float gamma2, float tiny, uint32_t *__restrict__ codes,
           float *__restrict__ proj, unsigned long long *__restrict__ rlist,
           unsigned long long *__restrict__ rcount)
{
    __shared__ __align__(16) float As[kBK][kBM + 4];
    __shared__ __align__(16) float Bs[kBK][kBN + 4];
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    const uint64_t row0 = uint64_t(blockIdx.x) * kBM;
    const uint32_t col0 = blockIdx.y * kBN;
    float p[8][4], s[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) p[i][j] = s[i][j] = 0.f;

    for (uint32_t k0 = 0; k0 < d; k0 += kBK) {
#pragma unroll
        for (int e = 0; e < (kBM * kBK) / kSrpThreads; ++e) {
            const int idx = tid + e * kSrpThreads;
            const int r = idx / kBK, kk = idx % kBK;
            const uint64_t gr = row0 + r;
            const uint32_t gk = k0 + kk;
            As[kk][r] = (gr < n && gk < d) ? X[gr * ldx + gk] : 0.f;
        }
#pragma unroll
        for (int e = 0; e < (kBN * kBK) / kSrpThreads; ++e) {
            const int idx = tid + e * kSrpThreads;
            const int r = idx / kBK, kk = idx % kBK;
            const uint32_t gc = col0 + r, gk = k0 + kk;
            Bs[kk][r] = (gc < P && gk < d) ? Wm[uint64_t(gc) * d + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            // k in order for every output, as before: the sums are the same
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][ty * 8 + 4]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    p[i][j] = fmaf(a[i], b[j], p[i][j]);
                    s[i][j] = fmaf(fabsf(a[i]), fabsf(b[j]), s[i][j]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint64_t gr = row0 + ty * 8 + i;
        if (gr >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t gc = col0 + tx * 4 + j;
            if (gc >= P) continue;
            if (proj) proj[gr * P + gc] = p[i][j];
            const float margin = fmaf(gamma2, s[i][j], tiny);
            if (fabsf(p[i][j]) > margin) {
                if (p[i][j] > 0.f) atomicOr(&codes[gr * L + gc / K], 1u << (gc % K));
            } else {
                const unsigned long long slot = atomicAdd(rcount, 1ull);
                rlist[slot] = (p[i][j] > 0.f ? kEntSign : 0ull) | ((unsigned long long)gr << 20) | gc;
            }
        }
    }
}

// Exact sign of sum_t a_t b_t with fp32 inputs: each product is an fp64
// value m * 2^(e-1075) with a 53-bit integer m; digits of 32 bits starting
// at 2^-384, kept in int64 so that sums over lanes and terms cannot overflow.
constexpr int kLimbs = 24;
constexpr int kLimbBias = 384;

__device__ void limb_add(long long *acc, double v)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int ex = int((bits >> 52) & 0x7FF);
    unsigned long long man = bits & ((1ull << 52) - 1);
    if (ex == 0 && man == 0) return;
    int lsb;
    if (ex == 0) {
        lsb = 1 - 1075;
    } else {
        man |= 1ull << 52;
        lsb = ex - 1075;
    }
    const int pos = lsb + kLimbBias;
    const int q = pos >> 5, r = pos & 31;
    const unsigned long long d0 = (man << r) & 0xffffffffull;
    const unsigned long long d1 = (r == 0 ? (man >> 32) : (man >> (32 - r))) & 0xffffffffull;
    const unsigned long long d2 = (r == 0) ? 0ull : (man >> (64 - r));
    const long long sg = (bits >> 63) ? -1 : 1;
    acc[q] += sg * (long long)d0;
    acc[q + 1] += sg * (long long)d1;
    acc[q + 2] += sg * (long long)d2;
}

__device__ int limb_sign(long long *acc)
{
    for (int i = 0; i < kLimbs - 1; ++i) {
        const long long c = acc[i] >> 32;   // arithmetic shift: floor division
        acc[i] -= c * 4294967296ll;
        acc[i + 1] += c;
    }
    if (acc[kLimbs - 1] != 0) return acc[kLimbs - 1] > 0 ? 1 : -1;
    for (int i = kLimbs - 2; i >= 0; --i)
        if (acc[i] != 0) return 1;
    return 0;
}

__global__ void k_srp_recheck(const float *__restrict__ X, uint64_t ldx,
                              const float *__restrict__ Wm, uint32_t d, uint32_t L,
                              uint32_t K, double gamma2,
                              const unsigned long long *__restrict__ rlist,
                              const unsigned long long *__restrict__ rcount,
                              uint32_t *__restrict__ codes,
                              unsigned long long *__restrict__ stats)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long nlist = *rcount;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long e = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
         e < nlist; e += nwarps) {
        const unsigned long long ent = rlist[e];
        const uint64_t gr = ent_row(ent);
        const uint32_t gc = ent_col(ent);
        const float *xr = X + gr * ldx;
        const float *wr = Wm + uint64_t(gc) * d;
        double p = 0.0, s = 0.0;
        for (uint32_t t = lane; t < d; t += 32) {
            const double prod = double(xr[t]) * double(wr[t]);
            p += prod;
            s += fabs(prod);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            p += __shfl_xor_sync(0xffffffffu, p, o);
            s += __shfl_xor_sync(0xffffffffu, s, o);
        }
        p = __shfl_sync(0xffffffffu, p, 0);
        s = __shfl_sync(0xffffffffu, s, 0);
        int positive;
        if (fabs(p) > gamma2 * s) {
            positive = p > 0.0;
        } else {
            long long acc[kLimbs + 2];
            for (int i = 0; i < kLimbs + 2; ++i) acc[i] = 0;
            for (uint32_t t = lane; t < d; t += 32) limb_add(acc, double(xr[t]) * double(wr[t]));
            for (int i = 0; i < kLimbs + 2; ++i) {
                long long v = acc[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                acc[i] = v;
            }
            // digits kLimbs, kLimbs+1 stay zero: fold them for safety
            acc[kLimbs - 1] += acc[kLimbs] * 4294967296ll;
            positive = limb_sign(acc) > 0;
            if (lane == 0) atomicAdd(&stats[1], 1ull);
        }
        if (lane == 0) {
            if (positive) atomicOr(&codes[gr * L + gc / K], 1u << (gc % K));
            atomicAdd(&stats[2], 1ull);
            if (positive != ((ent & kEntSign) != 0)) atomicAdd(&stats[4], 1ull);
        }
    }
}

__global__ void k_add_counter(unsigned long long *dst, const unsigned long long *src)
{
    *dst += *src;
}

// ------------------------------------------------------------------ DOPH

constexpr int kDophWarps = 8;
constexpr int kDophUnroll = 4;     // element loads in flight per lane

__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(kDophWarps * 32)
k_doph(const uint64_t *__restrict__ off, const uint32_t *__restrict__ elems,
       uint64_t n, uint32_t nb, uint32_t a, uint32_t b, uint64_t seed, uint32_t L,
       uint32_t K, uint32_t W, const uint64_t *__restrict__ ba,
       const uint64_t *__restrict__ bc, uint32_t *__restrict__ buckets,
       uint32_t *__restrict__ values)
{
    extern __shared__ uint32_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nbw = (nb + 31) / 32;
    uint32_t *val = sm + warp * (nb + nbw);
    uint32_t *occ = val + nb;
    const uint64_t gw = uint64_t(blockIdx.x) * kDophWarps + warp;
    const uint64_t stride = uint64_t(gridDim.x) * kDophWarps;
    for (uint64_t i = gw; i < n; i += stride) {
        for (uint32_t k = lane; k < nb; k += 32) val[k] = kEmpty32;
        for (uint32_t k = lane; k < nbw; k += 32) occ[k] = 0u;
        __syncwarp();
        const uint64_t beg = off[i], end = off[i + 1];
        // four element loads in flight per lane, then their bins
        for (uint64_t t0 = beg + lane; t0 < end; t0 += 32 * kDophUnroll) {
            uint32_t e[kDophUnroll];
#pragma unroll
            for (int u = 0; u < kDophUnroll; ++u) {
                const uint64_t t = t0 + 32u * u;
                e[u] = t < end ? elems[t] : 0u;
            }
#pragma unroll
            for (int u = 0; u < kDophUnroll; ++u) {
                if (t0 + 32u * u >= end) break;
                const uint32_t pe = a * e[u] + b;
                const uint32_t bin = __umulhi(pe, nb);
                atomicMin(&val[bin], pe);
                // a bin is occupied iff its minimum is below the empty marker,
                // or an element hashes to the marker's value itself (flagged
                // here; every other occupancy bit is read off val below, with
                // no atomic per element on the few bitmap words)
                if (pe == kEmpty32) atomicOr(&occ[bin >> 5], 1u << (bin & 31));
            }
        }
        __syncwarp();
        for (uint32_t k0 = 0; k0 < nb; k0 += 32) {                 // a ballot per 32 bins
            const uint32_t k = k0 + lane;
            const uint32_t bits = __ballot_sync(0xffffffffu, k < nb && val[k] != kEmpty32);
            if (lane == 0) occ[k0 >> 5] |= bits;
        }
        __syncwarp();
        if (end > beg) {
            const bool pow2 = (nb & (nb - 1u)) == 0u;     // z mod nb is a mask then
            for (uint32_t k = lane; k < nb; k += 32) {
                if ((occ[k >> 5] >> (k & 31)) & 1u) continue;
                bool found = false;
                for (uint32_t att = 1; att <= kDophMaxAttempts; ++att) {
                    const uint64_t z = splitmix64(seed ^ ((uint64_t(k) << 32) | att));
                    const uint32_t j = pow2 ? uint32_t(z) & (nb - 1u) : uint32_t(z % nb);
                    if ((occ[j >> 5] >> (j & 31)) & 1u) {
                        val[k] = val[j];
                        found = true;
                        break;
                    }
                }
                if (!found) {
                    for (uint32_t s = 1; s <= nb; ++s) {
                        const uint32_t j = (k + s) % nb;
                        if ((occ[j >> 5] >> (j & 31)) & 1u) {
                            val[k] = val[j];
                            break;
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (values)
            for (uint32_t k = lane; k < nb; k += 32) values[i * nb + k] = val[k];
        for (uint32_t l = lane; l < L; l += 32) {
            uint64_t h = bc[l];
            for (uint32_t j = 0; j < K; ++j) h += ba[l * K + j] * uint64_t(val[l * K + j]);
            buckets[i * L + l] = uint32_t(h >> (64 - W));
        }
        __syncwarp();
    }
}

}  // namespace

int add_counter(unsigned long long *dst, const unsigned long long *src, cudaStream_t st)
{
    k_add_counter<<<1, 1, 0, st>>>(dst, src);
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}

int srp_recheck_list(flinng_index *ix, const float *x, uint64_t ld, const unsigned long long *list,
                     const unsigned long long *count, uint32_t *codes)
{
    k_srp_recheck<<<152 * 4, 256, 0, ix->stream>>>(x, ld, ix->srp_w, ix->cfg.dim, ix->cfg.L, ix->cfg.K,
                                                   ix->srp_gamma64, list, count, codes, ix->stats);
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}

size_t srp_workspace_bytes(const flinng_index *ix, uint64_t n)
{
    if (ix->cfg.precision != FLINNG_PREC_FP32) return srp_tc_workspace_bytes(ix, n);
    const uint64_t rows = n < uint64_t(kSrpChunkRows) ? n : uint64_t(kSrpChunkRows);
    return carve_bytes<unsigned long long>(2) + carve_bytes<unsigned long long>(rows * ix->P + 1);
}

int srp_hash(flinng_index *ix, const float *x, uint64_t ld, uint64_t n,
             uint32_t *buckets, float *proj, void *ws, size_t ws_bytes)
{
    (void)ws_bytes;
    if (ix->cfg.precision != FLINNG_PREC_FP32) return srp_hash_tc(ix, x, ld, n, buckets, proj, ws);
    const cudaStream_t st = ix->stream;
    const uint32_t L = ix->cfg.L, K = ix->cfg.K, d = ix->cfg.dim, P = ix->P;
    Carver c(ws, ~size_t(0));
    unsigned long long *rcount = c.take<unsigned long long>(2);
    unsigned long long *rlist = c.take<unsigned long long>(uint64_t(kSrpChunkRows) * P + 1);
    FL_CUDA(cudaMemsetAsync(ix->stats, 0, kStats * sizeof(unsigned long long), st));
    if (n == 0) return FLINNG_OK;
    FL_CUDA(cudaMemsetAsync(buckets, 0, n * L * sizeof(uint32_t), st));
    // fp32 bound: 2 * gamma_d * sum|w x| + d * 2^-146 (underflow), see header comment
    const float tiny = float(d) * ldexpf(1.0f, -146);
    for (uint64_t r0 = 0; r0 < n; r0 += kSrpChunkRows) {
        const uint64_t rows = (n - r0) < uint64_t(kSrpChunkRows) ? (n - r0) : uint64_t(kSrpChunkRows);
        FL_CUDA(cudaMemsetAsync(rcount, 0, sizeof(unsigned long long), st));
        dim3 grid((unsigned)((rows + kBM - 1) / kBM), (P + kBN - 1) / kBN);
        k_srp_fp32<<<grid, kSrpThreads, 0, st>>>(x + r0 * ld, ld, rows, ix->srp_w, P, d, L, K,
                                                 ix->srp_margin_gamma, tiny, buckets + r0 * L,
                                                 proj ? proj + r0 * P : nullptr, rlist, rcount);
        count_launch();
        FL_CUDA(cudaGetLastError());
        FL_TRY(add_counter(ix->stats, rcount, st));        // undecided after the fp32 pass
        k_srp_recheck<<<152 * 4, 256, 0, st>>>(x + r0 * ld, ld, ix->srp_w, d, L, K, ix->srp_gamma64,
                                               rlist, rcount, buckets + r0 * L, ix->stats);
        count_launch();
        FL_CUDA(cudaGetLastError());
    }
    return FLINNG_OK;
}

int doph_hash(flinng_index *ix, const uint64_t *off, const uint32_t *elems,
              uint64_t n, uint32_t *buckets, uint32_t *values)
{
    if (n == 0) return FLINNG_OK;
    const uint32_t nb = ix->P;
    const size_t smem = size_t(kDophWarps) * (nb + (nb + 31) / 32) * sizeof(uint32_t);
    FL_TRY(ensure_dyn_smem((const void *)k_doph, smem));
    uint64_t blocks = (n + kDophWarps - 1) / kDophWarps;
    if (blocks > 152ull * 64) blocks = 152ull * 64;
    k_doph<<<(unsigned)blocks, kDophWarps * 32, smem, ix->stream>>>(
        off, elems, n, nb, ix->doph_a, ix->doph_b, ix->doph_seed, ix->cfg.L, ix->cfg.K,
        ix->cfg.range_bits, ix->bucket_a, ix->bucket_c, buckets, values);
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}

}  // namespace flinng
