// Synthetic embeddings streamed from a seed (the YFCC100M-shaped workload):
// not part of FLINNG, the input of its largest configuration, generated on
// the device so that 10^7 x 4096 vectors never need to be stored.
//
// Definitions (shared with the host generator, implemented separately):
//   Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11), key =
//   (seed low 32 bits, seed high 32 bits).
//   z(u0..u3) = (sum_i (u_i >> 10) - 2^23) * fp32(sqrt(3) * 2^-22): the sum of
//   four 22-bit uniforms, an approximate N(0, 1) (Irwin-Hall), one multiply.
//   centre[c][t] = z(philox(c, t, 0, 0xC0))
//   label[i]     = philox(i, 0, 1, 0xC0).x mod n_centers
//   point[i][t]  = ReLU(fma(sigma, z(philox(i, t, 2, 0xC0)), centre[label[i]][t]))
//   source[j]    = philox(j, 0, 3, 0xC0).x mod n_points
//   query[j][t]  = ReLU(fma(q_sigma, z(philox(j, t, 4, 0xC0)), pre[source[j]][t]))
// where pre is the point before ReLU and fma rounds once.
#include "internal.cuh"

namespace flinng {
namespace {

constexpr uint32_t kStream = 0xC0u;

__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ float irwin_hall(uint4 u)
{
    const int s = int(u.x >> 10) + int(u.y >> 10) + int(u.z >> 10) + int(u.w >> 10) - (1 << 23);
    return __fmul_rn(__int2float_rn(s), __int_as_float(0x34ddb3d7));   // sqrt(3) * 2^-22 in fp32
}

__device__ __forceinline__ float pre_value(const flinng_embed_spec &sp, uint32_t k0, uint32_t k1,
                                           uint32_t i, uint32_t t)
{
    const uint32_t lab = philox10(make_uint4(i, 0u, 1u, kStream), k0, k1).x % sp.n_centers;
    const float cen = irwin_hall(philox10(make_uint4(lab, t, 0u, kStream), k0, k1));
    const float z = irwin_hall(philox10(make_uint4(i, t, 2u, kStream), k0, k1));
    return __fmaf_rn(sp.sigma, z, cen);
}

__global__ void k_embed(flinng_embed_spec sp, int queries, uint64_t first, uint64_t n,
                        float *__restrict__ out, uint64_t ld)
{
    const uint32_t k0 = uint32_t(sp.seed), k1 = uint32_t(sp.seed >> 32);
    const uint64_t total = n * sp.dim;
    for (uint64_t e = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t row = e / sp.dim;
        const uint32_t t = uint32_t(e % sp.dim);
        const uint32_t i = uint32_t(first + row);
        float v;
        if (!queries) {
            v = pre_value(sp, k0, k1, i, t);
        } else {
            const uint32_t src = uint32_t(philox10(make_uint4(i, 0u, 3u, kStream), k0, k1).x % sp.n_points);
            const float pre = pre_value(sp, k0, k1, src, t);
            const float z = irwin_hall(philox10(make_uint4(i, t, 4u, kStream), k0, k1));
            v = __fmaf_rn(sp.q_sigma, z, pre);
        }
        out[row * ld + t] = v > 0.f ? v : 0.f;
    }
}

}  // namespace
}  // namespace flinng

using namespace flinng;

extern "C" int flinng_generate_embeddings(const flinng_embed_spec *spec, int queries, uint64_t first,
                                          uint64_t n, float *out, uint64_t ld, void *stream)
{
    if (!spec || (n > 0 && !out)) return set_error(FLINNG_ERR_INVALID_ARG, "generate: null argument");
    if (spec->dim == 0 || spec->n_centers == 0 || (queries && spec->n_points == 0) || ld < spec->dim)
        return set_error(FLINNG_ERR_INVALID_ARG, "generate: bad spec");
    if (first + n > (1ull << 32) || spec->n_points > (1ull << 32))
        return set_error(FLINNG_ERR_INVALID_ARG, "generate: indices must fit in 32 bits");
    if (n == 0) return FLINNG_OK;
    uint64_t blocks = (n * spec->dim + 255) / 256;
    if (blocks > 152ull * 64) blocks = 152ull * 64;
    k_embed<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(*spec, queries, first, n, out, ld);
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}
