// Exclusive prefix sum of uint32 counts (CSR offsets of the reverse index
// and of the member lists), reduce-then-scan: each tile of kTile values is
// summed (one read), the tile sums are scanned recursively, and each tile is
// scanned again with its offset added (one read, one write). A thread takes
// kItems consecutive values, as 16-byte accesses when both arrays are
// 16-byte aligned.
#include <cstdint>

#include "internal.cuh"

namespace flinng {

namespace {

constexpr int kScanThreads = 512;
constexpr int kItems = 16;
constexpr size_t kTile = size_t(kScanThreads) * kItems;

template <bool VEC>
__device__ __forceinline__ void load_items(const uint32_t *__restrict__ in, size_t base, size_t n, uint32_t *v)
{
    if (VEC && base + kItems <= n) {
#pragma unroll
        for (int i = 0; i < kItems; i += 4) {
            const uint4 x = *reinterpret_cast<const uint4 *>(in + base + i);
            v[i] = x.x;
            v[i + 1] = x.y;
            v[i + 2] = x.z;
            v[i + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kItems; ++i) v[i] = base + i < n ? in[base + i] : 0u;
    }
}

// Sum over the CTA; the result in every thread. Contains __syncthreads.
__device__ __forceinline__ uint32_t cta_sum(uint32_t x, uint32_t *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    if (lane == 0) red[warp] = x;
    __syncthreads();
    uint32_t t = lane < (kScanThreads >> 5) ? red[lane] : 0u;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
    return t;
}

template <bool VEC>
__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const uint32_t *__restrict__ in, size_t n, uint32_t *__restrict__ tile_sums)
{
    __shared__ uint32_t red[32];
    uint32_t v[kItems];
    load_items<VEC>(in, size_t(blockIdx.x) * kTile + size_t(threadIdx.x) * kItems, n, v);
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) s += v[i];
    s = cta_sum(s, red);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = s;
}

// tile_off: exclusive prefix of the tile sums (ntiles + 1 entries, total
// last); out[n] = the total.
template <bool VEC>
__global__ void __launch_bounds__(kScanThreads)
k_scan_down(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, size_t n,
            const uint32_t *__restrict__ tile_off, size_t ntiles)
{
    __shared__ uint32_t wtot[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t base = size_t(blockIdx.x) * kTile + size_t(threadIdx.x) * kItems;
    uint32_t v[kItems];
    load_items<VEC>(in, base, n, v);
    uint32_t tot = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) tot += v[i];
    uint32_t x = tot;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wtot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (kScanThreads >> 5) ? wtot[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        wtot[lane] = w;
    }
    __syncthreads();
    uint32_t run = tile_off[blockIdx.x] + (x - tot) + (warp > 0 ? wtot[warp - 1] : 0u);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const uint32_t e = v[i];
        v[i] = run;
        run += e;
    }
    if (VEC && base + kItems <= n) {
#pragma unroll
        for (int i = 0; i < kItems; i += 4)
            *reinterpret_cast<uint4 *>(out + base + i) = make_uint4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < kItems; ++i)
            if (base + i < n) out[base + i] = v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tile_off[ntiles];
}

// Scan of a single tile's worth (the recursion's last level): one CTA.
__global__ void __launch_bounds__(kScanThreads)
k_scan_single(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, size_t n)
{
    __shared__ uint32_t wtot[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t base = size_t(threadIdx.x) * kItems;
    uint32_t v[kItems];
    load_items<false>(in, base, n, v);
    uint32_t tot = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) tot += v[i];
    uint32_t x = tot;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wtot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (kScanThreads >> 5) ? wtot[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        wtot[lane] = w;
    }
    __syncthreads();
    uint32_t run = (x - tot) + (warp > 0 ? wtot[warp - 1] : 0u);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == kScanThreads - 1) out[n] = wtot[(kScanThreads >> 5) - 1];
}

}  // namespace

size_t scan_workspace_bytes(size_t n)
{
    size_t b = 0;
    while (n > kTile) {
        const size_t t = (n + kTile - 1) / kTile;
        b += carve_bytes<uint32_t>(t) + carve_bytes<uint32_t>(t + 1);
        n = t;
    }
    return b + 256;
}

int scan_exclusive(const uint32_t *in, uint32_t *out, size_t n, void *ws, cudaStream_t st)
{
    if (n <= kTile) {
        k_scan_single<<<1, kScanThreads, 0, st>>>(in, out, n);
        count_launch();
        FL_CUDA(cudaGetLastError());
        return FLINNG_OK;
    }
    const size_t ntiles = (n + kTile - 1) / kTile;
    Carver c(ws, ~size_t(0));
    uint32_t *sums = c.take<uint32_t>(ntiles);
    uint32_t *offs = c.take<uint32_t>(ntiles + 1);
    const bool vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
    if (vec) k_scan_reduce<true><<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, sums);
    else k_scan_reduce<false><<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, sums);
    count_launch();
    FL_CUDA(cudaGetLastError());
    FL_TRY(scan_exclusive(sums, offs, ntiles, c.base + ((c.used + 255) & ~size_t(255)), st));
    if (vec) k_scan_down<true><<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, out, n, offs, ntiles);
    else k_scan_down<false><<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, out, n, offs, ntiles);
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}

}  // namespace flinng
