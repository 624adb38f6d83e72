// Exclusive prefix sum of uint32 counts (CSR offsets of the reverse index
// and of the member lists). Tiles of 4096 values are scanned in shared
// memory; the per-tile totals are scanned recursively and added back.
#include "internal.cuh"

namespace flinng {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr size_t kTile = size_t(kScanThreads) * kScanItems;

__global__ void __launch_bounds__(kScanThreads)
k_scan_tile(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, size_t n,
            uint32_t *__restrict__ tile_sums)
{
    __shared__ uint32_t warp_tot[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t base = size_t(blockIdx.x) * kTile + size_t(threadIdx.x) * kScanItems;
    uint32_t v[kScanItems];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) v[i] = (base + i < n) ? in[base + i] : 0u;
    uint32_t incl[kScanItems];
    incl[0] = v[0];
#pragma unroll
    for (int i = 1; i < kScanItems; ++i) incl[i] = incl[i - 1] + v[i];
    const uint32_t tot = incl[kScanItems - 1];
    uint32_t x = tot;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < (kScanThreads >> 5)) ? warp_tot[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    const uint32_t pre = (x - tot) + (warp > 0 ? warp_tot[warp - 1] : 0u);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) out[base + i] = pre + incl[i] - v[i];
    if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = warp_tot[(kScanThreads >> 5) - 1];
}

__global__ void k_scan_add(uint32_t *__restrict__ out, size_t n,
                           const uint32_t *__restrict__ tile_off, size_t ntiles)
{
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_off[i / kTile];
    if (i == 0) out[n] = tile_off[ntiles];
}

__global__ void k_scan_total(uint32_t *__restrict__ out, size_t n,
                             const uint32_t *__restrict__ tile_sums)
{
    out[n] = tile_sums[0];
}

}  // namespace

size_t scan_workspace_bytes(size_t n)
{
    size_t b = 0;
    while (n > 0) {
        size_t t = (n + kTile - 1) / kTile;
        b += carve_bytes<uint32_t>(t) + carve_bytes<uint32_t>(t + 1);
        if (t == 1) break;
        n = t;
    }
    return b + 256;
}

int scan_exclusive(const uint32_t *in, uint32_t *out, size_t n, void *ws,
                   cudaStream_t st)
{
    if (n == 0) {
        FL_CUDA(cudaMemsetAsync(out, 0, sizeof(uint32_t), st));
        return FLINNG_OK;
    }
    const size_t ntiles = (n + kTile - 1) / kTile;
    Carver c(ws, ~size_t(0));
    uint32_t *sums = c.take<uint32_t>(ntiles);
    uint32_t *offs = c.take<uint32_t>(ntiles + 1);
    k_scan_tile<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, out, n, sums);
    count_launch();
    FL_CUDA(cudaGetLastError());
    if (ntiles == 1) {
        k_scan_total<<<1, 1, 0, st>>>(out, n, sums);
        count_launch();
        FL_CUDA(cudaGetLastError());
        return FLINNG_OK;
    }
    FL_TRY(scan_exclusive(sums, offs, ntiles, c.base + ((c.used + 255) & ~size_t(255)), st));
    const unsigned blocks = (unsigned)((n + 255) / 256);
    k_scan_add<<<blocks, 256, 0, st>>>(out, n, offs, ntiles);
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}

}  // namespace flinng
