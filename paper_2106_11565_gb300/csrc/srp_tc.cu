// Sign random projections on the tensor cores (the precision form): the
// dense contraction P = X W^T runs on tcgen05 with BF16 operands and FP32
// accumulation in tensor memory, and the sign bits stay exact.
//
// Exactness. Each fp32 operand is split as x1 = bf16(x), x2 = bf16(x - x1),
// so |x - x1 - x2| <= 2^-16 |x| (bf16 keeps 8 significant bits); likewise w.
// bf16 x bf16 products are exact in fp32. Per 64-wide k-block s the tensor
// cores compute hi_s = sum x1 w1 and lo_s = sum (x1 w2 + x2 w1) into a fresh
// pair of TMEM accumulators; the epilogue adds hi_s + lo_s into an fp32
// register per projection. Short accumulation chains keep the bound tight:
//   |p~ - w.x| <= [g'(64) + 2^-7 g'(128)] (1 + 2^-8)^2 ||x|| ||w||      (blocks)
//              + g(2m) (1 + g'(64)) (1 + 2^-7) (1 + 2^-8)^2 ||x|| ||w||  (sum of m blocks)
//              + 3.1 * 2^-16 ||x|| ||w||                                 (split)
//              + 8 d 2^-126 + sqrt(d) 2^-125 (||x|| + ||w||)           (underflow, flushes)
// with g(n) = n u / (1 - n u), u = 2^-24, and g' the same with u' = 2^-22:
// four units of fp32 rounding per product accumulated, which also covers a
// tensor-core adder that aligns and truncates. Projections whose |p~| does
// not clear that margin go to a compensated fp32 re-check (two-product,
// two-sum), and the few that stay ambiguous to the fp64 / exact re-check of
// hash.cu.
//
// Single-term forms. FLINNG_PREC_BF16 keeps x1 = bf16(x) only; FLINNG_PREC_FP8
// keeps xq = e4m3(x / s) with a power-of-two scale s per row (s chosen so the
// row's largest |x| / s <= 448; values that would be E4M3 subnormals become
// 0). The quantiser records each row's residual norm ||e_x|| = ||x - s xq||
// (exact fp64 differences, rounded up); with ||x|| and the same for every
// projection row w,
//   |w.x - s_x s_w sum xq wq| <= ||x|| ||e_w|| + ||e_x|| ||w|| + 3 ||e_x|| ||e_w||
// (Cauchy-Schwarz on x = s_x xq + e_x, w = s_w wq + e_w). The tensor cores sum
// the products of one k-block (64 bf16 or 128 e4m3 values) exactly-multiplied
// into fp32 (per-product error u' = 2^-22 of the running magnitude), the
// epilogue adds the blocks in fp32 and scales by s_x s_w (exact), so the
// margin is that residual term plus [g'(kb) + g(m)(1 + g'(kb))] (||x|| +
// ||e_x||) (||w|| + ||e_w||), 2^-23 |p~|, the underflow terms above, and a
// 2^-20 relative slack for evaluating the margin itself in fp32.
//
// Kernel layout (one CTA per 128 points x 128 projections, 320 threads):
//   warp 0     TMA producer: 3-stage ring of {X1, X2, W1, W2} tiles of 128 rows
//              x 64 bf16 (128-byte swizzle), one mbarrier per stage (single-term
//              forms: a 6-stage ring of {X, W} tiles of 128 rows x 128 bytes);
//   warp 1     allocates 512 TMEM columns (two buffers of {hi, lo}); one elected
//              thread issues the MMAs of k-block s into buffer s % 2 - per 16-wide
//              step x1 [w1 w2] (M=128, N=256: hi and the x1 w2 half of lo) and
//              x2 w1 (N=128, into lo) - then commits the stage back to the
//              producer and the buffer to the epilogue (single-term forms: one
//              N=128 MMA per 32-byte step into a 128-column buffer);
//   warps 2-9  epilogue: warp w reads TMEM lanes 32 (w % 4) .. +32 (one point per
//              thread) and 64 of the 128 columns, drains each buffer into fp32
//              registers and hands it back; at the end decides the signs,
//              writes the codes and lists ambiguous projections.
// Every wait on an mbarrier is bounded; on timeout the CTA sets an error flag,
// stops issuing work, waits (bounded) for its copies and MMAs, and frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "internal.cuh"

namespace flinng {
namespace {

constexpr int kTM = 128, kTN = 128, kTK = 64;     // tile rows, projections, bf16 K per stage
constexpr int kTileBytes = kTM * 128;             // 16 KB per operand tile (128-byte rows)
// forms of the kernel
constexpr int kFormBf16x2 = 0, kFormBf16 = 1, kFormFp8 = 2;

template <int FORM> struct TcForm;
template <> struct TcForm<kFormBf16x2> {
    static constexpr int kTiles = 4, kStages = 3, kKElems = 64;   // X1, X2, W1, W2
    static constexpr uint32_t kTmemCols = 512;                    // buffer b: hi at 256 b, lo at 256 b + 128
};
template <> struct TcForm<kFormBf16> {
    static constexpr int kTiles = 2, kStages = 6, kKElems = 64;   // X, W
    static constexpr uint32_t kTmemCols = 256;                    // buffer b at 128 b
};
template <> struct TcForm<kFormFp8> {
    static constexpr int kTiles = 2, kStages = 6, kKElems = 128;
    static constexpr uint32_t kTmemCols = 256;
};
template <int FORM>
constexpr size_t tc_smem_bytes() { return size_t(TcForm<FORM>::kStages) * TcForm<FORM>::kTiles * kTileBytes + 1024 + 256; }
constexpr int kEpiWarps = 8;                      // two per TMEM lane quarter, 64 columns each
constexpr int kTcThreads = 64 + 32 * kEpiWarps;
constexpr uint64_t kWaitNs = 1000000000ull;       // bounded mbarrier waits: 1 s
constexpr uint64_t kTcChunkRows = 16384;          // rows split and hashed per launch
constexpr size_t kRecheckRowBytes = 160 * 1024;   // largest row of x the re-check stages in shared memory

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: false if the phase has not completed within limit_ns
// (0: a single try).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns = kWaitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    if (limit_ns == 0) return false;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 256; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= uint64_t((addr & 0x3FFFFu) >> 4);
    d |= uint64_t(1) << 16;                 // leading byte offset (unused with 128B swizzle, K-major)
    d |= uint64_t(1024 >> 4) << 32;         // stride byte offset
    d |= uint64_t(1) << 46;                 // version
    d |= uint64_t(2) << 61;                 // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D fp32, A and B bf16, both K-major,
// M = 128 rows, N columns.
template <int N>
__host__ __device__ constexpr uint32_t mma_idesc()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(kTM >> 4) << 24);
}

template <int N>
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(mma_idesc<N>()), "r"(accumulate)
        : "memory");
}

// Instruction descriptor, kind::f8f6f4: D fp32, A and B E4M3 (format 0), both
// K-major, M = 128 rows, N columns.
template <int N>
__host__ __device__ constexpr uint32_t mma_idesc_e4m3()
{
    return (1u << 4) | (uint32_t(N >> 3) << 17) | (uint32_t(kTM >> 4) << 24);
}

template <int N>
__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(mma_idesc_e4m3<N>()), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

// 32 consecutive fp32 columns of this warp's 32 TMEM lanes; the caller waits
// (tmem_wait_ld) before reading the registers.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t r[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcArgs {
    uint64_t n;            // rows (points) in this launch
    uint32_t P, d, L, K;
    const float *xnorm;    // n: upper bounds of ||x||
    const float *wnorm;    // P: upper bounds of ||w||
    const float *xres;     // single-term forms: n upper bounds of ||x - s_x xq||
    const float *wres;     // P upper bounds of ||w - s_w wq||
    const float *xscale;   // FP8: n row scales s_x (powers of two)
    const float *wscale;   // FP8: P row scales s_w
    float c_norm;          // margin factor on ||x|| ||w||
    float c_sub;           // margin factor on ||x|| + ||w|| (subnormal flushes)
    float tiny;            // absolute margin (underflow)
    uint32_t *codes;       // n x L (zeroed)
    float *proj;           // optional n x P
    unsigned long long *rlist;
    unsigned long long *rcount;
    uint32_t *err;         // set to 1 on a wait timeout
    uint64_t wait_ns;      // limit of the pipeline's waits (the drains after an abort keep kWaitNs)
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int FORM>
__global__ void __launch_bounds__(kTcThreads, 1)
k_srp_tc(const __grid_constant__ CUtensorMap mx1, const __grid_constant__ CUtensorMap mx2,
         const __grid_constant__ CUtensorMap mw1, const __grid_constant__ CUtensorMap mw2, TcArgs a)
{
    using F = TcForm<FORM>;
    constexpr int kStages = F::kStages;
    constexpr int kStageBytes = F::kTiles * kTileBytes;
    constexpr int kW = F::kTiles / 2;                 // tile index of the first W tile in a stage
    constexpr uint32_t kBuf = F::kTmemCols / 2;        // TMEM columns per buffer
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    // 1024-byte aligned tile ring, then barriers and the TMEM address
    unsigned char *ring = tc_smem + ((1024u - (smem_u32(tc_smem) & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + kStages * kStageBytes);
    uint64_t *empty = full + kStages;        // stage consumed by the MMAs
    uint64_t *tfull = empty + kStages;       // TMEM buffer b holds a finished k-block
    uint64_t *tempty = tfull + 2;            // TMEM buffer b drained by the epilogue
    uint64_t *mdone = tempty + 2;            // every MMA issued has completed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mdone + 1);
    uint32_t *abort_flag = tmem_slot + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // projection blocks vary fastest: the CTAs that share one X tile run in
    // the same wave, so X is read from DRAM once and W stays in L2
    const uint32_t row0 = blockIdx.y * kTM, col0 = blockIdx.x * kTN;
    const uint32_t nkb = (a.d + F::kKElems - 1) / F::kKElems;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kEpiWarps);
        }
        mbar_init(mdone, 1);
        *abort_flag = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(F::kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    uint32_t issued = 0;   // producer: k-blocks whose copies were issued
    if (warp == 0) {
        if (lane == 0) {
            for (uint32_t kb = 0; kb < nkb; ++kb) {
                const int s = kb % kStages;
                if (kb >= uint32_t(kStages) && !mbar_wait(&empty[s], ((kb / kStages) - 1) & 1, a.wait_ns)) {
                    atomicExch(abort_flag, 1u);
                    break;
                }
                if (*(volatile uint32_t *)abort_flag) break;
                unsigned char *st = ring + s * kStageBytes;
                mbar_expect_tx(&full[s], kStageBytes);
                const int kx = int(kb * F::kKElems);
                tma_load_2d(st + 0 * kTileBytes, &mx1, &full[s], kx, int(row0));
                if constexpr (F::kTiles == 4) tma_load_2d(st + 1 * kTileBytes, &mx2, &full[s], kx, int(row0));
                tma_load_2d(st + kW * kTileBytes, &mw1, &full[s], kx, int(col0));
                if constexpr (F::kTiles == 4) tma_load_2d(st + 3 * kTileBytes, &mw2, &full[s], kx, int(col0));
                issued = kb + 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (uint32_t kb = 0; kb < nkb; ++kb) {
                const int s = kb % kStages;
                const uint32_t b = kb & 1u;
                if (!mbar_wait(&full[s], (kb / kStages) & 1, a.wait_ns) ||
                    (kb >= 2 && !mbar_wait(&tempty[b], ((kb >> 1) - 1) & 1, a.wait_ns))) {
                    atomicExch(abort_flag, 1u);
                    break;
                }
                if (*(volatile uint32_t *)abort_flag) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t st = smem_u32(ring + s * kStageBytes);
                const uint32_t t_hi = tmem + kBuf * b;
                // four 32-byte K steps per 128-byte stage row: 16 bf16 or 32 e4m3
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t off = kk * 32;
                    const uint32_t acc = kk > 0 ? 1u : 0u;     // each k-block starts a fresh accumulator
                    if constexpr (FORM == kFormBf16x2) {
                        // W1 and W2 tiles are adjacent in the stage, so [W1; W2] is one
                        // 256-row B operand: x1 [w1 w2] fills hi and lo in one MMA
                        // (N = 256), then x2 w1 adds into lo (N = 128)
                        const uint64_t x1 = smem_desc(st + 0 * kTileBytes + off);
                        const uint64_t x2 = smem_desc(st + 1 * kTileBytes + off);
                        const uint64_t w12 = smem_desc(st + 2 * kTileBytes + off);
                        mma_bf16<2 * kTN>(t_hi, x1, w12, acc);
                        mma_bf16<kTN>(t_hi + kTN, x2, w12, 1u);
                    } else {
                        const uint64_t xd = smem_desc(st + off);
                        const uint64_t wd = smem_desc(st + kTileBytes + off);
                        if constexpr (FORM == kFormBf16) mma_bf16<kTN>(t_hi, xd, wd, acc);
                        else mma_e4m3<kTN>(t_hi, xd, wd, acc);
                    }
                }
                mma_commit(&empty[s]);
                mma_commit(&tfull[b]);
            }
            mma_commit(mdone);     // arrives once every MMA issued above has completed
        }
    } else {
        // epilogue: TMEM lanes [32 (warp % 4), +32) = one point per thread;
        // columns [64 half, +64) of the tile
        const uint32_t quarter = (warp & 3) * 32;
        const uint32_t half = uint32_t(warp - 2) >> 2;
        const uint32_t tbase = tmem + (quarter << 16) + 64u * half;
        float acc[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) acc[j] = 0.f;
        bool abort = false;
        for (uint32_t kb = 0; kb < nkb; ++kb) {
            const uint32_t b = kb & 1u;
            uint32_t got = 0;
            if (lane == 0) got = mbar_wait(&tfull[b], (kb >> 1) & 1, a.wait_ns) ? 1u : 0u;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) {
                if (lane == 0) atomicExch(abort_flag, 1u);
                abort = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if constexpr (FORM == kFormBf16x2) {
                // two halves of 32 columns: hi and lo loads in flight together, one
                // wait each; the buffer goes back to the MMA issuer before the
                // second half is added
                uint32_t hv[32], lv[32];
                tmem_ld32(tbase + kBuf * b, hv);
                tmem_ld32(tbase + kBuf * b + kTN, lv);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] += __uint_as_float(hv[j]) + __uint_as_float(lv[j]);
                tmem_ld32(tbase + kBuf * b + 32, hv);
                tmem_ld32(tbase + kBuf * b + kTN + 32, lv);
                tmem_wait_ld();
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[b]);
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[32 + j] += __uint_as_float(hv[j]) + __uint_as_float(lv[j]);
            } else {
                uint32_t hv[32], hw[32];
                tmem_ld32(tbase + kBuf * b, hv);
                tmem_ld32(tbase + kBuf * b + 32, hw);
                tmem_wait_ld();
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[b]);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    acc[j] += __uint_as_float(hv[j]);
                    acc[32 + j] += __uint_as_float(hw[j]);
                }
            }
        }
        uint32_t ab = lane == 0 ? *(volatile uint32_t *)abort_flag : 0u;
        abort = abort || __shfl_sync(0xffffffffu, ab, 0) != 0u;    // warp-uniform
        const uint64_t row = uint64_t(row0) + quarter + lane;
        if (!abort && row < a.n) {
            const float xn = a.xnorm[row];
            float xr = 0.f, xs = 1.f;
            if constexpr (FORM != kFormBf16x2) xr = a.xres[row];
            if constexpr (FORM == kFormFp8) xs = a.xscale[row];
            uint32_t cur_l = 0xFFFFFFFFu, cur_bits = 0u;
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                const uint32_t col = col0 + 64u * half + j;
                if (col >= a.P) break;
                float p = acc[j];
                if constexpr (FORM == kFormFp8) p *= xs * a.wscale[col];    // powers of two: exact
                const float wn = a.wnorm[col];
                if (a.proj) a.proj[row * a.P + col] = p;
                float margin;
                if constexpr (FORM == kFormBf16x2) {
                    margin = fmaf(a.c_norm * xn, wn, fmaf(ldexpf(1.f, -23), fabsf(p), fmaf(a.c_sub, xn + wn, a.tiny)));
                } else {
                    // residual term (Cauchy-Schwarz on the quantisation errors) plus
                    // accumulation on the quantised operands' norms, then slack
                    const float wr = a.wres[col];
                    const float resid = fmaf(xn, wr, fmaf(xr, wn, 3.f * xr * wr));
                    const float accum = a.c_norm * (xn + xr) * (wn + wr);
                    margin = (resid + accum + fmaf(ldexpf(1.f, -23), fabsf(p), fmaf(a.c_sub, xn + wn, a.tiny))) *
                             (1.f + ldexpf(1.f, -20));
                }
                if (fabsf(p) > margin) {
                    if (p > 0.f) {
                        const uint32_t l = col / a.K;
                        if (l != cur_l) {
                            if (cur_bits) atomicOr(&a.codes[row * a.L + cur_l], cur_bits);
                            cur_l = l;
                            cur_bits = 0u;
                        }
                        cur_bits |= 1u << (col % a.K);
                    }
                } else {
                    const unsigned long long slot = atomicAdd(a.rcount, 1ull);
                    a.rlist[slot] = (p > 0.f ? kEntSign : 0ull) | ((unsigned long long)row << 20) | col;
                }
            }
            if (cur_bits) atomicOr(&a.codes[row * a.L + cur_l], cur_bits);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*(volatile uint32_t *)abort_flag) {
        if (threadIdx.x == 0) atomicExch(a.err, 1u);
        // let the copies this CTA issued land before its shared memory goes away
        if (warp == 0 && lane == 0) {
            for (uint32_t kb = (issued > uint32_t(kStages) ? issued - kStages : 0); kb < issued; ++kb)
                mbar_wait(&full[kb % kStages], (kb / kStages) & 1, kWaitNs);
        }
    }
    if (warp == 1) {
        // every MMA has completed before the columns are freed
        if (lane == 0) mbar_wait(mdone, 0, kWaitNs);
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(F::kTmemCols) : "memory");
    }
    __syncthreads();
}

// x -> (bf16(x), bf16(x - bf16(x))) and an upper bound of each row's norm
__global__ void k_split_rows(const float *__restrict__ x, uint64_t ld, uint64_t n, uint32_t d,
                             __nv_bfloat16 *__restrict__ x1, __nv_bfloat16 *__restrict__ x2,
                             float *__restrict__ norm)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t r = gw; r < n; r += nw) {
        double ss = 0.0;
        for (uint32_t t = lane; t < d; t += 32) {
            const float v = x[r * ld + t];
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
            x1[r * d + t] = h;
            x2[r * d + t] = l;
            ss += double(v) * double(v);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        // fp64 sum of d squares, sqrt, rounded up with room to spare
        if (lane == 0) norm[r] = __double2float_ru(sqrt(ss * (1.0 + 1e-12)) * (1.0 + 1e-7));
    }
}

// Single-term quantisers: q = bf16(x) (FORM kFormBf16) or q = e4m3(x / s) with
// s = 2^e, e the smallest with max |x| / s < 448 (FORM kFormFp8; a value whose
// quantised magnitude would be below 2^-6, an E4M3 subnormal, becomes 0). Per
// row: upper bounds of ||x|| and of ||x - s q|| (exact fp64 differences, fp64
// sums of squares, rounded up), and s.
template <int FORM>
__global__ void k_quant_rows(const float *__restrict__ x, uint64_t ld, uint64_t n, uint32_t d,
                             void *__restrict__ q, float *__restrict__ norm, float *__restrict__ res,
                             float *__restrict__ scale)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t r = gw; r < n; r += nw) {
        const float *xr = x + r * ld;
        float s = 1.f;
        if constexpr (FORM == kFormFp8) {
            float mx = 0.f;
            for (uint32_t t = lane; t < d; t += 32) mx = fmaxf(mx, fabsf(xr[t]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (mx > 0.f) {
                int e;
                frexpf(mx / 448.f, &e);      // mx / 448 = f 2^e with f in [0.5, 1): mx / 2^e < 448
                s = ldexpf(1.f, e);
            }
        }
        double ss = 0.0, rr = 0.0;
        for (uint32_t t = lane; t < d; t += 32) {
            const float v = xr[t];
            float back;
            if constexpr (FORM == kFormBf16) {
                const __nv_bfloat16 h = __float2bfloat16_rn(v);
                static_cast<__nv_bfloat16 *>(q)[r * d + t] = h;
                back = __bfloat162float(h);
            } else {
                __nv_fp8_e4m3 h(v / s);                       // round to nearest, saturating
                float hf = float(h);
                if (fabsf(hf) < ldexpf(1.f, -6)) {
                    h = __nv_fp8_e4m3(0.f);
                    hf = 0.f;
                }
                static_cast<__nv_fp8_e4m3 *>(q)[r * d + t] = h;
                back = hf * s;                                // exact: s is a power of two
            }
            const double e = double(v) - double(back);        // exact in fp64
            ss += double(v) * double(v);
            rr += e * e;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ss += __shfl_xor_sync(0xffffffffu, ss, o);
            rr += __shfl_xor_sync(0xffffffffu, rr, o);
        }
        if (lane == 0) {
            // fp64 sums of d squares, sqrt, rounded up with room to spare
            norm[r] = __double2float_ru(sqrt(ss * (1.0 + 1e-12)) * (1.0 + 1e-7));
            res[r] = __double2float_ru(sqrt(rr * (1.0 + 1e-12)) * (1.0 + 1e-7));
            if (scale) scale[r] = s;
        }
    }
}

// Compensated fp32 re-check of listed projections: two-product and two-sum
// per term (one warp per projection), error at most 2^-23 |p| + 2 g(2d)^2 S
// with S = sum |w x|. Decided bits are set; the rest go to the next list.
// xr: the entry's row of x (global or shared memory).
__device__ __forceinline__ void recheck2_entry(const float *xr, const float *__restrict__ Wm, uint32_t d,
                                               uint32_t L, uint32_t K, float g2, float tiny, unsigned long long ent,
                                               uint32_t *__restrict__ codes, unsigned long long *__restrict__ out_list,
                                               unsigned long long *__restrict__ out_count,
                                               unsigned long long *__restrict__ stats)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gr = ent_row(ent);
    const uint32_t gc = ent_col(ent);
    const float *wr = Wm + uint64_t(gc) * d;
    float s = 0.f, c = 0.f, sa = 0.f;
    for (uint32_t t = lane; t < d; t += 32) {
        const float xv = xr[t], wv = wr[t];
        const float h = xv * wv;
        const float l = fmaf(xv, wv, -h);          // exact product error
        const float sn = s + h;                     // two-sum
        const float z = sn - s;
        c += (s - (sn - z)) + (h - z) + l;
        s = sn;
        sa = fmaf(fabsf(xv), fabsf(wv), sa);
    }
    // combine the lanes: lane 0 adds the 32 (s, c) pairs with two-sums
    float ts = 0.f, tc = 0.f;
    for (int k = 0; k < 32; ++k) {
        const float sk = __shfl_sync(0xffffffffu, s, k);
        const float ck = __shfl_sync(0xffffffffu, c, k);
        const float sn = ts + sk;
        const float z = sn - ts;
        tc += (ts - (sn - z)) + (sk - z) + ck;
        ts = sn;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sa = __shfl_sync(0xffffffffu, sa, 0);
    const float p = ts + tc;
    const float margin = fmaf(ldexpf(1.f, -23), fabsf(p), fmaf(g2, sa, tiny));
    if (lane == 0) {
        if (fabsf(p) > margin) {
            if (p > 0.f) atomicOr(&codes[gr * L + gc / K], 1u << (gc % K));
            if ((p > 0.f) != ((ent & kEntSign) != 0)) atomicAdd(&stats[4], 1ull);
        } else {
            out_list[atomicAdd(out_count, 1ull)] = ent;
        }
        atomicAdd(&stats[3], 1ull);
    }
}

__global__ void k_srp_recheck2(const float *__restrict__ X, uint64_t ldx, const float *__restrict__ Wm, uint32_t d,
                               uint32_t L, uint32_t K, float g2, float tiny,
                               const unsigned long long *__restrict__ rlist,
                               const unsigned long long *__restrict__ rcount, uint32_t *__restrict__ codes,
                               unsigned long long *__restrict__ out_list, unsigned long long *__restrict__ out_count,
                               unsigned long long *__restrict__ stats)
{
    const unsigned long long nlist = *rcount;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long e = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
         e < nlist; e += nwarps) {
        const unsigned long long ent = rlist[e];
        recheck2_entry(X + ent_row(ent) * ldx, Wm, d, L, K, g2, tiny, ent, codes, out_list, out_count, stats);
    }
}

// The listed projections grouped by row (a counting sort on the row), so that
// the re-check stages each row of x once in shared memory for all of its
// entries (the tensor-core epilogue lists a row's projections far apart).
__global__ void k_rows_hist(const unsigned long long *__restrict__ rlist, const unsigned long long *__restrict__ rcount,
                            uint32_t *__restrict__ rowcnt)
{
    const unsigned long long n = *rcount;
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (unsigned long long)gridDim.x * blockDim.x)
        atomicAdd(&rowcnt[ent_row(rlist[e])], 1u);
}

__global__ void k_rows_scatter(const unsigned long long *__restrict__ rlist,
                               const unsigned long long *__restrict__ rcount, const uint32_t *__restrict__ rowoff,
                               uint32_t *__restrict__ fill, unsigned long long *__restrict__ sorted)
{
    const unsigned long long n = *rcount;
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long ent = rlist[e];
        const uint64_t r = ent_row(ent);
        sorted[rowoff[r] + atomicAdd(&fill[r], 1u)] = ent;
    }
}

// A CTA per row with listed entries: the row of x in shared memory, a warp per
// entry; the same arithmetic, in the same order, as k_srp_recheck2.
__global__ void k_srp_recheck2_rows(const float *__restrict__ X, uint64_t ldx, const float *__restrict__ Wm,
                                    uint32_t d, uint32_t L, uint32_t K, float g2, float tiny, uint32_t rows,
                                    const unsigned long long *__restrict__ sorted, const uint32_t *__restrict__ rowoff,
                                    uint32_t *__restrict__ codes, unsigned long long *__restrict__ out_list,
                                    unsigned long long *__restrict__ out_count, unsigned long long *__restrict__ stats)
{
    extern __shared__ float xs[];
    const uint32_t warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const uint32_t e0 = rowoff[r], e1 = rowoff[r + 1];
        if (e0 == e1) continue;                       // uniform over the CTA
        const float *xg = X + uint64_t(r) * ldx;
        for (uint32_t t = threadIdx.x; t < d; t += blockDim.x) xs[t] = xg[t];
        __syncthreads();
        for (uint32_t e = e0 + warp; e < e1; e += nw)
            recheck2_entry(xs, Wm, d, L, K, g2, tiny, sorted[e], codes, out_list, out_count, stats);
        __syncthreads();                              // before the next row overwrites xs
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int get_encoder(EncodeTiled *fn)
{
    static EncodeTiled cached = nullptr;
    if (!cached) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        FL_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (!p || q != cudaDriverEntryPointSuccess)
            return set_error(FLINNG_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        cached = reinterpret_cast<EncodeTiled>(p);
    }
    *fn = cached;
    return FLINNG_OK;
}

// 2-D map over rows x d (d contiguous, row stride d elements) of bf16 or
// 8-bit elements; the box is 128 bytes (64 bf16 or 128 e4m3) x 128 rows.
int make_map(CUtensorMap *m, const void *base, uint64_t rows, uint32_t d, bool bytes)
{
    EncodeTiled enc = nullptr;
    FL_TRY(get_encoder(&enc));
    const uint32_t esz = bytes ? 1u : 2u;
    const cuuint64_t dims[2] = {d, rows};
    const cuuint64_t strides[1] = {uint64_t(d) * esz};
    const cuuint32_t box[2] = {128u / esz, uint32_t(kTM)};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, bytes ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                           const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FLINNG_ERR_INVALID_ARG, "tensor map: error %d (d=%u)", int(r), d);
    return FLINNG_OK;
}

inline unsigned warp_grid(uint64_t items)
{
    uint64_t b = (items * 32 + 255) / 256;
    if (b > 152ull * 32) b = 152ull * 32;
    return (unsigned)(b ? b : 1);
}

// bytes of one quantised row
inline size_t qrow_bytes(uint32_t precision, uint32_t d)
{
    return precision == FLINNG_PREC_BF16X2 ? size_t(d) * 4 : precision == FLINNG_PREC_BF16 ? size_t(d) * 2 : size_t(d);
}

int quant_rows(uint32_t precision, const float *x, uint64_t ld, uint64_t n, uint32_t d, void *q, float *norm,
               float *res, float *scale, cudaStream_t st)
{
    if (precision == FLINNG_PREC_BF16X2) {
        __nv_bfloat16 *q1 = static_cast<__nv_bfloat16 *>(q);
        k_split_rows<<<warp_grid(n), 256, 0, st>>>(x, ld, n, d, q1, q1 + n * d, norm);
    } else if (precision == FLINNG_PREC_BF16) {
        k_quant_rows<kFormBf16><<<warp_grid(n), 256, 0, st>>>(x, ld, n, d, q, norm, res, nullptr);
    } else {
        k_quant_rows<kFormFp8><<<warp_grid(n), 256, 0, st>>>(x, ld, n, d, q, norm, res, scale);
    }
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}

template <int FORM>
int launch_tc(const CUtensorMap &mx1, const CUtensorMap &mx2, const CUtensorMap &mw1, const CUtensorMap &mw2,
              const TcArgs &a, uint64_t rows, cudaStream_t st)
{
    const size_t smem = tc_smem_bytes<FORM>();
    FL_TRY(ensure_dyn_smem((const void *)k_srp_tc<FORM>, smem));
    dim3 grid((a.P + kTN - 1) / kTN, (unsigned)((rows + kTM - 1) / kTM));
    k_srp_tc<FORM><<<grid, kTcThreads, smem, st>>>(mx1, mx2, mw1, mw2, a);
    count_launch();
    FL_CUDA(cudaGetLastError());
    return FLINNG_OK;
}

}  // namespace

int srp_tc_prepare_weights(flinng_index *ix)
{
    const uint32_t P = ix->P, d = ix->cfg.dim, prec = ix->cfg.precision;
    if (d % (prec == FLINNG_PREC_FP8 ? 16 : 8) != 0)
        return set_error(FLINNG_ERR_INVALID_ARG, "tensor-core SRP: dim %u is not a multiple of %d", d,
                         prec == FLINNG_PREC_FP8 ? 16 : 8);
    const size_t qb = qrow_bytes(prec, d) * P;
    FL_CUDA(cudaMalloc(&ix->w_split, qb));
    FL_CUDA(cudaMalloc(&ix->w_norm, size_t(P) * sizeof(float)));
    ix->device_bytes += qb + size_t(P) * 4;
    if (prec != FLINNG_PREC_BF16X2) {
        FL_CUDA(cudaMalloc(&ix->w_aux, size_t(P) * 2 * sizeof(float)));
        ix->device_bytes += size_t(P) * 8;
    }
    return quant_rows(prec, ix->srp_w, d, P, d, ix->w_split, ix->w_norm, ix->w_aux, ix->w_aux ? ix->w_aux + P : nullptr,
                      ix->stream);
}

size_t srp_tc_workspace_bytes(const flinng_index *ix, uint64_t n)
{
    const uint64_t rows = n < kTcChunkRows ? n : kTcChunkRows;
    return carve_bytes<char>(rows * qrow_bytes(ix->cfg.precision, ix->cfg.dim)) + 3 * carve_bytes<float>(rows) +
           carve_bytes<unsigned long long>(8) + 2 * carve_bytes<unsigned long long>(rows * ix->P + 1) +
           3 * carve_bytes<uint32_t>(rows + 1) + carve_bytes<char>(scan_workspace_bytes(rows + 1)) + 4096;
}

// Codes of n rows of x (stride ld) on the tensor cores; same contract as srp_hash.
int srp_hash_tc(flinng_index *ix, const float *x, uint64_t ld, uint64_t n, uint32_t *buckets, float *proj,
                void *ws)
{
    // a wait that timed out in an earlier call (the flag is sticky on the device)
    if (ix->h_flag[3]) return set_error(FLINNG_ERR_TIMEOUT, "tensor-core SRP: a pipeline wait timed out");
    const cudaStream_t st = ix->stream;
    const uint32_t L = ix->cfg.L, K = ix->cfg.K, d = ix->cfg.dim, P = ix->P, prec = ix->cfg.precision;
    const bool bytes = prec == FLINNG_PREC_FP8;
    const uint64_t chunk = kTcChunkRows;
    const uint64_t cap = n < chunk ? n : chunk;     // rows the workspace was sized for
    Carver c(ws, ~size_t(0));
    char *xq = c.take<char>(cap * qrow_bytes(prec, d));
    float *xn = c.take<float>(cap);
    float *xr = c.take<float>(cap);
    float *xsc = c.take<float>(cap);
    unsigned long long *cnt = c.take<unsigned long long>(8);
    unsigned long long *list1 = c.take<unsigned long long>(cap * P + 1);
    unsigned long long *list2 = c.take<unsigned long long>(cap * P + 1);
    uint32_t *rowcnt = c.take<uint32_t>(cap + 1);
    uint32_t *rowoff = c.take<uint32_t>(cap + 1);
    uint32_t *fill = c.take<uint32_t>(cap + 1);
    void *scan_ws = c.take<char>(scan_workspace_bytes(cap + 1));
    // stage 2 by row when a row of x fits in shared memory
    const bool rows_staged = size_t(d) * sizeof(float) <= kRecheckRowBytes;
    if (rows_staged) FL_TRY(ensure_dyn_smem((const void *)k_srp_recheck2_rows, size_t(d) * sizeof(float)));
    FL_CUDA(cudaMemsetAsync(ix->stats, 0, kStats * sizeof(unsigned long long), st));
    if (n == 0) return FLINNG_OK;
    FL_CUDA(cudaMemsetAsync(buckets, 0, n * L * sizeof(uint32_t), st));
    const char *wq = static_cast<const char *>(ix->w_split);
    CUtensorMap mw1, mw2;
    FL_TRY(make_map(&mw1, wq, P, d, bytes));
    if (prec == FLINNG_PREC_BF16X2) FL_TRY(make_map(&mw2, wq + size_t(P) * d * 2, P, d, false));
    else mw2 = mw1;
    // margin factors (see the header comment), in double then rounded up
    const double u = std::ldexp(1.0, -24), up = std::ldexp(1.0, -22);
    auto g = [](double m, double uu) { return m * uu / (1.0 - m * uu); };
    const double q = (1 + std::ldexp(1.0, -8)) * (1 + std::ldexp(1.0, -8));
    const double kb = prec == FLINNG_PREC_FP8 ? 128.0 : double(kTK);     // products per k-block
    const double m_blocks = std::ceil(double(d) / kb);
    double f;
    if (prec == FLINNG_PREC_BF16X2)
        f = (g(kTK, up) + std::ldexp(1.0, -7) * g(2 * kTK, up)) * q +
            g(2 * m_blocks, u) * (1 + g(kTK, up)) * (1 + std::ldexp(1.0, -7)) * q + 3.1 * std::ldexp(1.0, -16);
    else
        f = g(kb, up) + g(m_blocks, u) * (1 + g(kb, up));    // times (||x|| + ||e_x||)(||w|| + ||e_w||)
    const float c_norm = std::nextafter(float(f * 1.0001), INFINITY);
    const float c_sub = std::nextafter(float(std::sqrt(double(d)) * std::ldexp(1.0, -125)), INFINITY);
    const float tiny = std::nextafter(float(8.0 * d * std::ldexp(1.0, -126)), INFINITY);
    const double g2d = 2.0 * d * std::ldexp(1.0, -24) / (1.0 - 2.0 * d * std::ldexp(1.0, -24));
    const float g2 = std::nextafter(float(2.0 * g2d * g2d + std::ldexp(1.0, -40)), INFINITY);
    for (uint64_t r0 = 0; r0 < n; r0 += chunk) {
        const uint64_t rows = (n - r0) < chunk ? (n - r0) : chunk;
        FL_TRY(quant_rows(prec, x + r0 * ld, ld, rows, d, xq, xn, xr, xsc, st));
        CUtensorMap mx1, mx2;
        FL_TRY(make_map(&mx1, xq, rows, d, bytes));
        if (prec == FLINNG_PREC_BF16X2) FL_TRY(make_map(&mx2, xq + rows * d * 2, rows, d, false));
        else mx2 = mx1;
        FL_CUDA(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), st));
        TcArgs a{};
        a.n = rows;
        a.P = P;
        a.d = d;
        a.L = L;
        a.K = K;
        a.xnorm = xn;
        a.wnorm = ix->w_norm;
        a.xres = xr;
        a.wres = ix->w_aux;
        a.xscale = xsc;
        a.wscale = ix->w_aux ? ix->w_aux + P : nullptr;
        a.c_norm = c_norm;
        a.c_sub = c_sub;
        a.tiny = tiny;
        a.codes = buckets + r0 * L;
        a.proj = proj ? proj + r0 * P : nullptr;
        a.rlist = list1;
        a.rcount = cnt;
        a.err = ix->tc_err;
        a.wait_ns = ix->tc_wait_ns ? ix->tc_wait_ns - 1 : kWaitNs;
        if (prec == FLINNG_PREC_BF16X2) FL_TRY(launch_tc<kFormBf16x2>(mx1, mx2, mw1, mw2, a, rows, st));
        else if (prec == FLINNG_PREC_BF16) FL_TRY(launch_tc<kFormBf16>(mx1, mx2, mw1, mw2, a, rows, st));
        else FL_TRY(launch_tc<kFormFp8>(mx1, mx2, mw1, mw2, a, rows, st));
        // stage 2: compensated fp32; stage 3: fp64 / exact
        if (rows_staged) {
            // the list grouped by row into list2; stage 2 lists what stays undecided in list1
            FL_CUDA(cudaMemsetAsync(rowcnt, 0, (rows + 1) * sizeof(uint32_t), st));
            FL_CUDA(cudaMemsetAsync(fill, 0, (rows + 1) * sizeof(uint32_t), st));
            k_rows_hist<<<152 * 8, 256, 0, st>>>(list1, cnt, rowcnt);
            count_launch();
            FL_CUDA(cudaGetLastError());
            FL_TRY(scan_exclusive(rowcnt, rowoff, rows, scan_ws, st));
            k_rows_scatter<<<152 * 8, 256, 0, st>>>(list1, cnt, rowoff, fill, list2);
            count_launch();
            FL_CUDA(cudaGetLastError());
            const unsigned grid = unsigned(rows < 152ull * 8 ? rows : 152ull * 8);
            k_srp_recheck2_rows<<<grid, 256, size_t(d) * sizeof(float), st>>>(
                x + r0 * ld, ld, ix->srp_w, d, L, K, g2, tiny, uint32_t(rows), list2, rowoff, buckets + r0 * L, list1,
                cnt + 1, ix->stats);
            count_launch();
            FL_CUDA(cudaGetLastError());
            FL_TRY(srp_recheck_list(ix, x + r0 * ld, ld, list1, cnt + 1, buckets + r0 * L));
        } else {
            k_srp_recheck2<<<152 * 4, 256, 0, st>>>(x + r0 * ld, ld, ix->srp_w, d, L, K, g2, tiny, list1, cnt,
                                                   buckets + r0 * L, list2, cnt + 1, ix->stats);
            count_launch();
            FL_CUDA(cudaGetLastError());
            FL_TRY(srp_recheck_list(ix, x + r0 * ld, ld, list2, cnt + 1, buckets + r0 * L));
        }
        FL_TRY(add_counter(ix->stats, cnt, st));            // undecided after the tensor-core pass
    }
    // no synchronisation here (servers hash on their own streams): the flag
    // lands in pinned memory and the next call on this index reports it
    FL_CUDA(cudaMemcpyAsync(ix->h_flag + 3, ix->tc_err, 4, cudaMemcpyDeviceToHost, st));
    return FLINNG_OK;
}

}  // namespace flinng
