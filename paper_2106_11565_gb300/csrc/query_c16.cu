// The query kernels with 16-bit per-cell counts (indices with L > 255); the
// 8-bit instantiation is in query.cu. Separate translation units compile in
// parallel.
#include "query_impl.cuh"

namespace flinng {

const void *plain_kernel_c2(int NT, uint32_t rw) { return plain_kernel_t<2>(NT, rw); }
const void *fused_kernel_c2(int NT, uint32_t rw, bool srp) { return fused_kernel_t<2>(NT, rw, srp); }
const void *counts_kernel_c2() { return (const void *)k_counts<2>; }

}  // namespace flinng
