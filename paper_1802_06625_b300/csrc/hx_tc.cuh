// HX_b on tcgen05 tensor cores (placeholder until the tensor-core kernel lands).
#pragma once
#include "hx_cuda.cuh"
namespace prune {
__host__ inline bool hx_tc_supported(int N) { (void)N; return false; }
__host__ inline size_t hx_tc_b_elems(int N) { return static_cast<size_t>(N) * N * 8; }
__host__ inline cudaError_t hx_tc_prepare_b(const float2 *, int, uint16_t *, cudaStream_t) { return cudaErrorNotSupported; }
__host__ inline cudaError_t launch_hx_tc(const HxParams &, const uint16_t *, int, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace prune
