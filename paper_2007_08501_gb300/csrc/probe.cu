// FP32 FMA throughput probe: the denominator of the ALU rooflines (the fine
// pass's face tests, the nearest-neighbour distances) is measured on the
// device rather than derived from unit counts and a nominal clock.
//
// Every thread runs 8 independent chains of fused multiply-adds (enough
// independent work to cover the FMA latency at full occupancy); the chains
// are folded into one value per thread at the end so none is dead code.
#include <cuda_runtime.h>

#include "meshrast.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fma_probe(float *out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = __fmaf_rn(x[j], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" MESHRAST_API int meshrast_fma_probe(float *out, int64_t blocks, int32_t iters, void *stream) {
    if (!out || blocks < 1 || blocks > (1 << 20) || iters < 1) return MESHRAST_ERR_INVALID_ARG;
    // a = 1 - 2^-20, b = 2^-20 keep every chain finite for any iteration count
    k_fma_probe<<<(unsigned)blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(out, iters, 0.99999905f,
                                                                                       9.5367432e-7f);
    return cudaGetLastError() == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}
