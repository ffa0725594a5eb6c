// pt_probe.cu -- FP32 FMA-pipe throughput probe.  The Metropolis sweep is bound by FP32 arithmetic, not by
// memory, so its roofline needs the FP32 peak of the GPU it runs on, measured rather than taken from unit
// counts and a nominal clock: this kernel keeps every FP32 lane busy with independent fused multiply-add
// chains and the caller times it with CUDA events.
#include <cstdint>

#include "../../include/pt.h"
#include "pt_common.cuh"

namespace ptgb {
void set_global_error(const char *msg);
}

namespace {

constexpr int kChains = 8;  // independent accumulators per thread: enough to cover the FMA latency

// Packed variant: kChains FFMA2 per iteration (2 fused multiply-adds each); scalar variant: 2 kChains FFMA.
// Both do 4 kChains flops per thread and iteration.  The multiplier and addend keep the values finite; the
// result is stored only when it equals a value it cannot take, so nothing is optimised away and nothing is
// written in practice.
template <bool PACKED>
__global__ void __launch_bounds__(1024) fma_probe_kernel(int iters, float *sink) {
    const float x0 = 1.0f + 1e-3f * (float)(threadIdx.x & 31);
    const float2 m = make_float2(0.99999f, 1.00001f), c = make_float2(1e-6f, -1e-6f);
    float2 a[kChains];
#pragma unroll
    for (int r = 0; r < kChains; ++r) a[r] = make_float2(x0 + r, x0 - r);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < kChains; ++r) {
            if (PACKED) {
                a[r] = __ffma2_rn(a[r], m, c);
            } else {
                a[r].x = __fmaf_rn(a[r].x, m.x, c.x);
                a[r].y = __fmaf_rn(a[r].y, m.y, c.y);
            }
        }
    }
    float t = 0.f;
#pragma unroll
    for (int r = 0; r < kChains; ++r) t += a[r].x + a[r].y;
    if (t == -1.0f) sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace

extern "C" int pt_fma_probe(int packed, int blocks, int threads, int iters, float *sink, void *stream) {
    if (blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1 || !sink) {
        ptgb::set_global_error("pt_fma_probe: need blocks >= 1, threads a multiple of 32 in [32, 1024], iters >= 1, sink");
        return PT_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (packed) fma_probe_kernel<true><<<blocks, threads, 0, s>>>(iters, sink);
    else fma_probe_kernel<false><<<blocks, threads, 0, s>>>(iters, sink);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ptgb::set_global_error(cudaGetErrorString(e));
        return PT_ECUDA;
    }
    return PT_OK;
}
