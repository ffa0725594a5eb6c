// pt_learn_dev.cuh -- device helpers of the learned proposal shared by the sampling kernels (pt_learn.cu) and
// the fused network/sampling kernels on the tensor cores (pt_gemm.cu): one definition of the arithmetic,
// so that both paths draw bit-identical proposals.
#pragma once
#include <cstdint>
#include "pt_common.cuh"

namespace ptgb {

constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr float kLog2PiHalf = 0.91893853320467274178f;  // log(2 pi) / 2
constexpr float kRhoMax = 0.98f;
constexpr float kUScale = 0.25f;                          // input scale of logit(v)

// uniform in (0, 1) from the top 24 bits of a Philox word (FP32 draws)
__device__ __forceinline__ float u01f(uint32_t w) { return ((float)(w >> 8) + 0.5f) * (1.0f / 16777216.0f); }
__device__ __forceinline__ float softplusf(float x) { return x > 20.f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float wrap2pi(float x) { return x - kTwoPiF * floorf(x / kTwoPiF); }

// Input features of mode k: (logit(v_k)/4 clipped to [-4, 4], cos phi~_k, sin phi~_k).
__device__ __forceinline__ float feature_u(float u, int k, int N) {
    return (k <= N - 2) ? fminf(fmaxf(u * kUScale, -4.f), 4.f) : 0.f;
}
__device__ __forceinline__ void feature_triplet(float u, float ph, int k, int N, float f[3]) {
    f[0] = feature_u(u, k, N);
    float sn, cs;
    sincosf(ph, &sn, &cs);
    f[1] = cs;
    f[2] = sn;
}

// The state-independent part of a mode's draw, from the mode's Philox word w: the Box-Muller normal eps and
// the wrapped-Cauchy quantile factor t1 = tan(pi (U - 1/2)).
struct ModeNoise {
    float eps, t1;
};
__device__ __forceinline__ ModeNoise mode_noise(u32x4 w) {
    ModeNoise n;
    n.eps = sqrtf(-2.f * logf(u01f(w.x))) * cosf(kTwoPiF * u01f(w.y));
    n.t1 = tanf(3.14159265358979323846f * (u01f(w.z) - 0.5f));
    return n;
}
// u = mu + sigma eps (log sigma clipped to [-7, 3]) for k <= N-2, else 0
__device__ __forceinline__ float sample_u(float mu, float log_sigma, float eps, int k, int N) {
    if (k > N - 2) return 0.f;
    const float ls = fminf(fmaxf(log_sigma, -7.f), 3.f);
    return mu + expf(ls) * eps;
}
// phi~ by the wrapped-Cauchy inverse CDF around m with rho = 0.98 sigmoid(rho_raw) for k >= 2, else 0
__device__ __forceinline__ float sample_phi(float m, float rho_raw, float t1, int k) {
    if (k < 2) return 0.f;
    const float rho = kRhoMax / (1.f + expf(-rho_raw));
    return wrap2pi(m + 2.f * atanf((1.f - rho) / (1.f + rho) * t1));
}
// Draw of mode k from its conditionals, network outputs o = (mu, log sigma, m, rho_raw) and the mode's Philox
// word w: u = mu + sigma eps (Box-Muller, k <= N-2), phi~ by the wrapped-Cauchy inverse CDF (k >= 2).
__device__ __forceinline__ void sample_mode(const float o[4], u32x4 w, int k, int N, float *u, float *ph) {
    const ModeNoise n = mode_noise(w);
    *u = sample_u(o[0], o[1], n.eps, k, N);
    *ph = sample_phi(o[2], o[3], n.t1, k);
}

}  // namespace ptgb
