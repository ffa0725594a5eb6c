// pt_learn.cu -- kernels of the learned global-move proposal: gauge-fixed features, the proposal
// density and its gradient with respect to the network outputs, bias gradients, Adam, block-wise
// sampling, assembly of proposed configurations, FP64 energies and the exact Metropolis-Hastings step.
// The dense layers run on the tensor cores (pt_gemm.cu).  See pt_learn.h for the density.
#include <algorithm>
#include <cstdint>
#include <cuda_bf16.h>
#include "pt_common.cuh"
#include "pt_learn.h"
#include "pt_learn_dev.cuh"

namespace ptgb {

namespace {

__device__ __forceinline__ double warp_sumd(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// gauge-fixed features of configurations: one warp per row, N <= 64 (two modes per lane)
__global__ void features_kernel(FeatParams p) {
    const int s = blockIdx.y, row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (row >= p.rows_per_sample) return;
    const int N = p.N;
    const int64_t grow = (int64_t)s * p.rows_per_sample + row;
    double re[2] = {0, 0}, im[2] = {0, 0};
    if (p.slot) {
        const int slot = p.slot[grow];
        const SampleDev sd = p.samples[s];
        const int64_t base = sd.a_off + (int64_t)(slot - sd.chain0) * N;
        for (int q = 0; q < 2; ++q) {
            const int k = lane + 32 * q;
            if (k < N) {
                if (p.dbl) { const double2 v = reinterpret_cast<const double2 *>(p.a)[base + k]; re[q] = v.x; im[q] = v.y; }
                else { const float2 v = reinterpret_cast<const float2 *>(p.a)[base + k]; re[q] = v.x; im[q] = v.y; }
            }
        }
    } else {
        for (int q = 0; q < 2; ++q) {
            const int k = lane + 32 * q;
            if (k < N) {
                if (p.dbl) { const double2 v = reinterpret_cast<const double2 *>(p.a)[grow * N + k]; re[q] = v.x; im[q] = v.y; }
                else { const float2 v = reinterpret_cast<const float2 *>(p.a)[grow * N + k]; re[q] = v.x; im[q] = v.y; }
            }
        }
    }
    // intensity fractions s_k = |a_k|^4 / sum |a|^4 (exactly on the simplex)
    double sk[2], tot = 0.0;
    for (int q = 0; q < 2; ++q) {
        const double u = re[q] * re[q] + im[q] * im[q];
        sk[q] = (lane + 32 * q < N) ? u * u : 0.0;
        tot += sk[q];
    }
    tot = warp_sumd(tot);
    for (int q = 0; q < 2; ++q) sk[q] /= tot;
    // suffix sums R_k = sum_{i >= k} s_i and R_{k+1}, summed from the tail (no cancellation: a proposal's
    // intensities can fall off geometrically, and 1 - prefix would lose the tail entirely)
    double Rin[2], Rex[2];
    {
        double x0 = sk[0], x1 = sk[1];
        for (int o = 1; o < 32; o <<= 1) {
            const double y0 = __shfl_down_sync(0xffffffffu, x0, o), y1 = __shfl_down_sync(0xffffffffu, x1, o);
            if (lane + o < 32) { x0 += y0; x1 += y1; }
        }
        const double top = __shfl_sync(0xffffffffu, x1, 0);  // sum over modes 32..63
        const double n0 = __shfl_down_sync(0xffffffffu, x0, 1), n1 = __shfl_down_sync(0xffffffffu, x1, 1);
        Rin[0] = x0 + top;
        Rin[1] = x1;
        Rex[0] = (lane < 31 ? n0 : 0.0) + top;
        Rex[1] = lane < 31 ? n1 : 0.0;
    }
    // phases, gauge fixed.  The gauge phases phi_0 and phi_1 enter phi~_k k-fold and are taken in FP64; the
    // others need only the FP32 accuracy the stored phi~_k has.  log R_{k+1} is the next mode's log R_k.
    double phk[2], lr[2], ls[2];
    for (int q = 0; q < 2; ++q) {
        const int k = lane + 32 * q;
        phk[q] = k < 2 ? atan2(im[q], re[q]) : (double)atan2f((float)im[q], (float)re[q]);
        lr[q] = log(fmax(Rin[q], 1e-300));
        ls[q] = log(sk[q]);
    }
    const double ph0 = __shfl_sync(0xffffffffu, phk[0], 0);
    const double ph1 = __shfl_sync(0xffffffffu, phk[0], 1);
    double lr1[2];
    {
        const double n0 = __shfl_down_sync(0xffffffffu, lr[0], 1), n1 = __shfl_down_sync(0xffffffffu, lr[1], 1);
        const double b1 = __shfl_sync(0xffffffffu, lr[1], 0);  // log R_32
        lr1[0] = lane < 31 ? n0 : b1;
        lr1[1] = lane < 31 ? n1 : 0.0;  // k = 63 has no u
    }
    double extra = 0.0;
    const int64_t rrow = (int64_t)s * p.raw_stride + p.raw_off + row;
    for (int q = 0; q < 2; ++q) {
        const int k = lane + 32 * q;
        if (k >= N) continue;
        const float u = (k <= N - 2) ? (float)(ls[q] - (k + 1 < N ? lr1[q] : log(fmax(Rex[q], 1e-300)))) : 0.f;
        float ph = 0.f;
        if (k >= 2) ph = wrap2pi((float)(phk[q] - ph0 - (double)k * (ph1 - ph0)));
        if (k <= N - 2) extra -= lr[q];
        extra += 0.5 * ls[q];
        p.raw.u[rrow * N + k] = u;
        p.raw.phi[rrow * N + k] = ph;
        if (p.X) {
            float f[3];
            feature_triplet(u, ph, k, N, f);
            for (int c = 0; c < 3; ++c) {
                const int fi = 3 * k + c;
                const __nv_bfloat16 b = __float2bfloat16_rn(f[c]);
                p.X[((int64_t)s * p.x_stride + row) * p.Din + fi] = b;
                if (p.XT) p.XT[((int64_t)s * p.Din + fi) * p.ldxt + row] = b;
            }
        }
    }
    extra = warp_sumd(extra);
    if (lane == 0) {
        p.raw.extra[rrow] = (float)extra;
        if (p.cond_in) p.raw.cond[rrow] = p.cond_in[grow];
    }
}

cudaError_t launch_features(const FeatParams &p, int S, cudaStream_t s) {
    if (p.rows_per_sample <= 0) return cudaSuccess;
    dim3 grid(p.rows_per_sample, S);  // one row (warp) per block: the FP64 work spread over all SMs
    features_kernel<<<grid, 32, 0, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Position of element (n, k) of an N x K matrix in the sliced canonical K-major layout: four slices of
// NS = N/4 rows, each [K/8][NS][8] and contiguous.
__device__ __forceinline__ size_t sliced_canonical(size_t n, size_t k, size_t N, size_t K) {
    const size_t NS = N / 4;
    return ((n / NS) * (K / 8) + k / 8) * NS * 8 + (n % NS) * 8 + k % 8;
}

__global__ void cast_kernel(CastParams p) {
    const LearnShape &sh = p.sh;
    const int s = blockIdx.y;
    const float *P = p.P + (size_t)s * sh.psize;
    const size_t n1 = (size_t)sh.H * sh.Din, n2 = (size_t)sh.H * sh.H, n3 = (size_t)sh.Dout * sh.H;
    for (size_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2 + n3; i += gridDim.x * blockDim.x) {
        if (i < n1) {
            const __nv_bfloat16 w = __float2bfloat16_rn(P[sh.oW1 + i] * p.M1[i]);
            p.W1[s * n1 + i] = w;
            p.W1c[s * n1 + sliced_canonical(i / sh.Din, i % sh.Din, sh.H, sh.Din)] = w;
        } else if (i < n1 + n2) {
            const size_t j = i - n1;
            const __nv_bfloat16 w = __float2bfloat16_rn(P[sh.oW2 + j] * p.M2[j]);
            p.W2[s * n2 + j] = w;
            const size_t h2 = j / sh.H, h1 = j % sh.H;
            p.W2T[s * n2 + h1 * sh.H + h2] = w;
            p.W2c[s * n2 + sliced_canonical(h2, h1, sh.H, sh.H)] = w;
        } else {
            const size_t j = i - n1 - n2;
            const __nv_bfloat16 w = __float2bfloat16_rn(P[sh.oW3 + j] * p.M3[j]);
            p.W3[s * n3 + j] = w;
            const size_t o = j / sh.H, h = j % sh.H;
            p.W3T[s * n3 + h * sh.Dout + o] = w;
            p.W3c[s * n3 + sliced_canonical(o, h, sh.Dout, sh.H)] = w;
        }
    }
}

cudaError_t launch_cast(const CastParams &p, cudaStream_t s) {
    dim3 grid(128, p.sh.S);
    cast_kernel<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// log q per row and the gradient of mean(-log q) with respect to the outputs (mu, log sigma, m, rho_raw)
__global__ void density_kernel(DensityParams p) {
    const int s = blockIdx.y, row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (row >= p.rows_per_sample) return;
    const int N = p.N;
    const int64_t grow = (int64_t)s * p.rows_per_sample + row;
    const int64_t orow = (int64_t)s * p.o_stride + row;
    const float *o = p.O + orow * p.Dout;
    double lq = 0.0;
    for (int k = lane; k < N; k += 32) {
        float g[4] = {0.f, 0.f, 0.f, 0.f};
        if (k <= N - 2) {
            const float u = p.raw.u[grow * N + k];
            const float mu = o[4 * k], ls_raw = o[4 * k + 1];
            const float ls = fminf(fmaxf(ls_raw, -7.f), 3.f);
            const float sig = expf(ls);
            const float z = (u - mu) / sig;
            lq += (double)(-0.5f * z * z - ls - kLog2PiHalf + softplusf(-u) + softplusf(u));
            g[0] = z / sig;
            g[1] = (ls_raw > -7.f && ls_raw < 3.f) ? (z * z - 1.f) : 0.f;
        }
        if (k >= 2) {
            const float ph = p.raw.phi[grow * N + k];
            const float m = o[4 * k + 2], rr = o[4 * k + 3];
            const float sg = 1.f / (1.f + expf(-rr));
            const float rho = kRhoMax * sg;
            float sd, cd;
            sincosf(ph - m, &sd, &cd);
            const float D = 1.f + rho * rho - 2.f * rho * cd;
            lq += (double)(log1pf(-rho * rho) - 2.f * kLog2PiHalf - logf(D));
            g[2] = 2.f * rho * sd / D;
            const float dl_drho = -2.f * rho / (1.f - rho * rho) - (2.f * rho - 2.f * cd) / D;
            g[3] = dl_drho * kRhoMax * sg * (1.f - sg);
        }
        if (p.dO || p.dOb) {
            for (int c = 0; c < 4; ++c) {
                const float d = -g[c] * p.inv_rows;  // d mean(-log q) / d output
                const int col = 4 * k + c;
                if (p.dO) p.dO[orow * p.Dout + col] = d;
                const __nv_bfloat16 b = __float2bfloat16_rn(d);
                if (p.dOb) p.dOb[orow * p.Dout + col] = b;
                if (p.dOT) p.dOT[((int64_t)s * p.Dout + col) * p.lddt + row] = b;
            }
        }
    }
    lq = warp_sumd(lq);
    if (lane == 0) p.logq[grow] = lq;
}

cudaError_t launch_density(const DensityParams &p, int S, cudaStream_t s) {
    if (p.rows_per_sample <= 0) return cudaSuccess;
    dim3 grid(p.rows_per_sample, S);  // one row (warp) per block
    density_kernel<<<grid, 32, 0, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
__global__ void colsum_kernel(const float *dZ, int rows, int cols, float *db, float *dC, const int *cond,
                              int64_t strideZ, int64_t strideGrad, int64_t strideCond) {
    const int s = blockIdx.y, col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= cols) return;
    const float *z = dZ + s * strideZ;
    float acc = 0.f;
    for (int r = 0; r < rows; ++r) {
        const float v = z[(int64_t)r * cols + col];
        acc += v;
        if (dC) dC[s * strideGrad + (int64_t)cond[s * strideCond + r] * cols + col] += v;
    }
    db[s * strideGrad + col] = acc;
}

cudaError_t launch_colsum(const float *dZ, int rows, int cols, float *db, float *dC, const int *cond, int S,
                          int64_t strideZ, int64_t strideGrad, cudaStream_t s) {
    dim3 grid((cols + 127) / 128, S);
    colsum_kernel<<<grid, 128, 0, s>>>(dZ, rows, cols, db, dC, cond, strideZ, strideGrad, rows);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
__global__ void adam_kernel(float *P, const float *G, float *m, float *v, size_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float g = G[i];
        const float mi = b1 * m[i] + (1.f - b1) * g, vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

cudaError_t launch_adam(float *P, const float *G, float *m, float *v, size_t n, float lr, float b1, float b2,
                        float eps, int t, cudaStream_t s) {
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    adam_kernel<<<512, 256, 0, s>>>(P, G, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
__global__ void gather_kernel(GatherParams p) {
    const int s = blockIdx.y, row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (row >= p.rows) return;
    const int N = p.N;
    const u32x4 w = draw(p.seed, (uint32_t)s, p.step, (uint32_t)row, kTagBatch);
    const int idx = (int)(((uint64_t)w.x * (uint64_t)p.ndata) >> 32);
    const int64_t src = (int64_t)s * p.stride + idx, dst = (int64_t)s * p.rows + row;
    const int64_t xrow = (int64_t)s * p.x_stride + row;
    for (int k = lane; k < N; k += 32) {
        const float u = p.du[src * N + k], ph = p.dphi[src * N + k];
        p.raw.u[dst * N + k] = u;
        p.raw.phi[dst * N + k] = ph;
        float f[3];
        feature_triplet(u, ph, k, N, f);
        for (int c = 0; c < 3; ++c) {
            const int fi = 3 * k + c;
            const __nv_bfloat16 b = __float2bfloat16_rn(f[c]);
            p.X[xrow * p.Din + fi] = b;
            p.XT[((int64_t)s * p.Din + fi) * p.ldxt + row] = b;
        }
    }
    if (lane == 0) {
        p.raw.extra[dst] = p.dextra[src];
        p.raw.cond[dst] = p.dcond[src];
    }
}

cudaError_t launch_gather(const GatherParams &p, int S, cudaStream_t s) {
    dim3 grid((p.rows + 3) / 4, S);
    gather_kernel<<<grid, 128, 0, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// sampling pass for mode block b: u = mu + sigma * eps (Box-Muller), phi~ by the wrapped-Cauchy inverse CDF
__global__ void sample_block_kernel(SampleParams p) {
    const int s = blockIdx.y, row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (row >= p.rows_per_sample) return;
    const int N = p.N, per = N / kLearnBlocks;
    const int64_t grow = (int64_t)s * p.rows_per_sample + row;
    const uint32_t id = p.row_id[grow];
    if (p.block < first_block(p.seed, id, (uint32_t)p.ctl->global_rounds, N, p.lo, p.hi)) return;
    for (int t = lane; t < per; t += 32) {
        const int k = p.block * per + t;
        const float *o = p.O + ((int64_t)s * p.o_stride + row) * p.Dout + 4 * k;
        const u32x4 w = draw(p.seed, id, (uint32_t)p.ctl->global_rounds, (uint32_t)k, kTagGlobal);
        const float ov[4] = {o[0], o[1], o[2], o[3]};
        float u, ph;
        sample_mode(ov, w, k, N, &u, &ph);
        p.u[grow * N + k] = u;
        p.phi[grow * N + k] = ph;
        float f[3];
        feature_triplet(u, ph, k, N, f);
        for (int c = 0; c < 3; ++c) p.X[((int64_t)s * p.x_stride + row) * p.Din + 3 * k + c] = __float2bfloat16_rn(f[c]);
    }
}

cudaError_t launch_sample_block(const SampleParams &p, int S, cudaStream_t s) {
    dim3 grid((p.rows_per_sample + 3) / 4, S);
    sample_block_kernel<<<grid, 128, 0, s>>>(p);
    return cudaGetLastError();
}

// amplitudes: v_k = sigmoid(u_k), s_k = v_k r_k (stick breaking), |a_k| = (n s_k)^(1/4),
// phi_k = phi~_k + alpha + k theta.  With k0 = 8-mode-block start of the first resampled block:
// k0 = 0: r_0 = 1, n = N, (alpha, theta) fresh and uniform;
// k0 > 0: modes < k0 copied, r_{k0} = the current tail mass, n = the current sum |a|^4, gauge of the
// current configuration (alpha = phi_0, theta = phi_1 - phi_0), so the proposal moves only the tail.
// One warp per row, two modes per lane; r_k is an exclusive product scan over the lanes.
__global__ void assemble_kernel(AssembleParams p) {
    const int s = blockIdx.y, row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (row >= p.rows_per_sample) return;
    const int N = p.N;
    const int64_t grow = (int64_t)s * p.rows_per_sample + row;
    const uint32_t round = (uint32_t)p.ctl->global_rounds;
    const int k0 = first_block(p.seed, p.row_id[grow], round, N, p.lo, p.hi) * (N / kLearnBlocks);
    const SampleDev sd = p.samples[s];
    const int64_t base = sd.a_off + (int64_t)(p.slot[grow] - sd.chain0) * N;
    double2 cur[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    if (k0 > 0)
        for (int q = 0; q < 2; ++q) {
            const int k = lane + 32 * q;
            if (k < N) {
                if (p.dbl) cur[q] = reinterpret_cast<const double2 *>(p.a_cur)[base + k];
                else { const float2 v = reinterpret_cast<const float2 *>(p.a_cur)[base + k]; cur[q] = make_double2(v.x, v.y); }
            }
        }
    double alpha, theta, r0 = 1.0, n = (double)N;
    if (k0 == 0) {
        const u32x4 w = draw(p.seed, p.row_id[grow], round, (uint32_t)N, kTagGlobal);
        alpha = kTwoPi * u01(w.x);
        theta = kTwoPi * u01(w.y);
    } else {
        double tot = 0.0, tail = 0.0;
        for (int q = 0; q < 2; ++q) {
            const int k = lane + 32 * q;
            const double u = cur[q].x * cur[q].x + cur[q].y * cur[q].y;
            tot += u * u;
            if (k >= k0) tail += u * u;
        }
        tot = warp_sumd(tot);
        tail = warp_sumd(tail);
        n = tot;
        r0 = tail / tot;
        const double a0 = __shfl_sync(0xffffffffu, atan2(cur[0].y, cur[0].x), 0);
        const double a1 = __shfl_sync(0xffffffffu, atan2(cur[0].y, cur[0].x), 1);
        alpha = a0;
        theta = a1 - a0;
    }
    // per mode k >= k0: v_k and 1 - v_k from one exponential in (0, 1] (v + (1-v) = 1 to FP64 rounding):
    // v = 1/(1+t), 1-v = t/(1+t) with t = e^{-u} (u >= 0); v = w/(1+w), 1-v = 1/(1+w) with w = e^{u} (u < 0)
    double v[2], f[2];
    for (int q = 0; q < 2; ++q) {
        const int k = lane + 32 * q;
        v[q] = 0.0;
        f[q] = 1.0;
        if (k >= k0 && k <= N - 2) {
            const float u = p.u[grow * N + k];
            const double e = (double)expf(-fabsf(u)), d = 1.0 / (1.0 + e);
            v[q] = u >= 0.f ? d : e * d;
            f[q] = u >= 0.f ? e * d : d;
        } else if (k == N - 1) {
            v[q] = 1.0;  // the last mode takes the remaining mass
        }
    }
    // exclusive product scan of f over modes 0..63 (f = 1 below k0): r_k = r_{k0} prod_{k0 <= i < k} f_i
    double x0 = f[0], x1 = f[1];
    for (int o = 1; o < 32; o <<= 1) {
        const double y0 = __shfl_up_sync(0xffffffffu, x0, o), y1 = __shfl_up_sync(0xffffffffu, x1, o);
        if (lane >= o) { x0 *= y0; x1 *= y1; }
    }
    const double low_total = __shfl_sync(0xffffffffu, x0, 31);  // product over modes 0..31
    const double e0 = __shfl_up_sync(0xffffffffu, x0, 1), e1 = __shfl_up_sync(0xffffffffu, x1, 1);
    const double P[2] = {lane ? e0 : 1.0, (lane ? e1 : 1.0) * low_total};
    for (int q = 0; q < 2; ++q) {
        const int k = lane + 32 * q;
        if (k >= N) continue;
        if (k < k0) {
            p.a[grow * N + k] = cur[q];
            continue;
        }
        const double sk = r0 * P[q] * v[q];
        // phi~_k = phi_k - phi_0 - k (phi_1 - phi_0): errors in the phases of modes 0 and 1 come back k-fold
        // when the density is evaluated on the stored configuration, so those two are formed in FP64; the
        // others carry an FP32 rounding of the draw (as the stored draw itself does).
        double ph = (double)p.phi[grow * N + k] + alpha + (double)k * theta;
        if (!p.dbl) {
            // FP32 chains store the proposal rounded to FP32 (its density and energy are taken of that
            // rounding, the configuration the chain will hold), so the magnitude and the unit vector are
            // formed in FP32; (n s)^(1/4) of very small values is taken after an exact scaling by 2^128
            const double x = n * fmax(sk, 0.0);
            const bool tiny = x < 0x1p-100;
            const float Af = sqrtf(sqrtf((float)(tiny ? x * 0x1p128 : x))) * (tiny ? 0x1p-32f : 1.f);
            if (k < 2) {
                double sn, cs;
                sincos(ph, &sn, &cs);
                p.a[grow * N + k] = make_double2((float)((double)Af * cs), (float)((double)Af * sn));
            } else {
                float sf, cf;
                sincosf((float)(ph - kTwoPi * floor(ph * (1.0 / kTwoPi))), &sf, &cf);
                p.a[grow * N + k] = make_double2((double)(Af * cf), (double)(Af * sf));
            }
            continue;
        }
        // FP64 chains: the unit vector is renormalised in FP64 so that |a_k|^4 = n s_k holds to FP64 rounding
        const double A = sqrt(sqrt(n * fmax(sk, 0.0)));
        double sn, cs;
        if (k < 2) {
            sincos(ph, &sn, &cs);
        } else {
            ph -= kTwoPi * floor(ph / kTwoPi);
            float sf, cf;
            sincosf((float)ph, &sf, &cf);
            const double inv = 1.0 / sqrt((double)cf * cf + (double)sf * sf);
            sn = sf * inv;
            cs = cf * inv;
        }
        p.a[grow * N + k] = make_double2(A * cs, A * sn);
    }
}

cudaError_t launch_assemble(const AssembleParams &p, int S, cudaStream_t s) {
    dim3 grid(p.rows_per_sample, S);  // one row (warp) per block: the FP64 work spread over all SMs
    assemble_kernel<<<grid, 32, 0, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Index of the pair (x, y), x < y, in a table of the upper triangle stored diagonal by diagonal: the pairs of
// distance d = y - x are consecutive in x.  Consecutive quadruplets of the canonical order share their first
// pair and step their second pair (z, z + d) along a diagonal, so the lanes of a warp read one entry and
// consecutive entries (no shared-memory bank conflicts).
__device__ __forceinline__ int tri_index(int x, int y, int N) {
    const int d = y - x;
    return (d - 1) * N - (d - 1) * d / 2 + x;
}

// Double-float arithmetic (a value as an unevaluated sum hi + lo of two floats, ~48 significant bits) from
// the error-free transformations: Knuth's two-sum and the FMA form of Dekker's two-product.
struct dfloat {
    float hi, lo;
};
__device__ __forceinline__ dfloat two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dfloat fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfloat two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
// Re(u conj w) = u.re w.re + u.im w.im for double-float u = (re, im), w = (re, im) (float4: re.hi, re.lo,
// im.hi, im.lo)
__device__ __forceinline__ dfloat df_dot2(float4 u, float4 w) {
    const dfloat p1 = two_prod(u.x, w.x), p2 = two_prod(u.z, w.z);
    const dfloat s = two_sum(p1.hi, p2.hi);
    float lo = __fadd_rn(p1.lo, p2.lo);
    lo = __fmaf_rn(u.x, w.y, lo);
    lo = __fmaf_rn(u.y, w.x, lo);
    lo = __fmaf_rn(u.z, w.w, lo);
    lo = __fmaf_rn(u.w, w.z, lo);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, lo));
}
// conj(a_x) a_y for FP32 amplitudes, each component exact as a two-product pair, summed to double-float
__device__ __forceinline__ float4 df_pair(float2 ax, float2 ay) {
    const dfloat r1 = two_prod(ax.x, ay.x), r2 = two_prod(ax.y, ay.y);   // re = ax.x ay.x + ax.y ay.y
    const dfloat i1 = two_prod(ax.x, ay.y), i2 = two_prod(-ax.y, ay.x);  // im = ax.x ay.y - ax.y ay.x
    const dfloat rs = two_sum(r1.hi, r2.hi), is = two_sum(i1.hi, i2.hi);
    const dfloat re = fast_two_sum(rs.hi, __fadd_rn(rs.lo, __fadd_rn(r1.lo, r2.lo)));
    const dfloat im = fast_two_sum(is.hi, __fadd_rn(is.lo, __fadd_rn(i1.lo, i2.lo)));
    return make_float4(re.hi, re.lo, im.hi, im.lo);
}

// Energy H = -cc sum_q J_q Re(conj(a_x) a_y a_z conj(a_w)) of one row per block; blockIdx.z picks one of two
// row sets (the current configurations and the proposals of a round).
//  - The pair products P(x, y) = conj(a_x) a_y, x < y, are tabulated in shared memory (upper triangle by
//    diagonals, N(N-1)/2 entries of 16 bytes, 31.5 KB at N = 64, so that a launch's blocks fit in one wave);
//    a pair given in the other order is the conjugate, a sign flip done on the bits.  Each term is then
//    J_q Re(P(x, y) conj P(z, w)).
//  - kDF (FP32 configurations): P in double-float from exact two-products, the terms and the running sum
//    of a thread in double-float (about 30 FP32 operations per quadruplet), the threads' sums added in
//    FP64.  GB300 runs FP32 at many times its FP64 rate, and the sum stays within ~1e-14 of the FP64 one.
//  - otherwise FP64: three operations per quadruplet (nine for the direct product).
//  - Summing runs of quadruplets that share their first pair before multiplying by P(x, y) would save a
//    third of the FP64 operations, but the run boundaries differ between the lanes of a warp and the
//    divergent flushes cost the whole warp: it measured slower.
template <bool kDF>
__global__ void __launch_bounds__(256) energy_list_kernel(EnergyList2 pp) {
    extern __shared__ double2 pairs[];  // [N (N - 1) / 2] (as float4 (re.hi, re.lo, im.hi, im.lo) with kDF)
    __shared__ double2 sa[kLearnMaxN];
    __shared__ double red[8];
    const EnergyListParams &p = pp.set[blockIdx.z];
    const int s = blockIdx.y, row = blockIdx.x, N = p.N;
    if (row >= p.rows_per_sample) return;
    const int64_t grow = (int64_t)s * p.rows_per_sample + row;
    const SampleDev sd = p.samples[s];
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        if (p.slot) {
            const int64_t base = sd.a_off + (int64_t)(p.slot[grow] - sd.chain0) * N;
            if (p.dbl) sa[k] = reinterpret_cast<const double2 *>(p.a)[base + k];
            else { const float2 v = reinterpret_cast<const float2 *>(p.a)[base + k]; sa[k] = make_double2(v.x, v.y); }
        } else if (p.dbl) {
            sa[k] = reinterpret_cast<const double2 *>(p.a)[grow * N + k];
        } else {
            const float2 v = reinterpret_cast<const float2 *>(p.a)[grow * N + k];
            sa[k] = make_double2(v.x, v.y);
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < N * (N - 1) / 2; e += blockDim.x) {
        int d = 1, rem = e;  // e -> diagonal d, x (the inverse of tri_index)
        while (rem >= N - d) { rem -= N - d; ++d; }
        const int x = rem, y = x + d;
        const double2 ax = sa[x], ay = sa[y];
        if (kDF)
            reinterpret_cast<float4 *>(pairs)[e] =
                df_pair(make_float2((float)ax.x, (float)ax.y), make_float2((float)ay.x, (float)ay.y));
        else
            pairs[e] = make_double2(ax.x * ay.x + ax.y * ay.y, ax.x * ay.y - ax.y * ay.x);
    }
    __syncthreads();
    const int4 *Q = p.quads + sd.q_off;
    double acc = 0.0;
    if (kDF) {
        const float2 *J = p.Jdf + sd.q_off;
        const float4 *P4 = reinterpret_cast<const float4 *>(pairs);
        float ahi = 0.f, alo = 0.f;
        constexpr int kU = 4;  // quadruplets per batch: their loads are issued together (latency, not ALU, bounds)
        for (int64_t q0 = threadIdx.x; q0 < sd.nq; q0 += (int64_t)kU * blockDim.x) {
            int4 t[kU];
            float2 j[kU];
#pragma unroll
            for (int i = 0; i < kU; ++i) {
                const int64_t q = q0 + (int64_t)i * blockDim.x;
                const bool in = q < sd.nq;
                t[i] = in ? __ldg(Q + q) : make_int4(0, 1, 0, 1);
                j[i] = in ? __ldg(J + q) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < kU; ++i) {
                const bool f1 = t[i].x > t[i].y, f2 = t[i].z > t[i].w;
                const float4 u = P4[f1 ? tri_index(t[i].y, t[i].x, N) : tri_index(t[i].x, t[i].y, N)];
                float4 w = P4[f2 ? tri_index(t[i].w, t[i].z, N) : tri_index(t[i].z, t[i].w, N)];
                if (f1 != f2) { w.z = -w.z; w.w = -w.w; }  // one of the pairs stored the other way round
                const dfloat v = df_dot2(u, w);
                const dfloat m = two_prod(j[i].x, v.hi);
                const float mlo = __fmaf_rn(j[i].x, v.lo, __fmaf_rn(j[i].y, v.hi, m.lo));
                const dfloat s1 = two_sum(ahi, m.hi);
                ahi = s1.hi;
                alo = __fadd_rn(alo, __fadd_rn(s1.lo, mlo));
            }
        }
        acc = (double)ahi + (double)alo;
    } else {
        const double *J = p.Jq + sd.q_off;
        for (int64_t q = threadIdx.x; q < sd.nq; q += blockDim.x) {
            const int4 t = Q[q];
            const bool f1 = t.x > t.y, f2 = t.z > t.w;
            const double2 u = pairs[f1 ? tri_index(t.y, t.x, N) : tri_index(t.x, t.y, N)];
            const double2 w = pairs[f2 ? tri_index(t.w, t.z, N) : tri_index(t.z, t.w, N)];
            // Im P(x, y) Im P(z, w) changes sign when exactly one of the two pairs was stored the other way round
            const double wy = __longlong_as_double(__double_as_longlong(w.y) ^ ((long long)(f1 != f2) << 63));
            acc = fma(J[q], fma(u.x, w.x, u.y * wy), acc);
        }
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        p.E[grow] = -p.cc * t;
    }
}

cudaError_t launch_energy_list(const EnergyList2 &p, int n_sets, int S, cudaStream_t s) {
    int rows = 0;
    for (int i = 0; i < n_sets; ++i) {
        if (p.set[i].N < 1 || p.set[i].N > kLearnMaxN || p.set[i].N != p.set[0].N) return cudaErrorInvalidValue;
        if ((p.set[i].Jdf != nullptr) != (p.set[0].Jdf != nullptr)) return cudaErrorInvalidValue;
        rows = std::max(rows, p.set[i].rows_per_sample);
    }
    if (rows <= 0) return cudaSuccess;
    const size_t sm = sizeof(double2) * (size_t)p.set[0].N * (p.set[0].N - 1) / 2;
    dim3 grid(rows, S, n_sets);
    if (p.set[0].Jdf) energy_list_kernel<true><<<grid, 256, sm, s>>>(p);
    else energy_list_kernel<false><<<grid, 256, sm, s>>>(p);
    return cudaGetLastError();
}

__global__ void split_df_kernel(const double *J, float2 *Jdf, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float hi = (float)J[i];
        Jdf[i] = make_float2(hi, (float)(J[i] - (double)hi));
    }
}

cudaError_t launch_split_df(const double *J, float2 *Jdf, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    split_df_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(J, Jdf, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
__global__ void mh_kernel(MHParams p) {
    const int s = blockIdx.y, row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= p.rows_per_sample) return;
    const int64_t grow = (int64_t)s * p.rows_per_sample + row;
    const int slot = p.slot[grow];
    const int t = p.label[slot];
    const double beta = p.beta[t];
    const double lA = -beta * (p.H_prop[grow] - p.H_cur[grow]) + (p.logq_cur[grow] + (double)p.extra_cur[grow]) -
                      (p.logq_prop[grow] + (double)p.extra_prop[grow]);
    const u32x4 w = draw(p.seed, p.row_id[grow], (uint32_t)p.ctl->global_rounds, (uint32_t)(p.N + 1), kTagGlobal);
    const bool acc = isfinite(lA) && (lA >= 0.0 || log(u01(w.x)) < lA);
    atomicAdd(p.att + (int64_t)s * p.nT + t, 1ull);
    if (acc) {
        atomicAdd(p.acc + (int64_t)s * p.nT + t, 1ull);
        const SampleDev sd = p.samples[s];
        const int64_t base = sd.a_off + (int64_t)(slot - sd.chain0) * p.N;
        for (int k = 0; k < p.N; ++k) {
            const double2 v = p.a_prop[grow * p.N + k];
            if (p.dbl) reinterpret_cast<double2 *>(p.a)[base + k] = v;
            else reinterpret_cast<float2 *>(p.a)[base + k] = make_float2((float)v.x, (float)v.y);
        }
        p.E[slot] = p.H_prop[grow];
    }
}

cudaError_t launch_mh(const MHParams &p, int S, cudaStream_t s) {
    dim3 grid((p.rows_per_sample + 63) / 64, S);
    mh_kernel<<<grid, 64, 0, s>>>(p);
    return cudaGetLastError();
}

__global__ void learn_loss_kernel(const double *logq, const float *extra, int n, double *out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc -= logq[i] + (double)extra[i];
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
        *out = t / n;
    }
}

cudaError_t launch_learn_loss(const double *logq, const float *extra, int S, int rows, double *out, cudaStream_t s) {
    learn_loss_kernel<<<1, 256, 0, s>>>(logq, extra, S * rows, out);
    return cudaGetLastError();
}

__global__ void cold_rows_kernel(const int *perm, int S, int R, int nT, int ncold, int *slot, uint32_t *row_id,
                                 int *cond) {
    const int s = blockIdx.x, i = threadIdx.x;
    if (i >= ncold * R) return;
    const int t = i / R, r = i % R;
    const int64_t out = (int64_t)s * ncold * R + i;
    slot[out] = perm[((int64_t)s * R + r) * nT + t];
    row_id[out] = (uint32_t)((s * R + r) * nT + t);
    cond[out] = t;
}

cudaError_t launch_cold_rows(const int *perm, int S, int R, int nT, int ncold, int *slot, uint32_t *row_id,
                             int *cond, cudaStream_t s) {
    cold_rows_kernel<<<S, 1024, 0, s>>>(perm, S, R, nT, ncold, slot, row_id, cond);
    return cudaGetLastError();
}

}  // namespace ptgb
