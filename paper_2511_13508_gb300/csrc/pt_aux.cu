// pt_aux.cu -- chain initialisation, replica-exchange swaps, measurements and the plain FP64 path of
// the smoothed-cubic Parallel-Tempering engine (arXiv 2511.13508).
#include <cstdint>
#include "pt_common.cuh"
#include "pt_kernels.h"

namespace ptgb {

template <typename T> __device__ __forceinline__ T block_sum(T v, T *scratch) {
    // scratch: >= 32 entries; every thread of the block must call
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = (blockDim.x + 31) / 32;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    T t = T(0);
    for (int w = 0; w < nw; ++w) t += scratch[w];
    return t;
}

// ------------------------------------------------------------------------------------------------
// Initial chains: exact draws of the beta = 0 law (uniform on sum |a|^4 = N with uniform phases):
// u = sqrt(N) |g| / ||g||, g Gaussian by Box-Muller, a_k = sqrt(u_k) e^{i phi_k}.  Stream INIT with
// counter (chain id, mode, 0, tag), chain id = (s R + r) nT + t.
__global__ void init_kernel(InitParams p) {
    __shared__ double scratch[32];
    const int slot = blockIdx.x;
    const int s = p.chain_sample[slot];
    const SampleDev sd = p.samples[s];
    const int N = sd.N;
    const int r = (slot - sd.chain0) / p.nT, t = p.label[slot];
    const uint32_t cid = (uint32_t)((s * p.R + r) * p.nT + t);
    double g2 = 0.0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const u32x4 w = draw(p.seed, cid, (uint32_t)k, 0u, kTagInit);
        const double g = sqrt(-2.0 * log(u01(w.x))) * cos(kTwoPi * u01(w.y));
        g2 += g * g;
    }
    const double nrm = sqrt(block_sum(g2, scratch));
    const int64_t base = sd.a_off + (int64_t)(slot - sd.chain0) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const u32x4 w = draw(p.seed, cid, (uint32_t)k, 0u, kTagInit);
        const double g = sqrt(-2.0 * log(u01(w.x))) * cos(kTwoPi * u01(w.y));
        const double ph = kTwoPi * u01(w.z);
        const double u = sqrt((double)N) * fabs(g) / nrm;
        const double A = sqrt(u);
        const double re = A * cos(ph), im = A * sin(ph);
        if (p.dbl) reinterpret_cast<double2 *>(p.a)[base + k] = make_double2(re, im);
        else reinterpret_cast<float2 *>(p.a)[base + k] = make_float2((float)re, (float)im);
    }
}

cudaError_t launch_init(const InitParams &p, int n_chains, cudaStream_t s) {
    if (n_chains <= 0) return cudaSuccess;
    init_kernel<<<n_chains, 128, 0, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// One swap pass: per (sample, replica) ladder, sequentially i = 0 .. nT-2 (ascending T), exchange the
// temperatures of the chains at i and i+1 with probability min[1, exp((b_i - b_{i+1})(E_i - E_{i+1}))]
// (paper Eq. (15)).  Labels are exchanged instead of configurations.  The per-chain Metropolis
// counters are first folded into per-temperature counters under the labels they were earned with.
__global__ void swap_kernel(SwapParams p) {
    const int ladder = blockIdx.x * blockDim.x + threadIdx.x;
    if (ladder >= p.S * p.R) return;
    const int s = ladder / p.R;
    int *perm = p.perm + (int64_t)ladder * p.nT;
    for (int t = 0; t < p.nT; ++t) {
        const int slot = perm[t];
        atomicAdd(p.mcT_acc + (int64_t)s * p.nT + t, p.mc_acc[slot]);
        atomicAdd(p.mcT_att + (int64_t)s * p.nT + t, p.mc_att[slot]);
        p.mc_acc[slot] = 0ull;
        p.mc_att[slot] = 0ull;
    }
    const uint32_t pass = (uint32_t)p.ctl->swap_passes;
    for (int i = 0; i + 1 < p.nT; ++i) {
        const int c0 = perm[i], c1 = perm[i + 1];
        const double D = (p.beta[i] - p.beta[i + 1]) * (p.E[c0] - p.E[c1]);
        const u32x4 w = draw(p.seed, (uint32_t)ladder, pass, (uint32_t)i, kTagSwap);
        const int64_t pi = (int64_t)ladder * (p.nT - 1) + i;
        p.swap_att[pi] += 1ull;
        if (D >= 0.0 || u01(w.x) < exp(D)) {
            perm[i] = c1; perm[i + 1] = c0;
            p.label[c0] = i + 1; p.label[c1] = i;
            p.swap_acc[pi] += 1ull;
        }
    }
}

cudaError_t launch_swap(const SwapParams &p, cudaStream_t s) {
    const int n = p.S * p.R;
    if (n <= 0 || p.nT < 2) return cudaSuccess;
    swap_kernel<<<(n + 127) / 128, 128, 0, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Measurements of one (sample, temperature) per block over the snapshots and/or the live state:
// E, E^2 (specific heat, Eq. (21)), Y2, Y4 (Sec. IV.D), I, I^2 per chain; for every replica pair the
// overlap q = Re sum conj(a^c) a^d / N (Sec. IV.C), its moments and its 201-bin histogram.
template <typename V>
__device__ void measure_one(const MeasureParams &p, const V *a, const double *E, int s, int t, double *scratch) {
    const SampleDev sd = p.samples[s];
    const int N = sd.N;
    double *st = p.stat + ((int64_t)s * p.nT + t) * 7;
    double *qs = p.qstat + ((int64_t)s * p.nT + t) * 5;
    unsigned long long *h = p.qhist + ((int64_t)s * p.nT + t) * 201;
    const int *perm = p.perm + (int64_t)s * p.R * p.nT;
    for (int r = 0; r < p.R; ++r) {
        const int slot = perm[r * p.nT + t];
        const V *x = a + sd.a_off + (int64_t)(slot - sd.chain0) * N;
        double i2 = 0.0, i4 = 0.0, i8 = 0.0;
        for (int k = threadIdx.x; k < N; k += blockDim.x) {
            const V v = x[k];
            const double u = (double)v.x * v.x + (double)v.y * v.y;
            i2 += u; i4 += u * u; i8 += (u * u) * (u * u);
        }
        i2 = block_sum(i2, scratch);
        i4 = block_sum(i4, scratch);
        i8 = block_sum(i8, scratch);
        if (threadIdx.x == 0) {
            const double e = E[slot];
            st[0] += 1.0; st[1] += e; st[2] += e * e;
            st[3] += i4 / (i2 * i2); st[4] += i8 / (i4 * i4);
            st[5] += i2; st[6] += i2 * i2;
        }
    }
    for (int r1 = 0; r1 < p.R; ++r1)
        for (int r2 = r1 + 1; r2 < p.R; ++r2) {
            const V *x = a + sd.a_off + (int64_t)(perm[r1 * p.nT + t] - sd.chain0) * N;
            const V *y = a + sd.a_off + (int64_t)(perm[r2 * p.nT + t] - sd.chain0) * N;
            double d = 0.0;
            for (int k = threadIdx.x; k < N; k += blockDim.x) {
                const V u = x[k], v = y[k];
                d += (double)u.x * v.x + (double)u.y * v.y;
            }
            d = block_sum(d, scratch);
            if (threadIdx.x == 0) {
                const double q = d / (double)N;
                qs[0] += 1.0; qs[1] += q; qs[2] += q * q; qs[3] += q * q * q; qs[4] += (q * q) * (q * q);
                int b = (int)floor(100.0 * (q + 1.0) + 0.5);
                b = b < 0 ? 0 : (b > 200 ? 200 : b);
                h[b] += 1ull;
            }
        }
}

template <typename V> __global__ void measure_kernel(MeasureParams p) {
    __shared__ double scratch[32];
    const int s = blockIdx.x / p.nT, t = blockIdx.x % p.nT;
    for (int kk = 0; kk < p.n_snap; ++kk)
        measure_one<V>(p, reinterpret_cast<const V *>(p.snap_a) + (int64_t)kk * p.a_total,
                       p.snap_E + (int64_t)kk * p.n_chains, s, t, scratch);
    if (p.live) measure_one<V>(p, reinterpret_cast<const V *>(p.a), p.E, s, t, scratch);
}

cudaError_t launch_measure(const MeasureParams &p, cudaStream_t s) {
    if (p.n_snap <= 0 && !p.live) return cudaSuccess;
    if (p.dbl) measure_kernel<double2><<<p.S * p.nT, 128, 0, s>>>(p);
    else measure_kernel<float2><<<p.S * p.nT, 128, 0, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Plain FP64 path: the paper's GPU design restated (Sec. III.A.3): for every proposed pair move one
// thread per quadruplet holding j or k computes that quadruplet's energy change, the contributions are
// summed by a shared-memory tree reduction (O(log) depth), and one block simulates one chain; J is read
// from global memory by every chain separately.
__device__ __forceinline__ double2 cm(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double quad_term(double2 xa, double2 xb, double2 xc, double2 xd) {
    // Re( conj(a_a) a_b a_c conj(a_d) )
    const double2 ca = make_double2(xa.x, -xa.y), cd = make_double2(xd.x, -xd.y);
    return cm(cm(ca, xb), cm(xc, cd)).x;
}

__device__ __forceinline__ double tree_sum(double v, double *buf) {
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) buf[threadIdx.x] += buf[threadIdx.x + h];
        __syncthreads();
    }
    const double r = buf[0];
    __syncthreads();
    return r;
}

constexpr int kPlainThreads = 256;

__global__ void __launch_bounds__(kPlainThreads) plain_sweep_kernel(PlainParams p) {
    extern __shared__ double2 sa[];  // maxN amplitudes
    __shared__ double buf[kPlainThreads];
    __shared__ double2 s_new[2];
    __shared__ double s_U;
    const int slot = blockIdx.x;
    const int s = p.chain_sample[slot];
    const SampleDev sd = p.samples[s];
    const int N = sd.N, tid = threadIdx.x;
    const int r = (slot - sd.chain0) / p.nT, t = p.label[slot];
    const uint32_t cid = (uint32_t)((s * p.R + r) * p.nT + t);
    const double beta = p.beta[t];
    double2 *ag = p.a + sd.a_off + (int64_t)(slot - sd.chain0) * N;
    for (int k = tid; k < N; k += blockDim.x) sa[k] = ag[k];
    double E = p.E[slot];
    unsigned long long acc = 0, att = 0;
    const long long base = p.ctl->sweep_base;
    const int *inc_off = p.inc_off + sd.mode_off;
    const int *inc = p.inc + sd.inc_off;
    const int4 *quads = p.quads + sd.q_off;
    const double *Jq = p.Jq + sd.q_off;
    __syncthreads();
    for (int sw = 0; sw < p.n_sweeps; ++sw) {
        const uint32_t sweep = (uint32_t)(base + sw);
        for (int u = 0; u < N / 2; ++u) {
            int j, k;
            pair_jk(p.seed, (uint32_t)s, sweep, (uint32_t)u, N, j, k);
            if (tid == 0) {
                const u32x4 w = draw(p.seed, cid, sweep, (uint32_t)u, kTagPropose);
                const double2 aj = sa[j], ak = sa[k];
                const double uj = aj.x * aj.x + aj.y * aj.y, uk = ak.x * ak.x + ak.y * ak.y;
                const double K = sqrt(sqrt(uj * uj + uk * uk));
                const double phj = kTwoPi * u01(w.x), phk = kTwoPi * u01(w.y), th = kHalfPi * u01(w.z);
                const double Aj = K * sqrt(cos(th)), Ak = K * sqrt(sin(th));
                s_new[0] = make_double2(Aj * cos(phj), Aj * sin(phj));
                s_new[1] = make_double2(Ak * cos(phk), Ak * sin(phk));
                s_U = u01(w.w);
            }
            __syncthreads();
            const double2 nj = s_new[0], nk = s_new[1];
            const int oj = inc_off[j], nj_cnt = inc_off[j + 1] - oj;
            const int ok = inc_off[k], nk_cnt = inc_off[k + 1] - ok;
            double local = 0.0;
            for (int idx = tid; idx < nj_cnt + nk_cnt; idx += blockDim.x) {
                const int q = idx < nj_cnt ? inc[oj + idx] : inc[ok + idx - nj_cnt];
                const int4 Q = quads[q];
                const bool hasj = (Q.x == j || Q.y == j || Q.z == j || Q.w == j);
                if (idx >= nj_cnt && hasj) continue;  // counted once, from j's list
                double2 xa = sa[Q.x], xb = sa[Q.y], xc = sa[Q.z], xd = sa[Q.w];
                const double told = quad_term(xa, xb, xc, xd);
                if (Q.x == j) xa = nj; else if (Q.x == k) xa = nk;
                if (Q.y == j) xb = nj; else if (Q.y == k) xb = nk;
                if (Q.z == j) xc = nj; else if (Q.z == k) xc = nk;
                if (Q.w == j) xd = nj; else if (Q.w == k) xd = nk;
                local += Jq[q] * (quad_term(xa, xb, xc, xd) - told);
            }
            const double dH = -p.cc * tree_sum(local, buf);
            if (tid == 0) {
                ++att;
                if (dH <= 0.0 || s_U < exp(-beta * dH)) {
                    sa[j] = nj; sa[k] = nk;
                    E += dH;
                    ++acc;
                }
            }
            __syncthreads();
        }
        const long long done = base + sw + 1;
        if (p.measure_every > 0 && done % p.measure_every == 0 && sw + 1 < p.n_sweeps) {
            const int kk = (int)(done / p.measure_every - base / p.measure_every - 1);
            if (kk >= 0 && kk < p.n_snap_max) {
                double2 *dst = p.snap_a + (int64_t)kk * p.a_total + sd.a_off + (int64_t)(slot - sd.chain0) * N;
                for (int x = tid; x < N; x += blockDim.x) dst[x] = sa[x];
                if (tid == 0) p.snap_E[(int64_t)kk * p.n_chains + slot] = E;
            }
            __syncthreads();
        }
    }
    for (int x = tid; x < N; x += blockDim.x) ag[x] = sa[x];
    if (tid == 0) {
        p.E[slot] = E;
        p.mc_acc[slot] += acc;
        p.mc_att[slot] += att;
    }
}

__global__ void __launch_bounds__(kPlainThreads) plain_energy_kernel(PlainParams p) {
    extern __shared__ double2 sa[];
    __shared__ double buf[kPlainThreads];
    const int slot = blockIdx.x;
    const int s = p.chain_sample[slot];
    const SampleDev sd = p.samples[s];
    const int N = sd.N, tid = threadIdx.x;
    double2 *ag = p.a + sd.a_off + (int64_t)(slot - sd.chain0) * N;
    for (int k = tid; k < N; k += blockDim.x) sa[k] = ag[k];
    __syncthreads();
    if (p.renorm) {
        double s4 = 0.0;
        for (int k = tid; k < N; k += blockDim.x) {
            const double u = sa[k].x * sa[k].x + sa[k].y * sa[k].y;
            s4 += u * u;
        }
        s4 = tree_sum(s4, buf);
        if (!(s4 > 0.0) || !isfinite(s4)) record_error(p.ctl, kErrNaN, 20);
        const double f = sqrt(sqrt((double)N / s4));
        for (int k = tid; k < N; k += blockDim.x) {
            sa[k] = make_double2(sa[k].x * f, sa[k].y * f);
            ag[k] = sa[k];
        }
        __syncthreads();
    }
    const int4 *quads = p.quads + sd.q_off;
    const double *Jq = p.Jq + sd.q_off;
    const int64_t count = sd.nq;
    double local = 0.0;
    for (int64_t q = tid; q < count; q += blockDim.x) {
        const int4 Q = quads[q];
        local += Jq[q] * quad_term(sa[Q.x], sa[Q.y], sa[Q.z], sa[Q.w]);
    }
    const double E = -p.cc * tree_sum(local, buf);
    if (tid == 0) {
        if (!isfinite(E)) record_error(p.ctl, kErrNaN, 21);
        if (p.write_state) p.E[slot] = E;
        if (p.E_out) p.E_out[slot] = E;
    }
}

cudaError_t launch_plain_sweep(const PlainParams &p, int n_chains, cudaStream_t s) {
    if (n_chains <= 0 || p.n_sweeps <= 0) return cudaSuccess;
    plain_sweep_kernel<<<n_chains, kPlainThreads, (size_t)p.maxN * sizeof(double2), s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_plain_energy(const PlainParams &p, int n_chains, cudaStream_t s) {
    if (n_chains <= 0) return cudaSuccess;
    plain_energy_kernel<<<n_chains, kPlainThreads, (size_t)p.maxN * sizeof(double2), s>>>(p);
    return cudaGetLastError();
}

// Health check of the bounded waits: waits on a flag no kernel sets until the limit, then records the
// same timeout status as the engine's own waits.
__global__ void wait_probe_kernel(Control *ctl, unsigned long long limit_ns) {
    const volatile int *flag = &ctl->probe_flag;
    const unsigned long long t0 = global_ns();
    while (*flag == 0) {
        if (global_ns() - t0 > limit_ns) {
            record_error(ctl, kErrTimeout, 40);
            return;
        }
        __nanosleep(1000);
    }
}

cudaError_t launch_wait_probe(Control *ctl, unsigned long long limit_ns, cudaStream_t s) {
    wait_probe_kernel<<<1, 1, 0, s>>>(ctl, limit_ns);
    return cudaGetLastError();
}

__global__ void advance_kernel(Control *ctl, long long sweeps, long long passes, long long rounds) {
    ctl->sweep_base += sweeps;
    ctl->swap_passes += passes;
    ctl->global_rounds += rounds;
}

cudaError_t launch_advance(Control *ctl, long long sweeps, long long passes, long long rounds, cudaStream_t s) {
    advance_kernel<<<1, 1, 0, s>>>(ctl, sweeps, passes, rounds);
    return cudaGetLastError();
}

}  // namespace ptgb
