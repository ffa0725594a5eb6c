// pt_graph.cu -- FP32 sweep and energy kernels for explicit interaction lists (the random-frequency
// mode-locked graph of arXiv 2511.13508, Sec. II.C, or any list of quadruplets).
//
// One thread block per group of up to 8 chains of one disorder sample.  A lane is (chain c, worker w):
// the 128 workers of the block split the quadruplets that hold the updated modes j or k, and the 8
// lanes of a worker read each incidence record once for their 8 chains.  An incidence record of mode l
// is (the other three modes in position order, (q << 2) | position of l) with its coupling alongside,
// so a lane needs no search and no dependent load to evaluate a quadruplet.  Per chain the lane
// accumulates the local fields of j and k and the j-k cross term (Sec. III.A.1 and III.A.3; term of
// quadruplet (q0, q1, q2, q3): -cc J Re(conj(a_q0) a_q1 a_q2 conj(a_q3))):
//     h_l = sum_{q holding l} J_q (product of the other three factors), conjugated when l sits at
//           position 1 or 2, so that H = -cc Re(conj(a_l) h_l) + (terms without l);
//     dH  = -cc Re[ conj(dj) h_j + conj(dk) h_k + sum_{q holding j and k} J_q x x dxj dxk ],
// with dxl = conj(dl) at positions 0 and 3, dl at 1 and 2.  Products in FP32, energies in FP64.
#include <cstdint>
#include "pt_common.cuh"
#include "pt_kernels.h"

namespace ptgb {

namespace {

constexpr int kGG = 8;                      // chains per block
constexpr int kGThreads = 1024;             // 32 warps
constexpr int kGWarps = kGThreads / 32;
constexpr int kGWorkers = kGThreads / kGG;  // 128
// row stride of the amplitude table (float2), unpadded: a warp's four records then gather from two 64-byte halves
// of the banks instead of windows at 16 offsets (fewer bank conflicts; measured on GB300, random graph N = 64:
// 4.46M -> 4.73M chain-sweeps/s against a stride of kGG + 1)
constexpr int kGRS = kGraphRowStride;
static_assert(kGRS == kGG, "row stride");

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// factor of position p in the term: conjugated at positions 0 and 3
__device__ __forceinline__ float2 fac(float2 v, int p) { return (p == 0 || p == 3) ? make_float2(v.x, -v.y) : v; }

struct GraphProposal {
    float2 dj, dk, nj, nk;
    float U;
};

__device__ __forceinline__ GraphProposal graph_proposal(uint64_t seed, uint32_t chain_id, uint32_t sweep,
                                                        uint32_t update, float2 aj, float2 ak) {
    // the pair move of Sec. III.A.1: K^4 = |a_j|^4 + |a_k|^4, theta ~ U[0, pi/2], fresh uniform phases;
    // mode j receives K sqrt(cos theta), mode k receives K sqrt(sin theta)
    GraphProposal P;
    const u32x4 w = draw(seed, chain_id, sweep, update, kTagPropose);
    const float uj = aj.x * aj.x + aj.y * aj.y, uk = ak.x * ak.x + ak.y * ak.y;
    const float K = sqrtf(sqrtf(uj * uj + uk * uk));
    const float kInv = 2.3283064365386963e-10f;
    const float fj = ((float)w.x + 0.5f) * kInv, fk = ((float)w.y + 0.5f) * kInv, ft = ((float)w.z + 0.5f) * kInv;
    float sj, cj, sk, ck, st, ct;
    sincospif(2.0f * fj, &sj, &cj);
    sincospif(2.0f * fk, &sk, &ck);
    sincospif(0.5f * ft, &st, &ct);
    const float Aj = K * sqrtf(ct), Ak = K * sqrtf(st);
    P.nj = make_float2(Aj * cj, Aj * sj);
    P.nk = make_float2(Ak * ck, Ak * sk);
    P.dj = make_float2(P.nj.x - aj.x, P.nj.y - aj.y);
    P.dk = make_float2(P.nk.x - ak.x, P.nk.y - ak.y);
    P.U = ((float)w.w + 0.5f) * kInv;
    return P;
}

}  // namespace

// Variants by how an update's records reach the workers:
//  kPlain: each worker loads its records from global memory (L2) as it goes (the largest graphs).
//  kFew: every update's two record lists fit the workers (at most one record each, sparse graphs).  An
//    update is then bound by its fixed latencies, and the kernel trims them: the record offsets sit in
//    shared memory, each worker loads its record of the next update while the current one is reduced (the
//    pairs and the records do not depend on the state), and the leaders sum only the warps that held
//    records.
//  kStage: the two lists fit in shared memory; the whole block copies them there with asynchronous copies
//    while the leaders draw the proposal (one L2 latency per update instead of one per record and worker).
enum GraphVariant : int { kPlain = 0, kFew = 1, kStage = 2 };

// Shared-memory layout of the sweep kernel: amplitudes [maxN][kGRS] float2, record offsets [maxN + 1] int,
// then (kStage) the staged records [cap] int4 and couplings [cap] float.
struct GraphSmem {
    size_t inc, rec, J, total;
};
__host__ __device__ inline GraphSmem graph_smem(int maxN, int cap) {
    GraphSmem g;
    g.inc = (size_t)maxN * kGRS * sizeof(float2);
    g.rec = (g.inc + (size_t)(maxN + 1) * sizeof(int) + 15) / 16 * 16;
    g.J = g.rec + (size_t)cap * sizeof(int4);
    g.total = g.J + (size_t)cap * sizeof(float);
    return g;
}

template <int kVar>
__global__ void __launch_bounds__(kGThreads) graph_sweep_kernel(GraphParams p) {
    constexpr bool kFewV = kVar == kFew, kStageV = kVar == kStage;
    extern __shared__ __align__(16) float2 ga[];  // laid out as graph_smem
    __shared__ float red[kGWarps][kGG][5];
    __shared__ GraphProposal prop[kGG];
    const GroupDev gr = p.groups[blockIdx.x];
    const SampleDev sd = p.samples[gr.sample];
    const int N = sd.N, tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int c = lane % kGG, worker = warp * (32 / kGG) + lane / kGG;
    const bool leader = tid < kGG;  // warp 0, worker 0: chain c = tid
    float2 *A = p.a + sd.a_off + (int64_t)(gr.chain0 - sd.chain0) * N;
    for (int i = tid; i < N * kGG; i += kGThreads) {
        const int x = i / kGG, cc = i % kGG;
        ga[x * kGRS + cc] = cc < gr.count ? A[(int64_t)cc * N + x] : make_float2(0.f, 0.f);
    }
    double E = 0.0;
    float beta = 0.f;
    uint32_t cid = 0;
    unsigned long long acc = 0, att = 0;
    if (leader && c < gr.count) {
        const int slot = gr.chain0 + c;
        const int r = (slot - sd.chain0) / p.nT, t = p.label[slot];
        E = p.E[slot];
        beta = (float)p.beta[t];
        cid = (uint32_t)((gr.sample * p.R + r) * p.nT + t);
    }
    const int cap = 2 * p.max_deg;
    const GraphSmem lay = graph_smem(p.maxN, kStageV ? cap : 0);
    unsigned char *sbase = reinterpret_cast<unsigned char *>(ga);
    int *inc_off_s = reinterpret_cast<int *>(sbase + lay.inc);
    int4 *rec_s = reinterpret_cast<int4 *>(sbase + lay.rec);
    float *recJ_s = reinterpret_cast<float *>(sbase + lay.J);
    if (kFewV || kStageV)
        for (int i = tid; i <= N; i += kGThreads) inc_off_s[i] = p.inc_off[sd.mode_off + i];
    const int *inc_off = (kFewV || kStageV) ? inc_off_s : p.inc_off + sd.mode_off;
    const int4 *rec = p.rec + sd.inc_off;
    const float *recJ = p.recJ + sd.inc_off;
    const float cc_f = (float)p.cc;
    const long long base = p.ctl->sweep_base;
    // update trace: absolute sweep + 1 and update to record (0 = none)
    const long long tr_at = p.trace ? p.ctl->trace_at : 0ll;
    const int tr_u = p.trace ? p.ctl->trace_update : -1;
    __syncthreads();
    // kFew: the pair of the next update and this worker's record of it
    int jn = 0, kn = 0;
    int4 R4n = make_int4(0, 0, 0, 0);
    float Jn = 0.f;
    auto prefetch = [&](uint32_t sweep, uint32_t u) {
        pair_jk(p.seed, (uint32_t)gr.sample, sweep, u, N, jn, kn);
        const int oj = inc_off[jn], nj = inc_off[jn + 1] - oj, ok = inc_off[kn], nk = inc_off[kn + 1] - ok;
        if (worker < nj + nk) {
            const int r = worker < nj ? oj + worker : ok + worker - nj;
            R4n = __ldg(rec + r);
            Jn = __ldg(recJ + r);
        }
    };
    if (kFewV && p.n_sweeps > 0) prefetch((uint32_t)base, 0u);
    for (int sw = 0; sw < p.n_sweeps; ++sw) {
        const uint32_t sweep = (uint32_t)(base + sw);
        for (int u = 0; u < N / 2; ++u) {
            int j, k;
            int4 R4f;
            float Jf;
            if (kFewV) {
                j = jn; k = kn; R4f = R4n; Jf = Jn;
            } else {
                pair_jk(p.seed, (uint32_t)gr.sample, sweep, (uint32_t)u, N, j, k);
            }
            if (kStageV) {  // the update's records into shared memory (the previous update's reads are done)
                const int oj = inc_off[j], nj = inc_off[j + 1] - oj, ok = inc_off[k], nk = inc_off[k + 1] - ok;
                for (int i = tid; i < nj + nk; i += kGThreads) {
                    const int r = i < nj ? oj + i : ok + i - nj;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(rec_s + i)), "l"(rec + r)
                                 : "memory");
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(recJ_s + i)), "l"(recJ + r)
                                 : "memory");
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
            }
            if (leader) prop[c] = graph_proposal(p.seed, cid, sweep, (uint32_t)u, ga[j * kGRS + c], ga[k * kGRS + c]);
            if (kFewV) {
                if (u + 1 < N / 2) prefetch(sweep, (uint32_t)(u + 1));
                else if (sw + 1 < p.n_sweeps) prefetch(sweep + 1u, 0u);
            }
            if (kStageV) asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
            const GraphProposal P = prop[c];
            float2 hj = make_float2(0.f, 0.f), hk = make_float2(0.f, 0.f);
            float cr = 0.f;
            const int oj = inc_off[j], nj = inc_off[j + 1] - oj;
            const int ok = inc_off[k], nk = inc_off[k + 1] - ok;
            // one record of mode j (onj) or k: its field term, and for a quadruplet holding both (counted once,
            // from j's list) k's term and the cross term
            auto term = [&](const int4 R4, const float J, const bool onj) {
                const int pos = R4.w & 3;              // position of the record's own mode (j or k)
                const int otherR = (onj ? k : j) * kGRS;  // the other updated mode, possibly among the three
                const int o[3] = {R4.x, R4.y, R4.z};   // row offsets of A, B, C
                int po = -1;                           // index (0..2) of the other updated mode among them
#pragma unroll
                for (int m = 0; m < 3; ++m) if (o[m] == otherR) po = m;
                if (!onj && po >= 0) return;
                const float2 fa = ga[o[0] + c], fb = ga[o[1] + c], fc = ga[o[2] + c];
                // field of the record's mode: J a_A a_B conj(a_C)
                const float2 ab = cmulf(fa, fb);
                const float2 X = make_float2(J * (ab.x * fc.x + ab.y * fc.y), J * (ab.y * fc.x - ab.x * fc.y));
                if (onj) { hj.x += X.x; hj.y += X.y; } else { hk.x += X.x; hk.y += X.y; }
                if (onj && po >= 0) {
                    // the quadruplet holds j (this record) and k: k's field and the cross term, from the
                    // positions of the factors (conjugated at positions 0 and 3)
                    const int opos[3] = {(R4.w >> 2) & 3, (R4.w >> 4) & 3, (R4.w >> 6) & 3};
                    const float2 f[3] = {fac(fa, opos[0]), fac(fb, opos[1]), fac(fc, opos[2])};
                    const float2 own = fac(ga[j * kGRS + c], pos);
                    const int pk = opos[po];
                    float2 Y = make_float2(J * own.x, J * own.y), Z = make_float2(J, 0.f);
#pragma unroll
                    for (int m = 0; m < 3; ++m)
                        if (m != po) { Y = cmulf(Y, f[m]); Z = cmulf(Z, f[m]); }
                    if (pk == 1 || pk == 2) Y.y = -Y.y;
                    hk.x += Y.x; hk.y += Y.y;
                    const float2 dxj = (pos == 0 || pos == 3) ? make_float2(P.dj.x, -P.dj.y) : P.dj;
                    const float2 dxk = (pk == 0 || pk == 3) ? make_float2(P.dk.x, -P.dk.y) : P.dk;
                    cr += cmulf(Z, cmulf(dxj, dxk)).x;
                }
            };
            if (kFewV) {  // at most one record per worker, prefetched
                if (worker < nj + nk) term(R4f, Jf, worker < nj);
            } else {      // j's list, then k's (the list a record comes from is then known at compile time)
                for (int idx = worker; idx < nj; idx += kGWorkers)
                    term(kStageV ? rec_s[idx] : __ldg(rec + oj + idx), kStageV ? recJ_s[idx] : __ldg(recJ + oj + idx),
                         true);
                for (int idx = worker; idx < nk; idx += kGWorkers)
                    term(kStageV ? rec_s[nj + idx] : __ldg(rec + ok + idx),
                         kStageV ? recJ_s[nj + idx] : __ldg(recJ + ok + idx), false);
            }
            // reduce over the 4 workers of the warp, then over the warps in a fixed order
            float v[5] = {hj.x, hj.y, hk.x, hk.y, cr};
#pragma unroll
            for (int o = kGG; o < 32; o <<= 1)
#pragma unroll
                for (int e = 0; e < 5; ++e) v[e] += __shfl_xor_sync(0xffffffffu, v[e], o);
            if (lane < kGG) {
#pragma unroll
                for (int e = 0; e < 5; ++e) red[warp][c][e] = v[e];
            }
            __syncthreads();
            if (leader && c < gr.count) {
                float t[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
                // kFew: warps whose workers held no record contribute exact zeros; only the others are summed
                const int wmax = kFewV ? min(kGWarps, (nj + nk + (32 / kGG) - 1) / (32 / kGG)) : kGWarps;
                for (int w = 0; w < wmax; ++w)
#pragma unroll
                    for (int e = 0; e < 5; ++e) t[e] += red[w][c][e];
                // Re(conj(d) h) = d.x h.x + d.y h.y
                const float dH = -cc_f * (P.dj.x * t[0] + P.dj.y * t[1] + P.dk.x * t[2] + P.dk.y * t[3] + t[4]);
                ++att;
                const bool accept = dH <= 0.f || P.U < expf(-beta * dH);
                if (tr_at == base + sw + 1 && u == tr_u) {
                    // the record of this update and the chain's state before it (this leader is the only writer
                    // of its chain's column, so the table still holds the old a_j, a_k)
                    double *rec_o = p.trace + (int64_t)cid * kTraceRec;
                    const double v[kTraceRec] = {(double)j, (double)k, (double)t[0], (double)t[1], (double)t[2],
                                                 (double)t[3], (double)t[4], 0.0, 0.0, 0.0, (double)P.nj.x,
                                                 (double)P.nj.y, (double)P.nk.x, (double)P.nk.y, (double)P.U,
                                                 (double)dH, accept ? 1.0 : 0.0, (double)beta, E, 1.0};
                    for (int e = 0; e < kTraceRec; ++e) rec_o[e] = v[e];
                    double2 *st_o = reinterpret_cast<double2 *>(p.trace + (int64_t)p.n_chains * kTraceRec) + sd.a_off +
                                    (int64_t)(cid - (uint32_t)sd.chain0) * N;
                    for (int x = 0; x < N; ++x) {
                        const float2 a = ga[x * kGRS + c];
                        st_o[x] = make_double2((double)a.x, (double)a.y);
                    }
                }
                if (accept) {
                    ga[j * kGRS + c] = P.nj;
                    ga[k * kGRS + c] = P.nk;
                    E += (double)dH;
                    ++acc;
                }
            }
            // the leaders' amplitude writes are ordered before every read of the next update by the
            // barrier after its proposals
        }
        const long long done = base + sw + 1;
        if (p.measure_every > 0 && done % p.measure_every == 0 && sw + 1 < p.n_sweeps) {
            __syncthreads();
            const int kk = (int)(done / p.measure_every - base / p.measure_every - 1);
            if (kk >= 0 && kk < p.n_snap_max) {
                float2 *dst = p.snap_a + (int64_t)kk * p.a_total + sd.a_off + (int64_t)(gr.chain0 - sd.chain0) * N;
                for (int i = tid; i < N * gr.count; i += kGThreads) {
                    const int cc = i / N, x = i % N;
                    dst[(int64_t)cc * N + x] = ga[x * kGRS + cc];
                }
                if (leader && c < gr.count) p.snap_E[(int64_t)kk * p.n_chains + gr.chain0 + c] = E;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int i = tid; i < N * gr.count; i += kGThreads) {
        const int cc = i / N, x = i % N;
        A[(int64_t)cc * N + x] = ga[x * kGRS + cc];
    }
    if (leader && c < gr.count) {
        const int slot = gr.chain0 + c;
        if (!isfinite(E)) record_error(p.ctl, kErrNaN, 30);
        p.E[slot] = E;
        p.mc_acc[slot] += acc;
        p.mc_att[slot] += att;
    }
}

// Full energies of the chains of a group (optionally after rescaling to sum |a|^4 = N): each lane sums
// J_q Re(conj(a_q0) a_q1 a_q2 conj(a_q3)) for its chain over a share of the quadruplets, products in FP32,
// couplings and sums in FP64.
__global__ void __launch_bounds__(kGThreads) graph_energy_kernel(GraphParams p) {
    extern __shared__ float2 ga[];
    __shared__ double redd[kGWarps][kGG];
    __shared__ double s_f[kGG];
    const GroupDev gr = p.groups[blockIdx.x];
    const SampleDev sd = p.samples[gr.sample];
    const int N = sd.N, tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int c = lane % kGG, worker = warp * (32 / kGG) + lane / kGG;
    float2 *A = p.a + sd.a_off + (int64_t)(gr.chain0 - sd.chain0) * N;
    for (int i = tid; i < N * kGG; i += kGThreads) {
        const int x = i / kGG, cc = i % kGG;
        ga[x * kGRS + cc] = cc < gr.count ? A[(int64_t)cc * N + x] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (p.renorm) {
        double s4 = 0.0;
        for (int x = worker; x < N; x += kGWorkers) {
            const float2 v = ga[x * kGRS + c];
            const double uu = (double)v.x * v.x + (double)v.y * v.y;
            s4 += uu * uu;
        }
        for (int o = kGG; o < 32; o <<= 1) s4 += __shfl_xor_sync(0xffffffffu, s4, o);
        if (lane < kGG) redd[warp][c] = s4;
        __syncthreads();
        if (tid < kGG) {
            double t = 0.0;
            for (int w = 0; w < kGWarps; ++w) t += redd[w][tid];
            if (tid < gr.count && (!(t > 0.0) || !isfinite(t))) record_error(p.ctl, kErrNaN, 31);
            s_f[tid] = tid < gr.count ? sqrt(sqrt((double)N / t)) : 1.0;
        }
        __syncthreads();
        for (int i = tid; i < N * gr.count; i += kGThreads) {
            const int cc = i / N, x = i % N;
            const double f = s_f[cc];
            float2 v = ga[x * kGRS + cc];
            v = make_float2((float)((double)v.x * f), (float)((double)v.y * f));
            ga[x * kGRS + cc] = v;
            A[(int64_t)cc * N + x] = v;
        }
        __syncthreads();
    }
    const int4 *quads = p.quads + sd.q_off;
    const double *Jd = p.Jd + sd.q_off;
    double acc = 0.0;
    for (int64_t q = worker; q < sd.nq; q += kGWorkers) {
        const int4 Q = __ldg(quads + q);
        const float2 t = cmulf(cmulf(fac(ga[Q.x * kGRS + c], 0), ga[Q.y * kGRS + c]),
                               cmulf(ga[Q.z * kGRS + c], fac(ga[Q.w * kGRS + c], 3)));
        acc += __ldg(Jd + q) * (double)t.x;
    }
    for (int o = kGG; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane < kGG) redd[warp][c] = acc;
    __syncthreads();
    if (tid < gr.count) {
        double t = 0.0;
        for (int w = 0; w < kGWarps; ++w) t += redd[w][tid];
        const double Ec = -p.cc * t;
        const int slot = gr.chain0 + tid;
        if (!isfinite(Ec)) record_error(p.ctl, kErrNaN, 32);
        if (p.E_state) p.E_state[slot] = Ec;
        if (p.E_out) p.E_out[slot] = Ec;
    }
}

namespace {
constexpr size_t kGraphSmemMax = 227 * 1024 - 8 * 1024;  // dynamic part (the static reduction table aside)

int graph_variant(int maxN, int max_deg) {
    if (2 * max_deg <= kGWorkers) return kFew;
    if (graph_smem(maxN, 2 * max_deg).total <= kGraphSmemMax) return kStage;
    return kPlain;
}
}  // namespace

cudaError_t graph_prepare(int maxN, int max_deg) {
    const int var = graph_variant(maxN, max_deg);
    const int sm = (int)graph_smem(maxN, var == kStage ? 2 * max_deg : 0).total;
    cudaError_t e = cudaSuccess;
    if (var == kFew) e = cudaFuncSetAttribute(graph_sweep_kernel<kFew>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    else if (var == kStage)
        e = cudaFuncSetAttribute(graph_sweep_kernel<kStage>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    else e = cudaFuncSetAttribute(graph_sweep_kernel<kPlain>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    const int se = maxN * kGRS * (int)sizeof(float2);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(graph_energy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, se);
    return e;
}

cudaError_t launch_graph_sweep(const GraphParams &p, int n_groups, cudaStream_t s) {
    if (n_groups <= 0) return cudaSuccess;
    const int var = graph_variant(p.maxN, p.max_deg);
    const size_t sm = graph_smem(p.maxN, var == kStage ? 2 * p.max_deg : 0).total;
    if (var == kFew) graph_sweep_kernel<kFew><<<n_groups, kGThreads, sm, s>>>(p);
    else if (var == kStage) graph_sweep_kernel<kStage><<<n_groups, kGThreads, sm, s>>>(p);
    else graph_sweep_kernel<kPlain><<<n_groups, kGThreads, sm, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_graph_energy(const GraphParams &p, int n_groups, cudaStream_t s) {
    if (n_groups <= 0) return cudaSuccess;
    const size_t sm = (size_t)p.maxN * kGRS * sizeof(float2);
    graph_energy_kernel<<<n_groups, kGThreads, sm, s>>>(p);
    return cudaGetLastError();
}

}  // namespace ptgb
