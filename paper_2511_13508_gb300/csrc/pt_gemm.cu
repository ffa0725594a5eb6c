// pt_gemm.cu -- batched BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores (tcgen05, TMEM)
// for the learned global-move proposal's network (the paper has no counterpart; the proposal serves
// the Parallel-Tempering path of arXiv 2511.13508).
//
//   D[b] (M x N, FP32) = A[b] (M x K, BF16, row-major = K-major) * B[b]^T (B: N x K, BF16, K-major)
//
// One thread block computes a 128 x 64 tile with the accumulator in tensor memory: the
// operands are staged by asynchronous copies (cp.async, zero-filled outside the matrix) in shared memory
// in the canonical K-major no-swizzle layout (8 x 16-byte core matrices), two stages of K = 128 so that the
// copies of the next chunk overlap the MMAs of this one; one elected thread issues tcgen05.mma (M = 128,
// N = 64, K = 16 per instruction) and commits to the stage's mbarrier; four warps read the accumulator back
// with tcgen05.ld (warp w owns lanes 32w..32w+31) and transpose it through shared memory so that every
// global store of the epilogue is coalesced.
#include <algorithm>
#include <cstdint>
#include <cuda_bf16.h>
#include "pt_common.cuh"
#include "pt_gemm.h"

namespace ptgb {

namespace {

constexpr int kGemmM = 128;   // rows per thread block (= TMEM lanes)
constexpr int kGemmKC = 128;  // K per pipeline stage (8 MMAs of K = 16)
constexpr int kGemmNT = 64;   // output columns per thread block (the MMA's N); two stages of 48 KB

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, K-major, no swizzle: start address, leading-dimension byte offset
// (between core matrices adjacent in K), stride-dimension byte offset (between 8-row groups), version 1.
__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3fffu);
    d |= (uint64_t)((lbo >> 4) & 0x3fffu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3fffu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for sm_100-class tensor cores
    return d;                 // base offset 0, layout type 0 = no swizzle
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N.
__device__ __forceinline__ uint32_t make_idesc(int N) {
    uint32_t d = 0;
    d |= 1u << 4;                          // D format F32
    d |= 1u << 7;                          // A format BF16
    d |= 1u << 10;                         // B format BF16
    d |= (uint32_t)(N >> 3) << 17;         // N / 8
    d |= (uint32_t)(kGemmM >> 4) << 24;    // M / 16
    return d;
}

__device__ __forceinline__ void mbar_init1(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Issues the asynchronous copies of rows [r0, r0+rows) x K-chunk [k0, k0+KC) of a row-major BF16 matrix
// (leading dimension ld, valid rows < nrows, valid columns < K) into the canonical layout: element (r, k)
// at (k / 8) * lbo + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2 bytes.  Out-of-range parts are zero-filled.
// Lane l of a warp takes K-group (l & 1) of row (l >> 1): 32 contiguous bytes of one row per lane pair.
__device__ __forceinline__ void stage_async(uint32_t dst, const __nv_bfloat16 *src, int ld, int r0, int rows,
                                           int nrows, int k0, int K, uint32_t lbo) {
    constexpr int kGroups = kGemmKC / 8;
    const int pieces = rows * kGroups;
    for (int p = threadIdx.x; p < pieces; p += blockDim.x) {
        // p -> (row, K-group): bit 0 = low bit of the group, bits 1..4 = row within 16, then the rest
        const int kg = ((p >> 5) % (kGroups / 2)) * 2 + (p & 1);
        const int r = (p >> 5) / (kGroups / 2) * 16 + ((p >> 1) & 15);
        const int gr = r0 + r, gk = k0 + kg * 8;
        const bool ok = gr < nrows && gk < K;
        const __nv_bfloat16 *g = ok ? src + (int64_t)gr * ld + gk : src;
        const uint32_t d = dst + kg * lbo + (r / 8) * 128 + (r % 8) * 16;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(g), "r"(ok ? 16 : 0) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Bounded wait on an mbarrier phase; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity))
        if (global_ns() - t0 > kWaitNs) return false;
    return true;
}

}  // namespace

// Two-stage pipeline: the copies of chunk c+1 are in flight while the tensor cores work on chunk c.
__global__ void __launch_bounds__(128, 2) gemm_bf16_tc_kernel(GemmParams p) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_base_slot;
    const int b = blockIdx.z, m0 = blockIdx.x * kGemmM, n0 = blockIdx.y * kGemmNT;
    const int N = p.N, K = p.K, NT = min(kGemmNT, N - n0);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    constexpr uint32_t kStageA = kGemmM * kGemmKC * 2, kStage = kStageA + kGemmNT * kGemmKC * 2;
    const uint32_t s0 = smem_addr(gsm);
    const uint32_t lboA = (kGemmM / 8) * 128, lboB = (uint32_t)(NT / 8) * 128;
    const __nv_bfloat16 *A = p.A + (int64_t)b * p.strideA;
    const __nv_bfloat16 *Bm = p.B + (int64_t)b * p.strideB + (int64_t)n0 * p.ldb;  // rows n0 .. n0+NT of B

    // tensor-memory accumulator: 64 columns x 128 lanes of FP32
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_addr(&tmem_base_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) { mbar_init1(&mbar[0]); mbar_init1(&mbar[1]); }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_slot;
    const uint32_t idesc = make_idesc(NT);
    uint32_t phase[2] = {0u, 0u};
    bool pend[2] = {false, false};  // a commit on the stage's barrier not yet waited for
    bool ok = true;
    const int nchunks = (K + kGemmKC - 1) / kGemmKC;

    stage_async(s0, A, p.lda, m0, kGemmM, p.M, 0, K, lboA);
    stage_async(s0 + kStageA, Bm, p.ldb, 0, NT, NT, 0, K, lboB);
    for (int c = 0; c < nchunks && ok; ++c) {
        const int st = c & 1;
        if (c + 1 < nchunks) {
            const int nx = (c + 1) & 1;
            if (c >= 1) {  // the other stage was read by chunk c-1's MMAs
                ok = mbar_wait(&mbar[nx], phase[nx]);
                phase[nx] ^= 1u;
                pend[nx] = false;
                if (!ok) break;
            }
            const uint32_t base = s0 + nx * kStage;
            stage_async(base, A, p.lda, m0, kGemmM, p.M, (c + 1) * kGemmKC, K, lboA);
            stage_async(base + kStageA, Bm, p.ldb, 0, NT, NT, (c + 1) * kGemmKC, K, lboB);
            asm volatile("cp.async.wait_group 2;" ::: "memory");  // chunk c's two groups have landed
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> tensor core reads
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = s0 + st * kStage, sb = sa + kStageA;
            const int k0 = c * kGemmKC;
            const int ksteps = (min(kGemmKC, K - k0) + 15) / 16;
            for (int t = 0; t < ksteps; ++t) {
                const uint64_t da = make_sdesc(sa + t * 2 * lboA, lboA, 128);
                const uint64_t db = make_sdesc(sb + t * 2 * lboB, lboB, 128);
                const uint32_t acc = (c > 0 || t > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred pacc;\n\tsetp.ne.b32 pacc, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pacc;\n\t}" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&mbar[st]))
                         : "memory");
        }
        pend[st] = true;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // drain every outstanding commit (bounded), so no MMA or barrier arrival outlives the block
    for (int st = 0; st < 2; ++st)
        if (pend[st] && !mbar_wait(&mbar[st], phase[st])) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (!ok) {
        if (threadIdx.x == 0 && p.err) atomicCAS(p.err, 0, kErrTimeout);
    } else {
        // epilogue.  Phase 1 (lane = row): warp w reads TMEM lanes 32w..32w+31, 32 columns at a time, applies
        // bias / conditional bias / gate, writes the transposed BF16 copy (coalesced along rows) and parks the
        // values in a 32 x 33 shared tile.  Phase 2 (lane = column): row-major FP32 and BF16 stores, coalesced.
        float *tile = reinterpret_cast<float *>(gsm) + warp * (32 * 33);
        const int row = m0 + warp * 32 + lane;
        const bool relu = p.mode == kEpiRelu;
        for (int c0 = 0; c0 < NT; c0 += 32) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const bool live = row < p.M;
            const float *cb = (p.cbias && live)
                                  ? p.cbias + (int64_t)b * p.strideCbias + (int64_t)p.cond[(int64_t)b * p.strideCond + row] * N
                                  : nullptr;
            const float *gt = (p.mode == kEpiGate && live)
                                  ? p.gate + (int64_t)b * p.strideGate + (int64_t)row * p.ldgate : nullptr;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int col = n0 + c0 + q;
                float v = __uint_as_float(r[q]);
                if (p.mode == kEpiGate) {
                    v = (gt && col < N && gt[col] > 0.f) ? v : 0.f;
                } else {
                    if (p.bias && col < N) v += p.bias[(int64_t)b * p.strideBias + col];
                    if (cb && col < N) v += cb[col];
                }
                tile[lane * 33 + q] = v;
                if (p.HT && live && col < N)
                    p.HT[(int64_t)b * p.strideHT + (int64_t)col * p.ldht + row] = __float2bfloat16_rn(relu ? fmaxf(v, 0.f) : v);
            }
            __syncwarp();
            const int col = n0 + c0 + lane;
            for (int rr = 0; rr < 32; ++rr) {
                const int row2 = m0 + warp * 32 + rr;
                if (row2 >= p.M || col >= N) continue;
                const float v = tile[rr * 33 + lane];
                if (p.D) p.D[(int64_t)b * p.strideD + (int64_t)row2 * p.ldd + col] = v;
                if (p.H) p.H[(int64_t)b * p.strideH + (int64_t)row2 * p.ldh + col] = __float2bfloat16_rn(relu ? fmaxf(v, 0.f) : v);
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------------------------------------------
// Fused forward pass of the proposal network (see MlpParams), one thread block per sample.
//  - Weights arrive pre-arranged in the canonical K-major layout ([K/8][N][8] BF16, written by the cast
//    kernel), so one K-chunk of 64 (8 K-groups x N rows, up to 32 KB) is one contiguous bulk copy into a ring of
//    weight stages.  One thread issues the copies and the MMAs of all three layers in order; the copies of
//    later chunks (also of the next layers) stay in flight while the tensor cores consume earlier ones.
//  - Activations (input, H1, H2) live in shared memory in the canonical layout with a K-group stride of
//    Mp x 16 bytes (Mp = rows rounded up to 16).  The MMA always reads 128 rows; rows >= Mp read whatever
//    follows (each buffer is padded so that this stays inside the block's shared memory) and only produce
//    accumulator lanes that nobody reads.
//  - The accumulator of each layer occupies the same 256 TMEM columns; 16 warps read it back (warp w: TMEM
//    lanes 32 (w % 4) .., columns split four ways), add the biases, apply the ReLU and write the next layer's
//    BF16 input, or the FP32 outputs.
namespace {

constexpr int kMlpThreads = 512;
constexpr int kMlpKC = 64;                          // K per chunk (8 K-groups)
constexpr uint32_t kMlpStage = 256 * kMlpKC * 2;   // largest chunk: 256 rows x 64 K
constexpr int kMlpMaxStages = 6;
constexpr uint32_t kMlpPad = 2048;                 // rows Mp..127 of the last K-group

// rows [0, rows) (rows % 16 == 0) x K-groups [g0, g0 + groups) (groups even) of a row-major BF16 matrix into
// the canonical layout at dst; rows >= nrows are zero-filled
__device__ __forceinline__ void stage_rows(uint32_t dst, const __nv_bfloat16 *src, int ld, int rows, int nrows,
                                          int g0, int groups, uint32_t lbo) {
    const int pieces = rows * groups, half = groups / 2;
    for (int p = threadIdx.x; p < pieces; p += blockDim.x) {
        const int kg = ((p >> 5) % half) * 2 + (p & 1);
        const int r = (p >> 5) / half * 16 + ((p >> 1) & 15);
        const bool ok = r < nrows;
        const __nv_bfloat16 *g = ok ? src + (int64_t)r * ld + (int64_t)(g0 + kg) * 8 : src;
        const uint32_t d = dst + kg * lbo + (r / 8) * 128 + (r % 8) * 16;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(g), "r"(ok ? 16 : 0) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t r[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The chunk sequence of the three layers: layer l has ceil(K_l / 64) chunks of W_l (N_l rows).
struct MlpChunks {
    const unsigned char *W[3];
    int N[3], K[3], first[3], total;
    __device__ int layer_of(int g) const { return g >= first[2] ? 2 : (g >= first[1] ? 1 : 0); }
    __device__ uint32_t bytes(int g, int *groups) const {
        const int l = layer_of(g), c = g - first[l];
        *groups = min(kMlpKC, K[l] - c * kMlpKC) / 8;
        return (uint32_t)(*groups) * (uint32_t)N[l] * 16u;
    }
    __device__ const unsigned char *src(int g) const {
        const int l = layer_of(g), c = g - first[l];
        return W[l] + (size_t)c * 8 * N[l] * 16;
    }
};

// Epilogue of a hidden layer: relu(acc + bias (+ cbias[cond[row]])) as BF16 into the activation buffer.
__device__ void mlp_hidden_epilogue(uint32_t tmem, unsigned char *dst, uint32_t lboA, int Mp, int N, int M,
                                    const float *bias, const float *cbias, const int *cond) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, quad = warp % 4, part = warp / 4;
    const int row = quad * 32 + lane;
    if (quad * 32 >= Mp) return;  // the whole warp's rows are padding
    const bool live = row < M;
    const float *cb = (cbias && live) ? cbias + (int64_t)cond[row] * N : nullptr;
    const int span = N / 4;  // columns of this warp: [part * span, (part + 1) * span), span a multiple of 8
    for (int c0 = part * span; c0 < (part + 1) * span; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, r);
        const int ncol = min(32, (part + 1) * span - c0);
        if (row < Mp) {
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                if (8 * g >= ncol) break;
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float v0 = 0.f, v1 = 0.f;
                    if (live) {
                        const int k0 = c0 + 8 * g + 2 * e;
                        v0 = __uint_as_float(r[8 * g + 2 * e]) + bias[k0];
                        v1 = __uint_as_float(r[8 * g + 2 * e + 1]) + bias[k0 + 1];
                        if (cb) { v0 += cb[k0]; v1 += cb[k0 + 1]; }
                        v0 = fmaxf(v0, 0.f);
                        v1 = fmaxf(v1, 0.f);
                    }
                    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                    w[e] = *reinterpret_cast<const uint32_t *>(&h);
                }
                *reinterpret_cast<uint4 *>(dst + (uint32_t)((c0 + 8 * g) / 8) * lboA + (uint32_t)row * 16) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
}

}  // namespace

__global__ void __launch_bounds__(kMlpThreads, 1) fused_mlp_kernel(MlpParams p, int n_stages) {
    extern __shared__ __align__(1024) unsigned char msm[];
    __shared__ uint64_t full[kMlpMaxStages], empty[kMlpMaxStages], done;
    __shared__ uint32_t tmem_base_slot;
    const int b = blockIdx.x, warp = threadIdx.x / 32;
    const int Mp = (p.M + 15) & ~15;
    const uint32_t lboA = (uint32_t)Mp * 16u;
    const uint32_t act_bytes = 32u * lboA + kMlpPad;  // 256 columns
    unsigned char *act0 = msm, *act1 = msm + act_bytes;
    const uint32_t sAct0 = smem_addr(act0), sAct1 = smem_addr(act1), sW = smem_addr(msm + 2 * act_bytes);
    MlpChunks ch;
    ch.W[0] = reinterpret_cast<const unsigned char *>(p.W1c + (int64_t)b * p.strideW1);
    ch.W[1] = reinterpret_cast<const unsigned char *>(p.W2c + (int64_t)b * p.strideW2);
    ch.W[2] = reinterpret_cast<const unsigned char *>(p.W3c + (int64_t)b * p.strideW3);
    ch.N[0] = p.H; ch.N[1] = p.H; ch.N[2] = p.Dout;
    ch.K[0] = p.Din; ch.K[1] = p.H; ch.K[2] = p.H;
    ch.first[0] = 0;
    ch.first[1] = (p.Din + kMlpKC - 1) / kMlpKC;
    ch.first[2] = ch.first[1] + (p.H + kMlpKC - 1) / kMlpKC;
    ch.total = ch.first[2] + (p.H + kMlpKC - 1) / kMlpKC;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_addr(&tmem_base_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < n_stages; ++i) { mbar_init1(&full[i]); mbar_init1(&empty[i]); }
        mbar_init1(&done);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // the first chunks of the weights, then the input rows (rows M..Mp-1 zero)
    if (threadIdx.x == 0)
        for (int g = 0; g < min(n_stages, ch.total); ++g) {
            int groups;
            const uint32_t nb = ch.bytes(g, &groups);
            mbar_expect_tx(&full[g], nb);
            bulk_g2s(sW + g * kMlpStage, ch.src(g), nb, &full[g]);
        }
    stage_rows(sAct0, p.X + (int64_t)b * p.strideX, p.ldx, Mp, p.M, 0, p.Din / 8, lboA);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_slot;
    const float *P = p.P + (int64_t)b * p.psize;
    const int *cond = p.cond + (int64_t)b * p.strideCond;
    bool ok = true;
    int issued = min(n_stages, ch.total);
    for (int l = 0; l < 3; ++l) {
        const uint32_t abuf = (l == 1) ? sAct1 : sAct0;  // x -> H1 (act1) -> H2 (act0)
        if (threadIdx.x == 0) {
            const uint32_t idesc = make_idesc(ch.N[l]);
            const uint32_t lboB = (uint32_t)ch.N[l] * 16u;
            for (int g = ch.first[l]; g < (l < 2 ? ch.first[l + 1] : ch.total) && ok; ++g) {
                const int st = g % n_stages;
                if (!mbar_wait(&full[st], (uint32_t)(g / n_stages) & 1u)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                int groups;
                ch.bytes(g, &groups);
                const int c = g - ch.first[l];
                for (int t = 0; t < groups / 2; ++t) {
                    const uint64_t da = make_sdesc(abuf + (uint32_t)(c * 8 + 2 * t) * lboA, lboA, 128);
                    const uint64_t db = make_sdesc(sW + st * kMlpStage + 2 * t * lboB, lboB, 128);
                    const uint32_t acc = (c > 0 || t > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred pacc;\n\tsetp.ne.b32 pacc, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pacc;\n\t}" ::"r"(tmem),
                        "l"(da), "l"(db), "r"(idesc), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_addr(&empty[st]))
                             : "memory");
                // refill the stage of the previous chunk once its MMAs are done
                if (g >= 1 && issued < ch.total) {
                    const int gp = g - 1, sp = gp % n_stages;
                    if (!mbar_wait(&empty[sp], (uint32_t)(gp / n_stages) & 1u)) { ok = false; break; }
                    int gr;
                    const uint32_t nb = ch.bytes(issued, &gr);
                    mbar_expect_tx(&full[sp], nb);
                    bulk_g2s(sW + sp * kMlpStage, ch.src(issued), nb, &full[sp]);
                    ++issued;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&done))
                         : "memory");
        }
        __syncwarp();
        if (!mbar_wait(&done, (uint32_t)l & 1u)) ok = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        ok = __syncthreads_and(ok ? 1 : 0) != 0;
        if (!ok) break;
        if (l < 2) {
            mlp_hidden_epilogue(tmem, l == 0 ? act1 : act0, lboA, Mp, p.H, p.M, P + (l == 0 ? p.ob1 : p.ob2),
                                l == 0 ? P + p.oC1 : nullptr, l == 0 ? cond : nullptr);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core reads
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        } else {
            const int lane = threadIdx.x % 32, quad = warp % 4, part = warp / 4;
            const int row = quad * 32 + lane, span = p.Dout / 4;
            if (quad * 32 < Mp) {
                const float *b3 = P + p.ob3;
                for (int c0 = part * span; c0 < (part + 1) * span; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, r);
                    const int ncol = min(32, (part + 1) * span - c0);
                    if (row < p.M) {
                        float *o = p.O + (int64_t)b * p.strideO + (int64_t)row * p.ldo + c0;
#pragma unroll
                        for (int q = 0; q < 32; q += 4)
                            if (q < ncol)
                                *reinterpret_cast<float4 *>(o + q) = make_float4(
                                    __uint_as_float(r[q]) + b3[c0 + q], __uint_as_float(r[q + 1]) + b3[c0 + q + 1],
                                    __uint_as_float(r[q + 2]) + b3[c0 + q + 2], __uint_as_float(r[q + 3]) + b3[c0 + q + 3]);
                    }
                }
            }
        }
    }
    if (!ok && threadIdx.x == 0) {
        if (p.err) atomicCAS(p.err, 0, kErrTimeout);
        // let the bulk copies still in flight land before the block's shared memory is released
        for (int g = 0; g < issued; ++g) (void)mbar_wait(&full[g % n_stages], (uint32_t)(g / n_stages) & 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

cudaError_t launch_fused_mlp(const MlpParams &p, int batch, cudaStream_t s) {
    // M <= 128 rows, Din a multiple of 16 (<= 256), H = 256, Dout a multiple of 32 (<= 256), 16-byte aligned
    // canonical weights, O rows 16-byte aligned
    if (p.M < 1 || p.M > 128 || p.Din < 16 || p.Din > 256 || (p.Din % 16) || p.H != 256 || p.Dout < 32 ||
        p.Dout > 256 || (p.Dout % 32) || (p.ldo % 4) || batch < 1 || !p.W1c || !p.W2c || !p.W3c ||
        ((uintptr_t)p.W1c | (uintptr_t)p.W2c | (uintptr_t)p.W3c) % 16 ||
        ((p.strideW1 | p.strideW2 | p.strideW3) * 2) % 16)
        return cudaErrorInvalidValue;
    constexpr size_t kSmemMax = 227 * 1024 - 1024;  // minus the static part
    const int Mp = (p.M + 15) & ~15;
    const size_t act = 2 * (32 * (size_t)Mp * 16 + kMlpPad);
    const int n_stages = (int)std::min<size_t>(kMlpMaxStages, (kSmemMax - act) / kMlpStage);
    if (n_stages < 2) return cudaErrorInvalidValue;
    const size_t sm = act + (size_t)n_stages * kMlpStage;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(fused_mlp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    fused_mlp_kernel<<<batch, kMlpThreads, sm, s>>>(p, n_stages);
    return cudaGetLastError();
}

cudaError_t launch_gemm_bf16(const GemmParams &p, int batch, cudaStream_t s) {
    if (p.N < 16 || p.N > 256 || (p.N % 16) || p.K < 16 || (p.K % 8) || p.M < 1 || batch < 1)
        return cudaErrorInvalidValue;
    constexpr size_t sm = 2 * ((size_t)kGemmM * kGemmKC * 2 + (size_t)kGemmNT * kGemmKC * 2);
    static bool attr_set = false;  // per process; the attribute is a property of the function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((p.M + kGemmM - 1) / kGemmM, (p.N + kGemmNT - 1) / kGemmNT, batch);
    gemm_bf16_tc_kernel<<<grid, 128, sm, s>>>(p);
    return cudaGetLastError();
}

}  // namespace ptgb

// ------------------------------------------------------------------------------------------------
// C ABI: plain batched D = A B^T (see include/pt.h)
#include "../../include/pt.h"
namespace ptgb { void set_global_error(const char *msg); }

extern "C" int pt_gemm_bf16(int batch, int M, int N, int K, const void *A, const void *B, float *D, void *stream) {
    if (batch < 1 || M < 1 || N < 16 || N > 256 || (N % 16) || K < 16 || (K % 8) || !A || !B || !D) {
        ptgb::set_global_error("pt_gemm_bf16: need batch, M >= 1, 16 <= N <= 256 with N % 16 == 0, K >= 16 with K % 8 == 0");
        return PT_EINVAL;
    }
    ptgb::GemmParams p{};
    p.A = reinterpret_cast<const __nv_bfloat16 *>(A);
    p.B = reinterpret_cast<const __nv_bfloat16 *>(B);
    p.strideA = (int64_t)M * K; p.strideB = (int64_t)N * K;
    p.lda = K; p.ldb = K; p.M = M; p.N = N; p.K = K; p.mode = ptgb::kEpiF32;
    p.D = D; p.strideD = (int64_t)M * N; p.ldd = N;
    const cudaError_t e = ptgb::launch_gemm_bf16(p, batch, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        ptgb::set_global_error(cudaGetErrorString(e));
        return PT_ECUDA;
    }
    return PT_OK;
}
