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
#include "pt_learn.h"
#include "pt_learn_dev.cuh"

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
// Fused forward pass of the proposal network (see MlpParams): a cluster of kMlpCL thread blocks per sample,
// block r computing output columns [r N/kMlpCL, (r+1) N/kMlpCL) of every layer.
//  - Weights arrive in the sliced canonical layout (written by the cast kernel): block r's rows of a layer
//    are one contiguous run, loaded by a single bulk copy.  All three slices (at most 96 KB) are requested
//    at the start, so the copies overlap the input staging and the earlier layers.
//  - Activations (input, H1, H2) are held whole (all 256 K columns, Mp = rows rounded up to 16) in every
//    block, in the canonical layout with a K-group stride of Mp x 16 bytes.  The MMA reads 128 rows; rows
//    >= Mp read whatever follows (each buffer is padded so that this stays inside the block's shared memory)
//    and only produce accumulator lanes nobody reads.
//  - After a hidden layer each block writes its BF16 column slice of relu(acc + b (+ C1[cond])) into its own
//    next activation buffer (the slice is 8 contiguous K-groups) and one thread sends it to the three peers
//    with shared-to-shared bulk copies that complete on the peer's exchange mbarrier; a block starts the next
//    layer once its barrier has counted the three slices.
//  - 8 warps read the accumulator back: warp w takes TMEM lanes 32 (w % 4).. and half of the slice's columns.
//  - Biases and the C1 columns of the block are staged in shared memory at the start.
namespace {

constexpr int kMlpCL = 4;         // blocks per sample (cluster size)
constexpr int kMlpThreads = 256;
constexpr uint32_t kMlpPad = 2048;  // rows Mp..127 of the last K-group

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

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Bulk copy of `bytes` from this block's shared memory at `local` to the same offset in block `rank` of the
// cluster, completing (complete_tx) on the mbarrier at the same offset as `bar` in that block.
__device__ __forceinline__ void bulk_s2peer(uint32_t local, uint32_t bytes, uint64_t *bar, uint32_t rank) {
    uint32_t dst, rbar;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(dst) : "r"(local), "r"(rank));
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rbar) : "r"(smem_addr(bar)), "r"(rank));
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "r"(local), "r"(bytes), "r"(rbar)
                 : "memory");
}

// 2 bytes to the same shared-memory offset in block `rank` of the cluster
__device__ __forceinline__ void st_cluster2(uint32_t local, uint32_t rank, uint16_t v) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
    asm volatile("st.shared::cluster.u16 [%0], %1;" ::"r"(remote), "h"(v) : "memory");
}

constexpr size_t kMlpSmemMax = 227 * 1024 - 2048;  // dynamic shared memory of a cluster block (static part aside)
constexpr int kMlpMaxCond = 64;                     // conditions whose C1 columns are staged in shared memory

// One layer's products: TMEM[0..NS) = act (128 x K) * Wslice^T, issued by one thread, completion on `done`.
__device__ __forceinline__ void mlp_mma(uint32_t tmem, uint32_t abuf, uint32_t lboA, uint32_t wbuf, int NS, int K,
                                       uint64_t *done) {
    const uint32_t idesc = make_idesc(NS), lboB = (uint32_t)NS * 16u;
    // the start address (bits 0-13, in 16-byte units) advances by two K-groups per step; shared-memory
    // addresses stay below 256 KB, so the field never carries
    const uint64_t da0 = make_sdesc(abuf, lboA, 128), db0 = make_sdesc(wbuf, lboB, 128);
    const uint64_t dda = (uint64_t)((2 * lboA) >> 4), ddb = (uint64_t)((2 * lboB) >> 4);
    for (int t = 0; t < K / 16; ++t) {
        const uint64_t da = da0 + (uint64_t)t * dda, db = db0 + (uint64_t)t * ddb;
        const uint32_t acc = t > 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred pacc;\n\tsetp.ne.b32 pacc, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pacc;\n\t}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(done))
                 : "memory");
}

}  // namespace

// With kSampler the block also runs the autoregressive sampling of the learned proposal (see SamplerParams):
// one pass of the network per mode block b = lo..7 with the weights resident in shared memory; after pass b
// the block holding block b's outputs draws its modes for the rows that resample it, writes the draws to
// global memory and their input features into the input buffer of every block of the cluster.
template <bool kSampler>
__global__ void __cluster_dims__(kMlpCL, 1, 1) __launch_bounds__(kMlpThreads, 1)
    mlp_cluster_kernel(MlpParams p, SamplerExtra sx) {
    extern __shared__ __align__(1024) unsigned char msm[];
    __shared__ uint64_t full[3], done, xchg[2];  // weights; MMA completion; H1 / H2 slices from the peers
    __shared__ uint32_t tmem_base_slot;
    __shared__ float bsl[3][64];  // this block's slices of b1, b2, b3
    const uint32_t rank = cluster_rank();
    const int b = blockIdx.x / kMlpCL, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int NS = p.H / kMlpCL, NS3 = p.Dout / kMlpCL;
    const int Mp = (p.M + 15) & ~15;
    const uint32_t lboA = (uint32_t)Mp * 16u;
    const uint32_t act_bytes = 32u * lboA + kMlpPad;  // 256 K columns
    const uint32_t x_bytes = kSampler ? (uint32_t)(p.Din / 8) * lboA + kMlpPad : 0u;
    // H2 | H1 | [X] | W1 | W2 | W3 slices; without the sampler the input shares the H2 buffer
    const uint32_t sH2 = smem_addr(msm), sH1 = sH2 + act_bytes, sX = kSampler ? sH1 + act_bytes : sH2;
    const uint32_t wbytes[3] = {(uint32_t)p.Din * NS * 2u, (uint32_t)p.H * NS * 2u, (uint32_t)p.H * NS3 * 2u};
    const uint32_t w0 = sH1 + act_bytes + x_bytes;
    const uint32_t sW[3] = {w0, w0 + wbytes[0], w0 + wbytes[0] + wbytes[1]};
    // after the weights: C1's columns of this block (if staged), then (sampler) the outputs of a mode block
    // [Mp][32] and the first resampled block of each row
    const bool stage_c1 = p.ncond <= kMlpMaxCond;
    float *c1s = reinterpret_cast<float *>(msm + (w0 - sH2) + wbytes[0] + wbytes[1] + wbytes[2]);
    float *obuf = c1s + (stage_c1 ? p.ncond * NS : 0);
    ModeNoise *noise = reinterpret_cast<ModeNoise *>(obuf + (kSampler ? Mp * 32 : 0));  // [M][2 N/8]
    int *fbs = reinterpret_cast<int *>(noise + (kSampler ? p.M * 2 * (sx.N / kLearnBlocks) : 0));
    const unsigned char *gW[3] = {
        reinterpret_cast<const unsigned char *>(p.W1c + (int64_t)b * p.strideW1) + (size_t)rank * wbytes[0],
        reinterpret_cast<const unsigned char *>(p.W2c + (int64_t)b * p.strideW2) + (size_t)rank * wbytes[1],
        reinterpret_cast<const unsigned char *>(p.W3c + (int64_t)b * p.strideW3) + (size_t)rank * wbytes[2]};
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_addr(&tmem_base_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int l = 0; l < 3; ++l) mbar_init1(&full[l]);
        mbar_init1(&done);
        mbar_init1(&xchg[0]);
        mbar_init1(&xchg[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int l = 0; l < 3; ++l) {
            mbar_expect_tx(&full[l], wbytes[l]);
            bulk_g2s(sW[l], gW[l], wbytes[l], &full[l]);
        }
    const float *P = p.P + (int64_t)b * p.psize;
    if (threadIdx.x < 64) {
        bsl[0][threadIdx.x] = P[p.ob1 + rank * NS + threadIdx.x];
        bsl[1][threadIdx.x] = P[p.ob2 + rank * NS + threadIdx.x];
        bsl[2][threadIdx.x] = threadIdx.x < NS3 ? P[p.ob3 + rank * NS3 + threadIdx.x] : 0.f;
    }
    if (kSampler) {
        const uint32_t rnd = (uint32_t)sx.ctl->global_rounds;
        for (int rw = threadIdx.x; rw < p.M; rw += blockDim.x)
            fbs[rw] = first_block(sx.seed, sx.row_id[(int64_t)b * p.M + rw], rnd, sx.N, sx.lo, sx.hi);
        // the state-independent part of the draws of this block's modes (mode blocks 2 rank and 2 rank + 1)
        const int per = sx.N / kLearnBlocks, nm = 2 * per;
        for (int i = threadIdx.x; i < p.M * nm; i += blockDim.x) {
            const int rw = i / nm, k = 2 * (int)rank * per + i % nm;
            noise[i] = mode_noise(draw(sx.seed, sx.row_id[(int64_t)b * p.M + rw], rnd, (uint32_t)k, kTagGlobal));
        }
    }
    if (stage_c1)  // this block's columns of C1, all conditions
        for (int i = threadIdx.x; i < p.ncond * NS; i += blockDim.x)
            c1s[i] = P[p.oC1 + (int64_t)(i / NS) * p.H + rank * NS + i % NS];
    stage_rows(sX, p.X + (int64_t)b * p.strideX, p.ldx, Mp, p.M, 0, p.Din / 8, lboA);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    cluster_arrive();  // this block runs: the others may write into its shared memory once they have waited
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_slot;
    const int *cond = p.cond + (int64_t)b * p.strideCond;
    const int quad = warp % 4, part = warp / 4, row = quad * 32 + lane;
    bool ok = true;
    uint32_t n_commits = 0;
    const int pass0 = kSampler ? sx.lo : 0, pass1 = kSampler ? kLearnBlocks : 1;
    bool first_wait = true;
    for (int pass = pass0; pass < pass1; ++pass) {
        for (int l = 0; l < 3; ++l) {
            const int nsl = l < 2 ? NS : NS3;
            if (threadIdx.x == 0) {
                if (!first_wait || mbar_wait(&full[l], 0u)) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    mlp_mma(tmem, l == 0 ? sX : (l == 1 ? sH1 : sH2), lboA, sW[l], nsl, l == 0 ? p.Din : p.H, &done);
                } else {
                    ok = false;
                }
            }
            __syncwarp();
            if (!mbar_wait(&done, n_commits & 1u)) ok = false;
            ++n_commits;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // every block takes part in every cluster barrier, whatever its status, so that none waits forever
            const int span = nsl / 2, c0 = part * span, ncol = min(32, span);
            uint32_t r[32];
            if (l < 2) {
                if (quad * 32 < Mp) tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, r);
                if (quad * 32 < Mp && row < Mp && ok) {
                    const bool live = row < p.M;
                    const float *cb = (l == 0 && live) ? (stage_c1 ? c1s + cond[row] * NS + c0
                                                                   : P + p.oC1 + (int64_t)cond[row] * p.H + rank * NS + c0)
                                                       : nullptr;
                    float cv[32];
#pragma unroll
                    for (int q = 0; q < 32; ++q) cv[q] = (cb && q < ncol) ? cb[q] : 0.f;
                    const uint32_t dst = (l == 0 ? sH1 : sH2) + (uint32_t)row * 16u;
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        if (8 * g >= ncol) break;
                        uint32_t w[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int q = 8 * g + 2 * e;
                            float v0 = __uint_as_float(r[q]) + bsl[l][c0 + q] + cv[q];
                            float v1 = __uint_as_float(r[q + 1]) + bsl[l][c0 + q + 1] + cv[q + 1];
                            v0 = live ? fmaxf(v0, 0.f) : 0.f;
                            v1 = live ? fmaxf(v1, 0.f) : 0.f;
                            const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                            w[e] = *reinterpret_cast<const uint32_t *>(&h);
                        }
                        const uint32_t kg = (uint32_t)(rank * NS + c0 + 8 * g) / 8;
                        asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(dst + kg * lboA), "r"(w[0]),
                                     "r"(w[1]), "r"(w[2]), "r"(w[3])
                                     : "memory");
                    }
                }
                // the slice (K-groups [rank NS/8, (rank+1) NS/8), contiguous) goes to the peers by bulk copies that
                // complete on their exchange barrier; this block's own copy is read by its tensor cores
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> async proxy
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncthreads();
                if (first_wait && l == 0) cluster_wait();  // all blocks of the cluster have started
                const uint32_t slice = (uint32_t)(NS / 8) * lboA;
                if (threadIdx.x == 0) {
                    mbar_expect_tx(&xchg[l], (uint32_t)(kMlpCL - 1) * slice);
                    const uint32_t src = (l == 0 ? sH1 : sH2) + rank * slice;
                    for (uint32_t q = 1; q < (uint32_t)kMlpCL; ++q) bulk_s2peer(src, slice, &xchg[l], (rank + q) % kMlpCL);
                }
                if (!mbar_wait(&xchg[l], (uint32_t)(pass - pass0) & 1u)) ok = false;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            } else if (!kSampler) {
                if (quad * 32 < Mp) tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, r);
                if (quad * 32 < Mp && row < p.M && ok) {
                    float *o = p.O + (int64_t)b * p.strideO + (int64_t)row * p.ldo + rank * NS3 + c0;
#pragma unroll
                    for (int q = 0; q < 32; q += 4)
                        if (q < ncol)
                            *reinterpret_cast<float4 *>(o + q) = make_float4(
                                __uint_as_float(r[q]) + bsl[2][c0 + q], __uint_as_float(r[q + 1]) + bsl[2][c0 + q + 1],
                                __uint_as_float(r[q + 2]) + bsl[2][c0 + q + 2],
                                __uint_as_float(r[q + 3]) + bsl[2][c0 + q + 3]);
                }
            } else {
                // mode block `pass`: modes [pass per, (pass+1) per), output columns 4 per wide, held by block
                // rank pass / 2, warp part pass % 2 (each block's slice covers two mode blocks).  The owning warps
                // park the outputs (+ b3) in shared memory; then all threads of that block draw one (row, mode)
                // pair each.
                const int per = sx.N / kLearnBlocks;
                if ((int)rank == pass / 2) {
                    if (part == pass % 2 && quad * 32 < Mp) {
                        tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, r);
                        if (row < Mp)
#pragma unroll
                            for (int q = 0; q < 32; ++q)
                                if (q < 4 * per) obuf[row * 32 + q] = __uint_as_float(r[q]) + bsl[2][c0 + q];
                    }
                    __syncthreads();
                    // item (row, mode, half): half 0 draws u (feature 0), half 1 draws phi~ (features 1, 2)
                    for (int idx = threadIdx.x; idx < 2 * p.M * per && ok; idx += blockDim.x) {
                        const int half = idx & 1, rw = (idx >> 1) / per, t = (idx >> 1) % per, k = pass * per + t;
                        if (pass < fbs[rw]) continue;
                        const int64_t gr = (int64_t)b * p.M + rw;
                        const ModeNoise nz = noise[rw * 2 * per + (pass % 2) * per + t];
                        const float *o = obuf + rw * 32 + 4 * t;
                        float f[2];
                        int nf, f0;
                        if (half == 0) {
                            const float u = sample_u(o[0], o[1], nz.eps, k, sx.N);
                            sx.u[gr * sx.N + k] = u;
                            f[0] = feature_u(u, k, sx.N);
                            nf = 1; f0 = 0;
                        } else {
                            const float ph = sample_phi(o[2], o[3], nz.t1, k);
                            sx.phi[gr * sx.N + k] = ph;
                            float sn, cs;
                            sincosf(ph, &sn, &cs);
                            f[0] = cs; f[1] = sn;
                            nf = 2; f0 = 1;
                        }
                        for (int c = 0; c < nf; ++c) {
                            const uint32_t fi = (uint32_t)(3 * k + f0 + c);
                            const __nv_bfloat16 h = __float2bfloat16_rn(f[c]);
                            const uint16_t bits = *reinterpret_cast<const uint16_t *>(&h);
                            const uint32_t off = sX + (fi / 8) * lboA + (uint32_t)rw * 16u + (fi % 8) * 2u;
                            for (uint32_t dstr = 0; dstr < (uint32_t)kMlpCL; ++dstr) st_cluster2(off, dstr, bits);
                        }
                    }
                }
                asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                cluster_arrive();
                cluster_wait();
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
        }
        first_wait = false;
    }
    if (!kSampler) {  // the peers' bulk copies out of this block's shared memory are complete before it exits
        cluster_arrive();
        cluster_wait();
    }
    if (!ok && threadIdx.x == 0) {
        if (p.err) atomicCAS(p.err, 0, kErrTimeout);
        // let the bulk copies still in flight land before the block's shared memory is released
        for (int l = 0; l < 3; ++l) (void)mbar_wait(&full[l], 0u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

namespace {

// Shared memory of a cluster block, or 0 if the shapes are outside what the kernel handles.
size_t mlp_cluster_smem(const MlpParams &p, bool sampler) {
    // M <= 128 rows (<= 64 with the sampler); Din a multiple of 16 (<= 192); H = 256; Dout/4 a multiple of 16
    // (<= 64); 16-byte aligned weights; O rows 16-byte aligned
    if (p.M < 1 || p.M > (sampler ? 64 : 128) || p.ncond < 1 || p.Din < 16 || p.Din > 192 || (p.Din % 16) || p.H != 256 ||
        p.Dout < 64 || p.Dout > 256 || (p.Dout % 64) || (p.ldo % 4) || !p.W1c || !p.W2c || !p.W3c ||
        ((uintptr_t)p.W1c | (uintptr_t)p.W2c | (uintptr_t)p.W3c) % 16 || ((p.strideW1 | p.strideW2 | p.strideW3) * 2) % 16)
        return 0;
    const size_t Mp = (size_t)((p.M + 15) & ~15);
    size_t act = 2 * (32 * Mp * 16 + kMlpPad);
    if (sampler) act += (size_t)(p.Din / 8) * Mp * 16 + kMlpPad;
    const size_t w = ((size_t)p.Din + p.H) * (p.H / kMlpCL) * 2 + (size_t)p.H * (p.Dout / kMlpCL) * 2;
    size_t extra = p.ncond <= kMlpMaxCond ? (size_t)p.ncond * (p.H / kMlpCL) * 4 : 0;
    if (sampler) extra += Mp * 32 * 4 + (size_t)p.M * 2 * (p.Dout / 4 / kLearnBlocks) * sizeof(ModeNoise) + (size_t)p.M * 4;
    return act + w + extra <= kMlpSmemMax ? act + w + extra : 0;
}

template <bool kSampler>
cudaError_t launch_mlp_cluster(const MlpParams &p, const SamplerExtra &sx, int batch, cudaStream_t s) {
    const size_t sm = mlp_cluster_smem(p, kSampler);
    if (sm == 0 || batch < 1) return cudaErrorInvalidValue;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(mlp_cluster_kernel<kSampler>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kMlpSmemMax);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    mlp_cluster_kernel<kSampler><<<batch * kMlpCL, kMlpThreads, sm, s>>>(p, sx);
    return cudaGetLastError();
}

}  // namespace

bool fused_mlp_supported(const MlpParams &p, bool sampler) { return mlp_cluster_smem(p, sampler) != 0; }

cudaError_t launch_fused_mlp(const MlpParams &p, int batch, cudaStream_t s) {
    return launch_mlp_cluster<false>(p, SamplerExtra{}, batch, s);
}

cudaError_t launch_fused_sampler(const MlpParams &p, const SamplerExtra &sx, int batch, cudaStream_t s) {
    if (sx.N < kLearnBlocks || sx.N % kLearnBlocks || sx.N * 4 != p.Dout || sx.lo < 0 || sx.lo > sx.hi ||
        sx.hi >= kLearnBlocks || !sx.row_id || !sx.ctl || !sx.u || !sx.phi)
        return cudaErrorInvalidValue;
    return launch_mlp_cluster<true>(p, sx, batch, s);
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
