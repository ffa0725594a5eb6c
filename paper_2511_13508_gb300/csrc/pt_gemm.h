// pt_gemm.h -- batched BF16 tensor-core GEMM (tcgen05) with the epilogues of the proposal network.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace ptgb {

enum GemmEpilogue : int {
    kEpiF32 = 0,   // D = acc (+ bias)
    kEpiRelu = 1,  // z = acc + bias + cbias[cond[row]]; D = z; H = HT = bf16(max(z, 0))
    kEpiGate = 2,  // g = acc * [gate > 0]; D = g; H = HT = bf16(g)   (back-propagation through a ReLU)
};

struct GemmParams {
    const __nv_bfloat16 *A, *B;  // A: M x K row-major (lda); B: N x K row-major (ldb); per batch strides
    int64_t strideA, strideB;
    int lda, ldb, M, N, K, mode;
    float *D;                    // optional FP32 output, M x N (ldd)
    int64_t strideD;
    int ldd;
    const float *bias;           // optional, N per batch
    int64_t strideBias;
    const float *cbias;          // optional, [n_cond][N] per batch, row r uses cond[r]
    int64_t strideCbias;
    const int *cond;             // per batch, M entries (stride M_cond)
    int64_t strideCond;
    __nv_bfloat16 *H;            // optional BF16 output, M x N (ldh)
    int64_t strideH;
    int ldh;
    __nv_bfloat16 *HT;           // optional BF16 transposed output, N x M (ldht)
    int64_t strideHT;
    int ldht;
    const float *gate;           // for kEpiGate: M x N (ldgate)
    int64_t strideGate;
    int ldgate;
    int *err;
};

cudaError_t launch_gemm_bf16(const GemmParams &p, int batch, cudaStream_t s);

// The proposal network's whole forward pass for up to 128 rows per sample in one launch:
// O = W3 relu(W2 relu(W1 x + b1 + C1[cond]) + b2) + b3, the hidden activations kept in shared memory (BF16)
// and every product on the tensor cores.  One cluster of four thread blocks per sample (batch = samples).
struct MlpParams {
    const __nv_bfloat16 *X;  // [batch][rows of stride ldx] inputs, row-major (Din columns)
    int64_t strideX;
    int ldx, M, Din, H, Dout;
    // masked BF16 weights per sample in the sliced canonical K-major layout: for an N x K matrix cut into four
    // slices of NS = N/4 rows, element (n, k) at ((n / NS) (K / 8) + k / 8) NS 8 + (n % NS) 8 + k % 8, so that
    // each slice is contiguous: W1 (N = H, K = Din), W2 (H, H), W3 (Dout, H)
    const __nv_bfloat16 *W1c, *W2c, *W3c;
    int64_t strideW1, strideW2, strideW3;
    const float *P;          // FP32 master parameters [batch][psize]: biases b1, C1, b2, b3
    int64_t psize;
    int64_t ob1, oC1, ob2, ob3;
    const int *cond;         // [batch][strideCond] temperature index per row, in [0, ncond)
    int64_t strideCond;
    int ncond;               // rows of C1
    float *O;                // [batch][strideO], rows of ldo
    int64_t strideO;
    int ldo;
    int *err;
};
cudaError_t launch_fused_mlp(const MlpParams &p, int batch, cudaStream_t s);
// Whether the single-launch forward (sampler = false) or the one-launch sampler (true) takes these shapes.
bool fused_mlp_supported(const MlpParams &p, bool sampler);

struct Control;
// The autoregressive sampling of the learned proposal in one launch (network weights resident on chip): for
// mode blocks b = lo..7 a pass of the network over the input features X (the current configurations'
// features on entry; M = proposal rows per sample <= 64), then the draws of block b's modes for the rows whose
// first resampled block is <= b, written to u, phi ([batch][M][N]) and, as input features, into the next pass.
// The draws are those of the block-wise sampling kernel (same Philox streams, same arithmetic).
struct SamplerExtra {
    uint64_t seed;
    const uint32_t *row_id;  // [batch][M] chain ids (stream of the draws)
    const Control *ctl;      // global_rounds = round of the draws
    int lo, hi, N;           // range of the first resampled block; modes
    float *u, *phi;
};
cudaError_t launch_fused_sampler(const MlpParams &p, const SamplerExtra &sx, int batch, cudaStream_t s);

}  // namespace ptgb
