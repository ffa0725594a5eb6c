// pt_learn.h -- device kernels of the learned global-move proposal (internal to the library).
//
// The proposal is an independence Metropolis-Hastings move on a chain's whole configuration.  Its
// density q is a per-sample masked (MADE-style, block-autoregressive) MLP over gauge-fixed coordinates:
//   - global phase and comb gauge removed: phi~_k = phi_k - phi_0 - k (phi_1 - phi_0), so phi~_0 = phi~_1 = 0;
//   - intensities s_k = |a_k|^4 / N on the simplex, stick-broken into v_k = s_k / r_k, r_k = 1 - sum_{i<k} s_i;
//   - logit(v_k) ~ Normal(mu_k, sigma_k) (k <= N-2), phi~_k ~ wrapped Cauchy(m_k, rho_k) (k >= 2);
//   - the conditionals of mode block b depend on blocks < b and on the temperature index (conditional bias).
// The move draws a fresh gauge (alpha, theta) uniformly.  With log q the log density of (v_k, phi~_k) and
// extra = -sum_{k<=N-2} log r_k + 1/2 sum_k log s_k (stick-breaking Jacobian and the beta = 0 law of Eq. (8),
// prod_k s_k^(-1/2) ds dphi, as base measure), the acceptance
//   log A = -beta (H' - H) + [log q(x) + extra(x)] - [log q(x') + extra(x')]
// leaves the tempered target exactly invariant (the paper has no counterpart; it serves Sec. III.A).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include "pt_common.cuh"

namespace ptgb {

constexpr uint32_t kTagGlobal = 5u, kTagBatch = 6u;
constexpr int kLearnBlocks = 8;  // autoregressive blocks of modes
constexpr int kLearnMaxN = 64;   // largest N of the proposal network

struct LearnShape {
    int N, H, Din, Dout, ncold, S;
    size_t psize;  // FP32 parameters per sample
    size_t oW1, ob1, oC1, oW2, ob2, oW3, ob3;
};

// per-row inputs of the density: u_k = logit(v_k) (k <= N-2), phi~_k (k >= 2), extra = -sum log r_k + 1/2 sum log s_k
struct RawRows {
    float *u, *phi;   // [rows][N]
    float *extra;     // [rows]
    int *cond;        // [rows]
};

// Features of configurations taken from chain slots (slot[row] >= 0) of a state array, or from a proposal
// buffer (slot == nullptr: row-major [rows][N] complex, double2 if dbl else float2).  Writes X (bf16 [rows][Din]), XT (bf16 [Din][ldxt]),
// and the raw rows.
struct FeatParams {
    const void *a;          // chain states (float2 or double2) or proposals (float2 [rows][N])
    int dbl;                // chain states in FP64
    const SampleDev *samples;
    const int *slot;        // [S][rows_per_sample] chain slots, or nullptr for proposal rows
    int rows_per_sample;    // rows of one sample
    int N, Din;
    __nv_bfloat16 *X, *XT;  // optional [S][rows][Din], [S][Din][ldxt]
    int ldxt;
    RawRows raw;            // raw row (s, row) at s * raw_stride + raw_off + row
    int64_t raw_stride, raw_off;
    const int *cond_in;     // optional [S][rows]: copied to raw.cond
    int64_t x_stride;       // rows per sample in X
};
cudaError_t launch_features(const FeatParams &p, int S, cudaStream_t s);

// Masked BF16 copies of the weights (and the transposes the backward pass needs).
struct CastParams {
    const float *P;         // [S][psize]
    const float *M1, *M2, *M3;
    __nv_bfloat16 *W1, *W2, *W3, *W2T, *W3T;
    __nv_bfloat16 *W1c, *W2c, *W3c;  // the same weights in the sliced canonical K-major layout (MlpParams)
    LearnShape sh;
};
cudaError_t launch_cast(const CastParams &p, cudaStream_t s);

// Log density per row from the network outputs O ([S][rows][Dout] = (mu, log sigma, m, rho_raw) per mode),
// plus the gradient of mean(-log q) over the rows of each sample (optional).
struct DensityParams {
    const float *O;
    RawRows raw;
    int rows_per_sample, N, Dout;
    double *logq;           // [S][rows]
    float *dO;              // optional FP32 [S][rows][Dout]
    __nv_bfloat16 *dOb, *dOT;  // optional BF16 [S][rows][Dout], [S][Dout][lddt]
    int lddt;
    float inv_rows;         // 1 / rows (mean over the batch)
    int64_t o_stride;       // rows per sample in O, dO, dOb
};
cudaError_t launch_density(const DensityParams &p, int S, cudaStream_t s);

// Bias gradients: db[col] = sum_rows dZ[row][col]; dC[cond[row]][col] += dZ[row][col] (optional)
cudaError_t launch_colsum(const float *dZ, int rows, int cols, float *db, float *dC, const int *cond, int S,
                          int64_t strideZ, int64_t strideGrad, cudaStream_t s);

// Adam on [S][psize] parameters (grad G already averaged).
cudaError_t launch_adam(float *P, const float *G, float *m, float *v, size_t n, float lr, float b1, float b2,
                        float eps, int t, cudaStream_t s);

// Minibatch gather from the training set: rows of raw data -> raw rows + features.
struct GatherParams {
    const float *du, *dphi, *dextra;  // training set [S][ndata][N], [S][ndata]
    const int *dcond;
    int ndata, rows, N, Din, ldxt;
    int64_t stride;          // rows per sample in the training set
    uint64_t seed;
    uint32_t step;
    __nv_bfloat16 *X, *XT;
    RawRows raw;
    int64_t x_stride;
};
cudaError_t launch_gather(const GatherParams &p, int S, cudaStream_t s);

// First resampled block of a proposal row: uniform on [lo, hi], drawn from the row's stream.  Blocks below
// it keep the current configuration (and its gauge); block 0 resamples everything under a fresh gauge.
__device__ __forceinline__ int first_block(uint64_t seed, uint32_t id, uint32_t round, int N, int lo, int hi) {
    const u32x4 w = draw(seed, id, round, (uint32_t)(N + 2), kTagGlobal);
    return lo + (int)(((uint64_t)w.x * (uint64_t)(hi - lo + 1)) >> 32);
}

// One sampling pass: fill the variables of mode block b from the network outputs (rows = proposals);
// rows whose first resampled block is above b keep the current values already in X, u, phi.
struct SampleParams {
    const float *O;
    int rows_per_sample, N, Dout, Din, block;
    int lo, hi;              // range of the first resampled block
    uint64_t seed;
    const uint32_t *row_id;  // [S][rows] chain ids (stream of the draws)
    const Control *ctl;      // global_rounds = round of the draws
    __nv_bfloat16 *X;        // [S][x_stride][Din]
    float *u, *phi;          // raw proposal variables [S][rows][N]
    int64_t o_stride, x_stride;
};
cudaError_t launch_sample_block(const SampleParams &p, int S, cudaStream_t s);

// Amplitudes of the proposals from (u, phi~): modes below the first resampled block k0 are copied from the
// current configuration, the tail mass r_{k0} is the current one, and the gauge is the current one
// (fresh and uniform when k0 = 0).
struct AssembleParams {
    const float *u, *phi;
    int rows_per_sample, N;
    int lo, hi;
    uint64_t seed;
    const uint32_t *row_id;
    const Control *ctl;
    const void *a_cur;       // chain states (float2 or double2)
    int dbl;
    const SampleDev *samples;
    const int *slot;         // [S][rows] chain slots
    double2 *a;              // [S][rows][N]
};
cudaError_t launch_assemble(const AssembleParams &p, int S, cudaStream_t s);

// FP64 energies of configurations (quadruplet sum) from chain slots or from a proposal buffer.
struct EnergyListParams {
    const void *a;
    int dbl;
    const SampleDev *samples;
    const int *slot;         // or nullptr: proposal rows [S][rows][N] (double2 if dbl else float2)
    int rows_per_sample, N;
    const int4 *quads;
    const double *Jq;
    // FP32 configurations (values exact in FP32, also when given as double2): the sum in double-float
    // arithmetic from the couplings split into float pairs Jdf (J = hi + lo), instead of FP64
    const float2 *Jdf;
    double cc;
    double *E;               // [S][rows]
};
struct EnergyList2 {
    EnergyListParams set[2];
};
// All sets of one launch use the same arithmetic: double-float if set[0].Jdf is given, else FP64.
cudaError_t launch_energy_list(const EnergyList2 &p, int n_sets, int S, cudaStream_t s);
// Jdf[i] = (hi, lo) floats with hi + lo = J[i] to 48 bits.
cudaError_t launch_split_df(const double *J, float2 *Jdf, int64_t n, cudaStream_t s);

// Metropolis-Hastings decision and state update of every proposal row.
struct MHParams {
    const double *logq_cur, *logq_prop, *H_cur, *H_prop;
    const float *extra_cur, *extra_prop;
    const double2 *a_prop;   // proposals [S][rows][N]
    void *a;                 // chain states
    int dbl;
    double *E;               // running energies (chain slots)
    const int *slot;
    const SampleDev *samples;
    const double *beta;
    const int *label;
    int rows_per_sample, N, nT;
    uint64_t seed;
    const uint32_t *row_id;
    const Control *ctl;
    unsigned long long *acc, *att;  // [S][nT]
};
cudaError_t launch_mh(const MHParams &p, int S, cudaStream_t s);

// loss = mean over S x rows of -(logq + extra)
cudaError_t launch_learn_loss(const double *logq, const float *extra, int S, int rows, double *out, cudaStream_t s);

// Rows of the cold chains of every sample: slot and chain id (stream) for rows t * R + r, t < ncold.
cudaError_t launch_cold_rows(const int *perm, int S, int R, int nT, int ncold, int *slot, uint32_t *row_id,
                             int *cond, cudaStream_t s);

}  // namespace ptgb
