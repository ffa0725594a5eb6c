// pt_sweep.cu -- the J-sharing Metropolis sweep kernel (sm_103a), its field-only twin and the
// full-energy (resync) kernel, for the smoothed-cubic 4-body random-laser model (arXiv 2511.13508).
//
// Local field of the updated modes (paper Sec. III.A.3).  With z_P = a_x a_y for the pair P = {x,y},
// the field of mode l factorises over the pair sum s = x + y:
//     h_l = sum_s conj(a_{s-l}) acc_l[s],     acc_l[s] = sum_{P : x+y=s} J_l[s][P] z_P,
// where J_l[s][P] is the coupling of quadruplet {l, s-l} u P.  One pair product z_P therefore feeds
// both fields of a pair update (j,k), and all chains of a disorder sample read J_j and J_k once per
// thread block: the J rows stream HBM/L2 -> shared memory through cp.async.bulk (TMA) into a ring of
// stages, guarded by mbarriers, while the chains' amplitudes stay resident in shared memory.
//
// Delta H of a pair move (j,k) (Sec. III.A.1; cross term = reading R5 of the design notes):
//     dH = -cc Re[ conj(dj) h_j + conj(dk) h_k + conj(dj) dk B_jk + conj(dj) conj(dk) A_jk ],
//     B_jk = sum_s conj(a_{s-j}) J_j[s][{k, s-k}] a_{s-k},   A_jk = acc_j[j+k].
#include <cstdint>
#include <cstdio>
#include "pt_common.cuh"
#include "pt_kernels.h"

namespace ptgb {

// ------------------------------------------------------------------------------------------------
// PTX wrappers: mbarrier, bulk copy, named barriers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after kWaitNs of wall time, records the error and reports failure.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, Control *ctl, int where,
                                                  volatile int *abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t n = 1;; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if ((n & 63u) == 0 && global_ns() - t0 > kWaitNs) {
            record_error(ctl, kErrTimeout, where);
            *abort_flag = 1;
            return false;
        }
    }
}
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void named_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ------------------------------------------------------------------------------------------------
// complex arithmetic on float2/double2
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {  // conj(a) * b
    V r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.x * b.y - a.y * b.x;
    return r;
}
template <typename V, typename T> __device__ __forceinline__ void caxpy(V &acc, T s, V z) {
    acc.x = fma(s, z.x, acc.x);
    acc.y = fma(s, z.y, acc.y);
}
template <typename V> __device__ __forceinline__ void cadd(V &acc, V z) { acc.x += z.x; acc.y += z.y; }

// Row-stride of the shared amplitude table [x + APAD][chain] (complex elements): one pad element for
// 8-byte complex with 8 chains, so that four workers reading rows 8 apart hit distinct bank halves.
template <typename real, int G> struct RowStride {
    static constexpr int value = (sizeof(real) == 4 && G == 8) ? G + 1 : G;
};

// Loads one J column (TS reals: fixed x offset, the TS rows) of a block as vectors.
template <typename real> struct JRow;
template <> struct JRow<float> {
    float v[TX];
    __device__ __forceinline__ void load(const float *p) {
        const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
};
template <> struct JRow<double> {
    double v[TX];
    __device__ __forceinline__ void load(const double *p) {
#pragma unroll
        for (int i = 0; i < TX; i += 2) {
            const double2 a = *reinterpret_cast<const double2 *>(p + i);
            v[i] = a.x; v[i + 1] = a.y;
        }
    }
};

// Per-lane partial sums of one pair update.
template <typename real> struct Partials {
    typename vec2<real>::type hj, hk, B, A;
    __device__ __forceinline__ void zero() {
        hj.x = hj.y = hk.x = hk.y = B.x = B.y = A.x = A.y = real(0);
    }
};

// h += conj(m) acc, as four fused multiply-adds
template <typename V> __device__ __forceinline__ void cfma_conj(V &h, V m, V acc) {
    h.x = fma(m.x, acc.x, h.x);
    h.x = fma(m.y, acc.y, h.x);
    h.y = fma(m.x, acc.y, h.y);
    h.y = fma(-m.y, acc.x, h.y);
}

// One TS x TX block of pair products for chain c: accumulates the j field (MODE & 1), the k field
// (MODE & 2), and the j-k cross terms (with the j field).  as = shared amplitude table; Jj, Jk =
// column-major blocks.  The x offset i runs outside, the row r inside, so the 2*TS row accumulators
// are independent chains of fused multiply-adds.
template <typename real, int RS, int MODE, bool WB>
__device__ __forceinline__ void process_block(const typename vec2<real>::type *__restrict__ as, int c, int s0,
                                              int x0, int j, int k, int N, const real *Jj, const real *Jk,
                                              Partials<real> &p) {
    using V = typename vec2<real>::type;
    V ax[TX], ay[TS + TX - 1];
#pragma unroll
    for (int i = 0; i < TX; ++i) ax[i] = as[(x0 + i + APAD) * RS + c];
    const int ybase = s0 - x0 - (TX - 1) + APAD;
#pragma unroll
    for (int d = 0; d < TS + TX - 1; ++d) ay[d] = as[(ybase + d) * RS + c];
    V accj[TS], acck[TS];
#pragma unroll
    for (int r = 0; r < TS; ++r) accj[r].x = accj[r].y = acck[r].x = acck[r].y = real(0);
#pragma unroll
    for (int i = 0; i < TX; ++i) {
        JRow<real> cj, ck;
        if (MODE & 1) cj.load(Jj + i * TS);
        if (MODE & 2) ck.load(Jk + i * TS);
#pragma unroll
        for (int r = 0; r < TS; ++r) {
            const V z = cmul(ax[i], ay[r - i + TX - 1]);
            if (MODE & 1) caxpy(accj[r], cj.v[r], z);
            if (MODE & 2) caxpy(acck[r], ck.v[r], z);
        }
    }
#pragma unroll
    for (int r = 0; r < TS; ++r) {
        const int s = s0 + r;
        if (MODE & 1) cfma_conj(p.hj, as[(s - j + APAD) * RS + c], accj[r]);
        if (MODE & 2) cfma_conj(p.hk, as[(s - k + APAD) * RS + c], acck[r]);
    }
    if (MODE & 1) {
        // A_jk is the accumulator of row j+k: only the blocks of that row's s-tile hold it
        const int rs = j + k - s0;
        if (rs >= 0 && rs < TS) {
#pragma unroll
            for (int r = 0; r < TS; ++r)
                if (r == rs) cadd(p.A, accj[r]);
        }
    }
    if ((MODE & 1) && WB) {
        // B_jk: the element of row s at x* = min(k, s-k) belongs to this block for the rows s >= 2k of
        // the column tile holding k, and for the rows s - k in [x0, x0+TX) of the diagonal band.
        const bool col = (k >= x0 && k < x0 + TX);
        const bool diag = (s0 + TS - 1 >= x0 + k) && (s0 <= x0 + TX - 1 + k);
        if (col || diag) {
#pragma unroll
            for (int r = 0; r < TS; ++r) {
                const int s = s0 + r, y = s - k;
                const int xs = (y < k) ? y : k;
                if (y >= 0 && y < N && xs >= x0 && xs < x0 + TX) {
                    const real Jv = Jj[(xs - x0) * TS + r];
                    const V m = as[(s - j + APAD) * RS + c];
                    const V yv = as[(y + APAD) * RS + c];
                    caxpy(p.B, Jv, cmulc(m, yv));
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Packed-FP32 block arithmetic (the FP32 shapes of 8 chains per block).  Rows are taken in pairs (r, r+1)
// and every quantity is a float2 pair over the two rows, so each instruction is an FFMA2/FMUL2 doing two
// fused multiply-adds: with
//     sx = (Re a_x, Re a_x), sy = (Im a_x, Im a_x)                  (splats of a_x in registers)
//     WX = (Re a_y, Re a_{y+1}), WY = (Im a_y, Im a_{y+1})          (window table awin, y = s - x)
// the pair products of rows (s, s+1) at column x are
//     Re z = sx WX - sy WY,   Im z = sx WY + sy WX,
// and a field row pair accumulates acc += (J[s][x], J[s+1][x]) z with the column-major J block supplying
// the coupling pair directly.  Two FMUL2 + two FFMA2 make 2 products; one FFMA2 per field per component
// accumulates them: 2 instructions per coupling term when both fields use the block, 3 otherwise.
struct PartialsX2 {
    float2 hjx, hjy, hjyn, hkx, hky, hkyn;  // h = (hx.0 + hx.1, (hy.0 + hy.1) - (hyn.0 + hyn.1))
    float2 B, A;
    __device__ __forceinline__ void zero() {
        hjx = hjy = hjyn = hkx = hky = hkyn = B = A = make_float2(0.f, 0.f);
    }
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <int G, int MODE, bool WB>
__device__ __forceinline__ void process_block_x2(const float2 *__restrict__ as, const float4 *__restrict__ awin,
                                                 int c, int s0, int x0, int j, int k, int N, const float *Jj,
                                                 const float *Jk, PartialsX2 &p) {
    constexpr int RS = RowStride<float, G>::value;
    // Column i = 2h + pi pairs rows (2q, 2q+1) with the window starting at y-offset d = 2q - i + 7, of parity
    // 1 - pi: the columns run in two passes by parity, each holding the 7 windows of its parity
    // (d = 2m + 1 - pi, m = q - h + 3), so that only 7 windows are live at a time.
    const int ybase = s0 - x0 - (TX - 1) + APAD;
    float2 ajx[TS / 2], ajy[TS / 2], akx[TS / 2], aky[TS / 2];
#pragma unroll
    for (int q = 0; q < TS / 2; ++q) ajx[q] = ajy[q] = akx[q] = aky[q] = f2(0.f, 0.f);
#pragma unroll
    for (int pi = 0; pi < 2; ++pi) {
        float2 wx[7], wy[7];
#pragma unroll
        for (int m = 0; m < 7; ++m) {
            const float4 w = awin[(ybase + 2 * m + 1 - pi) * G + c];
            wx[m] = f2(w.x, w.y);
            wy[m] = f2(w.z, w.w);
        }
#pragma unroll
        for (int h = 0; h < TX / 2; ++h) {
            const int i = 2 * h + pi;
            // splats of a_x in registers (register moves cost less than the shared-memory bandwidth of a table)
            const float2 axv = as[(x0 + i + APAD) * RS + c];
            const float2 sx = f2(axv.x, axv.x), sy = f2(axv.y, axv.y), nsy = f2(-axv.y, -axv.y);
            float2 jp[TS / 2], kp[TS / 2];
            if (MODE & 1) {
                const float4 a = *reinterpret_cast<const float4 *>(Jj + i * TS), b = *reinterpret_cast<const float4 *>(Jj + i * TS + 4);
                jp[0] = f2(a.x, a.y); jp[1] = f2(a.z, a.w); jp[2] = f2(b.x, b.y); jp[3] = f2(b.z, b.w);
            }
            if (MODE & 2) {
                const float4 a = *reinterpret_cast<const float4 *>(Jk + i * TS), b = *reinterpret_cast<const float4 *>(Jk + i * TS + 4);
                kp[0] = f2(a.x, a.y); kp[1] = f2(a.z, a.w); kp[2] = f2(b.x, b.y); kp[3] = f2(b.z, b.w);
            }
            float2 tx[TS / 2], ty[TS / 2], zx[TS / 2], zy[TS / 2];
#pragma unroll
            for (int q = 0; q < TS / 2; ++q) {
                const int m = q - h + 3;
                tx[q] = __fmul2_rn(nsy, wy[m]);
                ty[q] = __fmul2_rn(sy, wx[m]);
            }
#pragma unroll
            for (int q = 0; q < TS / 2; ++q) {
                const int m = q - h + 3;
                zx[q] = __ffma2_rn(sx, wx[m], tx[q]);
                zy[q] = __ffma2_rn(sx, wy[m], ty[q]);
            }
#pragma unroll
            for (int q = 0; q < TS / 2; ++q) {
                if (MODE & 1) { ajx[q] = __ffma2_rn(jp[q], zx[q], ajx[q]); ajy[q] = __ffma2_rn(jp[q], zy[q], ajy[q]); }
                if (MODE & 2) { akx[q] = __ffma2_rn(kp[q], zx[q], akx[q]); aky[q] = __ffma2_rn(kp[q], zy[q], aky[q]); }
            }
        }
    }
    // close the rows: h += conj(m) acc with m = a_{s-l} for the row pair (s, s+1) from the window table
#pragma unroll
    for (int q = 0; q < TS / 2; ++q) {
        if (MODE & 1) {
            const float4 w = awin[(s0 + 2 * q - j + APAD) * G + c];
            const float2 mx = f2(w.x, w.y), my = f2(w.z, w.w);
            p.hjx = __ffma2_rn(mx, ajx[q], p.hjx);
            p.hjx = __ffma2_rn(my, ajy[q], p.hjx);
            p.hjy = __ffma2_rn(mx, ajy[q], p.hjy);
            p.hjyn = __ffma2_rn(my, ajx[q], p.hjyn);
        }
        if (MODE & 2) {
            const float4 w = awin[(s0 + 2 * q - k + APAD) * G + c];
            const float2 mx = f2(w.x, w.y), my = f2(w.z, w.w);
            p.hkx = __ffma2_rn(mx, akx[q], p.hkx);
            p.hkx = __ffma2_rn(my, aky[q], p.hkx);
            p.hky = __ffma2_rn(mx, aky[q], p.hky);
            p.hkyn = __ffma2_rn(my, akx[q], p.hkyn);
        }
    }
    if (MODE & 1) {
        // A_jk is the accumulator of row j+k
        const int rs = j + k - s0;
        if (rs >= 0 && rs < TS) {
#pragma unroll
            for (int q = 0; q < TS / 2; ++q) {
                if (rs == 2 * q) { p.A.x += ajx[q].x; p.A.y += ajy[q].x; }
                if (rs == 2 * q + 1) { p.A.x += ajx[q].y; p.A.y += ajy[q].y; }
            }
        }
    }
    if ((MODE & 1) && WB) {
        const bool col = (k >= x0 && k < x0 + TX);
        const bool diag = (s0 + TS - 1 >= x0 + k) && (s0 <= x0 + TX - 1 + k);
        if (col || diag) {
#pragma unroll
            for (int r = 0; r < TS; ++r) {
                const int s = s0 + r, y = s - k;
                const int xs = (y < k) ? y : k;
                if (y >= 0 && y < N && xs >= x0 && xs < x0 + TX) {
                    const float Jv = Jj[(xs - x0) * TS + r];
                    const float2 m = as[(s - j + APAD) * RS + c];
                    const float2 yv = as[(y + APAD) * RS + c];
                    caxpy(p.B, Jv, cmulc(m, yv));
                }
            }
        }
    }
}

template <int G, bool WB>
__device__ __forceinline__ void process_block_x2_dispatch(int mode, const float2 *as, const float4 *awin, int c,
                                                          int s0, int x0, int j, int k, int N, const float *Jj,
                                                          const float *Jk, PartialsX2 &p) {
    if (mode == 3) process_block_x2<G, 3, WB>(as, awin, c, s0, x0, j, k, N, Jj, Jk, p);
    else if (mode == 1) process_block_x2<G, 1, WB>(as, awin, c, s0, x0, j, k, N, Jj, Jk, p);
    else if (mode == 2) process_block_x2<G, 2, WB>(as, awin, c, s0, x0, j, k, N, Jj, Jk, p);
}

// Window entry of one amplitude-table row (shared-memory row index R = x + APAD): (Re a_R, Re a_{R+1},
// Im a_R, Im a_{R+1}).
template <int RS>
__device__ __forceinline__ void packed_rows(const float2 *as, float4 *awin, int G, int R, int rows, int c) {
    const float2 a = as[R * RS + c];
    const float2 b = (R + 1 < rows) ? as[(R + 1) * RS + c] : make_float2(0.f, 0.f);
    awin[R * G + c] = make_float4(a.x, b.x, a.y, b.y);
}

// WB: also pick the B_jk elements out of the block (the field-only kernel); the sweep kernel gathers them
// once per update instead (b_couplings).
template <typename real, int RS, bool WB>
__device__ __forceinline__ void process_block_dispatch(int mode, const typename vec2<real>::type *as, int c,
                                                       int s0, int x0, int j, int k, int N, const real *Jj,
                                                       const real *Jk, Partials<real> &p) {
    if (mode == 3) process_block<real, RS, 3, WB>(as, c, s0, x0, j, k, N, Jj, Jk, p);
    else if (mode == 1) process_block<real, RS, 1, WB>(as, c, s0, x0, j, k, N, Jj, Jk, p);
    else if (mode == 2) process_block<real, RS, 2, WB>(as, c, s0, x0, j, k, N, Jj, Jk, p);
}


// Block ranges of an update: union of the runs of j and k in the sample's block list.
struct Ranges {
    int jlo, jhi, klo, khi, ulo, uhi;  // sample-local block indices [lo, hi)
    int64_t jg, kg;                    // global block index of the first block of j's / k's run
};
__device__ __forceinline__ Ranges update_ranges(const SampleDev &sd, const int *bo, const int *mode_blk, int j,
                                                int k) {
    Ranges R;
    const int stlo_j = j / TS, sthi_j = min((j + sd.N - 1) / TS, sd.ST - 1);
    const int stlo_k = k / TS, sthi_k = min((k + sd.N - 1) / TS, sd.ST - 1);
    R.jlo = bo[stlo_j]; R.jhi = bo[sthi_j + 1];
    R.klo = bo[stlo_k]; R.khi = bo[sthi_k + 1];
    R.ulo = min(R.jlo, R.klo); R.uhi = max(R.jhi, R.khi);
    R.jg = sd.J_off + mode_blk[j];
    R.kg = sd.J_off + mode_blk[k];
    return R;
}

// Smallest N for which the FP32 sweep kernel gathers the B_jk couplings once per update (b_coupling, by the copy
// warp into a shared buffer) instead of picking them out of the blocks.  Measured on GB300 (chain-sweeps/s): with
// the gather from N = 48 on every FP32 shape, the ragged batch on 16 x 11 8.72M -> 8.82M and on 8 x 11 8.53M ->
// 8.62M, the others unchanged; when the field warps still did the gather themselves it paid only from N = 128 on.
constexpr int kGatherBMinN = 48;
template <typename real, int G> constexpr bool kGatherB = sizeof(real) == 4;
// With 8 chains per block the copy warp also draws the random part of every chain's proposal, up to kBD updates
// ahead, and warp 0 only finishes it at the update's start (measured on GB300: N = 256 bench workload +0.8%;
// with 16 or 32 chains per block warp 0 drawing the whole proposal itself measured 0.7-1.5% faster).
template <int G> constexpr bool kCopyDraws = G == 8;

// The coupling J_j[s][{k, s-k}] of quadruplet {j, s-j, k, s-k} (0 where the store holds no such entry):
// column x* = min(k, s-k) of row s in mode j's run, read from global memory (L2-resident: the run is
// being streamed for the same update).
template <typename real>
__device__ __forceinline__ real b_coupling(const real *__restrict__ J, const int *s_bo, const int *s_xtlo,
                                           const Ranges &Rg, int s, int k) {
    const int y = s - k, x = y < k ? y : k;
    const int st = s / TS, xt = x / TX;
    const int xi = xt - s_xtlo[st];
    if (xi < 0 || xi >= s_bo[st + 1] - s_bo[st]) return real(0);
    const int64_t gb = Rg.jg + (s_bo[st] + xi - Rg.jlo);
    return __ldg(J + gb * JStride<real>::value + (x - xt * TX) * TS + (s - st * TS));
}

// ------------------------------------------------------------------------------------------------
// Proposal of a pair move and Metropolis test (Sec. III.A.1, readings R3 and R6).
template <typename real> struct Proposal {
    typename vec2<real>::type aj, ak, nj, nk;  // old and proposed amplitudes
    real U;
};

// The pair move of Sec. III.A.1 in two parts: draw_proposal takes the random numbers of (chain, sweep, update)
// -- the angles as sqrt(cos theta), sqrt(sin theta), the phases as (cos, sin), and the Metropolis uniform U -- and
// needs no state, so the copy warp draws it ahead of the update; finish_proposal scales it by
// K = (|a_j|^4 + |a_k|^4)^(1/4) of the chain's current amplitudes (mode j receives K sqrt(cos theta)).
template <typename real> struct ProposalDraw {
    real sqc, sqs, cj, sj, ck, sk, U, pad;
};

template <typename real>
__device__ __forceinline__ ProposalDraw<real> draw_proposal(uint64_t seed, uint32_t chain_id, uint32_t sweep,
                                                            uint32_t update);

template <>
__device__ __forceinline__ ProposalDraw<float> draw_proposal<float>(uint64_t seed, uint32_t chain_id, uint32_t sweep,
                                                                    uint32_t update) {
    ProposalDraw<float> D;
    const u32x4 w = draw(seed, chain_id, sweep, update, kTagPropose);
    const float kInv = 2.3283064365386963e-10f;
    const float fj = ((float)w.x + 0.5f) * kInv, fk = ((float)w.y + 0.5f) * kInv, ft = ((float)w.z + 0.5f) * kInv;
    float st, ct;
    sincospif(2.0f * fj, &D.sj, &D.cj);
    sincospif(2.0f * fk, &D.sk, &D.ck);
    sincospif(0.5f * ft, &st, &ct);
    D.sqc = sqrtf(ct);
    D.sqs = sqrtf(st);
    D.U = ((float)w.w + 0.5f) * kInv;
    D.pad = 0.f;
    return D;
}

template <>
__device__ __forceinline__ ProposalDraw<double> draw_proposal<double>(uint64_t seed, uint32_t chain_id,
                                                                      uint32_t sweep, uint32_t update) {
    ProposalDraw<double> D;
    const u32x4 w = draw(seed, chain_id, sweep, update, kTagPropose);
    const double phj = kTwoPi * u01(w.x), phk = kTwoPi * u01(w.y), th = kHalfPi * u01(w.z);
    D.sqc = sqrt(cos(th));
    D.sqs = sqrt(sin(th));
    sincos(phj, &D.sj, &D.cj);
    sincos(phk, &D.sk, &D.ck);
    D.U = u01(w.w);
    D.pad = 0.0;
    return D;
}

template <typename real>
__device__ __forceinline__ Proposal<real> finish_proposal(const ProposalDraw<real> &D, typename vec2<real>::type aj,
                                                          typename vec2<real>::type ak) {
    Proposal<real> P;
    P.aj = aj; P.ak = ak;
    const real uj = aj.x * aj.x + aj.y * aj.y, uk = ak.x * ak.x + ak.y * ak.y;
    real K;
    if constexpr (sizeof(real) == 4) K = sqrtf(sqrtf(uj * uj + uk * uk));
    else K = sqrt(sqrt(uj * uj + uk * uk));
    const real Aj = K * D.sqc, Ak = K * D.sqs;
    P.nj.x = Aj * D.cj; P.nj.y = Aj * D.sj;
    P.nk.x = Ak * D.ck; P.nk.y = Ak * D.sk;
    P.U = D.U;
    return P;
}

template <typename real>
__device__ __forceinline__ real delta_h(const Proposal<real> &P, const Partials<real> &f, real cc) {
    using V = typename vec2<real>::type;
    V dj, dk;
    dj.x = P.nj.x - P.aj.x; dj.y = P.nj.y - P.aj.y;
    dk.x = P.nk.x - P.ak.x; dk.y = P.nk.y - P.ak.y;
    const V t1 = cmulc(dj, f.hj), t2 = cmulc(dk, f.hk);
    const V djdk = cmulc(dj, dk);  // conj(dj) dk
    V cdjcdk;                      // conj(dj) conj(dk)
    cdjcdk.x = dj.x * dk.x - dj.y * dk.y;
    cdjcdk.y = -(dj.x * dk.y + dj.y * dk.x);
    const V t3 = cmul(djdk, f.B), t4 = cmul(cdjcdk, f.A);
    return -cc * (t1.x + t2.x + t3.x + t4.x);
}

// Update trace: one chain's record of the traced update and its state before the update (modes j and k from
// the proposal's old amplitudes: the other warps may already have written the new ones).
template <typename real, int RS>
__device__ __noinline__ void trace_write(double *trace, int n_chains, int64_t a_off, int chain0, int N, uint32_t id,
                                         int j, int k, Partials<real> f, Proposal<real> P, real dH, bool acc,
                                         real beta, double E, const typename vec2<real>::type *as, int c) {
    using V = typename vec2<real>::type;
    double *rec = trace + (int64_t)id * kTraceRec;
    const double v[kTraceRec] = {(double)j, (double)k, (double)f.hj.x, (double)f.hj.y, (double)f.hk.x,
                                 (double)f.hk.y, (double)f.B.x, (double)f.B.y, (double)f.A.x, (double)f.A.y,
                                 (double)P.nj.x, (double)P.nj.y, (double)P.nk.x, (double)P.nk.y, (double)P.U,
                                 (double)dH, acc ? 1.0 : 0.0, (double)beta, E, 1.0};
    for (int e = 0; e < kTraceRec; ++e) rec[e] = v[e];
    double2 *st = reinterpret_cast<double2 *>(trace + (int64_t)n_chains * kTraceRec) + a_off +
                  (int64_t)(id - (uint32_t)chain0) * N;
    for (int x = 0; x < N; ++x) {
        const V a = (x == j) ? P.aj : (x == k) ? P.ak : as[(x + APAD) * RS + c];
        st[x] = make_double2((double)a.x, (double)a.y);
    }
}

__device__ __forceinline__ bool metropolis_accept(float dH, float beta, float U) {
    return dH <= 0.0f || U < expf(-beta * dH);
}
__device__ __forceinline__ bool metropolis_accept(double dH, double beta, double U) {
    return dH <= 0.0 || U < exp(-beta * dH);
}

// ------------------------------------------------------------------------------------------------
// The persistent sweep kernel.  NCW consumer warps + 1 producer warp.  A consumer lane is
// (chain c = lane % G, worker q = lane / G); worker w = warp * (32/G) + q takes block w of every
// chunk of CB = NCW*32/G blocks.  The producer (copy) warp streams the J runs of j and k, chunk by chunk,
// into a ring of NST stages, and fills one slot per update of a second ring (kBD slots): the update's B_jk
// couplings (FP32, N >= 48) and the random part of every chain's proposal (8 chains per block).  Work units = (group, run of sweeps) come from a ticket counter; a unit
// waits (bounded) until the previous run of its group has been written back.
// Ring depth: as many stages as fit next to the amplitude and window tables of the largest N (up to kNstMax), so
// that the copies of a chunk are issued several chunks ahead of its use (L2 misses of the coupling runs).
constexpr int kNstMax = 6, kNstMin = 2;
// Per-update slots (B_jk couplings for N >= 48 on the FP32 path, proposal draws with 8 chains per block): the copy
// warp fills an update's slot before it streams the update's coupling runs, up to kBD updates ahead of the field
// warps.
constexpr int kBD = 4;

template <typename real, int G, int NCW> struct SweepShape {
    static constexpr int WPW = 32 / G;
    static constexpr int NW = NCW * WPW;
    static constexpr int CB = NW;
    static constexpr int RS = RowStride<real, G>::value;
    static constexpr int NTHREADS = (NCW + 1) * 32;
    static constexpr int JS = JStride<real>::value;
    static constexpr size_t stage_bytes = (size_t)2 * CB * JS * sizeof(real);
    static constexpr bool PACKED = sizeof(real) == 4;  // packed-FP32 block arithmetic (every FP32 shape)
};

// Shared memory of the sweep kernel without the coupling ring.
template <typename real, int G, int NCW> size_t sweep_fixed_bytes(int maxN) {
    using Sh = SweepShape<real, G, NCW>;
    using V = typename vec2<real>::type;
    size_t b = 0;
    b += 2 * (kNstMax + kBD) * sizeof(uint64_t);                          // mbarriers
    b = (b + 127) / 128 * 128;
    b += (size_t)(maxN + 2 * APAD) * Sh::RS * sizeof(V);                  // amplitudes
    if (Sh::PACKED) b += (size_t)(maxN + 2 * APAD) * G * sizeof(float4);      // window table
    if (kGatherB<real, G>) b += (size_t)kBD * maxN * sizeof(real);            // gathered B_jk couplings
    b += (size_t)2 * NCW * G * 8 * sizeof(real);                          // reduction, double-buffered
    if (kCopyDraws<G>) b += (size_t)kBD * G * sizeof(ProposalDraw<real>);  // proposal draws of kBD updates
    b += (size_t)2 * G * sizeof(Proposal<real>) + 16;                     // proposals, double-buffered
    b += (size_t)G * (sizeof(double) + sizeof(real) + 2 * sizeof(uint32_t) + sizeof(unsigned long long));
    b += (size_t)(2 * 128 + 8) * sizeof(int);                             // bo / xtlo tables
    b += (size_t)(maxN / 2) * sizeof(int);                                // pair sequence of a sweep
    b += 64;
    return b;
}

// Ring stages for the largest N within `limit` bytes of shared memory per block (0 when fewer than kNstMin fit).
template <typename real, int G, int NCW> int sweep_stages(int maxN, size_t limit) {
    const size_t fixed = sweep_fixed_bytes<real, G, NCW>(maxN), st = SweepShape<real, G, NCW>::stage_bytes;
    if (fixed + kNstMin * st > limit) return 0;
    const size_t n = (limit - fixed) / st;
    return n > (size_t)kNstMax ? kNstMax : (int)n;
}

template <typename real, int G, int NCW> size_t sweep_smem_bytes(int maxN, int nst) {
    return sweep_fixed_bytes<real, G, NCW>(maxN) + (size_t)nst * SweepShape<real, G, NCW>::stage_bytes;
}

template <typename real, int G, int NCW>
__global__ void __launch_bounds__((NCW + 1) * 32, 1) sweep_kernel(SweepParams prm) {
    using Sh = SweepShape<real, G, NCW>;
    using V = typename vec2<real>::type;
    constexpr int RS = Sh::RS, CB = Sh::CB, WPW = Sh::WPW, JS = Sh::JS, NW = Sh::NW;
    const int NST = prm.nst;  // ring stages (kNstMin .. kNstMax), chosen by the launcher for the largest N
    constexpr int NCT = NCW * 32;  // consumer threads
    // decision step (see the end of an update): 16 chains per block spread it over 8 lanes per chain, 32 chains
    // leave it to warp 0, 8 chains take it redundantly in every warp
    constexpr bool kSpread = G == 16;
    constexpr bool kOneDecider = G == 32;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + kNstMax;
    uint64_t *bfull = empty + kNstMax;  // B-coupling buffers: filled (32 copy-warp lanes) / read (NCW warps)
    uint64_t *bempty = bfull + kBD;
    size_t off = (2 * (kNstMax + kBD) * sizeof(uint64_t) + 127) / 128 * 128;
    real *ring = reinterpret_cast<real *>(smem + off);
    off += NST * Sh::stage_bytes;
    V *as = reinterpret_cast<V *>(smem + off);
    off += (size_t)(prm.maxN + 2 * APAD) * RS * sizeof(V);
    float4 *awin = nullptr;
    if (Sh::PACKED) {
        awin = reinterpret_cast<float4 *>(smem + off);
        off += (size_t)(prm.maxN + 2 * APAD) * G * sizeof(float4);
    }
    real *bvals = nullptr;  // [kBD][maxN]: B_jk couplings of an update, s = max(j,k) + i
    if (kGatherB<real, G>) {
        bvals = reinterpret_cast<real *>(smem + off);
        off += (size_t)kBD * prm.maxN * sizeof(real);
    }
    real *red = reinterpret_cast<real *>(smem + off);
    off += (size_t)2 * NCW * G * 8 * sizeof(real);
    off = (off + 15) / 16 * 16;
    ProposalDraw<real> *pdraw = nullptr;  // [kBD][G]
    if (kCopyDraws<G>) {
        pdraw = reinterpret_cast<ProposalDraw<real> *>(smem + off);
        off += (size_t)kBD * G * sizeof(ProposalDraw<real>);
    }
    Proposal<real> *prop = reinterpret_cast<Proposal<real> *>(smem + off);
    off += (size_t)2 * G * sizeof(Proposal<real>);
    double *cE = reinterpret_cast<double *>(smem + off);
    off += G * sizeof(double);
    real *cBeta = reinterpret_cast<real *>(smem + off);
    off += G * sizeof(real);
    uint32_t *cId = reinterpret_cast<uint32_t *>(smem + off);
    off += G * sizeof(uint32_t);
    uint32_t *cAcc = reinterpret_cast<uint32_t *>(smem + off);
    off += G * sizeof(uint32_t);
    off = (off + 7) / 8 * 8;
    unsigned long long *cAtt = reinterpret_cast<unsigned long long *>(smem + off);
    off += G * sizeof(unsigned long long);
    int *s_bo = reinterpret_cast<int *>(smem + off);
    off += 129 * sizeof(int);
    int *s_xtlo = reinterpret_cast<int *>(smem + off);
    off += 129 * sizeof(int);
    int *s_unit = reinterpret_cast<int *>(smem + off);  // [0] group, [1] chunk, [2] abort
    volatile int *abort_flag = s_unit + 2;
    int *s_pair = s_unit + 4;  // (j | k << 16) of every update of the current sweep

    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const bool producer = (warp == NCW);
    const int c = lane % G, wq = lane / G;
    // warp 0 also draws the proposals, so it takes the last workers of a chunk: it is the one left without a
    // block when an update's last chunk is not full
    const int worker = (warp == 0 ? NCW - 1 : warp - 1) * WPW + wq;

    if (tid == 0) {
        for (int i = 0; i < NST; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NCW);
        }
        for (int i = 0; i < kBD; ++i) {
            mbar_init(&bfull[i], 32);
            mbar_init(&bempty[i], NCW);
        }
        s_unit[2] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();

    const long long sweep_base = prm.ctl->sweep_base;
    const int n_sweeps = prm.n_sweeps, spu = prm.sweeps_per_unit;
    const int chunks_per_group = (n_sweeps + spu - 1) / spu;
    const unsigned total_units = (unsigned)chunks_per_group * (unsigned)prm.n_groups;
    const real *J = reinterpret_cast<const real *>(prm.J);
    V *A = reinterpret_cast<V *>(prm.a);
    uint32_t q = 0;  // global chunk counter (ring position)
    // ring stage of chunk q (q mod NST) and the parity of its pass through the ring, advanced with q (NST is a
    // launch parameter: no division per chunk)
    int rst = 0;
    uint32_t rph = 0;
    int red_par = 0;
    uint32_t bcnt = 0;  // updates with gathered B couplings so far (buffer bcnt % kBD, phase (bcnt / kBD) & 1)

    for (;;) {
        __syncthreads();
        if (tid == 0) {
            int g = -1, ci = 0;
            if (!*abort_flag) {
                const unsigned t = atomicAdd(&prm.ctl->ticket, 1u);
                if (t < total_units) {
                    g = (int)(t % (unsigned)prm.n_groups);
                    ci = (int)(t / (unsigned)prm.n_groups);
                    // wait until the previous run of this group is written back
                    const unsigned long long t0 = global_ns();
                    while (true) {
                        int v;
                        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(prm.progress + g) : "memory");
                        if (v >= ci) break;
                        if (global_ns() - t0 > kWaitNs) { record_error(prm.ctl, kErrTimeout, 1); *abort_flag = 1; g = -1; break; }
                        __nanosleep(256);
                    }
                }
            }
            s_unit[0] = g; s_unit[1] = ci;
        }
        __syncthreads();
        const int g = s_unit[0], ci = s_unit[1];
        if (g < 0) break;
        const GroupDev gr = prm.groups[g];
        const SampleDev sd = prm.samples[gr.sample];
        const int N = sd.N;
        const int sw0 = ci * spu, sw1 = min(n_sweeps, sw0 + spu);
        const bool gatherB = kGatherB<real, G> && N >= kGatherBMinN;
        const bool useSlot = kCopyDraws<G> || gatherB;  // the copy warp fills a slot for every update

        // ---- unit set-up: tables, chain metadata, amplitudes (consumers); producer starts streaming
        if (!producer) {
            for (int i = tid; i <= sd.ST; i += NCT) s_bo[i] = prm.bo[sd.tab_off + i];
            for (int i = tid; i < sd.ST; i += NCT) s_xtlo[i] = prm.xtlo[sd.tab_off + i];
            if (tid < G) {
                const int slot = gr.chain0 + tid;
                if (tid < gr.count) {
                    const int t = prm.label[slot];
                    const int r = (slot - sd.chain0) / prm.nT;
                    cE[tid] = __ldcg(prm.E + slot);
                    cBeta[tid] = (real)prm.beta[t];
                    cId[tid] = (uint32_t)((gr.sample * prm.R + r) * prm.nT + t);
                } else {
                    cE[tid] = 0.0; cBeta[tid] = real(0); cId[tid] = 0u;
                }
                cAcc[tid] = 0u; cAtt[tid] = 0ull;
            }
            const int rows = N + 2 * APAD;
            for (int i = tid; i < rows * G; i += NCT) {
                const int x = i / G - APAD, cc = i % G;
                V v; v.x = v.y = real(0);
                if (x >= 0 && x < N && cc < gr.count) {
                    const V *src = A + sd.a_off + (int64_t)(gr.chain0 - sd.chain0 + cc) * N + x;
                    if (sizeof(real) == 4) {
                        const float2 t = __ldcg(reinterpret_cast<const float2 *>(src));
                        v.x = (real)t.x; v.y = (real)t.y;
                    } else {
                        const double2 t = __ldcg(reinterpret_cast<const double2 *>(src));
                        v.x = (real)t.x; v.y = (real)t.y;
                    }
                }
                as[(x + APAD) * RS + cc] = v;
            }
            named_bar(1, NCT);
            if (Sh::PACKED) {
                for (int i = tid; i < rows * G; i += NCT)
                    packed_rows<RS>(reinterpret_cast<const float2 *>(as), awin, G, i / G, rows, i % G);
                named_bar(1, NCT);
            }
        }

        if (producer) {
            // ---------------- producer warp: stream J runs of (j,k) for every update of the unit
            const int *bo_g = prm.bo + sd.tab_off;
            const int *xtlo_g = prm.xtlo + sd.tab_off;
            // identity of chain `lane` of the group (the Philox stream of its proposals): (sample, replica,
            // temperature index its slot holds)
            uint32_t pid = 0u;
            if (lane < gr.count) {
                const int slot = gr.chain0 + lane;
                pid = (uint32_t)((gr.sample * prm.R + (slot - sd.chain0) / prm.nT) * prm.nT + prm.label[slot]);
            }
            bool stop = false;
            for (int sw = sw0; sw < sw1 && !stop; ++sw) {
                const uint32_t sweep = (uint32_t)(sweep_base + sw);
                for (int u = 0; u < N / 2 && !stop; ++u) {
                    stop = __shfl_sync(0xffffffffu, *abort_flag, 0) != 0;  // warp-uniform
                    if (stop) break;
                    int j, k;
                    pair_jk(prm.seed, (uint32_t)gr.sample, sweep, (uint32_t)u, N, j, k);
                    const Ranges Rg = update_ranges(sd, bo_g, prm.mode_blk + sd.mode_off, j, k);
                    if (useSlot) {
                        // the update's slot (kBD in a ring, up to kBD updates ahead of the field warps): the random
                        // part of every chain's proposal (8 chains per block; lane = chain) and, for large N, the B_jk couplings
                        // J_j[s][{k, s-k}], s in [max(j,k), min(j,k) + N), gathered from L2 by the 32 lanes
                        const int slot = (int)(bcnt % kBD);
                        const uint32_t bph = (bcnt / kBD) & 1u;
                        ++bcnt;
                        if (mbar_wait_bounded(&bempty[slot], bph ^ 1u, prm.ctl, 4, abort_flag)) {
                            if (kCopyDraws<G> && lane < gr.count)
                                pdraw[slot * G + lane] = draw_proposal<real>(prm.seed, pid, sweep, (uint32_t)u);
                            if (kGatherB<real, G> && gatherB) {
                                const int sB0 = max(j, k), nB = min(j, k) + N - sB0;
                                real *bv = bvals + (size_t)slot * prm.maxN;
                                for (int i = lane; i < nB; i += 32)
                                    bv[i] = b_coupling<real>(J, bo_g, xtlo_g, Rg, sB0 + i, k);
                            }
                        }
                        mbar_arrive(&bfull[slot]);
                    }
                    for (int cb = Rg.ulo; cb < Rg.uhi; cb += CB, ++q, rph ^= (++rst == NST) ? 1u : 0u, rst = (rst == NST) ? 0 : rst) {
                        const int stage = rst;
                        const uint32_t ph = rph;
                        if (lane == 0) {
                            const bool ok = mbar_wait_bounded(&empty[stage], ph ^ 1u, prm.ctl, 2, abort_flag);
                            const int ce = min(cb + CB, Rg.uhi);
                            const int a0 = max(cb, Rg.jlo), a1 = min(ce, Rg.jhi);
                            const int b0 = max(cb, Rg.klo), b1 = min(ce, Rg.khi);
                            const uint32_t bj = a1 > a0 ? (uint32_t)(a1 - a0) * JS * sizeof(real) : 0u;
                            const uint32_t bk = b1 > b0 ? (uint32_t)(b1 - b0) * JS * sizeof(real) : 0u;
                            real *st_j = ring + (size_t)stage * 2 * CB * JS;
                            real *st_k = st_j + (size_t)CB * JS;
                            if (ok) mbar_arrive_expect_tx(&full[stage], bj + bk);
                            if (ok && bj) bulk_g2s(st_j + (size_t)(a0 - cb) * JS, J + (Rg.jg + (a0 - Rg.jlo)) * JS, bj, &full[stage]);
                            if (ok && bk) bulk_g2s(st_k + (size_t)(b0 - cb) * JS, J + (Rg.kg + (b0 - Rg.klo)) * JS, bk, &full[stage]);
                        }
                        __syncwarp();
                    }
                }
            }
        } else {
            // ---------------- consumer warps
            const int *mode_blk = prm.mode_blk + sd.mode_off;
            const uint32_t *binfo = prm.blkinfo + sd.blk_off;
            // update trace: absolute sweep + 1 and update to record (0 = none)
            const long long tr_at = prm.trace ? prm.ctl->trace_at : 0ll;
            const int tr_u = prm.trace ? prm.ctl->trace_update : -1;
            const real cc = (real)prm.cc;
            for (int sw = sw0; sw < sw1; ++sw) {
                const uint32_t sweep = (uint32_t)(sweep_base + sw);
                // the sweep's pair sequence, drawn once per block (every warp has read the previous sweep's
                // last entry before that update's barrier, which every thread here has passed)
                for (int i = tid; i < N / 2; i += NCT) {
                    int pj, pk;
                    pair_jk(prm.seed, (uint32_t)gr.sample, sweep, (uint32_t)i, N, pj, pk);
                    s_pair[i] = pj | (pk << 16);
                }
                named_bar(1, NCT);
                for (int u = 0; u < N / 2; ++u) {
                    const int jk = s_pair[u];
                    const int j = jk & 0xffff, k = jk >> 16;
                    const Ranges Rg = update_ranges(sd, s_bo, mode_blk, j, k);
                    // the update's slot from the copy warp (proposal draws with 8 chains per block, B couplings for
                    // large N); warp 0 puts chain c's proposal into the double-buffered table: finished from the
                    // copy warp's draw, or drawn whole
                    int pslot = 0;
                    uint32_t pph = 0u;
                    if (useSlot) {
                        pslot = (int)(bcnt % kBD);
                        pph = (bcnt / kBD) & 1u;
                        ++bcnt;
                    }
                    Proposal<real> *Pp = prop + red_par * G;
                    if (warp == 0) {
                        if constexpr (kCopyDraws<G>) {
                            const bool dok = mbar_wait_bounded(&bfull[pslot], pph, prm.ctl, 5, abort_flag);
                            if (dok && wq == 0) {
                                const V aj = as[(j + APAD) * RS + c], ak = as[(k + APAD) * RS + c];
                                Pp[c] = finish_proposal<real>(pdraw[pslot * G + c], aj, ak);
                            }
                        } else if (wq == 0) {
                            const V aj = as[(j + APAD) * RS + c], ak = as[(k + APAD) * RS + c];
                            Pp[c] = finish_proposal<real>(draw_proposal<real>(prm.seed, cId[c], sweep, (uint32_t)u), aj, ak);
                        }
                    }
                    Partials<real> pr;
                    pr.zero();
                    PartialsX2 prx;
                    prx.zero();
                    for (int cb = Rg.ulo; cb < Rg.uhi; cb += CB, ++q, rph ^= (++rst == NST) ? 1u : 0u, rst = (rst == NST) ? 0 : rst) {
                        const int stage = rst;
                        const uint32_t ph = rph;
                        // a chunk whose copies have landed is processed (its data are valid even after another
                        // wait gave up); a wait that gives up, or sees the abort flag, skips it
                        const bool landed = mbar_wait_bounded(&full[stage], ph, prm.ctl, 3, abort_flag);
                        const int b = cb + worker;
                        if (b < Rg.uhi && landed) {
                            const uint32_t info = __ldg(binfo + b);
                            const int st = (int)(info >> 16), xt = (int)(info & 0xffffu);
                            const int mode = ((b >= Rg.jlo && b < Rg.jhi) ? 1 : 0) | ((b >= Rg.klo && b < Rg.khi) ? 2 : 0);
                            const real *st_j = ring + (size_t)stage * 2 * CB * JS + (size_t)worker * JS;
                            const real *st_k = st_j + (size_t)CB * JS;
                            if constexpr (Sh::PACKED) {
                                const float2 *asf = reinterpret_cast<const float2 *>(as);
                                const float *fj = reinterpret_cast<const float *>(st_j), *fk = reinterpret_cast<const float *>(st_k);
                                if (gatherB) process_block_x2_dispatch<G, false>(mode, asf, awin, c, st * TS, xt * TX, j, k, N, fj, fk, prx);
                                else process_block_x2_dispatch<G, true>(mode, asf, awin, c, st * TS, xt * TX, j, k, N, fj, fk, prx);
                            } else {
                                if (gatherB) process_block_dispatch<real, RS, false>(mode, as, c, st * TS, xt * TX, j, k, N, st_j, st_k, pr);
                                else process_block_dispatch<real, RS, true>(mode, as, c, st * TS, xt * TX, j, k, N, st_j, st_k, pr);
                            }
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&empty[stage]);
                    }
                    if constexpr (Sh::PACKED) {
                        pr.hj.x = prx.hjx.x + prx.hjx.y;
                        pr.hj.y = (prx.hjy.x + prx.hjy.y) - (prx.hjyn.x + prx.hjyn.y);
                        pr.hk.x = prx.hkx.x + prx.hkx.y;
                        pr.hk.y = (prx.hky.x + prx.hky.y) - (prx.hkyn.x + prx.hkyn.y);
                        pr.B.x = prx.B.x; pr.B.y = prx.B.y;
                        pr.A.x = prx.A.x; pr.A.y = prx.A.y;
                    }
                    // B_jk = sum_s conj(a_{s-j}) J_j[s][{k, s-k}] a_{s-k} over s in [max(j,k), min(j,k)+N) (large N: the
                    // couplings come from the buffer the copy warp filled; worker w takes s = max(j,k) + w + m NW;
                    // for smaller N process_block picks them out of the blocks)
                    if (kGatherB<real, G> && gatherB) {
                        if (mbar_wait_bounded(&bfull[pslot], pph, prm.ctl, 5, abort_flag)) {
                            const real *bv = bvals + (size_t)pslot * prm.maxN;
                            const int sB0 = max(j, k), sB1 = min(j, k) + N;
                            for (int sb = sB0 + worker; sb < sB1; sb += NW)
                                caxpy(pr.B, bv[sb - sB0], cmulc(as[(sb - j + APAD) * RS + c], as[(sb - k + APAD) * RS + c]));
                        }
                    }
                    // every warp is done with the slot (warp 0 copied the proposals out at the update's start)
                    if (useSlot) {
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&bempty[pslot]);
                    }
                    // reduce over the workers of this warp, then across warps through shared memory
                    real v[8] = {pr.hj.x, pr.hj.y, pr.hk.x, pr.hk.y, pr.B.x, pr.B.y, pr.A.x, pr.A.y};
#pragma unroll
                    for (int o = G; o < 32; o <<= 1)
#pragma unroll
                        for (int e = 0; e < 8; ++e) v[e] += __shfl_xor_sync(0xffffffffu, v[e], o);
                    real *rb = red + (size_t)red_par * NCW * G * 8;
                    if constexpr (kSpread) {
                        // layout [warp][chain][value]: the 8 values of one (warp, chain) are consecutive, so that the
                        // reads after the barrier (32 lanes = 4 chains x 8 values of one warp) are 32 consecutive words
                        if (wq == 0) {
                            if constexpr (sizeof(real) == 4) {
                                float4 *d = reinterpret_cast<float4 *>(rb + ((size_t)warp * G + c) * 8);
                                d[0] = make_float4(v[0], v[1], v[2], v[3]);
                                d[1] = make_float4(v[4], v[5], v[6], v[7]);
                            } else {
                                double2 *d = reinterpret_cast<double2 *>(rb + ((size_t)warp * G + c) * 8);
                                d[0] = make_double2(v[0], v[1]); d[1] = make_double2(v[2], v[3]);
                                d[2] = make_double2(v[4], v[5]); d[3] = make_double2(v[6], v[7]);
                            }
                        }
                    } else if constexpr (Sh::PACKED) {
                        // layout [half][warp][chain] of float4: the chains of one (half, warp) are consecutive, so
                        // the stores and the reads after the barrier are free of bank conflicts
                        float4 *rb4 = reinterpret_cast<float4 *>(rb);
                        if (wq == 0) {
                            rb4[(0 * NCW + warp) * G + c] = make_float4(v[0], v[1], v[2], v[3]);
                            rb4[(1 * NCW + warp) * G + c] = make_float4(v[4], v[5], v[6], v[7]);
                        }
                    } else {
                        // layout [e][warp][chain]: the 8 chains of one (e, warp) are consecutive words, so both the
                        // stores below and the reads after the barrier (32 lanes = 4 warps x 8 chains) are free of
                        // bank conflicts
                        if (wq == 0) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) rb[(e * NCW + warp) * G + c] = v[e];
                        }
                    }
                    // packed: the neighbours of j and k for the window rows rewritten on acceptance (modes other
                    // than j and k keep their values during this update)
                    float2 nb[4];
                    if (Sh::PACKED && !kSpread && (!kOneDecider || warp == 0)) {
                        const float2 *asf = reinterpret_cast<const float2 *>(as);
                        nb[0] = asf[(j - 1 + APAD) * RS + c]; nb[1] = asf[(j + 1 + APAD) * RS + c];
                        nb[2] = asf[(k - 1 + APAD) * RS + c]; nb[3] = asf[(k + 1 + APAD) * RS + c];
                    }
                    named_bar(1, NCT);
                    // Decision (measured on GB300, per shape):
                    // - 16 chains per block: 8 lanes per chain, 4 chains per warp, warps in turn.  Lane e of a
                    //   chain's group adds value e over the warps in warp order; the group's first lane gathers
                    //   the 8 totals, decides and writes (+3.7% over warp 0 alone at N = 64);
                    // - 32 chains per block: warp 0 alone forms the totals, decides and writes (every other warp
                    //   would repeat the same reads of all partial sums: NCW x G x 8 words each; the 8-lane
                    //   groups measured 1.5% slower here);
                    // - 8 chains per block: every warp forms the same totals in the same order, takes the same
                    //   decision and writes the same values, with no second barrier (measured faster at N = 256).
                    // With one or more deciding warps a second barrier orders their writes before every warp's next
                    // update.
                    if constexpr (kSpread) {
                        for (int c4 = warp * 4; c4 < G; c4 += NCW * 4) {  // warp-uniform trip count
                            const int cd = c4 + (lane >> 3), e = lane & 7;
                            const bool mine = cd < G, lead = mine && e == 0;
                            // packed: the neighbours of j and k for the window rows rewritten on acceptance (modes
                            // other than j and k keep their values during this update)
                            float2 nbs[4];
                            if (Sh::PACKED && lead) {
                                const float2 *asf = reinterpret_cast<const float2 *>(as);
                                nbs[0] = asf[(j - 1 + APAD) * RS + cd]; nbs[1] = asf[(j + 1 + APAD) * RS + cd];
                                nbs[2] = asf[(k - 1 + APAD) * RS + cd]; nbs[3] = asf[(k + 1 + APAD) * RS + cd];
                            }
                            real s = 0;
                            if (mine) {
#pragma unroll
                                for (int w = 0; w < NCW; ++w) s += rb[((size_t)w * G + cd) * 8 + e];
                            }
                            real t[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i) t[i] = __shfl_sync(0xffffffffu, s, (lane & ~7) | i);
                            if (lead) {
                                Partials<real> f;
                                f.hj.x = t[0]; f.hj.y = t[1]; f.hk.x = t[2]; f.hk.y = t[3];
                                f.B.x = t[4]; f.B.y = t[5]; f.A.x = t[6]; f.A.y = t[7];
                                const Proposal<real> P = Pp[cd];
                                const real dH = delta_h<real>(P, f, cc);
                                const bool live = cd < gr.count;
                                const bool acc = live && metropolis_accept(dH, cBeta[cd], P.U);
                                if (tr_at == sweep_base + sw + 1 && u == tr_u && live)
                                    trace_write<real, RS>(prm.trace, prm.n_chains, sd.a_off, sd.chain0, N, cId[cd], j, k, f, P,
                                                          dH, acc, cBeta[cd], cE[cd], as, cd);
                                if (acc) {
                                    as[(j + APAD) * RS + cd] = P.nj;
                                    as[(k + APAD) * RS + cd] = P.nk;
                                    if constexpr (Sh::PACKED) {
                                        const float2 nj = P.nj, nk = P.nk;
                                        const float2 jm = (j - 1 == k) ? nk : nbs[0], jp = (j + 1 == k) ? nk : nbs[1];
                                        const float2 km = (k - 1 == j) ? nj : nbs[2], kp = (k + 1 == j) ? nj : nbs[3];
                                        awin[(j - 1 + APAD) * G + cd] = make_float4(jm.x, nj.x, jm.y, nj.y);
                                        awin[(j + APAD) * G + cd] = make_float4(nj.x, jp.x, nj.y, jp.y);
                                        awin[(k - 1 + APAD) * G + cd] = make_float4(km.x, nk.x, km.y, nk.y);
                                        awin[(k + APAD) * G + cd] = make_float4(nk.x, kp.x, nk.y, kp.y);
                                    }
                                }
                                if (live) {
                                    if (acc) { cE[cd] += (double)dH; cAcc[cd] += 1u; }
                                    cAtt[cd] += 1ull;
                                }
                            }
                        }
                    } else if (!kOneDecider || warp == 0) {
                        // lane (c, wq) adds the partials of warps wq, wq + WPW, ...: the trip count is the
                        // same on every lane (predicated body), so the warp is converged at the shuffles
                        real t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
                        for (int w0 = 0; w0 < NCW; w0 += WPW) {
                            const int w = w0 + wq;
                            if (w < NCW) {
                                if constexpr (Sh::PACKED) {
                                    const float4 *rb4 = reinterpret_cast<const float4 *>(rb);
                                    const float4 lo = rb4[(0 * NCW + w) * G + c], hi = rb4[(1 * NCW + w) * G + c];
                                    t[0] += lo.x; t[1] += lo.y; t[2] += lo.z; t[3] += lo.w;
                                    t[4] += hi.x; t[5] += hi.y; t[6] += hi.z; t[7] += hi.w;
                                } else {
#pragma unroll
                                    for (int e = 0; e < 8; ++e) t[e] += rb[(e * NCW + w) * G + c];
                                }
                            }
                        }
                        __syncwarp();
#pragma unroll
                        for (int o = G; o < 32; o <<= 1)
#pragma unroll
                            for (int e = 0; e < 8; ++e) t[e] += __shfl_xor_sync(0xffffffffu, t[e], o);
                        if (wq == 0) {
                            Partials<real> f;
                            f.hj.x = t[0]; f.hj.y = t[1]; f.hk.x = t[2]; f.hk.y = t[3];
                            f.B.x = t[4]; f.B.y = t[5]; f.A.x = t[6]; f.A.y = t[7];
                            const Proposal<real> P = Pp[c];
                            const real dH = delta_h<real>(P, f, cc);
                            const bool acc = (c < gr.count) && metropolis_accept(dH, cBeta[c], P.U);
                            if (tr_at == sweep_base + sw + 1 && u == tr_u && warp == 0 && c < gr.count)
                                trace_write<real, RS>(prm.trace, prm.n_chains, sd.a_off, sd.chain0, N, cId[c], j, k, f, P, dH, acc,
                                                      cBeta[c], cE[c], as, c);
                            if (acc) {
                                as[(j + APAD) * RS + c] = P.nj;
                                as[(k + APAD) * RS + c] = P.nk;
                                if constexpr (Sh::PACKED) {
                                    // the window rows j-1, j, k-1, k from registers: row R holds (a_R, a_{R+1});
                                    // a neighbour that is the other updated mode takes its new value
                                    const float2 nj = P.nj, nk = P.nk;
                                    const float2 jm = (j - 1 == k) ? nk : nb[0], jp = (j + 1 == k) ? nk : nb[1];
                                    const float2 km = (k - 1 == j) ? nj : nb[2], kp = (k + 1 == j) ? nj : nb[3];
                                    awin[(j - 1 + APAD) * G + c] = make_float4(jm.x, nj.x, jm.y, nj.y);
                                    awin[(j + APAD) * G + c] = make_float4(nj.x, jp.x, nj.y, jp.y);
                                    awin[(k - 1 + APAD) * G + c] = make_float4(km.x, nk.x, km.y, nk.y);
                                    awin[(k + APAD) * G + c] = make_float4(nk.x, kp.x, nk.y, kp.y);
                                }
                            }
                            if (warp == 0 && c < gr.count) {
                                if (acc) { cE[c] += (double)dH; cAcc[c] += 1u; }
                                cAtt[c] += 1ull;
                            }
                        }
                    }
                    red_par ^= 1;
                    if constexpr (kOneDecider || kSpread) named_bar(1, NCT);
                    else __syncwarp();
                }
                // interior measurement point: snapshot amplitudes and energies
                const long long done = sweep_base + sw + 1;
                if (prm.measure_every > 0 && done % prm.measure_every == 0 && sw + 1 < n_sweeps) {
                    named_bar(1, NCT);
                    // snapshot index = number of measurement points in (sweep_base, done], minus one
                    const int kk = (int)(done / prm.measure_every - sweep_base / prm.measure_every - 1);
                    if (kk >= 0 && kk < prm.n_snap_max) {
                        V *dst = reinterpret_cast<V *>(prm.snap_a) + (int64_t)kk * prm.a_total + sd.a_off +
                                 (int64_t)(gr.chain0 - sd.chain0) * N;
                        for (int i = tid; i < N * gr.count; i += NCT) {
                            const int cc2 = i / N, x = i % N;
                            dst[(int64_t)cc2 * N + x] = as[(x + APAD) * RS + cc2];
                        }
                        if (tid < gr.count) prm.snap_E[(int64_t)kk * prm.n_chains + gr.chain0 + tid] = cE[tid];
                    }
                    named_bar(1, NCT);
                }
            }
            // ---- write back the group's state and counters
            named_bar(1, NCT);
            for (int i = tid; i < N * gr.count; i += NCT) {
                const int cc2 = i / N, x = i % N;
                V *dst = A + sd.a_off + (int64_t)(gr.chain0 - sd.chain0 + cc2) * N + x;
                __stcg(dst, as[(x + APAD) * RS + cc2]);
            }
            if (tid < gr.count) {
                const int slot = gr.chain0 + tid;
                __stcg(prm.E + slot, cE[tid]);
                prm.mc_acc[slot] += cAcc[tid];
                prm.mc_att[slot] += cAtt[tid];
            }
            __threadfence();
            named_bar(1, NCT);
            if (tid == 0) {
                asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(prm.progress + g), "r"(ci + 1) : "memory");
            }
        }
    }
    // never leave bulk copies in flight behind an exiting block (only possible after an abort)
    if (producer && lane == 0) {
        const uint32_t first = q > (uint32_t)NST ? q - NST : 0u;
        for (uint32_t qq = first; qq < q; ++qq) {
            const unsigned long long t0 = global_ns();
            while (!mbar_try_wait(&full[qq % NST], (qq / NST) & 1u) && global_ns() - t0 < kWaitNs) {
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Field-only kernel: the same block arithmetic with J read straight from global memory; one thread
// block per group of the chosen sample.  Output: 8 doubles per chain (h_j, h_k, B_jk, A_jk).
template <typename real, int G>
__global__ void fields_kernel(FieldsParams prm) {
    using V = typename vec2<real>::type;
    constexpr int RS = RowStride<real, G>::value, NCW = 4, WPW = 32 / G, NW = NCW * WPW;
    extern __shared__ __align__(128) unsigned char smem[];
    V *as = reinterpret_cast<V *>(smem);
    const GroupDev gr = prm.groups[prm.group0 + blockIdx.x];
    const SampleDev sd = prm.samples[gr.sample];
    const int N = sd.N, tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int c = lane % G, worker = warp * WPW + lane / G;
    const V *A = reinterpret_cast<const V *>(prm.a);
    real *red = reinterpret_cast<real *>(smem + (size_t)(N + 2 * APAD) * RS * sizeof(V));
    for (int i = tid; i < (N + 2 * APAD) * G; i += blockDim.x) {
        const int x = i / G - APAD, cc = i % G;
        V v; v.x = v.y = real(0);
        if (x >= 0 && x < N && cc < gr.count) v = A[sd.a_off + (int64_t)(gr.chain0 - sd.chain0 + cc) * N + x];
        as[(x + APAD) * RS + cc] = v;
    }
    __syncthreads();
    const int j = prm.j, k = prm.k;
    const Ranges Rg = update_ranges(sd, prm.bo + sd.tab_off, prm.mode_blk + sd.mode_off, j, k);
    const real *J = reinterpret_cast<const real *>(prm.J);
    Partials<real> pr;
    pr.zero();
    for (int b = Rg.ulo + worker; b < Rg.uhi; b += NW) {
        const uint32_t info = prm.blkinfo[sd.blk_off + b];
        const int st = (int)(info >> 16), xt = (int)(info & 0xffffu);
        const int mode = ((b >= Rg.jlo && b < Rg.jhi) ? 1 : 0) | ((b >= Rg.klo && b < Rg.khi) ? 2 : 0);
        const real *Jj = J + (Rg.jg + (b - Rg.jlo)) * JStride<real>::value;
        const real *Jk = J + (Rg.kg + (b - Rg.klo)) * JStride<real>::value;
        process_block_dispatch<real, RS, true>(mode, as, c, st * TS, xt * TX, j, k, N, Jj, Jk, pr);
    }
    real v[8] = {pr.hj.x, pr.hj.y, pr.hk.x, pr.hk.y, pr.B.x, pr.B.y, pr.A.x, pr.A.y};
#pragma unroll
    for (int o = G; o < 32; o <<= 1)
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] += __shfl_xor_sync(0xffffffffu, v[e], o);
    if (lane < G)
        for (int e = 0; e < 8; ++e) red[(warp * G + c) * 8 + e] = v[e];
    __syncthreads();
    if (tid < G * 8 && tid / 8 < gr.count) {
        const int cc = tid / 8, e = tid % 8;
        double t = 0.0;
        for (int w = 0; w < NCW; ++w) t += (double)red[(w * G + cc) * 8 + e];
        prm.out[(int64_t)(gr.chain0 - sd.chain0 + cc) * 8 + e] = t;
    }
}

// ------------------------------------------------------------------------------------------------
// Full energy (resync).  With the partial fields h^>_x = sum_{m > x} conj(a_m) acc^>_x[x+m], where acc^>
// keeps only the pairs {p, q} of row x+m whose smaller mode (the block column) exceeds x,
//     H = -cc sum_x Re( conj(a_x) h^>_x ),
// which visits every quadruplet once, at its smallest mode x (partner m: the largest; the pair {p, q} of
// the two middle modes has p > x).  Blocks whose columns all lie at or below x are skipped.  Products and
// row sums in `real`, per-block sums accumulated in FP64.  A group's blocks are split over prm.parts thread
// blocks (block b of part p takes the work items p NW + worker, stepping by parts NW); each writes its per-chain
// FP64 sums to prm.part and energy_sum_kernel adds the parts in order.  With renorm != 0, renorm_kernel first
// rescales every chain onto sum |a|^4 = N.  The kernel waits on coupling loads from L2, so it runs as many
// warps per SM as fit: 3 blocks of 256 threads (FP32; 2 for FP64) and about 8 blocks per SM in all.  Measured on
// GB300 (resync of the N = 256 bench workload, 192 groups): 2.81 ms with one block per group, 2.08 ms with about
// 4 blocks per SM at 2 per SM, 1.45 ms now; batched N = 64: 0.166 -> 0.12 ms, ragged batch: 0.58 -> 0.24 ms.
template <typename real, int G>
__global__ void __launch_bounds__(256) renorm_kernel(EnergyParams prm) {
    using V = typename vec2<real>::type;
    const GroupDev gr = prm.groups[blockIdx.x];
    const SampleDev sd = prm.samples[gr.sample];
    const int N = sd.N, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    V *Ag = reinterpret_cast<V *>(prm.a);
    // sum |a|^4 per chain in FP64 (one warp per chain, round robin), then the rescaled amplitudes
    for (int cc = warp; cc < gr.count; cc += 8) {
        V *a = Ag + sd.a_off + (int64_t)(gr.chain0 - sd.chain0 + cc) * N;
        double s4 = 0.0;
        for (int x = lane; x < N; x += 32) {
            const V v = a[x];
            const double u = (double)v.x * v.x + (double)v.y * v.y;
            s4 += u * u;
        }
        for (int o = 16; o; o >>= 1) s4 += __shfl_xor_sync(0xffffffffu, s4, o);
        if (lane == 0 && (!(s4 > 0.0) || !isfinite(s4))) record_error(prm.ctl, kErrNaN, 10);
        const double f = sqrt(sqrt((double)N / s4));
        for (int x = lane; x < N; x += 32) {
            V v = a[x];
            v.x = (real)((double)v.x * f); v.y = (real)((double)v.y * f);
            a[x] = v;
        }
    }
}

template <typename real, int G>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 3 : 2) energy_kernel(EnergyParams prm) {
    using V = typename vec2<real>::type;
    constexpr int RS = RowStride<real, G>::value, NCW = 8, WPW = 32 / G, NW = NCW * WPW;
    extern __shared__ __align__(128) unsigned char smem[];
    const int part = (int)(blockIdx.x % (unsigned)prm.parts);
    const GroupDev gr = prm.groups[blockIdx.x / (unsigned)prm.parts];
    const SampleDev sd = prm.samples[gr.sample];
    const int N = sd.N, tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int c = lane % G, worker = warp * WPW + lane / G;
    V *as = reinterpret_cast<V *>(smem);
    double *dred = reinterpret_cast<double *>(smem + (size_t)(N + 2 * APAD) * RS * sizeof(V));
    V *Ag = reinterpret_cast<V *>(prm.a);
    for (int i = tid; i < (N + 2 * APAD) * G; i += blockDim.x) {
        const int x = i / G - APAD, cc = i % G;
        V v; v.x = v.y = real(0);
        if (x >= 0 && x < N && cc < gr.count) v = Ag[sd.a_off + (int64_t)(gr.chain0 - sd.chain0 + cc) * N + x];
        as[(x + APAD) * RS + cc] = v;
    }
    __syncthreads();
    const real *J = reinterpret_cast<const real *>(prm.J);
    const int *bo = prm.bo + sd.tab_off;
    const int *mode_blk = prm.mode_blk + sd.mode_off;
    const int *ebo = prm.ebo + sd.mode_off;  // prefix over x of the blocks with rows s > 2x
    const int total = ebo[N];
    double e = 0.0;
    int x = 0;
    for (int it = part * NW + worker; it < total; it += NW * prm.parts) {
        while (ebo[x + 1] <= it) ++x;
        const int stlo = x / TS;
        const int sta = (2 * x + 1) / TS;
        const int b = bo[sta] + (it - ebo[x]);
        const uint32_t info = prm.blkinfo[sd.blk_off + b];
        const int st = (int)(info >> 16), xt = (int)(info & 0xffffu);
        const real *Jx = J + (sd.J_off + mode_blk[x] + (b - bo[stlo])) * JStride<real>::value;
        const int s0 = st * TS, x0 = xt * TX;
        if (x0 + TX - 1 <= x) continue;  // every pair of the block has its smaller mode <= x
        V ax[TX], ay[TS + TX - 1], acc[TS];
#pragma unroll
        for (int i = 0; i < TX; ++i) ax[i] = as[(x0 + i + APAD) * RS + c];
        const int ybase = s0 - x0 - (TX - 1) + APAD;
#pragma unroll
        for (int d = 0; d < TS + TX - 1; ++d) ay[d] = as[(ybase + d) * RS + c];
#pragma unroll
        for (int r = 0; r < TS; ++r) acc[r].x = acc[r].y = real(0);
#pragma unroll
        for (int i = 0; i < TX; ++i) {
            if (x0 + i <= x) continue;  // pairs whose smaller mode is <= x: counted at that mode
            JRow<real> jc;
            jc.load(Jx + i * TS);
#pragma unroll
            for (int r = 0; r < TS; ++r) caxpy(acc[r], jc.v[r], cmul(ax[i], ay[r - i + TX - 1]));
        }
        const V axx = as[(x + APAD) * RS + c];
        real blk = real(0);
#pragma unroll
        for (int r = 0; r < TS; ++r) {
            const int m = s0 + r - x;
            if (m > x && m < N) {
                const V zz = cmul(axx, as[(m + APAD) * RS + c]);  // z_{x,m}
                blk += zz.x * acc[r].x + zz.y * acc[r].y;          // Re(conj(z) acc)
            }
        }
        e += (double)blk;
    }
    for (int o = G; o < 32; o <<= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane < G) dred[warp * G + c] = e;
    __syncthreads();
    if (tid < gr.count) {
        double t = 0.0;
        for (int w = 0; w < NCW; ++w) t += dred[w * G + tid];
        prm.part[((size_t)(blockIdx.x / (unsigned)prm.parts) * prm.parts + part) * 32 + tid] = t;
    }
}

// E = -cc (sum of the parts, in part order) per chain of a group; one thread per chain.
__global__ void energy_sum_kernel(EnergyParams prm) {
    const GroupDev gr = prm.groups[blockIdx.x];
    const int c = threadIdx.x;
    if (c >= gr.count) return;
    double t = 0.0;
    for (int p = 0; p < prm.parts; ++p) t += prm.part[((size_t)blockIdx.x * prm.parts + p) * 32 + c];
    const double E = -prm.cc * t;
    if (!isfinite(E)) record_error(prm.ctl, kErrNaN, 11);
    if (prm.E_out) prm.E_out[gr.chain0 + c] = E;
    if (prm.E_state) prm.E_state[gr.chain0 + c] = E;
}

// ------------------------------------------------------------------------------------------------
// host launchers
// Opt-in shared memory per block of the current device.
static size_t smem_limit() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return (size_t)v;
}

template <typename real, int G, int NCW>
static cudaError_t launch_sweep_t(const SweepParams &p, int grid, cudaStream_t s) {
    SweepParams q = p;
    q.nst = sweep_stages<real, G, NCW>(p.maxN, smem_limit());
    if (q.nst < kNstMin) return cudaErrorInvalidConfiguration;
    const size_t sm = sweep_smem_bytes<real, G, NCW>(p.maxN, q.nst);
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<real, G, NCW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    sweep_kernel<real, G, NCW><<<grid, (NCW + 1) * 32, sm, s>>>(q);
    return cudaGetLastError();
}

template <typename real, int G, int NCW>
static int occupancy_t(int maxN) {
    const int nst = sweep_stages<real, G, NCW>(maxN, smem_limit());
    if (nst < kNstMin) return 0;
    const size_t sm = sweep_smem_bytes<real, G, NCW>(maxN, nst);
    if (cudaFuncSetAttribute(sweep_kernel<real, G, NCW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<real, G, NCW>, (NCW + 1) * 32, sm) != cudaSuccess)
        return 0;
    return nb;
}

#define PT_SWEEP_VARIANTS(X)                                          \
    X(float, 8, 7) X(float, 8, 11) X(float, 8, 15)                    \
    X(float, 16, 7) X(float, 16, 11) X(float, 16, 15)                 \
    X(float, 32, 3) X(float, 32, 7) X(float, 32, 9) X(float, 32, 11)  \
    X(double, 8, 7) X(double, 16, 3)

bool sweep_variant_exists(bool dbl, int G, int ncw) {
#define X(T, g, n) if (dbl == (sizeof(T) == 8) && G == g && ncw == n) return true;
    PT_SWEEP_VARIANTS(X)
#undef X
    return false;
}

cudaError_t launch_sweep(bool dbl, int G, int ncw, const SweepParams &p, int grid, cudaStream_t s) {
#define X(T, g, n) \
    if (dbl == (sizeof(T) == 8) && G == g && ncw == n) return launch_sweep_t<T, g, n>(p, grid, s);
    PT_SWEEP_VARIANTS(X)
#undef X
    return cudaErrorInvalidValue;
}

int sweep_occupancy(bool dbl, int G, int ncw, int maxN) {
#define X(T, g, n) \
    if (dbl == (sizeof(T) == 8) && G == g && ncw == n) return occupancy_t<T, g, n>(maxN);
    PT_SWEEP_VARIANTS(X)
#undef X
    return 0;
}

template <typename real, int G>
static cudaError_t launch_fields_t(const FieldsParams &p, int ngroups, int maxN, cudaStream_t s) {
    using V = typename vec2<real>::type;
    const size_t sm = (size_t)(maxN + 2 * APAD) * RowStride<real, G>::value * sizeof(V) + 4 * G * 8 * sizeof(real) + 64;
    cudaError_t e = cudaFuncSetAttribute(fields_kernel<real, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    fields_kernel<real, G><<<ngroups, 128, sm, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fields(bool dbl, int G, const FieldsParams &p, int ngroups, int maxN, cudaStream_t s) {
    if (!dbl) {
        if (G == 8) return launch_fields_t<float, 8>(p, ngroups, maxN, s);
        if (G == 16) return launch_fields_t<float, 16>(p, ngroups, maxN, s);
        if (G == 32) return launch_fields_t<float, 32>(p, ngroups, maxN, s);
    } else {
        if (G == 8) return launch_fields_t<double, 8>(p, ngroups, maxN, s);
        if (G == 16) return launch_fields_t<double, 16>(p, ngroups, maxN, s);
    }
    return cudaErrorInvalidValue;
}

template <typename real, int G>
static cudaError_t launch_energy_t(const EnergyParams &p, int ngroups, int maxN, cudaStream_t s) {
    using V = typename vec2<real>::type;
    const size_t sm = (size_t)(maxN + 2 * APAD) * RowStride<real, G>::value * sizeof(V) + 8 * G * sizeof(double) + 64;
    cudaError_t e = cudaFuncSetAttribute(energy_kernel<real, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (p.parts < 1 || p.parts > kEnergyPartsMax || !p.part) return cudaErrorInvalidValue;
    if (p.renorm) {
        renorm_kernel<real, G><<<ngroups, 256, 0, s>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    energy_kernel<real, G><<<ngroups * p.parts, 256, sm, s>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    energy_sum_kernel<<<ngroups, 32, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_energy(bool dbl, int G, const EnergyParams &p, int ngroups, int maxN, cudaStream_t s) {
    if (!dbl) {
        if (G == 8) return launch_energy_t<float, 8>(p, ngroups, maxN, s);
        if (G == 16) return launch_energy_t<float, 16>(p, ngroups, maxN, s);
        if (G == 32) return launch_energy_t<float, 32>(p, ngroups, maxN, s);
    } else {
        if (G == 8) return launch_energy_t<double, 8>(p, ngroups, maxN, s);
        if (G == 16) return launch_energy_t<double, 16>(p, ngroups, maxN, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace ptgb
