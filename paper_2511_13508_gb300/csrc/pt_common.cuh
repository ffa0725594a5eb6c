// pt_common.cuh -- device helpers and kernel parameter blocks shared by the CUDA translation
// units of the smoothed-cubic Parallel-Tempering engine (arXiv 2511.13508).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ptgb {

// ------------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (x0,x1,x2,x3) -> (hi(M1*x2)^x1^k0, lo(M1*x2), hi(M0*x0)^x3^k1, lo(M0*x0)),
// key bumped by the Weyl increments between rounds.  Written from the published definition.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

// Stream tags of the counter's last word.
constexpr uint32_t kTagInit = 1u, kTagPair = 2u, kTagPropose = 3u, kTagSwap = 4u;

struct u32x4 { uint32_t x, y, z, w; };

__host__ __device__ inline u32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(kPhiloxM0, c0), lo0 = kPhiloxM0 * c0;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c2), lo1 = kPhiloxM1 * c2;
#else
        const uint64_t p0 = (uint64_t)kPhiloxM0 * c0, p1 = (uint64_t)kPhiloxM1 * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += kPhiloxW0; k1 += kPhiloxW1;
    }
    return {c0, c1, c2, c3};
}

__host__ __device__ inline u32x4 draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag) {
    return philox4x32_10(c0, c1, c2, tag, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
}

// uniform in (0,1): (w + 1/2) 2^-32, exact in FP64
__host__ __device__ inline double u01(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

// Pair choice: j = floor(w0 N / 2^32), k = (j + 1 + floor(w1 (N-1) / 2^32)) mod N.
__host__ __device__ inline void pair_jk(uint64_t seed, uint32_t sample, uint32_t sweep, uint32_t update, int N,
                                        int &j, int &k) {
    const u32x4 w = draw(seed, sample, sweep, update, kTagPair);
    const uint32_t jj = (uint32_t)(((uint64_t)w.x * (uint64_t)N) >> 32);
    const uint32_t off = (uint32_t)(((uint64_t)w.y * (uint64_t)(N - 1)) >> 32);
    j = (int)jj;
    k = (int)((jj + 1u + off) % (uint32_t)N);
}

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kHalfPi = 1.5707963267948966192313216916398;

// ------------------------------------------------------------------------------------------------
// complex helpers over float2 / double2
template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };

template <typename T> __host__ __device__ inline typename vec2<T>::type mk2(T x, T y) {
    typename vec2<T>::type r; r.x = x; r.y = y; return r;
}

// ------------------------------------------------------------------------------------------------
// Blocked per-mode coupling store.  Pair sums s = x + y (x < y) are tiled in TS-row s-tiles and
// TX-column x-tiles; block (st, xt) holds rows s in [st*TS, st*TS+TS) and x in [xt*TX, xt*TX+TX).
// For mode l, J_l[s][x] = J of the quadruplet {l, s-l, x, s-x} (0 where that is not a quadruplet),
// and the blocks of l are those of the s-tiles meeting [l, l+N-1]: a contiguous run of the sample's
// block list.
constexpr int TS = 8, TX = 8, TBLK = TS * TX;
// A block is stored column-major ([i][r], i = x offset, r = s offset) followed by 16 bytes of padding,
// so that blocks that sit next to each other in shared memory start in different banks.
template <typename real> struct JStride { static constexpr int value = TBLK + 16 / (int)sizeof(real); };
constexpr int APAD = 16;  // zero rows below and above the amplitude table in shared memory

// Per-sample descriptor (device copy).
struct SampleDev {
    int N;
    int ST;          // number of s-tiles
    int nblk;        // blocks in the sample's block list
    int chains;      // R * n_T
    int chain0;      // first chain slot of the sample
    int tab_off;     // offset of this sample in the bo / xtlo tables (ST+1 entries reserved)
    int blk_off;     // offset of this sample in the blkinfo table (nblk entries)
    int mode_off;    // offset of this sample in the mode_blk table (N+1 entries)
    int64_t J_off;   // offset (in blocks) of this sample in the J store
    int64_t a_off;   // offset (in complex numbers) of the sample's first chain state
    int64_t q_off;   // offset of the sample in the canonical quadruplet arrays (plain path)
    int64_t nq;      // quadruplets of the sample
    int64_t inc_off; // offset of the sample in the incidence arrays (plain path), N+1 entries at mode_off
};

// One scheduling group: up to G chains of one sample updated together by one thread block.
struct GroupDev {
    int sample;
    int chain0;  // first chain slot
    int count;   // chains in the group (<= G)
    int probe_flag;         // written by no kernel: the wait probe waits on it until its limit
};

// Kernel-wide control words in device memory.
struct Control {
    unsigned int ticket;    // persistent work queue ticket
    int error;              // first error code seen by a kernel (0 = none)
    int error_where;        // where a bounded wait ran out
    int probe_flag;         // written by no kernel: the wait probe waits on it until its limit
    long long sweep_base;   // sweeps done before the current sweep launch
    long long swap_passes;  // swap passes done
    long long global_rounds;  // learned global-move rounds done
    long long trace_at;     // update trace: absolute sweep index + 1 of the traced sweep (0 = off)
    int trace_update;       // update trace: pair update of that sweep
    int trace_pad;
};

// One record of the update trace (doubles per chain, canonical chain order): the pair, the reduced sums
// h_j, h_k, B_jk, A_jk, the proposal, the uniform, Delta H, the decision, beta, the running energy before
// the update and a written flag.
constexpr int kTraceRec = 20;

constexpr int kErrTimeout = 1, kErrNaN = 2, kErrBadArg = 3;
constexpr unsigned long long kWaitNs = 10000000000ull;  // bounded waits give up after 10 s of wall time

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ inline void record_error(Control *ctl, int code, int where) {
    if (atomicCAS(&ctl->error, 0, code) == 0) ctl->error_where = where;
}

}  // namespace ptgb
