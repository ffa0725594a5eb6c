// pt_capi.cu -- host orchestration and C ABI of the smoothed-cubic Parallel-Tempering engine
// (arXiv 2511.13508): argument checks, the blocked per-mode coupling packer, device memory, the
// sweep-segment scheduler (sweeps -> resync -> measure -> swap, replayed as CUDA graphs),
// checkpoints and the host watchdog.  The declarations and their contracts are in include/pt.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/pt.h"
#include "pt_common.cuh"
#include "pt_gemm.h"
#include "pt_kernels.h"
#include "pt_learn.h"

using namespace ptgb;

namespace {
thread_local std::string g_create_error;
}

namespace ptgb {
void set_global_error(const char *msg) { g_create_error = msg; }
}  // namespace ptgb

namespace {

// Counts the quadruplets of the N-mode comb: for every (a,b) with a<b the admissible c run over
// b+1 .. N-1-(b-a) (then d = b+c-a lies in (c, N)).
std::vector<int64_t> pair_offsets(int N, int64_t *total) {
    std::vector<int64_t> off((size_t)N * N, -1);
    int64_t n = 0;
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b) {
            off[(size_t)a * N + b] = n;
            const int cnt = N - 1 - 2 * b + a;
            if (cnt > 0) n += cnt;
        }
    *total = n;
    return off;
}

inline int xlo_of(int s, int N) { return std::max(0, s - (N - 1)); }
inline int xhi_of(int s) { return (s - 1) / 2; }

struct SampleLayout {
    int N, ST, nblk;
    std::vector<int> bo, xtlo, mode_blk, ebo;
    std::vector<uint32_t> blkinfo;
    int64_t jblocks;  // blocks of J stored for the sample
};

SampleLayout make_layout(int N) {
    SampleLayout L;
    L.N = N;
    L.ST = (2 * N - 2 + TS - 1) / TS;
    L.bo.assign(L.ST + 1, 0);
    L.xtlo.assign(L.ST, 0);
    for (int st = 0; st < L.ST; ++st) {
        int xl = 1 << 30, xh = -1;
        for (int s = st * TS; s < st * TS + TS; ++s) {
            if (s < 1 || s > 2 * N - 3) continue;
            const int lo = xlo_of(s, N), hi = xhi_of(s);
            if (lo > hi) continue;
            xl = std::min(xl, lo);
            xh = std::max(xh, hi);
        }
        L.bo[st + 1] = L.bo[st];
        if (xh >= 0) {
            L.xtlo[st] = xl / TX;
            for (int xt = xl / TX; xt <= xh / TX; ++xt) {
                L.blkinfo.push_back(((uint32_t)st << 16) | (uint32_t)xt);
                L.bo[st + 1]++;
            }
        }
    }
    L.nblk = L.bo[L.ST];
    L.mode_blk.assign(N + 1, 0);
    L.ebo.assign(N + 1, 0);
    for (int l = 0; l < N; ++l) {
        const int stlo = l / TS, sthi = std::min((l + N - 1) / TS, L.ST - 1);
        L.mode_blk[l + 1] = L.mode_blk[l] + (L.bo[sthi + 1] - L.bo[stlo]);
        const int sta = (2 * l + 1) / TS;
        L.ebo[l + 1] = L.ebo[l] + (sta <= sthi ? L.bo[sthi + 1] - L.bo[sta] : 0);
    }
    L.jblocks = L.mode_blk[N];
    return L;
}

// Fills the blocked store of one sample: for mode l and block (st, xt) of its run, entry (r, i) is
// J of the quadruplet {l, m = s-l, x, s-x} with s = st*TS+r, x = xt*TX+i, or 0 when that is not a
// quadruplet of distinct modes.  Blocks are column-major (entry (r, i) at i*TS + r) and padded to
// JStride reals.
template <typename real>
void pack_sample(const SampleLayout &L, const double *J, real *dst) {
    const int N = L.N;
    int64_t total;
    const std::vector<int64_t> off = pair_offsets(N, &total);
    for (int l = 0; l < N; ++l) {
        const int stlo = l / TS, sthi = std::min((l + N - 1) / TS, L.ST - 1);
        int64_t bpos = L.mode_blk[l];
        for (int b = L.bo[stlo]; b < L.bo[sthi + 1]; ++b, ++bpos) {
            const int st = (int)(L.blkinfo[b] >> 16), xt = (int)(L.blkinfo[b] & 0xffffu);
            real *blk = dst + bpos * JStride<real>::value;
            for (int e = TBLK; e < JStride<real>::value; ++e) blk[e] = real(0);
            for (int r = 0; r < TS; ++r)
                for (int i = 0; i < TX; ++i) {
                    const int s = st * TS + r, x = xt * TX + i, m = s - l, y = s - x;
                    real v = real(0);
                    if (m >= 0 && m < N && m != l && s >= 1 && s <= 2 * N - 3 && x >= xlo_of(s, N) &&
                        x <= xhi_of(s) && x != std::min(l, m)) {
                        int q[4] = {l, m, x, y};
                        std::sort(q, q + 4);
                        const int64_t idx = off[(size_t)q[0] * N + q[1]] + (q[2] - q[1] - 1);
                        v = (real)J[idx];
                    }
                    blk[i * TS + r] = v;
                }
        }
    }
}

struct SegKey {
    int seg, n_snap, resync, live, swap, global;
    bool operator<(const SegKey &o) const {
        return std::tie(seg, n_snap, resync, live, swap, global) <
               std::tie(o.seg, o.n_snap, o.resync, o.live, o.swap, o.global);
    }
};

// Learned global-move proposal: network parameters, training set and work buffers (device memory).
struct LearnState {
    ptgb::LearnShape sh{};
    int Mb = 0, ncap = 0, ndata = 0, nprop = 0, rows = 0, global_every = 0, adam_t = 0;
    bool one_launch = true;  // autoregressive sampling in one launch (nprop <= 64)
    cudaStream_t side = nullptr;  // the current configurations' density and energy, concurrent with the sampling
    cudaEvent_t ev_fork = nullptr, ev_mid = nullptr, ev_join = nullptr;
    float *Ocur = nullptr;        // network outputs of the current configurations, laid out as O [S][rows][Dout]
    float2 *Jdf = nullptr;        // FP32 chains: the couplings of the quadruplet lists as float pairs
    int blk_lo = 0, blk_hi = ptgb::kLearnBlocks - 1;  // range of the first resampled block
    uint32_t step = 0;
    uint64_t seed = 0;
    float *P = nullptr, *Gr = nullptr, *Am = nullptr, *Av = nullptr, *M1 = nullptr, *M2 = nullptr, *M3 = nullptr;
    __nv_bfloat16 *W1 = nullptr, *W2 = nullptr, *W3 = nullptr, *W2T = nullptr, *W3T = nullptr;
    __nv_bfloat16 *W1c = nullptr, *W2c = nullptr, *W3c = nullptr;  // canonical K-major copies (fused forward)
    float *du = nullptr, *dphi = nullptr, *dextra = nullptr;
    int *dcond = nullptr;
    __nv_bfloat16 *X = nullptr, *XT = nullptr, *H1 = nullptr, *H1T = nullptr, *H2 = nullptr, *H2T = nullptr;
    __nv_bfloat16 *dOb = nullptr, *dOT = nullptr, *dZ2b = nullptr, *dZ2T = nullptr, *dZ1T = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *O = nullptr, *dO = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    ptgb::RawRows raw{}, rcur{}, rprop{}, rsamp{};
    double *logq = nullptr, *lq_cur = nullptr, *lq_prop = nullptr, *H_cur = nullptr, *H_prop = nullptr;
    int *pslot = nullptr, *pcond = nullptr;
    uint32_t *prow = nullptr;
    __nv_bfloat16 *Xp = nullptr;
    double2 *a_prop = nullptr;
    double *losses = nullptr;
    int max_losses = 0;
};

}  // namespace

struct pt_ctx {
    pt_config cfg;
    int S = 0, R = 0, nT = 0, maxN = 0;
    std::vector<int> N;
    uint64_t seed = 0;
    bool dbl = false, plain = false;
    bool gfp32 = false;  // explicit interaction lists on the FP32 group kernels
    int max_deg = 0;     // largest number of quadruplets holding one mode (quadruplet-list paths)
    cudaStream_t stream = nullptr;
    pt_alloc_fn alloc = nullptr;
    pt_free_fn free_ = nullptr;
    void *user = nullptr;
    std::string err;
    int64_t sweeps_done = 0, swap_passes = 0, global_rounds = 0;
    int n_chains = 0;
    int64_t a_total = 0;
    size_t esize = 8;  // bytes of one real
    std::vector<SampleDev> samples;
    std::vector<GroupDev> groups;
    std::vector<int> chain_sample;
    std::vector<std::pair<void *, size_t>> allocs;
    // device buffers
    SampleDev *d_samples = nullptr;
    GroupDev *d_groups = nullptr;
    void *d_J = nullptr;
    int *d_bo = nullptr, *d_xtlo = nullptr, *d_mode_blk = nullptr, *d_ebo = nullptr;
    uint32_t *d_blkinfo = nullptr;
    void *d_a = nullptr;
    double *d_E = nullptr, *d_beta = nullptr, *d_Etmp = nullptr;
    int *d_label = nullptr, *d_perm = nullptr, *d_chain_sample = nullptr, *d_progress = nullptr;
    unsigned long long *d_mc_acc = nullptr, *d_mc_att = nullptr, *d_mcT_acc = nullptr, *d_mcT_att = nullptr;
    unsigned long long *d_swap_acc = nullptr, *d_swap_att = nullptr, *d_qhist = nullptr;
    double *d_stat = nullptr, *d_qstat = nullptr, *d_fields = nullptr;
    double *d_trace = nullptr;  // update trace of the sweep kernels (allocated by the first pt_trace_update)
    Control *d_ctl = nullptr;
    void *d_snap_a = nullptr;
    double *d_snap_E = nullptr;
    int n_snap_max = 0, max_seg = 0;
    int4 *d_quads = nullptr;
    int4 *d_rec = nullptr;     // incidence records of the FP32 quadruplet-list path
    float *d_recJ = nullptr;
    double *d_Jq = nullptr;
    int *d_inc_off = nullptr, *d_inc = nullptr;
    int G = 8, ncw = 8, spu = 1, grid = 1;
    std::map<SegKey, cudaGraphExec_t> graphs;
    std::vector<cudaGraph_t> graph_defs;
    bool own_stream = false;
    size_t max_groups = 0;  // capacity of d_groups / d_progress (groups of 8 chains)
    int sms = 0;            // streaming multiprocessors of the device
    double *d_epart = nullptr;  // partial energies of the resync, [max_groups][kEnergyPartsMax][32]
    LearnState *learn = nullptr;
    unsigned long long *d_gm_acc = nullptr, *d_gm_att = nullptr;  // [S][nT] global-move counters
};

namespace {

int fail(pt_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(pt_ctx *c, cudaError_t e, const char *where) {
    return fail(c, PT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);    \
    } while (0)

void *dev_alloc(pt_ctx *c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) / 256 * 256;
    void *p = nullptr;
    if (c->alloc) {
        p = c->alloc(bytes, c->user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        p = nullptr;
    }
    if (p) c->allocs.push_back({p, bytes});
    return p;
}

template <typename T> int dalloc(pt_ctx *c, T **out, size_t count) {
    *out = reinterpret_cast<T *>(dev_alloc(c, count * sizeof(T)));
    if (!*out) return fail(c, PT_ENOMEM, "device allocation failed");
    return PT_OK;
}

template <typename T> int upload(pt_ctx *c, T *dst, const T *src, size_t count) {
    if (count == 0) return PT_OK;
    CK(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    return PT_OK;
}

int watchdog_sync(pt_ctx *c) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaStreamQuery(c->stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(c, e, "device work failed");
        if (c->cfg.watchdog_ms > 0) {
            const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
            if (ms > c->cfg.watchdog_ms) return fail(c, PT_ETIMEOUT, "host watchdog: stream did not finish in time");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    Control h;
    CK(cudaMemcpy(&h, c->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost));
    if (h.error == kErrTimeout) return fail(c, PT_ETIMEOUT, "a bounded device wait ran out (site " + std::to_string(h.error_where) + ")");
    if (h.error == kErrNaN) return fail(c, PT_ENAN, "non-finite energy or constraint found on the device");
    if (h.error) return fail(c, PT_ECUDA, "device error status " + std::to_string(h.error));
    return PT_OK;
}

// ---------------------------------------------------------------------------------- kernels
GraphParams graph_params(pt_ctx *c) {
    GraphParams p{};
    p.samples = c->d_samples; p.groups = c->d_groups; p.quads = c->d_quads; p.Jd = c->d_Jq;
    p.inc_off = c->d_inc_off; p.max_deg = c->max_deg; p.rec = c->d_rec; p.recJ = c->d_recJ;
    p.a = reinterpret_cast<float2 *>(c->d_a);
    p.E = c->d_E; p.label = c->d_label; p.beta = c->d_beta; p.mc_acc = c->d_mc_acc; p.mc_att = c->d_mc_att;
    p.R = c->R; p.nT = c->nT; p.maxN = c->maxN; p.seed = c->seed; p.cc = c->cfg.cc_factor; p.ctl = c->d_ctl;
    p.measure_every = c->cfg.measure_every; p.snap_a = reinterpret_cast<float2 *>(c->d_snap_a);
    p.snap_E = c->d_snap_E; p.n_snap_max = c->n_snap_max; p.a_total = c->a_total; p.n_chains = c->n_chains;
    p.trace = c->d_trace;
    return p;
}

int run_energy(pt_ctx *c, int renorm, double *E_out, bool write_state) {
    if (c->gfp32) {
        GraphParams p = graph_params(c);
        p.renorm = renorm; p.E_out = E_out; p.E_state = write_state ? c->d_E : nullptr;
        CK(launch_graph_energy(p, (int)c->groups.size(), c->stream));
        return PT_OK;
    }
    if (c->plain) {
        PlainParams p{};
        p.samples = c->d_samples; p.chain_sample = c->d_chain_sample; p.quads = c->d_quads; p.Jq = c->d_Jq;
        p.inc_off = c->d_inc_off; p.inc = c->d_inc; p.a = reinterpret_cast<double2 *>(c->d_a); p.E = c->d_E;
        p.maxN = c->maxN; p.cc = c->cfg.cc_factor; p.ctl = c->d_ctl; p.renorm = renorm;
        p.write_state = write_state ? 1 : 0; p.E_out = E_out;
        CK(launch_plain_energy(p, c->n_chains, c->stream));
        return PT_OK;
    }
    EnergyParams p{};
    p.samples = c->d_samples; p.groups = c->d_groups; p.J = c->d_J; p.bo = c->d_bo; p.blkinfo = c->d_blkinfo;
    p.mode_blk = c->d_mode_blk; p.ebo = c->d_ebo; p.a = c->d_a; p.cc = c->cfg.cc_factor; p.renorm = renorm;
    p.E_out = E_out; p.E_state = write_state ? c->d_E : nullptr; p.ctl = c->d_ctl;
    // several thread blocks per group (their partial sums added in a fixed order by a second kernel), so that the
    // resync fills the GPU with more warps than one block per group gives (about 8 blocks per SM; measured on
    // GB300: see the energy kernel)
    const int ng = (int)c->groups.size();
    p.part = c->d_epart;
    p.parts = std::max(1, std::min(kEnergyPartsMax, (8 * std::max(c->sms, 1) + ng - 1) / std::max(ng, 1)));
    const int Ge = c->dbl ? std::min(c->G, 16) : c->G;
    CK(launch_energy(c->dbl, Ge, p, ng, c->maxN, c->stream));
    return PT_OK;
}

int run_measure(pt_ctx *c, int n_snap, int live) {
    MeasureParams p{};
    p.samples = c->d_samples; p.a = c->d_a; p.E = c->d_E; p.snap_a = c->d_snap_a; p.snap_E = c->d_snap_E;
    p.n_snap = n_snap; p.live = live; p.perm = c->d_perm; p.S = c->S; p.R = c->R; p.nT = c->nT;
    p.dbl = c->dbl ? 1 : 0; p.a_total = c->a_total; p.n_chains = c->n_chains; p.stat = c->d_stat;
    p.qstat = c->d_qstat; p.qhist = c->d_qhist; p.label = c->d_label;
    CK(launch_measure(p, c->stream));
    return PT_OK;
}

int run_swap(pt_ctx *c) {
    SwapParams p{};
    p.samples = c->d_samples; p.E = c->d_E; p.label = c->d_label; p.perm = c->d_perm; p.beta = c->d_beta;
    p.swap_acc = c->d_swap_acc; p.swap_att = c->d_swap_att; p.mc_acc = c->d_mc_acc; p.mc_att = c->d_mc_att;
    p.mcT_acc = c->d_mcT_acc; p.mcT_att = c->d_mcT_att; p.S = c->S; p.R = c->R; p.nT = c->nT; p.seed = c->seed;
    p.ctl = c->d_ctl;
    CK(launch_swap(p, c->stream));
    return PT_OK;
}

int run_sweeps(pt_ctx *c, int seg) {
    if (c->gfp32) {
        GraphParams p = graph_params(c);
        p.n_sweeps = seg;
        CK(launch_graph_sweep(p, (int)c->groups.size(), c->stream));
        return PT_OK;
    }
    if (c->plain) {
        PlainParams p{};
        p.samples = c->d_samples; p.chain_sample = c->d_chain_sample; p.quads = c->d_quads; p.Jq = c->d_Jq;
        p.inc_off = c->d_inc_off; p.inc = c->d_inc; p.a = reinterpret_cast<double2 *>(c->d_a); p.E = c->d_E;
        p.label = c->d_label; p.beta = c->d_beta; p.mc_acc = c->d_mc_acc; p.mc_att = c->d_mc_att; p.R = c->R;
        p.nT = c->nT; p.maxN = c->maxN; p.seed = c->seed; p.cc = c->cfg.cc_factor; p.ctl = c->d_ctl;
        p.n_sweeps = seg; p.measure_every = c->cfg.measure_every;
        p.snap_a = reinterpret_cast<double2 *>(c->d_snap_a); p.snap_E = c->d_snap_E; p.n_snap_max = c->n_snap_max;
        p.a_total = c->a_total; p.n_chains = c->n_chains;
        CK(launch_plain_sweep(p, c->n_chains, c->stream));
        return PT_OK;
    }
    CK(cudaMemsetAsync(c->d_ctl, 0, sizeof(unsigned int), c->stream));  // ticket
    CK(cudaMemsetAsync(c->d_progress, 0, sizeof(int) * c->groups.size(), c->stream));
    SweepParams p{};
    p.samples = c->d_samples; p.groups = c->d_groups; p.n_groups = (int)c->groups.size(); p.J = c->d_J;
    p.bo = c->d_bo; p.xtlo = c->d_xtlo; p.blkinfo = c->d_blkinfo; p.mode_blk = c->d_mode_blk; p.a = c->d_a;
    p.E = c->d_E; p.label = c->d_label; p.beta = c->d_beta; p.mc_acc = c->d_mc_acc; p.mc_att = c->d_mc_att;
    p.R = c->R; p.nT = c->nT; p.maxN = c->maxN; p.seed = c->seed; p.cc = c->cfg.cc_factor; p.ctl = c->d_ctl;
    p.progress = c->d_progress; p.n_sweeps = seg; p.sweeps_per_unit = std::min(c->spu, seg);
    p.measure_every = c->cfg.measure_every; p.snap_a = c->d_snap_a; p.snap_E = c->d_snap_E;
    p.n_snap_max = c->n_snap_max; p.a_total = c->a_total; p.n_chains = c->n_chains; p.trace = c->d_trace;
    const int units = ((seg + p.sweeps_per_unit - 1) / p.sweeps_per_unit) * p.n_groups;
    const int grid = std::max(1, std::min(c->grid, units));
    CK(launch_sweep(c->dbl, c->G, c->ncw, p, grid, c->stream));
    return PT_OK;
}


// ------------------------------------------------------------------------------------------- learned proposal
template <typename T> T *lalloc(pt_ctx *c, size_t count, int *rc) {
    T *p = reinterpret_cast<T *>(dev_alloc(c, count * sizeof(T)));
    if (!p && *rc == PT_OK) *rc = fail(c, PT_ENOMEM, "device allocation failed (learned proposal)");
    return p;
}

// Arguments of the single-launch network forward (one cluster of blocks per sample, outputs into L.O).
MlpParams mlp_params(pt_ctx *c, const __nv_bfloat16 *X, int rows, const int *cond, int64_t strideCond) {
    LearnState &L = *c->learn;
    const ptgb::LearnShape &sh = L.sh;
    const int64_t rc = L.rows;
    MlpParams m{};
    m.X = X; m.strideX = rc * sh.Din; m.ldx = sh.Din; m.M = rows; m.Din = sh.Din; m.H = sh.H; m.Dout = sh.Dout;
    m.W1c = L.W1c; m.W2c = L.W2c; m.W3c = L.W3c;
    m.strideW1 = (int64_t)sh.H * sh.Din; m.strideW2 = (int64_t)sh.H * sh.H; m.strideW3 = (int64_t)sh.Dout * sh.H;
    m.P = L.P; m.psize = (int64_t)sh.psize; m.ob1 = sh.ob1; m.oC1 = sh.oC1; m.ob2 = sh.ob2; m.ob3 = sh.ob3;
    m.cond = cond; m.strideCond = strideCond; m.ncond = sh.ncold;
    m.O = L.O; m.strideO = rc * sh.Dout; m.ldo = sh.Dout;
    m.err = &c->d_ctl->error;
    return m;
}

// Dense layers on the tensor cores: O = W3 relu(W2 relu(W1 x + b1 + C1[cond]) + b2) + b3 for `rows` rows of
// every sample; with `train` the transposed activations the weight gradients need are kept as well.
int learn_forward(pt_ctx *c, const __nv_bfloat16 *X, int rows, const int *cond, int64_t strideCond, bool train) {
    LearnState &L = *c->learn;
    const ptgb::LearnShape &sh = L.sh;
    const int64_t rc = L.rows;
    if (!train) {  // sampling passes: the whole network in one launch, activations on chip
        const MlpParams m = mlp_params(c, X, rows, cond, strideCond);
        if (fused_mlp_supported(m, false)) {
            CK(launch_fused_mlp(m, c->S, c->stream));
            return PT_OK;
        }
    }
    GemmParams g{};
    g.A = X; g.strideA = rc * sh.Din; g.lda = sh.Din;
    g.B = L.W1; g.strideB = (int64_t)sh.H * sh.Din; g.ldb = sh.Din;
    g.M = rows; g.N = sh.H; g.K = sh.Din; g.mode = kEpiRelu;
    g.D = L.Z1; g.strideD = rc * sh.H; g.ldd = sh.H;
    g.bias = L.P + sh.ob1; g.strideBias = (int64_t)sh.psize;
    g.cbias = L.P + sh.oC1; g.strideCbias = (int64_t)sh.psize; g.cond = cond; g.strideCond = strideCond;
    g.H = L.H1; g.strideH = rc * sh.H; g.ldh = sh.H;
    g.HT = train ? L.H1T : nullptr; g.strideHT = rc * sh.H; g.ldht = (int)rc;
    g.err = &c->d_ctl->error;
    CK(launch_gemm_bf16(g, c->S, c->stream));
    GemmParams g2 = g;
    g2.A = L.H1; g2.strideA = rc * sh.H; g2.lda = sh.H;
    g2.B = L.W2; g2.strideB = (int64_t)sh.H * sh.H; g2.ldb = sh.H; g2.K = sh.H;
    g2.D = L.Z2; g2.bias = L.P + sh.ob2; g2.cbias = nullptr; g2.cond = nullptr;
    g2.H = L.H2; g2.HT = train ? L.H2T : nullptr;
    CK(launch_gemm_bf16(g2, c->S, c->stream));
    GemmParams g3{};
    g3.A = L.H2; g3.strideA = rc * sh.H; g3.lda = sh.H;
    g3.B = L.W3; g3.strideB = (int64_t)sh.Dout * sh.H; g3.ldb = sh.H;
    g3.M = rows; g3.N = sh.Dout; g3.K = sh.H; g3.mode = kEpiF32;
    g3.D = L.O; g3.strideD = rc * sh.Dout; g3.ldd = sh.Dout;
    g3.bias = L.P + sh.ob3; g3.strideBias = (int64_t)sh.psize;
    g3.err = &c->d_ctl->error;
    CK(launch_gemm_bf16(g3, c->S, c->stream));
    return PT_OK;
}

// Gradient of mean(-log q) over `rows` rows (dO already written by the density kernel) into L.Gr.
int learn_backward(pt_ctx *c, int rows, const int *cond) {
    LearnState &L = *c->learn;
    const ptgb::LearnShape &sh = L.sh;
    const int64_t rc = L.rows, ps = (int64_t)sh.psize;
    CK(cudaMemsetAsync(L.Gr, 0, sizeof(float) * sh.psize * c->S, c->stream));
    GemmParams g{};  // dZ2 = (dO W3) * [Z2 > 0]
    g.A = L.dOb; g.strideA = rc * sh.Dout; g.lda = sh.Dout;
    g.B = L.W3T; g.strideB = (int64_t)sh.H * sh.Dout; g.ldb = sh.Dout;
    g.M = rows; g.N = sh.H; g.K = sh.Dout; g.mode = kEpiGate;
    g.gate = L.Z2; g.strideGate = rc * sh.H; g.ldgate = sh.H;
    g.D = L.dZ2; g.strideD = rc * sh.H; g.ldd = sh.H;
    g.H = L.dZ2b; g.strideH = rc * sh.H; g.ldh = sh.H;
    g.HT = L.dZ2T; g.strideHT = rc * sh.H; g.ldht = (int)rc;
    g.err = &c->d_ctl->error;
    CK(launch_gemm_bf16(g, c->S, c->stream));
    GemmParams w3{};  // dW3 = dO^T H2
    w3.A = L.dOT; w3.strideA = rc * sh.Dout; w3.lda = (int)rc;
    w3.B = L.H2T; w3.strideB = rc * sh.H; w3.ldb = (int)rc;
    w3.M = sh.Dout; w3.N = sh.H; w3.K = rows; w3.mode = kEpiF32;
    w3.D = L.Gr + sh.oW3; w3.strideD = ps; w3.ldd = sh.H;
    w3.err = &c->d_ctl->error;
    CK(launch_gemm_bf16(w3, c->S, c->stream));
    GemmParams g1 = g;  // dZ1 = (dZ2 W2) * [Z1 > 0]
    g1.A = L.dZ2b; g1.strideA = rc * sh.H; g1.lda = sh.H;
    g1.B = L.W2T; g1.strideB = (int64_t)sh.H * sh.H; g1.ldb = sh.H; g1.K = sh.H;
    g1.gate = L.Z1; g1.D = L.dZ1; g1.H = nullptr; g1.HT = L.dZ1T;
    CK(launch_gemm_bf16(g1, c->S, c->stream));
    GemmParams w2 = w3;  // dW2 = dZ2^T H1
    w2.A = L.dZ2T; w2.strideA = rc * sh.H; w2.B = L.H1T; w2.strideB = rc * sh.H;
    w2.M = sh.H; w2.N = sh.H; w2.D = L.Gr + sh.oW2; w2.ldd = sh.H;
    CK(launch_gemm_bf16(w2, c->S, c->stream));
    GemmParams w1 = w3;  // dW1 = dZ1^T X
    w1.A = L.dZ1T; w1.strideA = rc * sh.H; w1.B = L.XT; w1.strideB = rc * sh.Din;
    w1.M = sh.H; w1.N = sh.Din; w1.D = L.Gr + sh.oW1; w1.ldd = sh.Din;
    CK(launch_gemm_bf16(w1, c->S, c->stream));
    CK(launch_colsum(L.dO, rows, sh.Dout, L.Gr + sh.ob3, nullptr, nullptr, c->S, rc * sh.Dout, ps, c->stream));
    CK(launch_colsum(L.dZ2, rows, sh.H, L.Gr + sh.ob2, nullptr, nullptr, c->S, rc * sh.H, ps, c->stream));
    CK(launch_colsum(L.dZ1, rows, sh.H, L.Gr + sh.ob1, L.Gr + sh.oC1, cond, c->S, rc * sh.H, ps, c->stream));
    return PT_OK;
}

int learn_cast(pt_ctx *c) {
    LearnState &L = *c->learn;
    CastParams cp{};
    cp.P = L.P; cp.M1 = L.M1; cp.M2 = L.M2; cp.M3 = L.M3;
    cp.W1 = L.W1; cp.W2 = L.W2; cp.W3 = L.W3; cp.W2T = L.W2T; cp.W3T = L.W3T; cp.sh = L.sh;
    cp.W1c = L.W1c; cp.W2c = L.W2c; cp.W3c = L.W3c;
    CK(launch_cast(cp, c->stream));
    return PT_OK;
}

DensityParams density_params(LearnState &L, const float *O, const RawRows &raw, double *logq, int rows, bool grad) {
    DensityParams d{};
    d.O = O; d.raw = raw; d.rows_per_sample = rows; d.N = L.sh.N; d.Dout = L.sh.Dout; d.logq = logq;
    d.inv_rows = 1.0f / (float)rows;
    d.o_stride = L.rows;
    if (grad) { d.dO = L.dO; d.dOb = L.dOb; d.dOT = L.dOT; d.lddt = L.rows; }
    return d;
}

// One round of learned global moves on the chains at the ncold coldest temperatures of every sample.
// When the network's forward pass fits one launch, the current configurations' density and energy run on a
// second stream, concurrently with the sampling of the proposals (they share only the features X, which
// neither side writes after the fork), and so does the proposals' energy, beside their features, forward
// pass and density; the Metropolis-Hastings step waits for both streams.
int run_global(pt_ctx *c) {
    LearnState &L = *c->learn;
    const ptgb::LearnShape &sh = L.sh;
    const int np = L.nprop;
    int rc;
    CK(launch_cold_rows(c->d_perm, c->S, c->R, c->nT, sh.ncold, L.pslot, L.prow, L.pcond, c->stream));
    // current configurations: features, then density and exact FP64 energy
    FeatParams fp{};
    fp.a = c->d_a; fp.dbl = c->dbl ? 1 : 0; fp.samples = c->d_samples; fp.slot = L.pslot; fp.rows_per_sample = np;
    fp.N = sh.N; fp.Din = sh.Din; fp.X = L.X; fp.XT = nullptr; fp.ldxt = L.rows; fp.raw = L.rcur;
    fp.raw_stride = np; fp.raw_off = 0; fp.cond_in = nullptr; fp.x_stride = L.rows;
    CK(launch_features(fp, c->S, c->stream));
    EnergyList2 el{};
    EnergyListParams &ep = el.set[0];
    ep.a = c->d_a; ep.dbl = c->dbl ? 1 : 0; ep.samples = c->d_samples; ep.slot = L.pslot; ep.rows_per_sample = np;
    ep.N = sh.N; ep.quads = c->d_quads; ep.Jq = c->d_Jq; ep.Jdf = L.Jdf; ep.cc = c->cfg.cc_factor; ep.E = L.H_cur;
    MlpParams mc = mlp_params(c, L.X, np, L.pcond, np);
    mc.O = L.Ocur;
    const bool split = fused_mlp_supported(mc, false);
    if (split) {
        CK(cudaEventRecord(L.ev_fork, c->stream));
        CK(cudaStreamWaitEvent(L.side, L.ev_fork, 0));
        CK(launch_fused_mlp(mc, c->S, L.side));
        DensityParams dc = density_params(L, L.Ocur, L.rcur, L.lq_cur, np, false);
        CK(launch_density(dc, c->S, L.side));
        EnergyList2 e1{};
        e1.set[0] = ep;
        CK(launch_energy_list(e1, 1, c->S, L.side));
    } else {
        if ((rc = learn_forward(c, L.X, np, L.pcond, np, false)) != PT_OK) return rc;
        DensityParams dc = density_params(L, L.O, L.rcur, L.lq_cur, np, false);
        CK(launch_density(dc, c->S, c->stream));
    }
    // autoregressive sampling, one pass per block of modes from the first resampled block of each row on;
    // the blocks below it keep the current configuration's features (the assembly copies their amplitudes
    // from the current configuration and reads the drawn variables only from the first resampled mode on)
    const MlpParams ms = mlp_params(c, L.X, np, L.pcond, np);
    if (L.one_launch && fused_mlp_supported(ms, true)) {  // all passes in one launch, weights resident on chip
        SamplerExtra sx{};
        sx.seed = c->seed; sx.row_id = L.prow; sx.ctl = c->d_ctl; sx.lo = L.blk_lo; sx.hi = L.blk_hi; sx.N = sh.N;
        sx.u = L.rsamp.u; sx.phi = L.rsamp.phi;
        CK(launch_fused_sampler(ms, sx, c->S, c->stream));
    } else {  // one network pass and one sampling launch per block
        CK(cudaMemcpyAsync(L.Xp, L.X, sizeof(__nv_bfloat16) * (size_t)c->S * L.rows * sh.Din,
                           cudaMemcpyDeviceToDevice, c->stream));
        for (int b = L.blk_lo; b < ptgb::kLearnBlocks; ++b) {
            if ((rc = learn_forward(c, L.Xp, np, L.pcond, np, false)) != PT_OK) return rc;
            SampleParams sp{};
            sp.O = L.O; sp.rows_per_sample = np; sp.N = sh.N; sp.Dout = sh.Dout; sp.Din = sh.Din; sp.block = b;
            sp.lo = L.blk_lo; sp.hi = L.blk_hi;
            sp.seed = c->seed; sp.row_id = L.prow; sp.ctl = c->d_ctl; sp.X = L.Xp; sp.u = L.rsamp.u;
            sp.phi = L.rsamp.phi; sp.o_stride = L.rows; sp.x_stride = L.rows;
            CK(launch_sample_block(sp, c->S, c->stream));
        }
    }
    AssembleParams ap{};
    ap.u = L.rsamp.u; ap.phi = L.rsamp.phi; ap.rows_per_sample = np; ap.N = sh.N; ap.seed = c->seed;
    ap.lo = L.blk_lo; ap.hi = L.blk_hi;
    ap.row_id = L.prow; ap.ctl = c->d_ctl; ap.a = L.a_prop;
    ap.a_cur = c->d_a; ap.dbl = c->dbl ? 1 : 0; ap.samples = c->d_samples; ap.slot = L.pslot;
    CK(launch_assemble(ap, c->S, c->stream));
    EnergyListParams &eq = el.set[1];
    eq = ep;
    eq.a = L.a_prop; eq.dbl = 1; eq.slot = nullptr; eq.E = L.H_prop;
    if (split) {  // the proposals' energy on the side stream too, beside their features, forward pass and density
        CK(cudaEventRecord(L.ev_mid, c->stream));
        CK(cudaStreamWaitEvent(L.side, L.ev_mid, 0));
        EnergyList2 e2{};
        e2.set[0] = eq;
        CK(launch_energy_list(e2, 1, c->S, L.side));
        CK(cudaEventRecord(L.ev_join, L.side));
    }
    // proposed configurations as stored: features (into Xp: the side stream may still read X), density, energy
    FeatParams fq = fp;
    fq.a = L.a_prop; fq.dbl = 1; fq.slot = nullptr; fq.raw = L.rprop; fq.X = L.Xp;
    CK(launch_features(fq, c->S, c->stream));
    if ((rc = learn_forward(c, L.Xp, np, L.pcond, np, false)) != PT_OK) return rc;
    DensityParams dq = density_params(L, L.O, L.rprop, L.lq_prop, np, false);
    CK(launch_density(dq, c->S, c->stream));
    if (split) {
        CK(cudaStreamWaitEvent(c->stream, L.ev_join, 0));
    } else {
        CK(launch_energy_list(el, 2, c->S, c->stream));  // both sets in one launch
    }
    MHParams mp{};
    mp.logq_cur = L.lq_cur; mp.logq_prop = L.lq_prop; mp.H_cur = L.H_cur; mp.H_prop = L.H_prop;
    mp.extra_cur = L.rcur.extra; mp.extra_prop = L.rprop.extra; mp.a_prop = L.a_prop; mp.a = c->d_a;
    mp.dbl = c->dbl ? 1 : 0; mp.E = c->d_E; mp.slot = L.pslot; mp.samples = c->d_samples; mp.beta = c->d_beta;
    mp.label = c->d_label; mp.rows_per_sample = np; mp.N = sh.N; mp.nT = c->nT; mp.seed = c->seed;
    mp.row_id = L.prow; mp.ctl = c->d_ctl; mp.acc = c->d_gm_acc; mp.att = c->d_gm_att;
    CK(launch_mh(mp, c->S, c->stream));
    return PT_OK;
}

// One segment: seg sweeps, then resync / global moves / measure / swap as due at its end.
int enqueue_segment(pt_ctx *c, const SegKey &k) {
    int rc;
    if ((rc = run_sweeps(c, k.seg)) != PT_OK) return rc;
    if (k.resync && (rc = run_energy(c, 1, nullptr, true)) != PT_OK) return rc;
    if (k.global && (rc = run_global(c)) != PT_OK) return rc;
    if ((k.n_snap || k.live) && (rc = run_measure(c, k.n_snap, k.live)) != PT_OK) return rc;
    if (k.swap && (rc = run_swap(c)) != PT_OK) return rc;
    CK(launch_advance(c->d_ctl, k.seg, k.swap ? 1 : 0, k.global ? 1 : 0, c->stream));
    return PT_OK;
}

int run_segment(pt_ctx *c, const SegKey &k) {
    if (!c->cfg.use_graphs) return enqueue_segment(c, k);
    auto it = c->graphs.find(k);
    if (it == c->graphs.end()) {
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
        const int rc = enqueue_segment(c, k);
        cudaGraph_t gg = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->stream, &gg);
        if (rc != PT_OK) {
            if (gg) cudaGraphDestroy(gg);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
        g = gg;
        cudaGraphExec_t ex;
        CK(cudaGraphInstantiate(&ex, g, 0));
        c->graph_defs.push_back(g);
        it = c->graphs.emplace(k, ex).first;
    }
    CK(cudaGraphLaunch(it->second, c->stream));
    return PT_OK;
}

// Chain groups of G chains per sample, the most expensive (largest N) first.
void make_groups(pt_ctx *c, int G) {
    c->groups.clear();
    const int cps = c->R * c->nT;
    for (int s = 0; s < c->S; ++s)
        for (int g0 = 0; g0 < cps; g0 += G) c->groups.push_back({s, c->samples[s].chain0 + g0, std::min(G, cps - g0), 0});
    std::stable_sort(c->groups.begin(), c->groups.end(),
                     [&](const GroupDev &x, const GroupDev &y) { return c->N[x.sample] > c->N[y.sample]; });
}

void drop_graphs(pt_ctx *c) {
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    for (auto g : c->graph_defs) cudaGraphDestroy(g);
    c->graphs.clear();
    c->graph_defs.clear();
}

// Switches the sweep blocks to G chains x ncw field warps (sweeps_per_unit spu); rebuilds the groups.
int set_shape(pt_ctx *c, int G, int ncw, int spu) {
    if (!sweep_variant_exists(c->dbl, G, ncw)) return fail(c, PT_EINVAL, "unsupported sweep block shape");
    const int occ = sweep_occupancy(c->dbl, G, ncw, c->maxN);
    if (occ < 1) return fail(c, PT_EUNSUPPORTED, "sweep block shape does not fit on this GPU");
    make_groups(c, G);
    if (c->groups.size() > c->max_groups) return fail(c, PT_EINVAL, "too many groups for this context");
    CK(cudaMemcpy(c->d_groups, c->groups.data(), c->groups.size() * sizeof(GroupDev), cudaMemcpyHostToDevice));
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int bps = c->cfg.blocks_per_sm > 0 ? std::min(c->cfg.blocks_per_sm, occ) : occ;
    c->grid = std::max(1, std::min((int)c->groups.size(), sms * bps));
    c->G = G; c->ncw = ncw; c->spu = spu;
    drop_graphs(c);
    return PT_OK;
}

// Incidence lists of one quadruplet list (nq quadruplets of N modes, 4 ints each): inc[off[l] .. off[l+1]) are
// the indices of the quadruplets holding mode l, in list order.  off: N+1 ints; inc: 4 nq ints.
void incidence_lists(int N, int64_t nq, const int32_t *abcd, int *off, int *inc) {
    std::fill(off, off + N + 1, 0);
    for (int64_t q = 0; q < nq; ++q)
        for (int m = 0; m < 4; ++m) off[abcd[4 * q + m] + 1]++;
    for (int l = 0; l < N; ++l) off[l + 1] += off[l];
    std::vector<int> fill(N, 0);
    for (int64_t q = 0; q < nq; ++q)
        for (int m = 0; m < 4; ++m) {
            const int l = abcd[4 * q + m];
            inc[off[l] + fill[l]++] = (int)q;
        }
}

// Incidence records of the FP32 quadruplet-list kernels, one per (mode l, quadruplet q holding it) in the
// order of the incidence lists: the other three modes A, B, C as row offsets of the kernel's amplitude table
// (mode x kGraphRowStride), ordered so that l's field term is J a_A a_B conj(a_C) (the term of q is
// J conj(a_q0) a_q1 a_q2 conj(a_q3); the field of a mode at position 1 or 2 is the conjugate of its product
// of the other three factors), the positions of l, A, B, C packed in w (2 bits each), and J_q in FP32.
void incidence_records(int N, const int32_t *abcd, const double *J, const int *off, const int *inc, int4 *rec,
                       float *recJ) {
    for (int l = 0; l < N; ++l)
        for (int e = off[l]; e < off[l + 1]; ++e) {
            const int q = inc[e];
            const int32_t *m4 = abcd + 4 * (int64_t)q;
            int pos = 0, o[3] = {0, 0, 0}, n = 0;
            for (int m = 0; m < 4; ++m) {
                if (m4[m] == l) pos = m;
                else if (n < 3) o[n++] = m4[m];
            }
            // partner positions in ascending order (the positions other than pos), then the order A, B, C:
            // pos 0 -> (1, 2, 3); pos 1 -> (0, 3, 2); pos 2 -> (0, 3, 1); pos 3 -> (1, 2, 0)
            int op[3], n2 = 0;
            for (int m = 0; m < 4; ++m)
                if (m != pos) op[n2++] = m;
            const int perm[4][3] = {{0, 1, 2}, {0, 2, 1}, {0, 2, 1}, {1, 2, 0}};
            const int *pm = perm[pos];
            const int R = ptgb::kGraphRowStride;
            rec[e] = make_int4(o[pm[0]] * R, o[pm[1]] * R, o[pm[2]] * R,
                               pos | (op[pm[0]] << 2) | (op[pm[1]] << 4) | (op[pm[2]] << 6));
            recJ[e] = (float)J[q];
        }
}

void free_all(pt_ctx *c) {
    drop_graphs(c);
    for (auto &p : c->allocs) {
        if (c->free_) c->free_(p.first, c->user);
        else cudaFree(p.first);
    }
    c->allocs.clear();
}

}  // namespace

// ================================================================================================ C ABI
extern "C" {

void pt_config_default(pt_config *cfg) {
    if (!cfg) return;
    cfg->precision = PT_PREC_FP32;
    cfg->cc_factor = 2.0;
    cfg->swap_every = 64;
    cfg->measure_every = 16;
    cfg->resync_every = 64;
    cfg->chains_per_block = 0;
    cfg->sweeps_per_unit = 0;
    cfg->blocks_per_sm = 0;
    cfg->consumer_warps = 0;
    cfg->use_graphs = 1;
    cfg->watchdog_ms = 600000;
}

int pt_enumerate_quads(int N, int32_t *abcd, int64_t *count) {
    if (!count || N < 4 || N > 512) return fail(nullptr, PT_EINVAL, "pt_enumerate_quads: need 4 <= N <= 512 and count");
    int64_t n = 0;
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b)
            for (int c2 = b + 1; c2 < N; ++c2) {
                const int d = b + c2 - a;
                if (d >= N) break;
                if (abcd) {
                    abcd[4 * n] = a; abcd[4 * n + 1] = b; abcd[4 * n + 2] = c2; abcd[4 * n + 3] = d;
                }
                ++n;
            }
    *count = n;
    return PT_OK;
}

int pt_fmc_graph(int N, const double *omega, double gamma, int32_t *quads, int64_t *count) {
    if (!count || !omega || N < 4 || N > 512 || !(gamma > 0.0) || !std::isfinite(gamma))
        return fail(nullptr, PT_EINVAL, "pt_fmc_graph: need 4 <= N <= 512, omega, gamma > 0 and count");
    for (int k = 0; k < N; ++k)
        if (!std::isfinite(omega[k]) || (k && !(omega[k] > omega[k - 1])))
            return fail(nullptr, PT_EINVAL, "pt_fmc_graph: omega must be finite and strictly ascending");
    // For each a < b < c the fourth mode d > c of a matching splitting has a frequency in a window of
    // width 2 gamma: omega_b + omega_c - omega_a (splitting {a,d}|{b,c}), omega_a + omega_b - omega_c
    // ({a,b}|{c,d}) or omega_a + omega_c - omega_b ({a,c}|{b,d}); the windows are found by binary search
    // and the candidates kept in (d, splitting) order, so the list comes out in canonical order.
    int64_t n = 0;
    std::vector<std::pair<int, int>> cand;
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b)
            for (int c2 = b + 1; c2 < N; ++c2) {
                cand.clear();
                const double centre[3] = {omega[b] + omega[c2] - omega[a], omega[a] + omega[b] - omega[c2],
                                          omega[a] + omega[c2] - omega[b]};
                for (int t = 0; t < 3; ++t) {
                    const double *lo = std::lower_bound(omega + c2 + 1, omega + N, centre[t] - gamma);
                    for (const double *it = lo; it < omega + N && *it <= centre[t] + gamma; ++it) {
                        const int d = (int)(it - omega);
                        int p, q, u, v;  // conjugated {p, q}, plain {u, v}
                        if (t == 0) { p = a; q = d; u = b; v = c2; }
                        else if (t == 1) { p = a; q = b; u = c2; v = d; }
                        else { p = a; q = c2; u = b; v = d; }
                        if (std::fabs(omega[p] + omega[q] - omega[u] - omega[v]) < gamma) cand.push_back({d, t});
                    }
                }
                std::sort(cand.begin(), cand.end());
                for (const auto &dt : cand) {
                    const int d = dt.first, t = dt.second;
                    if (quads) {
                        int32_t *o = quads + 4 * n;
                        if (t == 0) { o[0] = a; o[1] = b; o[2] = c2; o[3] = d; }
                        else if (t == 1) { o[0] = a; o[1] = c2; o[2] = d; o[3] = b; }
                        else { o[0] = a; o[1] = b; o[2] = d; o[3] = c2; }
                    }
                    ++n;
                }
            }
    *count = n;
    return PT_OK;
}

static int create_impl(pt_ctx **out, const pt_config *cfg_in, int S, const int32_t *Nv, const int32_t *graph,
                       const double *J, const int64_t *J_offsets, int n_T, const double *temps, int replicas,
                       uint64_t seed, pt_alloc_fn alloc, pt_free_fn free_, void *alloc_user, void *stream);

// Default shape of the sweep blocks (chains sharing one J stream G, field warps ncw) for the largest N, the sample
// count and chains per sample, and the device's SM count; G_in > 0 keeps that G.  Measured on GB300
// (chain-sweeps/s):
// - N >= 160: 8 chains x 11 warps (N = 192, 32 samples x 64 chains: 1.48M against 1.41M with 16 x 11; N = 256,
//   16 x 96 chains: 0.694M against 0.481M);
// - 48 <= N < 160: the most chains per block that still give about one group per SM, from 32, 16, 8 below
//   N = 96 and from 16, 8 above (N = 64, 64 samples x 64 chains: 32 x 11 24.2M against 20.8M with 16 x 11
//   and 12.5M with 8 x 11; 16 samples x 64 chains: 8 x 11 10.0M against 5.7M with 32 x 11, which leaves most
//   SMs idle; N = 128, 64 samples x 64 chains: 16 x 11 4.71M against 4.50M with 32 x 11 and 3.81M with
//   8 x 11; the ragged batch N in {32..128}: 16 x 11 8.91M against 8.38M with 8 x 11), 32 x 11 (16 x 11 from
//   N = 96) when none does;
// - N < 48: 16 x 7;
// - at most 8 chains per sample: 8 chains per block.
// Field warps: 11 from N = 48 on (N = 64, 64 samples: 32 x 11 22.3M chain-sweeps/s against 21.6M with 32 x 7;
// ragged batch: 16 x 11 8.24M against 7.53M with 16 x 7), else 7.  FP64: 8 x 7 from N = 128 on, else 16 x 3
// (N = 64, 64 samples: 16 x 3 685k, 8 x 7 521k).
static void default_shape(bool dbl, int maxN, int S, int chains_ps, int sms, int G_in, int *G_out, int *ncw_out) {
    int G = G_in;
    if (G == 0) {
        if (dbl) G = (maxN >= 128) ? 8 : 16;
        else if (maxN >= 160) G = 8;
        else if (maxN >= 48) {
            const int gmax = maxN >= 96 ? 16 : 32;
            for (int g : {32, 16, 8}) {
                if (G == 0 && g <= gmax && sms > 0 && (int64_t)S * ((chains_ps + g - 1) / g) >= (int64_t)sms * 4 / 5) G = g;
            }
            if (G == 0) G = (gmax == 32 && chains_ps >= 32) ? 32 : 16;
        } else {
            G = 16;
        }
        if (G > 8 && chains_ps <= 8) G = 8;
    }
    *G_out = G;
    if (dbl) *ncw_out = (G == 16) ? 3 : 7;
    else *ncw_out = (maxN >= 48) ? 11 : 7;
}

int pt_default_shape(int precision, int max_n, int n_samples, int chains_per_sample, int sm_count,
                     int *chains_per_block, int *consumer_warps) {
    if ((precision != PT_PREC_FP32 && precision != PT_PREC_FP64) || max_n < 4 || max_n > 512 || (max_n & 1) ||
        n_samples < 1 || chains_per_sample < 1 || sm_count < 0 || !chains_per_block || !consumer_warps)
        return fail(nullptr, PT_EINVAL, "pt_default_shape: bad argument");
    default_shape(precision == PT_PREC_FP64, max_n, n_samples, chains_per_sample, sm_count, 0, chains_per_block,
                  consumer_warps);
    return PT_OK;
}

int pt_create(pt_ctx **out, const pt_config *cfg_in, int S, const int32_t *Nv, const double *J,
              const int64_t *J_offsets, int n_T, const double *temps, int replicas, uint64_t seed,
              pt_alloc_fn alloc, pt_free_fn free_, void *alloc_user, void *stream) {
    return create_impl(out, cfg_in, S, Nv, nullptr, J, J_offsets, n_T, temps, replicas, seed, alloc, free_,
                       alloc_user, stream);
}

int pt_create_graph(pt_ctx **out, const pt_config *cfg_in, int S, const int32_t *Nv, const int32_t *quads,
                    const double *J, const int64_t *q_offsets, int n_T, const double *temps, int replicas,
                    uint64_t seed, pt_alloc_fn alloc, pt_free_fn free_, void *alloc_user, void *stream) {
    if (!quads) return fail(nullptr, PT_EINVAL, "pt_create_graph: quads is NULL");
    return create_impl(out, cfg_in, S, Nv, quads, J, q_offsets, n_T, temps, replicas, seed, alloc, free_,
                       alloc_user, stream);
}

int pt_graph_records(int N, int64_t nq, const int32_t *quads, const double *J, int32_t *offsets, int32_t *rec,
                     float *recJ) {
    if (N < 4 || N > 2048 || nq < 0 || nq > (int64_t)1 << 28 || (nq > 0 && (!quads || !J)) || !offsets || (nq > 0 && (!rec || !recJ)))
        return fail(nullptr, PT_EINVAL, "pt_graph_records: need 4 <= N <= 2048, 0 <= nq <= 2^28, quads, J, offsets, rec, recJ");
    for (int64_t i = 0; i < 4 * nq; ++i)
        if (quads[i] < 0 || quads[i] >= N) return fail(nullptr, PT_EINVAL, "pt_graph_records: mode index out of range");
    std::vector<int> inc((size_t)std::max<int64_t>(4 * nq, 1));
    incidence_lists(N, nq, quads, offsets, inc.data());
    if (nq > 0) {
        std::vector<int4> r((size_t)(4 * nq));  // int4 is 16-byte aligned; the caller's buffer need not be
        incidence_records(N, quads, J, offsets, inc.data(), r.data(), recJ);
        std::memcpy(rec, r.data(), r.size() * sizeof(int4));
    }
    return PT_OK;
}

static int create_impl(pt_ctx **out, const pt_config *cfg_in, int S, const int32_t *Nv, const int32_t *graph,
                       const double *J, const int64_t *J_offsets, int n_T, const double *temps, int replicas,
                       uint64_t seed, pt_alloc_fn alloc, pt_free_fn free_, void *alloc_user, void *stream) {
    if (!out) return fail(nullptr, PT_EINVAL, "pt_create: out is NULL");
    *out = nullptr;
    pt_config cfg;
    pt_config_default(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if (S < 1 || !Nv || !J || !J_offsets || n_T < 1 || !temps || replicas < 1)
        return fail(nullptr, PT_EINVAL, "pt_create: need S >= 1, N, J, J_offsets, n_T >= 1, temps, replicas >= 1");
    if ((alloc == nullptr) != (free_ == nullptr)) return fail(nullptr, PT_EINVAL, "pt_create: give both alloc and free or neither");
    if (cfg.precision < PT_PREC_FP32 || cfg.precision > PT_PREC_FP64_PLAIN) return fail(nullptr, PT_EINVAL, "pt_create: bad precision");
    if (!(cfg.cc_factor > 0.0) || !std::isfinite(cfg.cc_factor)) return fail(nullptr, PT_EINVAL, "pt_create: cc_factor must be positive");
    if (cfg.swap_every < 0 || cfg.measure_every < 0 || cfg.resync_every < 0)
        return fail(nullptr, PT_EINVAL, "pt_create: negative schedule interval");
    for (int t = 0; t < n_T; ++t) {
        if (!(temps[t] > 0.0) || !std::isfinite(temps[t])) return fail(nullptr, PT_EINVAL, "pt_create: temperatures must be positive");
        if (t && !(temps[t] > temps[t - 1])) return fail(nullptr, PT_EINVAL, "pt_create: temperatures must be strictly ascending");
    }
    if ((int64_t)S * replicas * n_T > (1ll << 28)) return fail(nullptr, PT_EINVAL, "pt_create: too many chains");
    if (graph && cfg.precision == PT_PREC_FP64)
        return fail(nullptr, PT_EUNSUPPORTED, "pt_create_graph: explicit graphs run in PT_PREC_FP32 or PT_PREC_FP64_PLAIN");
    for (int s = 0; s < S; ++s) {
        if (Nv[s] < 4 || Nv[s] > (graph ? 2048 : 512) || (Nv[s] & 1))
            return fail(nullptr, PT_EINVAL, graph ? "pt_create_graph: every N must be even, 4..2048"
                                                  : "pt_create: every N must be even, 4..512");
        if (graph) {
            if (J_offsets[s + 1] < J_offsets[s] || (s == 0 && J_offsets[0] != 0))
                return fail(nullptr, PT_EINVAL, "pt_create_graph: q_offsets must start at 0 and not decrease");
            for (int64_t q = J_offsets[s]; q < J_offsets[s + 1]; ++q) {
                const int32_t *Q = graph + 4 * q;
                for (int m = 0; m < 4; ++m)
                    if (Q[m] < 0 || Q[m] >= Nv[s]) return fail(nullptr, PT_EINVAL, "pt_create_graph: mode index out of range");
                if (Q[0] == Q[1] || Q[0] == Q[2] || Q[0] == Q[3] || Q[1] == Q[2] || Q[1] == Q[3] || Q[2] == Q[3])
                    return fail(nullptr, PT_EINVAL, "pt_create_graph: the four modes of a quadruplet must be distinct");
            }
        } else {
            int64_t nq;
            pt_enumerate_quads(Nv[s], nullptr, &nq);
            if (J_offsets[s + 1] - J_offsets[s] != nq) return fail(nullptr, PT_EINVAL, "pt_create: J_offsets do not match the quadruplet counts");
        }
        for (int64_t i = J_offsets[s]; i < J_offsets[s + 1]; ++i)
            if (!std::isfinite(J[i])) return fail(nullptr, PT_ENAN, "pt_create: non-finite coupling");
    }
    pt_ctx *c = new pt_ctx();
    c->cfg = cfg;
    c->S = S; c->R = replicas; c->nT = n_T; c->seed = seed;
    c->N.assign(Nv, Nv + S);
    c->maxN = *std::max_element(c->N.begin(), c->N.end());
    c->dbl = cfg.precision != PT_PREC_FP32;
    c->plain = cfg.precision == PT_PREC_FP64_PLAIN;
    c->gfp32 = graph != nullptr && cfg.precision == PT_PREC_FP32;
    c->esize = c->dbl ? 8 : 4;
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    c->alloc = alloc; c->free_ = free_; c->user = alloc_user;
    if (c->stream == nullptr) {
        // the legacy default stream cannot be captured into graphs: run on a stream of our own
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            (void)cudaGetLastError();
            delete c;
            return fail(nullptr, PT_ECUDA, "pt_create: cannot create a CUDA stream");
        }
        c->own_stream = true;
    }
    auto bail = [&](int rc) {
        g_create_error = c->err;
        free_all(c);
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return rc;
    };
#undef CK
#define CK(call)                                                          \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return bail(cuda_fail(c, e_, #call));      \
    } while (0)
#define RC(x)                          \
    do {                               \
        int r_ = (x);                  \
        if (r_ != PT_OK) return bail(r_); \
    } while (0)

    // ---- scheduling shape
    const int chains_ps = replicas * n_T;
    int G = cfg.chains_per_block, ncw = 0;
    if (c->gfp32) G = 8;  // the group kernels hold 8 chains per block
    {
        int dev = 0, sms = 0;
        if (G == 0 && (cudaGetDevice(&dev) != cudaSuccess ||
                       cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess))
            sms = 0;
        default_shape(c->dbl, c->maxN, S, chains_ps, sms, G, &G, &ncw);
    }
    if (cfg.consumer_warps > 0) ncw = cfg.consumer_warps;
    if (!c->plain && !c->gfp32 && !sweep_variant_exists(c->dbl, G, ncw)) return bail(fail(c, PT_EINVAL, "pt_create: unsupported chains_per_block"));
    c->G = G; c->ncw = ncw;
    c->spu = cfg.sweeps_per_unit > 0 ? cfg.sweeps_per_unit
                                     : (c->maxN >= 192 ? 1 : c->maxN >= 96 ? 2 : c->maxN >= 48 ? 8 : 32);

    // ---- samples, chains, groups, layouts
    std::vector<SampleLayout> lay(S);
    std::vector<int> bo_all, xtlo_all, mode_all, ebo_all;
    std::vector<uint32_t> binfo_all;
    int64_t jblocks = 0, a_off = 0, q_off = 0, inc_total = 0;
    int chain0 = 0;
    for (int s = 0; s < S; ++s) {
        lay[s] = make_layout(c->N[s]);
        SampleDev sd{};
        sd.N = c->N[s]; sd.ST = lay[s].ST; sd.nblk = lay[s].nblk; sd.chains = chains_ps; sd.chain0 = chain0;
        sd.tab_off = (int)bo_all.size(); sd.blk_off = (int)binfo_all.size(); sd.mode_off = (int)mode_all.size();
        sd.J_off = jblocks; sd.a_off = a_off; sd.q_off = q_off; sd.nq = J_offsets[s + 1] - J_offsets[s];
        sd.inc_off = inc_total;
        bo_all.insert(bo_all.end(), lay[s].bo.begin(), lay[s].bo.end());
        xtlo_all.insert(xtlo_all.end(), lay[s].xtlo.begin(), lay[s].xtlo.end());
        xtlo_all.push_back(0);
        binfo_all.insert(binfo_all.end(), lay[s].blkinfo.begin(), lay[s].blkinfo.end());
        mode_all.insert(mode_all.end(), lay[s].mode_blk.begin(), lay[s].mode_blk.end());
        ebo_all.insert(ebo_all.end(), lay[s].ebo.begin(), lay[s].ebo.end());
        c->samples.push_back(sd);
        for (int i = 0; i < chains_ps; ++i) c->chain_sample.push_back(s);
        jblocks += lay[s].jblocks;
        a_off += (int64_t)c->N[s] * chains_ps;
        q_off += sd.nq;
        inc_total += 4 * sd.nq;
        chain0 += chains_ps;
    }
    // xtlo needs ST entries per sample at tab_off; pad to keep offsets aligned with bo (ST+1 entries)
    c->n_chains = chain0;
    c->a_total = a_off;
    make_groups(c, G);
    c->max_groups = std::max((size_t)S * ((chains_ps + 7) / 8), c->groups.size());
    // ---- schedule buffers
    int ev = 0;
    for (int e : {cfg.swap_every, cfg.resync_every}) if (e > 0) ev = ev ? std::min(ev, e) : e;
    c->max_seg = ev ? ev : 256;
    c->n_snap_max = cfg.measure_every > 0 ? std::max(1, (c->max_seg + cfg.measure_every - 1) / cfg.measure_every) : 1;

    // ---- device memory
    RC(dalloc(c, &c->d_samples, S));
    RC(dalloc(c, &c->d_groups, c->max_groups));
    RC(dalloc(c, &c->d_bo, bo_all.size()));
    RC(dalloc(c, &c->d_xtlo, xtlo_all.size()));
    RC(dalloc(c, &c->d_blkinfo, std::max<size_t>(1, binfo_all.size())));
    RC(dalloc(c, &c->d_mode_blk, mode_all.size()));
    RC(dalloc(c, &c->d_ebo, ebo_all.size()));
    c->d_a = dev_alloc(c, (size_t)c->a_total * 2 * c->esize);
    if (!c->d_a) return bail(fail(c, PT_ENOMEM, "device allocation failed (state)"));
    c->d_snap_a = dev_alloc(c, (size_t)c->n_snap_max * c->a_total * 2 * c->esize);
    if (!c->d_snap_a) return bail(fail(c, PT_ENOMEM, "device allocation failed (snapshots)"));
    RC(dalloc(c, &c->d_snap_E, (size_t)c->n_snap_max * c->n_chains));
    RC(dalloc(c, &c->d_E, c->n_chains));
    RC(dalloc(c, &c->d_Etmp, c->n_chains));
    RC(dalloc(c, &c->d_beta, n_T));
    RC(dalloc(c, &c->d_label, c->n_chains));
    RC(dalloc(c, &c->d_perm, c->n_chains));
    RC(dalloc(c, &c->d_chain_sample, c->n_chains));
    RC(dalloc(c, &c->d_progress, c->max_groups));
    RC(dalloc(c, &c->d_mc_acc, c->n_chains));
    RC(dalloc(c, &c->d_mc_att, c->n_chains));
    RC(dalloc(c, &c->d_mcT_acc, (size_t)S * n_T));
    RC(dalloc(c, &c->d_mcT_att, (size_t)S * n_T));
    RC(dalloc(c, &c->d_gm_acc, (size_t)S * n_T));
    RC(dalloc(c, &c->d_gm_att, (size_t)S * n_T));
    const size_t npair = (size_t)S * replicas * std::max(1, n_T - 1);
    RC(dalloc(c, &c->d_swap_acc, npair));
    RC(dalloc(c, &c->d_swap_att, npair));
    RC(dalloc(c, &c->d_qhist, (size_t)S * n_T * PT_QBINS));
    RC(dalloc(c, &c->d_stat, (size_t)S * n_T * PT_NSTAT));
    RC(dalloc(c, &c->d_qstat, (size_t)S * n_T * PT_NQSTAT));
    RC(dalloc(c, &c->d_fields, (size_t)chains_ps * 8));
    RC(dalloc(c, &c->d_ctl, 1));

    // ---- couplings: blocked store (J-sharing paths) or canonical list + incidences (plain path)
    if (!c->plain && !c->gfp32) {
        const size_t js = c->dbl ? JStride<double>::value : JStride<float>::value;
        c->d_J = dev_alloc(c, (size_t)jblocks * js * c->esize);
        if (!c->d_J) return bail(fail(c, PT_ENOMEM, "device allocation failed (couplings)"));
        std::vector<unsigned char> hJ((size_t)jblocks * js * c->esize);
        for (int s = 0; s < S; ++s) {
            if (c->dbl) pack_sample<double>(lay[s], J + J_offsets[s], reinterpret_cast<double *>(hJ.data()) + c->samples[s].J_off * js);
            else pack_sample<float>(lay[s], J + J_offsets[s], reinterpret_cast<float *>(hJ.data()) + c->samples[s].J_off * js);
        }
        CK(cudaMemcpy(c->d_J, hJ.data(), hJ.size(), cudaMemcpyHostToDevice));
    }
    if (c->plain || c->gfp32 || c->maxN <= 64) {
        std::vector<int4> hq((size_t)std::max<int64_t>(q_off, 1));
        std::vector<double> hJq((size_t)std::max<int64_t>(q_off, 1));
        std::vector<int> hinc_off, hinc((size_t)std::max<int64_t>(inc_total, 1));
        std::vector<int4> hrec(c->gfp32 ? hinc.size() : 0);
        std::vector<float> hrecJ(c->gfp32 ? hinc.size() : 0);
        for (int s = 0; s < S; ++s) {
            const int n = c->N[s];
            const SampleDev &sd = c->samples[s];
            std::vector<int32_t> abcd((size_t)4 * std::max<int64_t>(sd.nq, 1));
            int64_t cnt = sd.nq;
            if (graph) std::copy(graph + 4 * J_offsets[s], graph + 4 * J_offsets[s + 1], abcd.begin());
            else pt_enumerate_quads(n, abcd.data(), &cnt);
            for (int64_t q = 0; q < cnt; ++q) {
                hq[sd.q_off + q] = make_int4(abcd[4 * q], abcd[4 * q + 1], abcd[4 * q + 2], abcd[4 * q + 3]);
                hJq[sd.q_off + q] = J[J_offsets[s] + q];
            }
            std::vector<int> off(n + 1);
            incidence_lists(n, cnt, abcd.data(), off.data(), hinc.data() + sd.inc_off);
            for (int l = 0; l < n; ++l) c->max_deg = std::max(c->max_deg, off[l + 1] - off[l]);
            hinc_off.insert(hinc_off.end(), off.begin(), off.end());
            if (c->gfp32)
                incidence_records(n, abcd.data(), J + J_offsets[s], off.data(), hinc.data() + sd.inc_off,
                                  hrec.data() + sd.inc_off, hrecJ.data() + sd.inc_off);
        }
        RC(dalloc(c, &c->d_quads, hq.size()));
        RC(dalloc(c, &c->d_Jq, hJq.size()));
        RC(dalloc(c, &c->d_inc_off, hinc_off.size()));
        RC(dalloc(c, &c->d_inc, hinc.size()));
        CK(cudaMemcpy(c->d_quads, hq.data(), hq.size() * sizeof(int4), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_Jq, hJq.data(), hJq.size() * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_inc_off, hinc_off.data(), hinc_off.size() * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_inc, hinc.data(), hinc.size() * sizeof(int), cudaMemcpyHostToDevice));
        if (c->gfp32) {
            RC(dalloc(c, &c->d_rec, hrec.size()));
            RC(dalloc(c, &c->d_recJ, hrecJ.size()));
            CK(cudaMemcpy(c->d_rec, hrec.data(), hrec.size() * sizeof(int4), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c->d_recJ, hrecJ.data(), hrecJ.size() * sizeof(float), cudaMemcpyHostToDevice));
        }
    }
    std::vector<int> label(c->n_chains), perm(c->n_chains);
    for (int s = 0; s < S; ++s)
        for (int r = 0; r < replicas; ++r)
            for (int t = 0; t < n_T; ++t) {
                const int slot = c->samples[s].chain0 + r * n_T + t;
                label[slot] = t;
                perm[((size_t)s * replicas + r) * n_T + t] = slot;
            }
    std::vector<double> beta(n_T);
    for (int t = 0; t < n_T; ++t) beta[t] = 1.0 / temps[t];
    CK(cudaMemcpy(c->d_samples, c->samples.data(), S * sizeof(SampleDev), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_groups, c->groups.data(), c->groups.size() * sizeof(GroupDev), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_bo, bo_all.data(), bo_all.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_xtlo, xtlo_all.data(), xtlo_all.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (!binfo_all.empty()) CK(cudaMemcpy(c->d_blkinfo, binfo_all.data(), binfo_all.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_mode_blk, mode_all.data(), mode_all.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_ebo, ebo_all.data(), ebo_all.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_label, label.data(), label.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_perm, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_chain_sample, c->chain_sample.data(), c->chain_sample.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_beta, beta.data(), n_T * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemset(c->d_mc_acc, 0, c->n_chains * sizeof(unsigned long long)));
    CK(cudaMemset(c->d_mc_att, 0, c->n_chains * sizeof(unsigned long long)));
    CK(cudaMemset(c->d_mcT_acc, 0, (size_t)S * n_T * sizeof(unsigned long long)));
    CK(cudaMemset(c->d_mcT_att, 0, (size_t)S * n_T * sizeof(unsigned long long)));
    CK(cudaMemset(c->d_gm_acc, 0, (size_t)S * n_T * sizeof(unsigned long long)));
    CK(cudaMemset(c->d_gm_att, 0, (size_t)S * n_T * sizeof(unsigned long long)));
    CK(cudaMemset(c->d_swap_acc, 0, npair * sizeof(unsigned long long)));
    CK(cudaMemset(c->d_swap_att, 0, npair * sizeof(unsigned long long)));
    CK(cudaMemset(c->d_qhist, 0, (size_t)S * n_T * PT_QBINS * sizeof(unsigned long long)));
    CK(cudaMemset(c->d_stat, 0, (size_t)S * n_T * PT_NSTAT * sizeof(double)));
    CK(cudaMemset(c->d_qstat, 0, (size_t)S * n_T * PT_NQSTAT * sizeof(double)));
    CK(cudaMemset(c->d_ctl, 0, sizeof(Control)));

    if (c->gfp32) CK(graph_prepare(c->maxN, c->max_deg));
    // ---- persistent grid
    if (!c->plain && !c->gfp32) {
        int dev = 0, sms = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int occ = sweep_occupancy(c->dbl, G, ncw, c->maxN);
        if (occ < 1) return bail(fail(c, PT_EUNSUPPORTED, "pt_create: sweep kernel does not fit on this GPU for this N"));
        const int bps = cfg.blocks_per_sm > 0 ? std::min(cfg.blocks_per_sm, occ) : occ;
        c->grid = std::max(1, std::min((int)c->groups.size(), sms * bps));
        c->sms = sms;
        RC(dalloc(c, &c->d_epart, c->max_groups * (size_t)kEnergyPartsMax * 32));
    }

    // ---- initial chains (exact beta = 0 draws) and their energies
    InitParams ip{};
    ip.samples = c->d_samples; ip.chain_sample = c->d_chain_sample; ip.label = c->d_label; ip.a = c->d_a;
    ip.dbl = c->dbl ? 1 : 0; ip.R = replicas; ip.nT = n_T; ip.seed = seed;
    CK(launch_init(ip, c->n_chains, c->stream));
    RC(run_energy(c, 0, nullptr, true));
    RC(watchdog_sync(c));
#undef CK
#undef RC
    *out = c;
    return PT_OK;
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);    \
    } while (0)

int pt_sweep(pt_ctx *c, int64_t n) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_sweep: NULL context");
    if (n < 0) return fail(c, PT_EINVAL, "pt_sweep: negative sweep count");
    const pt_config &cf = c->cfg;
    while (n > 0) {
        const int64_t d = c->sweeps_done;
        int64_t nb = d + c->max_seg;
        const int ge = c->learn ? c->learn->global_every : 0;
        for (int e : {cf.swap_every, cf.resync_every, ge})
            if (e > 0) nb = std::min(nb, (d / e + 1) * e);
        const int seg = (int)std::min<int64_t>(n, nb - d);
        const int64_t end = d + seg;
        SegKey k{};
        k.seg = seg;
        k.n_snap = 0;
        if (cf.measure_every > 0) {
            const int64_t me = cf.measure_every;
            k.n_snap = (int)((end - 1) / me - d / me);  // measurement points in (d, end)
            k.live = (end % me == 0) ? 1 : 0;
        }
        k.resync = (cf.resync_every > 0 && end % cf.resync_every == 0) ? 1 : 0;
        k.swap = (cf.swap_every > 0 && end % cf.swap_every == 0 && c->nT > 1) ? 1 : 0;
        k.global = (ge > 0 && end % ge == 0) ? 1 : 0;
        if (k.n_snap > c->n_snap_max) return fail(c, PT_EINVAL, "pt_sweep: internal snapshot overflow");
        // a graph replays fixed sweep indices relative to the device counters: only the
        // segment shape enters the key
        const int rc = run_segment(c, k);
        if (rc != PT_OK) return rc;
        c->sweeps_done = end;
        c->swap_passes += k.swap;
        c->global_rounds += k.global;
        n -= seg;
    }
    return PT_OK;
}

int pt_swap(pt_ctx *c) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_swap: NULL context");
    if (c->nT < 2) return PT_OK;
    const int rc = run_swap(c);
    if (rc != PT_OK) return rc;
    CK(launch_advance(c->d_ctl, 0, 1, 0, c->stream));
    c->swap_passes++;
    return PT_OK;
}

int pt_resync(pt_ctx *c) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_resync: NULL context");
    return run_energy(c, 1, nullptr, true);
}

int pt_measure_now(pt_ctx *c) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_measure_now: NULL context");
    return run_measure(c, 0, 1);
}

int pt_measure(pt_ctx *c, pt_observables *o) {
    if (!c || !o) return fail(c, PT_EINVAL, "pt_measure: NULL argument");
    int rc = watchdog_sync(c);
    if (rc != PT_OK) return rc;
    const size_t ST = (size_t)c->S * c->nT, npair = (size_t)c->S * c->R * std::max(1, c->nT - 1);
    if (o->stat) CK(cudaMemcpy(o->stat, c->d_stat, ST * PT_NSTAT * sizeof(double), cudaMemcpyDeviceToHost));
    if (o->qstat) CK(cudaMemcpy(o->qstat, c->d_qstat, ST * PT_NQSTAT * sizeof(double), cudaMemcpyDeviceToHost));
    if (o->qhist) CK(cudaMemcpy(o->qhist, c->d_qhist, ST * PT_QBINS * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (o->swap_acc) CK(cudaMemcpy(o->swap_acc, c->d_swap_acc, npair * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (o->swap_att) CK(cudaMemcpy(o->swap_att, c->d_swap_att, npair * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (o->gm_acc) CK(cudaMemcpy(o->gm_acc, c->d_gm_acc, ST * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (o->gm_att) CK(cudaMemcpy(o->gm_att, c->d_gm_att, ST * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (o->mc_acc || o->mc_att) {
        std::vector<unsigned long long> ta(ST), tt(ST), ca(c->n_chains), ct(c->n_chains);
        std::vector<int> lab(c->n_chains);
        CK(cudaMemcpy(ta.data(), c->d_mcT_acc, ST * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(tt.data(), c->d_mcT_att, ST * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(ca.data(), c->d_mc_acc, c->n_chains * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(ct.data(), c->d_mc_att, c->n_chains * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(lab.data(), c->d_label, c->n_chains * sizeof(int), cudaMemcpyDeviceToHost));
        for (int slot = 0; slot < c->n_chains; ++slot) {
            const size_t i = (size_t)c->chain_sample[slot] * c->nT + lab[slot];
            ta[i] += ca[slot];
            tt[i] += ct[slot];
        }
        if (o->mc_acc) std::memcpy(o->mc_acc, ta.data(), ST * sizeof(uint64_t));
        if (o->mc_att) std::memcpy(o->mc_att, tt.data(), ST * sizeof(uint64_t));
    }
    return PT_OK;
}

int pt_reset_observables(pt_ctx *c) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_reset_observables: NULL context");
    const size_t ST = (size_t)c->S * c->nT, npair = (size_t)c->S * c->R * std::max(1, c->nT - 1);
    CK(cudaMemsetAsync(c->d_stat, 0, ST * PT_NSTAT * sizeof(double), c->stream));
    CK(cudaMemsetAsync(c->d_qstat, 0, ST * PT_NQSTAT * sizeof(double), c->stream));
    CK(cudaMemsetAsync(c->d_qhist, 0, ST * PT_QBINS * sizeof(uint64_t), c->stream));
    CK(cudaMemsetAsync(c->d_swap_acc, 0, npair * sizeof(uint64_t), c->stream));
    CK(cudaMemsetAsync(c->d_swap_att, 0, npair * sizeof(uint64_t), c->stream));
    CK(cudaMemsetAsync(c->d_mcT_acc, 0, ST * sizeof(uint64_t), c->stream));
    CK(cudaMemsetAsync(c->d_mcT_att, 0, ST * sizeof(uint64_t), c->stream));
    CK(cudaMemsetAsync(c->d_mc_acc, 0, c->n_chains * sizeof(uint64_t), c->stream));
    CK(cudaMemsetAsync(c->d_mc_att, 0, c->n_chains * sizeof(uint64_t), c->stream));
    CK(cudaMemsetAsync(c->d_gm_acc, 0, ST * sizeof(uint64_t), c->stream));
    CK(cudaMemsetAsync(c->d_gm_att, 0, ST * sizeof(uint64_t), c->stream));
    return PT_OK;
}

// canonical index of every chain slot: (s, r, label)
static int canonical_map(pt_ctx *c, std::vector<int> &canon) {
    std::vector<int> lab(c->n_chains);
    CK(cudaMemcpy(lab.data(), c->d_label, c->n_chains * sizeof(int), cudaMemcpyDeviceToHost));
    canon.resize(c->n_chains);
    for (int slot = 0; slot < c->n_chains; ++slot) {
        const int s = c->chain_sample[slot];
        const int r = (slot - c->samples[s].chain0) / c->nT;
        canon[slot] = c->samples[s].chain0 + r * c->nT + lab[slot];
    }
    return PT_OK;
}

int pt_get_state(pt_ctx *c, double *a, double *E) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_get_state: NULL context");
    int rc = watchdog_sync(c);
    if (rc != PT_OK) return rc;
    std::vector<int> canon;
    if ((rc = canonical_map(c, canon)) != PT_OK) return rc;
    if (a) {
        std::vector<unsigned char> h((size_t)c->a_total * 2 * c->esize);
        CK(cudaMemcpy(h.data(), c->d_a, h.size(), cudaMemcpyDeviceToHost));
        for (int slot = 0; slot < c->n_chains; ++slot) {
            const SampleDev &sd = c->samples[c->chain_sample[slot]];
            const int64_t src = sd.a_off + (int64_t)(slot - sd.chain0) * sd.N;
            const int64_t dst = sd.a_off + (int64_t)(canon[slot] - sd.chain0) * sd.N;
            for (int x = 0; x < 2 * sd.N; ++x)
                a[2 * dst + x] = c->dbl ? reinterpret_cast<double *>(h.data())[2 * src + x]
                                        : (double)reinterpret_cast<float *>(h.data())[2 * src + x];
        }
    }
    if (E) {
        std::vector<double> h(c->n_chains);
        CK(cudaMemcpy(h.data(), c->d_E, c->n_chains * sizeof(double), cudaMemcpyDeviceToHost));
        for (int slot = 0; slot < c->n_chains; ++slot) E[canon[slot]] = h[slot];
    }
    return PT_OK;
}

int pt_set_state(pt_ctx *c, const double *a) {
    if (!c || !a) return fail(c, PT_EINVAL, "pt_set_state: NULL argument");
    int rc = watchdog_sync(c);
    if (rc != PT_OK) return rc;
    std::vector<int> canon;
    if ((rc = canonical_map(c, canon)) != PT_OK) return rc;
    std::vector<unsigned char> h((size_t)c->a_total * 2 * c->esize);
    for (int slot = 0; slot < c->n_chains; ++slot) {
        const SampleDev &sd = c->samples[c->chain_sample[slot]];
        const int64_t dst = sd.a_off + (int64_t)(slot - sd.chain0) * sd.N;
        const int64_t src = sd.a_off + (int64_t)(canon[slot] - sd.chain0) * sd.N;
        for (int x = 0; x < 2 * sd.N; ++x) {
            const double v = a[2 * src + x];
            if (!std::isfinite(v)) return fail(c, PT_ENAN, "pt_set_state: non-finite amplitude");
            if (c->dbl) reinterpret_cast<double *>(h.data())[2 * dst + x] = v;
            else reinterpret_cast<float *>(h.data())[2 * dst + x] = (float)v;
        }
    }
    CK(cudaMemcpyAsync(c->d_a, h.data(), h.size(), cudaMemcpyHostToDevice, c->stream));
    if ((rc = run_energy(c, 0, nullptr, true)) != PT_OK) return rc;
    return watchdog_sync(c);
}

int pt_energy(pt_ctx *c, double *E) {
    if (!c || !E) return fail(c, PT_EINVAL, "pt_energy: NULL argument");
    int rc = run_energy(c, 0, c->d_Etmp, false);
    if (rc != PT_OK) return rc;
    if ((rc = watchdog_sync(c)) != PT_OK) return rc;
    std::vector<int> canon;
    if ((rc = canonical_map(c, canon)) != PT_OK) return rc;
    std::vector<double> h(c->n_chains);
    CK(cudaMemcpy(h.data(), c->d_Etmp, c->n_chains * sizeof(double), cudaMemcpyDeviceToHost));
    for (int slot = 0; slot < c->n_chains; ++slot) E[canon[slot]] = h[slot];
    return PT_OK;
}

int pt_fields(pt_ctx *c, int sample, int j, int k, double *out) {
    if (!c || !out) return fail(c, PT_EINVAL, "pt_fields: NULL argument");
    if (c->plain || c->gfp32) return fail(c, PT_EUNSUPPORTED, "pt_fields: not available for the quadruplet-list paths");
    if (sample < 0 || sample >= c->S) return fail(c, PT_EINVAL, "pt_fields: bad sample");
    const int N = c->N[sample];
    if (j < 0 || j >= N || k < 0 || k >= N || j == k) return fail(c, PT_EINVAL, "pt_fields: need distinct modes in [0, N)");
    int rc = watchdog_sync(c);
    if (rc != PT_OK) return rc;
    // the groups of one sample are contiguous (a stable sort by N keeps sample order within equal N)
    int g0 = -1, ng = 0;
    for (size_t i = 0; i < c->groups.size(); ++i)
        if (c->groups[i].sample == sample) { if (g0 < 0) g0 = (int)i; ++ng; }
    FieldsParams p{};
    p.samples = c->d_samples; p.groups = c->d_groups; p.group0 = g0; p.J = c->d_J; p.bo = c->d_bo;
    p.blkinfo = c->d_blkinfo; p.mode_blk = c->d_mode_blk; p.a = c->d_a; p.j = j; p.k = k; p.out = c->d_fields;
    const int Gf = c->dbl ? std::min(c->G, 16) : c->G;
    cudaError_t e = launch_fields(c->dbl, Gf, p, ng, c->maxN, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pt_fields");
    const int cps = c->R * c->nT;
    std::vector<double> h((size_t)cps * 8);
    CK(cudaMemcpy(h.data(), c->d_fields, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<int> canon;
    if ((rc = canonical_map(c, canon)) != PT_OK) return rc;
    const int c0 = c->samples[sample].chain0;
    for (int i = 0; i < cps; ++i) {
        const int dst = canon[c0 + i] - c0;
        for (int e2 = 0; e2 < 8; ++e2) out[(size_t)dst * 8 + e2] = h[(size_t)i * 8 + e2];
    }
    return PT_OK;
}

int pt_trace_update(pt_ctx *c, int update, double *rec, double *a) {
    if (!c || !rec) return fail(c, PT_EINVAL, "pt_trace_update: NULL argument");
    if (c->plain) return fail(c, PT_EUNSUPPORTED, "pt_trace_update: not available for PT_PREC_FP64_PLAIN");
    if (update < 0 || update >= c->maxN / 2) return fail(c, PT_EINVAL, "pt_trace_update: update must be in [0, maxN/2)");
    int rc = watchdog_sync(c);
    if (rc != PT_OK) return rc;
    const size_t nrec = (size_t)c->n_chains * kTraceRec, bytes = (nrec + (size_t)c->a_total * 2) * sizeof(double);
    if (!c->d_trace) {
        // allocated on first use; the sweep graphs captured before hold no trace buffer and are rebuilt
        if ((rc = dalloc(c, &c->d_trace, bytes / sizeof(double))) != PT_OK) return rc;
        drop_graphs(c);
    }
    CK(cudaMemsetAsync(c->d_trace, 0, bytes, c->stream));
    // arm the trace for the next sweep (its absolute index + 1), run it with its schedule, disarm
    struct { long long at; int u, pad; } on{c->sweeps_done + 1, update, 0}, off{0, -1, 0};
    static_assert(sizeof(on) == 16, "trace words");
    CK(cudaMemcpyAsync(&c->d_ctl->trace_at, &on, sizeof(on), cudaMemcpyHostToDevice, c->stream));
    rc = pt_sweep(c, 1);
    const cudaError_t e = cudaMemcpyAsync(&c->d_ctl->trace_at, &off, sizeof(off), cudaMemcpyHostToDevice, c->stream);
    if (rc != PT_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(c, e, "pt_trace_update: disarm");
    if ((rc = watchdog_sync(c)) != PT_OK) return rc;
    std::vector<double> h(nrec + (size_t)c->a_total * 2);
    CK(cudaMemcpy(h.data(), c->d_trace, bytes, cudaMemcpyDeviceToHost));
    std::memcpy(rec, h.data(), nrec * sizeof(double));
    if (a) std::memcpy(a, h.data() + nrec, (size_t)c->a_total * 2 * sizeof(double));
    return PT_OK;
}

// ---------------------------------------------------------------------------------- checkpoints
namespace {
const char kMagic[8] = {'P', 'T', 'G', 'B', 'C', 'K', 'P', '1'};
struct CkptHeader {
    char magic[8];
    int32_t version, S, R, nT, precision, n_chains;
    int64_t a_total, sweeps_done, swap_passes, global_rounds;
    uint64_t seed, layout_hash;
};
uint64_t fnv1a(const unsigned char *p, size_t n, uint64_t h = 1469598103934665603ull) {
    for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 1099511628211ull; }
    return h;
}
uint64_t layout_hash(const pt_ctx *c) {
    uint64_t h = fnv1a(reinterpret_cast<const unsigned char *>(c->N.data()), c->N.size() * sizeof(int));
    return fnv1a(reinterpret_cast<const unsigned char *>(&c->cfg.cc_factor), sizeof(double), h);
}
struct Blob { void *dev; size_t bytes; };
std::vector<Blob> blobs(pt_ctx *c) {
    const size_t ST = (size_t)c->S * c->nT, npair = (size_t)c->S * c->R * std::max(1, c->nT - 1);
    return {{c->d_a, (size_t)c->a_total * 2 * c->esize},
            {c->d_E, c->n_chains * sizeof(double)},
            {c->d_label, c->n_chains * sizeof(int)},
            {c->d_perm, c->n_chains * sizeof(int)},
            {c->d_mc_acc, c->n_chains * sizeof(uint64_t)},
            {c->d_mc_att, c->n_chains * sizeof(uint64_t)},
            {c->d_mcT_acc, ST * sizeof(uint64_t)},
            {c->d_mcT_att, ST * sizeof(uint64_t)},
            {c->d_stat, ST * PT_NSTAT * sizeof(double)},
            {c->d_qstat, ST * PT_NQSTAT * sizeof(double)},
            {c->d_qhist, ST * PT_QBINS * sizeof(uint64_t)},
            {c->d_swap_acc, npair * sizeof(uint64_t)},
            {c->d_swap_att, npair * sizeof(uint64_t)},
            {c->d_gm_acc, ST * sizeof(uint64_t)},
            {c->d_gm_att, ST * sizeof(uint64_t)}};
}
}  // namespace

int pt_save(pt_ctx *c, void *buf, size_t *len) {
    if (!c || !len) return fail(c, PT_EINVAL, "pt_save: NULL argument");
    auto bl = blobs(c);
    size_t need = sizeof(CkptHeader) + sizeof(uint64_t);
    for (auto &b : bl) need += b.bytes;
    if (!buf) { *len = need; return PT_OK; }
    if (*len < need) return fail(c, PT_EINVAL, "pt_save: buffer too small");
    int rc = watchdog_sync(c);
    if (rc != PT_OK) return rc;
    unsigned char *p = reinterpret_cast<unsigned char *>(buf);
    CkptHeader h{};
    std::memcpy(h.magic, kMagic, 8);
    h.version = 1; h.S = c->S; h.R = c->R; h.nT = c->nT; h.precision = c->cfg.precision; h.n_chains = c->n_chains;
    h.a_total = c->a_total; h.sweeps_done = c->sweeps_done; h.swap_passes = c->swap_passes; h.seed = c->seed;
    h.global_rounds = c->global_rounds;
    h.layout_hash = layout_hash(c);
    std::memcpy(p, &h, sizeof(h));
    size_t off = sizeof(h);
    for (auto &b : bl) {
        CK(cudaMemcpy(p + off, b.dev, b.bytes, cudaMemcpyDeviceToHost));
        off += b.bytes;
    }
    const uint64_t sum = fnv1a(p, off);
    std::memcpy(p + off, &sum, sizeof(sum));
    *len = need;
    return PT_OK;
}

int pt_load(pt_ctx *c, const void *buf, size_t len) {
    if (!c || !buf) return fail(c, PT_EINVAL, "pt_load: NULL argument");
    auto bl = blobs(c);
    size_t need = sizeof(CkptHeader) + sizeof(uint64_t);
    for (auto &b : bl) need += b.bytes;
    if (len != need) return fail(c, PT_ESTATE, "pt_load: checkpoint size does not match this context");
    const unsigned char *p = reinterpret_cast<const unsigned char *>(buf);
    CkptHeader h;
    std::memcpy(&h, p, sizeof(h));
    if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != 1) return fail(c, PT_ESTATE, "pt_load: not a checkpoint");
    if (h.S != c->S || h.R != c->R || h.nT != c->nT || h.precision != c->cfg.precision || h.n_chains != c->n_chains ||
        h.a_total != c->a_total || h.seed != c->seed || h.layout_hash != layout_hash(c))
        return fail(c, PT_ESTATE, "pt_load: checkpoint belongs to a different context");
    uint64_t sum;
    std::memcpy(&sum, p + need - sizeof(sum), sizeof(sum));
    if (fnv1a(p, need - sizeof(sum)) != sum) return fail(c, PT_ESTATE, "pt_load: checksum mismatch");
    int rc = watchdog_sync(c);
    if (rc != PT_OK) return rc;
    size_t off = sizeof(h);
    for (auto &b : bl) {
        CK(cudaMemcpy(b.dev, p + off, b.bytes, cudaMemcpyHostToDevice));
        off += b.bytes;
    }
    Control ctl{};
    ctl.sweep_base = h.sweeps_done;
    ctl.swap_passes = h.swap_passes;
    ctl.global_rounds = h.global_rounds;
    CK(cudaMemcpy(c->d_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice));
    c->sweeps_done = h.sweeps_done;
    c->swap_passes = h.swap_passes;
    c->global_rounds = h.global_rounds;
    return PT_OK;
}

int pt_autotune(pt_ctx *c, int trial_sweeps, int *chosen) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_autotune: NULL context");
    if (c->plain || c->gfp32) return fail(c, PT_EUNSUPPORTED, "pt_autotune: the quadruplet-list paths have one shape");
    if (trial_sweeps < 1) return fail(c, PT_EINVAL, "pt_autotune: trial_sweeps must be >= 1");
    size_t len = 0;
    int rc = pt_save(c, nullptr, &len);
    if (rc != PT_OK) return rc;
    std::vector<unsigned char> blob(len);
    if ((rc = pt_save(c, blob.data(), &len)) != PT_OK) return rc;
    const int cps = c->R * c->nT;
    const int spu0 = c->cfg.sweeps_per_unit > 0 ? c->cfg.sweeps_per_unit
                                                 : (c->maxN >= 192 ? 1 : c->maxN >= 96 ? 2 : c->maxN >= 48 ? 8 : 32);
    struct Cand { int G, ncw, spu; };
    std::vector<Cand> cands;
    const int Gs_f[] = {8, 16, 32}, Gs_d[] = {8, 16};
    const int ncws[] = {3, 7, 9, 11, 15};
    for (int G : (c->dbl ? std::vector<int>(Gs_d, Gs_d + 2) : std::vector<int>(Gs_f, Gs_f + 3))) {
        if (G > 8 && cps < G / 2) continue;  // mostly empty blocks
        for (int n : ncws)
            if (sweep_variant_exists(c->dbl, G, n))
                for (int sp : {spu0, spu0 * 4}) cands.push_back({G, n, sp});
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    Cand bestc = {c->G, c->ncw, c->spu};
    for (const Cand &cd : cands) {
        if (set_shape(c, cd.G, cd.ncw, cd.spu) != PT_OK) continue;
        if ((rc = pt_sweep(c, 1)) != PT_OK) break;  // warm-up (graph capture)
        if (cudaEventRecord(e0, c->stream) != cudaSuccess) break;
        if ((rc = pt_sweep(c, trial_sweeps)) != PT_OK) break;
        if (cudaEventRecord(e1, c->stream) != cudaSuccess) break;
        if ((rc = watchdog_sync(c)) != PT_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; bestc = cd; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int rc2 = set_shape(c, bestc.G, bestc.ncw, bestc.spu);
    const int rc3 = pt_load(c, blob.data(), len);  // the trials leave no trace
    if (rc != PT_OK) return rc;
    if (rc2 != PT_OK) return rc2;
    if (rc3 != PT_OK) return rc3;
    if (chosen) { chosen[0] = bestc.G; chosen[1] = bestc.ncw; chosen[2] = bestc.spu; }
    return PT_OK;
}

// ---------------------------------------------------------------------------------- learned proposal
int pt_learn_init(pt_ctx *c, int n_cold, int batch, int data_per_sample, uint64_t seed) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_learn_init: NULL context");
    if (c->learn) return fail(c, PT_EINVAL, "pt_learn_init: already initialised");
    const int N = c->N[0];
    for (int n : c->N)
        if (n != N) return fail(c, PT_EUNSUPPORTED, "pt_learn_init: the learned proposal needs one N for all samples");
    if (N < 16 || N > 64 || N % 16) return fail(c, PT_EUNSUPPORTED, "pt_learn_init: the learned proposal supports N in {16, 32, 48, 64}");
    if (n_cold < 1 || n_cold > c->nT || n_cold * c->R > 1024) return fail(c, PT_EINVAL, "pt_learn_init: need 1 <= n_cold <= n_T");
    if (batch < 128 || batch % 128) return fail(c, PT_EINVAL, "pt_learn_init: batch must be a positive multiple of 128");
    if (data_per_sample < batch) return fail(c, PT_EINVAL, "pt_learn_init: data_per_sample must be >= batch");
    int rc = PT_OK;
    LearnState *L = new LearnState();
    c->learn = L;
    ptgb::LearnShape &sh = L->sh;
    sh.N = N; sh.H = 256; sh.Din = 3 * N; sh.Dout = 4 * N; sh.ncold = n_cold; sh.S = c->S;
    sh.oW1 = 0;
    sh.ob1 = sh.oW1 + (size_t)sh.H * sh.Din;
    sh.oC1 = sh.ob1 + sh.H;
    sh.oW2 = sh.oC1 + (size_t)n_cold * sh.H;
    sh.ob2 = sh.oW2 + (size_t)sh.H * sh.H;
    sh.oW3 = sh.ob2 + sh.H;
    sh.ob3 = sh.oW3 + (size_t)sh.Dout * sh.H;
    sh.psize = (sh.ob3 + sh.Dout + 63) / 64 * 64;
    L->Mb = batch; L->ncap = data_per_sample; L->nprop = n_cold * c->R; L->seed = seed;
    L->rows = std::max(batch, (L->nprop + 127) / 128 * 128);
    const size_t S = c->S, ps = sh.psize, rows = L->rows;
    L->P = lalloc<float>(c, S * ps, &rc); L->Gr = lalloc<float>(c, S * ps, &rc);
    L->Am = lalloc<float>(c, S * ps, &rc); L->Av = lalloc<float>(c, S * ps, &rc);
    L->M1 = lalloc<float>(c, (size_t)sh.H * sh.Din, &rc); L->M2 = lalloc<float>(c, (size_t)sh.H * sh.H, &rc);
    L->M3 = lalloc<float>(c, (size_t)sh.Dout * sh.H, &rc);
    L->W1 = lalloc<__nv_bfloat16>(c, S * sh.H * sh.Din, &rc); L->W2 = lalloc<__nv_bfloat16>(c, S * sh.H * sh.H, &rc);
    L->W3 = lalloc<__nv_bfloat16>(c, S * sh.Dout * sh.H, &rc); L->W2T = lalloc<__nv_bfloat16>(c, S * sh.H * sh.H, &rc);
    L->W3T = lalloc<__nv_bfloat16>(c, S * sh.Dout * sh.H, &rc);
    L->W1c = lalloc<__nv_bfloat16>(c, S * sh.H * sh.Din, &rc); L->W2c = lalloc<__nv_bfloat16>(c, S * sh.H * sh.H, &rc);
    L->W3c = lalloc<__nv_bfloat16>(c, S * sh.Dout * sh.H, &rc);
    L->du = lalloc<float>(c, S * L->ncap * N, &rc); L->dphi = lalloc<float>(c, S * L->ncap * N, &rc);
    L->dextra = lalloc<float>(c, S * L->ncap, &rc); L->dcond = lalloc<int>(c, S * L->ncap, &rc);
    L->X = lalloc<__nv_bfloat16>(c, S * rows * sh.Din, &rc); L->XT = lalloc<__nv_bfloat16>(c, S * rows * sh.Din, &rc);
    L->Xp = lalloc<__nv_bfloat16>(c, S * rows * sh.Din, &rc);
    L->H1 = lalloc<__nv_bfloat16>(c, S * rows * sh.H, &rc); L->H1T = lalloc<__nv_bfloat16>(c, S * rows * sh.H, &rc);
    L->H2 = lalloc<__nv_bfloat16>(c, S * rows * sh.H, &rc); L->H2T = lalloc<__nv_bfloat16>(c, S * rows * sh.H, &rc);
    L->Z1 = lalloc<float>(c, S * rows * sh.H, &rc); L->Z2 = lalloc<float>(c, S * rows * sh.H, &rc);
    L->O = lalloc<float>(c, S * rows * sh.Dout, &rc); L->dO = lalloc<float>(c, S * rows * sh.Dout, &rc);
    L->dOb = lalloc<__nv_bfloat16>(c, S * rows * sh.Dout, &rc); L->dOT = lalloc<__nv_bfloat16>(c, S * rows * sh.Dout, &rc);
    L->dZ2 = lalloc<float>(c, S * rows * sh.H, &rc); L->dZ2b = lalloc<__nv_bfloat16>(c, S * rows * sh.H, &rc);
    L->dZ2T = lalloc<__nv_bfloat16>(c, S * rows * sh.H, &rc); L->dZ1 = lalloc<float>(c, S * rows * sh.H, &rc);
    L->dZ1T = lalloc<__nv_bfloat16>(c, S * rows * sh.H, &rc);
    auto raw_rows = [&](RawRows &r, size_t n) {
        r.u = lalloc<float>(c, n * N, &rc); r.phi = lalloc<float>(c, n * N, &rc);
        r.extra = lalloc<float>(c, n, &rc); r.cond = lalloc<int>(c, n, &rc);
    };
    raw_rows(L->raw, S * rows);
    raw_rows(L->rcur, S * L->nprop);
    raw_rows(L->rprop, S * L->nprop);
    raw_rows(L->rsamp, S * L->nprop);
    L->logq = lalloc<double>(c, S * rows, &rc);
    L->lq_cur = lalloc<double>(c, S * L->nprop, &rc); L->lq_prop = lalloc<double>(c, S * L->nprop, &rc);
    L->H_cur = lalloc<double>(c, S * L->nprop, &rc); L->H_prop = lalloc<double>(c, S * L->nprop, &rc);
    L->pslot = lalloc<int>(c, S * L->nprop, &rc); L->pcond = lalloc<int>(c, S * L->nprop, &rc);
    L->prow = lalloc<uint32_t>(c, S * L->nprop, &rc);
    L->a_prop = lalloc<double2>(c, S * L->nprop * N, &rc);
    L->Ocur = lalloc<float>(c, S * rows * sh.Dout, &rc);  // the strides of O
    if (!c->dbl) {
        int64_t nq_total = 0;
        for (const auto &sd : c->samples) nq_total = std::max<int64_t>(nq_total, sd.q_off + sd.nq);
        L->Jdf = lalloc<float2>(c, std::max<int64_t>(nq_total, 1), &rc);
        if (rc == PT_OK) CK(launch_split_df(c->d_Jq, L->Jdf, nq_total, c->stream));
    }
    if (rc == PT_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&L->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->ev_mid, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(c, e, "pt_learn_init: stream");
    }
    L->max_losses = 1 << 16;
    L->losses = lalloc<double>(c, (size_t)L->max_losses, &rc);
    if (rc != PT_OK) return rc;
    // block-autoregressive masks: input features of mode k have degree blk(k) + 1, hidden unit h degree h % 8,
    // output k depends on hidden units of degree <= blk(k)
    const int per = N / ptgb::kLearnBlocks;
    std::vector<float> m1((size_t)sh.H * sh.Din), m2((size_t)sh.H * sh.H), m3((size_t)sh.Dout * sh.H);
    for (int h = 0; h < sh.H; ++h)
        for (int i = 0; i < sh.Din; ++i) m1[(size_t)h * sh.Din + i] = ((i / 3) / per + 1 <= h % ptgb::kLearnBlocks) ? 1.f : 0.f;
    for (int h2 = 0; h2 < sh.H; ++h2)
        for (int h1 = 0; h1 < sh.H; ++h1) m2[(size_t)h2 * sh.H + h1] = (h1 % ptgb::kLearnBlocks <= h2 % ptgb::kLearnBlocks) ? 1.f : 0.f;
    for (int o = 0; o < sh.Dout; ++o)
        for (int h = 0; h < sh.H; ++h) m3[(size_t)o * sh.H + h] = (h % ptgb::kLearnBlocks <= (o / 4) / per) ? 1.f : 0.f;
    // initial weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)), output layer scaled by 0.1, biases 0
    std::vector<float> hp(S * ps, 0.f);
    uint64_t st = seed ^ 0x9E3779B97F4A7C15ull;
    auto urand = [&]() {  // splitmix64
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (size_t s = 0; s < S; ++s) {
        float *P = hp.data() + s * ps;
        const double a1 = 1.0 / std::sqrt((double)sh.Din), a2 = 1.0 / std::sqrt((double)sh.H);
        for (size_t i = 0; i < (size_t)sh.H * sh.Din; ++i) P[sh.oW1 + i] = (float)((2 * urand() - 1) * a1);
        for (size_t i = 0; i < (size_t)sh.H * sh.H; ++i) P[sh.oW2 + i] = (float)((2 * urand() - 1) * a2);
        for (size_t i = 0; i < (size_t)sh.Dout * sh.H; ++i) P[sh.oW3 + i] = (float)((2 * urand() - 1) * a2 * 0.1);
    }
    CK(cudaMemcpy(L->P, hp.data(), hp.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L->M1, m1.data(), m1.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L->M2, m2.data(), m2.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L->M3, m3.data(), m3.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemset(L->Am, 0, S * ps * sizeof(float)));
    CK(cudaMemset(L->Av, 0, S * ps * sizeof(float)));
    if ((rc = learn_cast(c)) != PT_OK) return rc;
    return watchdog_sync(c);
}

int pt_learn_params(pt_ctx *c, float *P, int set) {
    if (!c || !P) return fail(c, PT_EINVAL, "pt_learn_params: NULL argument");
    if (!c->learn) return fail(c, PT_EINVAL, "pt_learn_params: call pt_learn_init first");
    LearnState &L = *c->learn;
    int rc = watchdog_sync(c);
    if (rc != PT_OK) return rc;
    const size_t n = (size_t)c->S * L.sh.psize;
    if (set) {
        CK(cudaMemcpy(L.P, P, n * sizeof(float), cudaMemcpyHostToDevice));
        if ((rc = learn_cast(c)) != PT_OK) return rc;
        return watchdog_sync(c);
    }
    CK(cudaMemcpy(P, L.P, n * sizeof(float), cudaMemcpyDeviceToHost));
    return PT_OK;
}

int pt_learn_shape(pt_ctx *c, int64_t *out) {
    if (!c || !out) return fail(c, PT_EINVAL, "pt_learn_shape: NULL argument");
    if (!c->learn) return fail(c, PT_EINVAL, "pt_learn_shape: call pt_learn_init first");
    const ptgb::LearnShape &sh = c->learn->sh;
    const int64_t v[12] = {sh.N, sh.H, sh.Din, sh.Dout, sh.ncold, (int64_t)sh.psize, (int64_t)sh.oW1, (int64_t)sh.ob1,
                           (int64_t)sh.oC1, (int64_t)sh.oW2, (int64_t)sh.ob2, (int64_t)sh.oW3};
    for (int i = 0; i < 12; ++i) out[i] = v[i];
    out[12] = (int64_t)sh.ob3;
    out[13] = c->learn->ndata;
    return PT_OK;
}

int pt_learn_eval(pt_ctx *c, const double *a, const int *cond, int rows, double *logq, double *extra, float *grad) {
    if (!c || !a || !cond || !logq) return fail(c, PT_EINVAL, "pt_learn_eval: NULL argument");
    if (!c->learn) return fail(c, PT_EINVAL, "pt_learn_eval: call pt_learn_init first");
    LearnState &L = *c->learn;
    const ptgb::LearnShape &sh = L.sh;
    if (rows < 1 || rows > L.rows || (grad && rows % 8)) return fail(c, PT_EINVAL, "pt_learn_eval: bad row count");
    int rc = watchdog_sync(c);
    if (rc != PT_OK) return rc;
    const size_t S = c->S, N = sh.N;
    std::vector<int> hc(S * rows);
    for (size_t i = 0; i < hc.size(); ++i) {
        if (cond[i] < 0 || cond[i] >= sh.ncold) return fail(c, PT_EINVAL, "pt_learn_eval: condition out of range");
        hc[i] = cond[i];
    }
    const size_t na = S * rows * N;
    double2 *da = nullptr;
    int *dc = nullptr;
    CK(cudaMalloc(&da, na * sizeof(double2)));
    cudaError_t e = cudaMalloc(&dc, hc.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(da, a, na * sizeof(double2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dc, hc.data(), hc.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(da); cudaFree(dc); return cuda_fail(c, e, "pt_learn_eval upload"); }
    FeatParams fp{};
    fp.a = da; fp.dbl = 1; fp.samples = c->d_samples; fp.slot = nullptr; fp.rows_per_sample = rows; fp.N = sh.N;
    fp.Din = sh.Din; fp.X = L.X; fp.XT = grad ? L.XT : nullptr; fp.ldxt = L.rows; fp.raw = L.raw;
    fp.raw_stride = rows; fp.raw_off = 0; fp.cond_in = dc; fp.x_stride = L.rows;
    e = launch_features(fp, c->S, c->stream);
    if (e == cudaSuccess) {
        rc = learn_forward(c, L.X, rows, L.raw.cond, rows, grad != nullptr);
        if (rc == PT_OK) {
            DensityParams d = density_params(L, L.O, L.raw, L.logq, rows, grad != nullptr);
            e = launch_density(d, c->S, c->stream);
            if (e == cudaSuccess && grad) rc = learn_backward(c, rows, L.raw.cond);
        }
    }
    if (e == cudaSuccess && rc == PT_OK) e = cudaStreamSynchronize(c->stream);
    cudaFree(da);
    cudaFree(dc);
    if (e != cudaSuccess) return cuda_fail(c, e, "pt_learn_eval");
    if (rc != PT_OK) return rc;
    CK(cudaMemcpy(logq, L.logq, S * rows * sizeof(double), cudaMemcpyDeviceToHost));
    if (extra) {
        std::vector<float> hx(S * rows);
        CK(cudaMemcpy(hx.data(), L.raw.extra, hx.size() * sizeof(float), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < hx.size(); ++i) extra[i] = hx[i];
    }
    if (grad) CK(cudaMemcpy(grad, L.Gr, S * sh.psize * sizeof(float), cudaMemcpyDeviceToHost));
    return PT_OK;
}

int pt_collect(pt_ctx *c, int64_t every, int rounds) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_collect: NULL context");
    if (!c->learn) return fail(c, PT_EINVAL, "pt_collect: call pt_learn_init first");
    if (every < 0 || rounds < 0) return fail(c, PT_EINVAL, "pt_collect: negative argument");
    LearnState &L = *c->learn;
    int rc;
    for (int r = 0; r < rounds; ++r) {
        if (L.ndata + L.nprop > L.ncap) break;
        if (every > 0 && (rc = pt_sweep(c, every)) != PT_OK) return rc;
        CK(launch_cold_rows(c->d_perm, c->S, c->R, c->nT, L.sh.ncold, L.pslot, L.prow, L.pcond, c->stream));
        FeatParams fp{};
        fp.a = c->d_a; fp.dbl = c->dbl ? 1 : 0; fp.samples = c->d_samples; fp.slot = L.pslot;
        fp.rows_per_sample = L.nprop; fp.N = L.sh.N; fp.Din = L.sh.Din; fp.X = nullptr; fp.XT = nullptr;
        fp.raw.u = L.du; fp.raw.phi = L.dphi; fp.raw.extra = L.dextra; fp.raw.cond = L.dcond;
        fp.raw_stride = L.ncap; fp.raw_off = L.ndata; fp.cond_in = L.pcond; fp.x_stride = L.rows;
        CK(launch_features(fp, c->S, c->stream));
        L.ndata += L.nprop;
    }
    return PT_OK;
}

int pt_train(pt_ctx *c, int steps, double lr, double *losses) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_train: NULL context");
    if (!c->learn) return fail(c, PT_EINVAL, "pt_train: call pt_learn_init first");
    LearnState &L = *c->learn;
    if (L.ndata < 1) return fail(c, PT_EINVAL, "pt_train: no training configurations (pt_collect)");
    if (steps < 0 || steps > L.max_losses || !(lr > 0.0)) return fail(c, PT_EINVAL, "pt_train: bad steps or lr");
    const ptgb::LearnShape &sh = L.sh;
    int rc;
    for (int t = 0; t < steps; ++t) {
        GatherParams gp{};
        gp.du = L.du; gp.dphi = L.dphi; gp.dextra = L.dextra; gp.dcond = L.dcond;
        gp.ndata = L.ndata; gp.stride = L.ncap;  // rows of sample s live at s * ncap, ndata of them collected
        gp.rows = L.Mb; gp.N = sh.N; gp.Din = sh.Din; gp.ldxt = L.rows; gp.seed = L.seed; gp.step = L.step++;
        gp.X = L.X; gp.XT = L.XT; gp.raw = L.raw; gp.x_stride = L.rows;
        CK(launch_gather(gp, c->S, c->stream));
        if ((rc = learn_forward(c, L.X, L.Mb, L.raw.cond, L.Mb, true)) != PT_OK) return rc;
        DensityParams d = density_params(L, L.O, L.raw, L.logq, L.Mb, true);
        CK(launch_density(d, c->S, c->stream));
        if ((rc = learn_backward(c, L.Mb, L.raw.cond)) != PT_OK) return rc;
        CK(launch_adam(L.P, L.Gr, L.Am, L.Av, (size_t)c->S * sh.psize, (float)lr, 0.9f, 0.999f, 1e-8f, ++L.adam_t,
                       c->stream));
        if ((rc = learn_cast(c)) != PT_OK) return rc;
        if (losses) {
            // mean over samples and rows of -(log q + extra): the NLL on the constraint surface
            CK(launch_learn_loss(L.logq, L.raw.extra, c->S, L.Mb, L.losses + t, c->stream));
        }
    }
    if ((rc = watchdog_sync(c)) != PT_OK) return rc;
    if (losses && steps > 0) CK(cudaMemcpy(losses, L.losses, steps * sizeof(double), cudaMemcpyDeviceToHost));
    return PT_OK;
}

int pt_global_move(pt_ctx *c) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_global_move: NULL context");
    if (!c->learn) return fail(c, PT_EINVAL, "pt_global_move: call pt_learn_init first");
    const int rc = run_global(c);
    if (rc != PT_OK) return rc;
    CK(launch_advance(c->d_ctl, 0, 0, 1, c->stream));
    c->global_rounds++;
    return PT_OK;
}

int pt_set_global_every(pt_ctx *c, int every) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_set_global_every: NULL context");
    if (every < 0) return fail(c, PT_EINVAL, "pt_set_global_every: negative interval");
    if (every > 0 && !c->learn) return fail(c, PT_EINVAL, "pt_set_global_every: call pt_learn_init first");
    if (c->learn) c->learn->global_every = every;
    return PT_OK;
}

int pt_set_global_blocks(pt_ctx *c, int lo, int hi) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_set_global_blocks: NULL context");
    if (!c->learn) return fail(c, PT_EINVAL, "pt_set_global_blocks: call pt_learn_init first");
    if (lo < 0 || hi < lo || hi >= ptgb::kLearnBlocks) return fail(c, PT_EINVAL, "pt_set_global_blocks: need 0 <= lo <= hi <= 7");
    int rc = watchdog_sync(c);
    if (rc != PT_OK) return rc;
    c->learn->blk_lo = lo;
    c->learn->blk_hi = hi;
    drop_graphs(c);  // the range is baked into captured segments
    return PT_OK;
}

int pt_set_global_sampler(pt_ctx *c, int one_launch) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_set_global_sampler: NULL context");
    if (!c->learn) return fail(c, PT_EINVAL, "pt_set_global_sampler: call pt_learn_init first");
    int rc = watchdog_sync(c);
    if (rc != PT_OK) return rc;
    c->learn->one_launch = one_launch != 0;
    drop_graphs(c);  // the choice is baked into captured segments
    return PT_OK;
}

int pt_check_wait(pt_ctx *c, int limit_ms) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_check_wait: NULL context");
    if (limit_ms < 1 || limit_ms > 60000) return fail(c, PT_EINVAL, "pt_check_wait: limit_ms must be 1..60000");
    int rc = watchdog_sync(c);
    if (rc != PT_OK) return rc;
    CK(launch_wait_probe(c->d_ctl, (unsigned long long)limit_ms * 1000000ull, c->stream));
    rc = watchdog_sync(c);
    // clear the status the probe left, so that the context goes on
    const int zero[2] = {0, 0};
    CK(cudaMemcpy(&c->d_ctl->error, zero, sizeof(zero), cudaMemcpyHostToDevice));
    return rc;
}

int pt_counters(pt_ctx *c, int64_t *sweeps_done, int64_t *swap_passes) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_counters: NULL context");
    if (sweeps_done) *sweeps_done = c->sweeps_done;
    if (swap_passes) *swap_passes = c->swap_passes;
    return PT_OK;
}

int pt_sync(pt_ctx *c) {
    if (!c) return fail(nullptr, PT_EINVAL, "pt_sync: NULL context");
    return watchdog_sync(c);
}

int pt_destroy(pt_ctx *c) {
    if (!c) return PT_OK;
    cudaStreamSynchronize(c->stream);
    if (c->learn) {
        if (c->learn->side) { cudaStreamSynchronize(c->learn->side); cudaStreamDestroy(c->learn->side); }
        if (c->learn->ev_fork) cudaEventDestroy(c->learn->ev_fork);
        if (c->learn->ev_mid) cudaEventDestroy(c->learn->ev_mid);
        if (c->learn->ev_join) cudaEventDestroy(c->learn->ev_join);
        delete c->learn;
        c->learn = nullptr;
    }
    free_all(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return PT_OK;
}

const char *pt_last_error(const pt_ctx *c) {
    return c ? c->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
