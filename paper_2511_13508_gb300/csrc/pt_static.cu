// pt_static.cu -- pt_energy_fp64_static: full FP64 energies of a batch of chains without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Some callers must not allocate device memory: a host program whose device memory is handed out by
// another runtime's pool, a real-time loop in which cudaMalloc/cudaFree would synchronise the device,
// or a plug-in that may only use the buffers its host gives it.  They own the inputs and outputs;
// the only working memory this entry point needs -- the canonical quadruplet table of the comb --
// lives in the file-scope array below, which every GPU that loads the library holds until exit.
//
// The kernel is a variant of the plain FP64 energy kernel (one thread block per chain, one thread
// per quadruplet term, shared-memory tree reduction), reading its quadruplet table from that array.
#include <cuda.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pt.h"

namespace ptgb {
void set_global_error(const char *msg);  // message returned by pt_last_error(NULL)
}

namespace {

constexpr int kStaticMaxN = 64;           // largest mode count the table holds
constexpr int kStaticMaxQuads = 20336;    // quadruplets of the 64-mode comb
constexpr int kStaticThreads = 256;

// Working table shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) int4 g_static_quads[kStaticMaxQuads];

// The table's device address belongs to the CUDA context in which it was looked up: one entry per context
// (a plug-in host may run its own driver-API context next to the runtime's primary context).
struct TableAddr {
    CUcontext ctx;
    void *table;
};
std::vector<TableAddr> g_static_tables;
std::mutex g_static_mutex;

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
std::once_flag g_ctx_once;

// The context current on this thread (nullptr if none), through the driver entry point the runtime hands out
// (no link-time dependence on the driver library).
bool current_context(CUcontext *ctx) {
    std::call_once(g_ctx_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
        else
            (void)cudaGetLastError();
    });
    *ctx = nullptr;
    return g_ctx_get_current && g_ctx_get_current(ctx) == CUDA_SUCCESS;
}

// One thread per first index a: writes every a<b<c<d with a+d = b+c, in lexicographic (a,b,c) order,
// at the canonical position (the count of quadruplets with a smaller first index comes first).
__global__ void static_fill_quads(int4 *quads, int N) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    int64_t pos = 0;
    for (int a2 = 0; a2 < a; ++a2)
        for (int b = a2 + 1; b < N; ++b) {
            const int cnt = N - 1 - 2 * b + a2;
            if (cnt > 0) pos += cnt;
        }
    for (int b = a + 1; b < N; ++b)
        for (int c = b + 1; c < N; ++c) {
            const int d = b + c - a;
            if (d >= N) break;
            quads[pos++] = make_int4(a, b, c, d);
        }
}

__device__ __forceinline__ double2 cm(double2 x, double2 y) {
    return make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
}

// E = -cc sum_q J_q Re( conj(a_a) a_b a_c conj(a_d) ) for chain blockIdx.x.
__global__ void __launch_bounds__(kStaticThreads) static_energy_kernel(const int4 *quads, int64_t nq,
                                                                        const double *J, const double2 *a,
                                                                        int N, double cc, double *E) {
    __shared__ double2 sa[kStaticMaxN];
    __shared__ double buf[kStaticThreads];
    const double2 *x = a + (int64_t)blockIdx.x * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) sa[k] = x[k];
    __syncthreads();
    double local = 0.0;
    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) {
        const int4 Q = quads[q];
        const double2 ca = make_double2(sa[Q.x].x, -sa[Q.x].y), cd = make_double2(sa[Q.w].x, -sa[Q.w].y);
        local += J[q] * cm(cm(ca, sa[Q.y]), cm(sa[Q.z], cd)).x;
    }
    buf[threadIdx.x] = local;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) buf[threadIdx.x] += buf[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) E[blockIdx.x] = -cc * buf[0];
}

int static_fail(int code, const std::string &msg) {
    ptgb::set_global_error(msg.c_str());
    return code;
}

// Device address of the table in the current context.  Looked up with cudaGetSymbolAddress on every call
// made while the stream is not capturing (the address is then always the current context's, even after a
// device reset); a call made during stream capture takes the address an earlier call recorded for the
// current context.
int table_address(cudaStream_t s, void **table) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        return static_fail(PT_ECUDA, std::string("pt_energy_fp64_static: cannot query the stream: ") + cudaGetErrorString(e));
    }
    CUcontext ctx = nullptr;
    if (!current_context(&ctx))
        return static_fail(PT_ECUDA, "pt_energy_fp64_static: cannot read the current CUDA context");
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (cap == cudaStreamCaptureStatusNone || !ctx) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_quads);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return static_fail(PT_ECUDA, std::string("pt_energy_fp64_static: cudaGetSymbolAddress failed: ") +
                                             cudaGetErrorString(e));
        }
        if (!ctx && (!current_context(&ctx) || !ctx))  // the lookup above made the primary context current
            return static_fail(PT_ECUDA, "pt_energy_fp64_static: no current CUDA context");
        for (auto &t : g_static_tables)
            if (t.ctx == ctx) { t.table = p; *table = p; return PT_OK; }
        g_static_tables.push_back({ctx, p});
        *table = p;
        return PT_OK;
    }
    for (auto &t : g_static_tables)
        if (t.ctx == ctx) { *table = t.table; return PT_OK; }
    return static_fail(PT_EINVAL, "pt_energy_fp64_static: the first call in a CUDA context must come before any "
                                  "stream capture (it looks up the static table's address)");
}

}  // namespace

extern "C" int pt_energy_fp64_static(int N, int n_chains, const double *J, const double *a, double *E,
                                     double cc, void *stream) {
    if (N < 4 || N > kStaticMaxN)
        return static_fail(PT_EINVAL, "pt_energy_fp64_static: N must be in [4, 64] (size of the static table)");
    if (n_chains < 0 || (n_chains > 0 && (!J || !a || !E)))
        return static_fail(PT_EINVAL, "pt_energy_fp64_static: need n_chains >= 0 and device pointers J, a, E");
    if (n_chains == 0) return PT_OK;
    // an error left pending by earlier work on this thread is reported as such, not as this call's failure
    const cudaError_t pre = cudaGetLastError();
    if (pre != cudaSuccess)
        return static_fail(PT_ECUDA, std::string("pt_energy_fp64_static: CUDA error pending from earlier work: ") +
                                         cudaGetErrorString(pre));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    void *table = nullptr;
    const int rc = table_address(s, &table);
    if (rc != PT_OK) return rc;
    int64_t nq = 0;
    for (int aa = 0; aa < N; ++aa)
        for (int b = aa + 1; b < N; ++b) {
            const int cnt = N - 1 - 2 * b + aa;
            if (cnt > 0) nq += cnt;
        }
    int4 *quads = reinterpret_cast<int4 *>(table);
    static_fill_quads<<<1, kStaticMaxN, 0, s>>>(quads, N);
    static_energy_kernel<<<n_chains, kStaticThreads, 0, s>>>(quads, nq, J, reinterpret_cast<const double2 *>(a), N,
                                                             cc, E);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return static_fail(PT_ECUDA, std::string("pt_energy_fp64_static: kernel launch failed: ") + cudaGetErrorString(e));
    return PT_OK;
}
