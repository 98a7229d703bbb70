// lb_noalloc.cu -- lb_totals_noalloc: the FP64 mass/momentum reduction of
// the observe pass, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a fixed device
// arena it may not grow, or inside a framework that forbids allocation on its
// hot path.  lb_create allocates, and lb_create_in still needs a workspace for
// the reduction slots.  This entry point takes the caller's device fields and
// output and keeps its scratch -- one FP64 partial-sum slot per CTA and the
// CTA arrival ticket -- in a file-scope device array of fixed size, which
// every GPU that loads the library holds until the process exits.
#include <mutex>

#include "lb_internal.h"

namespace lbgb {
namespace {

constexpr int kThreads = 256;
constexpr int kSitesPerThread = 16;
constexpr long long kSitesPerBlock = (long long)kThreads * kSitesPerThread;   // 4096
constexpr int kMaxBlocks = LB_NOALLOC_MAX_SITES / kSitesPerBlock;              // 4096

// Layout of the scratch array: the CTA arrival ticket in the first 256
// bytes, then one slot of four FP64 partial sums per CTA.
struct NoAllocScratch {
    unsigned int ticket;           // must be zero when a call starts
    unsigned int pad_[63];
    double slots[kMaxBlocks][4];
};
static_assert(kMaxBlocks * kSitesPerBlock == LB_NOALLOC_MAX_SITES, "scratch sizing");
constexpr size_t kScratchDoubles = sizeof(NoAllocScratch) / sizeof(double);   // 128 KB + 256 B

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Each CTA sums kSitesPerBlock sites into its slot; the last CTA to arrive
// sums the slots in a fixed order (deterministic) and writes `out`.
__global__ void __launch_bounds__(kThreads)
    k_totals(NoAllocScratch* sc, long long n, const double* __restrict__ rA,
             const double* __restrict__ rB, const double* __restrict__ ux,
             const double* __restrict__ uy, double* __restrict__ out) {
    __shared__ double s_red[kThreads / 32][4];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const long long base = (long long)blockIdx.x * kSitesPerBlock;
    for (int k = 0; k < kSitesPerThread; ++k) {
        const long long i = base + (long long)k * kThreads + tid;
        if (i < n) {
            const double a = rA[i], b = rB[i], tot = a + b;
            v[0] += a;
            v[1] += b;
            v[2] += tot * ux[i];
            v[3] += tot * uy[i];
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = warp_sum_d(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) s_red[warp][k] = v[k];
    __syncthreads();
    if (tid == 0) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < kThreads / 32; ++w)
#pragma unroll
            for (int k = 0; k < 4; ++k) s[k] += s_red[w][k];
#pragma unroll
        for (int k = 0; k < 4; ++k) sc->slots[blockIdx.x][k] = s[k];
        __threadfence();
        s_last = atomicAdd(&sc->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const volatile double(*slots)[4] = sc->slots;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = tid; b < (int)gridDim.x; b += kThreads)
#pragma unroll
        for (int k = 0; k < 4; ++k) s[k] += slots[b][k];
#pragma unroll
    for (int k = 0; k < 4; ++k) s[k] = warp_sum_d(s[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) s_red[warp][k] = s[k];
    __syncthreads();
    if (tid == 0) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < kThreads / 32; ++w)
#pragma unroll
            for (int k = 0; k < 4; ++k) t[k] += s_red[w][k];
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = t[k];
        sc->ticket = 0u;
    }
}

// Unique id of the calling thread's current context (cuCtxGetId: unique over
// the life of the process, unlike the CUcontext handle, which a context
// created after a device reset may reuse).  False when there is no current
// context yet or the driver does not offer the call.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) ==
                cudaSuccess && qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) ==
                cudaSuccess && qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrentFn>(a);
            get_id = reinterpret_cast<CtxGetIdFn>(b);
        }
        cudaGetLastError();
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the scratch array, looked up once per device and
// context: a context created after a device reset loads the module again,
// possibly elsewhere, so its address is looked up afresh.
std::mutex g_mu;
void* g_addr[64] = {nullptr};
unsigned long long g_ctx[64] = {0};

lb_status scratch_address(NoAllocScratch** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LB_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);
    if (!g_addr[dev] || !have_id || g_ctx[dev] != id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return LB_ERR_CUDA;
        }
        // the lookup made the device's primary context current if it was not
        if (!have_id) have_id = current_context_id(&id);
        g_addr[dev] = p;
        g_ctx[dev] = have_id ? id : 0;
        if (!have_id) {   // no context id to key on: look up again next call
            *out = reinterpret_cast<NoAllocScratch*>(p);
            g_addr[dev] = nullptr;
            return LB_OK;
        }
    }
    *out = reinterpret_cast<NoAllocScratch*>(g_addr[dev]);
    return LB_OK;
}

}  // namespace
}  // namespace lbgb

extern "C" lb_status lb_totals_noalloc(int32_t nx, int32_t ny, const double* rho_A,
                                        const double* rho_B, const double* ux, const double* uy,
                                        double* totals, void* stream) {
    using namespace lbgb;
    if (nx < 1 || ny < 1 || !rho_A || !rho_B || !ux || !uy || !totals) return LB_ERR_INVALID;
    const long long n = (long long)nx * ny;
    if (n > LB_NOALLOC_MAX_SITES) return LB_ERR_INVALID;
    NoAllocScratch* sc = nullptr;
    lb_status s = scratch_address(&sc);
    if (s != LB_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // The ticket must start at zero; a call that was cut short could have
    // left it non-zero.  The slots are overwritten by every call.
    cudaError_t e = cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return LB_ERR_CUDA;
    const unsigned blocks = (unsigned)((n + kSitesPerBlock - 1) / kSitesPerBlock);
    k_totals<<<blocks, kThreads, 0, st>>>(sc, n, rho_A, rho_B, ux, uy, totals);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}
