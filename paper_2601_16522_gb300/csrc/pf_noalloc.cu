// pf_noalloc.cu -- per-field totals of a caller-owned device state without
// any allocation (see pf_totals_noalloc in include/pf.h).
//
// Some callers cannot allocate device memory at the point where they need the
// totals: cudaMalloc and cudaFree can synchronise the whole device, which a
// solver loop that keeps several streams busy (or a host thread with a
// latency budget) cannot afford; and a caller whose device memory is entirely
// owned by another allocator (a framework's caching arena) has nothing left
// to hand out.  This variant of the totals reduction therefore takes its
// per-block scratch from a fixed array in device global memory that the
// library reserves when it is loaded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "../../include/pf.h"

namespace {

// Maximum with NaN propagation: a NaN anywhere in a field makes its maximum
// NaN (as its sum is), instead of being skipped by the comparison.
__device__ __forceinline__ double nan_max(double m, double v) { return (v > m || v != v) ? v : m; }

constexpr int kBlocks = PF_NOALLOC_MAX_BLOCKS;   // per-field partial slots
constexpr int kThreads = 256;

// Scratch shared by every call on a device: [field][block][sum, max].  Each
// call writes every slot it later reads, so nothing has to be cleared, but
// calls whose kernels overlap on the GPU race on it.
static __device__ __align__(256) double g_scratch[(size_t)PF_NOALLOC_MAX_FIELDS * kBlocks * 2];

// Stage 1: block (b, f) reduces cells [b*chunk, (b+1)*chunk) of field f.
__global__ void totals_partial(const double *__restrict__ u, long long V, double *scratch, int nblk)
{
    const int f = blockIdx.y;
    const long long chunk = (V + nblk - 1) / nblk;
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = lo + chunk < V ? lo + chunk : V;
    const double *uf = u + (long long)f * V;
    double s = 0.0, m = -INFINITY;
    for (long long i = lo + threadIdx.x; i < hi; i += kThreads) {
        const double v = uf[i];
        s += v;
        m = nan_max(m, v);
    }
    __shared__ double ss[kThreads], sm[kThreads];
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = kThreads / 2; o >= 1; o >>= 1) {
        if ((int)threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sm[threadIdx.x] = nan_max(sm[threadIdx.x], sm[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double *slot = scratch + ((size_t)f * kBlocks + blockIdx.x) * 2;
        slot[0] = ss[0];
        slot[1] = sm[0];
    }
}

// Stage 2: one block per field folds the nblk partials in a fixed order.
__global__ void totals_final(const double *scratch, int nblk, double dv, double *sum_out, double *max_out)
{
    const int f = blockIdx.x;
    double s = 0.0, m = -INFINITY;
    for (int b = threadIdx.x; b < nblk; b += kThreads) {
        const double *slot = scratch + ((size_t)f * kBlocks + b) * 2;
        s += slot[0];
        m = nan_max(m, slot[1]);
    }
    __shared__ double ss[kThreads], sm[kThreads];
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = kThreads / 2; o >= 1; o >>= 1) {
        if ((int)threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sm[threadIdx.x] = nan_max(sm[threadIdx.x], sm[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (sum_out) sum_out[f] = ss[0] * dv;
        if (max_out) max_out[f] = sm[0];
    }
}

// Device address of g_scratch, looked up once per device and context (the
// host-side name of the array is only a stand-in and must never be handed
// to a kernel).  The cache is keyed on the current context's unique id, so a
// context created after cudaDeviceReset (which reloads the module and moves
// the array) is looked up afresh instead of reusing a stale address.
constexpr int kMaxDevices = 64;
std::mutex g_lock;
double *g_addr[kMaxDevices] = {nullptr};
unsigned long long g_ctx[kMaxDevices] = {0};

// Unique id of the current context (0 if the driver cannot say).
unsigned long long current_context_id()
{
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = (PFN_cuCtxGetCurrent_v4000)p;
        p = nullptr;
        if (cudaGetDriverEntryPoint("cuCtxGetId", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PFN_cuCtxGetId_v12000)p;
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_cur && get_id && get_cur(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
    return 0;
}

int scratch_for_current_device(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PF_EDEVICE;
    if (dev < 0 || dev >= kMaxDevices) return PF_EDEVICE;
    const unsigned long long ctx = current_context_id();   // 0 before the runtime made one current
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_addr[dev] || ctx == 0 || g_ctx[dev] != ctx) {
        // the lookup also initialises the device's primary context if needed
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return PF_EDEVICE;
        g_addr[dev] = static_cast<double *>(p);
        g_ctx[dev] = current_context_id();
    }
    *out = g_addr[dev];
    return PF_OK;
}

}  // namespace

extern "C" int pf_totals_noalloc(const double *u_dev, int n_fields, long long n_cells, double dv, double *sum_dev,
                                 double *max_dev, void *cuda_stream)
{
    if (!u_dev || n_cells < 1 || n_fields < 1 || (!sum_dev && !max_dev)) return PF_EINVAL;
    if (n_fields > PF_NOALLOC_MAX_FIELDS) return PF_EINVAL;
    double *scratch = nullptr;
    int st = scratch_for_current_device(&scratch);
    if (st) return st;
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    long long nb = (n_cells + 4095) / 4096;
    const int nblk = (int)(nb < kBlocks ? (nb > 0 ? nb : 1) : kBlocks);
    totals_partial<<<dim3(nblk, n_fields), kThreads, 0, s>>>(u_dev, n_cells, scratch, nblk);
    if (cudaGetLastError() != cudaSuccess) return PF_EDEVICE;
    totals_final<<<n_fields, kThreads, 0, s>>>(scratch, nblk, dv, sum_dev, max_dev);
    if (cudaGetLastError() != cudaSuccess) return PF_EDEVICE;
    return PF_OK;
}
