// gcmg_defect_noalloc: the defect and its max-norm for callers that cannot
// allocate device memory.
//
// Who needs it: code whose device memory is entirely owned by another
// allocator (a framework's caching pool, or an arena reserved up front under a
// fixed memory budget) and code running in a latency-critical loop that must
// not pay the implicit device-wide synchronisation of cudaMalloc / cudaFree.
// Such callers cannot create a gcmg context (gcmg_create allocates the level
// hierarchy), so this entry point takes every input and output as caller
// buffers and keeps its only scratch -- the per-block partial maxima of the
// norm reduction -- in a fixed-size array in the library's own device image.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents.  Each call overwrites every slot it reads before reading
// it, so nothing has to be cleared between calls; but two calls that overlap
// on the GPU (different streams, or different host threads on one device)
// race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "gcmg.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItemsPerThread = 4;
constexpr int kItemsPerBlock = kThreads * kItemsPerThread;
// capacity: 65536 blocks of 1024 items (grid nodes + ghosts), i.e. up to
// 67,108,864 items; 512 KiB of device memory held until the process exits
constexpr int kMaxBlocks = 65536;
constexpr long long kMaxItems = (long long)kMaxBlocks * kItemsPerBlock;
constexpr int kStencil = 27;   // per-ghost stencil stride (unused slots: weight 0)
constexpr int kMaxDevices = 64;

// slots [0, kMaxBlocks): per-block maxima of |r|; slot kMaxBlocks: the norm
static __device__ __align__(256) double g_noalloc_scratch[kMaxBlocks + 1];

// device addresses of g_noalloc_scratch, looked up once per device
double *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

__device__ __forceinline__ double block_max(double v) {
    __shared__ double wmax[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < kThreads / 32 ? wmax[threadIdx.x] : 0.0;
    if (threadIdx.x < 32)
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double abs_or_inf(double r) {
    const double a = fabs(r);
    return a != a ? __longlong_as_double(0x7ff0000000000000ll) : a;
}

// Items [0, nn) are grid nodes, [nn, nn + ng) ghosts.  Inside nodes:
// r = f + Lap_h u; outside nodes: r = 0; ghosts: r = g - sum_k w_k u(stn_k)
// over the 3^D slots a stencil can use (rows of kStencil slots).
// Each block stores its maximum |r| in partials[blockIdx.x].
template <int D>
__global__ void __launch_bounds__(kThreads)
k_defect_partials(long long nn, long long ng, long long s0, long long s1, double inv_h2, const uint8_t *__restrict__ type,
                  const double *__restrict__ u, const double *__restrict__ f, const int32_t *__restrict__ gnode,
                  const int32_t *__restrict__ stn, const double *__restrict__ w, const double *__restrict__ g,
                  double *__restrict__ r, double *__restrict__ partials) {
    double m = 0.0;
    const long long base = (long long)blockIdx.x * kItemsPerBlock;
#pragma unroll
    for (int k = 0; k < kItemsPerThread; k++) {
        const long long i = base + k * kThreads + threadIdx.x;
        if (i < nn) {
            const uint8_t t = type[i] & 3;
            if (t == 1) {
                const double up = u[i];
                double lap = (u[i - 1] - up) + (u[i + 1] - up) + (u[i - s0] - up) + (u[i + s0] - up);
                if (D == 3) lap += (u[i - s1] - up) + (u[i + s1] - up);
                const double ri = f[i] + lap * inv_h2;
                r[i] = ri;
                m = fmax(m, abs_or_inf(ri));
            } else if (t == 0) {
                r[i] = 0.0;
            }
        } else if (i < nn + ng) {
            const long long q = i - nn;
            double s = 0.0;
            constexpr int K = D == 2 ? 9 : 27;   // 2D stencils fill the first 9 slots of a row
#pragma unroll
            for (int j = 0; j < K; j++) s += w[q * kStencil + j] * u[stn[q * kStencil + j]];
            const double ri = g[q] - s;
            r[gnode[q]] = ri;
            m = fmax(m, abs_or_inf(ri));
        }
    }
    m = block_max(m);
    if (threadIdx.x == 0) partials[blockIdx.x] = m;
}

// single block: maximum of partials[0, nb) into partials[kMaxBlocks]
__global__ void __launch_bounds__(kThreads) k_reduce_partials(double *partials, int nb) {
    double m = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) m = fmax(m, partials[i]);
    m = block_max(m);
    if (threadIdx.x == 0) partials[kMaxBlocks] = m;
}

}  // namespace

extern "C" gcmg_status gcmg_defect_noalloc(int dim, int n, double h, const uint8_t *type_dev, const double *u_dev,
                                           const double *f_dev, int64_t ng, const int32_t *gnode_dev,
                                           const int32_t *stn_dev, const double *w_dev, const double *g_dev,
                                           double *r_dev, double *norm_host, void *stream) {
    if ((dim != 2 && dim != 3) || n < 3 || !(h > 0.0) || ng < 0 || !type_dev || !u_dev || !f_dev || !r_dev)
        return GCMG_E_ARG;
    if (ng > 0 && (!gnode_dev || !stn_dev || !w_dev || !g_dev)) return GCMG_E_ARG;
    // capacity, checked without overflow: n^dim grows one factor at a time
    if (n > kMaxItems || ng > kMaxItems) return GCMG_E_SIZE;
    long long nn = 1;
    for (int a = 0; a < dim; a++) {
        nn *= n;
        if (nn > kMaxItems) return GCMG_E_SIZE;
    }
    if (ng > kMaxItems - nn) return GCMG_E_SIZE;
    // one-time set-up per device: the device address of the scratch array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GCMG_E_CUDA;
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return GCMG_E_CUDA;
            }
            g_scratch_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((nn + ng + kItemsPerBlock - 1) / kItemsPerBlock);
    const long long s0 = dim == 2 ? n : (long long)n * n, s1 = n;
    const double inv_h2 = 1.0 / (h * h);
    if (dim == 2)
        k_defect_partials<2><<<nb, kThreads, 0, s>>>(nn, ng, s0, s1, inv_h2, type_dev, u_dev, f_dev, gnode_dev,
                                                     stn_dev, w_dev, g_dev, r_dev, scratch);
    else
        k_defect_partials<3><<<nb, kThreads, 0, s>>>(nn, ng, s0, s1, inv_h2, type_dev, u_dev, f_dev, gnode_dev,
                                                     stn_dev, w_dev, g_dev, r_dev, scratch);
    k_reduce_partials<<<1, kThreads, 0, s>>>(scratch, nb);
    if (cudaGetLastError() != cudaSuccess) return GCMG_E_CUDA;
    if (norm_host) {
        if (cudaMemcpyAsync(norm_host, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return GCMG_E_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return GCMG_E_CUDA;
    }
    return GCMG_OK;
}
