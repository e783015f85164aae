// Allocation-free forward operator K = Psi x = sum_i x_i a_i a_i^H.
//
// For callers that must not allocate device memory: code running inside a
// host framework whose allocator owns all device memory, real-time loops
// where cudaMalloc's implicit device synchronisation is not acceptable, or
// plug-ins that may only use the buffers they are handed.  Instead of a
// context (img_create allocates), this entry point keeps its working set -
// the separable steering tables and the split-K partial matrices - in one
// file-scope static device array of fixed size (g_psi_scratch below).  Every
// GPU that loads the library holds that array until the process exits.
//
// The arithmetic is the CUDA-core FP32 forward of img_psi: pixels are split
// into contiguous ranges, one CTA per range accumulates its partial p x p
// matrix, and a second kernel sums the partials in a fixed order in FP64.
#include <cuda.h>

#include <mutex>
#include <utility>

#include "../../include/img.h"
#include "cta_ops.cuh"

namespace img {
namespace {

constexpr int kNoAllocMaxP = 64;        // antennas
constexpr int kNoAllocMaxN = 256;       // grid lines per axis
constexpr int kNoAllocMaxQ = 65536;     // pixels
constexpr int kNoAllocParts = 64;       // split-K partial matrices

constexpr size_t kTableBytes = (size_t)kNoAllocMaxN * kNoAllocMaxP * sizeof(float2);
constexpr size_t kPartBytes = (size_t)kNoAllocParts * kNoAllocMaxP * kNoAllocMaxP * sizeof(float2);
constexpr size_t kScratchBytes = 2 * kTableBytes + kPartBytes;   // 2.25 MiB

// Shared by every call of img_psi_noalloc on a device.  Each call rewrites
// the tables and every partial it later reads, so nothing needs clearing;
// calls whose work overlaps on the GPU (different streams) race on it.
static __device__ __align__(256) unsigned char g_psi_scratch[kScratchBytes];

// Steering tables (as k_tables): El[il*p+k] = p^{-1/2} e^{-j2pi x_k l/lam},
// Em[im*p+k] = e^{-j2pi y_k m/lam}, FP64 phase reduction before sincospi.
__global__ void k_noalloc_tables(JobDev J) {
    const int p = J.p;
    const int total = p * (J.n_l + J.n_m);
    const double sc = rsqrt((double)p);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const bool isl = e < p * J.n_l;
        const int e2 = isl ? e : e - p * J.n_l;
        const int g = e2 / p, k = e2 - g * p;
        const double coord = isl ? J.ant[3 * k + 0] : J.ant[3 * k + 1];
        const double dir = isl ? J.lg[g] : J.mg[g];
        const double t = coord * dir / J.lam;
        const double r = t - rint(t);
        double s, c;
        sincospi(2.0 * r, &s, &c);
        if (isl) J.El[e2] = make_float2((float)(c * sc), (float)(-s * sc));
        else J.Em[e2] = make_float2((float)c, (float)(-s));
    }
}

// CTA b: part[b] = sum over pixels [b*per, (b+1)*per) of x_i a_i a_i^H.
__global__ void k_noalloc_partial(JobDev J, const double *x, float2 *part, int per) {
    extern __shared__ float4 smem4[];
    float2 *C = reinterpret_cast<float2 *>(smem4);
    __shared__ float wsm[kTile];
    const int i0 = blockIdx.x * per;
    const int n = max(0, min(per, J.Q - i0));
    const int p = J.p;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float2 *K = part + (size_t)blockIdx.x * p * p;
    // p <= 64: one 64 x 64 output tile per thread block
    const int r0 = ty * 4, c0 = tx * 4;
    float2 acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
    for (int j0 = 0; j0 < n; j0 += kTile) {
        const int np = min(kTile, n - j0);
        for (int e = threadIdx.x; e < kTile * p; e += kThreads) {
            const int j = e / p, k = e - j * p;
            float2 c = make_float2(0.f, 0.f);
            if (j < np) {
                const int i = i0 + j0 + j;
                const int im = i / J.n_l, il = i - im * J.n_l;
                c = steer(J, il, im, k);
            }
            C[e] = c;
        }
        if (threadIdx.x < kTile) wsm[threadIdx.x] = threadIdx.x < np ? (float)x[i0 + j0 + threadIdx.x] : 0.f;
        __syncthreads();
        if (r0 < p && c0 < p) {
            for (int j = 0; j < np; ++j) {
                const float wj = wsm[j];
                const float2 *cj = C + j * p;
                float2 ck[4], cl[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float2 t = (r0 + r < p) ? cj[r0 + r] : make_float2(0.f, 0.f);
                    ck[r] = make_float2(wj * t.x, wj * t.y);
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float2 t = (c0 + c < p) ? cj[c0 + c] : make_float2(0.f, 0.f);
                    cl[c] = make_float2(t.x, -t.y);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) cfma(acc[r][c], ck[r], cl[c]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int k = r0 + r, l = c0 + c;
            if (k < p && l < p) K[(size_t)l * p + k] = acc[r][c];
        }
}

__global__ void k_noalloc_reduce(const float2 *part, int nparts, int pp, double2 *Kout) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < pp; e += gridDim.x * blockDim.x) {
        double sx = 0.0, sy = 0.0;
        for (int b = 0; b < nparts; ++b) {
            const float2 v = part[(size_t)b * pp + e];
            sx += v.x;
            sy += v.y;
        }
        Kout[e] = make_double2(sx, sy);
    }
}

// Identity of the current CUDA context, or 0 when the driver cannot say.
// The driver's functions are reached through the runtime's entry-point query,
// so the library links no driver library.
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
std::mutex g_mu;
CtxGetCurrentFn g_get_cur = nullptr;
CtxGetIdFn g_get_id = nullptr;
bool g_looked = false;

unsigned long long context_id() {
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_looked) {
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", reinterpret_cast<void **>(&g_get_cur), 12000,
                                                 cudaEnableDefault, &q) != cudaSuccess ||
                q != cudaDriverEntryPointSuccess)
                g_get_cur = nullptr;
            if (cudaGetDriverEntryPointByVersion("cuCtxGetId", reinterpret_cast<void **>(&g_get_id), 12000,
                                                 cudaEnableDefault, &q) != cudaSuccess ||
                q != cudaDriverEntryPointSuccess)
                g_get_id = nullptr;
            g_looked = true;
        }
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!g_get_cur || !g_get_id || g_get_cur(&c) != CUDA_SUCCESS || !c || g_get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_psi_scratch for the current device (the host-side name
// is only a stand-in), looked up with cudaGetSymbolAddress once per device
// and context: cudaDeviceReset ends the context, and the array may sit
// elsewhere in the next one, so a new context identity triggers a new lookup.
struct ScratchAddr {
    unsigned long long ctx = 0;
    void *ptr = nullptr;
};
ScratchAddr g_addr[128];

cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    const unsigned long long ctx = context_id();
    std::lock_guard<std::mutex> lock(g_mu);
    ScratchAddr &a = g_addr[dev];
    if (!a.ptr || (ctx != 0 && ctx != a.ctx)) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_psi_scratch);
        if (e != cudaSuccess) return e;
        a.ptr = ptr;
        a.ctx = ctx;
    }
    *out = a.ptr;
    return cudaSuccess;
}

// One launch whose own status is returned (earlier errors of unrelated work
// are neither reported nor cleared here).
template <class... P, class... A>
cudaError_t launch(void (*k)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t st, A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

}  // namespace
}  // namespace img

extern "C" img_status img_psi_noalloc(int p, int n_l, int n_m, const double *ant_xyz,
                                      const double *l, const double *m, double lambda,
                                      const double *x, double *Kout, void *stream) {
    using namespace img;
    if (!ant_xyz || !l || !m || !x || !Kout) return IMG_EINVAL;
    if (p < 2 || n_l < 1 || n_m < 1 || !(lambda > 0.0)) return IMG_EINVAL;
    if (p > kNoAllocMaxP || n_l > kNoAllocMaxN || n_m > kNoAllocMaxN ||
        (long long)n_l * n_m > kNoAllocMaxQ)
        return IMG_ENOMEM;   // beyond the fixed capacity of the static scratch
    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return IMG_ECUDA;
    unsigned char *b = static_cast<unsigned char *>(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    JobDev J{};
    J.p = p;
    J.n_l = n_l;
    J.n_m = n_m;
    J.Q = n_l * n_m;
    J.lam = lambda;
    J.ant = ant_xyz;
    J.lg = l;
    J.mg = m;
    J.El = reinterpret_cast<float2 *>(b);
    J.Em = reinterpret_cast<float2 *>(b + kTableBytes);
    float2 *part = reinterpret_cast<float2 *>(b + 2 * kTableBytes);
    const int Q = J.Q;
    int per = (Q + kNoAllocParts - 1) / kNoAllocParts;
    per = ((per + kTile - 1) / kTile) * kTile;
    const int used = (Q + per - 1) / per;
    const size_t sm = (size_t)p * kTile * sizeof(float2);
    if (launch(k_noalloc_tables, 16, kThreads, 0, st, J) != cudaSuccess) return IMG_ECUDA;
    if (launch(k_noalloc_partial, used, kThreads, sm, st, J, x, part, per) != cudaSuccess) return IMG_ECUDA;
    if (launch(k_noalloc_reduce, (p * p + 255) / 256, 256, 0, st, (const float2 *)part, used, p * p,
               reinterpret_cast<double2 *>(Kout)) != cudaSuccess)
        return IMG_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return IMG_ECUDA;
    return IMG_OK;
}
