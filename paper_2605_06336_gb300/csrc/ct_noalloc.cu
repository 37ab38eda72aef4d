// ct_jacT_noalloc: the transposed angle/offset Jacobian (the same kernels as
// ct_jacT) for callers that cannot allocate device memory.
//
// Who needs it: a host application that owns all device memory through its
// own pool and does not let libraries call cudaMalloc, or a long-running
// service whose device-memory budget is fixed once it has started.  Such a
// caller cannot create a ct handle (ct_init allocates its workspaces), so
// this entry point takes the geometry directly and uses a file-scope
// device array as its workspace instead of allocating one.
//
// The array (below) is part of the library image: every GPU that loads the
// library holds it until the process exits, whether or not this entry point
// is ever called.  Its size is fixed by the limits in include/ctgb.h
// (CTGB_NOALLOC_MAX_N / _VIEWS / _BINS), about 1.7 MB.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ctgb.h"
#include "ct_internal.cuh"

namespace {

constexpr int kMaxN = CTGB_NOALLOC_MAX_N;
constexpr int kMaxV = CTGB_NOALLOC_MAX_VIEWS;
constexpr int kMaxB = CTGB_NOALLOC_MAX_BINS;
constexpr int kMaxChunks = (kMaxB + ctgb::kChunk - 1) / ctgb::kChunk;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace regions inside the array, each 256-byte aligned.
constexpr size_t kOffViews = 0;
constexpr size_t kOffFlag = align256(kOffViews + sizeof(ctgb::ViewGeo) * kMaxV);
constexpr size_t kOffPartial = align256(kOffFlag + sizeof(int));
constexpr size_t kOffPX = align256(kOffPartial + sizeof(double) * 4 * (size_t)kMaxV * kMaxChunks);
constexpr size_t kPairBytes = sizeof(float2) * (size_t)kMaxN * (kMaxN + 4);
constexpr size_t kOffPT = align256(kOffPX + kPairBytes);
constexpr size_t kScratchBytes = align256(kOffPT + kPairBytes);

// The workspace.  In host code this name is only a stand-in for the device
// object: its device address comes from cudaGetSymbolAddress (below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_base[kMaxDevices] = {};

// Device address of the workspace on the current device, looked up once per
// device (on the first call made with that device current).
cudaError_t scratch_base(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_base[dev] = p;
    }
    *out = g_base[dev];
    return cudaSuccess;
}

// Views whose angle or offset is not finite: their outputs become NaN, so that
// the caller sees the bad input in the result (this entry point has no status
// call; the kernels compute such a view at angle 0 and offset 0).
__global__ void k_mark_nonfinite(const double *__restrict__ theta, const double *__restrict__ delta, int V,
                                 double *__restrict__ gtheta, double *__restrict__ gdelta)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        if (isfinite(theta[v]) && (!delta || isfinite(delta[v]))) continue;
        gtheta[v] = __longlong_as_double(0x7ff8000000000000LL);
        if (gdelta) gdelta[v] = __longlong_as_double(0x7ff8000000000000LL);
    }
}

}  // namespace

extern "C" int ct_jacT_noalloc(int32_t N, int32_t B, int32_t n_views, const double *theta, const double *delta,
                               const float *x, const float *r, double *gtheta, double *gdelta, void *cuda_stream)
{
    if (!theta || !x || !r || !gtheta) return CT_ERR_ARG;
    if (N < 2 || N > kMaxN || B < 1 || B > kMaxB || n_views < 1 || n_views > kMaxV) return CT_ERR_ARG;
    void *base = nullptr;
    if (scratch_base(&base) != cudaSuccess) return CT_ERR_CUDA;
    unsigned char *s = static_cast<unsigned char *>(base);

    ctgb::Handle h;  // a view of the static workspace; owns nothing
    h.N = N;
    h.B = B;
    h.V = n_views;
    h.F = 1;
    h.max_batch = 1;
    h.precision = 0;
    h.Pp = N + 4;
    h.Pb = (B + 5) & ~1;  // even pair pitch, as ct_init sets it
    h.stream = (cudaStream_t)cuda_stream;
    h.d_views = reinterpret_cast<ctgb::ViewGeo *>(s + kOffViews);
    h.d_fov = nullptr;  // one frame
    h.d_flag = reinterpret_cast<int *>(s + kOffFlag);
    h.d_partial = reinterpret_cast<double *>(s + kOffPartial);
    h.d_px = s + kOffPX;
    h.d_pt = s + kOffPT;
    h.nchunks = (B + ctgb::kChunk - 1) / ctgb::kChunk;
    if (cudaGetDevice(&h.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h.num_sms, cudaDevAttrMultiProcessorCount, h.device) != cudaSuccess)
        return CT_ERR_CUDA;
    h.tune.der_split = 2;

    // The workspace keeps the previous call's contents: the per-view table
    // caches its constants by angle, so it must start invalid (zero) here.
    if (cudaMemsetAsync(h.d_views, 0, sizeof(ctgb::ViewGeo) * n_views, h.stream) != cudaSuccess ||
        cudaMemsetAsync(h.d_flag, 0, sizeof(int), h.stream) != cudaSuccess)
        return CT_ERR_CUDA;
    if (ctgb::launch_view_setup(h, theta, delta) != cudaSuccess) return CT_ERR_CUDA;
    if (ctgb::launch_pairs_img<float>(h, x, 1) != cudaSuccess) return CT_ERR_CUDA;
    if (ctgb::launch_vjp<float>(h, r, gtheta, gdelta, h.tune.der_split, 1, 0) != cudaSuccess) return CT_ERR_CUDA;
    k_mark_nonfinite<<<(n_views + 255) / 256, 256, 0, h.stream>>>(theta, delta, n_views, gtheta, gdelta);
    if (cudaGetLastError() != cudaSuccess) return CT_ERR_CUDA;
    return CT_OK;
}
