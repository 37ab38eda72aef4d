// Microbenchmarks of the on-chip levels that serve the operators' gathers:
// L2 -> SM read bandwidth and shared-memory read bandwidth.  They give the
// measured denominators of the gather roofline (the operators read pairs of
// pixels or bins from L2 through L1, or from shared memory when staged).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/ctgb.h"

namespace {

// Every thread streams float4 loads that bypass L1 (ld.global.cg) over a
// buffer that fits in L2, `reps` times; the sum is stored so the loads stay.
__global__ void __launch_bounds__(256) k_l2_read(const float4 *__restrict__ buf, long long n4, int reps,
                                                 float *__restrict__ sink)
{
    float acc = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc += (v.x + v.y) + (v.z + v.w);
        }
    }
    if (acc == 1234.5f) sink[0] = acc;  // practically never true; keeps the loads live
}

// Every thread reads consecutive 16-byte words of a 32 KB shared buffer
// (conflict-free: a warp reads 512 contiguous bytes per load).
__global__ void __launch_bounds__(256) k_smem_read(int reps, float *__restrict__ sink)
{
    constexpr int kWords = 2048;  // float4 words: 32 KB
    __shared__ float4 s[kWords];
    for (int i = threadIdx.x; i < kWords; i += blockDim.x) s[i] = make_float4(i, i + 1, i + 2, i + 3);
    __syncthreads();
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    int idx = threadIdx.x;
    for (int r = 0; r < reps; ++r) {
#pragma unroll 8
        for (int k = 0; k < kWords / 256; ++k) {
            const float4 v = s[(idx + k * 256) & (kWords - 1)];
            a.x += v.x;
            a.y += v.y;
            a.z += v.z;
            a.w += v.w;
        }
        idx += 32;
    }
    if (a.x + a.y + a.z + a.w == 1234.5f) sink[0] = a.x;
}

float time_ms(cudaStream_t s, void (*launch)(cudaStream_t), int reps)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch(s);  // warm-up
    std::vector<float> t(reps);
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, s);
        launch(s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t[r], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::sort(t.begin(), t.end());
    return t[0];
}

// launch parameters shared with the launch functions below
const float4 *g_buf = nullptr;
float *g_sink = nullptr;
long long g_n4 = 0;
int g_grid = 0, g_reps_l2 = 0, g_reps_smem = 0;

void launch_l2(cudaStream_t s) { k_l2_read<<<g_grid, 256, 0, s>>>(g_buf, g_n4, g_reps_l2, g_sink); }
void launch_smem(cudaStream_t s) { k_smem_read<<<g_grid, 256, 0, s>>>(g_reps_smem, g_sink); }

}  // namespace

extern "C" int ct_measure_peaks(double *l2_read_gbs, double *smem_read_gbs)
{
    if (!l2_read_gbs || !smem_read_gbs) return CT_ERR_ARG;
    int dev = 0, sms = 0, per_sm_l2 = 0, per_sm_smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CT_ERR_CUDA;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_l2, k_l2_read, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_smem, k_smem_read, 256, 0);
    const size_t bytes = 48u << 20;  // 48 MB: well inside the 126 MB L2
    void *buf = nullptr, *sink = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess || cudaMalloc(&sink, sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(buf);
        return CT_ERR_OOM;
    }
    cudaStream_t s = nullptr;
    int rc = CT_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMemsetAsync(buf, 0, bytes, s) != cudaSuccess) {
        rc = CT_ERR_CUDA;
    } else {
        g_buf = (const float4 *)buf;
        g_sink = (float *)sink;
        g_n4 = (long long)(bytes / sizeof(float4));
        g_grid = std::max(1, per_sm_l2) * sms;
        g_reps_l2 = 100;
        const float ms_l2 = time_ms(s, launch_l2, 5);
        g_grid = std::max(1, per_sm_smem) * sms;
        g_reps_smem = 4096;
        const float ms_smem = time_ms(s, launch_smem, 5);
        if (cudaGetLastError() != cudaSuccess || ms_l2 <= 0.f || ms_smem <= 0.f) {
            rc = CT_ERR_CUDA;
        } else {
            *l2_read_gbs = (double)bytes * g_reps_l2 / (ms_l2 * 1e-3) / 1e9;
            *smem_read_gbs = (double)g_grid * 256.0 * 16.0 * (2048 / 256) * g_reps_smem / (ms_smem * 1e-3) / 1e9;
        }
    }
    if (s) cudaStreamDestroy(s);
    cudaFree(buf);
    cudaFree(sink);
    return rc;
}
