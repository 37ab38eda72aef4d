// Device helpers shared by the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "ct_internal.cuh"

namespace ctgb {

template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };
template <typename T> using pair_t = typename Pair<T>::type;

__device__ __forceinline__ int cell_of(long long Q) { return (int)(Q >> kFracBits); }

// Fraction q - floor(q) of a fixed-point value: the top 23 (or 48) of the 48
// fractional bits placed in the mantissa of 1.m, minus one.
__device__ __forceinline__ float frac_of(long long Q, float)
{
    const unsigned m = (unsigned)((unsigned long long)Q >> (kFracBits - 23)) & 0x7FFFFFu;
    return __uint_as_float(m | 0x3F800000u) - 1.0f;
}
__device__ __forceinline__ double frac_of(long long Q, double)
{
    const unsigned long long m = ((unsigned long long)Q & ((1ull << kFracBits) - 1ull)) << (52 - kFracBits);
    return __longlong_as_double((long long)(m | 0x3FF0000000000000ull)) - 1.0;
}

// Fixed-point q of ray b at march index r (see ct_internal.cuh).
__device__ __forceinline__ long long line_at(const ViewGeo &g, int b, int r, int N)
{
    return g.Qc + (long long)(b + g.n0) * g.Qb + (long long)(2 * r - (N - 1)) * g.Qh;
}

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// floor(t) and t - floor(t) in [0, 1] for |t| < 2^22 without a conversion
// instruction: t - 1/2 is rounded to an integer by the 1.5 * 2^23 shift.
// When t is an integer the rounding may land on t - 1, giving f = 1, which
// the hat weights treat the same as f = 0 on the next cell.
__device__ __forceinline__ void floor_split(float t, int &m, float &f)
{
    const float magic = 12582912.0f;
    const float tr = __fadd_rn(__fsub_rn(t, 0.5f), magic);
    m = __float_as_int(tr) - 0x4B400000;
    f = __fsub_rn(t, __fsub_rn(tr, magic));
}
__device__ __forceinline__ void floor_split(double t, int &m, double &f)
{
    const double fl = floor(t);
    m = (int)fl;
    f = t - fl;
}

// Per-view derivative constants in the working precision.  The FP64 form
// recomputes them from (c, s) in double.
template <typename T> struct GeoT;
template <> struct GeoT<float> {
    __device__ static float w(const ViewGeo &g) { return g.w; }
    __device__ static float dw(const ViewGeo &g) { return g.dw; }
    __device__ static float gs(const ViewGeo &g) { return g.gs; }
    __device__ static float gh(const ViewGeo &g, int) { return g.gh; }
    __device__ static float gr(const ViewGeo &g) { return g.gr; }
    __device__ static float qb(const ViewGeo &g) { return g.qbf; }
    __device__ static float sb(const ViewGeo &g, int b) { return g.sb0 + (float)b; }
};
template <> struct GeoT<double> {
    __device__ static double w(const ViewGeo &g) { return g.mode ? 1.0 / fabs(g.s) : 1.0 / fabs(g.c); }
    __device__ static double dw(const ViewGeo &g)
    {
        return g.mode ? -copysign(1.0, g.s) * g.c / (g.s * g.s) : copysign(1.0, g.c) * g.s / (g.c * g.c);
    }
    __device__ static double gs(const ViewGeo &g) { return g.mode ? g.c / (g.s * g.s) : g.s / (g.c * g.c); }
    __device__ static double gh(const ViewGeo &g, int N)
    {
        const double h = 0.5 * (N - 1);
        return g.mode ? h / (g.s * g.s) : -h / (g.c * g.c);
    }
    __device__ static double gr(const ViewGeo &g) { return g.mode ? -1.0 / (g.s * g.s) : 1.0 / (g.c * g.c); }
    __device__ static double qb(const ViewGeo &g) { return g.mode ? -1.0 / g.s : 1.0 / g.c; }
    __device__ static double sb(const ViewGeo &g, int b) { return g.sb0d + (double)b; }
};

// Resident CTAs per SM of a kernel at a launch shape, queried once per
// (kernel, threads, shared memory) and cached: the occupancy query is a host
// API call that would otherwise cost several microseconds per launch.
inline int resident_per_sm(const void *kernel, int threads, size_t smem)
{
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, size_t>, int> cache;
    const auto key = std::make_tuple(kernel, threads, smem);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = per_sm;
    return per_sm;
}

// Persistent grid: as many CTAs as are resident at once, capped by the work.
template <typename K>
inline int persistent_grid(K kernel, int threads, size_t smem, long long work_blocks, int num_sms)
{
    const int per_sm = resident_per_sm((const void *)kernel, threads, smem);
    const long long cap = (long long)per_sm * num_sms;
    return (int)std::max<long long>(1, std::min(work_blocks, cap));
}

}  // namespace ctgb
