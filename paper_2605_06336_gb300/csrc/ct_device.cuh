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

// ---------------------------------------------------------------------------
// ray march arguments (ct_ray.cu, ct_band.cu)
// ---------------------------------------------------------------------------
enum RayMode { kFwd = 0, kJvp = 1, kVjp = 2, kGn = 3 };

template <typename T> struct RayArgs {
    const ViewGeo *vg;
    int V, N, B, nchunks, Pp;
    const pair_t<T> *PX, *PT;
    long long pimg_stride;  // pairs per batch element (F * N * Pp)
    int kbase, ngroups;
    T *Y;                   // FWD: [batch][V*B]; JVP: dY
    long long sino_stride;
    const double *dtheta, *ddelta;
    long long dir_stride;   // JVP: doubles between the directions of consecutive images (0: one for all)
    const T *R;             // VJP: r; GN: data b
    T *res;                 // GN: residual (nullable)
    long long r_stride;     // VJP / GN: elements between the R of consecutive images (0: one for all)
    double *partial;        // VJP / GN: [image][view][chunk][4]
    long long part_stride;  // doubles between the partials of consecutive images (V * nchunks * 4)
    const int *view_mask;   // GN: views with mask 0 are skipped (nullable)
    const int *skip;        // whole launch is a no-op when *skip != 0 (nullable)
    const int *order;       // view order (nullable: identity)
    int VW;                 // view slots per CTA
    int segs;               // band-staged forward: row segments per ray, one CTA each (1: whole rays)
    T *fpart;               // segments 1..segs-1 of the band-staged forward (segment 0 goes to Y)
    long long fpart_stride; // elements per segment in fpart
    const float *QX, *QT;   // interleaved images (FP32 forward)
    long long qimg_stride;  // floats per image in the interleaved layout (F * N * Pp)
    int kend;               // FWD: images k >= kend of a group are not written (a batch below the
                            // interleaved layout's ends inside a group)
};

// Warp-uniform row range [rlo, rhi] covering every row where one of the
// warp's rays has -1 < q < N; rows added by the union or by the two-row
// margin read exact zeros.
__device__ __forceinline__ void warp_rows(const ViewGeo &g, int b, bool active, int N, int &rlo, int &rhi)
{
    if (g.flags & kAllRows) {
        rlo = 0;
        rhi = N - 1;
        return;
    }
    const float r1 = fmaf((float)b, g.gam, g.alo);
    const float r2 = fmaf((float)b, g.gam, g.ahi);
    const float lo = fminf(fmaxf(fminf(r1, r2) - 2.0f, 0.0f), (float)N);
    const float hi = fmaxf(fminf(fmaxf(r1, r2) + 2.0f, (float)(N - 1)), -1.0f);
    int l = (int)floorf(lo), u = (int)ceilf(hi);
    if (!active) {
        l = N;
        u = -1;
    }
    rlo = __reduce_min_sync(0xffffffffu, l);
    rhi = __reduce_max_sync(0xffffffffu, u);
}

// Per-ray output of a march: the forward stores w * sum for each image, the
// JVP stores the directional derivative, the VJP and Gauss-Newton modes write
// per-(view, chunk) partial sums reduced over the warp in a fixed order.
template <typename T, int MODE, bool OFFS, int KB>
__device__ __forceinline__ void ray_epilogue(const RayArgs<T> &a, const ViewGeo &g, int v, int b, bool active, int k0,
                                             int chunk, int lane, const T (&acc)[(MODE == kFwd) ? KB : 3 * KB])
{
    const T wv = GeoT<T>::w(g);
    if constexpr (MODE == kFwd) {
        if (active) {
#pragma unroll
            for (int k = 0; k < KB; ++k)
                if (k0 + k < a.kend) a.Y[(size_t)(k0 + k) * a.sino_stride + (size_t)v * a.B + b] = wv * acc[k];
        }
    } else {
        // image k of the group: acc[3k] interpolated sum, acc[3k+1] slope x dq/dtheta, acc[3k+2] slopes
        const size_t vb = (size_t)v * a.B + b;
#pragma unroll
        for (int k = 0; k < KB; ++k) {
            const size_t img = (size_t)(k0 + k);
            const T jt = fma(GeoT<T>::dw(g), acc[3 * k], wv * acc[3 * k + 1]);
            const T jd = wv * GeoT<T>::qb(g) * acc[3 * k + 2];
            if constexpr (MODE == kJvp) {
                if (active) {
                    T out = (T)a.dtheta[img * a.dir_stride + v] * jt;
                    if (OFFS) out = fma((T)a.ddelta[img * a.dir_stride + v], jd, out);
                    a.Y[img * a.sino_stride + vb] = out;
                }
            } else if constexpr (MODE == kVjp) {
                double pt = 0.0, pd = 0.0;
                if (active) {
                    const T r = a.R[img * a.r_stride + vb];
                    pt = (double)(r * jt);
                    if (OFFS) pd = (double)(r * jd);
                }
                pt = warp_sum(pt);
                if (OFFS) pd = warp_sum(pd);
                if (lane == 0) {
                    double *p = a.partial + img * a.part_stride + ((size_t)v * a.nchunks + chunk) * 4;
                    p[0] = pt;
                    p[1] = pd;
                }
            } else {  // kGn
                // pr: the rounding scale |r| (|H x| + |b|) of the misfit (Armijo noise floor)
                double pg = 0.0, pj = 0.0, pf = 0.0, pr = 0.0;
                if (active) {
                    const T hx = wv * acc[3 * k];
                    const T bb = a.R[img * a.r_stride + vb];
                    const T rr = hx - bb;
                    if (a.res) a.res[img * a.sino_stride + vb] = rr;
                    pg = (double)rr * (double)jt;
                    pj = (double)jt * (double)jt;
                    pf = (double)rr * (double)rr;
                    pr = fabs((double)rr) * (fabs((double)hx) + fabs((double)bb));
                }
                pg = warp_sum(pg);
                pj = warp_sum(pj);
                pf = warp_sum(pf);
                pr = warp_sum(pr);
                if (lane == 0) {
                    double *p = a.partial + img * a.part_stride + ((size_t)v * a.nchunks + chunk) * 4;
                    p[0] = pg;
                    p[1] = pj;
                    p[2] = pf;
                    p[3] = pr;
                }
            }
        }
    }
}

// Band-staged FP32 ray march (ct_band.cu): the rows a CTA's rays cross are
// staged in shared memory block by block.  a.VW in {4, 8} view slots, rb in
// {4, 8} rows per staged block, kb in {1, 2, 4, 8} images (forward only).
// Results are bit-identical to k_ray with one row segment per ray.
bool band_shape_ok(int mode, int kb, int vw, int rb);
cudaError_t run_ray_band(const Handle &h, const RayArgs<float> &a, int mode, bool offs, int kb, int rb);
// Fan-beam ray march (ct_fan.cu) for the same arguments: mode kFwd (kb
// images), kJvp, kVjp (angle and, with offs, offset derivatives) or kGn
// (angle derivatives); split warps share a ray.
template <typename T>
cudaError_t run_fan_ray(const Handle &h, const RayArgs<T> &a, int mode, int kb, int split, bool offs);
// Y[k][v][b] = w_v * (Y + P_1 + ... + P_{segs-1}), summed in segment order.
cudaError_t launch_fwd_combine(const Handle &h, float *Y, const float *P, int segs, long long stride, int batch,
                               const int *skip);

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

// Grid of a work-item kernel: one CTA per item, so that the hardware hands
// items to SMs as CTAs finish (items differ in cost: chunks at the detector
// edge carry short rays).  Very large item counts are folded into a grid of
// 64 resident waves; the kernels loop over item += gridDim.x.
template <typename K>
inline int persistent_grid(K kernel, int threads, size_t smem, long long work_blocks, int num_sms)
{
    const int per_sm = resident_per_sm((const void *)kernel, threads, smem);
    const long long cap = 64LL * per_sm * num_sms;
    return (int)std::max<long long>(1, std::min(work_blocks, cap));
}

}  // namespace ctgb
