// CUDA kernels of the angle-dependent Joseph operator (sm_103a).
//
//   k_view_setup   per-view constants from (theta, delta), FP64 -> fixed point
//   k_transpose    X -> X^T so that column-sampled views also read rows
//   k_forward      Y = H X          ray-driven, one lane per ray, KB images per lane
//   k_jvp          dY = J dtheta    same march, accumulates the analytic derivative
//   k_vjp          J^T r            same march, per-view reduction in fixed order
//   k_gn           Gauss-Newton terms (residual, gradient, |J_v|^2, f_v)
//   k_adjoint      X = H^T Y        pixel-driven gather (no atomics)
//   k_finalize     per-view sums of the per-(view, bin-chunk) partials
//
// Forward model (Joseph rule, Sec. 6.2 "Radon transform at perturbed
// angles"): see the header ctgb.h for the geometry.  The ray kernels share
// one structure: a warp owns 32 consecutive bins of one view, computes the
// union of the rows its rays need (rays outside the image contribute exact
// zeros through predicated loads), and marches the rows in lock step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "ct_internal.cuh"

namespace ctgb {
namespace {

// ---------------------------------------------------------------------------
// fixed-point helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_of(long long Q) { return (int)(Q >> kFracBits); }

// Fraction q - floor(q) from the fixed-point value: the top 23 (52) of the
// 48 fractional bits placed in the mantissa of 1.m, minus one.
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

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Nearest integer n and remainder d = t - n, |d| <= 1/2 (|t| < 2^22).
__device__ __forceinline__ void round_split(float t, int &n, float &d)
{
    const float magic = 12582912.0f;  // 1.5 * 2^23
    const float tr = __fadd_rn(t, magic);
    n = __float_as_int(tr) - 0x4B400000;
    d = __fsub_rn(t, __fsub_rn(tr, magic));
}
__device__ __forceinline__ void round_split(double t, int &n, double &d)
{
    const double r = rint(t);
    n = (int)r;
    d = t - r;
}

// Row range [rlo, rhi] (inclusive, warp-uniform union) that covers every row
// where one of the warp's rays has -1 < q < N.  Rows added by the union or by
// the one-row safety margin contribute exact zeros.
__device__ __forceinline__ void warp_row_range(const ViewGeo &g, int b, bool active, int N, int &rlo,
                                               int &rhi)
{
    if (g.flags & kAllRows) {
        rlo = 0;
        rhi = N - 1;
        return;
    }
    const double r1 = fma((double)b, g.gam, g.alo);
    const double r2 = fma((double)b, g.gam, g.ahi);
    double lo = fmin(r1, r2) - 1.0, hi = fmax(r1, r2) + 1.0;
    lo = fmin(fmax(lo, 0.0), (double)N);
    hi = fmax(fmin(hi, (double)(N - 1)), -1.0);
    int l = (int)floor(lo), u = (int)ceil(hi);
    if (!active) {
        l = N;
        u = -1;
    }
    rlo = __reduce_min_sync(0xffffffffu, l);
    rhi = __reduce_max_sync(0xffffffffu, u);
}

// Fixed-point q of ray b at march index r (see ct_internal.cuh).
__device__ __forceinline__ long long line_start(const ViewGeo &g, int b, int r, int N)
{
    return g.Qc + (long long)(b + g.n0) * g.Qb + (long long)(2 * r - (N - 1)) * g.Qh;
}

template <typename T> struct GeoT;
template <> struct GeoT<float> {
    __device__ static float w(const ViewGeo &g) { return g.w; }
    __device__ static float dw(const ViewGeo &g) { return g.dw; }
    __device__ static float gs(const ViewGeo &g) { return g.gs; }
    __device__ static float gh(const ViewGeo &g) { return g.gh; }
    __device__ static float gr(const ViewGeo &g) { return g.gr; }
    __device__ static float qb(const ViewGeo &g) { return g.qbf; }
    __device__ static float sb0(const ViewGeo &g) { return g.sb0; }
};
// The FP64 form recomputes the few derivative constants in double from c, s.
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
};

template <typename T> __device__ __forceinline__ T geo_gh(const ViewGeo &g, int N);
template <> __device__ __forceinline__ float geo_gh<float>(const ViewGeo &g, int) { return g.gh; }
template <> __device__ __forceinline__ double geo_gh<double>(const ViewGeo &g, int N) { return GeoT<double>::gh(g, N); }
// ---------------------------------------------------------------------------
// per-view setup
// ---------------------------------------------------------------------------
__global__ void k_view_setup(const double *__restrict__ theta, const double *__restrict__ delta,
                             const int *__restrict__ fov, int V, int N, int B, ViewGeo *__restrict__ out,
                             int *__restrict__ flag)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    double th = theta[v];
    double dl = delta ? delta[v] : 0.0;
    if (!isfinite(th) || !isfinite(dl)) {
        *flag = 1;  // every writer stores the same value
        th = 0.0;
        dl = 0.0;
    }
    double s, c;
    sincos(th, &s, &c);
    const double h = 0.5 * (N - 1);
    const double sb0 = -0.5 * (B - 1) + dl;
    ViewGeo g;
    double q0, qb, qr;
    if (fabs(c) >= fabs(s)) {  // one sample per image row
        g.mode = 0;
        q0 = (sb0 - h * s) / c + h;
        qb = 1.0 / c;
        qr = s / c;
        const double ic2 = 1.0 / (c * c);
        g.w = (float)(1.0 / fabs(c));
        g.dw = (float)(copysign(1.0, c) * s * ic2);
        g.gs = (float)(s * ic2);
        g.gh = (float)(-h * ic2);
        g.gr = (float)ic2;
    } else {  // one sample per image column (rows of X^T)
        g.mode = 1;
        q0 = h - (sb0 + h * c) / s;
        qb = -1.0 / s;
        qr = c / s;
        const double is2 = 1.0 / (s * s);
        g.w = (float)(1.0 / fabs(s));
        g.dw = (float)(-copysign(1.0, s) * c * is2);
        g.gs = (float)(c * is2);
        g.gh = (float)(h * is2);
        g.gr = (float)(-is2);
    }
    // Fixed-point line anchored at the image centre with an integer bin offset.
    const double n0 = floor(sb0);
    g.n0 = (int)n0;
    g.Qc = __double2ll_rn(h * kFixScale) + __double2ll_rn((sb0 - n0) * qb * kFixScale);
    g.Qb = __double2ll_rn(qb * kFixScale);
    g.Qh = __double2ll_rn(qr * 0.5 * kFixScale);
    g.qbf = (float)qb;
    g.sb0 = (float)sb0;
    g.sb0d = sb0;
    if (fabs(qr) < 1e-9) {
        g.flags = kAllRows;
        g.alo = g.ahi = g.gam = 0.0;
    } else {
        g.flags = 0;
        const double iqr = 1.0 / qr;
        g.alo = (-1.0 - q0) * iqr;
        g.ahi = ((double)N - q0) * iqr;
        g.gam = -qb * iqr;
    }
    g.beta0 = h * (s - c) - dl + 0.5 * (B - 1);
    g.c = c;
    g.s = s;
    g.frame = fov ? fov[v] : 0;
    out[v] = g;
}

// ---------------------------------------------------------------------------
// transpose (X^T for column-sampled views)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_transpose(const T *__restrict__ X, T *__restrict__ XT, int N, int nimg)
{
    __shared__ T tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int img = blockIdx.z; img < nimg; img += gridDim.z) {
        const T *src = X + (size_t)img * N * N;
        T *dst = XT + (size_t)img * N * N;
        __syncthreads();
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            const int i = by + yy, j = bx + threadIdx.x;
            if (i < N && j < N) tile[yy][threadIdx.x] = src[(size_t)i * N + j];
        }
        __syncthreads();
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            const int j = bx + yy, i = by + threadIdx.x;
            if (i < N && j < N) dst[(size_t)j * N + i] = tile[threadIdx.x][yy];
        }
    }
}

// ---------------------------------------------------------------------------
// forward projection
// ---------------------------------------------------------------------------
template <typename T, int KB>
__global__ void __launch_bounds__(128) k_forward(const ViewGeo *__restrict__ vg, int V, int N, int B, int nchunks,
                                                 const T *__restrict__ X, const T *__restrict__ XT,
                                                 long long img_stride, int kbase, int ngroups, T *__restrict__ Y,
                                                 long long sino_stride)
{
    const int lane = threadIdx.x & 31;
    const int total = ngroups * V * nchunks;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nwarps) {
        const int chunk = w % nchunks;
        const int t = w / nchunks;
        const int v = t % V;
        const int grp = t / V;
        const ViewGeo &g = vg[v];
        const int b = chunk * kChunk + lane;
        const bool active = b < B;
        int rlo, rhi;
        warp_row_range(g, b, active, N, rlo, rhi);
        const int k0 = kbase + grp * KB;
        const T *img = (g.mode ? XT : X) + (size_t)g.frame * N * N + (size_t)k0 * img_stride + (size_t)rlo * N;
        long long Q = line_start(g, b, rlo, N);
        const long long dQ = 2 * g.Qh;
        T acc[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) acc[k] = T(0);
#pragma unroll 4
        for (int r = rlo; r <= rhi; ++r, img += N, Q += dQ) {
            const int cell = cell_of(Q);
            const T f = frac_of(Q, T());
            const T omf = T(1) - f;
            const bool p0 = (unsigned)cell < (unsigned)N;
            const bool p1 = (unsigned)(cell + 1) < (unsigned)N;
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                const T *p = img + (size_t)k * img_stride + cell;
                const T v0 = p0 ? ldg(p) : T(0);
                const T v1 = p1 ? ldg(p + 1) : T(0);
                acc[k] = fma(omf, v0, fma(f, v1, acc[k]));
            }
        }
        if (active) {
            const T wv = GeoT<T>::w(g);
#pragma unroll
            for (int k = 0; k < KB; ++k) Y[(size_t)(k0 + k) * sino_stride + (size_t)v * B + b] = wv * acc[k];
        }
    }
}

// One ray of the derivative march: value sum S0, sum of slope * dq/dtheta,
// and sum of slopes (for the offset derivative).
template <typename T, bool OFFS>
__device__ __forceinline__ void march_derivative(const ViewGeo &g, const T *img, int N, int b, int B, int rlo,
                                                 int rhi, T &s0, T &sg, T &s1)
{
    long long Q = line_start(g, b, rlo, N);
    const long long dQ = 2 * g.Qh;
    T sb;
    if constexpr (sizeof(T) == 4) sb = g.sb0 + (float)b;
    else sb = g.sb0d + (double)b;
    const T g0 = fma(sb, GeoT<T>::gs(g), geo_gh<T>(g, N));
    const T gr = GeoT<T>::gr(g);
    T rf = (T)rlo;
    s0 = sg = s1 = T(0);
    img += (size_t)rlo * N;
#pragma unroll 4
    for (int r = rlo; r <= rhi; ++r, img += N, Q += dQ, rf += T(1)) {
        const int cell = cell_of(Q);
        const T f = frac_of(Q, T());
        const T v0 = ((unsigned)cell < (unsigned)N) ? ldg(img + cell) : T(0);
        const T v1 = ((unsigned)(cell + 1) < (unsigned)N) ? ldg(img + cell + 1) : T(0);
        const T d = v1 - v0;
        s0 += fma(f, d, v0);
        sg = fma(d, fma(rf, gr, g0), sg);
        if (OFFS) s1 += d;
    }
}

template <typename T, bool OFFS>
__global__ void __launch_bounds__(128) k_jvp(const ViewGeo *__restrict__ vg, int V, int N, int B, int nchunks,
                                             const T *__restrict__ X, const T *__restrict__ XT,
                                             const double *__restrict__ dtheta, const double *__restrict__ ddelta,
                                             T *__restrict__ dY)
{
    const int lane = threadIdx.x & 31;
    const int total = V * nchunks;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nwarps) {
        const int chunk = w % nchunks;
        const int v = w / nchunks;
        const ViewGeo &g = vg[v];
        const int b = chunk * kChunk + lane;
        const bool active = b < B;
        int rlo, rhi;
        warp_row_range(g, b, active, N, rlo, rhi);
        const T *img = (g.mode ? XT : X) + (size_t)g.frame * N * N;
        T s0, sg, s1;
        march_derivative<T, OFFS>(g, img, N, b, B, rlo, rhi, s0, sg, s1);
        if (active) {
            const T wv = GeoT<T>::w(g);
            T out = (T)dtheta[v] * fma(GeoT<T>::dw(g), s0, wv * sg);
            if (OFFS) out += (T)ddelta[v] * (wv * GeoT<T>::qb(g) * s1);
            dY[(size_t)v * B + b] = out;
        }
    }
}

template <typename T, bool OFFS>
__global__ void __launch_bounds__(128) k_vjp(const ViewGeo *__restrict__ vg, int V, int N, int B, int nchunks,
                                             const T *__restrict__ X, const T *__restrict__ XT,
                                             const T *__restrict__ R, double *__restrict__ partial)
{
    const int lane = threadIdx.x & 31;
    const int total = V * nchunks;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nwarps) {
        const int chunk = w % nchunks;
        const int v = w / nchunks;
        const ViewGeo &g = vg[v];
        const int b = chunk * kChunk + lane;
        const bool active = b < B;
        int rlo, rhi;
        warp_row_range(g, b, active, N, rlo, rhi);
        const T *img = (g.mode ? XT : X) + (size_t)g.frame * N * N;
        T s0, sg, s1;
        march_derivative<T, OFFS>(g, img, N, b, B, rlo, rhi, s0, sg, s1);
        double pt = 0.0, pd = 0.0;
        if (active) {
            const T wv = GeoT<T>::w(g);
            const T r = R[(size_t)v * B + b];
            pt = (double)(r * fma(GeoT<T>::dw(g), s0, wv * sg));
            if (OFFS) pd = (double)(r * (wv * GeoT<T>::qb(g) * s1));
        }
        pt = warp_sum(pt);
        if (OFFS) pd = warp_sum(pd);
        if (lane == 0) {
            partial[((size_t)v * nchunks + chunk) * 4 + 0] = pt;
            partial[((size_t)v * nchunks + chunk) * 4 + 1] = pd;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(128) k_gn(const ViewGeo *__restrict__ vg, int V, int N, int B, int nchunks,
                                            const T *__restrict__ X, const T *__restrict__ XT,
                                            const T *__restrict__ bdata, T *__restrict__ res,
                                            double *__restrict__ partial)
{
    const int lane = threadIdx.x & 31;
    const int total = V * nchunks;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nwarps) {
        const int chunk = w % nchunks;
        const int v = w / nchunks;
        const ViewGeo &g = vg[v];
        const int b = chunk * kChunk + lane;
        const bool active = b < B;
        int rlo, rhi;
        warp_row_range(g, b, active, N, rlo, rhi);
        const T *img = (g.mode ? XT : X) + (size_t)g.frame * N * N;
        T s0, sg, s1;
        march_derivative<T, false>(g, img, N, b, B, rlo, rhi, s0, sg, s1);
        double pg = 0.0, pj = 0.0, pf = 0.0;
        if (active) {
            const T wv = GeoT<T>::w(g);
            const T jt = fma(GeoT<T>::dw(g), s0, wv * sg);
            const T rr = wv * s0 - bdata[(size_t)v * B + b];
            if (res) res[(size_t)v * B + b] = rr;
            pg = (double)rr * (double)jt;
            pj = (double)jt * (double)jt;
            pf = (double)rr * (double)rr;
        }
        pg = warp_sum(pg);
        pj = warp_sum(pj);
        pf = warp_sum(pf);
        if (lane == 0) {
            double *p = partial + ((size_t)v * nchunks + chunk) * 4;
            p[0] = pg;
            p[1] = pj;
            p[2] = pf;
        }
    }
}

// out_q[v] = scale_q * sum_c partial[v][c][q] for the requested slots.
__global__ void k_finalize(const double *__restrict__ partial, int V, int nchunks, double *out0, double *out1,
                           double *out2, double scale2)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    double a = 0.0, b = 0.0, c = 0.0;
    const double *p = partial + (size_t)v * nchunks * 4;
    for (int k = 0; k < nchunks; ++k) {
        a += p[4 * k + 0];
        b += p[4 * k + 1];
        c += p[4 * k + 2];
    }
    if (out0) out0[v] = a;
    if (out1) out1[v] = b;
    if (out2) out2[v] = scale2 * c;
}

// ---------------------------------------------------------------------------
// transpose operator H^T: one thread per pixel, loop over the frame's views
// ---------------------------------------------------------------------------
// For pixel (i, j) and view v the continuous bin coordinate of the pixel
// centre is beta = beta0 + j*c - i*s; the rays that sampled the pixel are the
// bins b with |b - beta| < 1/w, with weight w * (1 - |b - beta| * w) -- the
// same hat the forward interpolation assigns (at most two bins).  beta is
// split into an FP64 tile anchor (integer + fraction) and a small FP32
// in-tile offset.
template <typename T, int KB>
__global__ void __launch_bounds__(256) k_adjoint(const ViewGeo *__restrict__ vg, const int *__restrict__ fstart,
                                                 const int *__restrict__ fcount, int N, int B, int F, int tps,
                                                 int kbase, int ngroups, const T *__restrict__ Y,
                                                 long long sino_stride, T *__restrict__ X, long long img_stride)
{
    __shared__ T s_c[256], s_s[256], s_w[256], s_omw[256], s_bf[256];
    __shared__ int s_bi[256], s_off[256];
    const int tx = threadIdx.x & (kTile - 1), ty = threadIdx.x / kTile;
    const int tiles = tps * tps;
    const int total = ngroups * F * tiles;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int tile = item % tiles;
        const int t2 = item / tiles;
        const int f = t2 % F;
        const int grp = t2 / F;
        const int i0 = (tile / tps) * kTile, j0 = (tile % tps) * kTile;
        const int k0 = kbase + grp * KB;
        T acc[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) acc[k] = T(0);
        const T *Yg = Y + (size_t)k0 * sino_stride;
        const int vs = fstart[f], vc = fcount[f];
        const T fx = (T)tx, fy = (T)ty;
        for (int base = 0; base < vc; base += 256) {
            const int nv = min(256, vc - base);
            __syncthreads();
            if ((int)threadIdx.x < nv) {
                const int v = vs + base + threadIdx.x;
                const ViewGeo &g = vg[v];
                const double bt = g.beta0 + (double)j0 * g.c - (double)i0 * g.s;
                const double fl = floor(bt);
                const double wv = g.mode ? 1.0 / fabs(g.s) : 1.0 / fabs(g.c);
                s_bi[threadIdx.x] = (int)fl;
                s_bf[threadIdx.x] = (T)(bt - fl);
                s_c[threadIdx.x] = (T)g.c;
                s_s[threadIdx.x] = (T)g.s;
                s_w[threadIdx.x] = (T)wv;
                s_omw[threadIdx.x] = (T)(1.0 - wv);
                s_off[threadIdx.x] = v * B;
            }
            __syncthreads();
            for (int q = 0; q < nv; ++q) {
                const T t = fma(fx, s_c[q], fma(-fy, s_s[q], s_bf[q]));
                int n;
                T d;
                round_split(t, n, d);
                const T ad = fabs(d);
                const T wv = s_w[q];
                const T wn = fmax(T(0), fma(-ad, wv, T(1)));
                const T w2 = fmax(T(0), fma(ad, wv, s_omw[q]));
                const int b1 = s_bi[q] + n;
                const int b2 = b1 + ((d >= T(0)) ? 1 : -1);
                const bool p1 = (unsigned)b1 < (unsigned)B;
                const bool p2 = (unsigned)b2 < (unsigned)B;
                const T *yr = Yg + s_off[q];
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    const T y1 = p1 ? ldg(yr + (size_t)k * sino_stride + b1) : T(0);
                    const T y2 = p2 ? ldg(yr + (size_t)k * sino_stride + b2) : T(0);
                    acc[k] = fma(wv, fma(wn, y1, w2 * y2), acc[k]);
                }
            }
        }
        const int i = i0 + ty, j = j0 + tx;
        if (i < N && j < N) {
#pragma unroll
            for (int k = 0; k < KB; ++k)
                X[(size_t)(k0 + k) * img_stride + (size_t)f * N * N + (size_t)i * N + j] = acc[k];
        }
    }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
template <typename K>
int persistent_grid(K kernel, int threads, long long work_blocks, int num_sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long cap = (long long)per_sm * num_sms;
    return (int)std::max<long long>(1, std::min(work_blocks, cap));
}

}  // namespace

cudaError_t launch_view_setup(const Handle &h, const double *theta, const double *delta)
{
    const int threads = 128;
    k_view_setup<<<(h.V + threads - 1) / threads, threads, 0, h.stream>>>(theta, delta, h.d_fov, h.V, h.N, h.B,
                                                                           h.d_views, h.d_flag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_transpose(const Handle &h, const T *X, T *XT, int nimg)
{
    dim3 block(32, 8);
    dim3 grid((h.N + 31) / 32, (h.N + 31) / 32, std::min(nimg, 65535));
    k_transpose<T><<<grid, block, 0, h.stream>>>(X, XT, h.N, nimg);
    return cudaGetLastError();
}

template <typename T, int KB>
static cudaError_t fwd_part(const Handle &h, const T *X, const T *XT, T *Y, int kbase, int ngroups)
{
    const long long img_stride = (long long)h.F * h.N * h.N;
    const long long sino_stride = (long long)h.V * h.B;
    const long long warps = (long long)ngroups * h.V * h.nchunks;
    const int grid = persistent_grid(k_forward<T, KB>, 128, (warps + 3) / 4, h.num_sms);
    k_forward<T, KB><<<grid, 128, 0, h.stream>>>(h.d_views, h.V, h.N, h.B, h.nchunks, X, XT, img_stride, kbase,
                                                 ngroups, Y, sino_stride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_forward(const Handle &h, const T *X, const T *XT, T *Y, int batch)
{
    int k = 0;
    cudaError_t e = cudaSuccess;
    if (batch - k >= 8) {
        e = fwd_part<T, 8>(h, X, XT, Y, k, (batch - k) / 8);
        k += ((batch - k) / 8) * 8;
    }
    if (e == cudaSuccess && batch - k >= 4) {
        e = fwd_part<T, 4>(h, X, XT, Y, k, 1);
        k += 4;
    }
    if (e == cudaSuccess && batch - k >= 2) {
        e = fwd_part<T, 2>(h, X, XT, Y, k, 1);
        k += 2;
    }
    if (e == cudaSuccess && batch - k >= 1) {
        e = fwd_part<T, 1>(h, X, XT, Y, k, 1);
        k += 1;
    }
    return e;
}

template <typename T, int KB>
static cudaError_t adj_part(const Handle &h, const T *Y, T *X, int kbase, int ngroups)
{
    const long long img_stride = (long long)h.F * h.N * h.N;
    const long long sino_stride = (long long)h.V * h.B;
    const int tps = (h.N + kTile - 1) / kTile;
    const long long items = (long long)ngroups * h.F * tps * tps;
    const int grid = persistent_grid(k_adjoint<T, KB>, 256, items, h.num_sms);
    k_adjoint<T, KB><<<grid, 256, 0, h.stream>>>(h.d_views, h.d_fstart, h.d_fcount, h.N, h.B, h.F, tps, kbase,
                                                 ngroups, Y, sino_stride, X, img_stride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint(const Handle &h, const T *Y, T *X, int batch)
{
    int k = 0;
    cudaError_t e = cudaSuccess;
    if (batch - k >= 8) {
        e = adj_part<T, 8>(h, Y, X, k, (batch - k) / 8);
        k += ((batch - k) / 8) * 8;
    }
    if (e == cudaSuccess && batch - k >= 4) {
        e = adj_part<T, 4>(h, Y, X, k, 1);
        k += 4;
    }
    if (e == cudaSuccess && batch - k >= 2) {
        e = adj_part<T, 2>(h, Y, X, k, 1);
        k += 2;
    }
    if (e == cudaSuccess && batch - k >= 1) {
        e = adj_part<T, 1>(h, Y, X, k, 1);
        k += 1;
    }
    return e;
}

template <typename T>
cudaError_t launch_jvp(const Handle &h, const T *X, const T *XT, const double *dtheta, const double *ddelta, T *dY)
{
    const long long warps = (long long)h.V * h.nchunks;
    if (ddelta) {
        const int grid = persistent_grid(k_jvp<T, true>, 128, (warps + 3) / 4, h.num_sms);
        k_jvp<T, true><<<grid, 128, 0, h.stream>>>(h.d_views, h.V, h.N, h.B, h.nchunks, X, XT, dtheta, ddelta, dY);
    } else {
        const int grid = persistent_grid(k_jvp<T, false>, 128, (warps + 3) / 4, h.num_sms);
        k_jvp<T, false><<<grid, 128, 0, h.stream>>>(h.d_views, h.V, h.N, h.B, h.nchunks, X, XT, dtheta, nullptr, dY);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vjp(const Handle &h, const T *X, const T *XT, const T *R, double *gtheta, double *gdelta)
{
    const long long warps = (long long)h.V * h.nchunks;
    if (gdelta) {
        const int grid = persistent_grid(k_vjp<T, true>, 128, (warps + 3) / 4, h.num_sms);
        k_vjp<T, true><<<grid, 128, 0, h.stream>>>(h.d_views, h.V, h.N, h.B, h.nchunks, X, XT, R, h.d_partial);
    } else {
        const int grid = persistent_grid(k_vjp<T, false>, 128, (warps + 3) / 4, h.num_sms);
        k_vjp<T, false><<<grid, 128, 0, h.stream>>>(h.d_views, h.V, h.N, h.B, h.nchunks, X, XT, R, h.d_partial);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_finalize<<<(h.V + 127) / 128, 128, 0, h.stream>>>(h.d_partial, h.V, h.nchunks, gtheta, gdelta, nullptr, 1.0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gn(const Handle &h, const T *X, const T *XT, const T *bdata, T *res, double *grad, double *jnorm2,
                      double *fval)
{
    const long long warps = (long long)h.V * h.nchunks;
    const int grid = persistent_grid(k_gn<T>, 128, (warps + 3) / 4, h.num_sms);
    k_gn<T><<<grid, 128, 0, h.stream>>>(h.d_views, h.V, h.N, h.B, h.nchunks, X, XT, bdata, res, h.d_partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_finalize<<<(h.V + 127) / 128, 128, 0, h.stream>>>(h.d_partial, h.V, h.nchunks, grad, jnorm2, fval, 0.5);
    return cudaGetLastError();
}

#define CTGB_INSTANTIATE(T)                                                                                    \
    template cudaError_t launch_transpose<T>(const Handle &, const T *, T *, int);                            \
    template cudaError_t launch_forward<T>(const Handle &, const T *, const T *, T *, int);                   \
    template cudaError_t launch_adjoint<T>(const Handle &, const T *, T *, int);                              \
    template cudaError_t launch_jvp<T>(const Handle &, const T *, const T *, const double *, const double *, \
                                       T *);                                                                  \
    template cudaError_t launch_vjp<T>(const Handle &, const T *, const T *, const T *, double *, double *);  \
    template cudaError_t launch_gn<T>(const Handle &, const T *, const T *, const T *, T *, double *,        \
                                      double *, double *);

CTGB_INSTANTIATE(float)
CTGB_INSTANTIATE(double)

}  // namespace ctgb
