// Ray-driven kernels of the angle-dependent Joseph operator (sm_103a).
//
//   k_view_prep   per-view constants from (theta, delta), FP64 -> fixed point,
//                 and the view order of the ray kernels
//   k_pairs_img   X -> pair layouts of X and X^T (zero padded)
//   k_pairs_sino  Y -> pair layout of the sinogram (zero padded)
//   k_ray         one warp per 32 consecutive rays of one view (optionally
//                 SPLIT warps per ray group, each marching a row segment):
//                   FWD  Y = H X for KB images at once
//                   JVP  dY = J_theta dtheta (+ J_delta ddelta)
//                   VJP  J_theta^T r (and J_delta^T r), per-view partials
//                   GN   residual, J^T r, |J_v|^2, f_v partials
//   k_finalize    per-view sums of the partials in a fixed order
//
// Forward model: Joseph rule on a parallel-beam geometry with per-view angle
// theta_v and detector offset delta_v (the CT operator of Sec. 6.2, with the
// per-parameter derivatives H_{p_i} u of Alg. "UPDATE-PARAM").
#include <cuda_runtime.h>

#include <type_traits>

#include <algorithm>
#include <cmath>

#include "ct_device.cuh"
#include "ct_internal.cuh"

namespace ctgb {
namespace {

// ---------------------------------------------------------------------------
// per-view setup
// ---------------------------------------------------------------------------
// Joseph axis: one sample per image row iff |cos theta| >= |sin theta|, i.e.
// iff theta mod pi lies in [0, pi/4] or [3pi/4, pi).  The test runs on theta
// itself with exact operations (fmod is exact, one rounded addition for a
// negative angle) against the doubles nearest pi, pi/4 and 3pi/4: it differs
// from the exact rule only within ~3e-16 rad of a diagonal, where comparing
// |cos| with |sin| would depend on the last bit of the sine and cosine.
__device__ __forceinline__ bool march_rows(double theta)
{
    const double pi = 3.14159265358979323846, q1 = 0.78539816339744830962, q3 = 2.35619449019234492885;
    double t = fmod(theta, pi);
    if (t < 0.0) t = __dadd_rn(t, pi);
    return t <= q1 || t >= q3;
}

// Rebuilds the constants of view v when its (theta, delta) changed since the
// last call; returns whether it did.
__device__ bool view_setup_one(int v, const double *__restrict__ theta, const double *__restrict__ delta,
                               const int *__restrict__ fov, int N, int B, ViewGeo *__restrict__ out,
                               int *__restrict__ flag)
{
    double th = theta[v];
    double dl = delta ? delta[v] : 0.0;
    ViewGeo *gp = out + v;
    if ((gp->flags & kValid) && __double_as_longlong(gp->th) == __double_as_longlong(th) &&
        __double_as_longlong(gp->dl) == __double_as_longlong(dl))
        return false;  // unchanged since the last call
    const double th_in = th, dl_in = dl;
    int bad = 0;
    if (!isfinite(th) || !isfinite(dl)) {
        *flag = 1;  // every writer stores the same value
        th = 0.0;
        dl = 0.0;
        bad = 1;
    }
    double s, c;
    sincos(th, &s, &c);
    const double h = 0.5 * (N - 1);
    const double sb0 = -0.5 * (B - 1) + dl;
    ViewGeo g;
    double q0, qb, qr;
    if (march_rows(th)) {  // one sample per image row
        const double ic = 1.0 / c;
        const double ic2 = ic * ic;
        g.mode = 0;
        qb = ic;
        qr = s * ic;
        q0 = (sb0 - h * s) * ic + h;
        g.w = (float)fabs(ic);
        g.dw = (float)(copysign(1.0, c) * s * ic2);
        g.gs = (float)(s * ic2);
        g.gh = (float)(-h * ic2);
        g.gr = (float)ic2;
    } else {  // one sample per image column (rows of X^T)
        const double is = 1.0 / s;
        const double is2 = is * is;
        g.mode = 1;
        qb = -is;
        qr = c * is;
        q0 = h - (sb0 + h * c) * is;
        g.w = (float)fabs(is);
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
    int flags = kValid;
    if (fabs(qr) < kAllRowsBelow) {
        flags |= kAllRows;
        g.alo = g.ahi = g.gam = 0.0f;
    } else {
        const double iqr = 1.0 / qr;
        g.alo = (float)((-1.0 - q0) * iqr);
        g.ahi = (float)(((double)N - q0) * iqr);
        g.gam = (float)(-qb * iqr);
    }
    g.flags = bad ? (flags & ~kValid) : flags;  // a bad view is rebuilt (and reported) every call
    g.beta0 = h * (s - c) - dl + 0.5 * (B - 1);
    g.c = c;
    g.s = s;
    g.th = th_in;
    g.dl = dl_in;
    g.frame = fov ? fov[v] : 0;
    g.gen = gp->gen + 1;
    *gp = g;
    return true;
}

// Per-view setup and view order in one single-CTA launch.  The view order
// of the ray kernels sorts the views by frame, then by marching axis, then
// by ray slope qr (ties by index), so that consecutive entries read the same
// image and sweep nearly the same band of it; it is rebuilt only when a view
// changed.  Without an order buffer (nullable) only the constants are built.
constexpr int kOrderMaxV = 4096;

// What the view-table step of an operator call needs; `on` = 0: no step.
struct ViewPrep {
    const double *theta, *delta;
    const int *fov;
    int V, N, B, on;
    ViewGeo *vg;
    int *flag;
    int *order;  // nullable: constants only
};

__device__ void build_order(const ViewPrep &p, unsigned long long *key);

// The view-table step, run by one whole CTA; key: shared memory for
// min(V, kOrderMaxV) 64-bit keys.
__device__ void view_prep_block(const ViewPrep &p, unsigned long long *key)
{
    __shared__ int s_changed;
    if (threadIdx.x == 0) s_changed = 0;
    __syncthreads();
    int mine = 0;
    for (int v = threadIdx.x; v < p.V; v += blockDim.x)
        mine |= view_setup_one(v, p.theta, p.delta, p.fov, p.N, p.B, p.vg, p.flag);
    if (mine) s_changed = 1;  // every writer stores the same value
    __syncthreads();
    if (!p.order || !s_changed) return;
    build_order(p, key);
}

// The view order of a CTA from the current view records (see view_prep_block).
__device__ void build_order(const ViewPrep &p, unsigned long long *key)
{
    if (p.V > kOrderMaxV) {
        for (int i = threadIdx.x; i < p.V; i += blockDim.x) p.order[i] = i;
        return;
    }
    // One unsigned 64-bit key per view orders by (frame, axis, slope): the
    // fixed-point slope |Qh| < 2^47 is offset into 48 bits, the axis and the
    // frame sit above it.  The rank of a view counts the keys below it (ties by
    // index); integer compares, as the FP64 pipe of this part is narrow.
    for (int i = threadIdx.x; i < p.V; i += blockDim.x)
        key[i] = ((unsigned long long)p.vg[i].frame << 49) | ((unsigned long long)p.vg[i].mode << 48) |
                 (unsigned long long)(p.vg[i].Qh + (1LL << 47));
    __syncthreads();
    for (int i = threadIdx.x; i < p.V; i += blockDim.x) {
        const unsigned long long ki = key[i];
        int rank = 0;
        for (int j = 0; j < p.V; ++j) {
            const unsigned long long kj = key[j];
            rank += (kj < ki || (kj == ki && j < i)) ? 1 : 0;
        }
        p.order[rank] = i;
    }
}

__global__ void __launch_bounds__(1024) k_view_prep(ViewPrep p, const int *__restrict__ skip)
{
    __shared__ unsigned long long key[kOrderMaxV];
    if (skip && *skip) return;
    view_prep_block(p, key);
}

// The same step spread over many CTAs: the per-view constants in parallel
// (*changed = 1 when a view was rebuilt), then k_view_order in one CTA.
__global__ void k_view_setup_many(ViewPrep p, int *changed, const int *__restrict__ skip)
{
    if (skip && *skip) return;
    int mine = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < p.V; v += gridDim.x * blockDim.x)
        mine |= view_setup_one(v, p.theta, p.delta, p.fov, p.N, p.B, p.vg, p.flag);
    if (mine) *changed = 1;  // every writer stores the same value
}

__global__ void __launch_bounds__(1024) k_view_order(ViewPrep p, int *changed, const int *__restrict__ skip)
{
    __shared__ unsigned long long key[kOrderMaxV];
    if (skip && *skip) return;
    const int ch = *changed;
    __syncthreads();  // every thread has read the flag before it is cleared below
    if (!ch || !p.order) return;
    build_order(p, key);
    __syncthreads();
    if (threadIdx.x == 0) *changed = 0;
}

// ---------------------------------------------------------------------------
// pair layouts
// ---------------------------------------------------------------------------
// Tile of 32 rows x 32 pairs.  PX[img][r][cp] = (X[r][c], X[r][c+1]) and
// PT[img][r][cp] = (X[c][r], X[c+1][r]) with c = cp - 2, zero outside.
// With p.on, one extra column of CTAs is launched and its first CTA runs the
// view-table step of the call (the two are independent).
template <typename T>
__global__ void __launch_bounds__(256) k_pairs_img(const T *__restrict__ X, pair_t<T> *__restrict__ PX,
                                                   pair_t<T> *__restrict__ PT, int N, int Pp, int nimg, ViewPrep p,
                                                   const int *__restrict__ skip)
{
    extern __shared__ unsigned long long prep_key[];
    if (skip && *skip) return;
    if (p.on && blockIdx.x == gridDim.x - 1) {
        if (blockIdx.y == 0 && blockIdx.z == 0) view_prep_block(p, prep_key);
        return;
    }
    __shared__ T a[32][34];   // a[i][j] = X[r0 + i][c0 + j]
    __shared__ T bt[33][33];  // bt[i][j] = X[c0 + i][r0 + j]
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int cp0 = blockIdx.x * 32, r0 = blockIdx.y * 32, c0 = cp0 - 2;
    for (int img = blockIdx.z; img < nimg; img += gridDim.z) {
        const T *src = X + (size_t)img * N * N;
        __syncthreads();
        for (int i = ty; i < 32; i += 8) {
            const int r = r0 + i;
            for (int j = tx; j < 33; j += 32) {
                const int c = c0 + j;
                a[i][j] = (r < N && c >= 0 && c < N) ? src[(size_t)r * N + c] : T(0);
            }
        }
        for (int i = ty; i < 33; i += 8) {
            const int rr = c0 + i, cc = r0 + tx;
            bt[i][tx] = (rr >= 0 && rr < N && cc < N) ? src[(size_t)rr * N + cc] : T(0);
        }
        __syncthreads();
        pair_t<T> *px = PX + (size_t)img * N * Pp;
        pair_t<T> *pt = PT + (size_t)img * N * Pp;
        for (int i = ty; i < 32; i += 8) {
            const int r = r0 + i, cp = cp0 + tx;
            if (r < N && cp < Pp) {
                pair_t<T> p;
                p.x = a[i][tx];
                p.y = a[i][tx + 1];
                px[(size_t)r * Pp + cp] = p;
                pair_t<T> q;
                q.x = bt[tx][i];
                q.y = bt[tx + 1][i];
                pt[(size_t)r * Pp + cp] = q;
            }
        }
    }
}

// X -> interleaved images of X and X^T (FP32): each CTA writes a 32 x 32
// element tile of one orientation, of one frame of one group, with the
// group's images staged together so that every element is written as one
// vector of w floats.  With p.on the last column of CTAs carries the
// view-table step, as in k_pairs_img.
__global__ void __launch_bounds__(256) k_interleave_img(const float *__restrict__ X, float *__restrict__ QX,
                                                        float *__restrict__ QT, int N, int Pp, int F, int K,
                                                        ViewPrep p, const int *__restrict__ skip)
{
    extern __shared__ unsigned long long prep_key[];
    if (skip && *skip) return;
    if (p.on && blockIdx.x == gridDim.x - 1) {
        if (blockIdx.y == 0 && blockIdx.z == 0) view_prep_block(p, prep_key);
        return;
    }
    // rows of X:    t[j][i][e] = X_j[r0 + i][e0 - 2 + e]
    // columns of X: t[j][e][i] = X_j[e0 - 2 + e][r0 + i]
    __shared__ float t[4][32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int e0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int n4 = K & ~3, rem = K - n4;
    const int ngroups = n4 / 4 + (rem >= 2 ? 1 : 0) + (rem & 1);
    for (int z = blockIdx.z; z < 2 * F * ngroups; z += gridDim.z) {
        const int trans = z & 1, gf = z >> 1;
        const int gi = gf / F, f = gf - gi * F;
        int k0, w;
        interleave_group(gi < n4 / 4 ? 4 * gi : (gi == n4 / 4 && rem >= 2 ? n4 : K - 1), K, k0, w);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j < w) {
                const float *src = X + ((size_t)(k0 + j) * F + f) * N * N;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int i = ty + 8 * m;
                    const int rr = trans ? e0 - 2 + i : r0 + i, cc = trans ? r0 + tx : e0 - 2 + tx;
                    t[j][i][tx] = (rr >= 0 && rr < N && cc >= 0 && cc < N) ? src[(size_t)rr * N + cc] : 0.0f;
                }
            }
        }
        __syncthreads();
        float *Q = (trans ? QT : QX) + (size_t)k0 * F * N * Pp;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int i = ty + 8 * m;
            const int r = r0 + i, e = e0 + tx;
            if (r >= N || e >= Pp) continue;
            float v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = trans ? t[j][tx][i] : t[j][i][tx];
            float *q = Q + (((size_t)f * N + r) * Pp + e) * w;
            if (w == 4)
                *reinterpret_cast<float4 *>(q) = make_float4(v[0], v[1], v[2], v[3]);
            else if (w == 2)
                *reinterpret_cast<float2 *>(q) = make_float2(v[0], v[1]);
            else
                *q = v[0];
        }
    }
}

// Pair images of the first nimg images of a batch of K from the interleaved
// ones: pair e of a row is (element e, element e + 1), zero past the row end.
__global__ void k_interleaved_to_pairs(const float *__restrict__ QX, const float *__restrict__ QT,
                                       float2 *__restrict__ PX, float2 *__restrict__ PT, int N, int Pp, int F,
                                       int K, int nimg)
{
    const long long per = (long long)F * N * Pp;  // elements per image
    const long long total = (long long)nimg * per;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(idx / per);
        const long long el = idx - k * per;
        const int e = (int)(el % Pp);
        int k0, w;
        interleave_group(k, K, k0, w);
        const size_t o = (size_t)k0 * per + (size_t)el * w + (k - k0);
        const bool last = e + 1 >= Pp;
        PX[idx] = make_float2(QX[o], last ? 0.0f : QX[o + w]);
        PT[idx] = make_float2(QT[o], last ? 0.0f : QT[o + w]);
    }
}

// YP[row][bp] = (Y[row][bp - 2], Y[row][bp - 1]), zero outside [0, B).
// With p.on, the last CTA runs the view-table step of the call instead.
template <typename T>
__global__ void k_pairs_sino(const T *__restrict__ Y, pair_t<T> *__restrict__ YP, int B, int Pb, long long total,
                             ViewPrep p, const int *__restrict__ skip)
{
    extern __shared__ unsigned long long prep_key[];
    if (skip && *skip) return;
    const int nblk = gridDim.x - (p.on ? 1 : 0);
    if (p.on && blockIdx.x == nblk) {
        view_prep_block(p, prep_key);
        return;
    }
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)nblk * blockDim.x) {
        const long long row = idx / Pb;
        const int bp = (int)(idx - row * Pb);
        const int b0 = bp - 2, b1 = bp - 1;
        const T *y = Y + row * B;
        pair_t<T> p;
        p.x = (b0 >= 0 && b0 < B) ? y[b0] : T(0);
        p.y = (b1 >= 0 && b1 < B) ? y[b1] : T(0);
        YP[idx] = p;
    }
}

// ---------------------------------------------------------------------------
// ray march
// ---------------------------------------------------------------------------
// One CTA = VW view slots x SPLIT row segments, all on the same 32-bin chunk.
// The view slots take VW consecutive entries of the view order (views sorted
// by marching axis and ray slope), so the warps of a CTA sweep nearly the
// same image band row by row and share it in L1.  SPLIT warps march
// consecutive row segments of the same rays and are combined in shared memory
// in a fixed order.
// Both taps of the KB images of an interleaved group at element e of a row
// (q points at element e): one vector load at e and one at e + 1 for each
// group of 4 images (gstride floats per image between the groups).
template <int KB>
__device__ __forceinline__ void taps_interleaved(const float *__restrict__ q, long long gstride, float2 (&p)[KB])
{
    if constexpr (KB >= 4) {
#pragma unroll
        for (int h = 0; h < KB / 4; ++h) {
            const float4 *e = reinterpret_cast<const float4 *>(q + (size_t)h * 4 * gstride);
            const float4 x = __ldg(e), y = __ldg(e + 1);
            p[4 * h + 0] = make_float2(x.x, y.x);
            p[4 * h + 1] = make_float2(x.y, y.y);
            p[4 * h + 2] = make_float2(x.z, y.z);
            p[4 * h + 3] = make_float2(x.w, y.w);
        }
    } else if constexpr (KB == 2) {
        const float2 *e = reinterpret_cast<const float2 *>(q);
        const float2 x = __ldg(e), y = __ldg(e + 1);
        p[0] = make_float2(x.x, y.x);
        p[1] = make_float2(x.y, y.y);
    } else {
        p[0] = make_float2(__ldg(q), __ldg(q + 1));
    }
}

// QL (FP32 forward only): the images come from the interleaved layout; the
// taps, the fractions and the order of the sums are those of the pair form,
// so both give the same bits.
template <typename T, int MODE, bool OFFS, int KB, int SPLIT, bool QL = false>
__global__ void __launch_bounds__(512) k_ray(RayArgs<T> a)
{
    using P2 = pair_t<T>;
    constexpr int NACC = (MODE == kFwd) ? KB : 3 * KB;
    extern __shared__ unsigned char ray_smem[];
    T *red = reinterpret_cast<T *>(ray_smem);  // [VW][SPLIT][NACC][32], only when SPLIT > 1
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int seg = warp % SPLIT;
    const int slot = warp / SPLIT;
    const int VW = a.VW;
    const int N = a.N;
    const int ngv = (a.V + VW - 1) / VW;
    const int total = a.ngroups * ngv * a.nchunks;
    if (a.skip && *a.skip) return;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int chunk = item % a.nchunks;
        const int t = item / a.nchunks;
        const int vgi = t % ngv;
        const int grp = t / ngv;
        const int pos = vgi * VW + slot;
        const int v = pos < a.V ? (a.order ? a.order[pos] : pos) : -1;
        const bool live = v >= 0 && !(MODE == kGn && a.view_mask && a.view_mask[v] == 0);  // warp-uniform
        const ViewGeo &g = a.vg[live ? v : 0];
        const int b = chunk * kChunk + lane;
        const bool active = live && b < a.B;
        const int k0 = a.kbase + grp * KB;
        T acc[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) acc[k] = T(0);
        if (live) {
            int rlo, rhi;
            warp_rows(g, b, b < a.B, N, rlo, rhi);
            const int len = rhi - rlo + 1;
            const int per = (len + SPLIT - 1) / SPLIT;
            const int r0 = rlo + seg * per;
            const int r1 = min(rhi, r0 + per - 1);
            long long Q = line_at(g, b, r0, N);
            const long long dQ = 2 * g.Qh;
            const P2 *img = (g.mode ? a.PT : a.PX) + (size_t)g.frame * N * a.Pp + (size_t)k0 * a.pimg_stride +
                            (size_t)r0 * a.Pp + 2;
            // Rows are processed in blocks of U: all loads of a block are issued
            // before any of them is used, so U*KB gathers are in flight per warp.
            constexpr int U = KB >= 4 ? 4 : 8;
            const int pp = a.Pp;
            if constexpr (MODE == kFwd && QL) {
                constexpr int QW = KB >= 4 ? 4 : KB;  // floats per element of the group's layout
                const float *q = (g.mode ? a.QT : a.QX) + (size_t)k0 * a.qimg_stride +
                                 (((size_t)g.frame * N + r0) * pp + 2) * QW;
                int r = r0;
                for (; r + U - 1 <= r1; r += U) {
                    P2 p[U][KB];
                    T f[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const long long Qu = Q + (long long)u * dQ;
                        const int cell = min(max(cell_of(Qu), -2), N);
                        f[u] = frac_of(Qu, T());
                        taps_interleaved<KB>(q + ((size_t)u * pp + cell) * QW, a.qimg_stride, p[u]);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const T omf = T(1) - f[u];
#pragma unroll
                        for (int k = 0; k < KB; ++k) acc[k] = fma(omf, p[u][k].x, fma(f[u], p[u][k].y, acc[k]));
                    }
                    q += (size_t)U * pp * QW;
                    Q += (long long)U * dQ;
                }
                for (; r <= r1; ++r, q += (size_t)pp * QW, Q += dQ) {
                    const int cell = min(max(cell_of(Q), -2), N);
                    const T fr = frac_of(Q, T());
                    const T omf = T(1) - fr;
                    P2 p[KB];
                    taps_interleaved<KB>(q + (size_t)cell * QW, a.qimg_stride, p);
#pragma unroll
                    for (int k = 0; k < KB; ++k) acc[k] = fma(omf, p[k].x, fma(fr, p[k].y, acc[k]));
                }
            } else if constexpr (MODE == kFwd) {
                int r = r0;
                for (; r + U - 1 <= r1; r += U) {
                    P2 p[U][KB];
                    T f[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const long long Qu = Q + (long long)u * dQ;
                        const int cell = min(max(cell_of(Qu), -2), N);
                        f[u] = frac_of(Qu, T());
                        const P2 *row = img + (size_t)u * pp + cell;
#pragma unroll
                        for (int k = 0; k < KB; ++k) p[u][k] = __ldg(row + (size_t)k * a.pimg_stride);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const T omf = T(1) - f[u];
#pragma unroll
                        for (int k = 0; k < KB; ++k) acc[k] = fma(omf, p[u][k].x, fma(f[u], p[u][k].y, acc[k]));
                    }
                    img += (size_t)U * pp;
                    Q += (long long)U * dQ;
                }
                for (; r <= r1; ++r, img += pp, Q += dQ) {
                    const int cell = min(max(cell_of(Q), -2), N);
                    const T fr = frac_of(Q, T());
                    const T omf = T(1) - fr;
#pragma unroll
                    for (int k = 0; k < KB; ++k) {
                        const P2 q = __ldg(img + (size_t)k * a.pimg_stride + cell);
                        acc[k] = fma(omf, q.x, fma(fr, q.y, acc[k]));
                    }
                }
            } else {
                // per image k of the group: acc[3k] = sum of interpolated values,
                // acc[3k+1] = sum slope * dq/dtheta, acc[3k+2] = sum of slopes
                // (offset derivative); the line, cell and fraction serve all KB images
                const T g0 = fma(GeoT<T>::sb(g, b), GeoT<T>::gs(g), GeoT<T>::gh(g, N));
                const T gr = GeoT<T>::gr(g);
                T rf = (T)r0;
                int r = r0;
                for (; r + U - 1 <= r1; r += U) {
                    P2 p[U][KB];
                    T f[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const long long Qu = Q + (long long)u * dQ;
                        const int cell = min(max(cell_of(Qu), -2), N);
                        f[u] = frac_of(Qu, T());
                        const P2 *row = img + (size_t)u * pp + cell;
#pragma unroll
                        for (int k = 0; k < KB; ++k) p[u][k] = __ldg(row + (size_t)k * a.pimg_stride);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const T dq = fma(rf + T(u), gr, g0);
#pragma unroll
                        for (int k = 0; k < KB; ++k) {
                            const T d = p[u][k].y - p[u][k].x;
                            acc[3 * k] += fma(f[u], d, p[u][k].x);
                            acc[3 * k + 1] = fma(d, dq, acc[3 * k + 1]);
                            if (OFFS) acc[3 * k + 2] += d;
                        }
                    }
                    img += (size_t)U * pp;
                    Q += (long long)U * dQ;
                    rf += T(U);
                }
                for (; r <= r1; ++r, img += pp, Q += dQ, rf += T(1)) {
                    const int cell = min(max(cell_of(Q), -2), N);
                    const T fr = frac_of(Q, T());
                    const T dq = fma(rf, gr, g0);
#pragma unroll
                    for (int k = 0; k < KB; ++k) {
                        const P2 q = __ldg(img + (size_t)k * a.pimg_stride + cell);
                        const T d = q.y - q.x;
                        acc[3 * k] += fma(fr, d, q.x);
                        acc[3 * k + 1] = fma(d, dq, acc[3 * k + 1]);
                        if (OFFS) acc[3 * k + 2] += d;
                    }
                }
            }
        }
        if constexpr (SPLIT > 1) {
            T *mine = red + ((size_t)(slot * SPLIT + seg) * NACC) * 32;
#pragma unroll
            for (int k = 0; k < NACC; ++k) mine[k * 32 + lane] = acc[k];
            __syncthreads();
            if (seg == 0) {
                const T *base = red + ((size_t)slot * SPLIT * NACC) * 32;
#pragma unroll
                for (int k = 0; k < NACC; ++k) {
                    T s = base[k * 32 + lane];
#pragma unroll
                    for (int q = 1; q < SPLIT; ++q) s += base[(q * NACC + k) * 32 + lane];
                    acc[k] = s;
                }
            }
        }
        if (seg == 0 && live) ray_epilogue<T, MODE, OFFS, KB>(a, g, v, b, active, k0, chunk, lane, acc);
        if constexpr (SPLIT > 1) __syncthreads();  // red[] is reused by the next item
    }
}

// out_q[k][v] = scale_q * sum_c partial[k][v][c][q], summed in chunk order,
// for each of nimg images (partials part_stride doubles apart); with sum, one
// output per view summing the images in order (each image's chunks in order).
// One warp per output: the lanes load 32 chunks at a time in one round trip,
// and the sums run over them in chunk order through shuffles.
__global__ void k_finalize(const double *__restrict__ partial, int V, int nchunks, int nimg, long long part_stride,
                           int sum, double *out0, double *out1, double *out2, double scale2, double *out3,
                           const int *__restrict__ view_mask, const int *__restrict__ skip)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nout = sum ? 1 : nimg;
    if (w >= V * nout || (skip && *skip)) return;  // warp-uniform
    const int v = w % V, kout = w / V;
    if (view_mask && view_mask[v] == 0) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;  // sums over the images, each image's sum added in order
    const int klo = sum ? 0 : kout, khi = sum ? nimg : kout + 1;
    for (int k = klo; k < khi; ++k) {
        const double *p = partial + (size_t)k * part_stride + (size_t)v * nchunks * 4;
        double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;  // this image, chunks in order
        for (int base = 0; base < nchunks; base += 32) {
            double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
            if (base + lane < nchunks) {
                q0 = p[4 * (base + lane) + 0];
                q1 = p[4 * (base + lane) + 1];
                q2 = p[4 * (base + lane) + 2];
                if (out3) q3 = p[4 * (base + lane) + 3];
            }
            const int n = min(32, nchunks - base);
            for (int c = 0; c < n; ++c) {
                t0 += __shfl_sync(0xffffffffu, q0, c);
                t1 += __shfl_sync(0xffffffffu, q1, c);
                t2 += __shfl_sync(0xffffffffu, q2, c);
                if (out3) t3 += __shfl_sync(0xffffffffu, q3, c);
            }
        }
        s0 += t0;
        s1 += t1;
        s2 += t2;
        s3 += t3;
    }
    if (lane == 0) {
        const size_t o = (size_t)kout * V + v;
        if (out0) out0[o] = s0;
        if (out1) out1[o] = s1;
        if (out2) out2[o] = scale2 * s2;
        if (out3) out3[o] = s3;
    }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
template <typename T> RayArgs<T> base_args(const Handle &h)
{
    RayArgs<T> a{};
    a.vg = h.d_views;
    a.V = h.V;
    a.N = h.N;
    a.B = h.B;
    a.nchunks = h.nchunks;
    a.Pp = h.Pp;
    a.PX = (const pair_t<T> *)h.d_px;
    a.PT = (const pair_t<T> *)h.d_pt;
    a.pimg_stride = (long long)h.F * h.N * h.Pp;
    a.kbase = 0;
    a.ngroups = 1;
    a.sino_stride = (long long)h.V * h.B;
    a.order = h.d_order;
    a.VW = 1;
    a.segs = 1;
    a.kend = 1 << 30;
    return a;
}

template <typename T, int MODE, bool OFFS, int KB, int SPLIT, bool QL = false>
cudaError_t run_ray(const Handle &h, const RayArgs<T> &a)
{
    auto kern = k_ray<T, MODE, OFFS, KB, SPLIT, QL>;
    constexpr int NACC = (MODE == kFwd) ? KB : 3 * KB;
    const int threads = 32 * SPLIT * a.VW;
    const size_t smem = SPLIT > 1 ? (size_t)a.VW * SPLIT * NACC * 32 * sizeof(T) : 0;
    const long long items = (long long)a.ngroups * ((a.V + a.VW - 1) / a.VW) * a.nchunks;
    const int grid = persistent_grid(kern, threads, smem, items, h.num_sms);
    kern<<<grid, threads, smem, h.stream>>>(a);
    return cudaGetLastError();
}

template <typename T, int MODE, bool OFFS, int KB>
cudaError_t run_ray_split(const Handle &h, const RayArgs<T> &a, int split)
{
    switch (split) {
    case 1: return run_ray<T, MODE, OFFS, KB, 1>(h, a);
    case 2: return run_ray<T, MODE, OFFS, KB, 2>(h, a);
    case 4: return run_ray<T, MODE, OFFS, KB, 4>(h, a);
    default: return run_ray<T, MODE, OFFS, KB, 8>(h, a);
    }
}

// FP32 with a staged shape runs the band kernel (ct_band.cu); every other
// case runs k_ray.
template <typename T, int MODE, bool OFFS, int KB>
cudaError_t run_ray_any(const Handle &h, const RayArgs<T> &a, int split, int stage)
{
    if (h.fan_D > 0.0) return run_fan_ray<T>(h, a, MODE, KB, split, OFFS);
    if constexpr (std::is_same<T, float>::value) {
        if (stage > 0 && band_shape_ok(MODE, KB, a.VW, stage)) return run_ray_band(h, a, MODE, OFFS, KB, stage);
    }
    return run_ray_split<T, MODE, OFFS, KB>(h, a, split);
}

// The FP32 forward on the interleaved images: kb 8 (two groups of 4), 4, 2 or 1.
template <int KB>
cudaError_t run_fwd_interleaved(const Handle &h, const RayArgs<float> &a, int split)
{
    switch (split) {
    case 1: return run_ray<float, kFwd, false, KB, 1, true>(h, a);
    case 2: return run_ray<float, kFwd, false, KB, 2, true>(h, a);
    case 4: return run_ray<float, kFwd, false, KB, 4, true>(h, a);
    default: return run_ray<float, kFwd, false, KB, 8, true>(h, a);
    }
}

template <typename T>
cudaError_t fwd_groups(const Handle &h, RayArgs<T> a, int kb, int split, int stage)
{
    switch (kb) {
    case 1: return run_ray_any<T, kFwd, false, 1>(h, a, split, stage);
    case 2: return run_ray_any<T, kFwd, false, 2>(h, a, split, stage);
    case 4: return run_ray_any<T, kFwd, false, 4>(h, a, split, stage);
    default: return run_ray_any<T, kFwd, false, 8>(h, a, split, stage);
    }
}

}  // namespace

namespace {

ViewPrep view_prep_args(const Handle &h, const double *theta, const double *delta)
{
    ViewPrep p{};
    p.theta = theta;
    p.delta = delta;
    p.fov = h.d_fov;
    p.V = h.V;
    p.N = h.N;
    p.B = h.B;
    p.on = theta != nullptr;
    p.vg = h.d_views;
    p.flag = h.d_flag;
    p.order = h.d_order;
    return p;
}

size_t prep_smem(const ViewPrep &p) { return p.on ? sizeof(unsigned long long) * std::min(p.V, kOrderMaxV) : 0; }

// The layout kernels may carry the view-table step in up to 32 KB of dynamic shared memory.
template <auto Kernel> cudaError_t allow_prep_smem()
{
    static bool done = false;  // one flag per kernel; the attribute is idempotent, so a race is harmless
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(unsigned long long) * kOrderMaxV));
    if (e == cudaSuccess) done = true;
    return e;
}

}  // namespace

cudaError_t launch_view_setup(const Handle &h, const double *theta, const double *delta, const int *skip)
{
    k_view_prep<<<1, 1024, 0, h.stream>>>(view_prep_args(h, theta, delta), skip);
    if (h.fan_D > 0.0 && theta) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_fan_rays(h, skip);
    }
    return cudaGetLastError();
}

cudaError_t launch_view_setup_wide(const Handle &h, const double *theta, const double *delta, int *changed,
                                   const int *skip)
{
    const ViewPrep p = view_prep_args(h, theta, delta);
    const int grid = std::max(1, std::min((h.V + 127) / 128, 4 * h.num_sms));
    k_view_setup_many<<<grid, 128, 0, h.stream>>>(p, changed, skip);
    k_view_order<<<1, 1024, 0, h.stream>>>(p, changed, skip);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (h.fan_D > 0.0) return launch_fan_rays(h, skip);
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_pairs_img(const Handle &h, const T *X, int nimg, const int *skip, const double *theta,
                             const double *delta)
{
    const ViewPrep p = view_prep_args(h, theta, delta);
    cudaError_t e = allow_prep_smem<k_pairs_img<T>>();
    if (e != cudaSuccess) return e;
    dim3 grid((h.Pp + 31) / 32 + (p.on ? 1 : 0), (h.N + 31) / 32, std::max(1, std::min(nimg, 65535)));
    k_pairs_img<T><<<grid, 256, prep_smem(p), h.stream>>>(X, (pair_t<T> *)h.d_px, (pair_t<T> *)h.d_pt, h.N, h.Pp,
                                                          nimg, p, skip);
    if (h.fan_D > 0.0 && theta) {
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_fan_rays(h, skip);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prep_forward(const Handle &h, const T *X, int nimg, const int *skip, const double *theta,
                                const double *delta)
{
    return launch_pairs_img<T>(h, X, nimg, skip, theta, delta);
}

cudaError_t launch_interleave_img(const Handle &h, const float *X, int batch, const double *theta,
                                  const double *delta, const int *skip)
{
    if (!h.d_qx || h.fan_D > 0.0 || batch < 1 || batch > h.max_batch) return cudaErrorInvalidValue;
    const ViewPrep p = view_prep_args(h, theta, delta);
    cudaError_t e = allow_prep_smem<k_interleave_img>();
    if (e != cudaSuccess) return e;
    const int n4 = batch & ~3, rem = batch - n4;
    const int ngroups = n4 / 4 + (rem >= 2 ? 1 : 0) + (rem & 1);
    dim3 grid((h.Pp + 31) / 32 + (p.on ? 1 : 0), (h.N + 31) / 32, std::max(1, std::min(2 * h.F * ngroups, 65535)));
    k_interleave_img<<<grid, 256, prep_smem(p), h.stream>>>(X, h.d_qx, h.d_qt, h.N, h.Pp, h.F, batch, p, skip);
    return cudaGetLastError();
}

cudaError_t launch_interleaved_to_pairs(const Handle &h, int batch)
{
    if (!h.d_qx || h.precision != 0 || batch < 1 || batch > h.max_batch) return cudaErrorInvalidValue;
    const long long total = (long long)batch * h.F * h.N * h.Pp;
    const long long blocks = std::min<long long>((total + 255) / 256, (long long)h.num_sms * 16);
    k_interleaved_to_pairs<<<(int)std::max<long long>(1, blocks), 256, 0, h.stream>>>(
        h.d_qx, h.d_qt, (float2 *)h.d_px, (float2 *)h.d_pt, h.N, h.Pp, h.F, batch, batch);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pairs_sino(const Handle &h, const T *Y, int nsino, const int *skip, const double *theta,
                              const double *delta)
{
    const ViewPrep p = view_prep_args(h, theta, delta);
    cudaError_t e = allow_prep_smem<k_pairs_sino<T>>();
    if (e != cudaSuccess) return e;
    const long long total = (long long)nsino * h.V * h.Pb;
    const int threads = 256;
    const long long blocks = std::min<long long>((total + threads - 1) / threads, (long long)h.num_sms * 16);
    if (h.fan_D > 0.0) {
        // fan beam: the transpose reads the interleaved layout instead; the view-table
        // step (when the angles come with the call) runs on its own
        if (p.on) {
            e = launch_view_setup(h, theta, delta, skip);
            if (e != cudaSuccess) return e;
        }
        return launch_fan_sino<T>(h, Y, nsino, skip);
    }
    k_pairs_sino<T><<<(int)std::max<long long>(1, blocks) + (p.on ? 1 : 0), threads, prep_smem(p), h.stream>>>(
        Y, (pair_t<T> *)h.d_yp, h.B, h.Pb, total, p, skip);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_forward(const Handle &h, T *Y, int batch, int kb, int split, int vw, int stage, const int *skip,
                           bool interleaved, int layout_batch)
{
    RayArgs<T> a = base_args<T>(h);
    a.Y = Y;
    a.skip = skip;
    a.VW = vw;
    if (interleaved) {
        // The groups of the layout (a batch of layout_batch images: groups of 8 = two
        // interleaved groups of 4, or 4, then the remainder's 2 and 1) that hold one of
        // the first `batch` images; images past `batch` in the last of them are read
        // but not written.
        if constexpr (std::is_same<T, float>::value) {
            if (!h.d_qx || h.fan_D > 0.0 || layout_batch < batch || layout_batch > h.max_batch)
                return cudaErrorInvalidValue;
            a.QX = h.d_qx;
            a.QT = h.d_qt;
            a.qimg_stride = (long long)h.F * h.N * h.Pp;
            a.kend = batch;
            int k = 0;
            for (int width : {8, 4, 2, 1}) {
                if (width == 8 && kb < 8) continue;
                if (k >= batch) break;
                const int groups = std::min((layout_batch - k) / width, (batch - k + width - 1) / width);
                if (groups == 0) continue;
                a.kbase = k;
                a.ngroups = groups;
                cudaError_t e = width == 8   ? run_fwd_interleaved<8>(h, a, split)
                                : width == 4 ? run_fwd_interleaved<4>(h, a, split)
                                : width == 2 ? run_fwd_interleaved<2>(h, a, split)
                                             : run_fwd_interleaved<1>(h, a, split);
                if (e != cudaSuccess) return e;
                k += groups * width;
            }
            return cudaSuccess;
        } else {
            return cudaErrorInvalidValue;
        }
    }
    // band-staged FP32 march with `split` CTAs per ray: segment partials go to Y and d_segpart
    const bool band = std::is_same<T, float>::value && stage > 0 && band_shape_ok(kFwd, 1, vw, stage) &&
                      !(h.fan_D > 0.0);
    if (band && split > 1) {
        if (!h.d_segpart || split > 4) return cudaErrorInvalidValue;
        a.segs = split;
        a.fpart = (T *)h.d_segpart;
        a.fpart_stride = (long long)h.max_batch * h.V * h.B;
    }
    int k = 0;
    for (int width : {8, 4, 2, 1}) {
        if (width > kb) continue;
        const int groups = (batch - k) / width;
        if (groups == 0) continue;
        a.kbase = k;
        a.ngroups = groups;
        cudaError_t e = fwd_groups<T>(h, a, width, split, stage);
        if (e != cudaSuccess) return e;
        k += groups * width;
    }
    if constexpr (std::is_same<T, float>::value) {
        if (a.segs > 1) return launch_fwd_combine(h, Y, a.fpart, a.segs, a.fpart_stride, batch, skip);
    }
    return cudaSuccess;
}

// The derivative modes over `batch` images sharing the view table: groups of
// up to kb (1, 2 or 4) images per lane; the fan-beam and band-staged forms
// take one image per lane (their launches still cover the whole batch).
template <typename T, int MODE, bool OFFS>
cudaError_t der_groups(const Handle &h, RayArgs<T> a, int batch, int kb, int split, int stage)
{
    bool one = h.fan_D > 0.0;
    if constexpr (std::is_same<T, float>::value) one = one || (stage > 0 && band_shape_ok(MODE, 1, a.VW, stage));
    int k = 0;
    for (int width : {4, 2, 1}) {
        if (width > kb || (one && width > 1)) continue;
        const int groups = (batch - k) / width;
        if (groups == 0) continue;
        a.kbase = k;
        a.ngroups = groups;
        cudaError_t e;
        switch (width) {
        case 4: e = run_ray_any<T, MODE, OFFS, 4>(h, a, split, stage); break;
        case 2: e = run_ray_any<T, MODE, OFFS, 2>(h, a, split, stage); break;
        default: e = run_ray_any<T, MODE, OFFS, 1>(h, a, split, stage); break;
        }
        if (e != cudaSuccess) return e;
        k += groups * width;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_jvp(const Handle &h, const double *dtheta, const double *ddelta, T *dY, int split, int vw,
                       int stage, int batch, int kb, long long dir_stride)
{
    RayArgs<T> a = base_args<T>(h);
    a.VW = vw;
    a.Y = dY;
    a.dtheta = dtheta;
    a.ddelta = ddelta;
    a.dir_stride = dir_stride;
    return ddelta ? der_groups<T, kJvp, true>(h, a, batch, kb, split, stage)
                  : der_groups<T, kJvp, false>(h, a, batch, kb, split, stage);
}

template <typename T>
cudaError_t launch_vjp(const Handle &h, const T *R, double *gtheta, double *gdelta, int split, int vw, int stage,
                       int batch, int kb, long long r_stride, int sum)
{
    RayArgs<T> a = base_args<T>(h);
    a.VW = vw;
    a.R = R;
    a.r_stride = r_stride;
    a.partial = h.d_partial;
    a.part_stride = 4LL * h.V * h.nchunks;
    cudaError_t e = gdelta ? der_groups<T, kVjp, true>(h, a, batch, kb, split, stage)
                           : der_groups<T, kVjp, false>(h, a, batch, kb, split, stage);
    if (e != cudaSuccess) return e;
    const long long outs = (long long)h.V * (sum ? 1 : batch);
    k_finalize<<<(int)((outs + 7) / 8), 256, 0, h.stream>>>(h.d_partial, h.V, h.nchunks, batch, a.part_stride,
                                                            sum, gtheta, gdelta, nullptr, 1.0, nullptr, nullptr,
                                                            nullptr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gn(const Handle &h, const T *bdata, T *res, double *grad, double *jnorm2, double *fval, int split,
                      int vw, int stage, const int *view_mask, const int *skip, int batch, int kb, double *rscale)
{
    RayArgs<T> a = base_args<T>(h);
    a.VW = vw;
    a.R = bdata;
    a.r_stride = (long long)h.V * h.B;
    a.res = res;
    a.partial = h.d_partial;
    a.part_stride = 4LL * h.V * h.nchunks;
    a.view_mask = view_mask;
    a.skip = skip;
    cudaError_t e = der_groups<T, kGn, false>(h, a, batch, kb, split, stage);
    if (e != cudaSuccess) return e;
    const long long outs = (long long)h.V * batch;
    k_finalize<<<(int)((outs + 7) / 8), 256, 0, h.stream>>>(h.d_partial, h.V, h.nchunks, batch, a.part_stride, 0,
                                                            grad, jnorm2, fval, 0.5, rscale, view_mask, skip);
    return cudaGetLastError();
}

#define CTGB_RAY_INSTANTIATE(T)                                                                             \
    template cudaError_t launch_pairs_img<T>(const Handle &, const T *, int, const int *, const double *,   \
                                             const double *);                                              \
    template cudaError_t launch_pairs_sino<T>(const Handle &, const T *, int, const int *, const double *,  \
                                              const double *);                                             \
    template cudaError_t launch_prep_forward<T>(const Handle &, const T *, int, const int *, const double *, \
                                                const double *);                                           \
    template cudaError_t launch_forward<T>(const Handle &, T *, int, int, int, int, int, const int *, bool, int); \
    template cudaError_t launch_jvp<T>(const Handle &, const double *, const double *, T *, int, int, int, int, \
                                       int, long long);                                                   \
    template cudaError_t launch_vjp<T>(const Handle &, const T *, double *, double *, int, int, int, int, int, \
                                       long long, int);                                                   \
    template cudaError_t launch_gn<T>(const Handle &, const T *, T *, double *, double *, double *, int,    \
                                      int, int, const int *, const int *, int, int, double *);

CTGB_RAY_INSTANTIATE(float)
CTGB_RAY_INSTANTIATE(double)

}  // namespace ctgb
