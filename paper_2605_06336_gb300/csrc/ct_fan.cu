// Fan-beam form of the Joseph operator (sm_103a).
//
// Geometry (the fan-beam CT of Sec. 6.2; the paper gives no distances, so
// they are a reading): a point source at distance D from the rotation
// centre and a flat detector rescaled to the line through the centre, on
// which bin b keeps the parallel-beam centre s_b = b - (B-1)/2 + delta_v.
// With e = (cos, sin) and t = (-sin, cos), the source is S = -D t, bin b is
// P_b = s_b e, and ray (v,b) has direction r = P_b - S = s_b e + D t.  As D
// grows the rays become the parallel-beam rays.
//
// Every ray is marched like a parallel-beam ray, but with its own line: rows
// when |r_x| <= |r_y| (x(y) = A + C y, C = r_x / r_y, A = P_x - P_y C),
// columns otherwise (y(x) = A + C x, C = r_y / r_x, A = P_y - P_x C), weight
// sqrt(1 + C^2).  In march coordinates q(r) = q_h + (r - h) qr with
// q_h = h + A (rows) or h - A (columns), qr = -C, carried in the same 64-bit
// fixed point as the parallel-beam lines.  The geometry turns rigidly with
// theta (dr/dtheta = (-r_y, r_x), dP_b/dtheta = s_b t), so
// dq/dtheta = g0 + r gr with gr = -dC/dtheta, g0 = +-dA/dtheta + h dC/dtheta,
// and dw/dtheta = C dC/dtheta / w.  An offset delta_v moves every bin centre
// along e (ds_b/ddelta = 1, the source stays): dq/ddelta = s0 + r sr with
// sr = -dC/ds, s0 = +-dA/ds + h dC/ds, and dw/ddelta = C dC/ds / w.
//
//   k_fan_rays   per-ray table (fixed-point line, weight, derivative
//                constants, march range) from the view table, for the views
//                rebuilt since (generation stamps)
//   k_fan_views  per-view record of the transpose (FP32 constants, bin
//                ranges of row- and column-marched rays)
//   k_ray_fan    SPLIT warps (row segments) per 32 bins of one view: forward
//                (KB images), JVP, VJP and Gauss-Newton terms, each lane on
//                its own line
//   k_fan_sino   sinograms interleaved in blocks of 8 for the transpose
//   k_adj_fan    exact transpose in gather form: a pixel takes, per view,
//                the rays whose fixed-point sample at its row (row-marched
//                rays) or column (column-marched rays) falls in its
//                interpolation cell; the candidates come from the projective
//                inverse of the pixel's neighbourhood and are then tested
//                with the very values the forward uses, so the matrix
//                entries are those of the forward.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "ct_device.cuh"
#include "ct_internal.cuh"

namespace ctgb {
namespace {

template <typename T> struct __align__(16) FanRay {
    long long Qc, Qh;  // q(r) = (Qc + (2r - (N-1)) Qh) / 2^48
    T w, dw, g0, gr;   // weight, d w / d theta, dq/dtheta = g0 + r gr
    float rlo, rhi;    // march indices with -1 < q < N lie in [rlo, rhi] (two indices of margin)
    int mode;          // 0: rows of X, 1: rows of X^T (columns)
    int gen;           // generation of the view record the entry was built from (0: never)
    T dws, s0, sr;     // d w / d delta, dq/ddelta = s0 + r sr
};

// The fields of a ray the transpose's candidate search reads, in a table of
// their own after the FanRay table (24 bytes a ray instead of 64: the search
// touches a few records per pixel and view, scattered over the whole table).
template <typename T> struct FanLine {
    long long Qc, Qh;
    T w;
};
template <typename T> __host__ __device__ inline FanLine<T> *fan_lines(void *rays, long long nrays)
{
    return reinterpret_cast<FanLine<T> *>(reinterpret_cast<unsigned char *>(rays) + nrays * sizeof(FanRay<T>));
}

// Per view: FP32 constants of the transpose's candidate search and the bin
// ranges of the two march axes (the ray direction turns monotonically with
// s_b over a fan narrower than 90 degrees, so the axis changes at most once:
// bins [0, split) march along mode0, bins [split, B) along the other axis).
struct __align__(16) FanView {
    float c, sn, sb0, iD;
    int mode0, split, gen, pad;
};

template <typename T>
__global__ void __launch_bounds__(256) k_fan_rays(const ViewGeo *__restrict__ vg, int V, int B, int N, double D,
                                                  FanRay<T> *__restrict__ out, FanLine<T> *__restrict__ lines,
                                                  const int *__restrict__ skip)
{
    if (skip && *skip) return;
    const double h = 0.5 * (N - 1);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)V * B;
         idx += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(idx / B), b = (int)(idx - (long long)v * B);
        const ViewGeo &g = vg[v];
        if (out[idx].gen == g.gen) continue;  // built from this view record already
        const double c = g.c, sn = g.s, s = g.sb0d + (double)b;
        const double rx = s * c - D * sn, ry = s * sn + D * c;
        const double px = s * c, py = s * sn, dpx = -s * sn, dpy = s * c;
        double C, A, dC, dA, qh, g0, dCs, s0;
        int mode;
        if (fabs(rx) <= fabs(ry)) {
            mode = 0;
            C = rx / ry;
            A = px - py * C;
            dC = -(1.0 + C * C);
            dA = dpx - C * dpy - py * dC;
            qh = h + A;
            g0 = dA + h * dC;
            dCs = (c * ry - sn * rx) / (ry * ry);  // d/ds of C and A: P_b and r move by e
            s0 = (c - C * sn - py * dCs) + h * dCs;
        } else {
            mode = 1;
            C = ry / rx;
            A = py - px * C;
            dC = 1.0 + C * C;
            dA = dpy - C * dpx - px * dC;
            qh = h - A;
            g0 = -dA + h * dC;
            dCs = (sn * rx - c * ry) / (rx * rx);
            s0 = -(sn - C * c - px * dCs) + h * dCs;
        }
        const double qr = -C;
        const double w = sqrt(1.0 + C * C);
        FanRay<T> R;
        R.Qc = __double2ll_rn(qh * kFixScale);
        R.Qh = __double2ll_rn(qr * 0.5 * kFixScale);
        R.w = (T)w;
        R.dw = (T)(C * dC / w);
        R.g0 = (T)g0;
        R.gr = (T)(-dC);
        R.dws = (T)(C * dCs / w);
        R.s0 = (T)s0;
        R.sr = (T)(-dCs);
        R.mode = mode;
        R.gen = g.gen;
        if (fabs(qr) < 1e-12) {
            const bool in = qh > -1.0 && qh < (double)N;
            R.rlo = in ? 0.0f : (float)N;
            R.rhi = in ? (float)(N - 1) : -1.0f;
        } else {
            const double ra = h + (-1.0 - qh) / qr, rb = h + ((double)N - qh) / qr;
            R.rlo = (float)fmin(fmax(fmin(ra, rb) - 2.0, 0.0), (double)N);
            R.rhi = (float)fmax(fmin(fmax(ra, rb) + 2.0, (double)(N - 1)), -1.0);
        }
        out[idx] = R;
        FanLine<T> L;
        L.Qc = R.Qc;
        L.Qh = R.Qh;
        L.w = R.w;
        lines[idx] = L;
    }
}

// One warp per view: the per-view record of the transpose, rebuilt when the
// view record changed (after k_fan_rays has rebuilt its rays).
template <typename T>
__global__ void __launch_bounds__(256) k_fan_views(const ViewGeo *__restrict__ vg, int V, int B, double D,
                                                   const FanRay<T> *__restrict__ rays, FanView *__restrict__ out,
                                                   const int *__restrict__ skip)
{
    if (skip && *skip) return;
    const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= V) return;  // warp-uniform
    const ViewGeo &g = vg[v];
    if (out[v].gen == g.gen) return;
    const FanRay<T> *rv = rays + (size_t)v * B;
    const int mode0 = rv[0].mode;
    int split = B;
    for (int base = 0; base < B; base += 32) {
        const int b = base + lane;
        const unsigned other = __ballot_sync(0xffffffffu, b < B && rv[b].mode != mode0);
        if (other) {
            split = base + __ffs(other) - 1;
            break;
        }
    }
    if (lane == 0) {
        FanView f;
        f.c = (float)g.c;
        f.sn = (float)g.s;
        f.sb0 = (float)g.sb0d;
        f.iD = (float)(1.0 / D);
        f.mode0 = mode0;
        f.split = split;
        f.gen = g.gen;
        f.pad = 0;
        out[v] = f;
    }
}

// One CTA = SPLIT warps on one work item: 32 consecutive bins of one view
// (and one batch group of KB images for the forward).  The warps march
// consecutive segments of the warp-union row range; their sums are added in
// segment order in shared memory and warp 0 writes the result.
template <typename T, int MODE, int KB, int SPLIT, bool OFFS>
__global__ void __launch_bounds__(32 * SPLIT) k_ray_fan(RayArgs<T> a, const FanRay<T> *__restrict__ rays)
{
    using P2 = pair_t<T>;
    constexpr int NACC = (MODE == kFwd) ? KB : (OFFS ? 3 : 2);
    __shared__ T red[SPLIT > 1 ? SPLIT : 1][NACC][32];
    const int lane = threadIdx.x & 31;
    const int seg = threadIdx.x >> 5;
    const int N = a.N;
    const long long total = (long long)a.ngroups * a.V * a.nchunks;
    if (a.skip && *a.skip) return;
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {  // CTA-uniform
        const int chunk = (int)(item % a.nchunks);
        const long long t = item / a.nchunks;
        const int v = (int)(t % a.V);
        const int grp = (int)(t / a.V);
        if (MODE == kGn && a.view_mask && a.view_mask[v] == 0) continue;  // CTA-uniform
        const int b = chunk * kChunk + lane;
        const bool active = b < a.B;
        const FanRay<T> R = rays[(size_t)v * a.B + (active ? b : a.B - 1)];
        const int k0 = a.kbase + grp * KB;
        int rlo = active ? (int)floorf(R.rlo) : N, rhi = active ? (int)ceilf(R.rhi) : -1;
        rlo = __reduce_min_sync(0xffffffffu, rlo);
        rhi = __reduce_max_sync(0xffffffffu, rhi);
        const int per = rhi >= rlo ? (rhi - rlo + SPLIT) / SPLIT : 0;
        const int r0 = rlo + seg * per, r1 = min(rhi, r0 + per - 1);
        T acc[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) acc[k] = T(0);
        const P2 *img = (R.mode ? a.PT : a.PX) + (size_t)a.vg[v].frame * N * a.Pp + (size_t)k0 * a.pimg_stride + 2;
        const long long dQ = 2 * R.Qh;
        long long Q = R.Qc + (long long)(2 * r0 - (N - 1)) * R.Qh;
        constexpr int U = 4;
        int r = r0;
        if constexpr (MODE == kFwd) {
            for (; r + U - 1 <= r1; r += U) {
                P2 p[U][KB];
                T f[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long Qu = Q + (long long)u * dQ;
                    const int cell = min(max(cell_of(Qu), -2), N);
                    f[u] = frac_of(Qu, T());
                    const P2 *row = img + (size_t)(r + u) * a.Pp + cell;
#pragma unroll
                    for (int k = 0; k < KB; ++k) p[u][k] = __ldg(row + (size_t)k * a.pimg_stride);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const T omf = T(1) - f[u];
#pragma unroll
                    for (int k = 0; k < KB; ++k) acc[k] = fma(omf, p[u][k].x, fma(f[u], p[u][k].y, acc[k]));
                }
                Q += (long long)U * dQ;
            }
            for (; r <= r1; ++r, Q += dQ) {
                const int cell = min(max(cell_of(Q), -2), N);
                const T fr = frac_of(Q, T());
                const T omf = T(1) - fr;
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    const P2 q = __ldg(img + (size_t)r * a.Pp + (size_t)k * a.pimg_stride + cell);
                    acc[k] = fma(omf, q.x, fma(fr, q.y, acc[k]));
                }
            }
        } else {
            // acc[0] = sum of interpolated values, acc[1] = sum slope * dq/dtheta,
            // acc[2] (offsets) = sum slope * dq/ddelta; rows in blocks of U whose
            // loads are all issued first
            for (; r + U - 1 <= r1; r += U) {
                P2 p[U];
                T f[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long Qu = Q + (long long)u * dQ;
                    const int cell = min(max(cell_of(Qu), -2), N);
                    f[u] = frac_of(Qu, T());
                    p[u] = __ldg(img + (size_t)(r + u) * a.Pp + cell);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const T d = p[u].y - p[u].x;
                    acc[0] += fma(f[u], d, p[u].x);
                    acc[1] = fma(d, fma((T)(r + u), R.gr, R.g0), acc[1]);
                    if constexpr (OFFS) acc[NACC - 1] = fma(d, fma((T)(r + u), R.sr, R.s0), acc[NACC - 1]);
                }
                Q += (long long)U * dQ;
            }
            for (; r <= r1; ++r, Q += dQ) {
                const int cell = min(max(cell_of(Q), -2), N);
                const T fr = frac_of(Q, T());
                const P2 q = __ldg(img + (size_t)r * a.Pp + cell);
                const T d = q.y - q.x;
                acc[0] += fma(fr, d, q.x);
                acc[1] = fma(d, fma((T)r, R.gr, R.g0), acc[1]);
                if constexpr (OFFS) acc[NACC - 1] = fma(d, fma((T)r, R.sr, R.s0), acc[NACC - 1]);
            }
        }
        if constexpr (SPLIT > 1) {
#pragma unroll
            for (int k = 0; k < NACC; ++k) red[seg][k][lane] = acc[k];
            __syncthreads();
            if (seg == 0) {
#pragma unroll
                for (int k = 0; k < NACC; ++k) {
                    T sum = red[0][k][lane];
#pragma unroll
                    for (int q = 1; q < SPLIT; ++q) sum += red[q][k][lane];
                    acc[k] = sum;
                }
            }
        }
        if (seg == 0) {
            if constexpr (MODE == kFwd) {
                if (active) {
#pragma unroll
                    for (int k = 0; k < KB; ++k)
                        a.Y[(size_t)(k0 + k) * a.sino_stride + (size_t)v * a.B + b] = R.w * acc[k];
                }
            } else {
                // one image per lane in the derivative modes: image k0 of the batch
                const size_t img = (size_t)k0, vb = (size_t)v * a.B + b;
                const T jt = fma(R.dw, acc[0], R.w * acc[1]);
                T jd = T(0);
                if constexpr (OFFS) jd = fma(R.dws, acc[0], R.w * acc[NACC - 1]);
                if constexpr (MODE == kJvp) {
                    if (active) {
                        T out = (T)a.dtheta[img * a.dir_stride + v] * jt;
                        if constexpr (OFFS) out = fma((T)a.ddelta[img * a.dir_stride + v], jd, out);
                        a.Y[img * a.sino_stride + vb] = out;
                    }
                } else if constexpr (MODE == kVjp) {
                    double pt = 0.0, pd = 0.0;
                    if (active) {
                        const T rr = a.R[img * a.r_stride + vb];
                        pt = (double)(rr * jt);
                        if constexpr (OFFS) pd = (double)(rr * jd);
                    }
                    pt = warp_sum(pt);
                    if constexpr (OFFS) pd = warp_sum(pd);
                    if (lane == 0) {
                        double *p = a.partial + img * a.part_stride + ((size_t)v * a.nchunks + chunk) * 4;
                        p[0] = pt;
                        p[1] = pd;
                    }
                } else {  // kGn
                    double pg = 0.0, pj = 0.0, pf = 0.0, pr = 0.0;
                    if (active) {
                        const T hx = R.w * acc[0];
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
        if constexpr (SPLIT > 1) __syncthreads();  // red[] is reused by the next item
    }
}

// Detector coordinate of the point (x, y) for view (c, sn): the bin centre
// s of the ray through it, s = (x c + y sn) / (1 + (y c - x sn) / D).  Fast
// division: the candidate range keeps a margin of 0.05 bins.
__device__ __forceinline__ float fan_s(float x, float y, float c, float sn, float iD)
{
    return __fdividef(x * c + y * sn, 1.0f + (y * c - x * sn) * iD);
}

// YI[k / 8][v][b][k % 8] = Y[k][v][b] for k < nsino
template <typename T>
__global__ void k_fan_sino(const T *__restrict__ Y, T *__restrict__ YI, long long m, int nsino,
                           const int *__restrict__ skip)
{
    if (skip && *skip) return;
    const long long total = (long long)nsino * m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(idx / m);
        const long long e = idx - (long long)k * m;
        YI[((long long)(k >> 3) * m + e) * 8 + (k & 7)] = Y[idx];
    }
}

struct AdjFanArgs {
    const int *fstart, *fcount;
    int N, B, F, tps, Pb, kbase, ngroups;
    long long ysino_stride, img_stride;
    const int *skip;
};

// The KB values of one bin in the interleaved layout (16-byte loads where the
// group is 16-byte aligned: FP32 groups of 4 or 8, FP64 groups of 2 or more).
template <typename T, int KB> __device__ __forceinline__ void load_bin(const T *p, T (&out)[KB])
{
    if constexpr (std::is_same<T, float>::value && KB % 4 == 0) {
#pragma unroll
        for (int q = 0; q < KB / 4; ++q) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(p) + q);
            out[4 * q] = v.x;
            out[4 * q + 1] = v.y;
            out[4 * q + 2] = v.z;
            out[4 * q + 3] = v.w;
        }
    } else if constexpr (std::is_same<T, double>::value && KB % 2 == 0) {
#pragma unroll
        for (int q = 0; q < KB / 2; ++q) {
            const double2 v = __ldg(reinterpret_cast<const double2 *>(p) + q);
            out[2 * q] = v.x;
            out[2 * q + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < KB; ++k) out[k] = __ldg(p + k);
    }
}

// One CTA = one 16 x 16 pixel tile of one frame and KB sinograms, SPLIT
// thread groups of 256: group g of a pixel sums the views vs + g, vs + g +
// SPLIT, ... of its frame in order; the groups' sums are added in group
// order in shared memory.
template <typename T, int KB, int SPLIT>
__global__ void __launch_bounds__(256 * SPLIT) k_adj_fan(AdjFanArgs a, const FanLine<T> *__restrict__ rays,
                                                         const FanView *__restrict__ views,
                                                         const T *__restrict__ YI, T *__restrict__ X)
{
    __shared__ T red[SPLIT > 1 ? SPLIT - 1 : 1][KB][256];
    const int pix = threadIdx.x & 255, grp_v = threadIdx.x >> 8;
    const int tx = pix & (kTile - 1), ty = pix / kTile;
    const int N = a.N;
    const int tiles = a.tps * a.tps;
    const long long total = (long long)a.ngroups * a.F * tiles;
    const float h = 0.5f * (float)(N - 1);
    if (a.skip && *a.skip) return;
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {  // CTA-uniform
        const int tile = (int)(item % tiles);
        const long long t2 = item / tiles;
        const int f = (int)(t2 % a.F);
        const int grp = (int)(t2 / a.F);
        const int i = (tile / a.tps) * kTile + ty, j = (tile % a.tps) * kTile + tx;
        const int k0 = a.kbase + grp * KB;
        const bool inside = i < N && j < N;
        const float x = (float)j - h, y = h - (float)i;
        const long long Qrow = (long long)(2 * i - (N - 1)), Qcol = (long long)(2 * j - (N - 1));
        T acc[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) acc[k] = T(0);
        const int vs = a.fstart[f], vc = a.fcount[f];
        for (int v = vs + grp_v; inside && v < vs + vc; v += SPLIT) {
            const FanView fv = views[v];
            const FanLine<T> *rv = rays + (size_t)v * a.B;
            // the KB sinograms of this group at bin b: KB consecutive values (KB divides 8, and a
            // group starts at a multiple of its width)
            const T *yv = YI + ((size_t)(k0 >> 3) * a.ysino_stride + (size_t)v * a.B) * 8 + (k0 & 7);
            // rays marched along rows that sample row i inside (x - 1, x + 1), then
            // rays marched along columns that sample column j inside (y - 1, y + 1)
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
                const int mlo = fv.mode0 == pass ? 0 : fv.split;
                const int mhi = fv.mode0 == pass ? fv.split : a.B;  // bins [mlo, mhi) march along this axis
                if (mlo >= mhi) continue;
                const float s1 = pass == 0 ? fan_s(x - 1.0f, y, fv.c, fv.sn, fv.iD) : fan_s(x, y - 1.0f, fv.c, fv.sn, fv.iD);
                const float s2 = pass == 0 ? fan_s(x + 1.0f, y, fv.c, fv.sn, fv.iD) : fan_s(x, y + 1.0f, fv.c, fv.sn, fv.iD);
                // margin 0.05 bins: the FP32 detector coordinates are off by < 0.01 bins for N <= 4096
                const int blo = max(mlo, (int)floorf(fminf(s1, s2) - fv.sb0 - 0.05f));
                const int bhi = min(mhi - 1, (int)ceilf(fmaxf(s1, s2) - fv.sb0 + 0.05f));
                const long long Qr = pass == 0 ? Qrow : Qcol;
                const int me = pass == 0 ? j : i;
                for (int b = blo; b <= bhi; ++b) {
                    const long long Q = rv[b].Qc + Qr * rv[b].Qh;
                    const int cell = cell_of(Q);
                    if (cell != me && cell != me - 1) continue;
                    const T fr = frac_of(Q, T());
                    const T wt = rv[b].w * (cell == me ? T(1) - fr : fr);
                    T yk[KB];
                    load_bin<T, KB>(yv + (size_t)b * 8, yk);
#pragma unroll
                    for (int k = 0; k < KB; ++k) acc[k] = fma(wt, yk[k], acc[k]);
                }
            }
        }
        if constexpr (SPLIT > 1) {
            if (grp_v > 0) {
#pragma unroll
                for (int k = 0; k < KB; ++k) red[grp_v - 1][k][pix] = acc[k];
            }
            __syncthreads();
            if (grp_v == 0) {
#pragma unroll
                for (int k = 0; k < KB; ++k)
#pragma unroll
                    for (int q = 0; q < SPLIT - 1; ++q) acc[k] += red[q][k][pix];
            }
        }
        if (grp_v == 0 && inside) {
#pragma unroll
            for (int k = 0; k < KB; ++k)
                X[(size_t)(k0 + k) * a.img_stride + (size_t)f * N * N + (size_t)i * N + j] = acc[k];
        }
        if constexpr (SPLIT > 1) __syncthreads();  // red[] is reused by the next item
    }
}

template <typename T, int MODE, int KB, int SPLIT, bool OFFS = false>
cudaError_t run_fan(const Handle &h, const RayArgs<T> &a)
{
    auto kern = k_ray_fan<T, MODE, KB, SPLIT, OFFS>;
    const long long items = (long long)a.ngroups * a.V * a.nchunks;
    const int grid = persistent_grid(kern, 32 * SPLIT, 0, items, h.num_sms);
    kern<<<grid, 32 * SPLIT, 0, h.stream>>>(a, (const FanRay<T> *)h.d_rays);
    return cudaGetLastError();
}

template <typename T, int MODE, int KB, bool OFFS = false>
cudaError_t run_fan_split(const Handle &h, const RayArgs<T> &a, int split)
{
    switch (split) {
    case 1: return run_fan<T, MODE, KB, 1, OFFS>(h, a);
    case 2: return run_fan<T, MODE, KB, 2, OFFS>(h, a);
    default: return run_fan<T, MODE, KB, 4, OFFS>(h, a);
    }
}

template <typename T, int KB, int SPLIT> cudaError_t run_adj_fan(const Handle &h, const AdjFanArgs &a, T *X)
{
    auto kern = k_adj_fan<T, KB, SPLIT>;
    const long long items = (long long)a.ngroups * a.F * a.tps * a.tps;
    const int grid = persistent_grid(kern, 256 * SPLIT, 0, items, h.num_sms);
    kern<<<grid, 256 * SPLIT, 0, h.stream>>>(a, fan_lines<T>(h.d_rays, (long long)h.V * h.B),
                                             (const FanView *)h.d_fanview, (const T *)h.d_yi, X);
    return cudaGetLastError();
}

template <typename T, int KB> cudaError_t run_adj_fan_split(const Handle &h, const AdjFanArgs &a, T *X, int split)
{
    return split >= 4 ? run_adj_fan<T, KB, 4>(h, a, X)
                      : (split >= 2 ? run_adj_fan<T, KB, 2>(h, a, X) : run_adj_fan<T, KB, 1>(h, a, X));
}

}  // namespace

// bytes a ray takes in the handle's table: its FanRay and its FanLine
size_t fan_ray_bytes(int precision)
{
    return precision ? sizeof(FanRay<double>) + sizeof(FanLine<double>) : sizeof(FanRay<float>) + sizeof(FanLine<float>);
}
size_t fan_view_bytes() { return sizeof(FanView); }

cudaError_t launch_fan_rays(const Handle &h, const int *skip)
{
    const long long n = (long long)h.V * h.B;
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4LL * h.num_sms));
    const int vgrid = (h.V + 7) / 8;
    if (h.precision) {
        k_fan_rays<double><<<grid, 256, 0, h.stream>>>(h.d_views, h.V, h.B, h.N, h.fan_D,
                                                       (FanRay<double> *)h.d_rays, fan_lines<double>(h.d_rays, n),
                                                       skip);
        k_fan_views<double><<<vgrid, 256, 0, h.stream>>>(h.d_views, h.V, h.B, h.fan_D,
                                                         (const FanRay<double> *)h.d_rays, (FanView *)h.d_fanview,
                                                         skip);
    } else {
        k_fan_rays<float><<<grid, 256, 0, h.stream>>>(h.d_views, h.V, h.B, h.N, h.fan_D, (FanRay<float> *)h.d_rays,
                                                      fan_lines<float>(h.d_rays, n), skip);
        k_fan_views<float><<<vgrid, 256, 0, h.stream>>>(h.d_views, h.V, h.B, h.fan_D, (const FanRay<float> *)h.d_rays,
                                                        (FanView *)h.d_fanview, skip);
    }
    return cudaGetLastError();
}

// split: warps per work item (row segments), 1, 2 or 4 (larger values take 4);
// offs: the JVP / VJP also carry the offset derivatives
template <typename T>
cudaError_t run_fan_ray(const Handle &h, const RayArgs<T> &a, int mode, int kb, int split, bool offs)
{
    switch (mode) {
    case kFwd:
        switch (kb) {
        case 1: return run_fan_split<T, kFwd, 1>(h, a, split);
        case 2: return run_fan_split<T, kFwd, 2>(h, a, split);
        case 4: return run_fan_split<T, kFwd, 4>(h, a, split);
        default: return run_fan_split<T, kFwd, 8>(h, a, split);
        }
    case kJvp: return offs ? run_fan_split<T, kJvp, 1, true>(h, a, split) : run_fan_split<T, kJvp, 1>(h, a, split);
    case kVjp: return offs ? run_fan_split<T, kVjp, 1, true>(h, a, split) : run_fan_split<T, kVjp, 1>(h, a, split);
    default: return run_fan_split<T, kGn, 1>(h, a, split);
    }
}

// kb: sinograms per thread (the candidate search of a pixel and view is
// shared by them); split: thread groups per pixel (view subsets).
template <typename T>
cudaError_t launch_fan_adjoint(const Handle &h, T *X, int batch, int kb, int split, const int *skip)
{
    AdjFanArgs a{};
    a.fstart = h.d_fstart;
    a.fcount = h.d_fcount;
    a.N = h.N;
    a.B = h.B;
    a.F = h.F;
    a.tps = (h.N + kTile - 1) / kTile;
    a.Pb = h.Pb;
    a.ysino_stride = (long long)h.V * h.B;  // per block of 8 interleaved sinograms, in bins
    a.img_stride = (long long)h.F * h.N * h.N;
    a.skip = skip;
    int k = 0;
    for (int width : {8, 4, 2, 1}) {
        if (width > kb) continue;
        const int groups = (batch - k) / width;
        if (groups == 0) continue;
        a.kbase = k;
        a.ngroups = groups;
        cudaError_t e;
        switch (width) {
        case 1: e = run_adj_fan_split<T, 1>(h, a, X, split); break;
        case 2: e = run_adj_fan_split<T, 2>(h, a, X, split); break;
        case 4: e = run_adj_fan_split<T, 4>(h, a, X, split); break;
        default: e = run_adj_fan_split<T, 8>(h, a, X, split); break;
        }
        if (e != cudaSuccess) return e;
        k += groups * width;
    }
    return cudaSuccess;
}

template <typename T> cudaError_t launch_fan_sino(const Handle &h, const T *Y, int nsino, const int *skip)
{
    const long long m = (long long)h.V * h.B;
    const long long total = (long long)nsino * m;
    const int grid = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 8LL * h.num_sms));
    k_fan_sino<T><<<grid, 256, 0, h.stream>>>(Y, (T *)h.d_yi, m, nsino, skip);
    return cudaGetLastError();
}

template cudaError_t launch_fan_sino<float>(const Handle &, const float *, int, const int *);
template cudaError_t launch_fan_sino<double>(const Handle &, const double *, int, const int *);
template cudaError_t run_fan_ray<float>(const Handle &, const RayArgs<float> &, int, int, int, bool);
template cudaError_t run_fan_ray<double>(const Handle &, const RayArgs<double> &, int, int, int, bool);
template cudaError_t launch_fan_adjoint<float>(const Handle &, float *, int, int, int, const int *);
template cudaError_t launch_fan_adjoint<double>(const Handle &, double *, int, int, int, const int *);

}  // namespace ctgb
