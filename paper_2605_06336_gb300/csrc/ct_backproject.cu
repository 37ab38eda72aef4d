// Transpose operator X = H(theta)^T Y in gather form (sm_103a).
//
// One thread per pixel of a 16 x 16 tile, SPLIT thread groups per tile
// (each group a subset of the frame's views, combined in shared memory in a
// fixed order), KB sinograms per thread.  No atomics: every output pixel is
// written once by one thread.
//
// For pixel (i, j) and view v the continuous bin coordinate of the pixel
// centre is beta = beta0 + j*c - i*s.  The rays that sampled the pixel in
// the forward rule are the bins b with |b - beta| < 1/w, and the forward
// interpolation gave each of them the weight w * (1 - |b - beta| * w) -- at
// most two bins, floor(beta) and floor(beta) + 1, read as one sinogram pair.
// beta is split into an FP64 tile anchor (integer + fraction, once per tile
// and view) plus a small FP32 in-tile offset.  This is the residual step
// H^T (H u - b) of every MM-GKS iteration (Eq. (3.6), Alg. "Enlarge").
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "ct_device.cuh"
#include "ct_internal.cuh"

namespace ctgb {
namespace {

constexpr int kViewChunk = 256;  // per-view tile constants staged at a time

struct __align__(16) DoubleQuad {
    double x, y, z, w;
};
template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = DoubleQuad; };

template <typename T> struct AdjArgs {
    const ViewGeo *vg;
    const int *fstart, *fcount;
    int N, B, F, tps, Pb;
    const pair_t<T> *YP;
    long long ysino_stride;  // pairs per batch element (V * Pb)
    int kbase, ngroups;
    T *X;
    long long img_stride;    // F * N * N
    const int *skip;         // whole launch is a no-op when *skip != 0 (nullable)
};

template <typename T, int KB, int SPLIT>
__global__ void __launch_bounds__(256 * SPLIT) k_adjoint(AdjArgs<T> a)
{
    using V4 = typename Vec4<T>::type;
    using P2 = pair_t<T>;
    __shared__ V4 s_geo[kViewChunk];   // (c, s, w, fractional anchor)
    __shared__ int2 s_idx[kViewChunk]; // (integer anchor, view * Pb)
    __shared__ T red[SPLIT > 1 ? SPLIT - 1 : 1][256];
    const int tid = threadIdx.x & 255;
    const int grpv = threadIdx.x >> 8;
    const int tx = tid & (kTile - 1), ty = tid / kTile;
    const T fx = (T)tx, fy = (T)ty;
    const int tiles = a.tps * a.tps;
    const int total = a.ngroups * a.F * tiles;
    const int N = a.N;
    if (a.skip && *a.skip) return;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int tile = item % tiles;
        const int t2 = item / tiles;
        const int f = t2 % a.F;
        const int grp = t2 / a.F;
        const int i0 = (tile / a.tps) * kTile, j0 = (tile % a.tps) * kTile;
        const int k0 = a.kbase + grp * KB;
        T acc[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) acc[k] = T(0);
        const P2 *yp = a.YP + (size_t)k0 * a.ysino_stride;
        const int vs = a.fstart[f], vc = a.fcount[f];
        for (int base = 0; base < vc; base += kViewChunk) {
            const int nv = min(kViewChunk, vc - base);
            __syncthreads();
            for (int q = threadIdx.x; q < nv; q += blockDim.x) {
                const int v = vs + base + q;
                const ViewGeo &g = a.vg[v];
                const double bt = g.beta0 + (double)j0 * g.c - (double)i0 * g.s;
                const double fl = floor(bt);
                V4 gv;
                gv.x = (T)g.c;
                gv.y = (T)g.s;
                gv.z = GeoT<T>::w(g);
                gv.w = (T)(bt - fl);
                s_geo[q] = gv;
                s_idx[q] = make_int2((int)fl, v * a.Pb);
            }
            __syncthreads();
            // Views in blocks of U: the U*KB sinogram pairs of a block are loaded
            // before any is used (memory-level parallelism for the gathers).
            constexpr int U = KB >= 4 ? 2 : 4;
            int q = grpv;
            for (; q + (U - 1) * SPLIT < nv; q += U * SPLIT) {
                T wa[U], wb[U];
                P2 p[U][KB];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const V4 gv = s_geo[q + u * SPLIT];
                    const int2 ix = s_idx[q + u * SPLIT];
                    const T t = fma(fx, gv.x, fma(-fy, gv.y, gv.w));
                    int mm;
                    T fr;
                    floor_split(t, mm, fr);
                    const T wv = gv.z;
                    wa[u] = wv * fmax(T(0), fma(-fr, wv, T(1)));      // bin floor(beta)
                    wb[u] = wv * fmax(T(0), fma(fr, wv, T(1) - wv));  // bin floor(beta) + 1
                    const P2 *row = yp + ix.y + (min(max(ix.x + mm, -2), a.B) + 2);
#pragma unroll
                    for (int k = 0; k < KB; ++k) p[u][k] = __ldg(row + (size_t)k * a.ysino_stride);
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int k = 0; k < KB; ++k) acc[k] = fma(wa[u], p[u][k].x, fma(wb[u], p[u][k].y, acc[k]));
            }
            for (; q < nv; q += SPLIT) {
                const V4 gv = s_geo[q];
                const int2 ix = s_idx[q];
                const T t = fma(fx, gv.x, fma(-fy, gv.y, gv.w));
                int mm;
                T fr;
                floor_split(t, mm, fr);
                const T wv = gv.z;
                const T w0 = wv * fmax(T(0), fma(-fr, wv, T(1)));
                const T w1 = wv * fmax(T(0), fma(fr, wv, T(1) - wv));
                const P2 *row = yp + ix.y + (min(max(ix.x + mm, -2), a.B) + 2);
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    const P2 pk = __ldg(row + (size_t)k * a.ysino_stride);
                    acc[k] = fma(w0, pk.x, fma(w1, pk.y, acc[k]));
                }
            }
        }
        if constexpr (SPLIT > 1) {  // combine the view groups, one image at a time
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                if (grpv > 0) red[grpv - 1][tid] = acc[k];
                __syncthreads();
                if (grpv == 0) {
#pragma unroll
                    for (int q = 0; q < SPLIT - 1; ++q) acc[k] += red[q][tid];
                }
                __syncthreads();
            }
        }
        const int i = i0 + ty, j = j0 + tx;
        if (grpv == 0 && i < N && j < N) {
#pragma unroll
            for (int k = 0; k < KB; ++k)
                a.X[(size_t)(k0 + k) * a.img_stride + (size_t)f * N * N + (size_t)i * N + j] = acc[k];
        }
    }
}

template <typename T, int KB, int SPLIT>
cudaError_t run_adj(const Handle &h, const AdjArgs<T> &a)
{
    auto kern = k_adjoint<T, KB, SPLIT>;
    const long long items = (long long)a.ngroups * a.F * a.tps * a.tps;
    const int grid = persistent_grid(kern, 256 * SPLIT, 0, items, h.num_sms);
    kern<<<grid, 256 * SPLIT, 0, h.stream>>>(a);
    return cudaGetLastError();
}

template <typename T, int KB>
cudaError_t run_adj_split(const Handle &h, const AdjArgs<T> &a, int split)
{
    switch (split) {
    case 1: return run_adj<T, KB, 1>(h, a);
    case 2: return run_adj<T, KB, 2>(h, a);
    default: return run_adj<T, KB, 4>(h, a);
    }
}

}  // namespace

template <typename T>
cudaError_t launch_adjoint(const Handle &h, T *X, int batch, int kb, int split, int stage, const int *skip)
{
    if (h.fan_D > 0.0) return launch_fan_adjoint<T>(h, X, batch, kb, split, skip);
    if constexpr (std::is_same<T, float>::value) {
        if (stage > 0 && adj_band_ok(h, stage, split)) return launch_adjoint_band(h, X, batch, kb, split, stage, skip);
    }
    AdjArgs<T> a{};
    a.skip = skip;
    a.vg = h.d_views;
    a.fstart = h.d_fstart;
    a.fcount = h.d_fcount;
    a.N = h.N;
    a.B = h.B;
    a.F = h.F;
    a.tps = (h.N + kTile - 1) / kTile;
    a.Pb = h.Pb;
    a.YP = (const pair_t<T> *)h.d_yp;
    a.ysino_stride = (long long)h.V * h.Pb;
    a.X = X;
    a.img_stride = (long long)h.F * h.N * h.N;
    int k = 0;
    for (int width : {8, 4, 2, 1}) {
        if (width > kb) continue;
        const int groups = (batch - k) / width;
        if (groups == 0) continue;
        a.kbase = k;
        a.ngroups = groups;
        cudaError_t e;
        switch (width) {
        case 1: e = run_adj_split<T, 1>(h, a, split); break;
        case 2: e = run_adj_split<T, 2>(h, a, split); break;
        case 4: e = run_adj_split<T, 4>(h, a, split); break;
        default: e = run_adj_split<T, 8>(h, a, split); break;
        }
        if (e != cudaSuccess) return e;
        k += groups * width;
    }
    return cudaSuccess;
}

template cudaError_t launch_adjoint<float>(const Handle &, float *, int, int, int, int, const int *);
template cudaError_t launch_adjoint<double>(const Handle &, double *, int, int, int, int, const int *);

}  // namespace ctgb
