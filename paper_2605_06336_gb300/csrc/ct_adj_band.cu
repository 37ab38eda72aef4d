// Staged FP32 transpose operator: the sinogram windows a pixel tile reads
// are copied to shared memory, VB views at a time, before the pixels gather
// from them.
//
// A CTA owns one 16 x 16 pixel tile of one frame and KB sinograms of the
// batch.  For view v the tile's bin coordinates beta = beta0 + j*c - i*s
// span at most 15 (|c| + |s|) <= 21.3 bins, so the pairs a tile reads lie in
// a window of W = 32 pairs (one pair of margin below for the FP32 in-tile
// offset, aligned down to an even slot for 16-byte copies).  The per-(view,
// tile) constants of up to kViewCap views are computed first, one thread
// per view (the tile anchor is an FP64 sum, and FP64 issues slowly on this
// part).  While the windows of one block of VB views are read, those of the
// next block stream into the other buffer with cp.async.  A half-warp is one
// tile row, whose 16 pixels read at most 16 consecutive pairs: one
// shared-memory wavefront.
//
// With `segs` CTAs per tile, the CTAs of a tile form one thread-block
// cluster and CTA s takes the views s, s + segs, ... of the frame.  At the
// end of the tile each CTA leaves its partial sums in its shared memory and
// CTA 0 adds the others' through distributed shared memory, in segment
// order, before it writes the pixel: no partial images in global memory and
// no second kernel.  Every pixel sums its views in the same order with the
// same fused multiply-adds as k_adjoint with `segs` view groups, so the
// results are bit-identical to it.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "ct_device.cuh"
#include "ct_internal.cuh"

namespace ctgb {
namespace {

constexpr int kWin = 32;       // staged pairs per (view, sinogram)
constexpr int kViewCap = 128;  // views whose tile constants are staged at a time (a multiple of VB)

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct AdjBandArgs {
    const ViewGeo *vg;
    const int *fstart, *fcount;
    int N, B, F, tps, Pb;
    const float2 *YP;         // pair sinograms, pitch Pb (even)
    long long ysino_stride;   // pairs per batch element (V * Pb)
    int kbase, ngroups;
    float *X;
    long long img_stride;     // F * N * N
    int segs;                 // CTAs per tile (view subsets) = cluster size
    const int *skip;
};

// Per (view, tile) constants.
struct __align__(16) AdjView {
    float c, s, w, frac;  // direction, weight, fractional part of the tile anchor
    float w1;             // 1 - w
    int off;              // slot of in-tile offset m: min(max(m + off, 0), kWin - 1)
    int start;            // first staged pair of the view's window in its sinogram row
    int pad;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

template <int KB, int VB>
__global__ void __launch_bounds__(256) k_adj_band(AdjBandArgs a)
{
    static_assert(kViewCap % VB == 0, "view chunks hold whole blocks");
    extern __shared__ float4 adj_smem[];
    float2 *sbuf = reinterpret_cast<float2 *>(adj_smem);  // [2][VB][KB][kWin]
    __shared__ AdjView s_view[kViewCap];
    constexpr int BUF = VB * KB * kWin;
    const int tid = threadIdx.x;
    const int tx = tid & (kTile - 1), ty = tid / kTile;
    const float fx = (float)tx, fy = (float)ty;
    const int tiles = a.tps * a.tps;
    const int segs = a.segs;
    const int total = a.ngroups * a.F * tiles * segs;
    const int N = a.N;
    if (a.skip && *a.skip) return;
    // The grid is a whole number of clusters and total a multiple of segs, so
    // the CTAs of a cluster take the segments of one tile in every iteration
    // and leave the loop together (the cluster barriers below are uniform).
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int seg = item % segs;  // = rank of the CTA in its cluster
        int t2 = item / segs;
        const int tile = t2 % tiles;
        t2 /= tiles;
        const int f = t2 % a.F;
        const int grp = t2 / a.F;
        const int i0 = (tile / a.tps) * kTile, j0 = (tile % a.tps) * kTile;
        const int k0 = a.kbase + grp * KB;
        const float2 *yp = a.YP + (size_t)k0 * a.ysino_stride;
        const int vs = a.fstart[f], vc = a.fcount[f];
        const int nv = vc > seg ? (vc - seg + segs - 1) / segs : 0;  // this CTA's views: vs + seg + q * segs

        float acc[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) acc[k] = 0.0f;
        for (int cb = 0; cb < nv; cb += kViewCap) {
            const int nc = min(kViewCap, nv - cb);
            const int nblk = (nc + VB - 1) / VB;
            __syncthreads();  // the previous chunk (or item) is done with s_view and both buffers
            for (int q = tid; q < nc; q += blockDim.x) {
                const ViewGeo &g = a.vg[vs + seg + (cb + q) * segs];
                const double bt = g.beta0 + (double)j0 * g.c - (double)i0 * g.s;
                const double fl = floor(bt);
                const int ix = (int)fl;
                const float frac = (float)(bt - fl);
                const float c = (float)g.c, s = (float)g.s;
                // lowest in-tile offset floor, one pair of margin, even slot, inside the row
                const float tmin = frac + fminf(0.0f, 15.0f * c) + fminf(0.0f, -15.0f * s);
                int start = ix + 2 + (int)floorf(tmin) - 1;
                start = min(max(start, 0), a.Pb - kWin) & ~1;
                AdjView av;
                av.c = c;
                av.s = s;
                av.w = GeoT<float>::w(g);
                av.frac = frac;
                av.w1 = 1.0f - av.w;
                av.off = ix + 2 - start;
                av.start = start;
                av.pad = 0;
                s_view[q] = av;
            }
            __syncthreads();

            // Block blk of the chunk: thread t copies its share of the KB windows
            // of view q = t / (256 / VB) of the block.
            auto stage = [&](int blk, int buf) {
                constexpr int TPV = 256 / VB;         // threads per view
                constexpr int UNITS = KB * kWin / 2;  // 16-byte copies per view
                const int q = tid / TPV, r = tid % TPV;
                const int qq = blk * VB + q;
                if (qq >= nc) return;
                const int v = vs + seg + (cb + qq) * segs;
                float2 *dst = sbuf + (size_t)buf * BUF + (size_t)q * KB * kWin;
                const float2 *src = yp + (size_t)v * a.Pb + s_view[qq].start;
                for (int u = r; u < UNITS; u += TPV) {
                    const int k = u / (kWin / 2), c2 = 2 * (u % (kWin / 2));
                    cp_async16(dst + k * kWin + c2, src + (size_t)k * a.ysino_stride + c2);
                }
            };

            stage(0, 0);
            cp_async_commit();
            for (int blk = 0; blk < nblk; ++blk) {
                cp_async_wait0();
                // block blk is visible to every thread, and every thread has finished
                // block blk - 1, whose buffer the next copies overwrite
                __syncthreads();
                if (blk + 1 < nblk) stage(blk + 1, (blk + 1) & 1);
                cp_async_commit();
                const int nq = min(VB, nc - blk * VB);
                const float2 *base = sbuf + (size_t)(blk & 1) * BUF;
                const AdjView *sv = s_view + blk * VB;
#pragma unroll 4
                for (int q = 0; q < nq; ++q) {
                    const AdjView av = sv[q];
                    const float t = fmaf(fx, av.c, fmaf(-fy, av.s, av.frac));
                    int mm;
                    float fr;
                    floor_split(t, mm, fr);
                    const float wv = av.w;
                    const float wa = wv * fmaxf(0.0f, fmaf(-fr, wv, 1.0f));    // bin floor(beta)
                    const float wb = wv * fmaxf(0.0f, fmaf(fr, wv, av.w1));    // bin floor(beta) + 1
                    // Every cell the tile reads lies in the window unless the window
                    // was clamped to an end of the row; there the clamped slot is a
                    // zero padding pair, as is every pair beyond the detector.
                    const int slot = min(max(mm + av.off, 0), kWin - 1);
                    const float2 *sp = base + q * KB * kWin + slot;
#pragma unroll
                    for (int k = 0; k < KB; ++k) {
                        const float2 p = sp[k * kWin];
                        acc[k] = fmaf(wa, p.x, fmaf(wb, p.y, acc[k]));
                    }
                }
            }
            cp_async_wait0();  // the last group is empty
        }
        if (segs > 1) {
            // segment sums of the tile: CTA 0 adds those of CTAs 1..segs-1 in order
            namespace cg = cooperative_groups;
            cg::cluster_group cl = cg::this_cluster();
            float *red = reinterpret_cast<float *>(adj_smem);  // [KB][256], inside the staging buffers
            __syncthreads();  // every warp is done with the staging buffers
#pragma unroll
            for (int k = 0; k < KB; ++k) red[k * 256 + tid] = acc[k];
            cl.sync();
            if (seg == 0) {
                for (int q = 1; q < segs; ++q) {
                    const float *rq = cl.map_shared_rank(red, q);
#pragma unroll
                    for (int k = 0; k < KB; ++k) acc[k] += rq[k * 256 + tid];
                }
            }
            cl.sync();  // the others keep their shared memory until CTA 0 has read it
        }
        const int i = i0 + ty, j = j0 + tx;
        if (seg == 0 && i < N && j < N) {
#pragma unroll
            for (int k = 0; k < KB; ++k) a.X[(size_t)(k0 + k) * a.img_stride + (size_t)f * N * N + (size_t)i * N + j] = acc[k];
        }
    }
}

template <int KB, int VB>
cudaError_t launch_adj_band_kb(const Handle &h, const AdjBandArgs &a)
{
    static_assert(KB * 256 * sizeof(float) <= 2 * VB * KB * kWin * sizeof(float2), "segment sums fit the buffers");
    auto kern = k_adj_band<KB, VB>;
    const size_t smem = (size_t)2 * VB * KB * kWin * sizeof(float2);
    static bool attr_set = false;  // per instantiation; the attribute is idempotent, so a race is harmless
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const long long items = (long long)a.ngroups * a.F * a.tps * a.tps * a.segs;
    int grid = persistent_grid(kern, 256, smem, items, h.num_sms);
    grid -= grid % a.segs;  // whole clusters (items is a multiple of segs, so grid >= segs)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = h.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = a.segs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int VB>
cudaError_t launch_adj_band_vb(const Handle &h, const AdjBandArgs &a, int kb)
{
    switch (kb) {
    case 1: return launch_adj_band_kb<1, VB>(h, a);
    case 2: return launch_adj_band_kb<2, VB>(h, a);
    case 4: return launch_adj_band_kb<4, VB>(h, a);
    default: return launch_adj_band_kb<8, VB>(h, a);
    }
}

}  // namespace

bool adj_band_ok(const Handle &h, int stage, int segs)
{
    return (stage == 8 || stage == 16) && (segs == 1 || segs == 2 || segs == 4) && h.Pb >= kWin && (h.Pb & 1) == 0;
}

cudaError_t launch_adjoint_band(const Handle &h, float *X, int batch, int kb, int segs, int stage, const int *skip)
{
    if (!adj_band_ok(h, stage, segs)) return cudaErrorInvalidValue;
    AdjBandArgs a{};
    a.vg = h.d_views;
    a.fstart = h.d_fstart;
    a.fcount = h.d_fcount;
    a.N = h.N;
    a.B = h.B;
    a.F = h.F;
    a.tps = (h.N + kTile - 1) / kTile;
    a.Pb = h.Pb;
    a.YP = (const float2 *)h.d_yp;
    a.ysino_stride = (long long)h.V * h.Pb;
    a.X = X;
    a.img_stride = (long long)h.F * h.N * h.N;
    a.segs = segs;
    a.skip = skip;
    int k = 0;
    for (int width : {8, 4, 2, 1}) {
        if (width > kb) continue;
        const int groups = (batch - k) / width;
        if (groups == 0) continue;
        a.kbase = k;
        a.ngroups = groups;
        cudaError_t e = stage == 8 ? launch_adj_band_vb<8>(h, a, width) : launch_adj_band_vb<16>(h, a, width);
        if (e != cudaSuccess) return e;
        k += groups * width;
    }
    return cudaGetLastError();
}

}  // namespace ctgb
