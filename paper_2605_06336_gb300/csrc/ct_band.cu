// Band-staged FP32 ray march: the image rows a CTA's rays cross are copied to
// shared memory block by block, and the interpolation taps are read there.
//
// A CTA owns VW consecutive views of the sorted view order (one warp each,
// all on the same 32-bin chunk) and walks the union of their row ranges in
// blocks of RB rows.  For each block the columns its rays can touch form a
// band, found from the four corners (first/last bin, first/last row) of each
// view's part of the block: the fixed-point line is affine in the bin and
// the row, so its cell is monotone in each.  While block j is computed, the
// band of block j+1 streams into another of NS buffers with cp.async
// (16-byte copies when the pair pitch is even, 8-byte otherwise).  All KB
// images of a batch group sit at a compile-time stride in the buffer, so an
// image costs one shared load with an immediate offset, and the VW views
// reuse every staged pair.
//
// A block whose band is wider than kBandMax pairs is marched from the global
// pair images instead, and so is a whole item whose views do not share one
// frame and one marching axis.  Either way each ray is summed row by row in
// increasing row order with the same fused multiply-adds as k_ray with one
// row segment, so the results are bit-identical to it.
#include <cuda_runtime.h>

#include <algorithm>

#include "ct_device.cuh"
#include "ct_internal.cuh"

namespace ctgb {
namespace {

constexpr int kBandMax = 96;    // staged pairs per row
constexpr int kMaxBlocks = 1040;  // row blocks of one item: N / RB + 1 <= 1025 for N <= 4096, RB >= 4

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

template <int MODE, bool OFFS, int KB, int VW, int RB, int NS>
__global__ void __launch_bounds__(32 * VW) k_ray_band(RayArgs<float> a)
{
    constexpr int IMG = RB * kBandMax;  // pairs per image in one buffer
    constexpr int NACC = (MODE == kFwd) ? KB : 3;
    constexpr int NT = 32 * VW;
    extern __shared__ float4 band_smem[];
    float2 *sbuf = reinterpret_cast<float2 *>(band_smem);  // [NS][KB][RB][kBandMax]
    __shared__ int2 s_band[kMaxBlocks];  // (first staged pair slot, staged width); width 0: march from global
    __shared__ long long s_Qc[VW], s_Qb[VW], s_Qh[VW];
    __shared__ int s_lo[VW], s_hi[VW], s_n0[VW], s_key[VW];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int N = a.N;
    const int pp = a.Pp;
    const int ngv = (a.V + VW - 1) / VW;
    const int segs = MODE == kFwd ? a.segs : 1;
    const int total = a.ngroups * ngv * a.nchunks * segs;
    if (a.skip && *a.skip) return;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int chunk = item % a.nchunks;
        int t = item / a.nchunks;
        const int seg = t % segs;
        t /= segs;
        const int vgi = t % ngv;
        const int grp = t / ngv;
        const int pos = vgi * VW + warp;
        const int v = pos < a.V ? (a.order ? a.order[pos] : pos) : -1;
        const bool live = v >= 0 && !(MODE == kGn && a.view_mask && a.view_mask[v] == 0);  // warp-uniform
        const ViewGeo &g = a.vg[live ? v : 0];
        const int b = chunk * kChunk + lane;
        const bool active = live && b < a.B;
        const int k0 = a.kbase + grp * KB;
        int rlo = N, rhi = -1;
        if (live) warp_rows(g, b, b < a.B, N, rlo, rhi);
        if (segs > 1 && rlo <= rhi) {  // this CTA's segment of the rays, split as k_ray splits among warps
            const int per = (rhi - rlo + segs) / segs;
            const int r0 = rlo + seg * per;
            rhi = min(rhi, r0 + per - 1);
            rlo = r0;
        }

        __syncthreads();  // every warp is done with the previous item's tables and buffers
        if (lane == 0) {
            s_lo[warp] = rlo;
            s_hi[warp] = rhi;
            s_key[warp] = (live && rlo <= rhi) ? 2 * g.frame + g.mode : -1;
            s_Qc[warp] = g.Qc;
            s_Qb[warp] = g.Qb;
            s_Qh[warp] = g.Qh;
            s_n0[warp] = g.n0;
        }
        __syncthreads();
        // CTA-uniform: the union of the row ranges, and whether one frame and axis serve every view
        int R0 = N, R1 = -1, key0 = -1;
        bool uniform = true;
#pragma unroll 1
        for (int w = 0; w < VW; ++w) {
            const int kw = s_key[w];
            if (kw < 0) continue;
            R0 = min(R0, s_lo[w]);
            R1 = max(R1, s_hi[w]);
            if (key0 < 0) key0 = kw;
            else if (kw != key0) uniform = false;
        }
        const int nblk = R1 >= R0 ? (R1 - R0 + RB) / RB : 0;
        const bool staged = uniform && nblk > 0 && nblk <= kMaxBlocks;

        float acc[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) acc[k] = 0.0f;
        const long long dQ = 2 * g.Qh;
        float g0 = 0.0f, gr = 0.0f;
        if constexpr (MODE != kFwd) {
            g0 = fmaf(GeoT<float>::sb(g, b), GeoT<float>::gs(g), GeoT<float>::gh(g, N));
            gr = GeoT<float>::gr(g);
        }
        const float2 *gimg = (g.mode ? a.PT : a.PX) + (size_t)g.frame * N * pp + (size_t)k0 * a.pimg_stride + 2;

        // The warp's rows rlo..rhi are visited once each, in increasing order,
        // so the line position and the row index run on across row blocks.
        long long Q = line_at(g, b, rlo, N);
        float rf = (float)rlo;
        // one row from the global pair images (row = pair row of the current r, slot of cell 0)
        auto step_global = [&](const float2 *row) {
            const int cell = min(max(cell_of(Q), -2), N);
            const float f = frac_of(Q, 0.0f);
            if constexpr (MODE == kFwd) {
                const float omf = 1.0f - f;
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    const float2 p = __ldg(row + (size_t)k * a.pimg_stride + cell);
                    acc[k] = fmaf(omf, p.x, fmaf(f, p.y, acc[k]));
                }
            } else {
                const float2 p = __ldg(row + cell);
                const float d = p.y - p.x;
                acc[0] += fmaf(f, d, p.x);
                acc[1] = fmaf(d, fmaf(rf, gr, g0), acc[1]);
                if (OFFS) acc[2] += d;
            }
            Q += dQ;
            rf += 1.0f;
        };
        // one row from a staged block: srow = buffer row, off = 2 - first staged slot, wm1 = width - 1.
        // Cells inside [-2, N] lie in the band.  A cell below -2 (above N) only
        // occurs when a corner was clamped to -2 (N), so the band starts at slot 0
        // (ends at slot N+2 or N+3) and the clamped index reads the same zero pair
        // as the clamped cell of k_ray.
        auto step_shared = [&](const float2 *srow, int off, int wm1) {
            const int idx = min(max(cell_of(Q) + off, 0), wm1);
            const float f = frac_of(Q, 0.0f);
            const float2 *sp = srow + idx;
            if constexpr (MODE == kFwd) {
                const float omf = 1.0f - f;
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    const float2 p = sp[k * IMG];
                    acc[k] = fmaf(omf, p.x, fmaf(f, p.y, acc[k]));
                }
            } else {
                const float2 p = sp[0];
                const float d = p.y - p.x;
                acc[0] += fmaf(f, d, p.x);
                acc[1] = fmaf(d, fmaf(rf, gr, g0), acc[1]);
                if (OFFS) acc[2] += d;
            }
            Q += dQ;
            rf += 1.0f;
        };

        if (!staged) {
            for (int r = rlo; r <= rhi; ++r) step_global(gimg + (size_t)r * pp);
        } else {
            // bands of all row blocks of the item
            const int bb0 = chunk * kChunk, bb1 = chunk * kChunk + kChunk - 1;  // every lane, active or not
            for (int blk = threadIdx.x; blk < nblk; blk += NT) {
                const int ra = R0 + blk * RB, rb = min(ra + RB - 1, R1);
                int cmin = N + 1, cmax = -3;
#pragma unroll 1
                for (int w = 0; w < VW; ++w) {
                    if (s_key[w] < 0) continue;
                    const int r_a = max(ra, s_lo[w]), r_b = min(rb, s_hi[w]);
                    if (r_a > r_b) continue;
#pragma unroll 1
                    for (int e = 0; e < 4; ++e) {
                        const int bb = (e & 1) ? bb1 : bb0;
                        const int rr = (e & 2) ? r_b : r_a;
                        const long long Qe = s_Qc[w] + (long long)(bb + s_n0[w]) * s_Qb[w] +
                                             (long long)(2 * rr - (N - 1)) * s_Qh[w];
                        const int c = min(max(cell_of(Qe), -2), N);
                        cmin = min(cmin, c);
                        cmax = max(cmax, c);
                    }
                }
                int2 bd = make_int2(0, 0);
                if (cmin <= cmax) {
                    const int s0 = (cmin + 2) & ~1;                    // even: 16-byte aligned copies
                    const int width = ((cmax + 2 - s0 + 1) + 1) & ~1;  // pairs s0 .. s0 + width - 1 <= N + 3
                    if (width <= kBandMax) bd = make_int2(s0, width);
                }
                s_band[blk] = bd;
            }
            __syncthreads();
            const int frame0 = key0 >> 1, mode0 = key0 & 1;
            const float2 *base = (mode0 ? a.PT : a.PX) + (size_t)frame0 * N * pp + (size_t)k0 * a.pimg_stride;
            // copy the band of block blk into buffer buf: warp w takes rows w, w + VW, ...
            auto stage = [&](int blk, int buf) {
                const int2 bd = s_band[blk];
                if (bd.y == 0) return;  // CTA-uniform
                const int ra = R0 + blk * RB;
                const int nrow = min(RB, R1 - ra + 1);
                float2 *dst = sbuf + (size_t)buf * KB * IMG;
                for (int rr = warp; rr < nrow; rr += VW) {
                    const float2 *src = base + (size_t)(ra + rr) * pp + bd.x;
                    float2 *d = dst + rr * kBandMax;
                    if ((pp & 1) == 0) {
                        for (int c2 = 2 * lane; c2 < bd.y; c2 += 64) {
#pragma unroll
                            for (int k = 0; k < KB; ++k)
                                cp_async16(d + k * IMG + c2, src + (size_t)k * a.pimg_stride + c2);
                        }
                    } else {
                        for (int c = lane; c < bd.y; c += 32) {
#pragma unroll
                            for (int k = 0; k < KB; ++k) cp_async8(d + k * IMG + c, src + (size_t)k * a.pimg_stride + c);
                        }
                    }
                }
            };
#pragma unroll
            for (int st = 0; st < NS - 1; ++st) {
                if (st < nblk) stage(st, st);
                cp_async_commit();
            }
            for (int blk = 0; blk < nblk; ++blk) {
                cp_async_wait<NS - 2>();
                // block blk is visible to every thread, and every warp has finished
                // block blk - 1, whose buffer the next copies overwrite
                __syncthreads();
                if (blk + NS - 1 < nblk) stage(blk + NS - 1, (blk + NS - 1) % NS);
                cp_async_commit();
                const int ra = R0 + blk * RB, rb = min(ra + RB - 1, R1);
                const int r_a = max(ra, rlo), r_b = min(rb, rhi);
                if (r_a <= r_b) {  // warp-uniform
                    const int2 bd = s_band[blk];
                    if (bd.y > 0) {
                        const float2 *srow = sbuf + (size_t)(blk % NS) * KB * IMG + (r_a - ra) * kBandMax;
                        const int off = 2 - bd.x, wm1 = bd.y - 1;
                        if (r_b - r_a + 1 == RB) {
#pragma unroll
                            for (int i = 0; i < RB; ++i) step_shared(srow + i * kBandMax, off, wm1);
                        } else {
                            for (int r = r_a; r <= r_b; ++r, srow += kBandMax) step_shared(srow, off, wm1);
                        }
                    } else {
                        for (int r = r_a; r <= r_b; ++r) step_global(gimg + (size_t)r * pp);
                    }
                }
            }
            cp_async_wait<0>();  // the last groups are empty; nothing is left in flight
        }
        if (MODE == kFwd && segs > 1) {
            // unscaled segment sums; the combine kernel adds them in segment order and applies w
            if (active) {
                float *dst = seg == 0 ? a.Y : a.fpart + (size_t)(seg - 1) * a.fpart_stride;
#pragma unroll
                for (int k = 0; k < NACC; ++k) dst[(size_t)(k0 + k) * a.sino_stride + (size_t)v * a.B + b] = acc[k];
            }
        } else if (live) {
            ray_epilogue<float, MODE, OFFS, KB>(a, g, v, b, active, k0, chunk, lane, acc);
        }
    }
}

__global__ void k_fwd_combine(const ViewGeo *__restrict__ vg, float *__restrict__ Y, const float *__restrict__ P,
                              int segs, long long stride, int V, int B, long long total, const int *__restrict__ skip)
{
    if (skip && *skip) return;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int v = (int)((e / B) % V);
        float s = Y[e];
        for (int q = 1; q < segs; ++q) s += P[(q - 1) * stride + e];
        Y[e] = vg[v].w * s;
    }
}

template <int MODE, bool OFFS, int KB, int VW, int RB, int NS>
cudaError_t launch_band(const Handle &h, const RayArgs<float> &a)
{
    auto kern = k_ray_band<MODE, OFFS, KB, VW, RB, NS>;
    const size_t smem = (size_t)NS * KB * RB * kBandMax * sizeof(float2);
    static bool attr_set = false;  // per instantiation; the attribute is idempotent, so a race is harmless
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const long long items = (long long)a.ngroups * ((a.V + VW - 1) / VW) * a.nchunks * (MODE == kFwd ? a.segs : 1);
    const int grid = persistent_grid(kern, 32 * VW, smem, items, h.num_sms);
    kern<<<grid, 32 * VW, smem, h.stream>>>(a);
    return cudaGetLastError();
}

// Two buffers: the copies for block j+1 fly while block j is computed.
// Measured on the 256^2 / 180-view and 512^2 / 360-view workloads, a third
// buffer did not pay for the shared memory it takes from occupancy.
template <int MODE, bool OFFS, int KB, int VW, int RB>
cudaError_t band_ns(const Handle &h, const RayArgs<float> &a)
{
    return launch_band<MODE, OFFS, KB, VW, RB, 2>(h, a);
}

template <int MODE, bool OFFS, int KB>
cudaError_t band_vw_rb(const Handle &h, const RayArgs<float> &a, int rb)
{
    if (a.VW == 4) return rb == 4 ? band_ns<MODE, OFFS, KB, 4, 4>(h, a) : band_ns<MODE, OFFS, KB, 4, 8>(h, a);
    return rb == 4 ? band_ns<MODE, OFFS, KB, 8, 4>(h, a) : band_ns<MODE, OFFS, KB, 8, 8>(h, a);
}

}  // namespace

cudaError_t launch_fwd_combine(const Handle &h, float *Y, const float *P, int segs, long long stride, int batch,
                               const int *skip)
{
    const long long total = (long long)batch * h.V * h.B;
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = std::min<long long>((total + threads - 1) / threads, (long long)h.num_sms * 8);
    k_fwd_combine<<<(int)blocks, threads, 0, h.stream>>>(h.d_views, Y, P, segs, stride, h.V, h.B, total, skip);
    return cudaGetLastError();
}

bool band_shape_ok(int mode, int kb, int vw, int rb)
{
    const bool kb_ok = mode == kFwd ? (kb == 1 || kb == 2 || kb == 4 || kb == 8) : kb == 1;
    return kb_ok && (vw == 4 || vw == 8) && (rb == 4 || rb == 8);
}

cudaError_t run_ray_band(const Handle &h, const RayArgs<float> &a, int mode, bool offs, int kb, int rb)
{
    if (!band_shape_ok(mode, kb, a.VW, rb)) return cudaErrorInvalidValue;
    switch (mode) {
    case kFwd:
        switch (kb) {
        case 1: return band_vw_rb<kFwd, false, 1>(h, a, rb);
        case 2: return band_vw_rb<kFwd, false, 2>(h, a, rb);
        case 4: return band_vw_rb<kFwd, false, 4>(h, a, rb);
        default: return band_vw_rb<kFwd, false, 8>(h, a, rb);
        }
    case kJvp: return offs ? band_vw_rb<kJvp, true, 1>(h, a, rb) : band_vw_rb<kJvp, false, 1>(h, a, rb);
    case kVjp: return offs ? band_vw_rb<kVjp, true, 1>(h, a, rb) : band_vw_rb<kVjp, false, 1>(h, a, rb);
    default: return band_vw_rb<kGn, false, 1>(h, a, rb);
    }
}

}  // namespace ctgb
