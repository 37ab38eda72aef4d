// Device kernels of the NL-RMM-GKS driver (included by ct_solver.cu only).
//
// Vectors of the image space have n = F*N*N entries, of the data space
// m = V*B entries; a basis V (and H V) is stored column by column, each column
// contiguous, in the working precision T.  Small matrices (k <= kKMax) are
// FP64.  Every kernel that belongs to a predicated Enlarge step takes the
// device flag `stop` and returns at once when it is set, so a fixed launch
// sequence can run without host round trips.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <algorithm>

#include <cmath>

#include "ct_device.cuh"

namespace ctgb {
namespace solver {

constexpr int kKMax = 128;      // leading dimension of the k x k FP64 matrices in device memory
constexpr int kKSmem = 64;      // bases of up to this many columns keep the FP64 small algebra in shared memory
constexpr int kKLimit = 122;    // largest basis (columns): the register-blocked Gram's 4 x 4 block pairs fit 512 threads
constexpr int kRedBlocks = 608;  // largest partial-sum grid of the tall-skinny reductions (4 CTAs per SM of a GB300)
// Partial-sum grid for vectors of length len: 128 CTAs up to half a million
// elements, growing to kRedBlocks for the long image vectors (a fixed function
// of the length, so the summation order is fixed too).
inline int red_blocks(long long len)
{
    return (int)std::min<long long>(kRedBlocks, std::max<long long>(128, len / 4096));
}

// control words (int) and scalars (double) living on the device
enum Ctl { kStop = 0, kStopNext, kSteps, kActive, kBreakdown, kViewChanged, kArmijoDone, kCtlCount };
enum Scal { kLam = 0, kRnorm2, kDu2, kU2, kJreg, kBnorm2, kTmp0, kTmp1, kScalCount };

__device__ __forceinline__ bool stopped(const int *stop) { return stop && *stop; }

template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return 1.0f / sqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }

// ---------------------------------------------------------------------------
// block reductions (deterministic)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
        sh[32] = s;
    }
    __syncthreads();
    return sh[32];
}

// ---------------------------------------------------------------------------
// MM weights P^2 = (z^2 + eps^2)^(-1/2), z = Psi u (forward differences)
// edge layout: [F][N][N-1] horizontal, then [F][N-1][N] vertical, then (with
// temporal: the ANISO-TV operator D_1) [F-1][N][N] frame f+1 minus frame f
// ---------------------------------------------------------------------------
inline long long psi_edges(int N, int F, int temporal)
{
    return 2LL * F * N * (N - 1) + (temporal && F > 1 ? (long long)(F - 1) * N * N : 0);
}

template <typename T>
__global__ void k_weights(const T *__restrict__ u, T *__restrict__ w, int N, int F, int temporal, double eps,
                          const int *stop)
{
    if (stopped(stop)) return;
    const long long nx = (long long)F * N * (N - 1);
    const long long ne = 2 * nx + (temporal && F > 1 ? (long long)(F - 1) * N * N : 0);
    const T e2 = (T)(eps * eps);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
        T z;
        if (e < nx) {
            const long long f = e / ((long long)N * (N - 1));
            const long long rem = e - f * N * (N - 1);
            const int i = (int)(rem / (N - 1)), j = (int)(rem % (N - 1));
            const T *uf = u + f * N * N;
            z = uf[(size_t)i * N + j + 1] - uf[(size_t)i * N + j];
        } else if (e < 2 * nx) {
            const long long e2i = e - nx;
            const long long f = e2i / ((long long)(N - 1) * N);
            const long long rem = e2i - f * (N - 1) * N;
            const int i = (int)(rem / N), j = (int)(rem % N);
            const T *uf = u + f * N * N;
            z = uf[(size_t)(i + 1) * N + j] - uf[(size_t)i * N + j];
        } else {
            const long long et = e - 2 * nx;  // = f * N * N + pixel
            z = u[et + (long long)N * N] - u[et];
        }
        w[e] = rsqrt_t<T>(z * z + e2);
    }
}

// r += lambda Psi^T P^2 Psi u  (lambda = scal[kLam])
template <typename T>
__global__ void k_add_reg(T *__restrict__ r, const T *__restrict__ u, const T *__restrict__ w,
                          const double *__restrict__ scal, int N, int F, int temporal, const int *stop)
{
    if (stopped(stop)) return;
    const long long n = (long long)F * N * N;
    const long long nx = (long long)F * N * (N - 1);
    const T lam = (T)scal[kLam];
    const bool tm = temporal && F > 1;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const long long f = p / ((long long)N * N);
        const int rem = (int)(p - f * N * N);
        const int i = rem / N, j = rem % N;
        const T *uf = u + f * N * N;
        const T *wx = w + f * N * (N - 1);
        const T *wy = w + nx + f * (N - 1) * N;
        const T c = uf[rem];
        T acc = T(0);
        if (j < N - 1) acc -= wx[i * (N - 1) + j] * (uf[rem + 1] - c);      // edge (i,j)-(i,j+1)
        if (j > 0) acc += wx[i * (N - 1) + j - 1] * (c - uf[rem - 1]);      // edge (i,j-1)-(i,j)
        if (i < N - 1) acc -= wy[i * N + j] * (uf[rem + N] - c);            // edge (i,j)-(i+1,j)
        if (i > 0) acc += wy[(i - 1) * N + j] * (c - uf[rem - N]);          // edge (i-1,j)-(i,j)
        if (tm) {
            const T *wt = w + 2 * nx;                                       // [F-1][N*N]
            const long long nn = (long long)N * N;
            if (f < F - 1) acc -= wt[f * nn + rem] * (u[p + nn] - c);      // frame f -> f+1
            if (f > 0) acc += wt[(f - 1) * nn + rem] * (c - u[p - nn]);    // frame f-1 -> f
        }
        r[p] += lam * acc;
    }
}

// ---------------------------------------------------------------------------
// weighted Gram of Psi V:  G[a][b] = sum_e w_e (Psi v_a)_e (Psi v_b)_e,
// a <= b < k.  A fixed grid of CTAs walks the tiles (TR x 32 pixels of one
// frame) in a fixed order; for each tile the edges (right and down
// neighbour of every pixel) of all k columns are formed in shared memory,
// each thread sums its (a, b) entries over the tile's edges in T and adds the
// tile sum to an FP64 register accumulator.  Per-CTA FP64 partials;
// k_gram_reduce sums them in order.
// ---------------------------------------------------------------------------
constexpr int kGramPairs = kKMax * (kKMax + 1) / 2;
// register slots per thread of k_gram_psi: (pairs of a basis of kc columns) / 256
constexpr int gram_slots(int kc) { return (kc * (kc + 1) / 2 + 255) / 256; }

template <typename T, int TR, int kGramSlots>
__global__ void __launch_bounds__(256) k_gram_psi(const T *__restrict__ V, long long n, int k,
                                                  const T *__restrict__ w, int N, int F, int temporal,
                                                  double *__restrict__ part, const int *stop)
{
    if (stopped(stop)) return;
    extern __shared__ unsigned char smem_raw[];
    constexpr int TP = TR * 32;                  // pixels per tile
    const int EPP = (temporal && F > 1) ? 3 : 2;  // edges per pixel: right, down (, next frame)
    const int EP = EPP * TP + 1;                 // padded edge pitch (conflict-free column reads)
    T *E = reinterpret_cast<T *>(smem_raw);      // [k][EP]
    const int tiles_x = (N + 31) / 32, tiles_y = (N + TR - 1) / TR;
    const int ntiles = tiles_x * tiles_y * F;
    const long long nx = (long long)F * N * (N - 1);
    const int np = k * (k + 1) / 2;
    double acc[kGramSlots];
#pragma unroll
    for (int q = 0; q < kGramSlots; ++q) acc[q] = 0.0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tile = t % (tiles_x * tiles_y);
        const int f = t / (tiles_x * tiles_y);
        const int i0 = (tile / tiles_x) * TR, j0 = (tile % tiles_x) * 32;
        const T *wx = w + (long long)f * N * (N - 1);
        const T *wy = w + nx + (long long)f * (N - 1) * N;
        const T *wt = w + 2 * nx + (long long)f * N * N;  // temporal edges of frames (f, f + 1)
        __syncthreads();
        for (int idx = threadIdx.x; idx < k * TP; idx += blockDim.x) {
            const int a = idx / TP, pix = idx % TP;
            const int i = i0 + pix / 32, j = j0 + pix % 32;
            T ex = T(0), ey = T(0), et = T(0);
            if (i < N && j < N) {
                const T *va = V + (long long)a * n + (long long)f * N * N;
                const T c = va[(size_t)i * N + j];
                if (j < N - 1) ex = (va[(size_t)i * N + j + 1] - c) * sqrt(wx[i * (N - 1) + j]);
                if (i < N - 1) ey = (va[(size_t)(i + 1) * N + j] - c) * sqrt(wy[i * N + j]);
                if (EPP == 3 && f < F - 1)
                    et = (va[(size_t)N * N + (size_t)i * N + j] - c) * sqrt(wt[(size_t)i * N + j]);
            }
            E[a * EP + EPP * pix] = ex;
            E[a * EP + EPP * pix + 1] = ey;
            if (EPP == 3) E[a * EP + EPP * pix + 2] = et;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kGramSlots; ++q) {
            const int p = threadIdx.x + 256 * q;
            if (p >= np) break;
            // p -> (a, b) with a <= b, row-major over the upper triangle
            int a = 0, rem = p;
            while (rem >= k - a) {
                rem -= k - a;
                ++a;
            }
            const int b = a + rem;
            const T *ea = E + a * EP, *eb = E + b * EP;
            T s = T(0);
#pragma unroll 8
            for (int e = 0; e < EPP * TP; ++e) s = fma(ea[e], eb[e], s);
            acc[q] += (double)s;
        }
    }
#pragma unroll
    for (int q = 0; q < kGramSlots; ++q) {
        const int p = threadIdx.x + 256 * q;
        if (p < np) part[(long long)blockIdx.x * kGramPairs + p] = acc[q];
    }
}

// 4 x 4 register blocks for FP32 bases (k_gram_psi_pipe below).  A tile is
// 4 x 32 pixels of one frame; its edges (right, down, and with ANISO-TV the
// next frame) of all k columns go to shared memory as rows E[e][0..KP) (KP = k
// rounded up to 32), each 16-byte group of a row stored at group ^ (pixel & 7)
// so that the float4 stores of 8 consecutive pixels fall in distinct bank
// groups.  The k x k upper triangle is cut into 4 x 4 blocks; block pair
// (bi <= bj) and edge phase ph go to one thread, which sums its edges e = ph,
// ph + phases, ... with two float4 reads and 16 FMAs per edge.  Per tile the
// phases are added in FP32 in shared memory and the sum goes to the owner's
// FP64 accumulators; per-CTA FP64 partials as for k_gram_psi.  Up to 256
// block pairs (k <= 88).
constexpr int kRbRows = 4;                      // tile rows
constexpr int kRbPix = kRbRows * 32;            // tile pixels
inline size_t gram_rb_smem(int k, int epp, int nt = 256)
{
    const int kp = 32 * ((k + 31) / 32);
    return (size_t)epp * kRbPix * kp * sizeof(float) + (size_t)nt * 16 * sizeof(float);
}
// threads of the register-blocked Gram for k columns (one 4 x 4 block pair each)
inline int gram_rb_threads(int k)
{
    const int kb = (k + 3) / 4;
    return kb * (kb + 1) / 2 <= 256 ? 256 : 512;
}

// The raw values a tile needs (rows i0 .. i0 + 4 and columns j0 .. j0 + 32
// of every basis column, the next frame's rows with ANISO-TV, and the tile's
// weights) are copied to shared memory with cp.async, the next tile's while
// the current tile builds its edges and runs its products.
constexpr int kRawRows = kRbRows + 1, kRawCols = 33;  // rows and columns of a tile's raw block
constexpr size_t kGramPipeSmemMax = 200 * 1024;        // dynamic shared memory of the pipelined form
inline int gram_raw_floats(int k, int epp)
{
    return k * (kRawRows * kRawCols + (epp == 3 ? kRbRows * 32 : 0)) + 3 * kRbPix;
}
inline size_t gram_pipe_smem(int k, int epp)
{
    return gram_rb_smem(k, epp) + 2 * (size_t)gram_raw_floats(k, epp) * sizeof(float);
}

__device__ __forceinline__ void cp_async4_zfill(float *smem, const float *gmem, bool valid)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    const int bytes = valid ? 4 : 0;  // 0: the destination is zero-filled, the source is not read
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(bytes) : "memory");
}

__global__ void __launch_bounds__(256) k_gram_psi_pipe(const float *__restrict__ V, long long n, int k,
                                                       const float *__restrict__ w, int N, int F, int temporal,
                                                       double *__restrict__ part, const int *stop)
{
    if (stopped(stop)) return;
    extern __shared__ float4 rb_smem[];
    const int EPP = (temporal && F > 1) ? 3 : 2;
    const int KP = 32 * ((k + 31) / 32);
    const int NE = EPP * kRbPix;
    float *E = reinterpret_cast<float *>(rb_smem);  // [NE][KP], swizzled 16-byte groups
    float *red = E + (size_t)NE * KP;               // [16][256]
    float *raw0 = red + 256 * 16;                   // two raw buffers
    const int RAWC = k * kRawRows * kRawCols;        // per buffer: [k][5][33], then [k][4][32] (next frame), then weights
    const int RAWT = EPP == 3 ? k * kRbRows * 32 : 0;
    const int RAW = RAWC + RAWT + 3 * kRbPix;
    const int kb = (k + 3) / 4;
    const int P = kb * (kb + 1) / 2;
    const int phases = max(1, min(8, 256 / P));
    const int t = threadIdx.x;
    const bool busy = t < P * phases;
    const int p = t % P, ph = t / P;
    int bi = 0, rem = p;
    while (rem >= kb - bi) {
        rem -= kb - bi;
        ++bi;
    }
    const int bj = bi + rem;
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    const int tiles_x = (N + 31) / 32, tiles_y = (N + kRbRows - 1) / kRbRows;
    const int ntiles = tiles_x * tiles_y * F;
    const long long nx = (long long)F * N * (N - 1);

    // copies of tile tt into raw buffer dst
    auto issue = [&](int tt, float *dst) {
        const int tile = tt % (tiles_x * tiles_y);
        const int f = tt / (tiles_x * tiles_y);
        const int i0 = (tile / tiles_x) * kRbRows, j0 = (tile % tiles_x) * 32;
        for (int idx = t; idx < RAWC; idx += 256) {
            const int a = idx / (kRawRows * kRawCols), r = (idx / kRawCols) % kRawRows, c = idx % kRawCols;
            const int gi = i0 + r, gj = j0 + c;
            const bool ok = gi < N && gj < N;
            const float *col = V + (long long)a * n + (long long)f * N * N;
            cp_async4_zfill(dst + idx, ok ? col + (size_t)gi * N + gj : col, ok);
        }
        for (int idx = t; idx < RAWT; idx += 256) {  // the next frame's pixels of the tile
            const int a = idx / (kRbRows * 32), r = (idx / 32) % kRbRows, c = idx % 32;
            const int gi = i0 + r, gj = j0 + c;
            const bool ok = f < F - 1 && gi < N && gj < N;
            const float *col = V + (long long)a * n + (long long)(f + 1 < F ? f + 1 : f) * N * N;
            cp_async4_zfill(dst + RAWC + idx, ok ? col + (size_t)gi * N + gj : col, ok);
        }
        for (int idx = t; idx < 3 * kRbPix; idx += 256) {  // weights of the right, down, next-frame edges
            const int e = idx / kRbPix, pix = idx % kRbPix;
            const int gi = i0 + pix / 32, gj = j0 + pix % 32;
            bool ok;
            long long off;
            if (e == 0) {
                ok = gi < N && gj < N - 1;
                off = (long long)f * N * (N - 1) + (long long)gi * (N - 1) + gj;
            } else if (e == 1) {
                ok = gi < N - 1 && gj < N;
                off = nx + (long long)f * (N - 1) * N + (long long)gi * N + gj;
            } else {
                ok = EPP == 3 && f < F - 1 && gi < N && gj < N;
                off = 2 * nx + (long long)f * N * N + (long long)gi * N + gj;
            }
            cp_async4_zfill(dst + RAWC + RAWT + idx, ok ? w + off : w, ok);
        }
    };

    int buf = 0;
    if ((int)blockIdx.x < ntiles) issue(blockIdx.x, raw0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const int nxt = tt + gridDim.x;
        if (nxt < ntiles) issue(nxt, raw0 + (size_t)(buf ^ 1) * RAW);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // tile tt has landed
        __syncthreads();  // ... for every thread; the previous tile is done with E and red
        const float *rw = raw0 + (size_t)buf * RAW;
        const float *rwt = rw + RAWC, *rww = rw + RAWC + RAWT;
        const int tile = tt % (tiles_x * tiles_y);
        const int f = tt / (tiles_x * tiles_y);
        const int i0 = (tile / tiles_x) * kRbRows, j0 = (tile % tiles_x) * 32;
        for (int idx = t; idx < kb * kRbPix; idx += 256) {
            const int g = idx / kRbPix, pix = idx % kRbPix;
            const int li = pix / 32, lj = pix % 32;
            const int i = i0 + li, j = j0 + lj;
            float ex[4] = {0.f, 0.f, 0.f, 0.f}, ey[4] = {0.f, 0.f, 0.f, 0.f}, et[4] = {0.f, 0.f, 0.f, 0.f};
            if (i < N && j < N) {
                const float sx = j < N - 1 ? sqrtf(rww[pix]) : 0.f;
                const float sy = i < N - 1 ? sqrtf(rww[kRbPix + pix]) : 0.f;
                const float st = (EPP == 3 && f < F - 1) ? sqrtf(rww[2 * kRbPix + pix]) : 0.f;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int a = 4 * g + c;
                    if (a < k) {
                        const float *ra = rw + (size_t)a * kRawRows * kRawCols;
                        const float v0 = ra[li * kRawCols + lj];
                        if (j < N - 1) ex[c] = (ra[li * kRawCols + lj + 1] - v0) * sx;
                        if (i < N - 1) ey[c] = (ra[(li + 1) * kRawCols + lj] - v0) * sy;
                        if (EPP == 3 && f < F - 1) et[c] = (rwt[(size_t)a * kRbRows * 32 + li * 32 + lj] - v0) * st;
                    }
                }
            }
            const int col = (4 * g) ^ ((pix & 7) << 2);
            *reinterpret_cast<float4 *>(E + (size_t)(EPP * pix) * KP + col) = make_float4(ex[0], ex[1], ex[2], ex[3]);
            *reinterpret_cast<float4 *>(E + (size_t)(EPP * pix + 1) * KP + col) =
                make_float4(ey[0], ey[1], ey[2], ey[3]);
            if (EPP == 3)
                *reinterpret_cast<float4 *>(E + (size_t)(EPP * pix + 2) * KP + col) =
                    make_float4(et[0], et[1], et[2], et[3]);
        }
        __syncthreads();
        if (busy) {
            float sacc[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) sacc[q] = 0.f;
#pragma unroll 4
            for (int e = ph; e < NE; e += phases) {
                const int sw = ((e / EPP) & 7) << 2;
                const float4 A = *reinterpret_cast<const float4 *>(E + (size_t)e * KP + ((4 * bi) ^ sw));
                const float4 Bv = *reinterpret_cast<const float4 *>(E + (size_t)e * KP + ((4 * bj) ^ sw));
                const float av[4] = {A.x, A.y, A.z, A.w}, bv[4] = {Bv.x, Bv.y, Bv.z, Bv.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) sacc[4 * r + c] = fmaf(av[r], bv[c], sacc[4 * r + c]);
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) red[q * 256 + t] = sacc[q];  // conflict-free by thread
        }
        __syncthreads();
        if (t < P) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                float v = 0.f;
                for (int r = 0; r < phases; ++r) v += red[q * 256 + r * P + t];
                acc[q] += (double)v;
            }
        }
        buf ^= 1;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (t < P) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int a = 4 * bi + q / 4, b = 4 * bj + q % 4;
            if (a <= b && b < k) part[(long long)blockIdx.x * kGramPairs + a * k - a * (a - 1) / 2 + (b - a)] = acc[q];
        }
    }
}

// Large bases (k above what the pipelined 4 x 4 form holds in shared memory):
// the same cp.async pipeline over smaller tiles (TR = 2 or 1 rows of 32
// pixels) with 8 x 8 register blocks.  Block pair (bi <= bj) and edge phase ph
// go to one thread, which keeps its 64 sums in FP32 registers over kP8Flush
// tiles (four float4 reads and 64 FMAs per edge, a quarter of the
// shared-memory reads per FMA of the 4 x 4 blocks); every kP8Flush tiles and
// after the CTA's last tile the threads leave their sums in shared memory and
// the phases of each block pair are added in phase order, in FP64, to the
// CTA's FP64 sums (also in shared memory).  Per-CTA FP64 partials as for
// k_gram_psi; k_gram_reduce sums them in order.
constexpr int kP8Flush = 16;     // tiles summed in FP32 between two FP64 flushes
constexpr int kP8Threads = 384;  // threads of the large-basis form
inline int gram_p8_pairs(int k)
{
    const int kb = (k + 7) / 8;
    return kb * (kb + 1) / 2;
}
inline size_t gram_p8_smem(int k, int epp, int tr)
{
    const int kp = 32 * ((k + 31) / 32);
    const size_t e = (size_t)epp * tr * 32 * kp * sizeof(float);
    const size_t red = (size_t)kP8Threads * 32 * sizeof(float);
    const size_t raw = (size_t)k * ((tr + 1) * kRawCols + (epp == 3 ? tr * 32 : 0)) + 3 * tr * 32;
    return (e > red ? e : red) + 2 * raw * sizeof(float) + (size_t)gram_p8_pairs(k) * 64 * sizeof(double);
}
constexpr size_t kGramP8SmemMax = 226 * 1024;
// tile rows of the large-basis form: 2, or 1 when two rows do not fit (0: neither fits)
inline int gram_p8_rows(int k, int epp)
{
    return gram_p8_smem(k, epp, 2) <= kGramP8SmemMax ? 2 : (gram_p8_smem(k, epp, 1) <= kGramP8SmemMax ? 1 : 0);
}

template <int TR, int NT>
__global__ void __launch_bounds__(NT, 1) k_gram_psi_pipe8(const float *__restrict__ V, long long n, int k,
                                                          const float *__restrict__ w, int N, int F, int temporal,
                                                          double *__restrict__ part, const int *stop)
{
    if (stopped(stop)) return;
    extern __shared__ float4 p8_smem[];
    constexpr int TPIX = TR * 32;
    constexpr int RR = TR + 1;  // raw rows: the tile's and the one below
    const int EPP = (temporal && F > 1) ? 3 : 2;
    const int KP = 32 * ((k + 31) / 32);
    const int NE = EPP * TPIX;
    const size_t efl = max((size_t)NE * KP, (size_t)NT * 32);  // floats of E (and of the flush buffer)
    float *E = reinterpret_cast<float *>(p8_smem);               // [NE][KP], swizzled 16-byte groups
    const int RAWC = k * RR * kRawCols;                          // per buffer: [k][RR][33]
    const int RAWT = EPP == 3 ? k * TPIX : 0;                    // then [k][TR][32] (next frame)
    const int RAW = RAWC + RAWT + 3 * TPIX;                      // then the weights
    float *raw0 = E + efl;
    double *acc = reinterpret_cast<double *>(raw0 + 2 * (size_t)RAW);  // [64][P]
    const int kb = (k + 7) / 8;
    const int kg = (k + 3) / 4;  // column groups of 4 of the edge build
    const int P = kb * (kb + 1) / 2;
    const int phases = max(1, NT / P);
    const int t = threadIdx.x;
    const bool busy = t < P * phases;
    const int p = t % P, ph = t / P;
    int bi = 0, rem = p;
    while (rem >= kb - bi) {
        rem -= kb - bi;
        ++bi;
    }
    const int bj = bi + rem;
    for (int idx = t; idx < P * 64; idx += NT) acc[idx] = 0.0;
    float s[64];
#pragma unroll
    for (int q = 0; q < 64; ++q) s[q] = 0.f;
    const int tiles_x = (N + 31) / 32, tiles_y = (N + TR - 1) / TR;
    const int ntiles = tiles_x * tiles_y * F;
    const long long nx = (long long)F * N * (N - 1);

    // copies of tile tt into raw buffer dst
    auto issue = [&](int tt, float *dst) {
        const int tile = tt % (tiles_x * tiles_y);
        const int f = tt / (tiles_x * tiles_y);
        const int i0 = (tile / tiles_x) * TR, j0 = (tile % tiles_x) * 32;
        for (int idx = t; idx < RAWC; idx += NT) {
            const int a = idx / (RR * kRawCols), r = (idx / kRawCols) % RR, c = idx % kRawCols;
            const int gi = i0 + r, gj = j0 + c;
            const bool ok = gi < N && gj < N;
            const float *col = V + (long long)a * n + (long long)f * N * N;
            cp_async4_zfill(dst + idx, ok ? col + (size_t)gi * N + gj : col, ok);
        }
        for (int idx = t; idx < RAWT; idx += NT) {  // the next frame's pixels of the tile
            const int a = idx / TPIX, r = (idx / 32) % TR, c = idx % 32;
            const int gi = i0 + r, gj = j0 + c;
            const bool ok = f < F - 1 && gi < N && gj < N;
            const float *col = V + (long long)a * n + (long long)(f + 1 < F ? f + 1 : f) * N * N;
            cp_async4_zfill(dst + RAWC + idx, ok ? col + (size_t)gi * N + gj : col, ok);
        }
        for (int idx = t; idx < 3 * TPIX; idx += NT) {  // weights of the right, down, next-frame edges
            const int e = idx / TPIX, pix = idx % TPIX;
            const int gi = i0 + pix / 32, gj = j0 + pix % 32;
            bool ok;
            long long off;
            if (e == 0) {
                ok = gi < N && gj < N - 1;
                off = (long long)f * N * (N - 1) + (long long)gi * (N - 1) + gj;
            } else if (e == 1) {
                ok = gi < N - 1 && gj < N;
                off = nx + (long long)f * (N - 1) * N + (long long)gi * N + gj;
            } else {
                ok = EPP == 3 && f < F - 1 && gi < N && gj < N;
                off = 2 * nx + (long long)f * N * N + (long long)gi * N + gj;
            }
            cp_async4_zfill(dst + RAWC + RAWT + idx, ok ? w + off : w, ok);
        }
    };

    int buf = 0, batch = 0;
    if ((int)blockIdx.x < ntiles) issue(blockIdx.x, raw0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const int nxt = tt + gridDim.x;
        if (nxt < ntiles) issue(nxt, raw0 + (size_t)(buf ^ 1) * RAW);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // tile tt has landed
        __syncthreads();  // ... for every thread; the previous tile (or flush) is done with E
        const float *rw = raw0 + (size_t)buf * RAW;
        const float *rwt = rw + RAWC, *rww = rw + RAWC + RAWT;
        const int tile = tt % (tiles_x * tiles_y);
        const int f = tt / (tiles_x * tiles_y);
        const int i0 = (tile / tiles_x) * TR, j0 = (tile % tiles_x) * 32;
        // (columns 4 kg .. KP of a row are not written: they meet only entries with b >= k, not kept)
        for (int idx = t; idx < kg * TPIX; idx += NT) {
            const int g = idx / TPIX, pix = idx % TPIX;
            const int li = pix / 32, lj = pix % 32;
            const int i = i0 + li, j = j0 + lj;
            float ex[4] = {0.f, 0.f, 0.f, 0.f}, ey[4] = {0.f, 0.f, 0.f, 0.f}, et[4] = {0.f, 0.f, 0.f, 0.f};
            if (i < N && j < N) {
                const float sx = j < N - 1 ? sqrtf(rww[pix]) : 0.f;
                const float sy = i < N - 1 ? sqrtf(rww[TPIX + pix]) : 0.f;
                const float st = (EPP == 3 && f < F - 1) ? sqrtf(rww[2 * TPIX + pix]) : 0.f;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int a = 4 * g + c;
                    if (a < k) {
                        const float *ra = rw + (size_t)a * RR * kRawCols;
                        const float v0 = ra[li * kRawCols + lj];
                        if (j < N - 1) ex[c] = (ra[li * kRawCols + lj + 1] - v0) * sx;
                        if (i < N - 1) ey[c] = (ra[(li + 1) * kRawCols + lj] - v0) * sy;
                        if (EPP == 3 && f < F - 1) et[c] = (rwt[(size_t)a * TPIX + li * 32 + lj] - v0) * st;
                    }
                }
            }
            const int col = (4 * g) ^ ((pix & 7) << 2);
            *reinterpret_cast<float4 *>(E + (size_t)(EPP * pix) * KP + col) = make_float4(ex[0], ex[1], ex[2], ex[3]);
            *reinterpret_cast<float4 *>(E + (size_t)(EPP * pix + 1) * KP + col) =
                make_float4(ey[0], ey[1], ey[2], ey[3]);
            if (EPP == 3)
                *reinterpret_cast<float4 *>(E + (size_t)(EPP * pix + 2) * KP + col) =
                    make_float4(et[0], et[1], et[2], et[3]);
        }
        __syncthreads();
        if (busy) {
#pragma unroll 2
            for (int e = ph; e < NE; e += phases) {
                const int sw = ((e / EPP) & 7) << 2;
                const float *row = E + (size_t)e * KP;
                const float4 A0 = *reinterpret_cast<const float4 *>(row + ((8 * bi) ^ sw));
                const float4 A1 = *reinterpret_cast<const float4 *>(row + ((8 * bi + 4) ^ sw));
                const float4 B0 = *reinterpret_cast<const float4 *>(row + ((8 * bj) ^ sw));
                const float4 B1 = *reinterpret_cast<const float4 *>(row + ((8 * bj + 4) ^ sw));
                const float av[8] = {A0.x, A0.y, A0.z, A0.w, A1.x, A1.y, A1.z, A1.w};
                const float bv[8] = {B0.x, B0.y, B0.z, B0.w, B1.x, B1.y, B1.z, B1.w};
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) s[8 * r + c] = fmaf(av[r], bv[c], s[8 * r + c]);
            }
        }
        if (++batch == kP8Flush || nxt >= ntiles) {  // uniform over the CTA
            batch = 0;
            float *red = E;  // [32][NT], one half of the 64 sums at a time
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                __syncthreads();  // every thread is done with E (or with the previous half)
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    red[q * NT + t] = busy ? s[32 * half + q] : 0.f;
                    s[32 * half + q] = 0.f;
                }
                __syncthreads();
                for (int idx = t; idx < P * 32; idx += NT) {  // consecutive threads: consecutive block pairs
                    const int q = idx / P, pp = idx % P;
                    double v = 0.0;
                    for (int r = 0; r < phases; ++r) v += (double)red[q * NT + r * P + pp];
                    acc[(32 * half + q) * P + pp] += v;
                }
            }
        }
        buf ^= 1;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    for (int idx = t; idx < P * 64; idx += NT) {
        const int q = idx / P, pp = idx % P;
        int i = 0, rr = pp;
        while (rr >= kb - i) {
            rr -= kb - i;
            ++i;
        }
        const int a = 8 * i + q / 8, b = 8 * (i + rr) + q % 8;
        if (a <= b && b < k) part[(long long)blockIdx.x * kGramPairs + a * k - a * (a - 1) / 2 + (b - a)] = acc[idx];
    }
}

// G (ld kKMax, symmetric, k x k) = sum over nblk partials: one warp per entry,
// each lane sums the partials c = lane, lane + 32, ... and the warp adds the
// lanes in a fixed tree (FP64 is narrow on this part: no long dependent chains).
constexpr int kGramReduceWarps = 8;
inline int gram_reduce_blocks(int k) { return (k * (k + 1) / 2 + kGramReduceWarps - 1) / kGramReduceWarps; }

__global__ void __launch_bounds__(32 * kGramReduceWarps) k_gram_reduce(const double *__restrict__ part, int nblk,
                                                                       int k, double *__restrict__ G,
                                                                       const int *stop)
{
    if (stopped(stop)) return;
    const int np = k * (k + 1) / 2;
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < np; p += nw) {
        double s = 0.0;
        for (int c = lane; c < nblk; c += 32) s += part[(long long)c * kGramPairs + p];
        s = warp_sum(s);
        if (lane == 0) {
            int a = 0, rem = p;
            while (rem >= k - a) {
                rem -= k - a;
                ++a;
            }
            const int b = a + rem;
            G[a * kKMax + b] = s;
            G[b * kKMax + a] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// tall-skinny products: out[a] = sum_i A[a][i] * x[i] for a < k (A column-major
// with column stride lda); x2 (nullable) adds out[k] = x . x2 .
// kRedBlocks CTAs each own a contiguous slice; partials reduced in order.
// ---------------------------------------------------------------------------
// Columns are taken 16 at a time.  Every thread sums its elements of the 16
// products: in FP64 for T = double; for T = float in FP32 over runs of 16
// elements, each run then added in FP64 (the products are FP32 to begin with,
// and the FP64 pipe of this part is narrow: at 2048^2 per-element FP64 adds
// bound the kernel).  The 256 per-thread sums of a column are then added
// through shared memory: 16 threads per column sum 16 values each (strided)
// and combine them in a 16-lane tree, far fewer FP64 instructions than a
// shuffle tree per warp.  Fixed order throughout.
template <typename T>
__global__ void __launch_bounds__(256) k_dots(const T *__restrict__ A, long long len, long long lda, int k,
                                              const T *__restrict__ x, const T *__restrict__ x2,
                                              double *__restrict__ part, const int *stop)
{
    if (stopped(stop)) return;
    constexpr int G = 16;
    __shared__ double sh[G][257];
    const long long per = (len + gridDim.x - 1) / gridDim.x;
    const long long lo = blockIdx.x * per, hi = min(len, lo + per);
    const int kk = k + (x2 ? 1 : 0);
    for (int a0 = 0; a0 < kk; a0 += G) {
        const int na = min(G, kk - a0);
        const T *cols[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int a = min(a0 + q, kk - 1);
            cols[q] = (a < k) ? A + (long long)a * lda : x2;
        }
        double s[G];
#pragma unroll
        for (int q = 0; q < G; ++q) s[q] = 0.0;
        if constexpr (std::is_same<T, float>::value) {
            // FP32 fused multiply-adds over runs of 16 of the thread's
            // elements, each run added to the FP64 sum
            float fr[G];
#pragma unroll
            for (int q = 0; q < G; ++q) fr[q] = 0.0f;
            int run = 0;
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                const float xi = x[i];
#pragma unroll
                for (int q = 0; q < G; ++q)
                    if (q < na) fr[q] = fmaf(cols[q][i], xi, fr[q]);
                if (++run == 16) {
#pragma unroll
                    for (int q = 0; q < G; ++q) {
                        s[q] += (double)fr[q];
                        fr[q] = 0.0f;
                    }
                    run = 0;
                }
            }
#pragma unroll
            for (int q = 0; q < G; ++q) s[q] += (double)fr[q];
        } else {
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                const T xi = x[i];
#pragma unroll
                for (int q = 0; q < G; ++q)
                    if (q < na) s[q] = fma(cols[q][i], xi, s[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < G; ++q)
            if (q < na) sh[q][threadIdx.x] = s[q];
        __syncthreads();
        {
            const int q = threadIdx.x >> 4, seg = threadIdx.x & 15;
            double t = 0.0;
            if (q < na) {
#pragma unroll
                for (int e = 0; e < 16; ++e) t += sh[q][seg + 16 * e];  // conflict-free
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (seg == 0 && q < na) part[(long long)blockIdx.x * (kKMax + 2) + a0 + q] = t;
        }
        __syncthreads();
    }
}

// out[a] = sum_c part[c][a] for a < kk: one warp per output, lanes over the
// partials, a fixed warp tree
constexpr int kDotsReduceWarps = 8;
__global__ void __launch_bounds__(32 * kDotsReduceWarps) k_dots_reduce(const double *__restrict__ part, int nblk,
                                                                       int kk, double *__restrict__ out,
                                                                       const int *stop)
{
    if (stopped(stop)) return;
    const int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (a >= kk) return;
    double s = 0.0;
    for (int c = lane; c < nblk; c += 32) s += part[(long long)c * (kKMax + 2) + a];
    s = warp_sum(s);
    if (lane == 0) out[a] = s;
}

// out[i] = beta*out[i] + sgn * sum_a A[a][i] * y[a]  (+ bias[i] * bsgn)
template <typename T>
__global__ void k_gemv(const T *__restrict__ A, long long len, long long lda, int k, const double *__restrict__ y,
                       T *__restrict__ out, T beta, T sgn, const T *__restrict__ bias, T bsgn, const int *stop)
{
    if (stopped(stop)) return;
    __shared__ T ys[kKMax];
    for (int a = threadIdx.x; a < k; a += blockDim.x) ys[a] = (T)y[a];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
        T s = T(0);
        for (int a = 0; a < k; ++a) s = fma(A[(long long)a * lda + i], ys[a], s);
        T o = beta == T(0) ? T(0) : beta * out[i];
        o = fma(sgn, s, o);
        if (bias) o = fma(bsgn, bias[i], o);
        out[i] = o;
    }
}

// out[c][i] = sum_a A[a][i] * W[a][c]   (W: kKMax x kKMax row-major, c < kc)
template <typename T>
__global__ void k_gemm_small(const T *__restrict__ A, long long len, long long lda, int k,
                             const double *__restrict__ W, int kc, T *__restrict__ out, long long ldo)
{
    __shared__ T Ws[kKMax * 16];
    for (int idx = threadIdx.x; idx < k * kc; idx += blockDim.x) Ws[idx] = (T)W[(idx / kc) * kKMax + idx % kc];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
        T acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = T(0);
        for (int a = 0; a < k; ++a) {
            const T v = A[(long long)a * lda + i];
#pragma unroll
            for (int c = 0; c < 16; ++c)
                if (c < kc) acc[c] = fma(v, Ws[a * kc + c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < 16; ++c)
            if (c < kc) out[(long long)c * ldo + i] = acc[c];
    }
}

// squared norms of three vectors: a (|a|^2), a - b (|a - b|^2), b (|b|^2); per-block partials
template <typename T>
__global__ void k_norms3(const T *__restrict__ a, const T *__restrict__ b, long long len, double *__restrict__ part,
                         const int *stop)
{
    if (stopped(stop)) return;
    __shared__ double sh[33];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
        const double x = (double)a[i];
        const double y = b ? (double)b[i] : 0.0;
        s0 += x * x;
        s1 += (x - y) * (x - y);
        s2 += y * y;
    }
    s0 = block_sum(s0, sh);
    s1 = block_sum(s1, sh);
    s2 = block_sum(s2, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 3 + 0] = s0;
        part[blockIdx.x * 3 + 1] = s1;
        part[blockIdx.x * 3 + 2] = s2;
    }
}

// one warp: lanes over the partials, a fixed warp tree per output
__global__ void k_norms3_reduce(const double *__restrict__ part, int nblk, double *__restrict__ out3,
                                const int *stop)
{
    if (stopped(stop)) return;
    if (threadIdx.x >= 32) return;
    for (int q = 0; q < 3; ++q) {
        double s = 0.0;
        for (int c = threadIdx.x; c < nblk; c += 32) s += part[c * 3 + q];
        s = warp_sum(s);
        if (threadIdx.x == 0) out3[q] = s;
    }
}

// ---------------------------------------------------------------------------
// Enlarge step bookkeeping: normalise the new direction, decide whether the
// step is the last one (tol_1 test or a vanished residual).
//   scal[kRnorm2] = |r|^2, norms3 = {|u|^2, |u - u_old|^2, |u_old|^2}
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_normalize(T *__restrict__ r, long long len, const double *__restrict__ rn2, const int *stop)
{
    if (stopped(stop)) return;
    const double nr = sqrt(*rn2);
    const T inv = nr > 0.0 ? (T)(1.0 / nr) : T(0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
        r[i] *= inv;
}

__global__ void k_step_decide(const double *__restrict__ rn2, const double *__restrict__ norms3, double tol1,
                              int *__restrict__ ctl, double *__restrict__ scal)
{
    if (ctl[kStop]) return;
    const double uold2 = norms3[2];
    const bool small = uold2 > 0.0 && sqrt(norms3[1]) <= tol1 * sqrt(uold2);
    const bool vanished = !(*rn2 > 0.0);
    ctl[kSteps] += 1;
    scal[kDu2] = norms3[1];
    scal[kU2] = uold2;
    ctl[kStopNext] = (small || vanished) ? 1 : 0;
    if (vanished) ctl[kBreakdown] = 1;
}

// Append row/column kc of (HV)^T HV and entry kc of (HV)^T b from
// dots = {HV[:, j] . h_new for j <= kc, b . h_new}.
__global__ void k_gh_append(const double *__restrict__ dots, int kc, double *__restrict__ GH,
                            double *__restrict__ cvec, const int *stop)
{
    if (stopped(stop)) return;
    const int j = threadIdx.x;
    if (j <= kc) {
        GH[kc * kKMax + j] = dots[j];
        GH[j * kKMax + kc] = dots[j];
    }
    if (j == 0) cvec[kc] = dots[kc + 1];
}

// Ends a step: raises the stop flag when the step decided so, and mirrors
// it to host-mapped memory (nullable) for the host's issue loop.
__global__ void k_step_commit(int *__restrict__ ctl, volatile int *__restrict__ stop_mirror)
{
    if (!ctl[kStop] && ctl[kStopNext]) ctl[kStop] = 1;
    if (stop_mirror) *stop_mirror = ctl[kStop];
}

// ---------------------------------------------------------------------------
// FP64 small algebra in one CTA.  Its matrices have leading dimension KM + 1
// (KM = kKSmem: in shared memory, for bases of up to kKSmem columns;
// KM = kKMax: in a device workspace the solver allocates, for larger bases --
// __syncthreads orders a block's global accesses as it orders its shared ones).
// ---------------------------------------------------------------------------

// Cholesky A = L L^T in place (lower triangle); pivots clamped at tiny*A00.
template <int kLd>
__device__ void chol(double *A, int k, int *bad)
{
    for (int j = 0; j < k; ++j) {
        __syncthreads();
        if (threadIdx.x == 0) {
            double d = A[j * kLd + j];
            const double floor_ = 1e-300 + 1e-15 * fabs(A[0]);
            if (!(d > floor_)) {
                d = floor_;
                *bad = 1;
            }
            A[j * kLd + j] = sqrt(d);
        }
        __syncthreads();
        const double dj = A[j * kLd + j];
        for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) A[i * kLd + j] /= dj;
        __syncthreads();
        const int m = k - j - 1;
        for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
            const int i = j + 1 + idx / m, l = j + 1 + idx % m;
            if (l <= i) A[i * kLd + l] -= A[i * kLd + j] * A[l * kLd + j];
        }
    }
    __syncthreads();
}

// Cyclic Jacobi eigen-decomposition of the symmetric k x k matrix A
// (overwritten; its diagonal ends as the eigenvalues), eigenvectors in the
// columns of U.  Parallel round-robin ordering of the (p, q) rotations.
template <int kLd>
__device__ void jacobi_eig(double *A, double *U, int k, double *cs, double *sn, int *pp, int *qq, double *sh)
{
    for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
        const int i = idx / k, j = idx % k;
        U[i * kLd + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int kp = (k + 1) & ~1;  // even number of players, index k is a bye when k is odd
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
            const int i = idx / k, j = idx % k;
            const double v = A[i * kLd + j];
            tot += v * v;
            if (i != j) off += v * v;
        }
        off = block_sum(off, sh);
        tot = block_sum(tot, sh);
        if (!(off > 1e-30 * tot)) break;
        for (int round = 0; round < kp - 1; ++round) {
            for (int i = threadIdx.x; i < kp / 2; i += blockDim.x) {
                int p, q;
                if (i == 0) {
                    p = kp - 1;
                    q = round;
                } else {
                    p = (round + i) % (kp - 1);
                    q = (round - i + (kp - 1)) % (kp - 1);
                }
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                pp[i] = p;
                qq[i] = q;
                double c = 1.0, s = 0.0;
                if (q < k) {
                    const double apq = A[p * kLd + q];
                    if (apq != 0.0) {
                        const double tau = (A[q * kLd + q] - A[p * kLd + p]) / (2.0 * apq);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                cs[i] = c;
                sn[i] = s;
            }
            __syncthreads();
            const int npair = kp / 2;
            for (int idx = threadIdx.x; idx < npair * k; idx += blockDim.x) {  // rows p, q
                const int i = idx / k, j = idx % k;
                const int p = pp[i], q = qq[i];
                if (q >= k) continue;
                const double c = cs[i], s = sn[i];
                const double ap = A[p * kLd + j], aq = A[q * kLd + j];
                A[p * kLd + j] = c * ap - s * aq;
                A[q * kLd + j] = s * ap + c * aq;
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < npair * k; idx += blockDim.x) {  // columns p, q (and U)
                const int i = idx / k, j = idx % k;
                const int p = pp[i], q = qq[i];
                if (q >= k) continue;
                const double c = cs[i], s = sn[i];
                const double ap = A[j * kLd + p], aq = A[j * kLd + q];
                A[j * kLd + p] = c * ap - s * aq;
                A[j * kLd + q] = s * ap + c * aq;
                const double up = U[j * kLd + p], uq = U[j * kLd + q];
                U[j * kLd + p] = c * up - s * uq;
                U[j * kLd + q] = s * up + c * uq;
            }
            __syncthreads();
        }
    }
    __syncthreads();
}

// Work area of k_compress_basis (matrix, eigenvectors, rotation tables).
template <int KM> struct SmallShared {
    static constexpr int kLd = KM + 1;
    double A[KM * kLd];
    double U[KM * kLd];
    double vec[1][KM + 1];
    double cs[KM / 2 + 1], sn[KM / 2 + 1];
    int pp[KM / 2 + 1], qq[KM / 2 + 1];
    double sh[40];
};

// Reduced problem of one Enlarge step:
//   G_H = (H V)^T (H V), c = (H V)^T b (both maintained incrementally),
//   G_P = (P Psi V)^T (P Psi V).
// For a given lambda the normal equations (G_H + lambda G_P) y = c are solved
// by an L D L^T factorization, and the projected residual (the QR form
// |R_H y - Q_H^T b|^2 + |b|^2 - |Q_H^T b|^2 of the reduced problem) is
//   phi(lambda) = |H V y - b|^2 = |b|^2 - c.y - lambda y.G_P y,
// increasing in lambda with d phi / d lambda = 2 lambda w.(G_H + lambda G_P)^{-1} w,
// w = G_P y.  lambda: fixed, or the discrepancy principle phi = target solved
// in t = log10(lambda) over [lam_lo, lam_hi] by Newton steps safeguarded by
// bisection of the bracket (started from the previous lambda in scal[kLam]);
// a target at or below phi(10^lam_lo) gives 10^lam_lo, at or above
// phi(10^lam_hi) gives 10^lam_hi, as for plain bisection.  The search stops
// when |phi - target| <= 1e-10 target or the step falls below 1e-12 in t
// (lambda within ~2e-10 of the root).  The matrix is factored as L D L^T.
//
// FP64 on this part issues one warp instruction per 64 cycles per SM
// sub-partition, whatever the number of active lanes, so the solve is laid
// out for short FP64 chains and spread over the four sub-partitions: one CTA
// of four warps.  In the factorization thread 0 carries the pivot chain (it
// updates the next pivot and takes its reciprocal while warps 1-3 update the
// rest of the trailing block and the right-hand side); the substitutions and
// the small reductions run in warp 0.
constexpr int kSolveThreads = 128;

template <int KM> struct SolveShared {
    static constexpr int kLd = KM + 1;
    double GH[KM * kLd], GP[KM * kLd], L[KM * kLd];
    double c[KM], v[KM], y[KM], inv[KM];
    double fd[2];  // phi(lambda) and d phi / d t of the last evaluation
    int bad;
};
// bytes of device workspace the large-basis forms of k_small_solve and k_compress_basis need
constexpr size_t kSmallWorkBytes = sizeof(SolveShared<kKMax>) > sizeof(SmallShared<kKMax>)
                                       ? sizeof(SolveShared<kKMax>) : sizeof(SmallShared<kKMax>);

// L D L^T factorization of the lower triangle of L in place (all threads of a
// kSolveThreads CTA), with the forward substitution z = L^{-1} rhs done along
// the way (rhs overwritten).  The strict lower triangle becomes the unit
// factor and inv[j] = 1 / D_j.  Column j updates the trailing entries
// L[i][l] -= L[i][j] L[l][j] / D_j from the unscaled column; thread 0 updates
// the next pivot first and takes its reciprocal, warps 1-3 the other entries
// and rhs[i] -= (L[i][j] / D_j) rhs[j]; the columns are scaled at the end.
// Pivots at or below tiny * L_00 are clamped and flag *bad.
template <int kLd>
__device__ void ldlt_fwd(double *L, double *inv, double *rhs, int k, int *bad)
{
    constexpr int kWorkers = kSolveThreads - 32;
    const int tid = threadIdx.x;
    const double floor_ = 1e-300 + 1e-15 * fabs(L[0]);
    if (tid == 0) {
        double d = L[0];
        if (!(d > floor_)) {
            d = floor_;
            *bad = 1;
        }
        inv[0] = 1.0 / d;
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        const double id = inv[j];
        const int m = k - j - 1;
        if (tid == 0) {
            if (m > 0) {
                const int p = (j + 1) * kLd + j + 1, q = (j + 1) * kLd + j;
                L[p] -= L[q] * id * L[q];
                double d = L[p];
                if (!(d > floor_)) {
                    d = floor_;
                    *bad = 1;
                }
                inv[j + 1] = 1.0 / d;
            }
        } else if (tid >= 32) {
            // entry e of the trailing triangle (row i, column l <= i, e = i (i + 1) / 2 + l),
            // e = 1 .. m (m + 1) / 2 - 1 (e = 0 is the next pivot); e beyond the triangle
            // (row i = m) is the right-hand-side entry of row j + 1 + l
            const int e0 = tid - 31;
            int i = 0, l = e0;
            while (l > i) {
                l -= i + 1;
                ++i;
            }
            const double zj = rhs[j];
            for (int e = e0; e < m * (m + 1) / 2 + m; e += kWorkers) {
                if (i < m) {
                    const int ri = j + 1 + i, cl = j + 1 + l;
                    L[ri * kLd + cl] -= L[ri * kLd + j] * id * L[cl * kLd + j];
                } else {
                    const int r = j + 1 + l;
                    rhs[r] -= L[r * kLd + j] * id * zj;
                }
                l += kWorkers;
                while (l > i && i < m) {
                    l -= i + 1;
                    ++i;
                }
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < k * k; e += kSolveThreads) {  // unit factor
        const int r = e / k, c = e % k;
        if (c < r) L[r * kLd + c] *= inv[c];
    }
    __syncthreads();
}

// v := L^{-1} v for the unit factor (warp 0, lanes over rows)
template <int kLd>
__device__ void fwd_subst_warp(const double *L, double *v, int k)
{
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < k; ++j) {
        const double zj = v[j];
        for (int i = j + 1 + lane; i < k; i += 32) v[i] -= L[i * kLd + j] * zj;
        __syncwarp();
    }
}

// v := L^{-T} D^{-1} v (warp 0): the second half of an L D L^T solve
template <int kLd>
__device__ void back_subst_warp(const double *L, const double *inv, double *v, int k)
{
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < k; i += 32) v[i] *= inv[i];
    __syncwarp();
    for (int j = k - 1; j >= 0; --j) {
        const double yj = v[j];
        for (int i = lane; i < j; i += 32) v[i] -= L[j * kLd + i] * yj;
        __syncwarp();
    }
}

// KM = kKSmem: the work area in dynamic shared memory; KM = kKMax: in `work`
// (device, kSmallWorkBytes).  The threads of the block exchange values through
// the work area (pivots, phi(lambda), the convergence tests that steer every
// thread's control flow), so `work` must not be restrict-qualified: that would
// let the compiler assume no other thread writes it and keep stale copies,
// after which threads could take different branches around a barrier.
template <int KM>
__global__ void __launch_bounds__(kSolveThreads) k_small_solve(const double *__restrict__ GH,
                                                               const double *__restrict__ cvec,
                                                               const double *__restrict__ GP, int k, double bnorm2,
                                                               double target, double lam_fix, double lam_lo,
                                                               double lam_hi, int lam_iters, double *__restrict__ y,
                                                               double *__restrict__ scal, int *__restrict__ ctl,
                                                               double *work)
{
    if (ctl[kStop]) return;
    extern __shared__ unsigned char smem_raw[];
    constexpr int kLd = SolveShared<KM>::kLd;
    SolveShared<KM> &S = *reinterpret_cast<SolveShared<KM> *>(KM > kKSmem ? (unsigned char *)work : smem_raw);
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) S.bad = 0;
    for (int idx = tid; idx < k * k; idx += kSolveThreads) {
        const int i = idx / k, j = idx % k;
        S.GH[i * kLd + j] = GH[i * kKMax + j];
        S.GP[i * kLd + j] = GP[i * kKMax + j];
    }
    for (int i = tid; i < k; i += kSolveThreads) S.c[i] = cvec[i];
    const double lam_prev = scal[kLam];
    __syncthreads();
    // phi(lambda) (and d phi / d t, t = log10 lambda, when want_d); leaves y in
    // S.y.  Called by every thread with the same arguments; returns the same
    // value in every thread.
    auto eval = [&](double lam, bool want_d, double &dphi_dt) -> double {
        for (int idx = tid; idx < k * k; idx += kSolveThreads) {
            const int i = idx / k, j = idx % k;
            if (j <= i) S.L[i * kLd + j] = S.GH[i * kLd + j] + lam * S.GP[i * kLd + j];
        }
        for (int i = tid; i < k; i += kSolveThreads) S.y[i] = S.c[i];
        __syncthreads();
        ldlt_fwd<kLd>(S.L, S.inv, S.y, k, &S.bad);
        if (tid < 32) {
            back_subst_warp<kLd>(S.L, S.inv, S.y, k);
            double cy = 0.0, yw = 0.0;
            for (int i = lane; i < k; i += 32) {
                double t = 0.0;
                for (int l = 0; l < k; ++l) t += S.GP[i * kLd + l] * S.y[l];
                S.v[i] = t;
                cy += S.c[i] * S.y[i];
                yw += S.y[i] * t;
            }
            cy = warp_sum(cy);
            yw = warp_sum(yw);
            __syncwarp();
            double d = 0.0;
            if (want_d) {
                // w.(L D L^T)^{-1} w = sum_i (L^{-1} w)_i^2 / D_i, w = G_P y
                fwd_subst_warp<kLd>(S.L, S.v, k);
                double wz = 0.0;
                for (int i = lane; i < k; i += 32) wz += S.v[i] * S.v[i] * S.inv[i];
                wz = warp_sum(wz);
                d = 2.0 * lam * wz * lam * 2.302585092994045684;  // d/dt = lambda ln(10) d/dlambda
            }
            if (lane == 0) {
                S.fd[0] = bnorm2 - cy - lam * yw;
                S.fd[1] = d;
            }
        }
        __syncthreads();
        const double f = S.fd[0];
        dphi_dt = S.fd[1];
        __syncthreads();  // S.fd is rewritten by the next evaluation
        return f;
    };
    // 10^t (exp of t ln 10: the search only needs a smooth monotone map, and
    // the lambda returned is the one the last evaluation used)
    auto p10 = [](double t) { return exp(t * 2.302585092994045684); };
    double lam, dd;
    if (lam_fix > 0.0) {
        lam = lam_fix;
        eval(lam, false, dd);
    } else {
        // Newton in t on the bracket [lo, hi]; an end of the bracket that is
        // still lam_lo (lam_hi) is evaluated only when a step would leave it,
        // and ends the search when the target lies beyond it.  S.y always
        // holds the solution at the last evaluated t, which is returned.
        // Every thread runs this control flow on the same values.
        double lo = lam_lo, hi = lam_hi;
        bool lo_seen = false, hi_seen = false;
        double t = (lam_prev > 0.0) ? log10(lam_prev) : 0.5 * (lo + hi);
        if (!(t > lo && t < hi)) t = 0.5 * (lo + hi);
        double te = t;  // last evaluated t
        for (int it = 0; it < lam_iters + 2; ++it) {
            double dft;
            te = t;
            const double f = eval(p10(t), true, dft) - target;
            if (t == lam_lo && f >= 0.0) break;  // target at or below the smallest residual
            if (t == lam_hi && f <= 0.0) break;  // target at or above the largest residual
            // phi carries rounding errors near 1e-12 of the target here; once it
            // is this close, further steps only chase that noise (lambda is then
            // within ~2e-10 of the root)
            if (fabs(f) <= 1e-10 * target) break;
            if (f < 0.0) {
                lo = t;
                lo_seen = true;
            } else {
                hi = t;
                hi_seen = true;
            }
            double tn = t - f / dft;
            if (!(dft > 0.0) || !(tn > lo && tn < hi)) {
                if (!(tn > lo) && !lo_seen) tn = lo;        // check the lower end first
                else if (!(tn < hi) && !hi_seen) tn = hi;   // the upper end
                else tn = 0.5 * (lo + hi);
            }
            // phi carries rounding errors of ~1e-13 relative, so the root is
            // not defined more finely than this in t
            const double tol = 1e-12 * fmax(1.0, fabs(t));
            if (fabs(tn - t) <= tol || hi - lo <= tol) break;  // t is the root to tol
            t = tn;
        }
        lam = p10(te);
    }
    for (int i = tid; i < k; i += kSolveThreads) y[i] = S.y[i];
    if (tid == 0) {
        scal[kLam] = lam;
        if (S.bad) ctl[kBreakdown] = 1;
    }
}

// Compress: right singular vectors of [R_H; sqrt(lambda) R_P] are the
// eigenvectors of G_H + lambda G_P; W (row-major, ld kKMax) receives the
// keep = k_min - 1 of largest eigenvalue, ordered by decreasing eigenvalue
// (ties by index), each signed so its largest-magnitude entry is positive.
template <int KM>
__global__ void __launch_bounds__(256) k_compress_basis(const double *__restrict__ GH, const double *__restrict__ GP,
                                                        int k, const double *__restrict__ scal, int keep,
                                                        double *__restrict__ W, double *work)
{
    extern __shared__ unsigned char smem_raw[];
    constexpr int kLd = SmallShared<KM>::kLd;
    SmallShared<KM> &S = *reinterpret_cast<SmallShared<KM> *>(KM > kKSmem ? (unsigned char *)work : smem_raw);
    const double lam = scal[kLam];
    for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
        const int i = idx / k, j = idx % k;
        S.A[i * kLd + j] = GH[i * kKMax + j] + lam * GP[i * kKMax + j];
    }
    __syncthreads();
    jacobi_eig<kLd>(S.A, S.U, k, S.cs, S.sn, S.pp, S.qq, S.sh);
    if (threadIdx.x == 0) {  // selection of the `keep` largest eigenvalues
        bool used[kKMax];
        for (int i = 0; i < k; ++i) used[i] = false;
        for (int c = 0; c < keep && c < k; ++c) {
            int best = -1;
            for (int i = 0; i < k; ++i)
                if (!used[i] && (best < 0 || S.A[i * kLd + i] > S.A[best * kLd + best])) best = i;
            used[best] = true;
            S.vec[0][c] = (double)best;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < keep && c < k; c += blockDim.x) {
        const int src = (int)S.vec[0][c];
        int arg = 0;
        double big = 0.0;
        for (int i = 0; i < k; ++i) {
            const double v = fabs(S.U[i * kLd + src]);
            if (v > big) {
                big = v;
                arg = i;
            }
        }
        const double sgn = S.U[arg * kLd + src] < 0.0 ? -1.0 : 1.0;
        for (int i = 0; i < k; ++i) W[i * kKMax + c] = sgn * S.U[i * kLd + src];
    }
}

// Rounding scale sum |r| (|r + b| + |b|) of a misfit 1/2 |r|^2 formed from
// r = A - b (A = r + b); per-block partials in slot 0 of 3 (k_norms3_reduce).
template <typename T>
__global__ void k_round_scale(const T *__restrict__ r, const T *__restrict__ b, long long len,
                              double *__restrict__ part)
{
    __shared__ double sh[33];
    double s0 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
        const double x = (double)r[i], y = (double)b[i];
        s0 += fabs(x) * (fabs((double)(r[i] + b[i])) + fabs(y));
    }
    s0 = block_sum(s0, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 3 + 0] = s0;
        part[blockIdx.x * 3 + 1] = 0.0;
        part[blockIdx.x * 3 + 2] = 0.0;
    }
}

// VarPro reduced objective f = 1/2 |res|^2 + lambda/2 y^T G_P y (one thread).
__global__ void k_varpro_value(const double *__restrict__ norms3_res, const double *__restrict__ GP,
                               const double *__restrict__ y, int k, double lam, double *__restrict__ fval)
{
    double q = 0.0;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) q += y[i] * GP[i * kKMax + j] * y[j];
    *fval = 0.5 * norms3_res[0] + 0.5 * lam * q;
}

template <typename T> __global__ void k_fill(T *__restrict__ x, long long len, T value)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
        x[i] = value;
}

// ---------------------------------------------------------------------------
// Gauss-Newton per view (diagonal J^T J): direction and Armijo bookkeeping
// ---------------------------------------------------------------------------
// mu = mu_rel * max_v |J_v|^2; d_v = -g_v / (|J_v|^2 + mu); alpha = alpha0;
// theta_trial = theta + alpha d; every view active.
// Per-view damped Gauss-Newton direction d_v = -g_v / (|J_v|^2 + mu) and the
// first Armijo trial alpha0.  A view whose first-order change alpha0 |g_v d_v|
// is below u rho_v (rho_v the rounding scale of its misfit, u the unit
// roundoff of the misfit's precision) ends its search here with no step (the
// noise floor); ctl[kActive] counts the views that search.
__global__ void k_gn_direction(const double *__restrict__ g, const double *__restrict__ j2,
                               const double *__restrict__ rho, int V, double mu_rel, double alpha0, double unit,
                               const double *__restrict__ theta, double *__restrict__ d, double *__restrict__ alpha,
                               double *__restrict__ theta_trial, int *__restrict__ active, int *__restrict__ ctl)
{
    __shared__ int cnt[32];
    __shared__ double sh[40];
    double mx = 0.0;
    for (int v = threadIdx.x; v < V; v += blockDim.x) mx = fmax(mx, j2[v]);
    // block max
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, sh[i]);
        sh[32] = m;
    }
    __syncthreads();
    const double mu = mu_rel * fmax(sh[32], 1e-300);
    int mine = 0;
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
        const double dv = -g[v] / (j2[v] + mu);
        d[v] = dv;
        const bool on = !(alpha0 * fabs(g[v] * dv) < unit * rho[v]);
        alpha[v] = on ? alpha0 : 0.0;
        theta_trial[v] = on ? theta[v] + alpha0 * dv : theta[v];
        active[v] = on ? 1 : 0;
        mine += on ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0) cnt[threadIdx.x >> 5] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += cnt[i];
        ctl[kActive] = t;
        ctl[kArmijoDone] = t == 0;
    }
}

// Sums over the views, in a fixed order, of up to four per-view arrays (null
// entries give 0): out[q] = sum_v a_q[v].  One block.
__global__ void k_view_sums(const double *__restrict__ a0, const double *__restrict__ a1,
                            const double *__restrict__ a2, const double *__restrict__ a3, int V,
                            double *__restrict__ out)
{
    __shared__ double sh[40];
    const double *a[4] = {a0, a1, a2, a3};
    for (int q = 0; q < 4; ++q) {
        double s = 0.0;
        if (a[q])
            for (int v = threadIdx.x; v < V; v += blockDim.x) s += a[q][v];
        s = block_sum(s, sh);
        if (threadIdx.x == 0) out[q] = s;
    }
}

// Armijo test for the views still searching; shrinks alpha of the failures.
// A failure whose next first-order change alpha |g_v d_v| falls below u rho_v
// (the noise floor) ends its search with no step, as does a failure in the
// last round.  ctl[kArmijoDone] becomes 1 once no view searches; the trial
// kernels of the later rounds (and this kernel) then return at once.
__global__ void k_armijo(const double *__restrict__ f0, const double *__restrict__ ft, const double *__restrict__ g,
                         const double *__restrict__ d, const double *__restrict__ rho,
                         const double *__restrict__ theta, int V, double c1, double beta, double unit,
                         double *__restrict__ alpha, double *__restrict__ theta_trial, int *__restrict__ active,
                         int *__restrict__ ctl, int last)
{
    __shared__ int cnt[32];
    if (ctl[kArmijoDone]) return;
    int mine = 0;
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
        if (!active[v]) continue;
        if (ft[v] <= f0[v] + c1 * alpha[v] * g[v] * d[v]) {
            active[v] = 0;
        } else if (last) {  // no acceptable step: keep the old angle
            active[v] = 0;
            alpha[v] = 0.0;
            theta_trial[v] = theta[v];
        } else if ((alpha[v] * beta) * fabs(g[v] * d[v]) < unit * rho[v]) {  // noise floor: no step
            active[v] = 0;
            alpha[v] = 0.0;
            theta_trial[v] = theta[v];
        } else {
            alpha[v] *= beta;
            theta_trial[v] = theta[v] + alpha[v] * d[v];
            ++mine;
        }
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0) cnt[threadIdx.x >> 5] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += cnt[i];
        ctl[kActive] = t;
        ctl[kArmijoDone] = t == 0;
    }
}

// ---------------------------------------------------------------------------
// VarPro Gauss-Newton system (Sec. 4.2, Alg. "UPDATE-PARAM-VarPro")
// ---------------------------------------------------------------------------
// With the image restricted to span(V) (k columns), y(theta) the reduced
// solution, u = V y, r = H V y - b, s = P Psi V y, the sensitivity equation
// restricted to span(V) gives, for the angle of view j,
//   M y_j = -(G[:, j] + E[:, j]),  M = (HV)^T HV + lambda (P Psi V)^T (P Psi V),
//   G[c][j] = (H_j V_c)^T r,  E[c][j] = (H V_c)^T H_j u,
// and the Jacobian columns J_r[:, j] = H_j u + (HV) y_j, J_s[:, j] = (P Psi V) y_j
// (H_j = dH/dtheta_j, nonzero only in view j's samples).  Hence
//   J_r^T J_r + lambda J_s^T J_s = diag(|H_j u|^2) + E^T Y + Y^T E + Y^T M Y,
// a diagonal plus a rank-2k term: with U = [E; Y] (2k x V) and
// S = [[0, I], [I, M]] it is diag + U^T S U.  The damped system
// (diag + mu + U^T S U) d = -g is solved by the Woodbury identity with the
// 2k x 2k capacitance S^{-1} + U D^{-1} U^T, S^{-1} = [[-M, I], [I, 0]]
// (symmetric indefinite: Gaussian elimination with partial pivoting).
constexpr int kVpMax = 32;  // basis columns of the VarPro Gauss-Newton system

// Per-view dot products over view j's B samples: j2[j] = <a, a>_j,
// g[j] = <a, r>_j, E[c][j] = <(HV)_c, a>_j, where a = J_theta(u) 1 holds
// H_j u in view j's samples.  One CTA per view.
template <typename T>
__global__ void __launch_bounds__(128) k_view_dots(const T *__restrict__ HV, long long m, int k,
                                                   const T *__restrict__ a, const T *__restrict__ r, int V, int B,
                                                   double *__restrict__ E, double *__restrict__ j2,
                                                   double *__restrict__ g)
{
    __shared__ double red[4];
    for (int j = blockIdx.x; j < V; j += gridDim.x) {
        const size_t off = (size_t)j * B;
        for (int c = -2; c < k; ++c) {
            const T *x = c == -2 ? a : (c == -1 ? r : HV + (size_t)c * m);
            double s = 0.0;
            for (int q = threadIdx.x; q < B; q += blockDim.x) s += (double)a[off + q] * (double)x[off + q];
            s = warp_sum(s);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
            __syncthreads();
            if (threadIdx.x == 0) {
                const double t = (red[0] + red[1]) + (red[2] + red[3]);
                if (c == -2) j2[j] = t;
                else if (c == -1) g[j] = t;
                else E[(size_t)c * V + j] = t;
            }
            __syncthreads();
        }
    }
}

struct VpShared {
    static constexpr int kLd = kVpMax + 1;
    double M[kVpMax * kLd];                    // (HV)^T HV + lambda (P Psi V)^T (P Psi V)
    double L[kVpMax * kLd];                    // its Cholesky factor
    double C[2 * kVpMax][2 * kVpMax + 2];      // capacitance | right-hand side
    double z[2 * kVpMax];
    double red[40];
    double mu;
    int bad, piv;
};

// The damped Gauss-Newton direction d = -(J^T J + mu I)^{-1} g of the VarPro
// reduced objective, mu = mu_rel * max_j (J^T J)_jj, and gd = g . d.
// Y (k x V) and idel (V) are global work arrays written and read by this CTA.
// A numerically singular capacitance sets the breakdown flag and gives d = 0.
__global__ void __launch_bounds__(1024) k_varpro_direction(const double *__restrict__ GH,
                                                           const double *__restrict__ GP, double lam,
                                                           const double *__restrict__ E, const double *__restrict__ G,
                                                           const double *__restrict__ j2, const double *__restrict__ g,
                                                           int k, int V, double mu_rel, double *Y, double *idel,
                                                           double *__restrict__ d, double *__restrict__ gd_out,
                                                           int *__restrict__ ctl)
{
    extern __shared__ unsigned char smem_raw[];
    VpShared &S = *reinterpret_cast<VpShared *>(smem_raw);
    constexpr int kLd = VpShared::kLd;
    const int tid = threadIdx.x, nt = blockDim.x, K = 2 * k;
    if (tid == 0) S.bad = 0;
    for (int idx = tid; idx < k * k; idx += nt) {
        const int i = idx / k, l = idx % k;
        const double v = GH[i * kKMax + l] + lam * GP[i * kKMax + l];
        S.M[i * kLd + l] = v;
        S.L[i * kLd + l] = v;
    }
    __syncthreads();
    chol<VpShared::kLd>(S.L, k, &S.bad);
    __syncthreads();
    // Y[:, j] = -M^{-1} (G[:, j] + E[:, j]) by L z = -(G + E), L^T y = z; then
    // (J^T J)_jj = |H_j u|^2 + 2 E[:, j] . y + y^T M y, with y^T M y = |z|^2
    double dmax = 0.0;
    for (int j = tid; j < V; j += nt) {
        double z[kVpMax], yv[kVpMax];
        double zz = 0.0;
        for (int i = 0; i < k; ++i) {
            double s = -(G[(size_t)i * V + j] + E[(size_t)i * V + j]);
            for (int l = 0; l < i; ++l) s -= S.L[i * kLd + l] * z[l];
            z[i] = s / S.L[i * kLd + i];
            zz += z[i] * z[i];
        }
        double ey = 0.0;
        for (int i = k - 1; i >= 0; --i) {
            double s = z[i];
            for (int l = i + 1; l < k; ++l) s -= S.L[l * kLd + i] * yv[l];
            yv[i] = s / S.L[i * kLd + i];
            Y[(size_t)i * V + j] = yv[i];
            ey += E[(size_t)i * V + j] * yv[i];
        }
        dmax = fmax(dmax, j2[j] + 2.0 * ey + zz);
    }
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((tid & 31) == 0) S.red[tid >> 5] = dmax;
    __syncthreads();
    if (tid == 0) {
        double mx = 0.0;
        for (int i = 0; i < (nt >> 5); ++i) mx = fmax(mx, S.red[i]);
        S.mu = mu_rel * fmax(mx, 1e-300);
    }
    __syncthreads();
    for (int j = tid; j < V; j += nt) idel[j] = 1.0 / (j2[j] + S.mu);
    __syncthreads();  // Y and idel are visible to the whole CTA
    // capacitance C = S^{-1} + U D^{-1} U^T and right-hand side U D^{-1} g
    for (int idx = tid; idx < K * (K + 1); idx += nt) {
        const int p = idx / (K + 1), q = idx % (K + 1);
        const double *up = p < k ? E + (size_t)p * V : Y + (size_t)(p - k) * V;
        double s = 0.0;
        if (q < K) {
            const double *uq = q < k ? E + (size_t)q * V : Y + (size_t)(q - k) * V;
            for (int j = 0; j < V; ++j) s += up[j] * uq[j] * idel[j];
            if (p < k && q < k) s -= S.M[p * kLd + q];
            else if (q == p + k || p == q + k) s += 1.0;
        } else {
            for (int j = 0; j < V; ++j) s += up[j] * g[j] * idel[j];
        }
        S.C[p][q] = s;
    }
    __syncthreads();
    if (tid == 0) {
        double cmax = 0.0;
        for (int p = 0; p < K; ++p)
            for (int q = 0; q < K; ++q) cmax = fmax(cmax, fabs(S.C[p][q]));
        S.red[32] = cmax;
    }
    __syncthreads();
    const double cmax = S.red[32];
    for (int p = 0; p < K; ++p) {
        if (tid == 0) {
            int best = p;
            double bv = fabs(S.C[p][p]);
            for (int i = p + 1; i < K; ++i)
                if (fabs(S.C[i][p]) > bv) {
                    bv = fabs(S.C[i][p]);
                    best = i;
                }
            S.piv = best;
            if (!(bv > 1e-300 + 1e-15 * cmax)) S.bad |= 2;
        }
        __syncthreads();
        if (S.bad & 2) break;
        const int pv = S.piv;
        if (pv != p)
            for (int c = tid; c <= K; c += nt) {
                const double t = S.C[p][c];
                S.C[p][c] = S.C[pv][c];
                S.C[pv][c] = t;
            }
        __syncthreads();
        for (int i = p + 1 + tid; i < K; i += nt) S.z[i] = S.C[i][p] / S.C[p][p];
        __syncthreads();
        const int rows = K - p - 1, cols = K - p;  // rows p+1.., columns p+1..K (right-hand side included)
        for (int idx = tid; idx < rows * cols; idx += nt) {
            const int i = p + 1 + idx / cols, c = p + 1 + idx % cols;
            S.C[i][c] -= S.z[i] * S.C[p][c];
        }
        __syncthreads();
    }
    if (tid == 0 && !(S.bad & 2)) {
        for (int p = K - 1; p >= 0; --p) {
            double s = S.C[p][K];
            for (int c = p + 1; c < K; ++c) s -= S.C[p][c] * S.z[c];
            S.z[p] = s / S.C[p][p];
        }
    }
    __syncthreads();
    const bool bad = (S.bad & 2) != 0;
    // d = -(D^{-1} g - D^{-1} U^T C^{-1} U D^{-1} g)
    double gd = 0.0;
    for (int j = tid; j < V; j += nt) {
        double dj = 0.0;
        if (!bad) {
            double s = 0.0;
            for (int p = 0; p < k; ++p) s += E[(size_t)p * V + j] * S.z[p] + Y[(size_t)p * V + j] * S.z[k + p];
            dj = -(g[j] - s) * idel[j];
        }
        d[j] = dj;
        gd += g[j] * dj;
    }
    gd = block_sum(gd, S.red);
    if (tid == 0) {
        *gd_out = gd;
        if (S.bad) ctl[kBreakdown] = 1;
    }
}

// out = theta + alpha d
__global__ void k_theta_step(const double *__restrict__ theta, const double *__restrict__ d, double alpha, int V,
                             double *__restrict__ out)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x)
        out[v] = theta[v] + alpha * d[v];
}

}  // namespace solver
}  // namespace ctgb
