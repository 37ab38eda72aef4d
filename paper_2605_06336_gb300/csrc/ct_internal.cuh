// Internal declarations shared by the CUDA translation units of libctgb.
//
// Coordinates.  Every ray is marched in "march coordinates": for a view
// that samples once per image row (|cos| >= |sin|) the march index r is the
// row i and the in-row coordinate q is the column position u = x + (N-1)/2;
// for a view that samples once per column r is the column j and q is the row
// position t = (N-1)/2 - y, read from the transposed image.  In both cases
//     q(b, r) = h + s_b * qb + (r - h) * qr,   h = (N-1)/2,
// with s_b = b + n0 + phi (n0 integer, 0 <= phi < 1) the bin centre.  The
// kernels carry q in 64-bit fixed point with 48 fractional bits (kFracBits):
//     Q = Qc + (b + n0) * Qb + (2r - (N-1)) * Qh,
// Qc = h + phi*qb, Qb = qb, Qh = qr/2, each rounded once.  The cell floor(q)
// and the interpolation fraction come from integer shifts, so the cell
// choice agrees with an FP64 evaluation except within ~1e-11 pixels of a cell
// boundary, and exact coincidences at the image centre (the central ray of an
// odd-sized image meets the centre pixel exactly) stay exact.  That matters
// for the angle derivative, whose interpolation slope jumps at every cell
// boundary.
//
// Pair layouts.  The ray kernels read an image as "pairs": element c of row
// r holds (X[r][c], X[r][c+1]) for c = -2 .. N+1 (stored at c + 2, pitch
// Pp = N + 4 pairs), zero outside the image.  One 8-byte load then fetches
// both interpolation taps, and clamping the cell to [-2, N] keeps every load
// in bounds while rays outside the image read exact zeros.  The transpose
// operator reads sinograms the same way: pair b of view v holds
// (Y[v][b], Y[v][b+1]) for b = -2 .. B+1 (stored at b + 2, pitch Pb = B + 4
// rounded up to even, so that rows start on 16-byte boundaries).
//
// Interleaved images (FP32 forward, fwd_layout 1).  The forward of a batch
// may read its images from a second layout without the pair duplication:
// the batch is cut into groups of 4 images (a remainder of 2 or 3 gives one
// group of 2, an odd remainder one group of 1, in that order), and element
// c + 2 of row r holds X_k[r][c] of the group's w images side by side, for
// c = -2 .. N+1 (pitch Pp elements of w floats, zero outside the image).
// Group (k0, w) starts k0 * F * N * Pp floats into the buffer.  One 16-byte
// load at c and one at c + 1 then fetch both taps of 4 images, and a warp's
// rays touch half the bytes they touch in the pair layouts.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace ctgb {

constexpr int kFracBits = 48;
constexpr double kFixScale = 281474976710656.0;  // 2^48
constexpr int kMaxN = 4096;                      // keeps |q| * 2^48 inside int64
constexpr int kChunk = 32;                       // bins per warp work item
constexpr int kTile = 16;                        // transpose-operator pixel tile side
constexpr double kAllRowsBelow = 4e-3;           // |qr| below this: march every row

enum ViewFlags : int { kAllRows = 1, kValid = 2 };

// Per-view constants, rebuilt on the device from (theta, delta) whenever the
// angle or offset of the view changed since the previous call.
struct __align__(16) ViewGeo {
    long long Qc, Qb, Qh;  // h + phi*qb, qb, qr/2 in fixed point
    double beta0, c, s;    // transpose: bin coordinate of pixel (i,j) = beta0 + j*c - i*s
    double th, dl;         // the (theta, delta) the constants were built from
    double sb0d;           // s_b = sb0d + b (FP64 form)
    float alo, ahi, gam;   // rows with -1 < q < N lie between alo + b*gam and ahi + b*gam
    float w;               // 1/|cos| or 1/|sin|
    float dw;              // d w / d theta
    float gs, gh, gr;      // dq/dtheta (b, r) = (s_b*gs + gh) + r*gr
    float qbf;             // dq/ddelta = qb
    float sb0;             // s_b = sb0 + b
    int mode;              // 0: rows of X, 1: rows of X^T
    int frame;
    int flags;
    int n0;                // integer part of the bin-centre offset -(B-1)/2 + delta
    int gen;               // incremented at every rebuild (tables derived per view compare it)
};

// Launch shapes.  kb: images (or sinograms) per lane; split: warps sharing
// one ray (row segments, combined in shared memory) or thread groups sharing
// one pixel tile (view subsets, combined in shared memory).
// vw: view slots per CTA for the ray kernels (neighbouring views of the
// sorted view order, sharing the image band in L1 or shared memory).
// stage: 0 = gather through L1; 4 or 8 = rows per block of the band-staged
// FP32 march (vw 4 or 8).  There the forward's split is the number of CTAs
// that share one ray (row segments, combined by a second kernel); the
// derivative kernels march whole rays.  The staged transpose's split is the
// number of CTAs per pixel tile, one thread-block cluster.
struct Tuning {
    int fwd_kb = 8, fwd_split = 2, fwd_vw = 1;  // forward projection of a batch
    int adj_kb = 8, adj_split = 2;              // transpose of a batch
    int der_split = 4, der_vw = 1;              // JVP / VJP / Gauss-Newton terms
    int der_kb = 1;                             // images per lane of the batched derivative modes
    int fwd_stage = 0, der_stage = 0;
    int adj_stage = 0;  // 0: gather through L1; 8 or 16: views per shared-memory block of the
                        // staged FP32 transpose, whose adj_split is then CTAs per tile
    int fwd_layout = 0; // 1: the FP32 L1-gather forward (fwd_stage 0, fwd_kb 4 or 8, parallel
                        // beam) reads the interleaved images; 0: the pair images
};

// Group of image k in the interleaved layout of a batch of K: first image k0, width w.
__host__ __device__ inline void interleave_group(int k, int K, int &k0, int &w)
{
    const int n4 = K & ~3;
    if (k < n4) {
        k0 = k & ~3;
        w = 4;
    } else if (K - n4 >= 2 && k < n4 + 2) {
        k0 = n4;
        w = 2;
    } else {
        k0 = K - 1;
        w = 1;
    }
}

struct Handle {
    int N = 0, B = 0, V = 0, F = 1, max_batch = 1, precision = 0, device = 0;
    int Pp = 0, Pb = 0;  // pair pitches
    cudaStream_t stream = nullptr;
    std::vector<int> views_per_frame;
    ViewGeo *d_views = nullptr;
    int *d_fov = nullptr;     // frame of each view
    int *d_fstart = nullptr;  // first view of each frame
    int *d_fcount = nullptr;  // views of each frame
    int *d_flag = nullptr;    // device-side status bits
    int *d_order = nullptr;   // view order of the ray kernels (sorted by axis and slope)
    void *d_px = nullptr;     // pair images, rows of X:   (max_batch + 1) * F * N * Pp pairs
    void *d_pt = nullptr;     // pair images, rows of X^T: (max_batch + 1) * F * N * Pp pairs
    void *d_yp = nullptr;     // pair sinograms: max_batch * V * Pb pairs
    float *d_qx = nullptr;    // interleaved images, rows of X and of X^T: max_batch * F * N * Pp
    float *d_qt = nullptr;    // floats each, allocated when fwd_layout 1 is set (FP32 handles)
    double *d_partial = nullptr;  // per (image, view, chunk) reduction partials, 4 per item, max_batch images
    void *d_segpart = nullptr;    // segment partials of the staged forward (sinograms):
                                  // 3 * max_batch * max(V * B, F * N * N) floats, allocated
                                  // when a shape with several CTAs per ray is set
    int nchunks = 0;              // ceil(B / kChunk)
    double fan_D = 0.0;           // > 0: fan beam with the source at this distance (ct_fan.cu); 0: parallel
    void *d_rays = nullptr;       // fan beam: per-ray table, V * B entries
    void *d_fanview = nullptr;    // fan beam: per-view FP32 constants and march-axis bin ranges
    void *d_yi = nullptr;         // fan beam: sinograms interleaved in blocks of 8, [k / 8][V][B][k % 8]
    // Batch sizes whose forward (adjoint) inputs are still laid out in the
    // handle from the last ct_forward (ct_adjoint) call: ct_forward_repeat
    // (ct_adjoint_repeat) may rerun the projection kernel alone.  Any other
    // call that may change the view table or the pair layouts clears them.
    int fwd_ready = 0, adj_ready = 0;
    // Images (of F frames) whose pair layouts are current from the last
    // operator call that took images: a later call may pass X = null to use
    // them again (its batch at most this).  The solvers and the autotuner,
    // which lay out images of their own, clear it.
    int img_ready = 0;
    int img_kind = 0;  // the layout holding them: 0 pair images, 1 interleaved images
    int num_sms = 0;
    Tuning tune;
};

// Kernel launchers.  All launch on h.stream and return the launch status.
// `skip` (nullable, device) lets a caller that runs a fixed launch sequence
// (the solver's predicated Enlarge steps) turn a launch into a no-op: when
// *skip != 0 the kernel returns at once.
cudaError_t launch_view_setup(const Handle &h, const double *theta, const double *delta,
                              const int *skip = nullptr);
// The same step with the per-view constants spread over many CTAs (for large
// view counts) and the view order rebuilt by one more CTA when a view
// changed; *changed (device, zero on entry) is the flag between the two and
// is zero again afterwards.
cudaError_t launch_view_setup_wide(const Handle &h, const double *theta, const double *delta, int *changed,
                                   const int *skip = nullptr);

// Layout kernels.  With theta non-null the same launch also runs the view-table
// step of the call (what launch_view_setup does), in one extra CTA.
template <typename T>
cudaError_t launch_pairs_img(const Handle &h, const T *X, int nimg, const int *skip = nullptr,
                             const double *theta = nullptr, const double *delta = nullptr);
template <typename T>
cudaError_t launch_pairs_sino(const Handle &h, const T *Y, int nsino, const int *skip = nullptr,
                              const double *theta = nullptr, const double *delta = nullptr);
// Layout the forward projection reads (pair images of X and X^T).
template <typename T>
cudaError_t launch_prep_forward(const Handle &h, const T *X, int nimg, const int *skip = nullptr,
                                const double *theta = nullptr, const double *delta = nullptr);
// Interleaved images of X and X^T for a batch of `batch` images of F frames
// (into d_qx / d_qt), with the view-table step as in launch_pairs_img.
cudaError_t launch_interleave_img(const Handle &h, const float *X, int batch, const double *theta = nullptr,
                                  const double *delta = nullptr, const int *skip = nullptr);
// The pair images of the first `batch` images from the interleaved ones.
cudaError_t launch_interleaved_to_pairs(const Handle &h, int batch);

// stage > 0 (FP32 only): rows per shared-memory block of the band-staged
// march (ct_band.cu); 0: gathers through L1.  interleaved (FP32, parallel
// beam): the first `batch` images of the interleaved layout of a batch of
// layout_batch (>= batch) are read from d_qx / d_qt, 8 per lane when kb is 8,
// else 4 (stage is then ignored).
template <typename T>
cudaError_t launch_forward(const Handle &h, T *Y, int batch, int kb, int split, int vw, int stage,
                           const int *skip = nullptr, bool interleaved = false, int layout_batch = 0);
template <typename T>
cudaError_t launch_adjoint(const Handle &h, T *X, int batch, int kb, int split, int stage,
                           const int *skip = nullptr);
// Staged FP32 transpose (ct_adj_band.cu); adj_band_ok tells whether a shape can run on this handle.
bool adj_band_ok(const Handle &h, int stage, int segs);
cudaError_t launch_adjoint_band(const Handle &h, float *X, int batch, int kb, int segs, int stage, const int *skip);
// Derivative modes on `batch` images laid out in the pair buffers (kb images
// per lane: 1, 2 or 4), one launch of the ray kernel plus (VJP, GN) the
// per-view reduction.  JVP: image k uses dtheta + k * dir_stride (0: one
// direction for all) and writes dY + k * V * B.  VJP: image k reads
// R + k * r_stride (0: one r for all) and writes gtheta + k * V, or with sum
// one [V] vector summing the images in order.  GN: image k reads
// bdata + k * V * B and writes [k][V] outputs; rscale (nullable) receives
// sum_b |r_b| (|(H x)_b| + |b_b|) per view, the rounding scale of the misfit.
template <typename T>
cudaError_t launch_jvp(const Handle &h, const double *dtheta, const double *ddelta, T *dY, int split, int vw,
                       int stage, int batch = 1, int kb = 1, long long dir_stride = 0);
template <typename T>
cudaError_t launch_vjp(const Handle &h, const T *R, double *gtheta, double *gdelta, int split, int vw, int stage,
                       int batch = 1, int kb = 1, long long r_stride = 0, int sum = 0);
template <typename T>
cudaError_t launch_gn(const Handle &h, const T *bdata, T *res, double *grad, double *jnorm2, double *fval,
                      int split, int vw, int stage, const int *view_mask = nullptr, const int *skip = nullptr,
                      int batch = 1, int kb = 1, double *rscale = nullptr);

// Fan beam (ct_fan.cu).  launch_fan_rays rebuilds the per-ray table from the
// view table; every launcher that brings the view table up to date runs it
// on a fan-beam handle.  The transpose of a fan-beam handle reads the pair
// sinograms like the parallel-beam one.
size_t fan_ray_bytes(int precision);
size_t fan_view_bytes();
// YI[k / 8][v][b][k % 8] = Y[k][v][b]: the 8 sinograms of a block at one bin
// are contiguous for the fan-beam transpose (ct_fan.cu).
template <typename T> cudaError_t launch_fan_sino(const Handle &h, const T *Y, int nsino, const int *skip);
cudaError_t launch_fan_rays(const Handle &h, const int *skip);
template <typename T>
cudaError_t launch_fan_adjoint(const Handle &h, T *X, int batch, int kb, int split, const int *skip);

}  // namespace ctgb
