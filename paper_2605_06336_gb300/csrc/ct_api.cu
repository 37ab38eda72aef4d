// C ABI of libctgb (declared in include/ctgb.h): argument checks, handle
// workspaces and the launch sequence of each operator call.
#include <cuda_runtime.h>

#include <cstdio>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ctgb.h"
#include "ct_internal.cuh"

struct ct_handle {
    ctgb::Handle h;
};

namespace {

thread_local char g_cuda_msg[256] = "no error";

int cuda_fail(cudaError_t e)
{
    std::snprintf(g_cuda_msg, sizeof(g_cuda_msg), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return CT_ERR_CUDA;
}

#define CT_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_);   \
    } while (0)

size_t elem_size(const ctgb::Handle &h) { return h.precision ? sizeof(double) : sizeof(float); }

void free_all(ctgb::Handle &h)
{
    cudaFree(h.d_views);
    cudaFree(h.d_fov);
    cudaFree(h.d_fstart);
    cudaFree(h.d_fcount);
    cudaFree(h.d_flag);
    cudaFree(h.d_order);
    cudaFree(h.d_px);
    cudaFree(h.d_pt);
    cudaFree(h.d_yp);
    cudaFree(h.d_partial);
    cudaFree(h.d_segpart);
    cudaFree(h.d_rays);
    cudaFree(h.d_fanview);
    cudaFree(h.d_yi);
    cudaFree(h.d_qx);
    cudaFree(h.d_qt);
    h.d_qx = h.d_qt = nullptr;
    h.d_rays = nullptr;
    h.d_fanview = nullptr;
    h.d_yi = nullptr;
    h.d_views = nullptr;
    h.d_fov = h.d_fstart = h.d_fcount = h.d_flag = h.d_order = nullptr;
    h.d_px = h.d_pt = h.d_yp = nullptr;
    h.d_partial = nullptr;
    h.d_segpart = nullptr;
}

// The pair layouts of the call's images and the view table.  X == null: the
// layouts left by the previous call that took images are current (the caller
// checked h.img_ready; interleaved ones, left by a forward, are turned into
// pair layouts first); only the view table is brought up to date.
template <typename T>
cudaError_t prep_images(ctgb::Handle &h, const T *X, int nimg, const double *theta, const double *delta)
{
    if (X) {
        h.img_kind = 0;
        return ctgb::launch_pairs_img<T>(h, X, nimg, nullptr, theta, delta);
    }
    if (h.img_kind == 1) {
        const cudaError_t e = ctgb::launch_interleaved_to_pairs(h, h.img_ready);
        if (e != cudaSuccess) return e;
        h.img_kind = 0;
    }
    return ctgb::launch_view_setup(h, theta, delta);
}

// Whether a forward that takes images lays them out interleaved (the tuning
// asks for it and the handle can: FP32, parallel beam, workspace present).
bool forward_interleaves(const ctgb::Handle &h)
{
    return h.tune.fwd_layout == 1 && h.precision == 0 && h.fan_D == 0.0 && h.d_qx;
}

template <typename T>
int do_forward(ctgb::Handle &h, const double *theta, const double *delta, const void *X, void *Y, int batch)
{
    // X == null reads whichever layout the previous call left
    const bool inter = X ? forward_interleaves(h) : h.img_kind == 1;
    if (inter && X) {
        CT_CUDA(ctgb::launch_interleave_img(h, (const float *)X, batch, theta, delta));
        h.img_kind = 1;
    } else if (inter) {
        CT_CUDA(ctgb::launch_view_setup(h, theta, delta));
    } else {
        CT_CUDA(prep_images<T>(h, (const T *)X, batch * h.F, theta, delta));
    }
    CT_CUDA(ctgb::launch_forward<T>(h, (T *)Y, batch, h.tune.fwd_kb, h.tune.fwd_split, h.tune.fwd_vw, h.tune.fwd_stage,
                                    nullptr, inter, X ? batch : h.img_ready));
    return CT_OK;
}

template <typename T>
int do_adjoint(ctgb::Handle &h, const double *theta, const double *delta, const void *Y, void *X, int batch)
{
    CT_CUDA(ctgb::launch_pairs_sino<T>(h, (const T *)Y, batch, nullptr, theta, delta));
    CT_CUDA(ctgb::launch_adjoint<T>(h, (T *)X, batch, h.tune.adj_kb, h.tune.adj_split, h.tune.adj_stage));
    return CT_OK;
}

template <typename T>
int do_jac(ctgb::Handle &h, const double *theta, const double *delta, const void *x, const double *dtheta,
           const double *ddelta, void *dy)
{
    CT_CUDA(prep_images<T>(h, (const T *)x, h.F, theta, delta));
    CT_CUDA(ctgb::launch_jvp<T>(h, dtheta, ddelta, (T *)dy, h.tune.der_split, h.tune.der_vw, h.tune.der_stage));
    return CT_OK;
}

template <typename T>
int do_jacT(ctgb::Handle &h, const double *theta, const double *delta, const void *x, const void *r, double *gtheta,
            double *gdelta)
{
    CT_CUDA(prep_images<T>(h, (const T *)x, h.F, theta, delta));
    CT_CUDA(ctgb::launch_vjp<T>(h, (const T *)r, gtheta, gdelta, h.tune.der_split, h.tune.der_vw, h.tune.der_stage));
    return CT_OK;
}

template <typename T>
int do_jac_batch(ctgb::Handle &h, const double *theta, const double *delta, const void *X, const double *dtheta,
                 const double *ddelta, void *dY, int batch, int flags)
{
    const long long dstride = (flags & CT_BATCH_PER_IMAGE_DIRECTION) ? h.V : 0;
    CT_CUDA(prep_images<T>(h, (const T *)X, batch * h.F, theta, delta));
    CT_CUDA(ctgb::launch_jvp<T>(h, dtheta, ddelta, (T *)dY, h.tune.der_split, h.tune.der_vw, h.tune.der_stage, batch,
                                h.tune.der_kb, dstride));
    return CT_OK;
}

template <typename T>
int do_jacT_batch(ctgb::Handle &h, const double *theta, const double *delta, const void *X, const void *R,
                  double *gtheta, double *gdelta, int batch, int flags)
{
    const long long rstride = (flags & CT_BATCH_SHARED_R) ? 0 : (long long)h.V * h.B;
    CT_CUDA(prep_images<T>(h, (const T *)X, batch * h.F, theta, delta));
    CT_CUDA(ctgb::launch_vjp<T>(h, (const T *)R, gtheta, gdelta, h.tune.der_split, h.tune.der_vw, h.tune.der_stage,
                                batch, h.tune.der_kb, rstride, (flags & CT_BATCH_SUM) ? 1 : 0));
    return CT_OK;
}

template <typename T>
int do_gn_batch(ctgb::Handle &h, const double *theta, const double *delta, const void *X, const void *bdata,
                void *res, double *grad, double *jnorm2, double *fval, int batch)
{
    CT_CUDA(prep_images<T>(h, (const T *)X, batch * h.F, theta, delta));
    CT_CUDA(ctgb::launch_gn<T>(h, (const T *)bdata, (T *)res, grad, jnorm2, fval, h.tune.der_split, h.tune.der_vw,
                               h.tune.der_stage, nullptr, nullptr, batch, h.tune.der_kb));
    return CT_OK;
}

template <typename T>
int do_gn(ctgb::Handle &h, const double *theta, const double *delta, const void *x, const void *bdata, void *res,
          double *grad, double *jnorm2, double *fval)
{
    CT_CUDA(prep_images<T>(h, (const T *)x, h.F, theta, delta));
    CT_CUDA(ctgb::launch_gn<T>(h, (const T *)bdata, (T *)res, grad, jnorm2, fval, h.tune.der_split, h.tune.der_vw,
                                  h.tune.der_stage));
    return CT_OK;
}

// Workspace of the staged forward with several CTAs per ray (segment
// partials), allocated the first time such a shape is set.
int ensure_seg_partials(ctgb::Handle &h)
{
    if (h.d_segpart || h.precision != 0) return CT_OK;
    const size_t per = std::max((size_t)h.V * h.B, (size_t)h.F * h.N * h.N);
    const size_t bytes = sizeof(float) * 3 * (size_t)h.max_batch * per;
    if (cudaMalloc(&h.d_segpart, bytes) != cudaSuccess) {
        cudaGetLastError();
        h.d_segpart = nullptr;
        return CT_ERR_OOM;
    }
    return CT_OK;
}

// Workspace of the interleaved forward images, allocated the first time that
// layout is set (FP32 parallel-beam handles).
int ensure_interleaved(ctgb::Handle &h)
{
    if (h.d_qx) return CT_OK;
    if (h.precision != 0 || h.fan_D > 0.0) return CT_ERR_ARG;
    const size_t bytes = sizeof(float) * (size_t)h.max_batch * h.F * h.N * h.Pp;
    if (cudaMalloc(&h.d_qx, bytes) != cudaSuccess || cudaMalloc(&h.d_qt, bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h.d_qx);
        cudaFree(h.d_qt);
        h.d_qx = h.d_qt = nullptr;
        return CT_ERR_OOM;
    }
    return CT_OK;
}

// Default launch shapes before (or without) autotuning: enough warps per SM
// for the small workloads, batch folding for the large ones.
void default_tuning(ctgb::Handle &h)
{
    const int kb = h.max_batch >= 8 ? 8 : (h.max_batch >= 4 ? 4 : (h.max_batch >= 2 ? 2 : 1));
    h.tune.fwd_kb = std::min(kb, 4);
    h.tune.adj_kb = std::min(kb, 4);
    const long long rays = (long long)h.V * h.nchunks;  // warps per image
    h.tune.fwd_split = rays >= 16LL * h.num_sms ? 2 : 4;
    h.tune.adj_split = 2;
    h.tune.der_split = rays >= 32LL * h.num_sms ? 2 : 4;
    h.tune.fwd_vw = 2;
    h.tune.der_vw = 2;
    h.tune.der_kb = std::min(kb, 4);
    if (h.fan_D > 0.0) {
        // fan-beam transpose: one candidate search per pixel and view serves
        // every sinogram of a thread; two view groups per pixel keep the warps up
        h.tune.adj_kb = kb;
        h.tune.adj_split = 2;
    }
}

// Time one configuration: median over `reps` launches issued back to back
// (the GPU never idles between them, so its clock stays up), after two
// warm-up launches.
template <typename F> float time_config(cudaStream_t s, F &&launch, int reps = 9)
{
    std::vector<cudaEvent_t> ev(reps + 1);
    for (auto &e : ev) cudaEventCreate(&e);
    launch();
    launch();
    cudaEventRecord(ev[0], s);
    for (int r = 0; r < reps; ++r) {
        launch();
        cudaEventRecord(ev[r + 1], s);
    }
    cudaEventSynchronize(ev[reps]);
    std::vector<float> ms(reps);
    for (int r = 0; r < reps; ++r) cudaEventElapsedTime(&ms[r], ev[r], ev[r + 1]);
    for (auto &e : ev) cudaEventDestroy(e);
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
}

// About `target_ms` of back-to-back launches: the SM clock ramps up under
// sustained load, and the candidates timed first would otherwise see a
// lower clock than the later ones.
template <typename F> void clock_warmup(cudaStream_t s, F &&launch, float target_ms = 150.0f)
{
    const float one = std::max(time_config(s, launch, 3), 1e-3f);
    const int n = std::min(20000, (int)(target_ms / one) + 1);
    for (int i = 0; i < n; ++i) launch();
    cudaStreamSynchronize(s);
}

template <typename T> int autotune_impl(ctgb::Handle &h)
{
    // Representative inputs: evenly spaced angles, zero images and sinograms
    // (values do not change the timing), a scratch output.  Every candidate
    // is timed together with the layout kernel that precedes it in an
    // operator call, so its inputs are as warm in L2 as they are there.
    std::vector<double> th(h.V);
    for (int v = 0; v < h.V; ++v) th[v] = 3.14159265358979 * (v + 0.37) / h.V;
    double *d_th = nullptr, *d_g = nullptr;
    void *d_out = nullptr, *d_in = nullptr;
    const size_t out_elems = std::max((size_t)h.max_batch * h.V * h.B, (size_t)h.max_batch * h.F * h.N * h.N);
    if (cudaMalloc(&d_th, sizeof(double) * h.V) != cudaSuccess ||
        cudaMalloc(&d_g, sizeof(double) * h.V) != cudaSuccess ||
        cudaMalloc(&d_out, out_elems * sizeof(T)) != cudaSuccess ||
        cudaMalloc(&d_in, out_elems * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_th);
        cudaFree(d_g);
        cudaFree(d_out);
        cudaFree(d_in);
        return CT_ERR_OOM;
    }
    const T *X = (const T *)d_in;
    int rc = CT_OK;
    do {
        cudaError_t e = cudaMemcpy(d_th, th.data(), sizeof(double) * h.V, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_in, 0, out_elems * sizeof(T), h.stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_g, 0, sizeof(double) * h.V, h.stream);
        if (e == cudaSuccess) e = ctgb::launch_view_setup(h, d_th, nullptr);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h.stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(e);
            break;
        }
        const int K = h.max_batch;
        float best = 1e30f;
        ctgb::Tuning t = h.tune;
        clock_warmup(h.stream, [&] {
            ctgb::launch_prep_forward<T>(h, X, K * h.F);
            ctgb::launch_forward<T>(h, (T *)d_out, K, t.fwd_kb, t.fwd_split, t.fwd_vw, 0);
        });
        // L1-gather shapes (stage 0), then band-staged ones (FP32: stage = rows per block)
        const bool fp32 = h.precision == 0;
        for (int kb : {1, 2, 4, 8}) {
            if (kb > K) continue;
            for (int sp : {1, 2, 4, 8}) {
                for (int vw : {1, 2, 4, 8}) {
                    if (sp * vw > 16) continue;
                    const float ms = time_config(h.stream, [&] {
                        ctgb::launch_prep_forward<T>(h, X, K * h.F);
                        ctgb::launch_forward<T>(h, (T *)d_out, K, kb, sp, vw, 0);
                    });
                    if (ms < best) {
                        best = ms;
                        t.fwd_kb = kb;
                        t.fwd_split = sp;
                        t.fwd_vw = vw;
                        t.fwd_stage = 0;
                        t.fwd_layout = 0;
                    }
                }
            }
            // the same shapes reading the interleaved images (FP32 parallel beam, 4 or 8 per lane)
            if ((kb == 4 || kb == 8) && fp32 && h.fan_D == 0.0 && ensure_interleaved(h) == CT_OK) {
                for (int sp : {1, 2, 4, 8}) {
                    for (int vw : {1, 2, 4, 8}) {
                        if (sp * vw > 16) continue;
                        const float ms = time_config(h.stream, [&] {
                            ctgb::launch_interleave_img(h, (const float *)X, K);
                            ctgb::launch_forward<T>(h, (T *)d_out, K, kb, sp, vw, 0, nullptr, true, K);
                        });
                        if (ms < best) {
                            best = ms;
                            t.fwd_kb = kb;
                            t.fwd_split = sp;
                            t.fwd_vw = vw;
                            t.fwd_stage = 0;
                            t.fwd_layout = 1;
                        }
                    }
                }
            }
            for (int st : {4, 8}) {
                for (int vw : {4, 8}) {
                    for (int sp : {1, 2, 4}) {
                        if (!fp32 || (sp > 1 && ensure_seg_partials(h) != CT_OK)) continue;
                        const float ms = time_config(h.stream, [&] {
                            ctgb::launch_prep_forward<T>(h, X, K * h.F);
                            ctgb::launch_forward<T>(h, (T *)d_out, K, kb, sp, vw, st);
                        });
                        if (ms < best) {
                            best = ms;
                            t.fwd_kb = kb;
                            t.fwd_split = sp;
                            t.fwd_vw = vw;
                            t.fwd_stage = st;
                            t.fwd_layout = 0;
                        }
                    }
                }
            }
        }
        best = 1e30f;
        for (int kb : {1, 2, 4, 8}) {
            if (kb > K) continue;
            for (int st : {0, 8, 16}) {
                for (int sp : {1, 2, 4}) {
                    if (st > 0 && (!fp32 || !ctgb::adj_band_ok(h, st, sp)))
                        continue;
                    const float ms = time_config(h.stream, [&] {
                        ctgb::launch_pairs_sino<T>(h, X, K);
                        ctgb::launch_adjoint<T>(h, (T *)d_out, K, kb, sp, st);
                    });
                    if (ms < best) {
                        best = ms;
                        t.adj_kb = kb;
                        t.adj_split = sp;
                        t.adj_stage = st;
                    }
                }
            }
        }
        best = 1e30f;
        for (int sp : {1, 2, 4, 8}) {
            for (int vw : {1, 2, 4, 8}) {
                if (sp * vw > 16) continue;
                const float ms = time_config(h.stream, [&] {
                    ctgb::launch_pairs_img<T>(h, X, h.F);
                    ctgb::launch_jvp<T>(h, d_g, nullptr, (T *)d_out, sp, vw, 0);
                });
                if (ms < best) {
                    best = ms;
                    t.der_split = sp;
                    t.der_vw = vw;
                    t.der_stage = 0;
                }
            }
        }
        for (int st : {4, 8}) {
            for (int vw : {4, 8}) {
                if (!fp32) continue;
                const float ms = time_config(h.stream, [&] {
                    ctgb::launch_pairs_img<T>(h, X, h.F);
                    ctgb::launch_jvp<T>(h, d_g, nullptr, (T *)d_out, 1, vw, st);
                });
                if (ms < best) {
                    best = ms;
                    t.der_split = 1;
                    t.der_vw = vw;
                    t.der_stage = st;
                }
            }
        }
        // images per lane of the batched derivative modes, on the whole batch at
        // the chosen split / views per CTA (per image: the single-image time above)
        if (K > 1) {
            best = 1e30f;
            for (int kb : {1, 2, 4}) {
                if (kb > K) continue;
                const float ms = time_config(h.stream, [&] {
                    ctgb::launch_pairs_img<T>(h, X, K * h.F);
                    ctgb::launch_jvp<T>(h, d_g, nullptr, (T *)d_out, t.der_split, t.der_vw, t.der_stage, K, kb);
                });
                if (ms < best) {
                    best = ms;
                    t.der_kb = kb;
                }
            }
        }
        e = cudaStreamSynchronize(h.stream);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_fail(e);
            break;
        }
        h.tune = t;
    } while (0);
    cudaFree(d_th);
    cudaFree(d_g);
    cudaFree(d_out);
    cudaFree(d_in);
    // the view table now holds the tuning angles; force a rebuild on the next call
    cudaMemsetAsync(h.d_views, 0, sizeof(ctgb::ViewGeo) * h.V, h.stream);
    return rc;
}

}  // namespace

// After an operator call that took images (X) or reused the current layouts
// (X == null): the handle's layouts now hold the call's `batch` images, or
// (after an error) nothing usable.
int images_laid_out(ctgb::Handle &h, const void *X, int batch, int rc)
{
    if (rc != CT_OK) h.img_ready = 0;
    else if (X) h.img_ready = batch;
    return rc;
}

extern "C" {

int ct_init(const ct_geom *g, void *cuda_stream, ct_handle **out)
{
    if (!g || !out) return CT_ERR_ARG;
    *out = nullptr;
    if (g->N < 2 || g->N > ctgb::kMaxN || g->B < 1 || g->n_views < 1 || g->n_frames < 1 || g->max_batch < 1 ||
        (g->precision != 0 && g->precision != 1))
        return CT_ERR_ARG;
    // fan beam: the source must lie outside the disc that holds the image and
    // the detector line, with two pixels to spare: the fan is then narrower than
    // 90 degrees (one change of march axis per view at most) and the projective
    // map of the transpose's candidate search stays positive on every pixel and
    // its one-pixel neighbourhood (image depth at most N / sqrt(2) + sqrt(2))
    if (!(g->source_distance == 0.0 ||
          (g->source_distance > 0.0 && std::isfinite(g->source_distance) &&
           g->source_distance > 0.75 * std::max((double)g->N, (double)g->B) + 2.0)))
        return CT_ERR_ARG;
    std::vector<int> vpf;
    if (g->views_per_frame) {
        long long sum = 0;
        for (int f = 0; f < g->n_frames; ++f) {
            if (g->views_per_frame[f] < 0) return CT_ERR_ARG;
            vpf.push_back(g->views_per_frame[f]);
            sum += g->views_per_frame[f];
        }
        if (sum != g->n_views) return CT_ERR_ARG;
    } else {
        if (g->n_frames != 1) return CT_ERR_ARG;
        vpf.push_back(g->n_views);
    }
    ct_handle *H = new (std::nothrow) ct_handle();
    if (!H) return CT_ERR_OOM;
    ctgb::Handle &h = H->h;
    h.N = g->N;
    h.B = g->B;
    h.V = g->n_views;
    h.F = g->n_frames;
    h.max_batch = g->max_batch;
    h.precision = g->precision;
    h.stream = (cudaStream_t)cuda_stream;
    h.views_per_frame = vpf;
    h.nchunks = (h.B + ctgb::kChunk - 1) / ctgb::kChunk;
    h.Pp = h.N + 4;
    h.Pb = (h.B + 5) & ~1;  // B + 4 rounded up to even: sinogram pair rows start on 16-byte boundaries
    h.fan_D = g->source_distance;
    int rc = CT_OK;
    do {
        cudaError_t e = cudaGetDevice(&h.device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h.num_sms, cudaDevAttrMultiProcessorCount, h.device);
        if (e != cudaSuccess) {
            rc = cuda_fail(e);
            break;
        }
        std::vector<int> fov(h.V), fstart(h.F), fcount(h.F);
        int v = 0;
        for (int f = 0; f < h.F; ++f) {
            fstart[f] = v;
            fcount[f] = vpf[f];
            for (int k = 0; k < vpf[f]; ++k) fov[v++] = f;
        }
        const size_t pair_bytes = 2 * elem_size(h);
        const size_t img_pairs = (size_t)(h.max_batch + 1) * h.F * h.N * h.Pp;
        const size_t sino_pairs = (size_t)h.max_batch * h.V * h.Pb;
        bool ok = cudaMalloc(&h.d_views, sizeof(ctgb::ViewGeo) * h.V) == cudaSuccess &&
                  cudaMalloc(&h.d_fov, sizeof(int) * h.V) == cudaSuccess &&
                  cudaMalloc(&h.d_fstart, sizeof(int) * h.F) == cudaSuccess &&
                  cudaMalloc(&h.d_fcount, sizeof(int) * h.F) == cudaSuccess &&
                  cudaMalloc(&h.d_flag, sizeof(int)) == cudaSuccess &&
                  cudaMalloc(&h.d_order, sizeof(int) * h.V) == cudaSuccess &&
                  cudaMalloc(&h.d_px, img_pairs * pair_bytes) == cudaSuccess &&
                  cudaMalloc(&h.d_pt, img_pairs * pair_bytes) == cudaSuccess &&
                  cudaMalloc(&h.d_yp, sino_pairs * pair_bytes) == cudaSuccess &&
                  cudaMalloc(&h.d_partial, sizeof(double) * 4 * (size_t)h.max_batch * h.V * h.nchunks) ==
                      cudaSuccess &&
                  (h.fan_D == 0.0 ||
                   (cudaMalloc(&h.d_rays, ctgb::fan_ray_bytes(h.precision) * (size_t)h.V * h.B) == cudaSuccess &&
                    cudaMalloc(&h.d_fanview, ctgb::fan_view_bytes() * (size_t)h.V) == cudaSuccess &&
                    cudaMalloc(&h.d_yi, elem_size(h) * 8 * (size_t)((h.max_batch + 7) / 8) * h.V * h.B) ==
                        cudaSuccess));
        if (!ok) {
            cudaGetLastError();
            rc = CT_ERR_OOM;
            break;
        }
        e = cudaMemcpy(h.d_fov, fov.data(), sizeof(int) * h.V, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h.d_fstart, fstart.data(), sizeof(int) * h.F, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h.d_fcount, fcount.data(), sizeof(int) * h.F, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(h.d_flag, 0, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(h.d_views, 0, sizeof(ctgb::ViewGeo) * h.V);
        if (e == cudaSuccess) e = cudaMemset(h.d_px, 0, img_pairs * pair_bytes);
        if (e == cudaSuccess) e = cudaMemset(h.d_pt, 0, img_pairs * pair_bytes);
        if (e == cudaSuccess) e = cudaMemset(h.d_yp, 0, sino_pairs * pair_bytes);
        // fan beam: generation 0 marks every ray and view entry as not built (views start at 1)
        if (e == cudaSuccess && h.d_rays)
            e = cudaMemset(h.d_rays, 0, ctgb::fan_ray_bytes(h.precision) * (size_t)h.V * h.B);
        if (e == cudaSuccess && h.d_fanview) e = cudaMemset(h.d_fanview, 0, ctgb::fan_view_bytes() * (size_t)h.V);
        if (e != cudaSuccess) {
            rc = cuda_fail(e);
            break;
        }
    } while (0);
    if (rc != CT_OK) {
        free_all(h);
        delete H;
        return rc;
    }
    default_tuning(h);
    *out = H;
    return CT_OK;
}

void ct_destroy(ct_handle *H)
{
    if (!H) return;
    cudaStreamSynchronize(H->h.stream);
    free_all(H->h);
    delete H;
}

int ct_forward(ct_handle *H, const double *theta, const double *delta, const void *X, void *Y, int batch)
{
    if (!H || !theta || !Y || batch < 1 || batch > H->h.max_batch || (!X && batch > H->h.img_ready))
        return CT_ERR_ARG;
    H->h.fwd_ready = H->h.adj_ready = 0;
    const int rc = H->h.precision ? do_forward<double>(H->h, theta, delta, X, Y, batch)
                                  : do_forward<float>(H->h, theta, delta, X, Y, batch);
    if (rc == CT_OK) H->h.fwd_ready = batch;
    return images_laid_out(H->h, X, batch, rc);
}

int ct_forward_repeat(ct_handle *H, void *Y, int batch)
{
    if (!H || !Y || batch < 1 || batch > H->h.fwd_ready) return CT_ERR_ARG;
    ctgb::Handle &h = H->h;
    if (h.precision)
        CT_CUDA(ctgb::launch_forward<double>(h, (double *)Y, batch, h.tune.fwd_kb, h.tune.fwd_split, h.tune.fwd_vw,
                                             h.tune.fwd_stage));
    else
        CT_CUDA(ctgb::launch_forward<float>(h, (float *)Y, batch, h.tune.fwd_kb, h.tune.fwd_split, h.tune.fwd_vw,
                                            h.tune.fwd_stage, nullptr, h.img_kind == 1, h.img_ready));
    return CT_OK;
}

int ct_adjoint_repeat(ct_handle *H, void *X, int batch)
{
    if (!H || !X || batch < 1 || batch > H->h.adj_ready) return CT_ERR_ARG;
    ctgb::Handle &h = H->h;
    if (h.precision)
        CT_CUDA(ctgb::launch_adjoint<double>(h, (double *)X, batch, h.tune.adj_kb, h.tune.adj_split, h.tune.adj_stage));
    else
        CT_CUDA(ctgb::launch_adjoint<float>(h, (float *)X, batch, h.tune.adj_kb, h.tune.adj_split, h.tune.adj_stage));
    return CT_OK;
}

int ct_adjoint(ct_handle *H, const double *theta, const double *delta, const void *Y, void *X, int batch)
{
    if (!H || !theta || !X || !Y || batch < 1 || batch > H->h.max_batch) return CT_ERR_ARG;
    H->h.fwd_ready = H->h.adj_ready = 0;
    const int rc = H->h.precision ? do_adjoint<double>(H->h, theta, delta, Y, X, batch)
                                  : do_adjoint<float>(H->h, theta, delta, Y, X, batch);
    if (rc == CT_OK) H->h.adj_ready = batch;
    return rc;
}

int ct_jac(ct_handle *H, const double *theta, const double *delta, const void *x, const double *dtheta,
           const double *ddelta, void *dy)
{
    if (!H || !theta || (!x && H->h.img_ready < 1) || !dtheta || !dy) return CT_ERR_ARG;
    H->h.fwd_ready = H->h.adj_ready = 0;
    return images_laid_out(H->h, x, 1,
                           H->h.precision ? do_jac<double>(H->h, theta, delta, x, dtheta, ddelta, dy)
                                          : do_jac<float>(H->h, theta, delta, x, dtheta, ddelta, dy));
}

int ct_jacT(ct_handle *H, const double *theta, const double *delta, const void *x, const void *r, double *gtheta,
            double *gdelta)
{
    if (!H || !theta || (!x && H->h.img_ready < 1) || !r || !gtheta) return CT_ERR_ARG;
    H->h.fwd_ready = H->h.adj_ready = 0;
    return images_laid_out(H->h, x, 1,
                           H->h.precision ? do_jacT<double>(H->h, theta, delta, x, r, gtheta, gdelta)
                                          : do_jacT<float>(H->h, theta, delta, x, r, gtheta, gdelta));
}

int ct_gn_terms(ct_handle *H, const double *theta, const double *delta, const void *x, const void *bdata, void *res,
                double *grad, double *jnorm2, double *fval)
{
    if (!H || !theta || (!x && H->h.img_ready < 1) || !bdata || !grad || !jnorm2) return CT_ERR_ARG;
    H->h.fwd_ready = H->h.adj_ready = 0;
    return images_laid_out(H->h, x, 1,
                           H->h.precision ? do_gn<double>(H->h, theta, delta, x, bdata, res, grad, jnorm2, fval)
                                          : do_gn<float>(H->h, theta, delta, x, bdata, res, grad, jnorm2, fval));
}

int ct_jac_batch(ct_handle *H, const double *theta, const double *delta, const void *X, const double *dtheta,
                 const double *ddelta, void *dY, int batch, int flags)
{
    if (!H || !theta || !dtheta || !dY || batch < 1 || batch > H->h.max_batch || (!X && batch > H->h.img_ready) ||
        (flags & ~CT_BATCH_PER_IMAGE_DIRECTION))
        return CT_ERR_ARG;
    H->h.fwd_ready = H->h.adj_ready = 0;
    return images_laid_out(H->h, X, batch,
                           H->h.precision ? do_jac_batch<double>(H->h, theta, delta, X, dtheta, ddelta, dY, batch, flags)
                                          : do_jac_batch<float>(H->h, theta, delta, X, dtheta, ddelta, dY, batch, flags));
}

int ct_jacT_batch(ct_handle *H, const double *theta, const double *delta, const void *X, const void *R,
                  double *gtheta, double *gdelta, int batch, int flags)
{
    if (!H || !theta || !R || !gtheta || batch < 1 || batch > H->h.max_batch || (!X && batch > H->h.img_ready) ||
        (flags & ~(CT_BATCH_SHARED_R | CT_BATCH_SUM)))
        return CT_ERR_ARG;
    H->h.fwd_ready = H->h.adj_ready = 0;
    return images_laid_out(H->h, X, batch,
                           H->h.precision ? do_jacT_batch<double>(H->h, theta, delta, X, R, gtheta, gdelta, batch, flags)
                                          : do_jacT_batch<float>(H->h, theta, delta, X, R, gtheta, gdelta, batch, flags));
}

int ct_gn_terms_batch(ct_handle *H, const double *theta, const double *delta, const void *X, const void *bdata,
                      void *res, double *grad, double *jnorm2, double *fval, int batch)
{
    if (!H || !theta || !bdata || !grad || !jnorm2 || batch < 1 || batch > H->h.max_batch ||
        (!X && batch > H->h.img_ready))
        return CT_ERR_ARG;
    H->h.fwd_ready = H->h.adj_ready = 0;
    return images_laid_out(H->h, X, batch,
                           H->h.precision ? do_gn_batch<double>(H->h, theta, delta, X, bdata, res, grad, jnorm2, fval, batch)
                                          : do_gn_batch<float>(H->h, theta, delta, X, bdata, res, grad, jnorm2, fval, batch));
}

int ct_set_stream(ct_handle *H, void *cuda_stream)
{
    if (!H) return CT_ERR_ARG;
    H->h.stream = (cudaStream_t)cuda_stream;
    return CT_OK;
}

int ct_autotune(ct_handle *H)
{
    if (!H) return CT_ERR_ARG;
    H->h.fwd_ready = H->h.adj_ready = H->h.img_ready = 0;
    return H->h.precision ? autotune_impl<double>(H->h) : autotune_impl<float>(H->h);
}

int ct_get_tuning(ct_handle *H, int32_t *out)
{
    if (!H || !out) return CT_ERR_ARG;
    const ctgb::Tuning &t = H->h.tune;
    const int32_t v[CT_TUNING_COUNT] = {t.fwd_kb,    t.fwd_split, t.fwd_vw,    t.adj_kb,
                                        t.adj_split, t.der_split, t.der_vw,    t.fwd_stage,
                                        t.der_stage, t.adj_stage, t.der_kb,    t.fwd_layout};
    for (int i = 0; i < CT_TUNING_COUNT; ++i) out[i] = v[i];
    return CT_OK;
}

int ct_set_tuning(ct_handle *H, const int32_t *in)
{
    if (!H || !in) return CT_ERR_ARG;
    auto pow2 = [](int x, int hi) { return x >= 1 && x <= hi && (x & (x - 1)) == 0; };
    auto stage_ok = [](int st, int vw) { return st == 0 || ((st == 4 || st == 8) && (vw == 4 || vw == 8)); };
    if (!pow2(in[0], 8) || !pow2(in[1], 8) || !pow2(in[2], 8) || !pow2(in[3], 8) || !pow2(in[4], 4) ||
        !pow2(in[5], 8) || !pow2(in[6], 8) || (in[7] == 0 && in[1] * in[2] > 16) ||
        (in[8] == 0 && in[5] * in[6] > 16) || !stage_ok(in[7], in[2]) || !stage_ok(in[8], in[6]) ||
        (in[7] > 0 && in[1] > 4) || (in[9] != 0 && in[9] != 8 && in[9] != 16) || !pow2(in[10], 4) ||
        (in[11] != 0 && in[11] != 1) || (in[11] == 1 && (in[7] != 0 || in[0] < 4)))
        return CT_ERR_ARG;
    if (in[7] > 0 && in[1] > 1) {
        const int rc = ensure_seg_partials(H->h);
        if (rc != CT_OK) return rc;
    }
    if (in[11] == 1) {
        const int rc = ensure_interleaved(H->h);
        if (rc != CT_OK) return rc;
    }
    ctgb::Tuning &t = H->h.tune;
    t.fwd_kb = in[0];
    t.fwd_split = in[1];
    t.fwd_vw = in[2];
    t.adj_kb = in[3];
    t.adj_split = in[4];
    t.der_split = in[5];
    t.der_vw = in[6];
    t.fwd_stage = in[7];
    t.der_stage = in[8];
    t.adj_stage = in[9];
    t.der_kb = in[10];
    t.fwd_layout = in[11];
    return CT_OK;
}

int ct_status(ct_handle *H)
{
    if (!H) return CT_ERR_ARG;
    CT_CUDA(cudaStreamSynchronize(H->h.stream));
    CT_CUDA(cudaGetLastError());
    int flag = 0;
    CT_CUDA(cudaMemcpy(&flag, H->h.d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        CT_CUDA(cudaMemset(H->h.d_flag, 0, sizeof(int)));
        return CT_ERR_NAN;
    }
    return CT_OK;
}

const char *ct_strerror(int code)
{
    switch (code) {
    case CT_OK: return "ok";
    case CT_ERR_ARG: return "invalid argument (null pointer, size or batch out of range)";
    case CT_ERR_CUDA: return "CUDA runtime error";
    case CT_ERR_OOM: return "device allocation failed";
    case CT_ERR_TIMEOUT: return "bounded device-side wait ran out";
    case CT_ERR_NAN: return "non-finite angle/offset or numerical breakdown";
    case CT_ERR_NOCONV: return "iteration limit reached (outputs valid)";
    default: return "unknown error code";
    }
}

const char *ct_last_cuda_error(void) { return g_cuda_msg; }

}  // extern "C"
