// C ABI of libctgb (declared in include/ctgb.h): argument checks, handle
// workspaces and the launch sequence of each operator call.
#include <cuda_runtime.h>

#include <cstdio>
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
    cudaFree(h.d_xt);
    cudaFree(h.d_partial);
    h.d_views = nullptr;
    h.d_fov = h.d_fstart = h.d_fcount = h.d_flag = nullptr;
    h.d_xt = nullptr;
    h.d_partial = nullptr;
}

template <typename T>
int do_forward(ct_handle *H, const double *theta, const double *delta, const void *X, void *Y, int batch)
{
    ctgb::Handle &h = H->h;
    CT_CUDA(ctgb::launch_view_setup(h, theta, delta));
    CT_CUDA(ctgb::launch_transpose<T>(h, (const T *)X, (T *)h.d_xt, batch * h.F));
    CT_CUDA(ctgb::launch_forward<T>(h, (const T *)X, (const T *)h.d_xt, (T *)Y, batch));
    return CT_OK;
}

template <typename T>
int do_adjoint(ct_handle *H, const double *theta, const double *delta, const void *Y, void *X, int batch)
{
    ctgb::Handle &h = H->h;
    CT_CUDA(ctgb::launch_view_setup(h, theta, delta));
    CT_CUDA(ctgb::launch_adjoint<T>(h, (const T *)Y, (T *)X, batch));
    return CT_OK;
}

template <typename T>
int do_jac(ct_handle *H, const double *theta, const double *delta, const void *x, const double *dtheta,
           const double *ddelta, void *dy)
{
    ctgb::Handle &h = H->h;
    CT_CUDA(ctgb::launch_view_setup(h, theta, delta));
    CT_CUDA(ctgb::launch_transpose<T>(h, (const T *)x, (T *)h.d_xt, h.F));
    CT_CUDA(ctgb::launch_jvp<T>(h, (const T *)x, (const T *)h.d_xt, dtheta, ddelta, (T *)dy));
    return CT_OK;
}

template <typename T>
int do_jacT(ct_handle *H, const double *theta, const double *delta, const void *x, const void *r, double *gtheta,
            double *gdelta)
{
    ctgb::Handle &h = H->h;
    CT_CUDA(ctgb::launch_view_setup(h, theta, delta));
    CT_CUDA(ctgb::launch_transpose<T>(h, (const T *)x, (T *)h.d_xt, h.F));
    CT_CUDA(ctgb::launch_vjp<T>(h, (const T *)x, (const T *)h.d_xt, (const T *)r, gtheta, gdelta));
    return CT_OK;
}

template <typename T>
int do_gn(ct_handle *H, const double *theta, const double *delta, const void *x, const void *bdata, void *res,
          double *grad, double *jnorm2, double *fval)
{
    ctgb::Handle &h = H->h;
    CT_CUDA(ctgb::launch_view_setup(h, theta, delta));
    CT_CUDA(ctgb::launch_transpose<T>(h, (const T *)x, (T *)h.d_xt, h.F));
    CT_CUDA(ctgb::launch_gn<T>(h, (const T *)x, (const T *)h.d_xt, (const T *)bdata, (T *)res, grad, jnorm2, fval));
    return CT_OK;
}

}  // namespace

extern "C" {

int ct_init(const ct_geom *g, void *cuda_stream, ct_handle **out)
{
    if (!g || !out) return CT_ERR_ARG;
    *out = nullptr;
    if (g->N < 2 || g->N > ctgb::kMaxN || g->B < 1 || g->n_views < 1 || g->n_frames < 1 || g->max_batch < 1 ||
        (g->precision != 0 && g->precision != 1))
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
        const size_t img_elems = (size_t)h.max_batch * h.F * h.N * h.N;
        bool ok = cudaMalloc(&h.d_views, sizeof(ctgb::ViewGeo) * h.V) == cudaSuccess &&
                  cudaMalloc(&h.d_fov, sizeof(int) * h.V) == cudaSuccess &&
                  cudaMalloc(&h.d_fstart, sizeof(int) * h.F) == cudaSuccess &&
                  cudaMalloc(&h.d_fcount, sizeof(int) * h.F) == cudaSuccess &&
                  cudaMalloc(&h.d_flag, sizeof(int)) == cudaSuccess &&
                  cudaMalloc(&h.d_xt, img_elems * elem_size(h)) == cudaSuccess &&
                  cudaMalloc(&h.d_partial, sizeof(double) * 4 * (size_t)h.V * h.nchunks) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            rc = CT_ERR_OOM;
            break;
        }
        e = cudaMemcpy(h.d_fov, fov.data(), sizeof(int) * h.V, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h.d_fstart, fstart.data(), sizeof(int) * h.F, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h.d_fcount, fcount.data(), sizeof(int) * h.F, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(h.d_flag, 0, sizeof(int));
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
    if (!H || !theta || !X || !Y || batch < 1 || batch > H->h.max_batch) return CT_ERR_ARG;
    return H->h.precision ? do_forward<double>(H, theta, delta, X, Y, batch)
                          : do_forward<float>(H, theta, delta, X, Y, batch);
}

int ct_adjoint(ct_handle *H, const double *theta, const double *delta, const void *Y, void *X, int batch)
{
    if (!H || !theta || !X || !Y || batch < 1 || batch > H->h.max_batch) return CT_ERR_ARG;
    return H->h.precision ? do_adjoint<double>(H, theta, delta, Y, X, batch)
                          : do_adjoint<float>(H, theta, delta, Y, X, batch);
}

int ct_jac(ct_handle *H, const double *theta, const double *delta, const void *x, const double *dtheta,
           const double *ddelta, void *dy)
{
    if (!H || !theta || !x || !dtheta || !dy) return CT_ERR_ARG;
    return H->h.precision ? do_jac<double>(H, theta, delta, x, dtheta, ddelta, dy)
                          : do_jac<float>(H, theta, delta, x, dtheta, ddelta, dy);
}

int ct_jacT(ct_handle *H, const double *theta, const double *delta, const void *x, const void *r, double *gtheta,
            double *gdelta)
{
    if (!H || !theta || !x || !r || !gtheta) return CT_ERR_ARG;
    return H->h.precision ? do_jacT<double>(H, theta, delta, x, r, gtheta, gdelta)
                          : do_jacT<float>(H, theta, delta, x, r, gtheta, gdelta);
}

int ct_gn_terms(ct_handle *H, const double *theta, const double *delta, const void *x, const void *bdata, void *res,
                double *grad, double *jnorm2, double *fval)
{
    if (!H || !theta || !x || !bdata || !grad || !jnorm2) return CT_ERR_ARG;
    return H->h.precision ? do_gn<double>(H, theta, delta, x, bdata, res, grad, jnorm2, fval)
                          : do_gn<float>(H, theta, delta, x, bdata, res, grad, jnorm2, fval);
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
