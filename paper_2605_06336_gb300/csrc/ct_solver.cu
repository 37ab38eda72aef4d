// nlrmm_gks_solve: the alternating NL-RMM-GKS driver on the GPU.
//
// Algorithms followed: "NL-RMM-GKS" (Sec. 4.3, without the optional
// high-lambda solve), "RMM-GKS" (Sec. 3.3) with "Enlarge" and "Compress"
// (supplementary Sec. S1.2), "UPDATE-PARAM" (Sec. 4.1.2) or, with
// opts.varpro, "UPDATE-PARAM-VarPro" (Sec. 4.2).  Operators are the
// ct kernels of this library in the handle's precision; every small matrix
// (k <= 122) is FP64 on the device.
//
// Differences from the printed form, none of which changes the iterates in
// exact arithmetic:
//   * R_H and R_Psi enter the reduced problem and the Compress SVD only as
//     R_H^T R_H = (HV)^T HV, R_Psi^T R_Psi = (P Psi V)^T (P Psi V) and
//     R_H^T Q_H^T b = (HV)^T b, so those FP64 Gram products are formed
//     directly; (HV)^T HV and (HV)^T b grow by one row per Enlarge step.
//   * lambda is found on the generalized eigenbasis of the two Gram
//     matrices, where the projected discrepancy is a closed-form sum.
//   * H u is formed as (HV) y (no extra projection per step).
//   * An Enlarge step is a fixed launch sequence predicated on a device stop
//     flag (no host round trip inside Enlarge).
//   * With per-view angles J^T J is diagonal, so the Gauss-Newton step and
//     its Armijo backtracking are per view.
//   * VarPro: the Gauss-Newton matrix of the reduced residuals is a diagonal
//     plus a rank-2k term (k basis columns); it is never formed: the damped
//     system is solved by the Woodbury identity with a 2k x 2k capacitance.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include "../../include/ctgb.h"
#include "ct_internal.cuh"
#include "ct_solver_kernels.cuh"

struct ct_handle {
    ctgb::Handle h;
};

namespace {

using namespace ctgb;
using namespace ctgb::solver;

thread_local char g_solver_msg[256] = "";

#define SV_CUDA(call)                                                                                     \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) {                                                                          \
            std::snprintf(g_solver_msg, sizeof(g_solver_msg), "%s:%d %s", __FILE__, __LINE__,             \
                          cudaGetErrorString(e_));                                                        \
            return CT_ERR_CUDA;                                                                           \
        }                                                                                                 \
    } while (0)

#define SV_TRY(expr)                  \
    do {                              \
        int rc_ = (expr);             \
        if (rc_ != CT_OK) return rc_; \
    } while (0)

constexpr int kThreads = 256;

template <typename T> struct Solver {
    Handle h;  // copy of the caller's handle, running on the solver's private stream
    const nlrmm_opts &o;
    const T *b;
    const double *delta;
    long long n = 0, m = 0, ne = 0;
    int KC = 0;         // basis capacity (columns)
    int gram_blocks = 0;
    std::vector<void *> allocs;
    // device buffers
    T *V = nullptr, *HV = nullptr, *u = nullptr, *uold = nullptr, *uprev = nullptr, *w = nullptr, *res = nullptr,
      *Vtmp = nullptr;
    double *GH = nullptr, *GP = nullptr, *cvec = nullptr, *y = nullptr, *W = nullptr, *dots = nullptr,
           *part_gram = nullptr, *part_dot = nullptr, *part_n = nullptr, *norms = nullptr, *norms2 = nullptr,
           *scal = nullptr;
    double *th_k = nullptr, *th_n = nullptr, *th_t = nullptr, *d = nullptr, *alpha = nullptr, *g = nullptr,
           *j2 = nullptr, *f0 = nullptr, *ft = nullptr, *rho = nullptr, *scratch_v = nullptr;
    int *ctl = nullptr, *active = nullptr;
    // VarPro Gauss-Newton work (allocated on first use)
    T *vp_a = nullptr, *vp_u = nullptr;
    double *vp_E = nullptr, *vp_G = nullptr, *vp_Y = nullptr, *vp_idel = nullptr, *vp_ones = nullptr,
           *vp_scal = nullptr, *vp_rho = nullptr;
    double *small_work = nullptr;  // device work area of the FP64 small algebra above kKSmem columns
    int *vp_ctl = nullptr;
    int *h_ctl = nullptr;       // pinned mirror of ctl
    double *h_scal = nullptr;   // pinned mirror of small results
    int *h_stop = nullptr;      // host-mapped mirror of the Enlarge stop flag
    int *d_stop = nullptr;      // its device address
    cudaEvent_t ev[2] = {nullptr, nullptr};
    std::vector<cudaGraphExec_t> step_graph;  // one captured Enlarge step per basis size
    bool use_graphs = true;  // off in the plain form
    double noise = 0.0;      // noise norm of the discrepancy principle for the bound data
    // unit roundoff of the Armijo noise floor: the option, or that of the misfit's precision
    double armijo_u() const { return o.armijo_eps >= 0.0 ? o.armijo_eps : (sizeof(T) == 4 ? 0x1p-24 : 0x1p-53); }
    long long m_cap = 0;     // streaming: capacities over all blocks (0: this handle's)
    int v_cap = 0;

    Solver(const Handle &h_, cudaStream_t s_, const nlrmm_opts &o_, const T *b_, const double *delta_)
        : h(h_), o(o_), b(b_), delta(delta_), noise(o_.noise_norm)
    {
        h.stream = s_;
        if (o.plain) use_graphs = false;
    }

    ~Solver()
    {
        for (cudaGraphExec_t g : step_graph)
            if (g) cudaGraphExecDestroy(g);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        for (void *p : allocs) cudaFree(p);
        if (h_ctl) cudaFreeHost(h_ctl);
        if (h_scal) cudaFreeHost(h_scal);
        if (h_stop) cudaFreeHost(h_stop);
    }

    template <typename U> int alloc(U *&p, size_t count)
    {
        void *q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(1, count) * sizeof(U)) != cudaSuccess) {
            cudaGetLastError();
            return CT_ERR_OOM;
        }
        allocs.push_back(q);
        p = (U *)q;
        return CT_OK;
    }

    int grid_for(long long len) const
    {
        return (int)std::max<long long>(1, std::min<long long>((len + kThreads - 1) / kThreads, 8LL * h.num_sms));
    }

    int setup()
    {
        n = (long long)h.F * h.N * h.N;
        m = (long long)h.V * h.B;
        ne = psi_edges(h.N, h.F, o.temporal);
        KC = o.k_max + 2;
        // tiles of the Gram kernel: kRbRows x 32 pixels (FP32, register-blocked), 4 x 32 (FP64)
        const int tile_rows = sizeof(T) == 4 ? kRbRows : 4;
        const int tiles = ((h.N + 31) / 32) * ((h.N + tile_rows - 1) / tile_rows) * h.F;
        gram_blocks = std::min(tiles, 2 * h.num_sms);
        const long long m_all = std::max(m, m_cap);
        const int v_all = std::max(h.V, v_cap);
        SV_TRY(alloc(V, (size_t)KC * n));
        SV_TRY(alloc(HV, (size_t)KC * m_all));
        SV_TRY(alloc(u, n));
        SV_TRY(alloc(uold, n));
        SV_TRY(alloc(uprev, n));
        SV_TRY(alloc(w, ne));
        SV_TRY(alloc(res, m_all));
        SV_TRY(alloc(Vtmp, (size_t)o.k_min * n));
        SV_TRY(alloc(GH, kKMax * kKMax));
        SV_TRY(alloc(GP, kKMax * kKMax));
        SV_TRY(alloc(cvec, kKMax + 2));
        SV_TRY(alloc(y, kKMax + 2));
        SV_TRY(alloc(W, kKMax * kKMax));
        SV_TRY(alloc(dots, kKMax + 2));
        SV_TRY(alloc(part_gram, (size_t)gram_blocks * kGramPairs));
        SV_TRY(alloc(part_dot, (size_t)kRedBlocks * (kKMax + 2)));
        SV_TRY(alloc(part_n, (size_t)kRedBlocks * 3));
        SV_TRY(alloc(norms, 3));
        SV_TRY(alloc(norms2, 3));
        SV_TRY(alloc(scal, kScalCount));
        for (double **p : {&th_k, &th_n, &th_t, &d, &alpha, &g, &j2, &f0, &ft, &rho, &scratch_v})
            SV_TRY(alloc(*p, v_all));
        SV_TRY(alloc(ctl, kCtlCount));
        SV_TRY(alloc(active, v_all));
        if (cudaMallocHost(&h_ctl, sizeof(int) * kCtlCount) != cudaSuccess ||
            cudaMallocHost(&h_scal, sizeof(double) * 16) != cudaSuccess ||
            cudaHostAlloc(&h_stop, sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            return CT_ERR_OOM;
        }
        SV_CUDA(cudaHostGetDevicePointer((void **)&d_stop, h_stop, 0));
        *(volatile int *)h_stop = 0;
        SV_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
        SV_CUDA(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
        step_graph.assign(KC + 1, nullptr);
        SV_CUDA(cudaMemsetAsync(GH, 0, sizeof(double) * kKMax * kKMax, h.stream));
        SV_CUDA(cudaMemsetAsync(GP, 0, sizeof(double) * kKMax * kKMax, h.stream));
        SV_CUDA(cudaMemsetAsync(ctl, 0, sizeof(int) * kCtlCount, h.stream));
        SV_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * kScalCount, h.stream));
        SV_CUDA(cudaFuncSetAttribute(k_small_solve<kKSmem>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(SolveShared<kKSmem>)));
        SV_CUDA(cudaFuncSetAttribute(k_compress_basis<kKSmem>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(SmallShared<kKSmem>)));
        if (KC > kKSmem) SV_TRY(alloc(small_work, kSmallWorkBytes / sizeof(double) + 1));
        if constexpr (sizeof(T) == 4) {
            SV_CUDA(cudaFuncSetAttribute(k_gram_psi_pipe8<2, kP8Threads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kGramP8SmemMax));
            SV_CUDA(cudaFuncSetAttribute(k_gram_psi_pipe8<1, kP8Threads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kGramP8SmemMax));
            SV_CUDA(cudaFuncSetAttribute(k_gram_psi_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kGramPipeSmemMax));
        } else {
            SV_CUDA(cudaFuncSetAttribute(k_gram_psi<T, 4, gram_slots(kKSmem)>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gram_smem(kKSmem, true, 4)));
            SV_CUDA(cudaFuncSetAttribute(k_gram_psi<T, 1, gram_slots(kKLimit)>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gram_smem(kKLimit, true, 1)));
        }
        return CT_OK;
    }

    // FP64 small algebra: shared-memory form up to kKSmem columns, device workspace above
    void small_solve(int k, double target, double lam_fix, double lam_lo, double lam_hi, int lam_iters, double *yout,
                     double *scal_out, int *ctl_out)
    {
        if (k <= kKSmem)
            k_small_solve<kKSmem><<<1, kSolveThreads, sizeof(SolveShared<kKSmem>), h.stream>>>(
                GH, cvec, GP, k, bnorm2, target, lam_fix, lam_lo, lam_hi, lam_iters, yout, scal_out, ctl_out, nullptr);
        else
            k_small_solve<kKMax><<<1, kSolveThreads, 0, h.stream>>>(GH, cvec, GP, k, bnorm2, target, lam_fix, lam_lo,
                                                                     lam_hi, lam_iters, yout, scal_out, ctl_out,
                                                                     small_work);
    }
    void compress_basis(int k, int keep)
    {
        if (k <= kKSmem)
            k_compress_basis<kKSmem><<<1, 256, sizeof(SmallShared<kKSmem>), h.stream>>>(GH, GP, k, scal, keep, W,
                                                                                       nullptr);
        else
            k_compress_basis<kKMax><<<1, 256, 0, h.stream>>>(GH, GP, k, scal, keep, W, small_work);
    }

    // k columns of the edges of one tile of TR x 32 pixels: 2 per pixel, 3 with the temporal edge (ANISO-TV)
    static size_t gram_smem(int k, bool temporal, int tr)
    {
        return (size_t)k * ((temporal ? 3 : 2) * tr * 32 + 1) * sizeof(T);
    }

    // GP = (P Psi V)^T (P Psi V) over V[:, :k] with the weights in w
    int gram_psi(int k, const int *stop)
    {
        const bool tm = o.temporal && h.F > 1;
        if constexpr (sizeof(T) == 4) {
            const int epp = tm ? 3 : 2;
            if (k <= 32 && gram_pipe_smem(k, epp) <= kGramPipeSmemMax && gram_rb_threads(k) == 256)
                // 4 x 4 blocks over 4-row tiles for small bases (above 32 columns the 8 x 8 blocks
                // measured faster: C5 streaming 6.98 -> 6.78 s per pass)
                k_gram_psi_pipe<<<gram_blocks, kThreads, gram_pipe_smem(k, epp), h.stream>>>(
                    V, n, k, w, h.N, h.F, o.temporal, part_gram, stop);
            else if (gram_p8_rows(k, epp) == 2)  // larger bases: 2-row tiles, 8 x 8 blocks
                k_gram_psi_pipe8<2, kP8Threads><<<gram_blocks, kP8Threads, gram_p8_smem(k, epp, 2), h.stream>>>(
                    V, n, k, w, h.N, h.F, o.temporal, part_gram, stop);
            else  // 1-row tiles (fits up to the largest basis)
                k_gram_psi_pipe8<1, kP8Threads><<<gram_blocks, kP8Threads, gram_p8_smem(k, epp, 1), h.stream>>>(
                    V, n, k, w, h.N, h.F, o.temporal, part_gram, stop);
        } else {
            if (k <= kKSmem)
                k_gram_psi<T, 4, gram_slots(kKSmem)><<<gram_blocks, kThreads, gram_smem(k, tm, 4), h.stream>>>(
                    V, n, k, w, h.N, h.F, o.temporal, part_gram, stop);
            else
                k_gram_psi<T, 1, gram_slots(kKLimit)><<<gram_blocks, kThreads, gram_smem(k, tm, 1), h.stream>>>(
                    V, n, k, w, h.N, h.F, o.temporal, part_gram, stop);
        }
        k_gram_reduce<<<gram_reduce_blocks(k), 32 * kGramReduceWarps, 0, h.stream>>>(part_gram, gram_blocks, k, GP,
                                                                                     stop);
        SV_CUDA(cudaGetLastError());
        return CT_OK;
    }

    T *col(T *base, long long len, int j) const { return base + (long long)j * len; }

    // ---- building blocks --------------------------------------------------
    // out[0..k) = A[:, 0..k)^T x  (+ out[k] = x2 . x when x2 != null)
    int dots_into(const T *A, long long len, int k, const T *x, const T *x2, double *out, const int *stop)
    {
        const int nblk = red_blocks(len);
        k_dots<T><<<nblk, kThreads, 0, h.stream>>>(A, len, len, k, x, x2, part_dot, stop);
        const int kk = k + (x2 ? 1 : 0);
        k_dots_reduce<<<(kk + kDotsReduceWarps - 1) / kDotsReduceWarps, 32 * kDotsReduceWarps, 0, h.stream>>>(
            part_dot, nblk, kk, out, stop);
        SV_CUDA(cudaGetLastError());
        return CT_OK;
    }

    // norms3 of (a, b): {|a|^2, |a-b|^2, |b|^2}
    int norms3(const T *a, const T *bb, long long len, double *out, const int *stop)
    {
        const int nblk = red_blocks(len);
        k_norms3<T><<<nblk, kThreads, 0, h.stream>>>(a, bb, len, part_n, stop);
        k_norms3_reduce<<<1, 32, 0, h.stream>>>(part_n, nblk, out, stop);
        SV_CUDA(cudaGetLastError());
        return CT_OK;
    }

    // r <- r - V[:, :k] V[:, :k]^T r, twice
    int cgs2(T *r, int k, const int *stop)
    {
        if (k == 0) return CT_OK;
        for (int pass = 0; pass < 2; ++pass) {
            SV_TRY(dots_into(V, n, k, r, nullptr, dots, stop));
            k_gemv<T><<<grid_for(n), kThreads, 0, h.stream>>>(V, n, n, k, dots, r, T(1), T(-1), nullptr, T(0),
                                                                stop);
        }
        SV_CUDA(cudaGetLastError());
        return CT_OK;
    }

    // columns per projection launch: the Krylov block (max_batch), or one in the plain form
    int block() const { return o.plain ? 1 : h.max_batch; }

    // HV[:, j0:j0+cnt) = H(theta) V[:, j0:j0+cnt), in chunks of block() columns; a chunk
    // of two or more columns reads them interleaved when the handle's forward does
    // (the same bits; one column reads the pair images, which are as fast there)
    int project(const double *theta, int j0, int cnt, const int *stop)
    {
        if (cnt <= 0) SV_CUDA(launch_view_setup(h, theta, delta, stop));
        for (int j = j0; j < j0 + cnt; j += block()) {
            const int nb = std::min(block(), j0 + cnt - j);
            const double *th = j == j0 ? theta : nullptr;  // the first layout launch also updates the view table
            if constexpr (std::is_same<T, float>::value) {
                if (nb >= 2 && h.tune.fwd_layout == 1 && h.d_qx && h.fan_D == 0.0) {
                    SV_CUDA(launch_interleave_img(h, col(V, n, j), nb, th, delta, stop));
                    SV_CUDA(launch_forward<T>(h, col(HV, m, j), nb, h.tune.fwd_kb, h.tune.fwd_split, h.tune.fwd_vw,
                                              0, stop, true, nb));
                    continue;
                }
            }
            SV_CUDA(launch_prep_forward<T>(h, col(V, n, j), nb * h.F, stop, th, delta));
            SV_CUDA(launch_forward<T>(h, col(HV, m, j), nb, h.tune.fwd_kb, h.tune.fwd_split, h.tune.fwd_vw,
                                      h.tune.fwd_stage, stop));
        }
        return CT_OK;
    }

    // out = H(theta)^T yin  (n vector)
    int backproject(const double *theta, const T *yin, T *out, const int *stop)
    {
        SV_CUDA(launch_pairs_sino<T>(h, yin, 1, stop, theta, delta));
        SV_CUDA(launch_adjoint<T>(h, out, 1, h.tune.adj_kb, h.tune.adj_split, h.tune.adj_stage, stop));
        return CT_OK;
    }

    int sync_ctl()
    {
        SV_CUDA(cudaMemcpyAsync(h_ctl, ctl, sizeof(int) * kCtlCount, cudaMemcpyDeviceToHost, h.stream));
        SV_CUDA(cudaStreamSynchronize(h.stream));
        return CT_OK;
    }

    int read_doubles(const double *src, int cnt, double *dst)
    {
        SV_CUDA(cudaMemcpyAsync(h_scal, src, sizeof(double) * cnt, cudaMemcpyDeviceToHost, h.stream));
        SV_CUDA(cudaStreamSynchronize(h.stream));
        std::memcpy(dst, h_scal, sizeof(double) * cnt);
        return CT_OK;
    }

    // ---- Golub-Kahan bidiagonalization start basis --------------------------
    int gkb(const double *theta, int k)
    {
        double nb[3];
        SV_TRY(norms3(b, nullptr, m, norms, nullptr));
        SV_TRY(read_doubles(norms, 3, nb));
        const double bn = std::sqrt(nb[0]);
        if (!(bn > 0.0)) return CT_ERR_ARG;
        // ubuf (m) = b / |b| ; v = H^T ubuf
        T *ubuf = res;
        SV_CUDA(cudaMemcpyAsync(ubuf, b, sizeof(T) * m, cudaMemcpyDeviceToDevice, h.stream));
        scale(ubuf, m, 1.0 / bn);
        SV_TRY(backproject(theta, ubuf, col(V, n, 0), nullptr));
        double nv[3];
        SV_TRY(norms3(col(V, n, 0), nullptr, n, norms, nullptr));
        SV_TRY(read_doubles(norms, 3, nv));
        double alpha_ = std::sqrt(nv[0]);
        scale(col(V, n, 0), n, 1.0 / alpha_);
        for (int j = 1; j < k; ++j) {
            // p = H v_{j-1} - alpha u ; beta = |p| ; u = p / beta
            SV_TRY(project(theta, j - 1, 1, nullptr));
            axpby(ubuf, col(HV, m, j - 1), m, -alpha_, 1.0);  // ubuf = HV[:, j-1] - alpha * ubuf
            SV_TRY(norms3(ubuf, nullptr, m, norms, nullptr));
            SV_TRY(read_doubles(norms, 3, nv));
            const double beta_ = std::sqrt(nv[0]);
            scale(ubuf, m, 1.0 / beta_);
            // q = H^T u - beta v_{j-1}, reorthogonalized
            SV_TRY(backproject(theta, ubuf, col(V, n, j), nullptr));
            axpby(col(V, n, j), col(V, n, j - 1), n, 1.0, -beta_);  // V_j = V_j - beta V_{j-1}
            SV_TRY(cgs2(col(V, n, j), j, nullptr));
            SV_TRY(norms3(col(V, n, j), nullptr, n, norms, nullptr));
            SV_TRY(read_doubles(norms, 3, nv));
            alpha_ = std::sqrt(nv[0]);
            scale(col(V, n, j), n, 1.0 / alpha_);
        }
        SV_CUDA(cudaGetLastError());
        return CT_OK;
    }

    // small elementwise helpers (host-known scalars)
    void scale(T *x, long long len, double s)
    {
        k_gemv<T><<<grid_for(len), kThreads, 0, h.stream>>>(x, len, len, 0, y, x, (T)s, T(0), nullptr, T(0),
                                                              nullptr);
    }
    // x = a*x + c*z
    void axpby(T *x, const T *z, long long len, double a, double c)
    {
        k_gemv<T><<<grid_for(len), kThreads, 0, h.stream>>>(x, len, len, 0, y, x, (T)a, T(0), z, (T)c, nullptr);
    }

    // ---- one predicated Enlarge step with kc basis columns ------------------
    int enlarge_step(const double *theta, int kc)
    {
        const int *stop = ctl + kStop;
        // P^2 from the previous iterate
        k_weights<T><<<grid_for(ne), kThreads, 0, h.stream>>>(uold, w, h.N, h.F, o.temporal, o.eps, stop);
        // G_P = (P Psi V)^T (P Psi V)
        SV_TRY(gram_psi(kc, stop));
        // lambda and the reduced solution
        const double target = (o.tau * noise) * (o.tau * noise);
        small_solve(kc, target, o.lam_fix, o.lam_lo, o.lam_hi, o.lam_iters, y, scal, ctl);
        // u = V y ; res = (HV) y - b
        k_gemv<T><<<grid_for(n), kThreads, 0, h.stream>>>(V, n, n, kc, y, u, T(0), T(1), nullptr, T(0), stop);
        k_gemv<T><<<grid_for(m), kThreads, 0, h.stream>>>(HV, m, m, kc, y, res, T(0), T(1), b, T(-1), stop);
        SV_CUDA(cudaGetLastError());
        // r = H^T res + lambda Psi^T P^2 Psi u, written straight into the next basis column
        T *r = col(V, n, kc);
        SV_TRY(backproject(theta, res, r, stop));
        k_add_reg<T><<<grid_for(n), kThreads, 0, h.stream>>>(r, u, w, scal, h.N, h.F, o.temporal, stop);
        SV_TRY(cgs2(r, kc, stop));
        SV_TRY(norms3(r, nullptr, n, norms2, stop));        // |r|^2
        SV_TRY(norms3(u, uold, n, norms, stop));            // |u|^2, |u - u_old|^2, |u_old|^2
        k_step_decide<<<1, 1, 0, h.stream>>>(norms2, norms, o.tol1, ctl, scal);
        k_normalize<T><<<grid_for(n), kThreads, 0, h.stream>>>(r, n, norms2, stop);
        // H v_new and the new row of (HV)^T HV, (HV)^T b
        SV_TRY(project(theta, kc, 1, stop));
        SV_TRY(dots_into(HV, m, kc + 1, col(HV, m, kc), b, dots, stop));
        k_gh_append<<<1, kKMax + 2, 0, h.stream>>>(dots, kc, GH, cvec, stop);
        SV_CUDA(cudaMemcpyAsync(uold, u, sizeof(T) * n, cudaMemcpyDeviceToDevice, h.stream));  // (u_old = u)
        k_step_commit<<<1, 1, 0, h.stream>>>(ctl, d_stop);
        SV_CUDA(cudaGetLastError());
        return CT_OK;
    }

    // One Enlarge step: replay the captured graph for this basis size (capture
    // it on first use); launch eagerly if capture is not available.
    int run_step(int kc)
    {
        if (use_graphs && !step_graph[kc]) {
            cudaGraph_t g = nullptr;
            bool ok = cudaStreamBeginCapture(h.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            int rc = ok ? enlarge_step(th_k, kc) : CT_ERR_CUDA;
            if (ok) ok = cudaStreamEndCapture(h.stream, &g) == cudaSuccess && rc == CT_OK;
            cudaGraphExec_t ge = nullptr;
            if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
            if (!ok) {
                cudaGetLastError();
                use_graphs = false;  // fall back to plain launches for the rest of the solve
            } else {
                step_graph[kc] = ge;
            }
        }
        if (use_graphs) {
            SV_CUDA(cudaGraphLaunch(step_graph[kc], h.stream));
            return CT_OK;
        }
        return enlarge_step(th_k, kc);
    }

    double bnorm2 = 0.0;

    int full_gram(int kc)
    {
        // (HV)^T HV and (HV)^T b from scratch
        for (int j = 0; j < kc; ++j) {
            SV_TRY(dots_into(HV, m, j + 1, col(HV, m, j), b, dots, nullptr));
            k_gh_append<<<1, kKMax + 2, 0, h.stream>>>(dots, j, GH, cvec, nullptr);
        }
        SV_CUDA(cudaGetLastError());
        return CT_OK;
    }

    // ---- Gauss-Newton / Armijo per view ---------------------------------------
    int update_param(const T *uimg)
    {
        SV_CUDA(cudaMemcpyAsync(th_n, th_k, sizeof(double) * h.V, cudaMemcpyDeviceToDevice, h.stream));
        for (int it = 0; it < o.maxiter_p; ++it) {
            SV_CUDA(launch_pairs_img<T>(h, uimg, h.F, nullptr, th_n, delta));
            SV_CUDA(launch_gn<T>(h, b, nullptr, g, j2, f0, h.tune.der_split, h.tune.der_vw, h.tune.der_stage,
                                 nullptr, nullptr, 1, 1, rho));
            k_gn_direction<<<1, 1024, 0, h.stream>>>(g, j2, rho, h.V, o.mu_rel, o.alpha0, armijo_u(), th_n, d, alpha,
                                                     th_t, active, ctl);
            // Trial rounds run predicated on ctl[kArmijoDone] (set by k_armijo when no
            // view searches any more); the host reads the flag after rounds 1, 3, 7, 15
            // and the last only, so a search that needs many halvings costs few round
            // trips and one that ends early enqueues few idle rounds.
            const int *done = ctl + kArmijoDone;
            int next_check = 1;
            for (int hv = 0; hv <= o.max_halvings; ++hv) {
                SV_CUDA(launch_view_setup_wide(h, th_t, delta, ctl + kViewChanged, done));
                SV_CUDA(launch_gn<T>(h, b, nullptr, scratch_v, scratch_v, ft, h.tune.der_split, h.tune.der_vw,
                                     h.tune.der_stage, active, done));
                k_armijo<<<1, 1024, 0, h.stream>>>(f0, ft, g, d, rho, th_n, h.V, o.c1, o.beta, armijo_u(), alpha,
                                                   th_t, active, ctl, hv == o.max_halvings ? 1 : 0);
                if (hv + 1 == next_check || hv == o.max_halvings || o.plain) {
                    SV_TRY(sync_ctl());
                    if (h_ctl[kArmijoDone]) break;
                    next_check = 2 * next_check + 1;
                }
            }
            SV_CUDA(cudaMemcpyAsync(th_n, th_t, sizeof(double) * h.V, cudaMemcpyDeviceToDevice, h.stream));
        }
        SV_CUDA(cudaGetLastError());
        return CT_OK;
    }

    // ---- UPDATE-PARAM for one offset shared by every view ------------------------
    // theta = theta_k + p 1: Gauss-Newton on p from the per-view terms summed in a
    // fixed order (g = sum_v g_v, J^T J = sum_v |J_v|^2, f = sum_v f_v, rho = sum_v
    // rho_v), Armijo on the total misfit with its noise floor; the step d fills the
    // per-view direction array so that the trial angles are th_n + alpha d.
    int update_param_shared(const T *uimg)
    {
        SV_CUDA(cudaMemcpyAsync(th_n, th_k, sizeof(double) * h.V, cudaMemcpyDeviceToDevice, h.stream));
        for (int it = 0; it < o.maxiter_p; ++it) {
            SV_CUDA(launch_pairs_img<T>(h, uimg, h.F, nullptr, th_n, delta));
            SV_CUDA(launch_gn<T>(h, b, nullptr, g, j2, f0, h.tune.der_split, h.tune.der_vw, h.tune.der_stage,
                                 nullptr, nullptr, 1, 1, rho));
            k_view_sums<<<1, 1024, 0, h.stream>>>(g, j2, f0, rho, h.V, part_n);
            double s4[4];
            SV_TRY(read_doubles(part_n, 4, s4));
            const double G = s4[0], JJ = s4[1], F = s4[2], R = s4[3];
            const double dp = -G / (JJ + o.mu_rel * std::max(JJ, 1e-300));
            k_fill<double><<<grid_for(h.V), kThreads, 0, h.stream>>>(d, h.V, dp);
            bool accepted = false;
            double alpha = o.alpha0;
            for (int hv = 0; hv <= o.max_halvings; ++hv) {
                if (alpha * std::fabs(G * dp) < armijo_u() * R) break;  // noise floor: no step
                k_theta_step<<<grid_for(h.V), kThreads, 0, h.stream>>>(th_n, d, alpha, h.V, th_t);
                SV_CUDA(launch_view_setup_wide(h, th_t, delta, ctl + kViewChanged, nullptr));
                SV_CUDA(launch_gn<T>(h, b, nullptr, scratch_v, scratch_v, ft, h.tune.der_split, h.tune.der_vw,
                                     h.tune.der_stage));
                k_view_sums<<<1, 1024, 0, h.stream>>>(ft, nullptr, nullptr, nullptr, h.V, part_n);
                double fsum[1];
                SV_TRY(read_doubles(part_n, 1, fsum));
                if (fsum[0] <= F + o.c1 * alpha * G * dp) {
                    accepted = true;
                    break;
                }
                alpha *= o.beta;
            }
            if (!accepted) break;  // the offset stays
            SV_CUDA(cudaMemcpyAsync(th_n, th_t, sizeof(double) * h.V, cudaMemcpyDeviceToDevice, h.stream));
        }
        SV_CUDA(cudaGetLastError());
        return CT_OK;
    }

    // ---- VarPro Gauss-Newton update (Alg. "UPDATE-PARAM-VarPro", Sec. 4.2) --------
    int varpro_setup()
    {
        if (vp_a) return CT_OK;
        const long long m_all = std::max(m, m_cap);
        const int v_all = std::max(h.V, v_cap);
        SV_TRY(alloc(vp_a, m_all));
        SV_TRY(alloc(vp_u, n));
        for (double **p : {&vp_E, &vp_G, &vp_Y}) SV_TRY(alloc(*p, (size_t)kVpMax * v_all));
        SV_TRY(alloc(vp_idel, v_all));
        SV_TRY(alloc(vp_ones, v_all));
        SV_TRY(alloc(vp_scal, kScalCount));
        SV_TRY(alloc(vp_rho, 3));
        SV_TRY(alloc(vp_ctl, kCtlCount));
        k_fill<double><<<grid_for(v_all), kThreads, 0, h.stream>>>(vp_ones, v_all, 1.0);
        SV_CUDA(cudaMemsetAsync(vp_ctl, 0, sizeof(int) * kCtlCount, h.stream));
        SV_CUDA(cudaMemsetAsync(vp_scal, 0, sizeof(double) * kScalCount, h.stream));
        SV_CUDA(cudaFuncSetAttribute(k_varpro_direction, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(VpShared)));
        return CT_OK;
    }

    // f(theta) on V[:, :k] with G_P already formed: HV, (HV)^T HV, (HV)^T b,
    // the fixed-lambda reduced solve y, u = V y (vp_u), res = HV y - b; f goes to *fslot
    int varpro_eval(const double *theta, int k, double lam, double *fslot)
    {
        SV_TRY(project(theta, 0, k, nullptr));
        SV_CUDA(cudaMemsetAsync(GH, 0, sizeof(double) * kKMax * kKMax, h.stream));
        SV_TRY(full_gram(k));
        small_solve(k, 1.0, lam, 0.0, 0.0, 1, y, vp_scal, vp_ctl);
        k_gemv<T><<<grid_for(n), kThreads, 0, h.stream>>>(V, n, n, k, y, vp_u, T(0), T(1), nullptr, T(0), nullptr);
        k_gemv<T><<<grid_for(m), kThreads, 0, h.stream>>>(HV, m, m, k, y, res, T(0), T(1), b, T(-1), nullptr);
        SV_TRY(norms3(res, nullptr, m, norms, nullptr));
        k_varpro_value<<<1, 1, 0, h.stream>>>(norms, GP, y, k, lam, fslot);
        SV_CUDA(cudaGetLastError());
        return CT_OK;
    }

    // maxiter_p damped Gauss-Newton steps on the reduced objective over the
    // basis V[:, :k] with the weights in w and lambda_hat = lam, from
    // theta_in; the angles reached go to theta_out (device, V).  Per step:
    // f and its reduced solution at theta; a = J_theta(u) 1 (one JVP);
    // per-view dots E, |a|^2, g; G by one VJP per basis column; the
    // direction (k_varpro_direction); Armijo backtracking on f, each trial one
    // more evaluation of f.  No accepted step ends the update.  f_hist
    // (host, nullable): f before the first step and after each step.
    int varpro_update(const double *theta_in, int k, double lam, double *theta_out, double *f_hist)
    {
        if (k < 1 || k > kVpMax) return CT_ERR_ARG;
        SV_TRY(varpro_setup());
        SV_TRY(gram_psi(k, nullptr));
        SV_CUDA(cudaMemcpyAsync(th_n, theta_in, sizeof(double) * h.V, cudaMemcpyDeviceToDevice, h.stream));
        double f_last = 0.0;
        for (int it = 0; it < o.maxiter_p; ++it) {
            SV_TRY(varpro_eval(th_n, k, lam, vp_scal + kTmp0));
            {  // rounding scale of f's data term at theta (Armijo noise floor)
                const int nblk = red_blocks(m);
                k_round_scale<T><<<nblk, kThreads, 0, h.stream>>>(res, b, m, part_n);
                k_norms3_reduce<<<1, 32, 0, h.stream>>>(part_n, nblk, vp_rho, nullptr);
            }
            SV_CUDA(launch_pairs_img<T>(h, vp_u, h.F, nullptr, th_n, delta));
            SV_CUDA(launch_jvp<T>(h, vp_ones, nullptr, vp_a, h.tune.der_split, h.tune.der_vw, h.tune.der_stage));
            k_view_dots<T><<<std::min(h.V, 8 * h.num_sms), 128, 0, h.stream>>>(HV, m, k, vp_a, res, h.V, h.B, vp_E,
                                                                               j2, g);
            // G[c][j] = (H_j V_c)^T r: the basis columns in batches of max_batch, one
            // batched VJP against the shared residual per batch
            for (int c = 0; c < k; c += block()) {
                const int nb = std::min(block(), k - c);
                SV_CUDA(launch_pairs_img<T>(h, col(V, n, c), nb * h.F, nullptr, nullptr, delta));
                SV_CUDA(launch_vjp<T>(h, res, vp_G + (size_t)c * h.V, nullptr, h.tune.der_split, h.tune.der_vw,
                                      h.tune.der_stage, nb, h.tune.der_kb, 0, 0));
            }
            k_varpro_direction<<<1, 1024, sizeof(VpShared), h.stream>>>(GH, GP, lam, vp_E, vp_G, j2, g, k, h.V,
                                                                        o.mu_rel, vp_Y, vp_idel, d, vp_scal + kTmp1,
                                                                        ctl);
            SV_CUDA(cudaGetLastError());
            double fg[2], rho0;
            SV_TRY(read_doubles(vp_scal + kTmp0, 2, fg));
            SV_TRY(read_doubles(vp_rho, 1, &rho0));
            const double f0 = fg[0], gd = fg[1];
            if (it == 0 && f_hist) f_hist[0] = f0;
            f_last = f0;
            bool accepted = false;
            double alpha = o.alpha0;
            if (gd < 0.0) {
                for (int hv = 0; hv <= o.max_halvings; ++hv) {
                    if (alpha * std::fabs(gd) < armijo_u() * rho0) break;  // noise floor: no step
                    k_theta_step<<<grid_for(h.V), kThreads, 0, h.stream>>>(th_n, d, alpha, h.V, th_t);
                    SV_TRY(varpro_eval(th_t, k, lam, vp_scal + kRnorm2));
                    double ft;
                    SV_TRY(read_doubles(vp_scal + kRnorm2, 1, &ft));
                    if (ft <= f0 + o.c1 * alpha * gd) {
                        accepted = true;
                        f_last = ft;
                        break;
                    }
                    alpha *= o.beta;
                }
            }
            if (!accepted) {
                if (f_hist)
                    for (int r = it + 1; r <= o.maxiter_p; ++r) f_hist[r] = f_last;
                break;
            }
            if (f_hist) f_hist[it + 1] = f_last;
            SV_CUDA(cudaMemcpyAsync(th_n, th_t, sizeof(double) * h.V, cudaMemcpyDeviceToDevice, h.stream));
        }
        if (theta_out != th_n)
            SV_CUDA(cudaMemcpyAsync(theta_out, th_n, sizeof(double) * h.V, cudaMemcpyDeviceToDevice, h.stream));
        SV_CUDA(cudaStreamSynchronize(h.stream));
        return CT_OK;
    }

    // UPDATE-PARAM of an outer iteration (or block visit) after Compress left
    // kc columns in V: per-view AltMin, or VarPro on the compressed basis with
    // the MM weights of u and the lambda of the last Enlarge step.  th_k -> th_n.
    int param_update(int kc)
    {
        if (!o.update_theta || (o.varpro && kc < 1)) {
            SV_CUDA(cudaMemcpyAsync(th_n, th_k, sizeof(double) * h.V, cudaMemcpyDeviceToDevice, h.stream));
            return CT_OK;
        }
        if (o.shared_offset) return update_param_shared(u);
        if (!o.varpro) return update_param(u);
        k_weights<T><<<grid_for(ne), kThreads, 0, h.stream>>>(u, w, h.N, h.F, o.temporal, o.eps, nullptr);
        double lam;
        SV_TRY(read_doubles(scal + kLam, 1, &lam));
        return varpro_update(th_k, kc, lam, th_n, nullptr);
    }

    // ---- VarPro reduced objective and gradient on a given basis -----------------
    // f(theta) = min_y 1/2 |H(theta) V y - b|^2 + lambda/2 |P Psi V y|^2, and
    // grad f = J_theta(V y)^T (H(theta) V y - b) (Golub-Pereyra envelope form).
    int varpro(const double *theta, const T *Vin, int k, double lam, const T *u_w, double *fval, double *grad,
               T *u_out)
    {
        SV_TRY(setup());
        double nb[3];
        SV_TRY(norms3(b, nullptr, m, norms, nullptr));
        SV_TRY(read_doubles(norms, 3, nb));
        bnorm2 = nb[0];
        SV_CUDA(cudaMemcpyAsync(V, Vin, sizeof(T) * n * k, cudaMemcpyDeviceToDevice, h.stream));
        SV_TRY(project(theta, 0, k, nullptr));
        SV_CUDA(cudaMemsetAsync(GH, 0, sizeof(double) * kKMax * kKMax, h.stream));
        SV_TRY(full_gram(k));
        if (u_w) {
            k_weights<T><<<grid_for(ne), kThreads, 0, h.stream>>>(u_w, w, h.N, h.F, o.temporal, o.eps, nullptr);
        } else {
            k_fill<T><<<grid_for(ne), kThreads, 0, h.stream>>>(w, ne, T(1));
        }
        SV_TRY(gram_psi(k, nullptr));
        small_solve(k, 1.0, lam, 0.0, 0.0, 1, y, scal, ctl);
        k_gemv<T><<<grid_for(n), kThreads, 0, h.stream>>>(V, n, n, k, y, u, T(0), T(1), nullptr, T(0), nullptr);
        k_gemv<T><<<grid_for(m), kThreads, 0, h.stream>>>(HV, m, m, k, y, res, T(0), T(1), b, T(-1), nullptr);
        SV_TRY(norms3(res, nullptr, m, norms, nullptr));
        k_varpro_value<<<1, 1, 0, h.stream>>>(norms, GP, y, k, lam, fval);
        SV_CUDA(cudaGetLastError());
        if (grad) {
            SV_CUDA(launch_pairs_img<T>(h, u, h.F, nullptr, theta, delta));
            SV_CUDA(launch_vjp<T>(h, res, grad, nullptr, h.tune.der_split, h.tune.der_vw, h.tune.der_stage));
        }
        if (u_out) SV_CUDA(cudaMemcpyAsync(u_out, u, sizeof(T) * n, cudaMemcpyDeviceToDevice, h.stream));
        SV_CUDA(cudaStreamSynchronize(h.stream));
        return CT_OK;
    }

    // ---- streaming (Alg. "s-NL-RMM-GKS", Sec. 5) --------------------------------
    // Bind block j: its handle (views, layouts, launch shapes) on the solver's
    // stream, its data, offsets and noise norm.  Basis, image and the small
    // algebra state stay.
    int bind(const Handle &hj, const T *bj, const double *deltaj, double noise_j)
    {
        const cudaStream_t s_ = h.stream;
        h = hj;
        h.stream = s_;
        b = bj;
        delta = deltaj;
        noise = noise_j;
        m = (long long)h.V * h.B;
        double nb[3];
        SV_TRY(norms3(b, nullptr, m, norms, nullptr));
        SV_TRY(read_doubles(norms, 3, nb));
        bnorm2 = nb[0];
        return CT_OK;
    }

    // One visit of the bound block: an RMM-GKS cycle (Enlarge + Compress) from
    // the carried image and basis (kc columns), then UPDATE-PARAM for the
    // block's angles theta_j (device, updated in place).  |theta change|^2 is
    // added to *dth2.
    int visit(double *theta_j, int &kc, int &steps_out, double &lam_out, double *dth2)
    {
        SV_CUDA(cudaMemcpyAsync(th_k, theta_j, sizeof(double) * h.V, cudaMemcpyDeviceToDevice, h.stream));
        SV_TRY(project(th_k, 0, kc, nullptr));
        SV_CUDA(cudaMemsetAsync(GH, 0, sizeof(double) * kKMax * kKMax, h.stream));
        SV_TRY(full_gram(kc));
        SV_CUDA(cudaMemsetAsync(ctl, 0, sizeof(int) * kCtlCount, h.stream));
        SV_CUDA(cudaStreamSynchronize(h.stream));
        *(volatile int *)h_stop = 0;
        const int s_steps = o.k_max - o.k_min;
        for (int step = 0; step < s_steps && kc + step + 1 < KC; ++step) {
            if (step >= 2) {
                SV_CUDA(cudaEventSynchronize(ev[step & 1]));
                if (*(volatile int *)h_stop) break;
            }
            SV_TRY(run_step(kc + step));
            SV_CUDA(cudaEventRecord(ev[step & 1], h.stream));
        }
        SV_TRY(sync_ctl());
        steps_out = h_ctl[kSteps];
        const int k_used = kc + steps_out - 1;
        SV_TRY(compress(k_used, kc));
        SV_TRY(param_update(kc));
        k_norms3<double><<<red_blocks(h.V), kThreads, 0, h.stream>>>(th_n, th_k, h.V, part_n, nullptr);
        k_norms3_reduce<<<1, 32, 0, h.stream>>>(part_n, red_blocks(h.V), norms, nullptr);
        double dth3[3], lam_now[1];
        SV_TRY(read_doubles(norms, 3, dth3));
        SV_TRY(read_doubles(scal + kLam, 1, lam_now));
        *dth2 += dth3[1];
        lam_out = lam_now[0];
        SV_CUDA(cudaMemcpyAsync(theta_j, th_n, sizeof(double) * h.V, cudaMemcpyDeviceToDevice, h.stream));
        return CT_OK;
    }

    // Compress: the k_min - 1 leading directions of the reduced problem on the
    // k_used columns, then the normalized part of u outside them; kc = the
    // columns kept.
    int compress(int k_used, int &kc)
    {
        const int keep = std::min(o.k_min - 1, k_used);
        compress_basis(k_used, keep);
        for (int c0 = 0; c0 < keep; c0 += 16)  // 16 output columns per pass over V
            k_gemm_small<T><<<grid_for(n), kThreads, 0, h.stream>>>(V, n, n, k_used, W + c0,
                                                                    std::min(16, keep - c0), col(Vtmp, n, c0), n);
        SV_CUDA(cudaMemcpyAsync(V, Vtmp, sizeof(T) * n * keep, cudaMemcpyDeviceToDevice, h.stream));
        SV_TRY(dots_into(V, n, keep, u, nullptr, dots, nullptr));
        k_gemv<T><<<grid_for(n), kThreads, 0, h.stream>>>(V, n, n, keep, dots, col(V, n, keep), T(0), T(-1), u,
                                                            T(1), nullptr);
        SV_TRY(norms3(col(V, n, keep), u, n, norms, nullptr));
        double nu[3];
        SV_TRY(read_doubles(norms, 3, nu));
        kc = keep;
        if (std::sqrt(nu[0]) > 1e-14 * std::max(std::sqrt(nu[2]), 1e-300)) {
            scale(col(V, n, keep), n, 1.0 / std::sqrt(nu[0]));
            kc = keep + 1;
        }
        SV_CUDA(cudaGetLastError());
        return CT_OK;
    }

    // Alg. "s-NL-RMM-GKS": passes over the blocks, each block visited once per
    // pass, until the image and all angles change less than tol_u / tol_p
    // over a pass (or outer_iters passes).  The first basis is the GKB basis
    // of block 0.  Statistics are per pass.
    int stream_run(int nb, const Handle *const *hs, const T *const *bs, double *const *thetas,
                   const double *const *deltas, const double *noises, void *x_out, const T *x_true,
                   nlrmm_stats *st)
    {
        for (int j = 0; j < nb; ++j) {
            m_cap = std::max(m_cap, (long long)hs[j]->V * hs[j]->B);
            v_cap = std::max(v_cap, hs[j]->V);
        }
        use_graphs = false;  // a captured Enlarge step would hold one block's buffers
        SV_TRY(setup());
        double xt2 = 0.0, nb3[3];
        if (x_true) {
            SV_TRY(norms3(x_true, nullptr, n, norms, nullptr));
            SV_TRY(read_doubles(norms, 3, nb3));
            xt2 = nb3[0];
        }
        SV_TRY(bind(*hs[0], bs[0], deltas ? deltas[0] : nullptr, noises ? noises[0] : 0.0));
        SV_CUDA(cudaMemsetAsync(u, 0, sizeof(T) * n, h.stream));
        SV_CUDA(cudaMemsetAsync(uold, 0, sizeof(T) * n, h.stream));
        SV_CUDA(cudaMemsetAsync(uprev, 0, sizeof(T) * n, h.stream));
        SV_TRY(gkb(thetas[0], o.k_min));
        int kc = o.k_min;
        int rc_final = CT_ERR_NOCONV;
        if (st) std::memset(st, 0, sizeof(*st));
        for (int pass = 0; pass < o.outer_iters; ++pass) {
            const auto t0 = std::chrono::steady_clock::now();
            SV_CUDA(cudaMemcpyAsync(uprev, u, sizeof(T) * n, cudaMemcpyDeviceToDevice, h.stream));
            double dth2 = 0.0, lam = 0.0;
            int steps_pass = 0;
            for (int j = 0; j < nb; ++j) {
                SV_TRY(bind(*hs[j], bs[j], deltas ? deltas[j] : nullptr, noises ? noises[j] : 0.0));
                int steps = 0;
                SV_TRY(visit(thetas[j], kc, steps, lam, &dth2));
                steps_pass += steps;
            }
            SV_TRY(norms3(u, uprev, n, norms, nullptr));
            double du3[3];
            SV_TRY(read_doubles(norms, 3, du3));
            double rre = -1.0;
            if (x_true) {
                SV_TRY(norms3(u, x_true, n, norms, nullptr));
                double e3[3];
                SV_TRY(read_doubles(norms, 3, e3));
                rre = std::sqrt(e3[1] / std::max(xt2, 1e-300));
            }
            const double du = du3[2] > 0.0 ? std::sqrt(du3[1] / du3[2]) : INFINITY;
            const double dth = std::sqrt(dth2);
            SV_CUDA(cudaStreamSynchronize(h.stream));
            const double ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (st) {
                st->outer_done = pass + 1;
                if (pass < NLRMM_MAX_HIST) {
                    st->enlarge_steps[pass] = steps_pass;
                    st->lambda[pass] = lam;
                    st->du[pass] = du;
                    st->dtheta[pass] = dth;
                    st->rre[pass] = rre;
                    st->ms[pass] = ms;
                }
                st->breakdown |= h_ctl[kBreakdown];
            }
            if (o.stop_on_convergence && du < o.tol_u && dth < o.tol_p) {
                rc_final = CT_OK;
                if (st) st->converged = 1;
                break;
            }
        }
        if (!o.stop_on_convergence) rc_final = CT_OK;
        SV_CUDA(cudaMemcpyAsync(x_out, u, sizeof(T) * n, cudaMemcpyDeviceToDevice, h.stream));
        SV_CUDA(cudaStreamSynchronize(h.stream));
        return rc_final;
    }

    // ---- the whole solve ---------------------------------------------------------
    int run(double *theta_io, void *x_out, const T *x_true, nlrmm_stats *st)
    {
        SV_TRY(setup());
        double nb[3];
        SV_TRY(norms3(b, nullptr, m, norms, nullptr));
        SV_TRY(read_doubles(norms, 3, nb));
        bnorm2 = nb[0];
        double xt2 = 0.0;
        if (x_true) {
            SV_TRY(norms3(x_true, nullptr, n, norms, nullptr));
            SV_TRY(read_doubles(norms, 3, nb));
            xt2 = nb[0];
        }
        SV_CUDA(cudaMemcpyAsync(th_k, theta_io, sizeof(double) * h.V, cudaMemcpyDeviceToDevice, h.stream));
        SV_CUDA(cudaMemsetAsync(u, 0, sizeof(T) * n, h.stream));
        SV_CUDA(cudaMemsetAsync(uold, 0, sizeof(T) * n, h.stream));
        SV_CUDA(cudaMemsetAsync(uprev, 0, sizeof(T) * n, h.stream));
        SV_TRY(gkb(th_k, o.k_min));
        int kc = o.k_min;
        const int s = o.k_max - o.k_min;
        int rc_final = CT_ERR_NOCONV;
        if (st) {
            std::memset(st, 0, sizeof(*st));
        }
        for (int it = 0; it < o.outer_iters; ++it) {
            const auto t0 = std::chrono::steady_clock::now();
            // H(theta_k) V and its Gram data
            SV_TRY(project(th_k, 0, kc, nullptr));
            SV_CUDA(cudaMemsetAsync(GH, 0, sizeof(double) * kKMax * kKMax, h.stream));
            SV_TRY(full_gram(kc));
            SV_CUDA(cudaMemsetAsync(ctl, 0, sizeof(int) * kCtlCount, h.stream));
            SV_CUDA(cudaStreamSynchronize(h.stream));
            *(volatile int *)h_stop = 0;
            // Enlarge: predicated steps issued one step ahead of the device's stop decision
            for (int step = 0; step < s && kc + step + 1 < KC; ++step) {
                if (step >= 2) {
                    SV_CUDA(cudaEventSynchronize(ev[step & 1]));
                    if (*(volatile int *)h_stop) break;
                }
                SV_TRY(run_step(kc + step));
                SV_CUDA(cudaEventRecord(ev[step & 1], h.stream));
            }
            SV_TRY(sync_ctl());
            const int steps = h_ctl[kSteps];
            const int k_used = kc + steps - 1;  // columns the last reduced problem used
            // Compress
            SV_TRY(compress(k_used, kc));
            // parameter update
            SV_TRY(param_update(kc));
            // residual of the normal equations at H_k, new weights, appended to V
            k_weights<T><<<grid_for(ne), kThreads, 0, h.stream>>>(u, w, h.N, h.F, o.temporal, o.eps, nullptr);
            SV_CUDA(launch_prep_forward<T>(h, u, h.F, nullptr, th_k, delta));
            SV_CUDA(launch_forward<T>(h, res, 1, h.tune.fwd_kb, h.tune.fwd_split, h.tune.fwd_vw, h.tune.fwd_stage));
            axpby(res, b, m, 1.0, -1.0);
            SV_TRY(backproject(th_k, res, col(V, n, kc), nullptr));
            k_add_reg<T><<<grid_for(n), kThreads, 0, h.stream>>>(col(V, n, kc), u, w, scal, h.N, h.F, o.temporal,
                                                                nullptr);
            SV_TRY(cgs2(col(V, n, kc), kc, nullptr));
            SV_TRY(norms3(col(V, n, kc), nullptr, n, norms2, nullptr));
            // convergence data
            SV_TRY(norms3(u, uprev, n, norms, nullptr));
            double du3[3], dr[3], lam_now[1];
            SV_TRY(read_doubles(norms, 3, du3));
            SV_TRY(read_doubles(norms2, 3, dr));
            SV_TRY(read_doubles(scal + kLam, 1, lam_now));
            if (dr[0] > 0.0) {
                scale(col(V, n, kc), n, 1.0 / std::sqrt(dr[0]));
                kc += 1;
            }
            k_norms3<double><<<red_blocks(h.V), kThreads, 0, h.stream>>>(th_n, th_k, h.V, part_n, nullptr);
            k_norms3_reduce<<<1, 32, 0, h.stream>>>(part_n, red_blocks(h.V), norms, nullptr);
            double dth3[3];
            SV_TRY(read_doubles(norms, 3, dth3));
            double rre = -1.0;
            if (x_true) {
                SV_TRY(norms3(u, x_true, n, norms, nullptr));
                double e3[3];
                SV_TRY(read_doubles(norms, 3, e3));
                rre = std::sqrt(e3[1] / std::max(xt2, 1e-300));
            }
            const double du = du3[2] > 0.0 ? std::sqrt(du3[1] / du3[2]) : INFINITY;
            const double dth = std::sqrt(dth3[1]);
            SV_CUDA(cudaMemcpyAsync(th_k, th_n, sizeof(double) * h.V, cudaMemcpyDeviceToDevice, h.stream));
            SV_CUDA(cudaMemcpyAsync(uprev, u, sizeof(T) * n, cudaMemcpyDeviceToDevice, h.stream));
            SV_CUDA(cudaStreamSynchronize(h.stream));
            const double ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (st) {
                st->outer_done = it + 1;
                if (it < NLRMM_MAX_HIST) {
                    st->enlarge_steps[it] = steps;
                    st->lambda[it] = lam_now[0];
                    st->du[it] = du;
                    st->dtheta[it] = dth;
                    st->rre[it] = rre;
                    st->ms[it] = ms;
                }
                st->breakdown |= h_ctl[kBreakdown];
            }
            if (o.stop_on_convergence && du < o.tol_u && dth < o.tol_p) {
                rc_final = CT_OK;
                if (st) st->converged = 1;
                break;
            }
        }
        if (!o.stop_on_convergence) rc_final = CT_OK;
        SV_CUDA(cudaMemcpyAsync(x_out, u, sizeof(T) * n, cudaMemcpyDeviceToDevice, h.stream));
        SV_CUDA(cudaMemcpyAsync(theta_io, th_k, sizeof(double) * h.V, cudaMemcpyDeviceToDevice, h.stream));
        SV_CUDA(cudaStreamSynchronize(h.stream));
        return rc_final;
    }
};

}  // namespace

extern "C" {

void nlrmm_default_opts(nlrmm_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->k_min = 5;
    o->k_max = 25;
    o->outer_iters = 20;
    o->maxiter_p = 3;
    o->max_halvings = 20;
    o->lam_iters = 60;
    o->update_theta = 1;
    o->stop_on_convergence = 1;
    o->eps = 1e-3;
    o->tol1 = 1e-3;
    o->tau = 1.01;
    o->noise_norm = 0.0;
    o->lam_fix = 0.0;
    o->lam_lo = -10.0;
    o->lam_hi = 10.0;
    o->c1 = 1e-4;
    o->beta = 0.5;
    o->alpha0 = 1.0;
    o->mu_rel = 1e-8;
    o->tol_u = 1e-3;
    o->tol_p = 1e-4;
    o->armijo_eps = -1.0;
}

int nlrmm_gks_solve(ct_handle *H, const void *b, double *theta_inout, const double *delta, void *x_out,
                    const void *x_true, const nlrmm_opts *opts, nlrmm_stats *stats)
{
    if (!H || !b || !theta_inout || !x_out || !opts) return CT_ERR_ARG;
    const nlrmm_opts &o = *opts;
    if (o.k_min < 2 || o.k_max <= o.k_min || o.k_max + 2 > ctgb::solver::kKLimit || o.k_min > 32 ||
        o.outer_iters < 1 || o.maxiter_p < 0 || o.max_halvings < 0 || o.lam_iters < 1 || !(o.eps > 0.0) ||
        !(o.tau > 0.0) || (o.lam_fix <= 0.0 && !(o.noise_norm > 0.0)))
        return CT_ERR_ARG;
    if ((o.plain != 0 && o.plain != 1) || (o.shared_offset != 0 && o.shared_offset != 1) ||
        (o.shared_offset && o.varpro))
        return CT_ERR_ARG;
    ctgb::Handle &h = H->h;
    h.fwd_ready = h.adj_ready = h.img_ready = 0;
    // The solve runs on a private stream ordered after the work already queued
    // on the handle's stream; it synchronises before returning.
    cudaStream_t ps = nullptr;
    cudaEvent_t e0 = nullptr;
    if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(e0, h.stream) != cudaSuccess || cudaStreamWaitEvent(ps, e0, 0) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        if (ps) cudaStreamDestroy(ps);
        return CT_ERR_CUDA;
    }
    int rc;
    if (h.precision) {
        Solver<double> s(h, ps, o, (const double *)b, delta);
        rc = s.run(theta_inout, x_out, (const double *)x_true, stats);
    } else {
        Solver<float> s(h, ps, o, (const float *)b, delta);
        rc = s.run(theta_inout, x_out, (const float *)x_true, stats);
    }
    cudaStreamSynchronize(ps);
    cudaEventDestroy(e0);
    cudaStreamDestroy(ps);
    return rc;
}

int nlrmm_stream_solve(ct_handle *const *blocks, int nblocks, const void *const *b, double *const *theta_inout,
                       const double *const *delta, const double *noise_norms, void *x_out, const void *x_true,
                       const nlrmm_opts *opts, nlrmm_stats *stats)
{
    if (!blocks || nblocks < 1 || !b || !theta_inout || !x_out || !opts) return CT_ERR_ARG;
    const nlrmm_opts &o = *opts;
    if (o.k_min < 2 || o.k_max <= o.k_min || o.k_max + 2 > ctgb::solver::kKLimit || o.k_min > 32 ||
        o.outer_iters < 1 || o.maxiter_p < 0 || o.max_halvings < 0 || o.lam_iters < 1 || !(o.eps > 0.0) ||
        !(o.tau > 0.0) || (o.lam_fix <= 0.0 && !noise_norms))
        return CT_ERR_ARG;
    if ((o.plain != 0 && o.plain != 1) || o.shared_offset != 0 ||
        (o.shared_offset && o.varpro))
        return CT_ERR_ARG;
    std::vector<const ctgb::Handle *> hs(nblocks);
    for (int j = 0; j < nblocks; ++j) {
        if (!blocks[j] || !b[j] || !theta_inout[j]) return CT_ERR_ARG;
        const ctgb::Handle &hj = blocks[j]->h;
        const ctgb::Handle &h0 = blocks[0]->h;
        if (hj.N != h0.N || hj.F != h0.F || hj.precision != h0.precision || hj.device != h0.device)
            return CT_ERR_ARG;
        if (o.lam_fix <= 0.0 && !(noise_norms[j] > 0.0)) return CT_ERR_ARG;
        hs[j] = &hj;
    }
    for (int j = 0; j < nblocks; ++j) blocks[j]->h.fwd_ready = blocks[j]->h.adj_ready = blocks[j]->h.img_ready = 0;
    ctgb::Handle &h = blocks[0]->h;
    cudaStream_t ps = nullptr;
    cudaEvent_t e0 = nullptr;
    if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        if (ps) cudaStreamDestroy(ps);
        return CT_ERR_CUDA;
    }
    // ordered after the work already queued on every block's stream
    for (int j = 0; j < nblocks; ++j) {
        if (cudaEventRecord(e0, blocks[j]->h.stream) != cudaSuccess || cudaStreamWaitEvent(ps, e0, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaEventDestroy(e0);
            cudaStreamDestroy(ps);
            return CT_ERR_CUDA;
        }
    }
    int rc;
    if (h.precision) {
        Solver<double> s(h, ps, o, (const double *)b[0], delta ? delta[0] : nullptr);
        rc = s.stream_run(nblocks, hs.data(), (const double *const *)b, theta_inout, delta, noise_norms, x_out,
                          (const double *)x_true, stats);
    } else {
        Solver<float> s(h, ps, o, (const float *)b[0], delta ? delta[0] : nullptr);
        rc = s.stream_run(nblocks, hs.data(), (const float *const *)b, theta_inout, delta, noise_norms, x_out,
                          (const float *)x_true, stats);
    }
    cudaStreamSynchronize(ps);
    cudaEventDestroy(e0);
    cudaStreamDestroy(ps);
    return rc;
}

int nlrmm_varpro(ct_handle *H, const void *b, const double *theta, const double *delta, const void *V, int k,
                 double lam, const void *u_w, double eps, double *fval, double *grad, void *u_out)
{
    if (!H || !b || !theta || !V || !fval || k < 1 || k + 2 > ctgb::solver::kKLimit || !(lam > 0.0) ||
        (u_w && !(eps > 0.0)))
        return CT_ERR_ARG;
    ctgb::Handle &h = H->h;
    h.fwd_ready = h.adj_ready = h.img_ready = 0;
    nlrmm_opts o;
    nlrmm_default_opts(&o);
    o.k_min = 2;
    o.k_max = k;
    o.eps = eps > 0.0 ? eps : 1e-3;
    o.lam_fix = lam;
    cudaStream_t ps = nullptr;
    cudaEvent_t e0 = nullptr;
    if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(e0, h.stream) != cudaSuccess || cudaStreamWaitEvent(ps, e0, 0) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        if (ps) cudaStreamDestroy(ps);
        return CT_ERR_CUDA;
    }
    int rc;
    if (h.precision) {
        Solver<double> s(h, ps, o, (const double *)b, delta);
        rc = s.varpro(theta, (const double *)V, k, lam, (const double *)u_w, fval, grad, (double *)u_out);
    } else {
        Solver<float> s(h, ps, o, (const float *)b, delta);
        rc = s.varpro(theta, (const float *)V, k, lam, (const float *)u_w, fval, grad, (float *)u_out);
    }
    cudaStreamSynchronize(ps);
    cudaEventDestroy(e0);
    cudaStreamDestroy(ps);
    return rc;
}

int nlrmm_varpro_update(ct_handle *H, const void *b, double *theta_inout, const double *delta, const void *V, int k,
                        double lam, const void *u_w, double eps, const nlrmm_opts *opts, double *f_hist)
{
    if (!H || !b || !theta_inout || !V || k < 1 || k > ctgb::solver::kVpMax || !(lam > 0.0) ||
        (u_w && !(eps > 0.0)))
        return CT_ERR_ARG;
    nlrmm_opts o;
    nlrmm_default_opts(&o);
    if (opts) {
        if (opts->maxiter_p < 0 || opts->max_halvings < 0 || !(opts->beta > 0.0 && opts->beta < 1.0) ||
            !(opts->alpha0 > 0.0) || !(opts->mu_rel >= 0.0))
            return CT_ERR_ARG;
        o.maxiter_p = opts->maxiter_p;
        o.max_halvings = opts->max_halvings;
        o.c1 = opts->c1;
        o.beta = opts->beta;
        o.alpha0 = opts->alpha0;
        o.mu_rel = opts->mu_rel;
        o.temporal = opts->temporal;
        o.armijo_eps = opts->armijo_eps;
        if (opts->plain != 0 && opts->plain != 1) return CT_ERR_ARG;
        o.plain = opts->plain;
    }
    ctgb::Handle &h = H->h;
    h.fwd_ready = h.adj_ready = h.img_ready = 0;
    o.k_min = 2;
    o.k_max = std::max(k, 3);
    o.eps = u_w ? eps : 1e-3;
    o.lam_fix = lam;
    cudaStream_t ps = nullptr;
    cudaEvent_t e0 = nullptr;
    if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(e0, h.stream) != cudaSuccess || cudaStreamWaitEvent(ps, e0, 0) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        if (ps) cudaStreamDestroy(ps);
        return CT_ERR_CUDA;
    }
    auto run = [&](auto tag) -> int {
        using T = decltype(tag);
        Solver<T> s(h, ps, o, (const T *)b, delta);
        SV_TRY(s.setup());
        SV_CUDA(cudaMemcpyAsync(s.V, V, sizeof(T) * s.n * k, cudaMemcpyDeviceToDevice, ps));
        if (u_w) {
            k_weights<T><<<s.grid_for(s.ne), kThreads, 0, ps>>>((const T *)u_w, s.w, h.N, h.F, o.temporal, o.eps,
                                                                   nullptr);
        } else {
            k_fill<T><<<s.grid_for(s.ne), kThreads, 0, ps>>>(s.w, s.ne, T(1));
        }
        SV_CUDA(cudaGetLastError());
        return s.varpro_update(theta_inout, k, lam, theta_inout, f_hist);
    };
    const int rc = h.precision ? run(double(0)) : run(float(0));
    cudaStreamSynchronize(ps);
    cudaEventDestroy(e0);
    cudaStreamDestroy(ps);
    return rc;
}

}  // extern "C"
