/*
 * ctgb -- angle-dependent parallel-beam CT operators (GB300 / sm_103a).
 *
 * C ABI of the hot path of NL-RMM-GKS (nonlinear recycled MM-GKS with
 * uncertain forward operators).  The forward model is H(p)u + e = b
 * (Eq. (1.1)); the joint problem is min_{u,p} 1/2 ||H(p)u - b||^2 +
 * lambda ||Psi u||_1 (Eq. (1.2), Eq. (4.1)).  Here H(p) is the Radon
 * transform at perturbed view angles (Sec. 6.2), discretised with the
 * Joseph rule, and p holds one angle theta_v per view (plus, optionally,
 * one detector offset delta_v per view).
 *
 * Geometry (unit pixels, unit bins):
 *   image   N x N, row-major X[i*N + j], pixel centre x_j = j - (N-1)/2,
 *           y_i = (N-1)/2 - i
 *   bins    B, bin centre s_b = b - (B-1)/2 + delta_v
 *   ray     x cos(theta_v) + y sin(theta_v) = s_b
 *   Joseph  |cos| >= |sin|: one linear interpolation per image row at
 *           x = (s_b - y_i sin)/cos, weight 1/|cos|; otherwise one per
 *           column at y = (s_b - x_j cos)/sin, weight 1/|sin|; pixels outside
 *           the image are zero.  The axis is decided on theta itself: rows
 *           iff fmod(theta, pi) (+ pi when negative) <= pi/4 or >= 3pi/4,
 *           with the doubles nearest pi, pi/4, 3pi/4 (exact operations, so
 *           the decision does not depend on the last bit of a sine).
 *
 * Frames (block-diagonal operator of the dynamic problem, Sec. 7): the flat
 * view list is split into consecutive frames, views_per_frame[f] views for
 * frame f; views of frame f see image f.  An "image" argument is therefore
 * n_frames * N * N elements and a "sinogram" n_views * B elements.  A batch
 * of K images / sinograms is K such blocks back to back (the Krylov block
 * H V of Sec. 3.2, stored column by column).
 *
 * Conventions for every call below:
 *   * All array arguments are DEVICE pointers owned by the caller, on the
 *     device that was current at ct_init.  Element type of images and
 *     sinograms is float (precision 0) or double (precision 1); angle,
 *     offset and gradient arrays are always double.
 *   * Calls are asynchronous on the stream given to ct_init; they never
 *     synchronise.  A handle is bound to that stream and is not thread safe.
 *   * Outputs are overwritten, never accumulated into.
 *   * Return value: CT_OK (0) or a negative CT_ERR_* code; on error nothing
 *     has been launched.  ct_status() synchronises and reports device-side
 *     conditions (non-finite angles) found by earlier calls.
 */
#ifndef CTGB_H
#define CTGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CT_OK = 0,
    CT_ERR_ARG = -1,      /* null pointer, bad size or batch out of range */
    CT_ERR_CUDA = -2,     /* a CUDA runtime call failed (see ct_last_cuda_error) */
    CT_ERR_OOM = -3,      /* device allocation failed in ct_init / the solver */
    CT_ERR_TIMEOUT = -4,  /* a bounded device-side wait ran out */
    CT_ERR_NAN = -5,      /* non-finite angle / offset or solver breakdown */
    CT_ERR_NOCONV = -6    /* solver hit its iteration limit; outputs are valid */
};

typedef struct {
    int32_t N;                        /* image side, 2 <= N <= 4096 */
    int32_t B;                        /* detector bins, 1 <= B */
    int32_t n_views;                  /* total views over all frames */
    int32_t n_frames;                 /* >= 1 */
    const int32_t *views_per_frame;   /* HOST array of n_frames counts, or NULL for one frame */
    int32_t max_batch;                /* largest batch any call will pass, >= 1 */
    int32_t use_offsets;              /* reserved: offsets are accepted whenever delta != NULL */
    int32_t precision;                /* 0 = float32 images/sinograms, 1 = float64 */
    double source_distance;           /* 0: parallel beam.  > 0: fan beam (the geometry of the
                                         paper's CT experiments, Sec. 6.2, whose distances it does not
                                         give): point source at this distance (pixels) from the
                                         rotation centre, flat detector rescaled to the line through
                                         the centre, bin b centred at s_b = b - (B-1)/2 + delta_v on
                                         it; ray (v,b) joins the source and s_b (cos, sin)(theta_v).
                                         Must exceed 0.75 max(N, B) + 2.  Fan-beam handles run H, H^T,
                                         the angle and offset derivatives and the solvers (an offset
                                         moves the bin centres along the detector line; the source
                                         stays). */
} ct_geom;

typedef struct ct_handle ct_handle;

/*
 * Create a handle: copies the geometry, allocates the workspaces it needs
 * on the current device (per-view tables; zero-padded "pair" copies of
 * max_batch images, of their transposes and of max_batch sinograms, about
 * 4 x 8 bytes per pixel and 8 bytes per sample and image in float32; the
 * reduction partials) and binds it to cuda_stream (a cudaStream_t; NULL =
 * legacy default stream).  *out receives the handle.
 */
int ct_init(const ct_geom *g, void *cuda_stream, ct_handle **out);

/* Release every workspace of the handle (synchronises its stream first). */
void ct_destroy(ct_handle *h);

/*
 * Y = H(theta, delta) X for a batch of `batch` images (forward projection
 * "H u" in the residual of every MM-GKS step, Eq. (3.6), Alg. "Enlarge").
 *   theta  [n_views] radians; delta [n_views] bins or NULL (zero offsets)
 *   X      [batch][n_frames][N][N]      Y [batch][n_views][B]
 *
 * Image reuse (this call, ct_jac, ct_jacT, ct_gn_terms and the batched
 * forms): every call that takes images lays them out in the handle (pairs
 * of neighbouring pixels along rows and along columns; for this call, with
 * tuning value [11] = 1 on an FP32 parallel-beam handle, the images
 * interleaved in groups of 4 instead, see ct_set_tuning).  Passing X (x) =
 * NULL uses the layouts of the previous such call on the handle again,
 * i.e. that call's first `batch` images, at this call's angles and offsets:
 * the Jacobian and its transpose at one image (a Gauss-Newton step, an
 * inner least-squares solve on J) then lay the image out once.  A Jacobian
 * product after a forward on interleaved images first turns them into pair
 * layouts (one more kernel launch); the results are the same either way.
 * CT_ERR_ARG when no layouts are current (none yet, or an error,
 * ct_autotune or a solver call on the handle since) or batch exceeds that
 * call's.  Calls that take no image (ct_adjoint, the repeats) keep them.
 * No counterpart in the paper.
 */
int ct_forward(ct_handle *h, const double *theta, const double *delta,
               const void *X, void *Y, int batch);

/*
 * X = H(theta, delta)^T Y, the exact transpose of ct_forward in gather form
 * (one thread per pixel, no atomics); used in the residual
 * H^T (H u - b) + lambda Psi^T P^2 Psi u of every MM-GKS step (Eq. (3.6)).
 *   Y [batch][n_views][B]  ->  X [batch][n_frames][N][N]
 */
int ct_adjoint(ct_handle *h, const double *theta, const double *delta,
               const void *Y, void *X, int batch);

/*
 * Rerun only the projection kernel of the last ct_forward (ct_adjoint) call
 * on this handle, on the angles, offsets and inputs that call laid out in
 * the handle, writing Y (X) for its first `batch` images (sinograms).  For
 * callers that need the same product again (and for timing the kernel
 * alone).  No counterpart in the paper.  CT_ERR_ARG when batch exceeds that
 * call's batch, or when any other call on the handle (ct_forward for
 * ct_adjoint_repeat and the reverse, ct_jac, ct_jacT, ct_gn_terms,
 * ct_autotune, the solvers) has run since.  Same layouts as ct_forward
 * (ct_adjoint); the inputs of that call need not be alive any more.
 */
int ct_forward_repeat(ct_handle *h, void *Y, int batch);
int ct_adjoint_repeat(ct_handle *h, void *X, int batch);

/*
 * Angle (and offset) Jacobian-vector product of the forward projection at a
 * fixed image x: dy[v,b] = dtheta_v d(Hx)[v,b]/dtheta_v
 *                        + ddelta_v d(Hx)[v,b]/ddelta_v
 * (the columns H_{p_i} u of Alg. "UPDATE-PARAM").  The derivative of the
 * linear interpolation uses the slope of the cell floor(u) (right derivative
 * at integer u).
 *   x [n_frames][N][N] or NULL (the image of the previous call, see
 *   ct_forward), dtheta [n_views] (device, double),
 *   ddelta [n_views] or NULL, dy [n_views][B]
 */
int ct_jac(ct_handle *h, const double *theta, const double *delta,
           const void *x, const double *dtheta, const double *ddelta,
           void *dy);

/*
 * Transposed Jacobian: gtheta[v] = sum_b r[v,b] d(Hx)[v,b]/dtheta_v and
 * gdelta[v] = sum_b r[v,b] d(Hx)[v,b]/ddelta_v (gradient of the data term
 * with respect to p, (H_{p_i} u)^T (H u - b), appendix lemma on the
 * Lipschitz gradient).  Per-view sums are reduced in a fixed order (no
 * atomics): results are bitwise reproducible.
 *   x [n_frames][N][N] or NULL (the image of the previous call, see
 *   ct_forward), r [n_views][B], gtheta [n_views] (device double),
 *   gdelta [n_views] or NULL
 */
int ct_jacT(ct_handle *h, const double *theta, const double *delta,
            const void *x, const void *r, double *gtheta, double *gdelta);

/*
 * Fused per-view Gauss-Newton terms at image x and data b, one ray march:
 *   res[v,b]  = (H x)[v,b] - bdata[v,b]          (may be NULL: not stored)
 *   grad[v]   = sum_b res[v,b] d(Hx)[v,b]/dtheta_v
 *   jnorm2[v] = sum_b (d(Hx)[v,b]/dtheta_v)^2
 *   fval[v]   = 1/2 sum_b res[v,b]^2
 * With per-view angles the Gauss-Newton matrix J^T J of Alg. "UPDATE-PARAM"
 * is diagonal, so these four arrays are all the parameter update needs.
 * grad, jnorm2, fval: [n_views] device double (fval may be NULL); x may be
 * NULL (the image of the previous call, see ct_forward).
 */
int ct_gn_terms(ct_handle *h, const double *theta, const double *delta,
                const void *x, const void *bdata, void *res, double *grad,
                double *jnorm2, double *fval);

/*
 * Batched Jacobian products: `batch` images x_k (1 <= batch <= max_batch)
 * sharing the angles and offsets, one ray-march launch for the whole batch
 * (the block V of basis vectors of Sec. 3.2 whose sensitivities H_{p_i} V_c
 * enter the VarPro Gauss-Newton system of Sec. 4.2, Alg.
 * "UPDATE-PARAM-VarPro"; the batched backward of the autograd projection).
 * Each image's result equals the single-image call's (ct_jac, ct_jacT,
 * ct_gn_terms) on that image, up to the summation order within a ray.
 *
 * ct_jac_batch: dY[k][v,b] = dtheta_k[v] d(H x_k)[v,b]/dtheta_v
 *                           (+ ddelta_k[v] d(H x_k)[v,b]/ddelta_v)
 *   X [batch][n_frames][N][N]; dY [batch][n_views][B];
 *   dtheta, ddelta (nullable): [n_views] shared by every image, or
 *   [batch][n_views] with flags & CT_BATCH_PER_IMAGE_DIRECTION.
 * ct_jacT_batch: gtheta[k][v] = sum_b R_k[v,b] d(H x_k)[v,b]/dtheta_v (and gdelta)
 *   R [batch][n_views][B], or one [n_views][B] shared by every image with
 *   flags & CT_BATCH_SHARED_R; gtheta, gdelta (nullable) [batch][n_views], or
 *   with flags & CT_BATCH_SUM one [n_views] vector: the sum over the images,
 *   added in image order after each image's fixed-order sum over bins (the
 *   gradient of sum_k <R_k, H(theta) x_k> with respect to theta).
 * ct_gn_terms_batch: the four ct_gn_terms outputs for each image, against
 *   data bdata [batch][n_views][B]: res [batch][n_views][B] (nullable),
 *   grad, jnorm2, fval (nullable) [batch][n_views].
 * X may be NULL: the first `batch` images of the previous call that took
 * images (see ct_forward).
 * CT_ERR_ARG for batch out of range, null required pointers or unknown flags.
 */
#define CT_BATCH_PER_IMAGE_DIRECTION 1
#define CT_BATCH_SHARED_R 2
#define CT_BATCH_SUM 4
int ct_jac_batch(ct_handle *h, const double *theta, const double *delta, const void *X, const double *dtheta,
                 const double *ddelta, void *dY, int batch, int flags);
int ct_jacT_batch(ct_handle *h, const double *theta, const double *delta, const void *X, const void *R,
                  double *gtheta, double *gdelta, int batch, int flags);
int ct_gn_terms_batch(ct_handle *h, const double *theta, const double *delta, const void *X, const void *bdata,
                      void *res, double *grad, double *jnorm2, double *fval, int batch);

/*
 * Rebind the handle to another stream (for example a stream being captured
 * into a CUDA graph).  Later calls launch on it.
 */
int ct_set_stream(ct_handle *h, void *cuda_stream);

/*
 * Pick launch shapes for this handle's geometry by timing the candidates on
 * its stream: images per lane (1, 2, 4, 8), warps per ray (1, 2, 4, 8) and
 * neighbouring views per CTA (1, 2, 4, 8) for the forward projection at
 * max_batch, images per thread and view groups per pixel tile (1, 2, 4) for
 * the transpose, warps per ray and views per CTA for the Jacobian kernels
 * (and, for max_batch > 1, images per lane of the batched ones),
 * and (FP32 handles) the staged forms: the forward and Jacobian kernels
 * with 4 or 8 views per CTA, 4 or 8 rows per shared-memory block and 1, 2
 * or 4 CTAs per ray, the transpose with 8 or 16 views per block and 1, 2 or
 * 4 CTAs per tile.  Synchronises; allocates and frees scratch buffers; must not run
 * during stream capture.  Results of every operator are independent of the
 * chosen shapes up to floating-point summation order.
 */
int ct_autotune(ct_handle *h);

/*
 * Read / set the launch shapes, CT_TUNING_COUNT values:
 *   [0] forward images per lane, [1] forward warps per ray (row segments),
 *   [2] forward views per CTA, [3] transpose images per thread,
 *   [4] transpose view groups per pixel tile, [5] Jacobian warps per ray,
 *   [6] Jacobian views per CTA, [7] forward staging, [8] Jacobian staging,
 *   [9] transpose staging, [10] images per lane of the batched Jacobian
 *   products (1, 2 or 4; the staged and fan-beam forms take 1), [11] forward
 *   image layout: 0 pair images (each pixel stored beside its neighbour), 1
 *   images interleaved in groups of 4 (FP32 parallel-beam handles, forward
 *   staging 0, [0] 4 or 8; the forward then reads both taps of 4 images with
 *   two 16-byte loads; a later call that passes X = NULL to a Jacobian
 *   product converts them to pair images first).  Layout 1 allocates two
 *   buffers of max_batch x n_frames x N x (N + 4) floats the first time
 *   (CT_ERR_OOM if that fails; CT_ERR_ARG on an FP64 or fan-beam handle).
 * [0]..[6] are powers of two, at most 8 (view groups at most 4), warps per
 * ray x views per CTA at most 16 (unstaged kernels).  Forward / Jacobian
 * staging is 0 (gathers through L1) or 4 / 8 (rows per shared-memory block of
 * the band-staged march, which needs 4 or 8 views per CTA).  Transpose
 * staging is 0 or 8 / 16 (views per shared-memory block of the staged
 * transpose).  Staging applies to FP32 handles only.  With forward staging,
 * [1] is the number of CTAs sharing one ray (row segments, at most 4); with
 * transpose staging, [4] is the number of CTAs sharing one pixel tile (view
 * subsets).  A value above 1 there allocates a workspace of
 * 3 x max_batch x max(V x B, F x N x N) floats the first time (CT_ERR_OOM if
 * that fails).  The Jacobian kernels ignore [5] when staged.  CT_ERR_ARG for
 * any other value.
 */
#define CT_TUNING_COUNT 12
int ct_get_tuning(ct_handle *h, int32_t *out);
int ct_set_tuning(ct_handle *h, const int32_t *in);

/*
 * Measure, on the current device, the read bandwidth of the two on-chip
 * levels that serve the operators' gathers (a microbenchmark with no
 * counterpart in the paper; it gives the measured denominators of the
 * gather roofline):
 *   *l2_read_gbs    float4 loads that bypass L1 over a 48 MB buffer held
 *                   in L2, all SMs, GB/s;
 *   *smem_read_gbs  conflict-free 16-byte shared-memory loads, all SMs, GB/s.
 * Best of 5 timed launches each.  Allocates and frees 48 MB; synchronises a
 * private stream.  CT_ERR_ARG for null outputs, CT_ERR_OOM, CT_ERR_CUDA.
 */
int ct_measure_peaks(double *l2_read_gbs, double *smem_read_gbs);

/* ------------------------------------------------------------------------
 * NL-RMM-GKS (alternating form) on the handle's geometry.
 * ------------------------------------------------------------------------ */
#define NLRMM_MAX_HIST 256

typedef struct {
    int32_t k_min;          /* compressed basis size (Sec. 6 default 5); 2 <= k_min <= 32 */
    int32_t k_max;          /* enlarged basis size (default 25); k_min < k_max <= 120 (bases above 62
                               columns keep the FP64 small algebra in a device work area) */
    int32_t outer_iters;    /* outer iteration limit */
    int32_t maxiter_p;      /* Gauss-Newton iterations per outer iteration (default 3) */
    int32_t max_halvings;   /* Armijo backtracking halvings (default 20) */
    int32_t lam_iters;      /* step limit of the discrepancy-principle search for lambda (default 60;
                               the device runs safeguarded Newton steps in log10 lambda, at most
                               lam_iters + 2 evaluations, stopping at |phi - target| <= 1e-10 target) */
    int32_t update_theta;   /* 0: angles fixed (the solve is RMM-GKS) */
    int32_t stop_on_convergence; /* stop when du < tol_u and dtheta < tol_p */
    double eps;             /* smoothing of the l1 term, P = diag((z^2 + eps^2)^(-1/4)) (default 1e-3) */
    double tol1;            /* Enlarge stops when |u_new - u_old| <= tol1 |u_old| (default 1e-3) */
    double tau;             /* discrepancy safety factor (default 1.01) */
    double noise_norm;      /* |e| for the discrepancy principle (required unless lam_fix > 0) */
    double lam_fix;         /* > 0: fixed lambda instead of the discrepancy principle */
    double lam_lo, lam_hi;  /* log10 bracket of lambda (default -10, 10) */
    double c1, beta, alpha0;/* Armijo constants (default 1e-4, 0.5, 1) */
    double mu_rel;          /* damping mu = mu_rel * max_v |J_v|^2 (default 1e-8) */
    double tol_u, tol_p;    /* outer stopping tolerances (default 1e-3, 1e-4) */
    int32_t temporal;       /* 1: ANISO-TV, Psi also takes the difference of consecutive frames
                               (operator D_1 of Alg. "Dynamic NL-RMM-GKS"); default 0 */
    int32_t varpro;         /* 1: parameter update by Alg. "UPDATE-PARAM-VarPro" (Sec. 4.2) on the
                               compressed basis (see nlrmm_varpro_update) instead of the per-view
                               AltMin update; default 0 */
    double armijo_eps;      /* noise floor of the Armijo searches: a search whose first-order change
                               alpha |g d| of the misfit f = 1/2 |r|^2 is below armijo_eps * rho, with
                               rho = sum_b |r_b| (|(H u)_b| + |b_b|) the rounding scale of f (one view's
                               residual in the AltMin update, the data residual of the reduced
                               objective in the VarPro update), ends before that trial with no
                               acceptable step: its test would compare two misfits closer than their
                               rounding (the paper's descent lemmas assume exact arithmetic).  < 0
                               (default): the unit roundoff of the handle's precision, 2^-24 (float32
                               residuals) or 2^-53; 0: no floor */
    int32_t plain;          /* 1: the unpackaged form, for comparison: no CUDA graphs, every projection
                               of the basis one column per launch (no Krylov-block batching), the
                               Armijo flag read after every trial round; same iterates.  Default 0 */
    int32_t shared_offset;  /* 1: one angle offset p shared by every view and frame, theta_v = theta_v^0 + p
                               (the scalar parameter of the paper's CT experiments, Sec. 6.2, shared by
                               all frames in its dynamic CT, Sec. 7): Gauss-Newton on p with gradient
                               sum_v g_v and J^T J = sum_v |J_v|^2 (damped by mu_rel J^T J), Armijo and
                               its noise floor on the total misfit; no accepted step ends the update.
                               Not with varpro, not in nlrmm_stream_solve.  Default 0: one angle per view */
} nlrmm_opts;

typedef struct {
    int32_t outer_done;     /* outer iterations run */
    int32_t converged;      /* stopping rule met */
    int32_t breakdown;      /* a pivot of the reduced problem's L D L^T was clamped or a residual vanished */
    int32_t enlarge_steps[NLRMM_MAX_HIST];
    double lambda[NLRMM_MAX_HIST];   /* lambda of the last Enlarge step */
    double du[NLRMM_MAX_HIST];       /* |u_{k+1} - u_k| / |u_k| */
    double dtheta[NLRMM_MAX_HIST];   /* |theta_{k+1} - theta_k| */
    double rre[NLRMM_MAX_HIST];      /* |u - x_true| / |x_true| (-1 without x_true) */
    double ms[NLRMM_MAX_HIST];       /* wall time of the outer iteration, milliseconds */
} nlrmm_stats;

/* Fill *opts with the defaults above. */
void nlrmm_default_opts(nlrmm_opts *opts);

/*
 * Joint reconstruction min_{u,theta} 1/2 |H(theta) u - b|^2 + lambda |Psi u|_1
 * (Eq. (4.1)) by alternating NL-RMM-GKS (Alg. "NL-RMM-GKS" without the
 * high-lambda solve): per outer iteration one Enlarge (<= k_max - k_min
 * MM-GKS steps, lambda by the discrepancy principle on the projected
 * problem) and one Compress of the generalized Krylov basis at the current
 * angles, then per-view damped Gauss-Newton with Armijo backtracking on the
 * angles (Alg. "UPDATE-PARAM"; with opts->varpro, the VarPro update of
 * nlrmm_varpro_update on the compressed basis with the MM weights of the new
 * image and the last lambda), then the normal-equation residual appended
 * to the basis.  Psi = forward differences per frame (with opts->temporal,
 * also between consecutive frames: ANISO-TV).  The basis starts
 * from k_min Golub-Kahan steps on b and u starts at zero.
 *   b [n_views][B] (device, handle precision); theta_inout [n_views] device
 *   double, initial angles in, estimated angles out; delta [n_views] or NULL
 *   (fixed offsets); x_out [n_frames][N][N] device; x_true (nullable) for
 *   the RRE history; stats (host, nullable).
 * Operators run in the handle's precision; every small matrix is FP64 on the
 * device.  Allocates its workspace (about (k_max + 2)(n + m) elements) on
 * entry and frees it on return; synchronises the handle's stream.  Returns
 * CT_OK, CT_ERR_NOCONV (iteration limit reached with stopping enabled;
 * outputs valid), CT_ERR_ARG, CT_ERR_OOM or CT_ERR_CUDA.
 */
int nlrmm_gks_solve(ct_handle *h, const void *b, double *theta_inout, const double *delta, void *x_out,
                    const void *x_true, const nlrmm_opts *opts, nlrmm_stats *stats);

/*
 * Streaming NL-RMM-GKS over blocks of views (Alg. "s-NL-RMM-GKS", Sec. 5,
 * blocks as in Sec. 2.4): each pass visits the blocks in order; a visit is
 * one Enlarge + Compress on block j's data, started from the carried image
 * and compressed basis, then per-view Gauss-Newton with Armijo (with
 * opts->varpro: the VarPro update of nlrmm_varpro_update) on block j's
 * angles; the compressed basis (k_min columns) goes on to the next block.
 * Passes repeat until the image and all angles change less than tol_u /
 * tol_p over a pass, or outer_iters passes.  The first basis is k_min
 * Golub-Kahan steps on block 0's data; u starts at zero; no residual is
 * appended after a parameter update (the next block's first Enlarge step
 * appends its own).
 *   blocks [nblocks]      host array of handles, one per block (its views);
 *                         same N, n_frames, precision and device; each
 *                         keeps its own launch shapes
 *   b [nblocks]           host array of device [V_j][B] data
 *   theta_inout [nblocks] host array of device [V_j] double angles, updated
 *   delta                 host array of device [V_j] offsets (entries may be
 *                         NULL) or NULL: no offsets
 *   noise_norms [nblocks] host, |e_j| for block j's discrepancy principle
 *                         (NULL allowed when opts->lam_fix > 0)
 *   x_out [n_frames][N][N] device; x_true nullable, for the RRE history
 *   stats                 one entry per pass: Enlarge steps summed over the
 *                         blocks, lambda of the last block, du, dtheta (all
 *                         blocks), rre, ms
 * Workspace about (k_max + 2)(n + max_j m_j) elements, allocated on entry and
 * freed on return; runs on a private stream ordered after every block's
 * stream and synchronises it.  CT_OK, CT_ERR_NOCONV, CT_ERR_ARG, CT_ERR_OOM,
 * CT_ERR_CUDA.
 */
int nlrmm_stream_solve(ct_handle *const *blocks, int nblocks, const void *const *b, double *const *theta_inout,
                       const double *const *delta, const double *noise_norms, void *x_out, const void *x_true,
                       const nlrmm_opts *opts, nlrmm_stats *stats);

/*
 * VarPro reduced objective on a fixed basis (Sec. 4.2, Alg.
 * "UPDATE-PARAM-VarPro"): with the image restricted to span(V) and the MM
 * weights frozen,
 *   f(theta) = min_y 1/2 |H(theta) V y - b|^2 + lam/2 |P Psi V y|^2,
 *   P^2 = diag((z^2 + eps^2)^(-1/2)), z = Psi u_w   (u_w == NULL: P = I),
 * and its gradient grad[v] = d f / d theta_v.  y is optimal for every theta,
 * so the gradient is J_theta(u)^T (H(theta) u - b) at u = V y (the
 * Golub-Pereyra / envelope form): one batched projection of V, the FP64
 * reduced solve and one transposed-Jacobian pass; nothing of the inner solve
 * is kept between calls.
 *   b [n_views][B]; theta, delta [n_views] device double (delta nullable);
 *   V [k][n_frames][N][N] device, k <= 120 columns; u_w [n_frames][N][N] or NULL;
 *   fval: one device double; grad [n_views] device double or NULL;
 *   u_out [n_frames][N][N] device or NULL.
 * Allocates and frees its workspace; synchronises.  CT_OK, CT_ERR_ARG,
 * CT_ERR_OOM or CT_ERR_CUDA.
 */
int nlrmm_varpro(ct_handle *h, const void *b, const double *theta, const double *delta, const void *V, int k,
                 double lam, const void *u_w, double eps, double *fval, double *grad, void *u_out);

/*
 * One VarPro parameter update (Alg. "UPDATE-PARAM-VarPro", Sec. 4.2) on a
 * fixed basis: opts->maxiter_p damped Gauss-Newton steps on the reduced
 * objective f(theta) of nlrmm_varpro, each followed by Armijo backtracking on
 * f (c1, beta, alpha0, at most max_halvings halvings; when no step is
 * accepted the angles stay and the update ends).  The Gauss-Newton matrix is
 * J_r^T J_r + lam J_s^T J_s of the reduced residuals r = H(theta) V y(theta) - b
 * and s = P Psi V y(theta), whose columns follow the sensitivity equation
 * restricted to span(V); it is a diagonal plus a rank-2k term, damped by
 * mu = mu_rel * its largest diagonal entry and solved by the Woodbury identity
 * (FP64).  The gradient is J_theta(V y)^T r.  Per step: one projection of the
 * k basis columns per evaluation of f, one JVP, k VJPs.
 *   b [n_views][B]; theta_inout [n_views] device double, updated in place;
 *   delta [n_views] device or NULL; V [k][n_frames][N][N] device, 1 <= k <= 32;
 *   lam > 0; u_w [n_frames][N][N] device or NULL (P = I), eps > 0 with u_w;
 *   opts: maxiter_p, max_halvings, c1, beta, alpha0, mu_rel, temporal are
 *   read (NULL: defaults); f_hist (host, nullable): maxiter_p + 1 values,
 *   f before the first step and after each step (repeated once the update ends).
 * Allocates and frees its workspace; synchronises.  CT_OK, CT_ERR_ARG,
 * CT_ERR_OOM or CT_ERR_CUDA.
 */
int nlrmm_varpro_update(ct_handle *h, const void *b, double *theta_inout, const double *delta, const void *V, int k,
                        double lam, const void *u_w, double eps, const nlrmm_opts *opts, double *f_hist);

/* ------------------------------------------------------------------------
 * Allocation-free transposed Jacobian (this entry point has no counterpart in
 * the paper; it exists for callers that cannot allocate device memory).
 * ------------------------------------------------------------------------ */
#define CTGB_NOALLOC_MAX_N 256      /* image side */
#define CTGB_NOALLOC_MAX_VIEWS 512  /* views */
#define CTGB_NOALLOC_MAX_BINS 1024  /* detector bins */

/*
 * Same result as ct_jacT (float32, one frame) without a handle and without
 * allocating: for callers that cannot call cudaMalloc, such as a host
 * application that owns all device memory through its own pool, or a
 * service whose device-memory budget is fixed after start-up.
 *   N, B, n_views   geometry (as in ct_geom), at most the CTGB_NOALLOC_MAX_*
 *                   limits above; larger sizes return CT_ERR_ARG
 *   theta, delta    [n_views] device double (delta may be NULL)
 *   x               [N][N] device float image;  r [n_views][B] device float
 *   gtheta, gdelta  [n_views] device double outputs (gdelta may be NULL)
 *   cuda_stream     cudaStream_t the kernels run on (NULL = legacy default)
 * The workspace is a file-scope device array of about 1.7 MB compiled into
 * the library, so every GPU that loads the library holds it until the
 * process exits.  The first call made on a device looks up that array's
 * device address (cudaGetSymbolAddress) for the device current at the call;
 * make that first call before any stream capture.  All calls share the one
 * array: calls that may overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  No cudaMalloc,
 * cudaFree or allocating library routine is called.  A view whose angle or
 * offset is not finite gets NaN in gtheta (and gdelta): there is no status
 * call here (ct_jacT reports the same input through ct_status).  Returns
 * CT_OK, CT_ERR_ARG or CT_ERR_CUDA; asynchronous, like ct_jacT.
 */
int ct_jacT_noalloc(int32_t N, int32_t B, int32_t n_views, const double *theta, const double *delta,
                    const float *x, const float *r, double *gtheta, double *gdelta, void *cuda_stream);

/*
 * Synchronise the handle's stream and report device-side conditions found
 * since the last ct_status: CT_ERR_NAN if a non-finite angle or offset was
 * passed, CT_ERR_CUDA on an asynchronous CUDA error, else CT_OK.
 */
int ct_status(ct_handle *h);

/* Static description of an error code. */
const char *ct_strerror(int code);

/* Text of the last CUDA runtime error seen by this library (thread-local). */
const char *ct_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CTGB_H */
