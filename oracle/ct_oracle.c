/*
 * FP64 CPU oracle for the angle-dependent parallel-beam CT operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header or constant with the CUDA
 * path.
 *
 * What it computes (the forward model H(p)u of Eq. (1.1) with p = per-view
 * angles theta_v and optional per-view detector offsets delta_v; the paper's
 * CT experiments use "the Radon transform at perturbed angles", Sec. 6.2):
 *
 *   image      N x N, row-major X[i*N + j]; pixel (i,j) centre at
 *              x_j = j - (N-1)/2,  y_i = (N-1)/2 - i   (unit pixels)
 *   detector   B bins, bin b centre s_b = b - (B-1)/2 + delta_v
 *   ray (v,b)  { (x,y) : x cos(theta_v) + y sin(theta_v) = s_b }
 *
 *   Joseph rule.  If |cos| >= |sin| the ray is sampled once per image row i
 *   (decided on theta itself, see march_rows):
 *   x = (s_b - y_i sin)/cos, column coordinate u = x + (N-1)/2, linear
 *   interpolation between columns floor(u) and floor(u)+1 (pixels outside
 *   the image are zero), weight 1/|cos| (path length per row).  Otherwise it
 *   is sampled once per column j: y = (s_b - x_j cos)/sin, row coordinate
 *   t = (N-1)/2 - y, interpolation between rows floor(t), floor(t)+1,
 *   weight 1/|sin|.
 *
 * The angle derivative d(Hu)/dtheta_v (the Jacobian columns H_{p_i} u of
 * Algorithm "UPDATE-PARAM", Sec. 4.1.2) is the exact derivative of the
 * expression above, taking the slope of the interpolation cell floor(u)
 * (right derivative at the kinks where u is an integer).  Each function is
 * written as a plain loop over rays and samples; nothing is blocked, fused
 * or reordered.
 *
 * Frames: view v reads the image of frame fov[v] (block-diagonal H of the
 * dynamic problem, Sec. 7); fov == NULL means every view reads frame 0.
 */
#include <math.h>
#include <stddef.h>
#include <string.h>

/*
 * Joseph axis of a view: rows iff |cos theta| >= |sin theta|, i.e. iff theta
 * mod pi lies in [0, pi/4] or [3pi/4, pi).  Decided on theta with exact
 * operations (fmod is exact; one rounded addition for negative angles) and
 * the doubles nearest pi, pi/4 and 3pi/4, so that any implementation of this
 * rule takes the same decision; evaluating |cos| >= |sin| on a library's
 * cosine and sine could go either way within an ulp of the diagonals.  It
 * differs from the exact rule only within about 3e-16 rad of a diagonal.
 */
static int march_rows(double theta)
{
    const double pi = 3.14159265358979323846, q1 = 0.78539816339744830962, q3 = 2.35619449019234492885;
    double t = fmod(theta, pi);
    if (t < 0.0)
        t += pi;
    return t <= q1 || t >= q3;
}

/* Pixel value with the zero extension outside the image. */
static double pixel(const double *X, int N, int i, int j)
{
    if (i < 0 || i >= N || j < 0 || j >= N)
        return 0.0;
    return X[(size_t)i * N + j];
}

/*
 * One ray.  Returns the line integral and, if requested, its derivatives
 * with respect to theta and delta.
 */
static void ray_integral(const double *X, int N, int B, double theta,
                         double delta, int b, double *val, double *d_theta,
                         double *d_delta)
{
    const double c = cos(theta), s = sin(theta);
    const double h = 0.5 * (N - 1);
    const double sb = (b - 0.5 * (B - 1)) + delta;
    double sum = 0.0, sum_theta = 0.0, sum_delta = 0.0;
    double w, dw;

    if (march_rows(theta)) {
        /* march over rows */
        w = 1.0 / fabs(c);
        dw = (c > 0 ? 1.0 : -1.0) * s / (c * c); /* d(1/|cos|)/dtheta */
        for (int i = 0; i < N; i++) {
            const double y = h - i;
            const double x = (sb - y * s) / c;
            const double u = x + h;
            const double u0 = floor(u);
            const int j0 = (int)u0;
            const double f = u - u0;
            const double v0 = pixel(X, N, i, j0);
            const double v1 = pixel(X, N, i, j0 + 1);
            const double slope = v1 - v0;
            sum += (1.0 - f) * v0 + f * v1;
            sum_theta += slope * (sb * s - y) / (c * c); /* du/dtheta */
            sum_delta += slope / c;                      /* du/ddelta */
        }
    } else {
        /* march over columns */
        w = 1.0 / fabs(s);
        dw = -(s > 0 ? 1.0 : -1.0) * c / (s * s); /* d(1/|sin|)/dtheta */
        for (int j = 0; j < N; j++) {
            const double x = j - h;
            const double y = (sb - x * c) / s;
            const double t = h - y;
            const double t0 = floor(t);
            const int i0 = (int)t0;
            const double f = t - t0;
            const double v0 = pixel(X, N, i0, j);
            const double v1 = pixel(X, N, i0 + 1, j);
            const double slope = v1 - v0;
            sum += (1.0 - f) * v0 + f * v1;
            sum_theta += slope * (sb * c - x) / (s * s); /* dt/dtheta */
            sum_delta += slope * (-1.0 / s);             /* dt/ddelta */
        }
    }
    *val = w * sum;
    if (d_theta)
        *d_theta = dw * sum + w * sum_theta;
    if (d_delta)
        *d_delta = w * sum_delta;
}

static const double *frame_image(const double *X, int N, const int *fov, int v)
{
    const int f = fov ? fov[v] : 0;
    return X + (size_t)f * N * N;
}

/* Y[v*B + b] = (H(theta, delta) X)[v, b]. */
void orc_forward(int N, int B, int V, const int *fov, const double *theta,
                 const double *delta, const double *X, double *Y)
{
    for (int v = 0; v < V; v++) {
        const double *Xv = frame_image(X, N, fov, v);
        const double dl = delta ? delta[v] : 0.0;
        for (int b = 0; b < B; b++)
            ray_integral(Xv, N, B, theta[v], dl, b, &Y[(size_t)v * B + b],
                         NULL, NULL);
    }
}

/*
 * X = H(theta, delta)^T Y by scattering: every ray adds its interpolation
 * weights times Y[v,b] into the two pixels it sampled.  X (n_frames images)
 * is overwritten.
 */
void orc_adjoint(int N, int B, int V, int n_frames, const int *fov,
                 const double *theta, const double *delta, const double *Y,
                 double *X)
{
    memset(X, 0, sizeof(double) * (size_t)n_frames * N * N);
    const double h = 0.5 * (N - 1);
    for (int v = 0; v < V; v++) {
        double *Xv = X + (size_t)(fov ? fov[v] : 0) * N * N;
        const double c = cos(theta[v]), s = sin(theta[v]);
        const double dl = delta ? delta[v] : 0.0;
        for (int b = 0; b < B; b++) {
            const double yv = Y[(size_t)v * B + b];
            const double sb = (b - 0.5 * (B - 1)) + dl;
            if (march_rows(theta[v])) {
                const double w = 1.0 / fabs(c);
                for (int i = 0; i < N; i++) {
                    const double u = (sb - (h - i) * s) / c + h;
                    const double u0 = floor(u);
                    const int j0 = (int)u0;
                    const double f = u - u0;
                    if (j0 >= 0 && j0 < N)
                        Xv[(size_t)i * N + j0] += w * (1.0 - f) * yv;
                    if (j0 + 1 >= 0 && j0 + 1 < N)
                        Xv[(size_t)i * N + j0 + 1] += w * f * yv;
                }
            } else {
                const double w = 1.0 / fabs(s);
                for (int j = 0; j < N; j++) {
                    const double t = h - (sb - (j - h) * c) / s;
                    const double t0 = floor(t);
                    const int i0 = (int)t0;
                    const double f = t - t0;
                    if (i0 >= 0 && i0 < N)
                        Xv[(size_t)i0 * N + j] += w * (1.0 - f) * yv;
                    if (i0 + 1 >= 0 && i0 + 1 < N)
                        Xv[(size_t)(i0 + 1) * N + j] += w * f * yv;
                }
            }
        }
    }
}

/*
 * Per-sample derivatives: Dth[v,b] = d(HX)[v,b]/dtheta_v and
 * Ddl[v,b] = d(HX)[v,b]/ddelta_v (either may be NULL).
 */
void orc_dsample(int N, int B, int V, const int *fov, const double *theta,
                 const double *delta, const double *X, double *Dth,
                 double *Ddl)
{
    for (int v = 0; v < V; v++) {
        const double *Xv = frame_image(X, N, fov, v);
        const double dl = delta ? delta[v] : 0.0;
        for (int b = 0; b < B; b++) {
            double val, dt, dd;
            ray_integral(Xv, N, B, theta[v], dl, b, &val, &dt, &dd);
            if (Dth)
                Dth[(size_t)v * B + b] = dt;
            if (Ddl)
                Ddl[(size_t)v * B + b] = dd;
        }
    }
}

/*
 * Jacobian-vector product: dY[v,b] = dtheta_v d(HX)/dtheta_v
 *                                  + ddelta_v d(HX)/ddelta_v.
 * ddelta may be NULL (no offset direction).
 */
void orc_jac(int N, int B, int V, const int *fov, const double *theta,
             const double *delta, const double *X, const double *dtheta,
             const double *ddelta, double *dY)
{
    for (int v = 0; v < V; v++) {
        const double *Xv = frame_image(X, N, fov, v);
        const double dl = delta ? delta[v] : 0.0;
        for (int b = 0; b < B; b++) {
            double val, dt, dd;
            ray_integral(Xv, N, B, theta[v], dl, b, &val, &dt, &dd);
            double out = dtheta[v] * dt;
            if (ddelta)
                out += ddelta[v] * dd;
            dY[(size_t)v * B + b] = out;
        }
    }
}

/*
 * Transposed Jacobian: g_theta[v] = sum_b R[v,b] d(HX)[v,b]/dtheta_v and
 * g_delta[v] = sum_b R[v,b] d(HX)[v,b]/ddelta_v (g_delta may be NULL).
 * This is the gradient [grad_p J]_i = (H_{p_i} u)^T (H u - b) of the
 * Lipschitz-gradient lemma of the appendix when R is the residual.
 */
void orc_jacT(int N, int B, int V, const int *fov, const double *theta,
              const double *delta, const double *X, const double *R,
              double *g_theta, double *g_delta)
{
    for (int v = 0; v < V; v++) {
        const double *Xv = frame_image(X, N, fov, v);
        const double dl = delta ? delta[v] : 0.0;
        double gt = 0.0, gd = 0.0;
        for (int b = 0; b < B; b++) {
            double val, dt, dd;
            ray_integral(Xv, N, B, theta[v], dl, b, &val, &dt, &dd);
            gt += R[(size_t)v * B + b] * dt;
            gd += R[(size_t)v * B + b] * dd;
        }
        g_theta[v] = gt;
        if (g_delta)
            g_delta[v] = gd;
    }
}

/*
 * Fan-beam variant (the paper's CT experiments are fan-beam, Sec. 6.2; its
 * source and detector distances are not given).  Reading: point source at
 * distance D from the rotation centre, flat detector rescaled to the line
 * through the centre, so bin b keeps the parallel-beam centre s_b on that
 * line.  With t = (-sin, cos) (the parallel-beam ray direction) and
 * e = (cos, sin) (the detector axis), the source sits at S = -D t, bin b at
 * P_b = s_b e, and ray (v,b) is the line through S and P_b, direction
 * r = P_b - S = (s_b cos - D sin, s_b sin + D cos).  As D -> infinity it
 * becomes the parallel-beam ray { x cos + y sin = s_b }.
 *
 * Joseph rule per ray: rows if |r_x| <= |r_y| (one sample per image row,
 * x(y) = A + C y with C = r_x / r_y, A = P_x - P_y C), else columns
 * (y(x) = A + C x with C = r_y / r_x, A = P_y - P_x C); weight sqrt(1 + C^2)
 * (path length per row or column).  Interpolation, zero extension and the
 * kink convention as for the parallel beam.
 *
 * Derivatives: the geometry rotates rigidly with theta, so dr/dtheta =
 * (-r_y, r_x) and dP_b/dtheta = s_b (-sin, cos); with respect to delta,
 * dr/ds_b = dP_b/ds_b = e.  Hence, for rows,
 *   dC/dtheta = -(1 + C^2),  dA/dtheta = dP_x - C dP_y - P_y dC/dtheta,
 *   dC/ds = (cos r_y - sin r_x) / r_y^2,  dA/ds = cos - C sin - P_y dC/ds,
 * for columns
 *   dC/dtheta = 1 + C^2,  dA/dtheta = dP_y - C dP_x - P_x dC/dtheta,
 *   dC/ds = (sin r_x - cos r_y) / r_x^2,  dA/ds = sin - C cos - P_x dC/ds,
 * and dw = C dC / w.
 */
static void fan_ray(const double *X, int N, int B, double D, double theta,
                    double delta, int b, double *val, double *d_theta,
                    double *d_delta)
{
    const double c = cos(theta), sn = sin(theta);
    const double h = 0.5 * (N - 1);
    const double s = (b - 0.5 * (B - 1)) + delta;
    const double rx = s * c - D * sn, ry = s * sn + D * c;
    const double px = s * c, py = s * sn;
    const double dpx = -s * sn, dpy = s * c; /* dP_b/dtheta */
    double sum = 0.0, st = 0.0, sd = 0.0;
    double C, A, w, dC, dA, dw, dCs, dAs, dws;

    if (fabs(rx) <= fabs(ry)) {
        /* one sample per image row */
        C = rx / ry;
        A = px - py * C;
        w = sqrt(1.0 + C * C);
        dC = -(1.0 + C * C);
        dA = dpx - C * dpy - py * dC;
        dCs = (c * ry - sn * rx) / (ry * ry);
        dAs = c - C * sn - py * dCs;
        for (int i = 0; i < N; i++) {
            const double y = h - i;
            const double u = A + C * y + h;
            const double u0 = floor(u);
            const int j0 = (int)u0;
            const double f = u - u0;
            const double v0 = pixel(X, N, i, j0);
            const double v1 = pixel(X, N, i, j0 + 1);
            const double slope = v1 - v0;
            sum += (1.0 - f) * v0 + f * v1;
            st += slope * (dA + y * dC); /* du/dtheta */
            sd += slope * (dAs + y * dCs); /* du/ds */
        }
    } else {
        /* one sample per image column */
        C = ry / rx;
        A = py - px * C;
        w = sqrt(1.0 + C * C);
        dC = 1.0 + C * C;
        dA = dpy - C * dpx - px * dC;
        dCs = (sn * rx - c * ry) / (rx * rx);
        dAs = sn - C * c - px * dCs;
        for (int j = 0; j < N; j++) {
            const double x = j - h;
            const double t = h - (A + C * x);
            const double t0 = floor(t);
            const int i0 = (int)t0;
            const double f = t - t0;
            const double v0 = pixel(X, N, i0, j);
            const double v1 = pixel(X, N, i0 + 1, j);
            const double slope = v1 - v0;
            sum += (1.0 - f) * v0 + f * v1;
            st += slope * (-(dA + x * dC)); /* dt/dtheta */
            sd += slope * (-(dAs + x * dCs)); /* dt/ds */
        }
    }
    dw = C * dC / w;
    dws = C * dCs / w;
    *val = w * sum;
    if (d_theta)
        *d_theta = dw * sum + w * st;
    if (d_delta)
        *d_delta = dws * sum + w * sd;
}

/* Fan-beam Y[v*B + b] = (H(theta, delta) X)[v, b], source distance D. */
void orc_fan_forward(int N, int B, int V, const int *fov, double D,
                     const double *theta, const double *delta, const double *X,
                     double *Y)
{
    for (int v = 0; v < V; v++) {
        const double *Xv = frame_image(X, N, fov, v);
        const double dl = delta ? delta[v] : 0.0;
        for (int b = 0; b < B; b++)
            fan_ray(Xv, N, B, D, theta[v], dl, b, &Y[(size_t)v * B + b], NULL,
                    NULL);
    }
}

/* Fan-beam X = H^T Y by scattering the interpolation weights of every ray. */
void orc_fan_adjoint(int N, int B, int V, int n_frames, const int *fov,
                     double D, const double *theta, const double *delta,
                     const double *Y, double *X)
{
    memset(X, 0, sizeof(double) * (size_t)n_frames * N * N);
    const double h = 0.5 * (N - 1);
    for (int v = 0; v < V; v++) {
        double *Xv = X + (size_t)(fov ? fov[v] : 0) * N * N;
        const double c = cos(theta[v]), sn = sin(theta[v]);
        const double dl = delta ? delta[v] : 0.0;
        for (int b = 0; b < B; b++) {
            const double yv = Y[(size_t)v * B + b];
            const double s = (b - 0.5 * (B - 1)) + dl;
            const double rx = s * c - D * sn, ry = s * sn + D * c;
            const double px = s * c, py = s * sn;
            if (fabs(rx) <= fabs(ry)) {
                const double C = rx / ry, A = px - py * C;
                const double w = sqrt(1.0 + C * C);
                for (int i = 0; i < N; i++) {
                    const double u = A + C * (h - i) + h;
                    const double u0 = floor(u);
                    const int j0 = (int)u0;
                    const double f = u - u0;
                    if (j0 >= 0 && j0 < N)
                        Xv[(size_t)i * N + j0] += w * (1.0 - f) * yv;
                    if (j0 + 1 >= 0 && j0 + 1 < N)
                        Xv[(size_t)i * N + j0 + 1] += w * f * yv;
                }
            } else {
                const double C = ry / rx, A = py - px * C;
                const double w = sqrt(1.0 + C * C);
                for (int j = 0; j < N; j++) {
                    const double t = h - (A + C * (j - h));
                    const double t0 = floor(t);
                    const int i0 = (int)t0;
                    const double f = t - t0;
                    if (i0 >= 0 && i0 < N)
                        Xv[(size_t)i0 * N + j] += w * (1.0 - f) * yv;
                    if (i0 + 1 >= 0 && i0 + 1 < N)
                        Xv[(size_t)(i0 + 1) * N + j] += w * f * yv;
                }
            }
        }
    }
}

/* Fan-beam per-sample derivatives (d/dtheta_v, d/ddelta_v of (HX)[v,b]). */
void orc_fan_dsample(int N, int B, int V, const int *fov, double D,
                     const double *theta, const double *delta, const double *X,
                     double *Dth, double *Ddl)
{
    for (int v = 0; v < V; v++) {
        const double *Xv = frame_image(X, N, fov, v);
        const double dl = delta ? delta[v] : 0.0;
        for (int b = 0; b < B; b++) {
            double val, dt, dd;
            fan_ray(Xv, N, B, D, theta[v], dl, b, &val, &dt, &dd);
            if (Dth)
                Dth[(size_t)v * B + b] = dt;
            if (Ddl)
                Ddl[(size_t)v * B + b] = dd;
        }
    }
}
