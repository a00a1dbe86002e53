/*
 * FP64 CPU oracle for the OS-TV statistical iterative MVCT reconstruction of
 * Ozaki et al. (arXiv:1903.10088). TEST INFRASTRUCTURE ONLY: it is loaded by the
 * tests, by the smoke check and by the benchmark's CPU-baseline leg, never by the
 * product path. It shares no code with the CUDA library.
 *
 * Plain, slow, obviously correct: every operator is written out the way the
 * method defines it, in double precision, with no blocking, fusion or
 * reordering. It runs on one thread unless oracle_set_threads() asks for more
 * (a timed CPU baseline over all host cores); then only two loops are shared
 * out, each without changing a single rounding: the reprojection's rays (each
 * ray's sum is its own) and the transpose's views (every view still scatters
 * into its own private image, and the view images are added to the result in
 * view order, pixel by pixel). Results are bit-identical for any thread count.
 *
 *   Problem (Sec. 2, Eq. 1-2): maximise ln P(mu|y) = L(mu) + alpha R(mu) subject
 *     to mu > 0; L from Poisson statistics, R the total variation.
 *     Reading used here: L is the penalised-weighted-least-squares (log-domain
 *     quadratic) form of the Poisson likelihood and R = -TV_eps, i.e. minimise
 *     Psi(mu) = 1/2 sum_i w_i ([A mu]_i - p_i)^2 + beta TV_eps(mu).
 *   Reprojection (Sec. 4.4, "reprojection"): A = Joseph fan-beam projector.
 *   Estimation (Sec. 4.4): the transpose A^T, written as a literal scatter.
 *   Gradient step (Eq. 3) with adaptive lambda (Eq. 4-5, lambda0 = 0.01,
 *     +1e-4 when the square difference falls, -2e-4 when it rises).
 *   Homogeneous initial image mu0 (Sec. 3.3.2).
 *   Ordered subsets by thinning the views at a fixed spacing; the
 *     regulariser weight multiplied by the thinning parameter 1/S (Sec. 3.4).
 *   Best iterate at the minimum of the oscillating square difference (Sec. 4.2).
 *
 * Parity status of each function (what pins it) is stated in its comment.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads used by oracle_forward / oracle_back (1 unless set). */
static int g_threads = 1;

/* Set the thread count (clamped to >= 1); returns the count in effect, which is
 * 1 when the library was built without OpenMP. */
int oracle_set_threads(int threads)
{
#ifdef _OPENMP
    g_threads = threads < 1 ? 1 : threads;
#else
    (void)threads;
    g_threads = 1;
#endif
    return g_threads;
}

typedef struct {
    int32_t n;              /* image n x n, row-major, row i = y, column j = x */
    double fov_cm;          /* pixel size delta = fov_cm / n */
    double sad_cm;          /* source to isocentre */
    double sdd_cm;          /* source to detector (does not enter an arc detector's line integrals) */
    int32_t n_views;        /* V, uniform over 2 pi */
    int32_t n_channels;     /* C, equiangular */
    double view0_rad;       /* angle of view 0 */
    double fan_angle_rad;   /* <= 0 selects 2 asin((fov/2)/sad) */
    double channel_offset;  /* in channels */
} oracle_geometry;

typedef struct {
    double lambda0;         /* Eq. 4-5: initial convergence parameter, 0.01 */
    double dlambda_up;      /* Eq. 4: +1e-4 when the square difference decreased */
    double dlambda_down;    /* Eq. 5: -2e-4 when it increased */
    double lambda_min;      /* floor on lambda (reading: lambda stays positive) */
    double kappa;           /* step tau = kappa * lambda on the preconditioned gradient */
    double tv_eps;          /* smoothing inside the TV square root */
    double mu0;             /* homogeneous initial value, 1/cm (Sec. 3.3.2) */
    int32_t init_from_input;/* 1: start from the caller's image instead of mu0 */
    int32_t data_term;      /* 0: weighted least squares on log projections; 1: Poisson log-likelihood */
    const int32_t *subset_order; /* S entries, a permutation of 0..S-1 visited cyclically; NULL: 0, 1, ..., S-1 */
    int32_t lambda_rule;    /* which square difference drives Eq. 4-5 (see oracle_recon) */
} oracle_recon_params;

/* Readings of Sec. 3.3.2 (lambda follows the squared difference between the
 * reprojection and the measured projection) under ordered subsets, where a
 * sub-iteration sees only its own subset (Sec. 3.4). */
enum {
    LAMBDA_SUBSET = 0,       /* Phi_n against Phi_{n-1}: consecutive sub-iterations (different subsets) */
    LAMBDA_PASS = 1,         /* once per pass: the sum over the last complete pass against the pass before */
    LAMBDA_PASS_SLIDING = 2  /* every sub-iteration: the pass sum P_n = Phi_{n-S+1} + ... + Phi_n against
                                P_{n-1}, i.e. Phi_n against Phi_{n-S} (the same subset one pass earlier) */
};

static const double PI = 3.14159265358979323846;

static double fan_angle(const oracle_geometry *g)
{
    if (g->fan_angle_rad > 0) return g->fan_angle_rad;
    return 2.0 * asin((g->fov_cm / 2.0) / g->sad_cm);
}

/* Source point and unit direction of ray (view v, channel c). */
static void ray(const oracle_geometry *g, int v, int c,
                double *sx, double *sy, double *dx, double *dy)
{
    double beta = g->view0_rad + 2.0 * PI * (double)v / (double)g->n_views;
    double gamma = ((double)c - (g->n_channels - 1) / 2.0 + g->channel_offset)
                   * (fan_angle(g) / (double)g->n_channels);
    double bx = -cos(beta), by = -sin(beta);        /* towards the isocentre */
    *sx = g->sad_cm * cos(beta);
    *sy = g->sad_cm * sin(beta);
    *dx = cos(gamma) * bx - sin(gamma) * by;         /* rotate by the channel angle */
    *dy = sin(gamma) * bx + cos(gamma) * by;
}

static double pixel_centre(const oracle_geometry *g, int k)
{
    double delta = g->fov_cm / g->n;
    return ((double)k - (g->n - 1) / 2.0) * delta;
}

/* Joseph line integral of img along one ray.
 * If |dx| >= |dy| the ray is x-driven: for every column j, take the ray's height
 * y at the column centre, interpolate linearly between the two rows that
 * bracket it (rows outside the image read 0) and sum; the sum times
 * delta/|dx| (the path length per column) is the integral. Otherwise the same
 * with rows and columns exchanged. */
static double joseph_ray(const oracle_geometry *g, const double *img, int v, int c)
{
    int n = g->n;
    double delta = g->fov_cm / n;
    double origin = pixel_centre(g, 0);
    double sx, sy, dx, dy;
    ray(g, v, c, &sx, &sy, &dx, &dy);
    double sum = 0.0;
    if (fabs(dx) >= fabs(dy)) {
        for (int j = 0; j < n; ++j) {
            double y = sy + (pixel_centre(g, j) - sx) * dy / dx;
            double u = (y - origin) / delta;
            double fl = floor(u);
            int i0 = (int)fl;
            double f = u - fl;
            if (i0 >= 0 && i0 < n) sum += (1.0 - f) * img[(size_t)i0 * n + j];
            if (i0 + 1 >= 0 && i0 + 1 < n) sum += f * img[(size_t)(i0 + 1) * n + j];
        }
        return sum * delta / fabs(dx);
    } else {
        for (int i = 0; i < n; ++i) {
            double x = sx + (pixel_centre(g, i) - sy) * dx / dy;
            double u = (x - origin) / delta;
            double fl = floor(u);
            int j0 = (int)fl;
            double f = u - fl;
            if (j0 >= 0 && j0 < n) sum += (1.0 - f) * img[(size_t)i * n + j0];
            if (j0 + 1 >= 0 && j0 + 1 < n) sum += f * img[(size_t)i * n + j0 + 1];
        }
        return sum * delta / fabs(dy);
    }
}

/* The transpose of joseph_ray: scatter value * (the same weights) into acc. */
static void joseph_ray_transpose(const oracle_geometry *g, double value, int v, int c, double *acc)
{
    int n = g->n;
    double delta = g->fov_cm / n;
    double origin = pixel_centre(g, 0);
    double sx, sy, dx, dy;
    ray(g, v, c, &sx, &sy, &dx, &dy);
    if (fabs(dx) >= fabs(dy)) {
        double s = value * delta / fabs(dx);
        for (int j = 0; j < n; ++j) {
            double y = sy + (pixel_centre(g, j) - sx) * dy / dx;
            double u = (y - origin) / delta;
            double fl = floor(u);
            int i0 = (int)fl;
            double f = u - fl;
            if (i0 >= 0 && i0 < n) acc[(size_t)i0 * n + j] += (1.0 - f) * s;
            if (i0 + 1 >= 0 && i0 + 1 < n) acc[(size_t)(i0 + 1) * n + j] += f * s;
        }
    } else {
        double s = value * delta / fabs(dy);
        for (int i = 0; i < n; ++i) {
            double x = sx + (pixel_centre(g, i) - sy) * dx / dy;
            double u = (x - origin) / delta;
            double fl = floor(u);
            int j0 = (int)fl;
            double f = u - fl;
            if (j0 >= 0 && j0 < n) acc[(size_t)i * n + j0] += (1.0 - f) * s;
            if (j0 + 1 >= 0 && j0 + 1 < n) acc[(size_t)i * n + j0 + 1] += f * s;
        }
    }
}

/* Number of rows of a subset's sinogram and the view held in row k.
 * subset < 0: all views in natural order. Otherwise views v = subset + k*S
 * (Sec. 3.4: views thinned at a fixed spacing). */
static int subset_rows(const oracle_geometry *g, int subset, int n_subsets)
{
    return subset < 0 ? g->n_views : g->n_views / n_subsets;
}
static int subset_view(int subset, int n_subsets, int k)
{
    return subset < 0 ? k : subset + k * n_subsets;
}

static int check(const oracle_geometry *g, int subset, int n_subsets)
{
    if (!g || g->n < 1 || g->n_views < 1 || g->n_channels < 1 || !(g->fov_cm > 0)) return -1;
    if (!(g->sad_cm > g->fov_cm * sqrt(2.0) / 2.0)) return -1;
    if (n_subsets < 1 || g->n_views % n_subsets != 0) return -1;
    if (subset >= n_subsets) return -1;
    return 0;
}

/* Reprojection: sino[k][c] = (A img) for the rays of the subset.
 * Pinned by: analytic disk/ellipse integrals, exactness on affine images,
 * the axis-aligned-ray special case, and an explicit 8x8 system matrix. */
int oracle_forward(const oracle_geometry *g, const double *img, int subset, int n_subsets, double *sino)
{
    if (check(g, subset, n_subsets)) return -1;
    int rows = subset_rows(g, subset, n_subsets), C = g->n_channels;
    long long n_rays = (long long)rows * C;
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
    for (long long i = 0; i < n_rays; ++i) {
        int k = (int)(i / C), c = (int)(i % C);
        sino[i] = joseph_ray(g, img, subset_view(subset, n_subsets, k), c);
    }
    return 0;
}

/* Estimation: img = A^T sino over the subset's rays, as a literal scatter of the
 * forward weights; each view scatters into a private image and the views are
 * summed in order. Pinned by the adjoint identity and the explicit matrix. */
int oracle_back(const oracle_geometry *g, const double *sino, int subset, int n_subsets, double *img)
{
    if (check(g, subset, n_subsets)) return -1;
    size_t nn = (size_t)g->n * g->n;
    int T = g_threads;                       /* views scattered at a time */
    double *view_img = (double *)malloc((size_t)T * nn * sizeof(double));
    if (!view_img) return -2;
    memset(img, 0, nn * sizeof(double));
    int rows = subset_rows(g, subset, n_subsets);
    for (int k0 = 0; k0 < rows; k0 += T) {
        int kn = rows - k0 < T ? rows - k0 : T;
        /* views k0 .. k0+kn-1, each into its own image */
#pragma omp parallel for schedule(static, 1) num_threads(T) if (T > 1)
        for (int t = 0; t < kn; ++t) {
            int v = subset_view(subset, n_subsets, k0 + t);
            double *vi = view_img + (size_t)t * nn;
            memset(vi, 0, nn * sizeof(double));
            for (int c = 0; c < g->n_channels; ++c)
                joseph_ray_transpose(g, sino[(size_t)(k0 + t) * g->n_channels + c], v, c, vi);
        }
        /* and added to the result in view order */
#pragma omp parallel for schedule(static) num_threads(T) if (T > 1)
        for (long long r = 0; r < (long long)nn; ++r)
            for (int t = 0; t < kn; ++t) img[r] += view_img[(size_t)t * nn + r];
    }
    free(view_img);
    return 0;
}

/* Smoothed isotropic total variation (Sec. 2 names TV as the regulariser):
 *   TV_eps = sum_{i,j} sqrt(dx^2 + dy^2 + eps),
 *   dx = mu[i][j+1] - mu[i][j] (0 in the last column),
 *   dy = mu[i+1][j] - mu[i][j] (0 in the last row),
 * and, if grad is given, its exact gradient, accumulated term by term.
 * Pinned by closed forms (constant and step images) and finite differences. */
double oracle_tv(int n, const double *img, double eps, double *grad)
{
    double tv = 0.0;
    if (grad) memset(grad, 0, (size_t)n * n * sizeof(double));
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            double m = img[(size_t)i * n + j];
            double dx = (j + 1 < n) ? img[(size_t)i * n + j + 1] - m : 0.0;
            double dy = (i + 1 < n) ? img[(size_t)(i + 1) * n + j] - m : 0.0;
            double phi = sqrt(dx * dx + dy * dy + eps);
            tv += phi;
            if (grad) {
                if (j + 1 < n) {
                    grad[(size_t)i * n + j + 1] += dx / phi;
                    grad[(size_t)i * n + j] -= dx / phi;
                }
                if (i + 1 < n) {
                    grad[(size_t)(i + 1) * n + j] += dy / phi;
                    grad[(size_t)i * n + j] -= dy / phi;
                }
            }
        }
    }
    return tv;
}

/* Psi(mu) = 1/2 sum_i w_i ([A mu]_i - p_i)^2 + beta TV_eps(mu) over all views. */
double oracle_objective(const oracle_geometry *g, const double *img, const double *p, const double *w,
                        double beta, double eps)
{
    if (check(g, -1, 1)) return NAN;
    size_t R = (size_t)g->n_views * g->n_channels;
    double *q = (double *)malloc(R * sizeof(double));
    if (!q) return NAN;
    oracle_forward(g, img, -1, 1, q);
    double phi = 0.0;
    for (size_t i = 0; i < R; ++i) {
        double r = q[i] - p[i];
        phi += w[i] * r * r;
    }
    free(q);
    return 0.5 * phi + beta * oracle_tv(g->n, img, eps, NULL);
}

/* Curvature bound of TV_eps used in the separable surrogate: the Hessian of
 * sqrt(a^2+b^2+eps) is at most 1/sqrt(eps) in (a,b), and a pixel enters three
 * terms whose difference operators have absolute row sums 4, 2 and 2. */
static double tv_curvature_bound(double eps) { return 8.0 / sqrt(eps); }

/* Set-up of the loop. Support mask M_r = [(A^T 1)_r > 0] over all views (pixels
 * no ray reaches are held at 0), and the separable-quadratic-surrogate diagonal
 *   D_r = 1 / ( (A^T (w .* (A 1)))_r + beta * 8/sqrt(eps) )   on M, else 0,
 * which majorises the Hessian of Psi so that a unit step (tau = kappa*lambda = 1)
 * decreases Psi for a full-gradient step. */
int oracle_setup(const oracle_geometry *g, const double *w, double beta, double eps,
                 double *D, unsigned char *M)
{
    if (check(g, -1, 1)) return -1;
    size_t nn = (size_t)g->n * g->n, R = (size_t)g->n_views * g->n_channels;
    double *ones_img = (double *)malloc(nn * sizeof(double));
    double *t = (double *)malloc(R * sizeof(double));
    double *a1t = (double *)malloc(nn * sizeof(double));
    double *awa = (double *)malloc(nn * sizeof(double));
    if (!ones_img || !t || !a1t || !awa) { free(ones_img); free(t); free(a1t); free(awa); return -2; }
    for (size_t i = 0; i < R; ++i) t[i] = 1.0;
    oracle_back(g, t, -1, 1, a1t);                  /* A^T 1 */
    for (size_t r = 0; r < nn; ++r) ones_img[r] = 1.0;
    oracle_forward(g, ones_img, -1, 1, t);          /* A 1 */
    for (size_t i = 0; i < R; ++i) t[i] *= w[i];    /* w .* A 1 */
    oracle_back(g, t, -1, 1, awa);
    double cb = beta * tv_curvature_bound(eps);
    for (size_t r = 0; r < nn; ++r) {
        M[r] = a1t[r] > 0.0;
        D[r] = M[r] ? 1.0 / (awa[r] + cb) : 0.0;
    }
    free(ones_img); free(t); free(a1t); free(awa);
    return 0;
}

/* The ordered-subset gradient loop (Eq. 3 with Eq. 4-5, Sec. 3.3.2, 3.4, 4.2).
 *
 * Sub-iteration n = 0 .. n_iter-1 uses subset s = n mod S (or subset_order[n mod S]):
 *   q   = A_s mu                         (reprojection of the subset's views)
 *   r   = q - p_s,  Phi_n = sum r^2 (the square difference)
 *   e   = w_s .* r                    (weighted least squares, data_term 0), or
 *   e   = w_s - exp(-q)               (data_term 1: gradient of the negative Poisson
 *                                      log-likelihood sum(y q + I0 exp(-q)) divided by
 *                                      I0, with counts y = I0 w)
 *   lambda_n = lambda0 at n = 0; otherwise lambda_{n-1} + up if the square
 *              difference fell, - down if it rose, unchanged on a tie or when the
 *              rule makes no comparison at n; floored at lambda_min. Which square
 *              differences are compared (lambda_rule):
 *                SUBSET        Phi_n with Phi_{n-1} (n >= 1);
 *                PASS          at n = kS, k >= 2: Phi_{n-S} + ... + Phi_{n-1} with
 *                              Phi_{n-2S} + ... + Phi_{n-S-1} (the last two passes);
 *                PASS_SLIDING  Phi_n with Phi_{n-S} (n >= S): the pass sum P_n with P_{n-1}.
 *              (lambda_schedule, if given, replaces the rule.)
 *   g   = A_s^T e                        (estimation)
 *   mu' = max(0, mu - kappa lambda_n D .* (S g + beta grad TV_eps(mu))), 0 off M
 *        (descent on Phi_{w,s} + (beta/S) TV_eps, scaled by S to full-gradient size)
 * Best iterate: for n >= S-1 the pass sum P_n = Phi_{n-S+1} + ... + Phi_n; the
 * image mu^(n) at the first minimum of P_n is copied to best_img.
 *
 * img_inout: in = initial image if init_from_input, out = mu^(n_iter).
 * phi_out, lambda_out: n_iter entries (may be NULL). */
int oracle_recon(const oracle_geometry *g, int n_subsets, const double *p, const double *w,
                 double beta, int n_iter, const oracle_recon_params *prm,
                 const double *lambda_schedule, double *img_inout, double *best_img,
                 double *phi_out, double *lambda_out, int *best_n_out, double *best_pass_out)
{
    if (check(g, 0, n_subsets) || n_iter < 0 || !prm || !img_inout) return -1;
    int n = g->n, C = g->n_channels, S = n_subsets, Vs = g->n_views / n_subsets;
    size_t nn = (size_t)n * n, Rs = (size_t)Vs * C;
    double *D = (double *)malloc(nn * sizeof(double));
    unsigned char *M = (unsigned char *)malloc(nn);
    double *q = (double *)malloc(Rs * sizeof(double));
    double *gr = (double *)malloc(nn * sizeof(double));
    double *tvg = (double *)malloc(nn * sizeof(double));
    double *next = (double *)malloc(nn * sizeof(double));
    double *phis = (double *)malloc(((size_t)n_iter + 1) * sizeof(double));
    int rc = 0;
    if (!D || !M || !q || !gr || !tvg || !next || !phis) { rc = -2; goto done; }

    if (oracle_setup(g, w, beta, prm->tv_eps, D, M)) { rc = -1; goto done; }
    for (size_t r = 0; r < nn; ++r)
        img_inout[r] = M[r] ? (prm->init_from_input ? img_inout[r] : prm->mu0) : 0.0;

    double lambda = prm->lambda0, phi_prev = 0.0, best_pass = INFINITY;
    int best_n = -1;
    for (int it = 0; it < n_iter; ++it) {
        int s = prm->subset_order ? prm->subset_order[it % S] : it % S;
        oracle_forward(g, img_inout, s, S, q);
        double phi = 0.0;
        for (int k = 0; k < Vs; ++k) {
            int v = s + k * S;
            for (int c = 0; c < C; ++c) {
                size_t i = (size_t)k * C + c, iv = (size_t)v * C + c;
                double r = q[i] - p[iv];
                phi += r * r;
                q[i] = prm->data_term == 1 ? w[iv] - exp(-q[i])   /* e, reusing q's storage */
                                           : w[iv] * r;
            }
        }
        phis[it] = phi;
        /* the two square differences Eq. 4-5 compare at this sub-iteration, if any */
        int decide = 0;
        double now = 0.0, before = 0.0;
        if (prm->lambda_rule == LAMBDA_PASS_SLIDING) {
            if (it >= S) { decide = 1; now = phi; before = phis[it - S]; }
        } else if (prm->lambda_rule == LAMBDA_PASS) {
            if (it >= 2 * S && it % S == 0) {
                decide = 1;
                for (int k = it - S; k < it; ++k) now += phis[k];
                for (int k = it - 2 * S; k < it - S; ++k) before += phis[k];
            }
        } else if (it > 0) {
            decide = 1; now = phi; before = phi_prev;
        }
        if (lambda_schedule) {
            lambda = lambda_schedule[it];
        } else if (decide) {
            if (now < before) lambda += prm->dlambda_up;
            else if (now > before) lambda -= prm->dlambda_down;
            if (lambda < prm->lambda_min) lambda = prm->lambda_min;
        }
        phi_prev = phi;
        if (phi_out) phi_out[it] = phi;
        if (lambda_out) lambda_out[it] = lambda;

        if (it >= S - 1) {
            double pass = 0.0;
            for (int k = it - S + 1; k <= it; ++k) pass += phis[k];
            if (pass < best_pass) {
                best_pass = pass;
                best_n = it;
                if (best_img) memcpy(best_img, img_inout, nn * sizeof(double));
            }
        }

        oracle_back(g, q, s, S, gr);
        oracle_tv(n, img_inout, prm->tv_eps, tvg);
        double tau = prm->kappa * lambda;
        for (size_t r = 0; r < nn; ++r) {
            double m = img_inout[r] - tau * D[r] * ((double)S * gr[r] + beta * tvg[r]);
            next[r] = M[r] ? (m > 0.0 ? m : 0.0) : 0.0;
        }
        memcpy(img_inout, next, nn * sizeof(double));
    }
    if (best_n_out) *best_n_out = best_n;
    if (best_pass_out) *best_pass_out = best_pass;
done:
    free(D); free(M); free(q); free(gr); free(tvg); free(next); free(phis);
    return rc;
}
