/*
 * mvct.h -- C ABI of the GB300 (sm_103a) OS-TV statistical iterative MVCT
 * reconstruction library, libmvct.so.
 *
 * Method: Ozaki et al., "Fast Statistical Iterative Reconstruction for MVCT in
 * TomoTherapy", arXiv:1903.10088. The library runs the ordered-subset gradient
 * loop of Sec. 2-3 (Eq. 1-5, Sec. 3.3.2, Sec. 3.4) on one GPU: per
 * sub-iteration it reprojects the current image along the fan-beam rays of one
 * view subset, forms the weighted residual against the measured log
 * projections, backprojects it with the matched adjoint, adds the smoothed TV
 * gradient and steps with the adaptive convergence parameter.
 *
 * Conventions shared by every entry point
 *  - Image: float32, n x n, row-major, row i = y, column j = x; pixel centres
 *    x_j = (j - (n-1)/2) * delta, y_i = (i - (n-1)/2) * delta, delta = fov/n.
 *  - Sinogram: float32, view-major [rows][n_channels]. "subset = -1" means all
 *    views in natural order (rows = n_views); "subset = s" means the thinned
 *    sinogram of views v = s + k*S, k = 0 .. n_views/S - 1 (Sec. 3.4).
 *  - View v: source at sad*(cos b, sin b), b = view0 + 2 pi v / n_views.
 *    Channel c: angle g = (c - (C-1)/2 + channel_offset) * fan / C on an
 *    equiangular arc; ray direction = Rot(g) (-cos b, -sin b).
 *  - All d_* pointers are caller-owned DEVICE memory on the plan's device,
 *    float32 unless stated, contiguous, 4-byte aligned; the library never frees
 *    them. Host pointers are named without the d_ prefix.
 *  - stream is a cudaStream_t (NULL = legacy default stream). Calls are
 *    asynchronous on it except mvct_plan_create and mvct_recon (see below).
 *    A plan owns scratch buffers: calls on one plan must not overlap in time
 *    (issue them on one stream or synchronise between streams).
 *  - Return value: MVCT_OK (0) or a negative MVCT_E* code; the message of the
 *    last failure on the calling thread is returned by mvct_last_error().
 *    Arguments are validated before anything is enqueued.
 */
#ifndef MVCT_H_
#define MVCT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MVCT_OK 0
#define MVCT_EINVAL (-1)   /* invalid argument or geometry */
#define MVCT_ENOMEM (-2)   /* device or host allocation failed */
#define MVCT_ECUDA (-3)    /* a CUDA runtime call failed */
#define MVCT_ELAUNCH (-4)  /* the persistent grid cannot be co-resident */
#define MVCT_ETIMEOUT (-5) /* a grid barrier of the persistent loop timed out */
#define MVCT_EDATA (-6)    /* non-finite or negative input data */

#define MVCT_MAX_N 4096        /* largest image side */
#define MVCT_MAX_SUBSETS 1024  /* largest number of ordered subsets */
#define MVCT_NOALLOC_MAX_BLOCKS 2048 /* FP64 slots (16 KiB) of mvct_tv_grad_noalloc's static scratch */

/* Scanner and image grid (Sec. 3.1, 3.4). Lengths in cm, angles in rad. */
typedef struct mvct_geometry {
    int32_t n;              /* image side, 1 .. MVCT_MAX_N */
    double fov_cm;          /* field of view; pixel size delta = fov_cm / n */
    double sad_cm;          /* source-isocentre distance; must exceed fov_cm*sqrt(2)/2 */
    double sdd_cm;          /* source-detector distance (not used by an arc detector) */
    int32_t n_views;        /* V >= 1, uniform over 2 pi */
    int32_t n_channels;     /* C >= 1, equiangular */
    double view0_rad;       /* angle of view 0 */
    double fan_angle_rad;   /* <= 0 selects 2 asin((fov/2)/sad) */
    double channel_offset;  /* detector shift in channels */
} mvct_geometry;

typedef struct mvct_plan_s *mvct_plan;

/* Loop state carried between calls to resume a reconstruction (host memory).
 * A run of N sub-iterations resumed after K equals one run of K + N, bit for bit. */
typedef struct mvct_recon_state {
    int64_t n_done;       /* sub-iterations already run (0 for a fresh run) */
    double lambda;        /* lambda of the last sub-iteration */
    double phi_prev;      /* square difference of the last sub-iteration */
    double best_pass;     /* smallest pass sum so far (+inf if none) */
    int64_t best_n;       /* its sub-iteration (-1 if none) */
    double phi_ring[MVCT_MAX_SUBSETS]; /* last S square differences, slot n mod S */
    double pass_prev;     /* MVCT_LAMBDA_PASS: the last complete pass sum that was recorded */
} mvct_recon_state;

/* Options of mvct_recon. Fill with mvct_recon_opts_init() first. */
typedef struct mvct_recon_opts {
    double lambda0;       /* Eq. 4-5 initial convergence parameter (0.01) */
    double dlambda_up;    /* Eq. 4 increment when the square difference fell (1e-4) */
    double dlambda_down;  /* Eq. 5 decrement when it rose (2e-4) */
    double lambda_min;    /* floor of lambda (1e-4) */
    double kappa;         /* step tau = kappa * lambda on the preconditioned gradient (50: lambda0 = 0.01 is
                             half the separable-surrogate step) */
    double tv_eps;        /* TV smoothing inside the square root (1e-6) */
    double mu0;           /* homogeneous initial image in 1/cm, Sec. 3.3.2 (0.05) */
    int32_t init_from_input;       /* 1: start from d_img_inout instead of mu0 */
    float *d_best_out;             /* device n*n: image at the best pass sum, or NULL */
    const double *lambda_schedule; /* host, n_iter values replacing Eq. 4-5, or NULL */
    mvct_recon_state *state;       /* host in/out resume state, or NULL */
    double barrier_timeout_ms;     /* grid-barrier wait limit (2000) */
    int32_t debug_unreachable_barrier; /* test knob: the first barrier can never complete */
    int32_t data_term;             /* MVCT_DATA_WLS (0, default) or MVCT_DATA_POISSON (1) */
    int32_t storage;               /* MVCT_STORAGE_F32 (0, default), _BF16 (1) or _F16 (2); mvct_recon only */
    const int32_t *subset_order;   /* host, S entries: a permutation of 0..S-1 visited cyclically
                                      (sub-iteration n uses subset subset_order[n mod S]); NULL: the
                                      paper's equal-interval subsets in order 0, 1, ..., S-1 (Sec. 3.4).
                                      mvct_recon only; MVCT_EINVAL if not a permutation */
    int32_t lambda_rule;           /* which square differences Eq. 4-5 compare: MVCT_LAMBDA_* below
                                      (default MVCT_LAMBDA_PASS_SLIDING) */
    double *psi_record;            /* host, n_iter/S + 1 doubles, or NULL: the convergence record of
                                      Sec. 4.2 -- psi_record[k] = Psi (mvct_objective over all views) of
                                      the iterate after k*S sub-iterations of this call, k = 0 ..
                                      n_iter/S (k = 0: the start image). The loop then runs one pass
                                      per launch, resumed bit for bit. mvct_recon only */
} mvct_recon_opts;

/* Readings of Eq. 4-5 under ordered subsets. Sec. 3.3.2 raises lambda while the
 * squared difference between reprojection and measured projection falls and
 * lowers it when that difference grows; with subsets each sub-iteration n only
 * has the square difference Phi_n of its own subset's rays. The rules say which values
 * are compared (lambda unchanged on a tie and where no comparison is made):
 *   SUBSET        Phi_n with Phi_{n-1}, n >= 1 (consecutive sub-iterations, i.e.
 *                 different subsets);
 *   PASS          once per pass: at n = kS, k >= 2, the sum over the last complete
 *                 pass Phi_{n-S} + ... + Phi_{n-1} with the pass before it;
 *   PASS_SLIDING  every sub-iteration n >= S: the pass sum P_n = Phi_{n-S+1} + ... +
 *                 Phi_n with P_{n-1}, i.e. Phi_n with Phi_{n-S}, the same subset one
 *                 pass earlier (the whole-sinogram square difference, refreshed one
 *                 subset at a time). */
#define MVCT_LAMBDA_SUBSET 0
#define MVCT_LAMBDA_PASS 1
#define MVCT_LAMBDA_PASS_SLIDING 2

/* Storage precision of mvct_recon. F32: every buffer FP32. BF16 / F16: the copies
 * of the iterate that the reprojection reads (the image and its transpose) and
 * the measured p and w are stored in that 16-bit type (round to nearest) and
 * widened to FP32 on load; the iterate itself stays FP32 (the update of Eq. 3
 * is applied to the FP32 image, then rounded into the 16-bit copies). All
 * arithmetic is FP32 (projection, backprojection, TV, update); Phi and the
 * objective are summed in FP64. mvct_batch_* accept F32 only. */
#define MVCT_STORAGE_F32 0
#define MVCT_STORAGE_BF16 1
#define MVCT_STORAGE_F16 2

/* Data terms of mvct_recon (Sec. 2: Poisson photon statistics).
 * WLS:     1/2 sum w_i ([A mu]_i - p_i)^2, the quadratic (log-domain) approximation.
 * POISSON: sum w_i [A mu]_i + exp(-[A mu]_i), the negative Poisson log-likelihood
 *          with counts y_i = I0 w_i divided by I0 (p is not used by its gradient).
 * The adaptive lambda of Eq. 4-5 is driven by sum (A mu - p)^2 in both cases. */
#define MVCT_DATA_WLS 0
#define MVCT_DATA_POISSON 1

/* Results of mvct_recon (host memory; arrays caller-owned, may be NULL). */
typedef struct mvct_recon_stats {
    double *phi;          /* n_iter square differences Phi_n (unweighted, subset rays) */
    double *lambda;       /* n_iter convergence parameters lambda_n */
    int64_t best_n;       /* sub-iteration of the smallest pass sum (-1 if none) */
    double best_pass;     /* that pass sum */
    double loop_ms;       /* device time of the persistent loop kernel */
    double setup_ms;      /* device time of the set-up kernels */
    double forward_ms;    /* loop time in reprojection + residual (incl. its grid barrier) */
    double back_ms;       /* loop time in estimation + TV + update (incl. its grid barrier) */
    int32_t grid_blocks;  /* persistent grid size used */
    int32_t block_threads;
} mvct_recon_stats;

/* Default options (the paper's constants: lambda0 0.01, +1e-4, -2e-4; mu0 0.05; kappa 50 and
 * MVCT_LAMBDA_PASS_SLIDING, the readings under which the paper's convergence claims hold). */
void mvct_recon_opts_init(mvct_recon_opts *opts);

/* Build a plan for geometry *g with n_subsets ordered subsets (Sec. 3.4:
 * views thinned at a fixed spacing; n_views % n_subsets must be 0). Allocates
 * the ray and view tables and scratch on the CURRENT device and computes the
 * support mask (A^T 1 > 0) there; synchronous. *out receives the plan. */
int mvct_plan_create(const mvct_geometry *g, int32_t n_subsets, mvct_plan *out);

/* Free a plan and its device memory (NULL is ignored). Synchronises the device. */
void mvct_plan_destroy(mvct_plan plan);

/* Reprojection (Sec. 4.4): d_sino = A_s d_img, Joseph interpolation along each
 * fan-beam ray. d_img: n*n; d_sino: rows*C with rows = V (subset -1) or V/S. */
int mvct_forward(mvct_plan plan, const float *d_img, float *d_sino, int32_t subset, void *stream);

/* Estimation (Sec. 4.4): d_img = A_s^T d_sino, the matched adjoint of
 * mvct_forward (the projector's own Joseph weights, so <A x, y> = <x, A^T y>
 * up to FP32 rounding). Computed ray-driven, not pixel-driven: each 32x32 pixel
 * tile is owned by one block, whose warps walk the rays of the tile's channel
 * window through it and add their weighted values into warp-private
 * shared-memory copies of the tile, which are then summed in a fixed order (per
 * tile, view groups are merged in group order). No global atomics and no
 * floating-point race, so results are bit-identical from run to run.
 * Overwrites all n*n pixels. */
int mvct_back(mvct_plan plan, const float *d_sino, float *d_img, int32_t subset, void *stream);

/* Gradient of the smoothed TV regulariser (Sec. 2):
 * TV_eps = sum sqrt(dx^2 + dy^2 + eps), forward differences, zero across the
 * last row/column. d_grad: n*n; d_tv_or_null: one double (device) receiving
 * TV_eps, reduced in FP64 in a fixed order. */
int mvct_tv_grad(mvct_plan plan, const float *d_img, double eps, float *d_grad,
                 double *d_tv_or_null, void *stream);

/* Objective Psi = 1/2 sum_i w_i ([A img]_i - p_i)^2 + beta TV_eps(img) over all
 * views (Eq. 2 in its weighted-least-squares reading), FP64 reduction.
 * d_sino, d_weights: V*C; d_out: one double (device). */
int mvct_objective(mvct_plan plan, const float *d_img, const float *d_sino, const float *d_weights,
                   double beta, double eps, double *d_out, void *stream);

/* Gradient of the objective over all views (the direction Eq. 3 steps along,
 * in the weighted-least-squares reading of Eq. 2):
 *   d_grad = A^T (w .* (A img - p)) + beta grad TV_eps(img)        (FP32, n*n),
 * and, if d_out_or_null is given, Psi(img) as mvct_objective computes it (one
 * device double, FP64 reduction). Projection and backprojection are the plan's
 * matched pair (mvct_forward / mvct_back), the TV gradient that of mvct_tv_grad.
 * d_sino, d_weights: V*C; d_grad must not alias d_img. Uses the plan's scratch;
 * asynchronous on stream. */
int mvct_objective_grad(mvct_plan plan, const float *d_img, const float *d_sino, const float *d_weights,
                        double beta, double eps, float *d_grad, double *d_out_or_null, void *stream);

/* The ordered-subset TV reconstruction (Eq. 3-5, Sec. 3.3.2, 3.4, 4.2).
 * d_sino: measured log projections p [V][C]; d_weights: statistical weights w
 * [V][C] (>= 0); beta: TV weight; n_iter: sub-iterations (each uses one subset,
 * s = n mod S). d_img_inout: n*n, in = starting image if opts->init_from_input,
 * out = final iterate. Runs the set-up kernels and one persistent cooperative
 * kernel on `stream`, then synchronises it and fills *stats (may be NULL).
 * Returns MVCT_ETIMEOUT if a grid barrier exceeded opts->barrier_timeout_ms,
 * MVCT_EDATA on non-finite p/w or negative w, MVCT_ELAUNCH if the grid cannot
 * be co-resident. */
int mvct_recon(mvct_plan plan, const float *d_sino, const float *d_weights, double beta,
               int32_t n_iter, const mvct_recon_opts *opts, float *d_img_inout,
               mvct_recon_stats *stats, void *stream);

/* Filtered backprojection (the paper's comparison image, Sec. 1 and 4.5, and the
 * plain start image of the loop): equiangular fan-beam FBP with cosine
 * pre-weighting D cos(gamma), the fan-beam ramp filter
 * g(k a) = 1/2 (k a / sin(k a))^2 h(k a) (h the band-limited ramp, a the channel
 * pitch) and 1/L^2-weighted backprojection over the full rotation, dbeta = 2 pi/V.
 * d_sino: log projections [V][C] (all views); d_img: n*n output (1/cm).
 * Uses the plan's scratch; asynchronous on stream. */
int mvct_fbp(mvct_plan plan, const float *d_sino, float *d_img, void *stream);

/* ---- Batches: many slices (uneven geometries) in one persistent launch ----
 * The plans (one per slice, all on one device, each in at most one batch) are
 * reconstructed together: the co-resident grid is split into block groups, each
 * group runs the ordered-subset loop of mvct_recon on its own slices with
 * group-local barriers. With at most as many slices as co-resident blocks each
 * slice is a group of at least one block, and the remaining blocks are dealt one
 * at a time to the slice with the most work (views/S x channels x n) per block;
 * with more slices, single-block groups take the slices longest first. A plan in
 * a batch may not be passed to mvct_recon until the batch is destroyed. */
typedef struct mvct_batch_s *mvct_batch;

/* Create a batch over `count` distinct plans (host array). Synchronous. */
int mvct_batch_create(const mvct_plan *plans, int32_t count, mvct_batch *out);

/* Free a batch (synchronises the device); its plans become usable again. */
void mvct_batch_destroy(mvct_batch batch);

/* Bind the slices' data (host arrays of `count` entries, in plan order): device
 * pointers to p and w ([V][C] of each plan's geometry), TV weights beta, and the
 * images (n*n, in = start image if opts->init_from_input, out = final iterate),
 * plus the largest n_iter that mvct_batch_run will be given. opts as for
 * mvct_recon (NULL = defaults); lambda_schedule, state and d_best_out must be
 * NULL. Synchronous; pointers are kept until the next bind. */
int mvct_batch_bind(mvct_batch batch, const float *const *d_sinos, const float *const *d_weights,
                    const double *betas, float *const *d_imgs, int32_t max_iter,
                    const mvct_recon_opts *opts);

/* Enqueue the set-up of every slice, one persistent cooperative launch running
 * n_iter sub-iterations on every slice, and the copy of each final image into
 * its bound buffer. Asynchronous on `stream`: no host synchronisation, no host
 * memory access. */
int mvct_batch_run(mvct_batch batch, int32_t n_iter, void *stream);

/* Synchronise the device, then fill *stats (may be NULL) for one slice (plan
 * order) of the last run: Phi and lambda per sub-iteration, best pass, and the
 * device times of the whole batch (setup_ms, loop_ms; -1 after a CUDA-graph
 * replay of mvct_batch_run). stats->phi and stats->lambda, when not NULL, must
 * each hold the last run's n_iter doubles (caller-owned host memory). Returns
 * MVCT_ETIMEOUT / MVCT_EDATA if the run failed. */
int mvct_batch_stats(mvct_batch batch, int32_t slice, mvct_recon_stats *stats);

/* ---- Learned warm start (a start image for mvct_recon from the FBP image) ----
 * An 8-layer 3x3 convolutional network: 1 -> 32 channels, six 32 -> 32 layers,
 * 32 -> 1, ReLU after layers 1-7, zero padding, residual output:
 *   out = x + f(s x) / s   (s = the input scale given at creation),
 * BF16 weights and activations with FP32 accumulation; the 32 -> 32 layers run
 * on BF16 tensor cores in the forward and both backward convolutions. The
 * network is trained on (FBP image, converged OS-TV image) pairs that the
 * reconstruction itself produces; the paper (Sec. 3.3.2, 4.2) motivates it by
 * the effect of the start image on convergence, and has no network of its own.
 * Parameter vector (FP32, mvct_cnn_param_count() entries, host order):
 *   W1[9][32] b1[32] | 6 x (W[9][32 in][32 out] b[32]) | W8[9][32] b8[1],
 *   tap = 3*ky + kx, out[y][x] = sum x[y+ky-1][x+kx-1] W[tap] (cross-correlation). */
typedef struct mvct_cnn_s *mvct_cnn;

int32_t mvct_cnn_param_count(void);

/* Network for batches of up to batch_max images of h x w on the current device;
 * params: host array of initial parameters. Synchronous. */
int mvct_cnn_create(int32_t batch_max, int32_t h, int32_t w, double scale, const float *params,
                    mvct_cnn *out);
void mvct_cnn_destroy(mvct_cnn cnn);

/* Copy the FP32 master parameters to the host array params. Synchronous. */
int mvct_cnn_get_params(mvct_cnn cnn, float *params);

/* Inference: d_out[n][h][w] = network(d_in[n][h][w]) (FP32, device). */
int mvct_cnn_forward(mvct_cnn cnn, const float *d_in, int32_t n, float *d_out, void *stream);

/* Waits of the tensor-core convolutions: each wait on a pipeline barrier gives
 * up after timeout_ms of GPU time (default 1000; at most 60000), records the
 * failure and lets the launch finish. debug_stall = 1 is a test knob: the copy
 * warps issue nothing, so the first wait of every block runs out. Host-side
 * setting, applies to launches made after the call. */
int mvct_cnn_set_wait(mvct_cnn cnn, double timeout_ms, int32_t debug_stall);

/* Synchronise the stream and report whether a tensor-core convolution of the
 * network gave up waiting since the last status call or training step
 * (MVCT_ETIMEOUT: the outputs of those launches are invalid); clears the flag.
 * mvct_cnn_forward is asynchronous and graph-capturable and does not check. */
int mvct_cnn_status(mvct_cnn cnn, void *stream);

/* Mean squared error of the network on (d_in, d_target) in the scaled domain,
 * mean over all n*h*w pixels, written to *loss (host; the call synchronises
 * the stream), and its gradient with respect to the parameters into d_grad
 * (device, param_count floats) if not NULL. Deterministic. */
int mvct_cnn_grad(mvct_cnn cnn, const float *d_in, const float *d_target, int32_t n, float *d_grad,
                  double *loss, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the batch;
 * *loss receives the batch loss before the step. Synchronises the stream. */
int mvct_cnn_train_step(mvct_cnn cnn, const float *d_in, const float *d_target, int32_t n, double lr,
                        double *loss, void *stream);

/* Allocation-free variant of mvct_tv_grad for callers that may not allocate
 * device memory (applications that hand out all GPU memory through their own
 * allocator, or latency-critical paths where cudaMalloc/cudaFree, which can
 * synchronise the device, are not allowed). The paper has no counterpart; this
 * is a library-level service. Same operation and outputs as mvct_tv_grad, but
 * no plan: d_img and d_grad are caller-owned n*n float32 device arrays, n in
 * 1..MVCT_MAX_N; d_tv_or_null receives TV_eps (one device double) or is NULL.
 * Allocates nothing: the FP64 partial sums live in a 16 KiB static device array
 * of the library (MVCT_NOALLOC_MAX_BLOCKS slots) that every GPU loading the
 * library holds until process exit. The first call on a device, made with that
 * device current, looks up the array's address there; make that first call
 * before any stream capture. All calls share the array: calls that overlap on
 * the GPU (unordered streams) race and corrupt the TV value -- order them.
 * Returns MVCT_EINVAL for null pointers, n outside 1..MVCT_MAX_N or eps <= 0. */
int mvct_tv_grad_noalloc(const float *d_img, int32_t n, double eps, float *d_grad,
                         double *d_tv_or_null, void *stream);

/* ---- Autotuner (launch shapes of the loop) ---------------------------------
 * The loop's work split has two knobs that change speed, not the method: the
 * blocks of the one-slice launch (co-resident blocks per SM x SMs) and the
 * number of view groups each 32x32 tile's backprojection (Sec. 4.4
 * "estimation") is dealt to. The tuners time short runs of every candidate on
 * the caller's data (each candidate twice, the second run counts) and keep the
 * fastest; results of a tuned run equal an untuned run up to the summation
 * order of the groups' partial tiles. */
#define MVCT_TUNE_MAX 32
typedef struct mvct_tune_report {
    int32_t groups;              /* chosen view groups per tile (0 = the default rule: for one slice the
                                    balanced plan where the sizes allow it, see mvct_plan_set_shape) */
    int32_t grid_blocks;         /* chosen blocks of the loop launch */
    double ms_per_iter;          /* loop time per sub-iteration of the choice */
    double default_ms_per_iter;  /* the same for the untuned default */
    int32_t n_candidates;        /* entries below (the first is the default) */
    int32_t cand_groups[MVCT_TUNE_MAX];
    int32_t cand_grid[MVCT_TUNE_MAX];
    double cand_ms_per_iter[MVCT_TUNE_MAX];
} mvct_tune_report;

/* Tune the plan's one-slice loop on (d_sino, d_weights, beta) with n_iter_probe
 * sub-iterations per run (homogeneous start, default options) and keep the
 * fastest shape for later mvct_recon calls. Device memory of the caller is only
 * read; a scratch image is allocated for the duration. report may be NULL.
 * Synchronises the stream. Errors: as mvct_recon; MVCT_EINVAL for a plan that
 * belongs to a batch. */
int mvct_plan_tune(mvct_plan plan, const float *d_sino, const float *d_weights, double beta,
                   int32_t n_iter_probe, mvct_tune_report *report, void *stream);

/* Set the one-slice launch shape explicitly (e.g. a shape an earlier
 * mvct_plan_tune reported): groups = view groups per tile (0 = the default
 * rule, at most min(8, views per subset)), grid_blocks = blocks of the loop
 * launch (0 = every co-resident block). MVCT_EINVAL outside those ranges.
 * The default rule with every co-resident block uses the balanced plan where
 * the sizes allow it (r blocks per SM, 2 <= r: r - 1 items of half a tile's
 * views per SM and one item of a tile split into 2..8 groups, one block left
 * for the reduction of Phi; e.g. 512^2 with 40 views per subset on 152 SMs);
 * otherwise every tile is split into min(8, views per subset, blocks / tiles)
 * groups. A groups value > 0 always splits every tile into that many groups. */
int mvct_plan_set_shape(mvct_plan plan, int32_t groups, int32_t grid_blocks);

/* The balanced plan of phase B that a one-slice launch of the default shape
 * uses (see mvct_plan_set_shape), as plain host arithmetic: n_tiles 32x32
 * tiles, views_per_subset views per subset, groups_cap = min(8, views per
 * subset) partial-tile buffers per tile, grid blocks on num_sms SMs (block b
 * assumed on SM b mod num_sms). Group h of a tile split into H groups holds the
 * subset's views h, h + H, h + 2H, ... On success writes 4 * grid int32 to
 * items (per block: tile, view group, view groups of that tile, first
 * partial-tile slot of that tile; tile -1 for a block without an item) and the
 * item-less block that reduces Phi_n to *idle_block, and returns 1; returns 0,
 * writing nothing, when the sizes do not allow the plan (the launch then splits
 * every tile into the same number of groups); MVCT_EINVAL for a NULL pointer or
 * a size < 1. Makes no CUDA call. */
int mvct_phase_b_plan(int32_t n_tiles, int32_t views_per_subset, int32_t groups_cap, int32_t grid,
                      int32_t num_sms, int32_t *items, int32_t *idle_block);

/* Tune a bound batch: the view groups per tile of every slice (the default
 * rule, or 1, 2, 3, 4, 6, 8) with runs of min(n_iter_probe, max_iter)
 * sub-iterations on the bound data; the bound images are saved before and
 * restored after the runs, and the batch stays bound with the fastest choice.
 * Synchronises the stream. report may be NULL. */
int mvct_batch_tune(mvct_batch batch, int32_t n_iter_probe, mvct_tune_report *report, void *stream);

/* Message of the last failed call on this thread ("" if none). */
const char *mvct_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MVCT_H_ */
