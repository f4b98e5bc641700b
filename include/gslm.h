/*
 * gslm.h - C ABI of the GB300 (sm_103a) Levenberg-Marquardt / PCG hot path for
 * 3D Gaussian Splatting, after 3DGS-LM (arXiv 2409.12892).
 *
 * What the calls compute (paper sections in brackets):
 *   gslm_render        images of the splatted scene [Sec. 3.1, Eq. alpha-blending]
 *   gslm_build_cache   residual F = c - C, cost ||F||^2, the per-(pixel, splat)
 *                      gradient cache and b = -J^T F [Sec. 3.3 "buildCache",
 *                      "sortCacheByGaussians"; Algorithm 1, first two lines]
 *   gslm_apply_J       u = J p  [Sec. A, Eq. apply-j]
 *   gslm_apply_JT      g = J^T u  [Sec. A, Eq. apply-jt]
 *   gslm_jacobi_diag   M = diag(J^T J)  [Sec. A, Eq. diag-jtj]
 *   gslm_pcg_solve     Algorithm 1 on (J^T J + lambda M) x = b  [Sec. 3.3]
 *   gslm_pcg_solve_batch  the same for several image subsets in lock step
 *   gslm_combine_*     weighted mean of subset directions [Eq. combine-pcg]
 *   gslm_lm_step       one LM iteration over image subsets [Sec. 3.2,
 *                      Eq. norm-eq, Eq. tr-update, Eq. combine-pcg]
 *
 * Conventions
 *   - Every array pointer is a DEVICE pointer unless its comment says "host".
 *     Arrays passed in are owned by the caller; the library never frees them.
 *   - The library owns gslm_ctx and gslm_cache objects and the device memory
 *     behind them (allocated with cudaMallocAsync on the context's stream, from
 *     the device's default memory pool). gslm_create sets that pool to keep
 *     freed memory (release threshold: maximum), so caches rebuilt every LM
 *     step reuse it; gslm_destroy trims the pool back to the driver.
 *   - All work is enqueued on the context's CUDA stream. Outputs are valid
 *     once that stream has been synchronised. gslm_build_cache synchronises
 *     once (to size the cache); gslm_lm_step synchronises to fill its stats;
 *     gslm_pcg_solve synchronises when stats is non-NULL and, for more than 16
 *     iterations, every 16 iterations: it reads the break-test flag back and
 *     launches no further iterations once the solve has ended.
 *   - Errors are returned as gslm_status codes; nothing throws across the
 *     ABI; gslm_last_error() gives a message for the last failure on a
 *     context. The library never traps on the device.
 *
 * Layouts
 *   - Gaussian parameters and every parameter-space vector (b, p, g, x, M,
 *     preconditioner, Delta): structure of arrays, float32 [59][ld], element
 *     (k, i) at offset k*ld + i for parameter k of Gaussian i; ld >= N and a
 *     multiple of 4; gslm_pcg_solve's vectors start on a 16-byte boundary
 *     (every cudaMalloc'd or torch-allocated buffer does). Parameter order per Gaussian: position (3), log-scale (3),
 *     quaternion w,x,y,z (4, not normalised), opacity logit (1), SH (48, index
 *     3*coeff + channel, coeff l-major, degree <= 3). This is the paper's
 *     per-attribute layout q (Sec. A, "Design of applyJ and diagJTJ").
 *   - Residual-space vectors (targets, F, u, images): float32, the views of a
 *     call concatenated in order, each view row-major [H][W][3].
 */
#ifndef GSLM_H
#define GSLM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GSLM_OK = 0,
  GSLM_E_INVALID = -1,        /* bad argument (null pointer, size, layout) */
  GSLM_E_OOM = -2,            /* device allocation failed or budget exceeded */
  GSLM_E_CUDA = -3,           /* a CUDA runtime call failed */
  GSLM_E_CACHE_OVERFLOW = -4, /* the cache would exceed options.mem_budget */
  GSLM_E_TIMEOUT = -5,        /* a bounded device wait ran out */
  GSLM_E_NUMERIC = -6,        /* non-finite value where one is not allowed */
  GSLM_W_PCG_BREAKDOWN = 1    /* PCG stopped early: p^T g <= 0 or not finite */
} gslm_status;

/* Cache formats. FP32, BF16 and FP16S store one entry per contributing
 * (pixel, splat) pair: its weight alpha T and alpha dc/dalpha, in float32, in
 * bfloat16, or in float16 scaled per (tile, splat) segment.
 * GSLM_CACHE_THIN stores no entries: the cache keeps, per (tile, splat)
 * segment, the projected splat; per pixel, its final colour and how many of its
 * tile's segments reach it before blending stops; and a checkpoint of the
 * pixel's transmittance and colour prefix before every 32nd segment of its tile
 * (the memory-saving thinning the paper's limitations section proposes). J p,
 * J^T u and diag(J^T J) then blend each pixel's splats again, J^T u and the
 * diagonal window by window from those checkpoints. It takes several times
 * less memory and more time per product; gslm_pcg_solve_batch and the batched
 * gslm_lm_step solve thin caches one subset after another. */
typedef enum { GSLM_CACHE_FP32 = 0, GSLM_CACHE_BF16 = 1, GSLM_CACHE_FP16S = 2, GSLM_CACHE_THIN = 3 } gslm_cache_fmt;

/* The energy the LM step minimises.
 * GSLM_OBJ_L2: residual c - C per pixel channel, E = ||c - C||^2.
 * GSLM_OBJ_L1_SSIM: Eq. gn-loss, two residuals per pixel channel,
 *   r1 = sqrt(l1 |c - C|), r2 = sqrt(l2 (1 - SSIM)), E = sum of l1 |c - C| + l2 (1 - SSIM);
 *   SSIM per channel with an 11 x 11 Gaussian window (sd 1.5, zero outside the
 *   view), C1 = 0.01^2, C2 = 0.03^2; dSSIM/dc keeps only the centre pixel's own
 *   term (Sec. C). Their Jacobian enters through the per pixel channel weights
 *   w = (dr1/dc)^2 + (dr2/dc)^2 and e = (dr1/dc) r1 + (dr2/dc) r2 (Sec. C,
 *   "Precomputation Of Residual-To-Pixel Weights"): J^T J p = (dc/dx)^T (w (dc/dx) p),
 *   J^T F = (dc/dx)^T e, diag(J^T J) = sum w (dc/dx)^2. Under the square roots of
 *   the derivatives |c - C| and 1 - SSIM are floored at options.res_eps. */
typedef enum { GSLM_OBJ_L2 = 0, GSLM_OBJ_L1_SSIM = 1 } gslm_objective;

/* A posed pinhole camera. World point X maps to camera point R X + t (OpenCV
 * axes: x right, y down, z forward) and to pixel (fx x/z + cx, fy y/z + cy).
 * Pixel (px, py) has its centre at (px + 0.5, py + 0.5). */
typedef struct {
  float R[9];          /* row-major world -> camera rotation */
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
} gslm_camera;

typedef struct {
  int32_t cache_fmt;   /* gslm_cache_fmt */
  int32_t n_iters;     /* PCG loop iterations after the initial product (paper: 8) */
  float break_rel2;    /* stop when ||r||^2 < break_rel2 ||b||^2 (paper: 0.01); 0 = never */
  float lambda_min;    /* LM damping clamp (paper: 1e-4 .. 1e4) */
  float lambda_max;
  int32_t smooth;      /* test mode: no alpha clamp/skip, no T stop, no SH clamp, no tile culling */
  size_t mem_budget;   /* bytes a cache may take; 0 = no limit */
  int32_t group;       /* reserved: lanes per cache segment in the apply kernels (0 or 32) */
  int32_t profile;     /* 1: gslm_lm_step records CUDA events per phase (ms_phase in its stats) */
  int32_t autotune;    /* 1 (default): on first use per cache format, time every apply kernel
                          variant once on the real cache and keep the fastest; 0: fixed variant */
  int32_t batch;       /* 1 (default): gslm_lm_step solves all subsets in lock step, one launch per
                          phase over every subset (gslm_pcg_solve_batch); 0: one subset after another */
  int32_t graph;       /* 1 (default): a batched solve is captured into one CUDA graph and launched
                          once (after the first batched solve of a context, which also autotunes) */
  int32_t batch_ctas;  /* resident CTAs per SM of the persistent batched tile kernels; 0 = autotune */
  int32_t apply_variant; /* 0: autotuned (or default) apply kernel variant; 1..10: always variant 0..9 */
  int32_t line_search; /* gslm_lm_step: 0 = full step (gamma = 1); n > 0 = Eq. line-search over
                          gamma = 1, 1/2, ..., 2^(1-n) on the first 30% of the step's views,
                          stopping at the first cost increase (default 8) */
  int32_t pad;
  size_t batch_mem;    /* gslm_lm_step with batch: bytes the stacked PCG vectors of a group of
                          subsets may take (0 = as much as the device gives); a group above it,
                          or whose vectors cannot be allocated, is solved subset by subset */
  int32_t objective;   /* gslm_objective (default GSLM_OBJ_L2) */
  float lambda_l1;     /* GSLM_OBJ_L1_SSIM weights (paper: 0.8 and 0.2) */
  float lambda_ssim;
  float res_eps;       /* floor under the square roots of the residual derivatives (1e-4) */
} gslm_options;

typedef struct gslm_ctx gslm_ctx;
typedef struct gslm_cache gslm_cache;

typedef struct {
  int64_t entries;       /* (pixel, splat) cache entries */
  int64_t segments;      /* non-empty (tile, splat) segments */
  int64_t splats;        /* visible (view, Gaussian) splats */
  int64_t active_splats; /* splats with at least one entry */
  int64_t keys;          /* tile keys sorted while building */
  int64_t bytes;         /* device bytes held by the cache */
  int64_t pixels;        /* residual pixels covered (sum of W*H over the views) */
  int32_t views;
  int32_t cache_fmt;
} gslm_cache_info;

typedef struct {
  int32_t iters;         /* loop iterations run */
  int32_t breakdown;     /* 1 if p^T g <= 0 or non-finite stopped the loop */
  double rr;             /* ||r||^2 of the recursive residual at exit */
  double bb;             /* ||b||^2 */
} gslm_pcg_stats;

typedef struct {
  float lambda;          /* in: damping for this step; out: updated damping */
  int32_t step;          /* in/out: LM step counter (incremented) */
} gslm_lm_state;

typedef struct {
  double cost;           /* ||F(x)||^2 over all subsets' views */
  double cost_new;       /* ||F(x + Delta)||^2 */
  double predicted;      /* sum_i ||J_i Delta + F_i||^2 */
  double rho;            /* Eq. tr-update */
  int32_t accepted;
  int32_t pcg_iters;     /* summed over subsets */
  int64_t cache_entries; /* summed over subsets */
  int64_t cache_bytes;
  double ms_total;       /* device time of the step (CUDA events) */
  /* With options.profile: device ms per phase, summed over the step:
   * [0] cache build, [1] Jacobi diagonal, [2] tangent (dy/dx) p, [3] apply_J tile
   * kernel, [4] apply_JT tile kernel, [5] adjoint (dy/dx)^T ybar, [6] PCG vector
   * kernels, [7] rho evaluation (J Delta and the trial render). */
  double ms_phase[8];
  int32_t n_pairs;       /* J p + J^T u pairs executed (initial product + PCG iterations) */
  int32_t trial_overflows; /* trial renders (line search and rho) whose splats needed more than
                              2^32 tile keys; each counted one as cost +inf */
  /* Algorithmic bytes of those pairs: per pair on a cache with E entries of B_e
   * payload bytes, P pixels, N Gaussians and S active splats:
   * 2 E (B_e + 1) + 24 P + 472 N + 192 S. */
  double pair_bytes;
  int64_t cache_segments; /* non-empty (tile, splat) segments, summed over subsets */
  int64_t active_splats;  /* splats with at least one cache entry, summed over subsets */
  double gamma;           /* step scale the line search chose (1 without line search) */
  int32_t ls_evals;       /* line-search cost evaluations */
  int32_t seq_groups;     /* groups of subsets solved one after another because their stacked
                             PCG vectors did not fit in device memory beside the caches (batch mode) */
} gslm_lm_stats;

/* Default options: FP32 cache, 8 iterations, break 0.01, lambda in [1e-4, 1e4]. */
void gslm_default_options(gslm_options* opt);

/* Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
gslm_status gslm_create(const gslm_options* opt, void* cuda_stream, gslm_ctx** out);
void gslm_destroy(gslm_ctx* ctx);
const char* gslm_last_error(const gslm_ctx* ctx);
/* Replace the context's options (e.g. to switch cache format). */
gslm_status gslm_set_options(gslm_ctx* ctx, const gslm_options* opt);

/* Render the V views [Sec. 3.1, Eq. alpha-blending].
 * params: [59][ld]; cams: host array of V cameras; img: [sum W*H][3].
 * If targets is non-NULL, also writes cost[0] = E of options.objective:
 * ||img - targets||^2 or Eq. gn-loss (cost: host double*, may be NULL). */
gslm_status gslm_render(gslm_ctx* ctx, const float* params, int64_t N, int64_t ld,
                        const gslm_camera* cams, int32_t V, float* img,
                        const float* targets, double* cost);

/* Build the gradient cache of one image subset [Sec. 3.3; the inputs F and b of Algorithm 1].
 * Writes F = img - targets into F (may be NULL), b = -J^T F into b ([59][ld], may be
 * NULL) and cost ||F||^2 into *cost (host, may be NULL); with GSLM_OBJ_L1_SSIM,
 * F is e (see gslm_objective) and cost is Eq. gn-loss. The cache holds its
 * own device copy of params, so the caller may change or free params afterwards.
 * Returns GSLM_E_CACHE_OVERFLOW (and no cache) if options.mem_budget is exceeded. */
gslm_status gslm_build_cache(gslm_ctx* ctx, const float* params, int64_t N, int64_t ld,
                             const gslm_camera* cams, int32_t V, const float* targets,
                             gslm_cache** cache, float* F, float* b, double* cost);
gslm_status gslm_cache_stats(const gslm_cache* cache, gslm_cache_info* info);
/* The cache's residual-to-pixel weights w = (dr/dc)^2 summed over the pixel
 * channel's residuals, [pixels][3] into w (device): 1 everywhere for
 * GSLM_OBJ_L2. With GSLM_OBJ_L1_SSIM the cache's F (gslm_build_cache's F
 * output) is e = sum (dr/dc) r, and cost is Eq. gn-loss. */
gslm_status gslm_cache_weights(const gslm_cache* cache, float* w);
void gslm_cache_free(gslm_cache* cache);

/* u = J p [Eq. apply-j]. p: [59][ld]; u: [pixels][3]. With GSLM_OBJ_L1_SSIM
 * the cache's weights are applied: u = w . ((dc/dx) p), the vector
 * (u-hat . grad r) of Eq. apply-jtj-simplified-vec-vec that gslm_apply_JT
 * takes, so that gslm_apply_JT(gslm_apply_J(p)) = J^T J p. */
gslm_status gslm_apply_J(gslm_ctx* ctx, const gslm_cache* cache, const float* p, float* u);
/* g = J^T u [Eq. apply-jt]. u: [pixels][3]; g: [59][ld]. */
gslm_status gslm_apply_JT(gslm_ctx* ctx, const gslm_cache* cache, const float* u, float* g);
/* g = J^T u like gslm_apply_JT, for callers that must not allocate device
 * memory once running (a service whose memory another allocator reserved up
 * front, or a thread that may not call cudaMalloc). The paper has no
 * counterpart. The per-segment partial sums live in one fixed 24 MiB
 * __device__ array inside the library instead of a context buffer; the call
 * allocates nothing. gslm_create looks up the array's address on the
 * context's device, which places the array there: every device on which a
 * context was created holds it until the process exits.
 * Limits and rules: caches with more than 2^19 (tile, splat) segments
 * (gslm_cache_info.segments) are rejected with GSLM_E_INVALID, and so is a call
 * made while another device than the context's is current. It runs the same
 * apply_JT kernel variant as gslm_apply_JT on that context. With CUDA's lazy
 * module loading the first launch of a kernel in a process loads its code,
 * which takes device memory: make one call (or one gslm_apply_JT call) during
 * set-up, or set CUDA_MODULE_LOADING=EAGER. All calls share the array: calls
 * whose work overlaps on the GPU (other streams, other contexts) race; calls
 * on one stream are ordered and need no clearing in between. */
gslm_status gslm_apply_JT_noalloc(gslm_ctx* ctx, const gslm_cache* cache, const float* u, float* g);

/* M = diag(J^T J) [Eq. diag-jtj]. diag: [59][ld]. */
gslm_status gslm_jacobi_diag(gslm_ctx* ctx, const gslm_cache* cache, float* diag);

/* Algorithm 1 [Sec. 3.3]: x ~ (J^T J + lambda M)^-1 b with M = diag(J^T J) as
 * given, clamped to [1e-6, 1e32] (the LM diagonal bounds of Ceres, whose LM the
 * paper follows) both in the damping term and in the Jacobi preconditioner
 * M^-1 = 1/M; if precond is non-NULL, the given positive diagonal D ([59][ld])
 * replaces M^-1. x: [59][ld] output.
 * stats: host pointer or NULL (NULL: no synchronisation). Returns
 * GSLM_W_PCG_BREAKDOWN if the loop stopped on p^T g <= 0. */
gslm_status gslm_pcg_solve(gslm_ctx* ctx, const gslm_cache* cache, const float* b,
                           const float* diag, const float* precond, float lambda,
                           float* x, gslm_pcg_stats* stats);

/* Algorithm 1 for the systems of n_b image subsets of the same Gaussians at
 * once [Sec. 3.2-3.3]: the solves advance in lock step and each phase (tangent,
 * J p, J^T u, adjoint, vector update, scalars) is one launch over every
 * subset; the tile kernels are persistent and take the tiles of all subsets
 * from one queue, so subsets of uneven size share the GPU. Each subset's
 * arithmetic is that of gslm_pcg_solve, with its own break test. With
 * options.graph the solve is replayed from one captured CUDA graph.
 * caches, b, diag, precond (may be NULL, or hold NULL entries: Jacobi), x:
 * host arrays of n_b entries (device vectors [59][ld] as in gslm_pcg_solve).
 * All caches must share N, ld, cache format and mode. stats: host array of n_b
 * or NULL. Synchronises. Returns GSLM_W_PCG_BREAKDOWN if any subset broke down. */
gslm_status gslm_pcg_solve_batch(gslm_ctx* ctx, const gslm_cache* const* caches, int32_t n_b,
                                 const float* const* b, const float* const* diag,
                                 const float* const* precond, float lambda, float* const* x,
                                 gslm_pcg_stats* stats);

/* Eq. combine-pcg, accumulated subset by subset:
 * gslm_combine_accumulate: num += M_i * Delta_i, den += M_i;
 * gslm_combine_finish:     Delta = num / den (0 where den == 0). All [59][ld]. */
gslm_status gslm_combine_accumulate(gslm_ctx* ctx, int64_t N, int64_t ld, const float* delta_i,
                                    const float* diag_i, float* num, float* den);
gslm_status gslm_combine_finish(gslm_ctx* ctx, int64_t N, int64_t ld, const float* num,
                                const float* den, float* delta);

/* One LM step [Sec. 3.2]: for each of the n_b subsets build the cache, the
 * Jacobi diagonal and the PCG direction; combine [Eq. combine-pcg]; evaluate
 * rho [Eq. tr-update] with gamma = 1; on acceptance (rho > 1e-5) params +=
 * gamma Delta in place (gamma from the line search of Eq. line-search when
 * options.line_search > 0, else 1), else params are unchanged; lambda is
 * updated and clamped.
 * cams: host array of all cameras; targets: [sum over all cams W*H][3] in camera
 * order; subset_views: host, concatenated camera indices of the subsets;
 * subset_off: host, n_b + 1 offsets into subset_views. precond: optional
 * per-subset preconditioners (host array of n_b device pointers, or NULL).
 * Memory: every subset's cache stays resident until the step ends (they read
 * params in place, so params must not change during the call). With
 * options.batch the subsets' solves run in groups of up to 16 that keep six
 * stacked [59][ld] vectors per subset (seven with a preconditioner); a group
 * whose vectors do not fit beside its caches is solved one subset after
 * another instead (reported in stats->seq_groups), with the same arithmetic. */
gslm_status gslm_lm_step(gslm_ctx* ctx, float* params, int64_t N, int64_t ld,
                         const gslm_camera* cams, int32_t n_cams, const float* targets,
                         const int32_t* subset_views, const int32_t* subset_off, int32_t n_b,
                         const float* const* precond, gslm_lm_state* state, gslm_lm_stats* stats);

/* ---------------------------------------------------------------------------
 * Learned diagonal preconditioner. The paper has no counterpart: it uses the
 * Jacobi preconditioner M^-1 of Algorithm 1. This is a per-Gaussian network
 * whose output scales that preconditioner entry by entry:
 *   phi (64 features per Gaussian): log(M_k + 1e-12) for the 59 entries of the
 *     subset's diag(J^T J), the 3 log-scales, sigmoid(opacity logit) and
 *     log(1 + cache entries of the Gaussian), standardised with a stored
 *     per-feature mean and standard deviation;
 *   h1 = GELU(W1 phi + b1), h2 = GELU(W2 h1 + b2), o = W3 h2 + b3
 *     (64 -> 64 -> 64 -> 59, GELU(x) = x Phi(x));
 *   D_k = softplus(o_k) / clamp(M_k), used as D in gslm_pcg_solve.
 * The network computes with its weight matrices W1, W2, W3 rounded to
 * bfloat16 (round to nearest even) and float32 biases, activations and sums;
 * the weights held, set, got and updated by Adam are float32, and the weight
 * gradient is that of the rounded matrices.
 * Training minimises L = 1/2 log(||r_K||^2 / ||b||^2), the relative residual
 * after K iterations of Algorithm 1 run with D (x0 = D b, z = D r), by reverse
 * mode through those iterations and then through the network, with Adam.
 * Weights: float32 vector of gslm_precond_weight_count() values in the order
 * W1 (64 x 64, row = output), b1, W2 (64 x 64), b2, W3 (59 x 64), b3.
 * Feature arrays phi: device, float32 [N][64] row-major. */
typedef struct gslm_precond gslm_precond;

/* 12,155: the number of network weights. */
int32_t gslm_precond_weight_count(void);

/* Creates a network on ctx's device and stream. weights (host, or NULL):
 * initial weights; NULL starts at the Jacobi preconditioner (W3 = 0,
 * b3 = log(e - 1), so D = 1/clamp(M)) with W1, W2 ~ N(0, 0.25/64) drawn from
 * SplitMix64(seed) by Box-Muller. mean, std (host [64], or NULL for 0 and 1):
 * the standardisation. Adam state starts at zero. */
gslm_status gslm_precond_create(gslm_ctx* ctx, const float* weights, const float* mean, const float* std,
                                uint64_t seed, gslm_precond** out);
void gslm_precond_free(gslm_precond* pc);
/* Host copies of the weights / standardisation (any pointer may be NULL). Synchronises. */
gslm_status gslm_precond_get(const gslm_precond* pc, float* weights, float* mean, float* std);
/* Replaces the weights and/or the standardisation from host arrays (NULL = keep). */
gslm_status gslm_precond_set(gslm_precond* pc, const float* weights, const float* mean, const float* std);

/* Features phi [N][64] of a cache's system; diag = its diag(J^T J) [59][ld]. */
gslm_status gslm_precond_features(gslm_ctx* ctx, const gslm_cache* cache, const float* diag, float* phi);
/* Sets the standardisation to the per-feature mean and standard deviation
 * (floored at 1e-6) of phi [N][64]. Synchronises. */
gslm_status gslm_precond_fit_standardizer(gslm_precond* pc, const float* phi, int64_t N);
/* D [59][ld] = softplus(o) / clamp(diag) for features phi [N][64]. */
gslm_status gslm_precond_apply(gslm_precond* pc, const float* phi, int64_t N, int64_t ld, const float* diag,
                               float* D);
/* Weight gradient for an upstream gradient dD = dL/dD [59][ld]; added to
 * grad (device, [weight_count]) when accumulate != 0, written otherwise. */
gslm_status gslm_precond_backward(gslm_precond* pc, const float* phi, int64_t N, int64_t ld, const float* diag,
                                  const float* dD, float* grad, int32_t accumulate);
/* The unrolled loss for a given diagonal D on the cache's system
 * A = J^T J + lambda clamp(diag) with right-hand side b: *loss (host) = L and
 * dD (may be NULL) = dL/dD [59][ld]. K >= 1 iterations. Synchronises. Uses
 * about (3K + 8) vectors of [59][ld] floats of device memory. */
gslm_status gslm_precond_unrolled_grad(gslm_ctx* ctx, const gslm_cache* cache, const float* b, const float* diag,
                                       float lambda, const float* D, int32_t K, double* loss, float* dD);
/* One training contribution: D from the network, the unrolled loss and its
 * weight gradient, added (scaled by weight) to the network's own gradient
 * accumulator. *loss (host, may be NULL) = L. Synchronises. */
gslm_status gslm_precond_accumulate(gslm_precond* pc, const gslm_cache* cache, const float* phi, const float* b,
                                    const float* diag, float lambda, int32_t K, float weight, double* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the accumulated
 * gradient, which is then cleared. */
gslm_status gslm_precond_adam(gslm_precond* pc, float lr);
/* Makes gslm_lm_step use the network for every subset that gets no explicit
 * preconditioner (NULL restores Jacobi). The network must outlive its use. */
gslm_status gslm_set_precond(gslm_ctx* ctx, gslm_precond* pc);

/* Library version string. */
const char* gslm_version(void);
/* Number of CUDA kernels this library has launched in this process. */
int64_t gslm_kernel_launches(void);
/* Device memory of the pool the library allocates from (the context device's
 * default pool, see Conventions), host out[3]: out[0] bytes in use, out[1]
 * bytes the pool holds (in use + kept for reuse), out[2] the most bytes in use
 * since the last reset. reset_peak != 0 then resets out[2]'s mark to the
 * bytes in use. Reads only; nothing is enqueued. */
gslm_status gslm_memory_usage(const gslm_ctx* ctx, int32_t reset_peak, int64_t out[3]);
/* Kernel variants the autotuner chose on this context: out[0..2] apply_J and
 * out[3..5] apply_JT for the FP32, BF16 and FP16S caches (-1 = not tuned yet);
 * ms[0..5] (may be NULL) the time of the chosen variant when it was tuned. */
gslm_status gslm_autotune_info(const gslm_ctx* ctx, int32_t out[6], float ms[6]);

#ifdef __cplusplus
}
#endif
#endif /* GSLM_H */
