/*
 * gsopt.h — C ABI of libgsopt.so, the GB300 (sm_103a) AdamW-GS optimizer step
 * of "A Step to Decouple Optimization in 3DGS" (arXiv 2601.16736).
 *
 * The library updates the attributes of N Gaussian primitives in place with
 * the paper's recomposed optimizer: Sparse Adam over the primitives visible
 * from the current view (Sec. 3.1, Eq. meth::sparse_beta), Decoupled
 * Attribute Regularization on opacity and scale (Sec. 3.3,
 * Eq. disentangled_adam; App. Eqs. disentangled_opacity / _scaling),
 * Re-State Regularization of StSS-sampled primitives (Sec. 3.2,
 * Eq. meth::restate), and it keeps its per-primitive optimizer state
 * consistent when the primitive set changes (Sec. 2: densification, pruning,
 * MCMC relocation; App. "Scaling in RSR" item 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns a gs_status.  Arguments are validated on the host
 *   before anything is launched; an invalid argument returns
 *   GS_ERR_INVALID_ARG and launches nothing.  Device pointers are checked to
 *   be device allocations that hold the stated number of bytes (driver
 *   address-range query, cached per pointer).
 * - "device" pointers are CUDA global memory on the context's device,
 *   owned by the caller unless stated otherwise; "host" pointers are host
 *   memory (pinned memory gives asynchronous copies).
 * - Work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default
 *   stream) and is asynchronous unless stated otherwise.  A CUDA error during
 *   a call returns GS_ERR_CUDA and latches the context: later calls return
 *   GS_ERR_STATE until it is destroyed.
 * - A context is not thread-safe; calls on one context must be ordered on
 *   one stream (or externally synchronised).
 * - Primitive attributes use a structure-of-arrays layout, one float32
 *   array per group, row-major within the group:
 *       xyz [N][3]  position mu
 *       scale [N][3]  log-scale kappa (s = exp(kappa))
 *       rot [N][4]  quaternion
 *       opacity [N][1]  opacity logit tau (o = sigmoid(tau))
 *       sh [N][48]  16 SH coefficients x RGB; columns 0-2 are the DC term
 *   59 values per primitive.  rot and sh must be 16-byte aligned, the others
 *   4-byte aligned.  The canonical 59-column row used by the state
 *   export/import concatenates the groups in that order.
 * - N (the row count) must be below 2^31 - 1.
 */
#ifndef GSOPT_H
#define GSOPT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_ABI_VERSION 2
#define GS_NUM_COLS 59

typedef enum gs_status {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or value; nothing launched */
    GS_ERR_CUDA = 2,        /* a CUDA runtime/driver call failed; context latched   */
    GS_ERR_OOM = 3,         /* device allocation failed                               */
    GS_ERR_UNSUPPORTED = 4, /* valid request the library does not implement          */
    GS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up                     */
    GS_ERR_STATE = 6        /* context latched by an earlier error                    */
} gs_status;

/* Storage of the Adam moments m, v.  Arithmetic is FP32 in every case; only
 * the stored copy of each updated moment is rounded.  With beta2 = 0.999 the
 * second moment moves ~0.1 % per step, below BF16's resolution, so BF16
 * second moments drift (round-to-nearest) or carry noise (stochastic
 * rounding); how much that moves the attributes depends on each column's
 * learning rate relative to its magnitude.  Measured group errors after 1000
 * steps of the 3 M-primitive workload against the FP64 reference are
 * reported by the tests and the bench (GS_MOM_BF16: about 1e-2 on opacity;
 * GS_MOM_BF16_HYBRID: 3e-4; GS_MOM_FP16_BLOCK: 6e-4). */
typedef enum gs_moment_prec {
    GS_MOM_FP32 = 0,
    GS_MOM_BF16 = 1,        /* all 59 columns BF16: m round-to-nearest-even, v
                               stochastically rounded from a counter hash of (seed,
                               iteration, row, slot)                              */
    GS_MOM_FP8E4M3 = 2,     /* all 59 columns e4m3 (64 B per moment and row, t in
                               the m row) with one FP32 scale per column and block
                               of 256 rows, a power of two that keeps the block's
                               magnitudes within e4m3's 448.  On most steps a scale
                               only grows, when the changed rows' values need it (to
                               8 x the smallest fitting power of two once it is
                               set); on one step in 128 per block (iteration + block
                               a multiple of 128) it is recomputed from all 256 rows
                               and shrinks, to 8 x the smallest fitting, when that
                               is more than 3 binades below (import sets the
                               smallest that fits).  A scale change
                               re-encodes that column in the block's other rows.
                               m rounded to nearest, v stochastically (+-1/2
                               e4m3 ulp dither, then nearest); a positive v is never
                               stored as zero.  3 mantissa bits: far outside a 1e-3
                               error budget (measured by the tests and the bench).
                               Not with the optional terms (noise, AIU, active
                               count) or in a batch: GS_ERR_UNSUPPORTED.  */
    GS_MOM_BF16_HYBRID = 3, /* the 45 SH-rest columns BF16 (m round-to-nearest, v
                               stochastically rounded from a counter hash of (seed,
                               iteration, row, slot)); the other 14 columns FP32  */
    GS_MOM_FP16_BLOCK = 4   /* all 59 columns FP16 with one shared exponent per
                               group of columns a work item updates (8 SH columns;
                               rotation; xyz + scale + opacity): the group's largest
                               magnitude is scaled into FP16's top binade, so every
                               value within 2^29 of it keeps FP16's 10-bit mantissa.
                               m rounded to nearest, v stochastically (dithered by
                               +-1/2 FP16 ulp from a counter hash per group, then
                               rounded to nearest; values further than 2^29 below
                               their group's largest round to nearest).  128 B per
                               moment and row, as BF16.
                               The step count t saturates at 65535 (the
                               bias-correction factors are exactly 1 from step
                               15936 on).                                         */
} gs_moment_prec;

/* Regulariser form.  GS_REG_DAR is the paper's AdamW-GS (Eq. disentangled_adam);
 * the others are the ablations of App. "AdamW Style Decoupling" and
 * Sec. 3.2 (Eqs. disentangled_adam2, disentangled_adamwithcliping,
 * meth::undisentangled_mom). */
typedef enum gs_reg_mode {
    GS_REG_DAR = 0,
    GS_REG_COUPLED = 1,
    GS_REG_ADAMW = 2,
    GS_REG_ADAMW_CLIP = 3
} gs_reg_mode;

/* Which primitives take the position noise of App. Eq. disentangled_mu.  The
 * equation writes it as a term of the visible primitives' update
 * (GS_NOISE_VISIBLE); the 3DGS-MCMC regulariser it is taken from moves every
 * primitive (GS_NOISE_ALL). */
typedef enum gs_noise_mode {
    GS_NOISE_OFF = 0,
    GS_NOISE_VISIBLE = 1,
    GS_NOISE_ALL = 2
} gs_noise_mode;

typedef struct gs_attrs {        /* device, caller-owned, updated in place */
    float *xyz, *scale, *rot, *opacity, *sh;
} gs_attrs;

typedef struct gs_grads {        /* device (host for gs_step_host), read-only */
    const float *xyz, *scale, *rot, *opacity, *sh;
} gs_grads;

/* Static configuration (paper defaults in brackets, App. "Hyperparameter
 * Selection"). */
typedef struct gs_opt_config {
    double beta1, beta2;     /* Adam decay rates [0.9, 0.999]; 0 <= beta < 1          */
    float eps;               /* added outside the square root, Eq. meth::adam_update   */
    float lambda_o;          /* DAR weight on opacity [1e-3]                            */
    float lambda_s;          /* DAR weight on scale [1e-5]                              */
    float clip_o, clip_s;    /* C_t [10, 10]                                            */
    float alpha1, alpha2;    /* RSR factors [0.2, 0.04]; 0 <= alpha < 1                 */
    int32_t prec;            /* gs_moment_prec                                          */
    int32_t bias_mode;       /* 0: per-primitive step count t (Sec. 3.2), 1: global k  */
    int32_t reg_mode;        /* gs_reg_mode                                             */
    int32_t reserved;        /* must be 0                                               */
    int64_t n_pixels;        /* training-image pixel count; the DAR normaliser N_I is
                                derived from it by the paper's rule (keep the leading
                                decimal digit, divide by ten: 800x800 -> 60000)          */
} gs_opt_config;

/* Pinhole camera of the current view: p = R mu + t (R row-major,
 * world -> camera, camera looking down +z).  A mean is visible iff
 * z_near <= p.z <= z_far, |p.x| <= p.z tan_half_fovx, |p.y| <= p.z tan_half_fovy
 * (Eq. meth::sparse_beta's V, read as the frustum test of the mean), decided
 * exactly for the given FP32 values: the test is evaluated in FP32 and taken
 * again in FP64 for every mean within twice the FP32 evaluation's rounding
 * bound of a plane, so the decision can differ from exact arithmetic only
 * within ~1e-14 (relative to the coordinates) of a plane. */
typedef struct gs_camera {
    float R[9];
    float t[3];
    float tan_half_fovx, tan_half_fovy, znear, zfar;
} gs_camera;

/* Per-iteration parameters.
 *
 * Random draws.  Every draw is output number `counter` of the SplitMix64
 * stream seeded with `seed` (state seed + (counter + 1) * 0x9E3779B97F4A7C15,
 * then the published finaliser), with counter = tag << 62 | k << 32 | row:
 *   tag 0  StSS membership: sampled iff the top 53 bits, read as a fraction
 *          of 2^53, are below restate_ratio;
 *   tag 1  AIU membership: the same test against aiu_prob;
 *   tag 2, 3  the noise vector gamma ~ N(0, I_3) by the Box-Muller transform:
 *          from each word w, ua = (w >> 40 + 1) / 2^24 and
 *          ub = ((w >> 16) & 0xFFFFFF) / 2^24; with (ua1, ub1) from tag 2 and
 *          (ua2, ub2) from tag 3, gamma = (r1 cos 2 pi ub1, r1 sin 2 pi ub1,
 *          r2 cos 2 pi ub2), r = sqrt(-2 ln ua) (FP32 on the device).
 *
 * Position noise (App. Eq. disentangled_mu): the chosen primitives'
 * positions move by -noise_lr * lr[0] * sigmoid(-noise_k (o - noise_t)) *
 * Sigma gamma, with o = sigmoid(tau), Sigma = R diag(exp(2 kappa)) R^T and R
 * the rotation of the normalised quaternion (w, x, y, z) (q / max(|q|,
 * 1e-12)), all taken from the primitive's values before this step's update.
 * The paper gives no values for noise_lr, noise_k, noise_t (3DGS-MCMC: 5e5,
 * 100, 0.005).
 *
 * AIU (Sec. 3.2): each invisible primitive is sampled with probability
 * aiu_prob; a sampled one whose step count t is non-zero (per-primitive
 * mode; any, with bias_mode 1) moves by -lr_group * aiu_scale *
 * m^/(sqrt(v^) + eps) from its current moments, bias-corrected with its t
 * (or k), which all stay unchanged.  No regulariser applies to that step.
 *
 * n_active: the number of primitives whose opacity sigmoid(tau) exceeds
 * 1/255 after the step (Sec. 4: active; the others are dead) is added to
 * this device int64.  The decision is exact: tau > -ln 254 for FP32 tau.
 *
 * The batched entry points (gs_batch_*) reject noise, AIU and n_active with
 * GS_ERR_UNSUPPORTED.
 */
typedef struct gs_step_params {
    float lr[6];             /* xyz, scale, rot, opacity, SH DC (sh cols 0-2), SH rest   */
    int32_t dar_opacity;     /* apply the opacity regulariser this step                   */
    int32_t dar_scale;       /* apply the scale regulariser this step                     */
    int32_t restate;         /* apply RSR to the StSS-sampled rows after this step        */
    int32_t reserved;        /* must be 0                                                  */
    double restate_ratio;    /* StSS sampling probability in [0, 1]                        */
    uint64_t seed;           /* seed of every random draw of the step (see above)          */
    int64_t iteration;       /* global iteration k, 1 <= k < 2^30: keys the random draws and
                                is the bias-correction step when bias_mode = 1             */
    int64_t n_visible;       /* N_v for GS_REG_COUPLED (host-known visible count), else 0  */
    int32_t noise;           /* gs_noise_mode                                              */
    int32_t aiu;             /* apply AIU this step                                        */
    float noise_lr;          /* eta_Ro of Eq. disentangled_mu, finite                      */
    float noise_k;           /* lambda_mu, finite                                          */
    float noise_t;           /* lambda_t, finite                                           */
    float aiu_prob;          /* Pro_AIU in [0, 1]                                          */
    float aiu_scale;         /* eta_AIU, finite                                            */
    int32_t reserved2;       /* must be 0                                                  */
    int64_t *n_active;       /* device int64, optional (NULL): N_a is added to it          */
} gs_step_params;

typedef struct gs_opt gs_opt;   /* opaque context */

/* Name of a status code (static string). */
const char *gs_status_string(gs_status s);

/* GS_ABI_VERSION of the loaded library. */
int32_t gs_abi_version(void);

/* N_I of App. "DAR": the leading decimal digit of n_pixels kept, divided by
 * ten (640000 -> 60000).  0 for n_pixels <= 0. */
double gs_dar_normaliser(int64_t n_pixels);

/*
 * Create a context for n_rows primitives (0 <= n_rows < 2^31 - 1).
 * Allocates and zeroes the library-owned state on the current CUDA device:
 * moments m, v in the configured precision, per-primitive step counters t
 * (all start at 0, as for newly created primitives, App. "Scaling in RSR"
 * item 1), and the FP64 bias-correction table 1 - beta^k computed on the GPU.
 * *out receives the context (NULL on failure).  Errors: GS_ERR_INVALID_ARG
 * (config out of range, reserved fields non-zero), GS_ERR_OOM, GS_ERR_CUDA.
 */
gs_status gs_opt_init(gs_opt **out, const gs_opt_config *cfg, int64_t n_rows, void *stream);

/* Free the context and its device memory (synchronises the device first).
 * NULL is ignored. */
void gs_opt_destroy(gs_opt *opt);

/* Current row count (changes with gs_reindex_state), -1 for NULL. */
int64_t gs_opt_rows(const gs_opt *opt);

/*
 * Visibility filter V of Eq. meth::sparse_beta for the view `cam`: the
 * frustum test of each mean (see gs_camera).
 *   xyz          device [n_rows][3] float32 means, read-only.
 *   mask         device [n_rows] uint8 out: 1 visible, 0 not.  Required.
 *   visible_rows device [n_rows] int32 out, optional (NULL): the visible row
 *                indices, compacted (ascending within each tile of rows,
 *                tiles in completion order; a tile is 2048 rows when xyz is
 *                16-B and mask 4-B aligned, else 256).
 *   n_visible    device int64 out, optional (NULL): the visible count; required
 *                when visible_rows is given.
 */
gs_status gs_visibility(gs_opt *opt, const float *xyz, const gs_camera *cam, uint8_t *mask,
                        int32_t *visible_rows, int64_t *n_visible, void *stream);

/*
 * One AdamW-GS step over the rows whose mask byte is non-zero.
 *   attrs  device attribute groups, updated in place for visible rows only.
 *   grads  device photometric gradients (the mean-loss gradient, i.e. already
 *          divided by N_I as a renderer returns it), same layout; read for
 *          visible rows only.
 *   mask   device [n_rows] uint8 visibility (e.g. from gs_visibility or a
 *          rasterizer's radii > 0); NULL = every row visible (dense Adam).
 * Visible row: t += 1; m, v updated by Eq. disentangled_mom; theta moved by
 * Eq. disentangled_adam with the bias-corrected moments of this step and the
 * regulariser evaluated at the attribute before the update.  Invisible row:
 * attributes, m, v, t untouched (beta' = 1).  If params->restate, every row
 * the StSS draw selects (visible or not) then has m *= alpha1, v *= alpha2
 * (Eq. meth::restate).
 */
gs_status gs_step(gs_opt *opt, const gs_attrs *attrs, const gs_grads *grads, const uint8_t *mask,
                  const gs_step_params *params, void *stream);

/*
 * gs_visibility followed by gs_step, fused into one pass over the rows:
 * each tile of rows tests its means against `cam`, compacts its visible rows
 * in shared memory and updates them.
 *   mask_out   device [n_rows] uint8 out, optional (NULL).
 *   n_visible  device int64, optional (NULL): this step's visible count is
 *              ADDED to it (atomically); zero it beforehand for a plain count.
 */
gs_status gs_step_camera(gs_opt *opt, const gs_attrs *attrs, const gs_grads *grads,
                         const gs_camera *cam, uint8_t *mask_out, int64_t *n_visible,
                         const gs_step_params *params, void *stream);

/*
 * gs_step_camera with the gradients in HOST memory; copies the visible count
 * back to *n_visible_host and synchronises `stream` before returning
 * (blocking).  When all five gradient groups are pinned host memory the
 * device can address (cudaHostAlloc / cudaHostRegister under unified
 * addressing; rot and sh 16-byte aligned), the step kernel reads the visible
 * rows' gradients in place over the CPU-GPU link and nothing else is copied.
 * Otherwise the groups are first copied into a library-owned device staging
 * buffer on `stream` (allocated on first use).  Both give the same result.
 */
gs_status gs_step_host(gs_opt *opt, const gs_attrs *attrs, const gs_grads *grads_host,
                       const gs_camera *cam, const gs_step_params *params,
                       int64_t *n_visible_host, void *stream);

/*
 * Batched step: several independent scenes (one context each, all with the
 * same moment precision, on the same device) updated by ONE persistent launch
 * whose CTAs pull (scene, tile) work items from a shared counter, so scenes
 * of very different sizes keep every SM busy until the whole batch is done.
 * Each scene has its own camera, parameters and step counters; the result of
 * every scene is identical to gs_step_camera on that scene alone.
 */
#define GS_MAX_BATCH 64
typedef struct gs_batch gs_batch;   /* opaque */

/* Create a batch over n_scenes (1..GS_MAX_BATCH) existing contexts (not
 * owned: they must outlive the batch).  Allocates a device scene table, two
 * pinned staging buffers and the work counters. */
gs_status gs_batch_create(gs_batch **out, gs_opt *const *scenes, int32_t n_scenes);

/* Free the batch (synchronises the device); NULL is ignored. */
void gs_batch_destroy(gs_batch *b);

/*
 * One step of every scene: scene s uses attrs[s], grads[s], cams[s],
 * params[s] (host arrays of n_scenes entries; the pointers inside are device
 * memory, validated as for gs_step_camera).  n_visible: optional device
 * int64[n_scenes]; each scene's visible count is added to its entry.
 * The scene table is staged in pinned memory and copied to the device on
 * `stream` before the launch.  Autotuning: the first calls of a batch run
 * each candidate launch configuration (rows per tile, SH columns per work
 * item, CTAs per SM) in turn — 3 times each — and time them with CUDA events;
 * afterwards the fastest is used.  All candidates compute identical results,
 * so tuning happens on real steps.
 */
gs_status gs_batch_step(gs_batch *b, const gs_attrs *attrs, const gs_grads *grads, const gs_camera *cams,
                        const gs_step_params *params, int64_t *n_visible, void *stream);

/*
 * gs_batch_step through a CUDA graph that the batch builds itself (a copy
 * node for the scene table and the kernel node) once tuning has finished;
 * each call refreshes the copy node's source (alternating between the two
 * pinned buffers) and launches the graph.  Before tuning has finished it
 * behaves as gs_batch_step.
 */
gs_status gs_batch_graph_step(gs_batch *b, const gs_attrs *attrs, const gs_grads *grads, const gs_camera *cams,
                              const gs_step_params *params, int64_t *n_visible, void *stream);

/* The launch configuration in use: rows per tile, SH columns per work item,
 * CTAs per SM of the persistent form (0: one CTA per tile of the whole batch,
 * scheduled by the hardware), and whether tuning has finished (1) or not (0).
 * Any output may be NULL. */
gs_status gs_batch_config(const gs_batch *b, int32_t *tile_rows, int32_t *sh_width, int32_t *blocks_per_sm,
                          int32_t *tuned);

/* Largest primitive count gs_step_host_noalloc accepts. */
#define GS_NOALLOC_MAX_ROWS 65536

/*
 * gs_step_host that allocates nothing.  The paper has no counterpart: this
 * is a deployment variant of the library's own host-gradient entry point.
 *
 * gs_step_host creates a device staging buffer for the gradients and a pinned
 * host word for the count (cudaMalloc / cudaMallocHost) the first time it runs
 * on a context.  Some callers cannot allocate at the moment they step: a
 * process that committed its whole device-memory budget at start-up, a
 * latency-critical or real-time thread on which a synchronising allocation is
 * not allowed, or a host runtime that owns the CUDA allocator and forbids
 * allocations behind its back.  This variant stages the gradients in a fixed
 * array that the library keeps in device global memory: a file-scope array
 * sized for GS_NOALLOC_MAX_ROWS rows (about 15.5 MB).  The array is reserved
 * on a GPU when the library's code is loaded there: gs_opt_init looks up its
 * device address (cudaGetSymbolAddress) on the context's device, which also
 * loads that code under CUDA's lazy module loading, so the reservation happens
 * at set-up and lasts until the process exits.  gs_step_host_noalloc itself
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Arguments, semantics, blocking behaviour and errors are those of
 * gs_step_host, plus: a context with more than GS_NOALLOC_MAX_ROWS rows gives
 * GS_ERR_INVALID_ARG and nothing is launched.  If gs_opt_init could not look
 * the address up, the first call on that device tries again (with the device
 * current, so make that call before any stream capture) and returns
 * GS_ERR_CUDA if it fails.  The address is cached per device: after a
 * cudaDeviceReset the cache is stale, and contexts from before the reset must
 * not be used anyway.  Every call in the
 * process shares the one array, which keeps the previous call's contents: the
 * visible counter is cleared on each call and the gradient staging is
 * overwritten for all rows.  Calls that overlap on the GPU (other streams,
 * threads or contexts) race on the array and must be serialised by the caller.
 */
gs_status gs_step_host_noalloc(gs_opt *opt, const gs_attrs *attrs, const gs_grads *grads_host,
                               const gs_camera *cam, const gs_step_params *params,
                               int64_t *n_visible_host, void *stream);

/*
 * Re-index the optimizer state for a new primitive set of n_new rows
 * (densify / prune / relocate).  Output row j inherits the state of old row
 * src_rows[j]; src_rows[j] < 0, or reset[j] != 0, starts it at zero m, v and
 * t = 0 (a new or relocated primitive).  Re-indexing the attribute arrays is
 * the caller's job (or gs_gather_attrs).
 *   src_rows device [n_new] int32, read-only; values must be < the old row count.
 *   reset    device [n_new] uint8, optional (NULL).
 * A source index out of range is not read: that row is zeroed and the
 * context records GS_ERR_INVALID_ARG, returned by the next gs_opt_sync_errors.
 * 0 <= n_new < 2^31 - 1; the state grows if needed (allocation is synchronous).
 */
gs_status gs_reindex_state(gs_opt *opt, const int32_t *src_rows, const uint8_t *reset,
                           int64_t n_new, void *stream);

/*
 * Gather attribute rows for a new primitive set: out row j = in row
 * src_rows[j] for every group (src_rows[j] must be in [0, n_in)); a negative
 * entry leaves out row j untouched.  in and out are distinct device buffers
 * of n_in and n_new rows.  Out-of-range sources are skipped and recorded as
 * for gs_reindex_state.
 */
gs_status gs_gather_attrs(gs_opt *opt, const gs_attrs *in, int64_t n_in, const gs_attrs *out,
                          const int32_t *src_rows, int64_t n_new, void *stream);

/*
 * Copy the state out in the canonical layout (float32 m, v [n_rows][59] in
 * the column order xyz, scale, rot, opacity, sh; uint32 t [n_rows]), decoding
 * low-precision moments.  Any of m, v, t may be NULL.  Device buffers.
 */
gs_status gs_opt_export_state(gs_opt *opt, float *m, float *v, uint32_t *t, void *stream);

/* Inverse of gs_opt_export_state (checkpoint resume); NULL leaves that part
 * unchanged.  Low-precision moments are re-encoded. */
gs_status gs_opt_import_state(gs_opt *opt, const float *m, const float *v, const uint32_t *t,
                              void *stream);

/*
 * The active primitives (opacity sigmoid(tau) > 1/255, Sec. 4 "Dataset and
 * Metric"; exactly tau > -ln 254 for FP32 tau) of the context's n_rows, in
 * ascending order: the source list of a prune of the dead primitives, ready
 * for gs_reindex_state (n_new = the count) and gs_gather_attrs.
 *   opacity  device [n_rows] float32 logits tau, read-only.
 *   rows     device [n_rows] int32 out, optional (NULL: count only).
 *   n_active device int64 out (overwritten), required.
 * Two launches (per-block counts; the ordered write, where each block adds
 * up the counts of the blocks before it); a scratch array of one int32 per
 * 4096 rows is kept by the context (allocated synchronously on first use or
 * growth).
 */
gs_status gs_active_rows(gs_opt *opt, const float *opacity, int32_t *rows, int64_t *n_active, void *stream);

/*
 * Diagnostic: the memory traffic of one step over the listed rows, without
 * the update.  For each listed row, every attribute, gradient, moment and
 * step-counter byte that gs_step reads for a visible row is read, and every
 * byte it writes is written back with the value just read, so nothing
 * changes.  Its time beside gs_step's on the same rows separates what the
 * scattered row accesses cost from what the update adds.
 *   attrs, grads  as for gs_step (device buffers of the context's n_rows).
 *   rows          device [n_listed] int32, each in [0, n_rows), e.g.
 *                 gs_visibility's visible_rows; 0 <= n_listed <= n_rows.
 * An out-of-range row is skipped and recorded as for gs_reindex_state.  One
 * launch; no allocation.
 */
gs_status gs_copy_rows(gs_opt *opt, const gs_attrs *attrs, const gs_grads *grads, const int32_t *rows,
                       int64_t n_listed, void *stream);

/* Length of the context's bias-correction table: the first step count k at
 * which both FP32 factors 1/(1 - beta1^k) and 1/sqrt(1 - beta2^k) round to
 * exactly 1 (15 936 for beta2 = 0.999), at most 2^22.  -1 for NULL. */
int64_t gs_bias_table_len(const gs_opt *opt);

/* Copy the FP64 bias-correction denominators 1 - beta1^k, 1 - beta2^k for
 * k = 0 .. len-1 (computed on the GPU at init, beta^k by binary
 * exponentiation) into device buffers; len <= gs_bias_table_len(opt). */
gs_status gs_bias_table(gs_opt *opt, double *one_minus_b1k, double *one_minus_b2k, int64_t len,
                        void *stream);

/* Synchronise `stream` and return (then clear) the first error recorded by a
 * device-side check since the last call, GS_OK if none. */
gs_status gs_opt_sync_errors(gs_opt *opt, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GSOPT_H */
