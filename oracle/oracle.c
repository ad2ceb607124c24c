/*
 * FP64 CPU oracle for the AdamW-GS optimizer hot path
 * ("A Step to Decouple Optimization in 3DGS", arXiv 2601.16736).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may build, load or call it.  It
 * shares no code, header, table or constant generator with the CUDA library;
 * neither side includes or links the other.
 *
 * Every floating-point quantity of the method is carried in FP64, widened from
 * the FP32 inputs (attributes, gradients).  The visibility filter is decided
 * in FP64 too, as the sign of the distance to the nearest frustum plane
 * (orc_frustum_margin_f64).  orc_visibility_f32 is the same test evaluated in
 * plain FP32 (round-to-nearest, no fused multiply-add, fixed order); the tests
 * use it to pin how far an FP32 evaluation can stray from the FP64 decision.
 * Compile with -ffp-contract=off.
 *
 * Row layout (canonical column order of one primitive, 59 values):
 *   0-2   position mu (xyz)
 *   3-5   log-scale kappa, s = exp(kappa)            (App. Eq. "scale")
 *   6-9   rotation quaternion
 *   10    opacity logit tau, o = sigmoid(tau)        (App. Eq. "opacity")
 *   11-58 SH colour, 16 coefficients x RGB; 11-13 = DC, 14-58 = rest
 * Learning-rate groups: 0 xyz, 1 scale, 2 rotation, 3 opacity, 4 SH DC,
 * 5 SH rest.
 *
 * Parity status of each function is stated in its comment; all are pinned
 * by tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#define ORC_NCOL 59

/* Static hyper-parameters (Sec. 3, App. "Hyperparameter Selection"). */
typedef struct {
    double beta1, beta2;   /* Adam decay rates, Eq. meth::first_grad          */
    double eps;            /* outside the square root, Eq. meth::adam_update  */
    double lambda_o;       /* DAR weight on opacity, App. "DAR": 1e-3         */
    double lambda_s;       /* DAR weight on scale,   App. "DAR": 1e-5         */
    double clip_o, clip_s; /* C_t of Eq. disentangled_adam: 10 and 10         */
    double n_i;            /* DAR normaliser N_I after the digit rule          */
    double alpha1, alpha2; /* RSR factors, Eq. meth::restate: 0.2, 0.04       */
    int32_t bias_mode;     /* 0: per-primitive t (Sec. 3.2), 1: global step   */
    int32_t reg_mode;      /* 0 DAR (Eq. disentangled_adam)
                              1 coupled L1 in the moments (Eq. meth::undisentangled_mom)
                              2 AdamW-style constant penalty (Eq. disentangled_adam2)
                              3 clipped AdamW-style (Eq. disentangled_adamwithcliping) */
} orc_config;

/* ---------------------------------------------------------------- helpers */

static int lr_group(int c)
{
    if (c < 3) return 0;
    if (c < 6) return 1;
    if (c < 10) return 2;
    if (c == 10) return 3;
    if (c < 14) return 4;
    return 5;
}

/*
 * N_I rule of App. "DAR": keep only the most significant decimal digit of the
 * image pixel count, then scale down by one order of magnitude.
 * 800 x 800 = 640000 -> 600000 -> 60000.
 */
double orc_dar_normaliser(int64_t n_pixels)
{
    if (n_pixels <= 0) return 0.0;
    int64_t p = 1;
    while (n_pixels / p >= 10) p *= 10;
    int64_t msd = n_pixels / p;
    return (double)(msd * p) / 10.0;
}

/*
 * SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the state advances by the
 * golden-gamma 0x9E3779B97F4A7C15 and each output is the state passed through
 * the two xor-shift-multiply rounds of the published finaliser.  Counter-based
 * use: output number `counter` (0-based) of the stream seeded with `seed`.
 */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t counter)
{
    uint64_t z = seed + (counter + 1u) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/*
 * StSS membership (Sec. 3.2, App. "StSS in RSR"): the schedule samples the
 * existing primitives uniformly.  Read here as an independent Bernoulli(ratio)
 * draw per primitive and sampling event: u = top 53 bits of the SplitMix64
 * output for counter (k << 32 | row) scaled to [0, 1); sampled iff u < ratio.
 */
int32_t orc_stss_sampled(uint64_t seed, int64_t k, int64_t row, double ratio)
{
    uint64_t h = orc_splitmix64_at(seed, ((uint64_t)k << 32) | (uint64_t)(uint32_t)row);
    double u = (double)(h >> 11) * (1.0 / 9007199254740992.0); /* 2^-53 */
    return u < ratio;
}

/* ------------------------------------------------------------- visibility */

/*
 * Visibility filter V of Eq. meth::sparse_beta: 1 for a primitive whose mean
 * lies inside the current camera frustum, 0 otherwise.
 * cam[16] = { R (3x3 row-major world->camera), t (3), tan(fov_x/2),
 *             tan(fov_y/2), z_near, z_far }, camera looks down +z.
 * p = R mu + t;  visible iff z_near <= p.z <= z_far, |p.x| <= p.z tan_x,
 * |p.y| <= p.z tan_y.  Evaluated in FP32, products rounded before each sum,
 * sums taken left to right: near a plane this can differ from the FP64
 * decision of orc_frustum_margin_f64, which is the oracle's visibility.
 */
void orc_visibility_f32(const float *xyz, int64_t n, const float *cam, uint8_t *mask)
{
    for (int64_t i = 0; i < n; ++i) {
        const float mx = xyz[3 * i + 0], my = xyz[3 * i + 1], mz = xyz[3 * i + 2];
        float px = cam[0] * mx;
        px = px + cam[1] * my;
        px = px + cam[2] * mz;
        px = px + cam[9];
        float py = cam[3] * mx;
        py = py + cam[4] * my;
        py = py + cam[5] * mz;
        py = py + cam[10];
        float pz = cam[6] * mx;
        pz = pz + cam[7] * my;
        pz = pz + cam[8] * mz;
        pz = pz + cam[11];
        const float wx = pz * cam[12];
        const float wy = pz * cam[13];
        int vis = (pz >= cam[14]) && (pz <= cam[15]) && (fabsf(px) <= wx) && (fabsf(py) <= wy);
        mask[i] = (uint8_t)(vis ? 1 : 0);
    }
}

/*
 * The same frustum in FP64 as a signed margin: the minimum over the six
 * bounding planes of the Euclidean distance of the mean to the plane, positive
 * inside.  margin >= 0 is the oracle's visibility decision V; |margin| is how
 * far the mean is from flipping it (in world units, R being a rotation).
 */
void orc_frustum_margin_f64(const float *xyz, int64_t n, const float *cam,
                            double *margin, uint8_t *mask64)
{
    const double tx = cam[12], ty = cam[13];
    const double nx = sqrt(1.0 + tx * tx), ny = sqrt(1.0 + ty * ty);
    for (int64_t i = 0; i < n; ++i) {
        double p[3];
        for (int r = 0; r < 3; ++r)
            p[r] = (double)cam[3 * r + 0] * xyz[3 * i + 0] + (double)cam[3 * r + 1] * xyz[3 * i + 1] +
                   (double)cam[3 * r + 2] * xyz[3 * i + 2] + (double)cam[9 + r];
        double d[6];
        d[0] = p[2] - (double)cam[14];      /* near   */
        d[1] = (double)cam[15] - p[2];      /* far    */
        d[2] = (p[2] * tx - p[0]) / nx;     /* right  */
        d[3] = (p[2] * tx + p[0]) / nx;     /* left   */
        d[4] = (p[2] * ty - p[1]) / ny;     /* bottom */
        d[5] = (p[2] * ty + p[1]) / ny;     /* top    */
        double s = d[0];
        for (int j = 1; j < 6; ++j) s = d[j] < s ? d[j] : s;
        if (margin) margin[i] = s;
        if (mask64) mask64[i] = (uint8_t)(s >= 0.0);
    }
}

/* ------------------------------------------------------------------- step */

/*
 * One AdamW-GS optimizer step over n primitives, in place.
 *   theta [n*59] FP64 attributes, grad [n*59] FP32 photometric gradients
 *   (already the mean-loss gradient dl/N_I a renderer returns), m, v [n*59]
 *   FP64 moments, t [n] per-primitive step counters, mask [n] visibility
 *   (NULL = every primitive visible, i.e. dense Adam), lr[6] per group,
 *   dar_o / dar_s switch the opacity / scale regularisers, k the global
 *   iteration (1-based), n_visible the visible count N_v (reg_mode 1 only).
 *
 * Visible primitive (V = 1), Sec. 3.1 and 3.3:
 *   t += 1                                 (own asynchronous index, Sec. 3.2)
 *   m = b1 m + (1-b1) g,  v = b2 v + (1-b2) g^2     Eq. disentangled_mom
 *   m^ = m / (1 - b1^t),  v^ = v / (1 - b2^t)       bias correction
 *   d  = sqrt(v^) + eps
 *   u  = m^ / d                                     Eq. meth::adam_update
 *   opacity (tau):  u += min(l_o * sig'(tau) / N_I / d, C_o)   Eq. disentangled_opacity
 *   scale (kappa):  u += min(l_s * exp(kappa) / N_I / d, C_s)  Eq. disentangled_scaling
 *   theta -= lr_group * u                           (regulariser at the old theta)
 * Invisible primitive (V = 0): beta' = 1 in Eq. meth::sparse_beta and the
 * update is skipped, so theta, m, v and t are left exactly as they were.
 */
void orc_step(const orc_config *cfg, int64_t n, double *theta, const float *grad,
              double *m, double *v, uint32_t *t, const uint8_t *mask,
              const double *lr, int32_t dar_o, int32_t dar_s, int64_t k, int64_t n_visible)
{
    const double b1 = cfg->beta1, b2 = cfg->beta2;
    for (int64_t i = 0; i < n; ++i) {
        if (mask && !mask[i]) continue;
        t[i] += 1u;
        const double tt = cfg->bias_mode ? (double)k : (double)t[i];
        const double bc1 = 1.0 - pow(b1, tt);
        const double bc2 = 1.0 - pow(b2, tt);
        for (int c = 0; c < ORC_NCOL; ++c) {
            const int64_t e = i * ORC_NCOL + c;
            const double th = theta[e];
            double g = (double)grad[e];

            /* derivative of the L1 regulariser through the activation,
               App. Eq. opacity / Eq. scale; zero for other attributes */
            double grad_r = 0.0, lam = 0.0, clip = 0.0;
            int reg_on = 0;
            if (c == 10 && dar_o) {
                /* sig(tau) (1 - sig(tau)), with 1 - sig(tau) taken as
                   sig(-tau) so the tail does not cancel to zero */
                const double o = 1.0 / (1.0 + exp(-th));
                const double one_minus_o = 1.0 / (1.0 + exp(th));
                grad_r = o * one_minus_o;
                lam = cfg->lambda_o;
                clip = cfg->clip_o;
                reg_on = 1;
            } else if (c >= 3 && c < 6 && dar_s) {
                grad_r = exp(th);
                lam = cfg->lambda_s;
                clip = cfg->clip_s;
                reg_on = 1;
            }
            if (reg_on && cfg->reg_mode == 1)   /* gradient-coupled: into the moments */
                g += lam * grad_r / (double)n_visible;

            m[e] = b1 * m[e] + (1.0 - b1) * g;
            v[e] = b2 * v[e] + (1.0 - b2) * g * g;
            const double mh = m[e] / bc1;
            const double vh = v[e] / bc2;
            const double d = sqrt(vh) + cfg->eps;
            double u = mh / d;
            if (reg_on) {
                if (cfg->reg_mode == 0)
                    u += fmin(lam * (grad_r / cfg->n_i) / d, clip);
                else if (cfg->reg_mode == 2)
                    u += lam * grad_r;
                else if (cfg->reg_mode == 3)
                    u += fmin(lam * grad_r, clip);
            }
            theta[e] = th - lr[lr_group(c)] * u;
        }
    }
}

/*
 * Re-State Regularization, Eq. meth::restate: for every primitive the StSS
 * draw selects, m <- alpha1 m and v <- alpha2 v on all 59 attributes; t and
 * theta unchanged.  row_ids gives the global primitive id of each local row
 * (NULL = identity), so that a subset of rows draws the same samples.
 * Returns the number of sampled rows.
 */
int64_t orc_restate(const orc_config *cfg, int64_t n, double *m, double *v,
                    const int64_t *row_ids, uint64_t seed, int64_t k, double ratio)
{
    int64_t count = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t gid = row_ids ? row_ids[i] : i;
        if (!orc_stss_sampled(seed, k, gid, ratio)) continue;
        ++count;
        for (int c = 0; c < ORC_NCOL; ++c) {
            m[i * ORC_NCOL + c] *= cfg->alpha1;
            v[i * ORC_NCOL + c] *= cfg->alpha2;
        }
    }
    return count;
}

/*
 * Optimizer-state re-indexing across densify / prune / relocate (Sec. 2,
 * App. "Scaling in RSR" item (1): new and reallocated primitives start from
 * zero state, i.e. RSR with alpha1 = alpha2 = 0).  Output row j takes the
 * state of input row src[j]; src[j] < 0 or reset[j] != 0 gives zero m, v and
 * t = 0.  Returns 0, or -1 if a source index is out of range (nothing written
 * past the failing row).
 */
int32_t orc_reindex(int64_t n_old, const double *m, const double *v, const uint32_t *t,
                    int64_t n_new, const int32_t *src, const uint8_t *reset,
                    double *m_out, double *v_out, uint32_t *t_out)
{
    for (int64_t j = 0; j < n_new; ++j) {
        const int64_t s = src[j];
        if (s >= n_old) return -1;
        if (s < 0 || (reset && reset[j])) {
            for (int c = 0; c < ORC_NCOL; ++c) {
                m_out[j * ORC_NCOL + c] = 0.0;
                v_out[j * ORC_NCOL + c] = 0.0;
            }
            t_out[j] = 0u;
        } else {
            for (int c = 0; c < ORC_NCOL; ++c) {
                m_out[j * ORC_NCOL + c] = m[s * ORC_NCOL + c];
                v_out[j * ORC_NCOL + c] = v[s * ORC_NCOL + c];
            }
            t_out[j] = t[s];
        }
    }
    return 0;
}

/* Bias-correction denominators 1 - beta^k for k = 0 .. len-1, FP64. */
void orc_bias_denominators(double beta, int64_t len, double *out)
{
    for (int64_t k = 0; k < len; ++k) out[k] = 1.0 - pow(beta, (double)k);
}

/* ------------------------------------------- position noise, AIU, N_a / N_d */

/*
 * Random streams.  All draws come from the SplitMix64 stream of the step's
 * seed; the top two bits of the counter name the use, so no two uses share a
 * draw: 0 = StSS membership (orc_stss_sampled, iteration k < 2^30), 1 = AIU
 * membership, 2 and 3 = the two words behind the position noise.  Bits 32-61
 * carry the iteration k, bits 0-31 the row.
 */
static uint64_t orc_counter(uint64_t tag, int64_t k, int64_t row)
{
    return (tag << 62) | ((uint64_t)k << 32) | (uint64_t)(uint32_t)row;
}

/*
 * AIU membership (Sec. 3.2, "Artificial Implicit Update"): a uniform sampler
 * over the invisible primitives, read as an independent Bernoulli(prob) draw
 * per primitive and iteration on stream tag 1 (top 53 bits as a fraction of
 * 2^53, sampled iff below prob).
 */
int32_t orc_aiu_sampled(uint64_t seed, int64_t k, int64_t row, double prob)
{
    uint64_t h = orc_splitmix64_at(seed, orc_counter(1, k, row));
    double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
    return u < prob;
}

/*
 * gamma ~ N(0, I_3) of App. Eq. disentangled_mu, by the Box-Muller transform
 * (Box & Muller, Ann. Math. Stat. 1958).  Each of two SplitMix64 words
 * (tags 2 and 3) gives two 24-bit uniforms: ua = (bits 40..63 + 1) / 2^24 in
 * (0, 1] and ub = (bits 16..39) / 2^24 in [0, 1).  Then
 *   gamma0 = sqrt(-2 ln ua1) cos(2 pi ub1),  gamma1 = sqrt(-2 ln ua1) sin(2 pi ub1),
 *   gamma2 = sqrt(-2 ln ua2) cos(2 pi ub2).
 * The uniforms are exact in FP32 and FP64 alike; the transform runs in FP64.
 */
void orc_gauss3(uint64_t seed, int64_t k, int64_t row, double g[3])
{
    const double inv24 = 1.0 / 16777216.0;
    const double pi = 3.14159265358979323846;
    uint64_t h1 = orc_splitmix64_at(seed, orc_counter(2, k, row));
    uint64_t h2 = orc_splitmix64_at(seed, orc_counter(3, k, row));
    double ua1 = (double)((h1 >> 40) + 1u) * inv24, ub1 = (double)((h1 >> 16) & 0xFFFFFFu) * inv24;
    double ua2 = (double)((h2 >> 40) + 1u) * inv24, ub2 = (double)((h2 >> 16) & 0xFFFFFFu) * inv24;
    double r1 = sqrt(-2.0 * log(ua1)), r2 = sqrt(-2.0 * log(ua2));
    g[0] = r1 * cos(2.0 * pi * ub1);
    g[1] = r1 * sin(2.0 * pi * ub1);
    g[2] = r2 * cos(2.0 * pi * ub2);
}

/*
 * Covariance of a primitive, Sigma = R S S^T R^T, S = diag(exp(kappa)), R the
 * rotation of the quaternion q = (w, x, y, z) (real part first) after
 * normalisation q / max(|q|, 1e-12).  Row-major 3x3.
 */
void orc_covariance(const double q[4], const double kappa[3], double sig[9])
{
    double nrm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (nrm < 1e-12) nrm = 1e-12;
    const double w = q[0] / nrm, x = q[1] / nrm, y = q[2] / nrm, z = q[3] / nrm;
    const double R[9] = {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z),       2.0 * (x * z + w * y),
                         2.0 * (x * y + w * z),       1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
                         2.0 * (x * z - w * y),       2.0 * (y * z + w * x),       1.0 - 2.0 * (x * x + y * y)};
    double s2[3];
    for (int j = 0; j < 3; ++j) s2[j] = exp(2.0 * kappa[j]);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int j = 0; j < 3; ++j) acc += R[3 * a + j] * s2[j] * R[3 * b + j];
            sig[3 * a + b] = acc;
        }
}

/*
 * Position noise of App. Eq. disentangled_mu for one primitive (its 59
 * values before this iteration's update), the amount subtracted from mu:
 *   R_mu = eta_mu * sigmoid(-lambda_mu (o - lambda_t)) * Sigma gamma,  o = sigmoid(tau);
 * the bracket of Eq. disentangled_mu scales R_mu by eta_Ro / eta_mu and the
 * outer factor by eta_mu, which leaves eta_Ro * R_mu.
 */
void orc_noise_term(const double *row, double eta_ro, double eta_mu, double lam_mu, double lam_t,
                    const double gamma[3], double out[3])
{
    double sig[9];
    orc_covariance(row + 6, row + 3, sig);
    const double o = 1.0 / (1.0 + exp(-row[10]));
    const double gate = 1.0 / (1.0 + exp(lam_mu * (o - lam_t)));
    for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (int j = 0; j < 3; ++j) acc += sig[3 * a + j] * gamma[j];
        out[a] = eta_ro * eta_mu * gate * acc;
    }
}

/* Active primitive (Sec. 4, "Dataset and Metric"): opacity sigmoid(tau) >
 * 1/255; dead otherwise. */
int32_t orc_is_active(double tau)
{
    return 1.0 / (1.0 + exp(-tau)) > 1.0 / 255.0;
}

/* The active rows among n opacity logits (FP32, as stored), ascending, into
 * rows (may be NULL); returns their number N_a (N_d = n - N_a). */
int64_t orc_active_rows(const float *tau, int64_t n, int32_t *rows)
{
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        if (orc_is_active((double)tau[i])) {
            if (rows) rows[c] = (int32_t)i;
            ++c;
        }
    return c;
}

/* Switches and constants of the noise and AIU terms for one iteration. */
typedef struct {
    int32_t noise_mode;    /* 0 off, 1 visible primitives, 2 every primitive       */
    int32_t aiu;           /* AIU active this iteration                            */
    double noise_lr;       /* eta_Ro                                               */
    double noise_k;        /* lambda_mu                                            */
    double noise_t;        /* lambda_t                                             */
    double aiu_prob;       /* Pro_AIU                                              */
    double aiu_scale;      /* eta_AIU                                              */
    uint64_t seed;         /* stream seed (row ids as in orc_restate)              */
} orc_ext;

/*
 * orc_step extended by the position noise, AIU and the active count; returns
 * N_a after the iteration.  Per primitive (global id from row_ids, NULL =
 * local index):
 *   visible: the orc_step update, and with noise_mode >= 1 mu -= the noise
 *     term of the primitive's values before this update (eta_mu = lr[0]);
 *   invisible, AIU on and sampled, with a step count t > 0 (a primitive never
 *     seen has no moments): theta -= lr_group * eta_AIU * m^ / (sqrt(v^) + eps)
 *     from its current moments and t (global k when bias_mode = 1); m, v and t
 *     are kept (Sec. 3.2: moments unchanged while invisible); no DAR;
 *   invisible with noise_mode = 2: mu -= the noise term as above.
 */
int64_t orc_step_ext(const orc_config *cfg, int64_t n, double *theta, const float *grad,
                     double *m, double *v, uint32_t *t, const uint8_t *mask,
                     const double *lr, int32_t dar_o, int32_t dar_s, int64_t k, int64_t n_visible,
                     const orc_ext *x, const int64_t *row_ids)
{
    int64_t active = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t gid = row_ids ? row_ids[i] : i;
        double *th = theta + i * ORC_NCOL;
        double *mi = m + i * ORC_NCOL, *vi = v + i * ORC_NCOL;
        double old[ORC_NCOL];
        memcpy(old, th, sizeof(old));
        const int vis = !mask || mask[i];
        if (vis) {
            orc_step(cfg, 1, th, grad + i * ORC_NCOL, mi, vi, t + i, NULL, lr, dar_o, dar_s, k, n_visible);
        } else if (x->aiu && orc_aiu_sampled(x->seed, k, gid, x->aiu_prob) && (cfg->bias_mode || t[i] > 0)) {
            const double tt = cfg->bias_mode ? (double)k : (double)t[i];
            const double bc1 = 1.0 - pow(cfg->beta1, tt), bc2 = 1.0 - pow(cfg->beta2, tt);
            for (int c = 0; c < ORC_NCOL; ++c) {
                const double u = (mi[c] / bc1) / (sqrt(vi[c] / bc2) + cfg->eps);
                th[c] -= lr[lr_group(c)] * x->aiu_scale * u;
            }
        }
        if (x->noise_mode == 2 || (x->noise_mode == 1 && vis)) {
            double g[3], d[3];
            orc_gauss3(x->seed, k, gid, g);
            orc_noise_term(old, x->noise_lr, lr[0], x->noise_k, x->noise_t, g, d);
            for (int a = 0; a < 3; ++a) th[a] -= d[a];
        }
        active += orc_is_active(th[10]);
    }
    return active;
}
