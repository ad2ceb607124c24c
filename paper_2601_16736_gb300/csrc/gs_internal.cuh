// Internal declarations shared by the translation units of libgsopt.so:
// the optimizer-state layout, the kernel argument block and the device-side
// pieces of the method (frustum test, StSS draw, moment update).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "gsopt.h"

namespace gs {

// ---------------------------------------------------------------- layout
//
// Optimizer state is library-owned, so it is laid out for the step kernel,
// not in the caller's structure of arrays: one padded row of 64 slots per
// primitive for m and one for v, so that a visible primitive's 59 moments
// are one contiguous run of sectors (256 B in FP32) instead of five
// scattered runs.  Slot order inside a row:
//   0-47  SH (same column order as the sh group)
//   48-51 rotation, 52-54 xyz, 55-57 scale, 58 opacity
//   59    (m rows only) the primitive's step counter t as uint32 bits
//   60-63 padding, never read
// BF16 uses the same slots at 2 B each (128-B rows; slot 59 unused, t is one
// uint32 at byte 120, i.e. slots 60-61).
// The BF16 hybrid row (160 B) has an FP32 part of 16 slots (bytes 0-63) for
// the 14 columns whose learning rate is large relative to their magnitude —
// [0-2] SH DC, [3] t (m only), [4-7] rotation, [8-10] xyz, [11-13] scale,
// [14] opacity, [15] unused — followed by a BF16 part of the 48 SH columns
// (bytes 64-159; its slots 0-2 are unused, the DC moments live in the FP32
// part).
constexpr int kSlots = 64;
constexpr int kRowBytesF32 = 256, kTByteF32 = 4 * 59;
constexpr int kRowBytesBf16 = 128, kTByteBf16 = 120;
constexpr int kRowBytesHyb = 160, kTByteHyb = 12, kHybShByte = 64;
// GS_MOM_FP16_BLOCK rows (128 B): SH columns as FP16 at byte 2j (items of 8
// columns at 16i), the 8 item exponents at 96 + item, rotation at 104,
// xyz / scale / opacity at 112 .. 125, t (uint16) at 126.
constexpr int kRowBytesF16B = 128, kTByteF16B = 126, kF16BExp = 96, kF16BRot = 104, kF16BXso = 112;
constexpr int kSlotSh = 0, kSlotRot = 48, kSlotXyz = 52, kSlotScale = 55, kSlotOpacity = 58;
constexpr int kSlotT = 59;
constexpr int kNumCols = 59;

// canonical column (xyz, scale, rot, opacity, sh) -> state slot
__host__ __device__ inline int slot_of_col(int c)
{
    if (c < 3) return kSlotXyz + c;
    if (c < 6) return kSlotScale + (c - 3);
    if (c < 10) return kSlotRot + (c - 6);
    if (c == 10) return kSlotOpacity;
    return kSlotSh + (c - 11);
}

enum VisSource : int { kVisAll = 0, kVisMask = 1, kVisCamera = 2 };

// Floats of the camera argument the kernels take: gs_camera's 16, then the
// frustum band constants (see frustum_visible).
constexpr int kCamFloats = 20;

// ------------------------------------------------------------ arguments

struct StepArgs {
    float *a_xyz, *a_scale, *a_rot, *a_op, *a_sh;
    const float *g_xyz, *g_scale, *g_rot, *g_op, *g_sh;
    void *m, *v;                 // state rows
    const float2 *fac;           // per step count k: {1/(1-b1^k), 1/sqrt(1-b2^k)}
    int32_t fac_len;             // factors are exactly 1.0f from here on
    int32_t n_rows;
    const uint8_t *mask_in;      // kVisMask
    uint8_t *mask_out;           // optional
    unsigned long long *n_visible;  // optional, accumulated with atomicAdd
    int32_t *err;                // device error word (first error wins)
    float cam[kCamFloats];       // gs_camera as 16 floats + the frustum band constants (camera_arg)
    float lr[6];
    float c1, c2;                // 1 - beta1, 1 - beta2 (FP32 of the FP64 values)
    float eps;
    float lam_o, lam_s;          // regulariser weights as the reg_mode consumes them
    float clip_o, clip_s;
    float alpha1, alpha2;
    int32_t dar_o, dar_s, restate, bias_mode, reg_mode;
    uint32_t k_bias;             // step used for bias correction when bias_mode == 1
    uint64_t seed;
    uint64_t k_ctr;              // iteration k: bits 32-61 of every draw counter
    uint64_t rs_thr;             // row sampled iff (draw >> 11) < rs_thr
    // position noise (App. Eq. disentangled_mu), AIU (Sec. 3.2), active count
    int32_t noise;               // gs_noise_mode
    int32_t aiu;                 // AIU on this step
    float noise_scale;           // eta_Ro * lr[0]
    float noise_k, noise_t;      // lambda_mu, lambda_t
    float aiu_scale;             // eta_AIU
    float tau_act;               // active iff tau > tau_act (largest float below -ln 254)
    uint64_t aiu_thr;            // AIU-sampled iff (draw >> 11) < aiu_thr
    unsigned long long *n_active;   // optional, accumulated with atomicAdd
    int32_t g_host;              // gradients are pinned host memory read in place
    int32_t tile_ahead;          // CTAs resident at once (0: no look-ahead prefetch)
    float *msc, *vsc;            // FP8 moments: per-(256-row block, column) scales of m, v
};

// ------------------------------------------------------- device helpers

// Frustum test of one mean (z_near <= p_z <= z_far, |p_x| <= p_z tan_x,
// |p_y| <= p_z tan_y with p = R mu + t), decided exactly.
//
// Fast path: FP32, each coordinate by three fused multiply-adds
// (t_r + R_r2 mu_2, then + R_r1 mu_1, then + R_r0 mu_0) and each plane's slack
// (p_z - z_near, z_far - p_z, p_z tan - |p_x|, p_z tan - |p_y|) by one more
// rounding.  Unrolling the roundings, each computed coordinate is within
// gamma_3 S_r of the exact one, S_r = sum_j |R_rj mu_j| + |t_r| (gamma_n =
// n u / (1 - n u), u = 2^-24).  The kernels take e = 2^-21 (rs max_j |mu_j| +
// max_r |t_r|), rs = max_r sum_j |R_rj|, which bounds 2^-21 S_r for every r,
// more than twice gamma_3 S_r.  Wherever the slack exceeds e for the near and
// far planes and e (1 + tan) for the sides, the FP32 decision is the exact
// one (a slack's own rounding keeps its sign).  A mean inside that band (a
// few per million for scenes of this extent) is decided again in FP64: the
// products of FP32 values are exact there and the sums round at 2^-53, so the
// decision is exact up to ~1e-14 of a plane.
//
// The camera as the kernels see it: the 16 floats of gs_camera, then
// {2^-21 rs, 2^-21 max_r |t_r|, 1 + tan_x, 1 + tan_y} (camera_arg), each
// rounded up.
inline void camera_arg(const float *cam16, float *out)
{
    double rs = 0.0, tm = 0.0;
    for (int r = 0; r < 3; ++r) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j) s += cam16[3 * r + j] < 0 ? -(double)cam16[3 * r + j] : (double)cam16[3 * r + j];
        rs = s > rs ? s : rs;
        const double t = cam16[9 + r] < 0 ? -(double)cam16[9 + r] : (double)cam16[9 + r];
        tm = t > tm ? t : tm;
    }
    constexpr double kUp = 1.0 + 0x1p-20;    // covers the rounding of these factors to FP32
    for (int i = 0; i < 16; ++i) out[i] = cam16[i];
    out[16] = (float)(rs * 0x1p-21 * kUp);
    out[17] = (float)(tm * 0x1p-21 * kUp);
    out[18] = (float)((1.0 + (double)cam16[12]) * kUp);
    out[19] = (float)((1.0 + (double)cam16[13]) * kUp);
}

static __device__ __noinline__ bool frustum_visible_f64(float x, float y, float z, float c0, float c1, float c2,
                                                        float c3, float c4, float c5, float c6, float c7, float c8,
                                                        float t0, float t1, float t2, float tx, float ty, float zn,
                                                        float zf)
{
    const double X = x, Y = y, Z = z;
    const double px = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(c0, X), __dmul_rn(c1, Y)), __dmul_rn(c2, Z)), t0);
    const double py = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(c3, X), __dmul_rn(c4, Y)), __dmul_rn(c5, Z)), t1);
    const double pz = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(c6, X), __dmul_rn(c7, Y)), __dmul_rn(c8, Z)), t2);
    return (pz >= (double)zn) && (pz <= (double)zf) && (fabs(px) <= __dmul_rn(pz, (double)tx)) &&
           (fabs(py) <= __dmul_rn(pz, (double)ty));
}

// c: kCamFloats floats (camera_arg).
__device__ __forceinline__ bool frustum_visible(float x, float y, float z, const float *c)
{
    const float px = fmaf(c[0], x, fmaf(c[1], y, fmaf(c[2], z, c[9])));
    const float py = fmaf(c[3], x, fmaf(c[4], y, fmaf(c[5], z, c[10])));
    const float pz = fmaf(c[6], x, fmaf(c[7], y, fmaf(c[8], z, c[11])));
    const float s_near = pz - c[14], s_far = c[15] - pz;
    const float s_x = fmaf(pz, c[12], -fabsf(px)), s_y = fmaf(pz, c[13], -fabsf(py));
    const bool vis = (s_near >= 0.f) && (s_far >= 0.f) && (s_x >= 0.f) && (s_y >= 0.f);
    const float e = fmaf(c[16], fmaxf(fmaxf(fabsf(x), fabsf(y)), fabsf(z)), c[17]);
    const bool near_plane = (fabsf(s_near) <= e) || (fabsf(s_far) <= e) || (fabsf(s_x) <= e * c[18]) ||
                            (fabsf(s_y) <= e * c[19]);
    if (!near_plane) return vis;
    return frustum_visible_f64(x, y, z, c[0], c[1], c[2], c[3], c[4], c[5], c[6], c[7], c[8], c[9], c[10], c[11],
                               c[12], c[13], c[14], c[15]);
}

// SplitMix64 (Steele, Lea & Flood 2014), counter-based: output number
// `counter` of the stream seeded with `seed`.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t counter)
{
    uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Counter of a draw: the use in bits 62-63 (0 StSS, 1 AIU, 2-3 noise), the
// iteration in bits 32-61, the row in bits 0-31.
__device__ __forceinline__ uint64_t draw_counter(uint64_t tag, uint64_t k, int32_t row)
{
    return (tag << 62) | (k << 32) | (uint64_t)(uint32_t)row;
}

// StSS membership of `row` at the sampling event a.k_ctr.
__device__ __forceinline__ bool stss_sampled(const StepArgs &a, int32_t row)
{
    const uint64_t h = splitmix64_at(a.seed, draw_counter(0, a.k_ctr, row));
    return (h >> 11) < a.rs_thr;
}

// AIU membership of an invisible `row` (Sec. 3.2: a uniform sampler).
__device__ __forceinline__ bool aiu_sampled(const StepArgs &a, int32_t row)
{
    const uint64_t h = splitmix64_at(a.seed, draw_counter(1, a.k_ctr, row));
    return (h >> 11) < a.aiu_thr;
}

// Derivative of the L1 regulariser through the opacity activation,
// sig(tau)(1 - sig(tau)), written as e/(1+e)^2 with e = exp(-|tau|) so the
// tails do not cancel (the two forms are equal for every tau).
__device__ __forceinline__ float dsigmoid(float tau)
{
    const float e = expf(-fabsf(tau));
    const float d = 1.0f + e;
    return e / (d * d);
}

// Square root by the hardware approximation (PTX sqrt.approx.f32: relative
// error within 2^-23, exact at 0, +inf at +inf).  The correctly rounded
// square root and division cost the FP16-block step 4 % of its time; their
// difference from these is far below the step's other FP32 rounding.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One element of the step: moments (Eq. disentangled_mom, as the
// equivalent update m += (1-b1)(g - m), v += (1-b2)(g^2 - v), which keeps the
// FP32 decay exactly complementary to the FP32 gain), bias-corrected
// direction m^/(sqrt(v^)+eps) (Eq. meth::adam_update) and the regulariser
// term of the configured reg_mode (Eq. disentangled_adam for DAR).  Returns
// the new attribute value.  `gr` is dR/dtheta at the old attribute; `has_reg`
// selects whether this element carries a regulariser this step.  The
// quotients use the fast division (__fdividef, within 2 ulp): d lies far
// inside [2^-126, 2^126] whenever v > 0 or eps > 0 (sqrt(v) >= 2^-75, and
// below 2^70 for any finite v), where that division is accurate.
__device__ __forceinline__ float step_element(float th, float g, float &m, float &v, float r1, float r2,
                                              const StepArgs &a, float lr, bool has_reg, float gr,
                                              float lam, float clip)
{
    if (has_reg && a.reg_mode == GS_REG_COUPLED) g = fmaf(lam, gr, g);
    m = fmaf(a.c1, g - m, m);
    v = fmaf(a.c2, fmaf(g, g, -v), v);
    const float d = fmaf(sqrt_approx(v), r2, a.eps);
    float u = __fdividef(m * r1, d);
    if (has_reg) {
        if (a.reg_mode == GS_REG_DAR) u += fminf(__fdividef(lam * gr, d), clip);
        else if (a.reg_mode == GS_REG_ADAMW) u += lam * gr;
        else if (a.reg_mode == GS_REG_ADAMW_CLIP) u += fminf(lam * gr, clip);
    }
    return fmaf(-lr, u, th);
}

// GS_MOM_FP16_BLOCK encoding.  A group of values shares one exponent byte:
// the largest biased FP32 exponent e among them (0 when every magnitude is
// below 2^-112).  Values are stored as FP16 of x * 2^(141 - e), which puts
// the largest magnitude in [2^14, 2^15).
__device__ __forceinline__ uint32_t group_exponent(const float *x, int n)
{
    uint32_t b = 0;                       // the largest magnitude's bits
    for (int q = 0; q < n; ++q) b = max(b, __float_as_uint(x[q]) & 0x7fffffffu);
    const uint32_t e = b >> 23;
    return e < 15u ? 0u : e;
}
// 2^(141 - e) and 2^(e - 141) as exact FP32 powers of two (15 <= e <= 254)
__device__ __forceinline__ float enc_scale(uint32_t e) { return __uint_as_float((268u - e) << 23); }
__device__ __forceinline__ float dec_scale(uint32_t e) { return e ? __uint_as_float((e - 14u) << 23) : 0.f; }

__device__ __forceinline__ uint32_t h_bits(float y) { return __half_as_ushort(__float2half_rn(y)); }


// Canonical column c -> byte offset of its FP16 value in an FP16-block row
// and the index of its group exponent.
__host__ __device__ inline void f16b_slot(int c, int &byte, int &group)
{
    if (c < 6) { byte = kF16BXso + 2 * c; group = 7; }                  // xyz, scale
    else if (c < 10) { byte = kF16BRot + 2 * (c - 6); group = 6; }      // rotation
    else if (c == 10) { byte = kF16BXso + 12; group = 7; }              // opacity
    else { byte = 2 * (c - 11); group = (c - 11) / 8; }                 // SH
}

// Scene table of one batched launch (in device memory, written by one
// host-to-device copy before each launch or graph replay).
constexpr int kMaxBatch = 64;
struct BatchParams {
    int32_t n_scenes;
    int32_t total_tiles;
    int32_t tile_start[kMaxBatch + 1];
    StepArgs args[kMaxBatch];
};

// Programmatic dependent launch.  The kernels of this library are launched
// with programmatic stream serialisation, so a kernel may start while the
// kernel before it in the stream is still running: every CTA first lets the
// next launch be scheduled (once all of this grid's CTAs have started, its
// CTAs may take SM slots as this grid's last wave drains), then waits until
// the previous grid has completed and its writes are visible, before
// touching any data.  The next kernel's CTAs are thus resident when this one
// ends, instead of being launched then (2 % per step on the 1 M workload).
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <class... Args>
inline cudaError_t launch_pdl(void (*kernel)(Args...), unsigned grid, unsigned block, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// --------------------------------------------------- launch entry points
// (defined in the kernel translation units, called by api.cu)

cudaError_t launch_step(const StepArgs &a, int prec, int vis_src, cudaStream_t s);
// the step with AIU or noise on every row (launch_step forwards to it; the count
// and noise on visible rows alone take the plain kernel's terms form)
cudaError_t launch_step_ext(const StepArgs &a, int prec, int vis_src, cudaStream_t s);
// Batched launch with candidate configuration `cand` (0 .. batch_candidates-1)
// over the device scene table p (tile_start built for that candidate's tile
// size, see batch_candidate_info; total_tiles its tile count); *grid receives
// the grid (the persistent grid, or total_tiles for the one-CTA-per-tile
// form, min_blocks 0).  With fn != NULL nothing is launched: *fn receives the
// kernel (for graph nodes).
int batch_candidates(int prec);
void batch_candidate_info(int prec, int cand, int *tile, int *width, int *min_blocks);
cudaError_t launch_batch(const BatchParams *p, unsigned *work, unsigned *done, int total_tiles, int prec, int cand,
                         cudaStream_t s, int *grid, void **fn);
cudaError_t launch_active_rows(const float *tau, int32_t n, float tau_act, int32_t *blk, int32_t *rows,
                               long long *n_active, cudaStream_t s);
int64_t active_rows_scratch(int64_t n);     // int32 entries of scratch launch_active_rows needs
cudaError_t launch_visibility(const float *xyz, int32_t n, const float cam[kCamFloats], uint8_t *mask,
                              int32_t *list, unsigned long long *count, cudaStream_t s);
cudaError_t launch_bias_table(double beta1, double beta2, int32_t len, double *t1, double *t2,
                              float2 *fac, cudaStream_t s);
// State of one context as the kernels see it: its format and m, v rows.
struct StateView {
    int prec;
    void *m, *v;
    float *msc = nullptr, *vsc = nullptr;     // FP8 block scales (64 floats per 256 rows)
};

// FP8 (e4m3) moments with per-256-row block scales (csrc/step_fp8.cu).
constexpr int kRowBytesF8 = 64, kF8BlockRows = 256;
cudaError_t launch_step_fp8(const StepArgs &a, int vis_src, cudaStream_t s);
cudaError_t launch_export_fp8(const StateView &st, int32_t n, float *m_out, float *v_out, uint32_t *t_out,
                              cudaStream_t s);
cudaError_t launch_import_fp8(const StateView &st, int32_t n, const float *m_in, const float *v_in,
                              const uint32_t *t_in, cudaStream_t s);
cudaError_t launch_reindex_fp8(const StateView &in, int32_t n_in, const StateView &out, int32_t n_out,
                               const int32_t *src, const uint8_t *reset, int32_t *err, cudaStream_t s);

cudaError_t launch_reindex(const StateView &in, int32_t n_in, const StateView &out, int32_t n_out,
                           const int32_t *src, const uint8_t *reset, int32_t *err, cudaStream_t s);
cudaError_t launch_export(const StateView &st, int32_t n, float *m_out, float *v_out, uint32_t *t_out,
                          cudaStream_t s);
cudaError_t launch_import(const StateView &st, int32_t n, const float *m_in, const float *v_in,
                          const uint32_t *t_in, cudaStream_t s);
cudaError_t launch_copy_rows(const gs_attrs &a, const gs_grads &g, void *m, void *v, int32_t row_bytes,
                             int32_t used_bytes, const int32_t *rows, int64_t n_listed, int32_t n, int32_t *err,
                             cudaStream_t s);
cudaError_t launch_gather_attrs(const gs_attrs &in, int32_t n_in, const gs_attrs &out,
                                const int32_t *src, int32_t n_new, int32_t *err, cudaStream_t s);

}  // namespace gs
