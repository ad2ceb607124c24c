// FP8 (e4m3) moments with per-256-row block scales.
//
// Storage: m and v rows of 64 bytes, the 59 e4m3 codes in work-chunk order
// (SH 0-47, rotation 48-51, xyz 52-54, opacity 55, scale 56-58; byte 59 is
// padding and bytes 60-63 of the m row hold the step counter t), so that
// each 4-value work chunk is one 32-bit word; and for every block of 256
// rows one FP32 scale per slot for m and one for v (a power of two, 0 for a
// slot that is zero throughout the block).  A value is code x scale.
//
// A block's scale is a power of two that keeps the largest magnitude of its
// slot within e4m3's finite range (448).  Sparse Adam updates only the
// visible rows of a block, but the scale belongs to all 256, so one CTA
// takes one block, in one of two ways:
//   * on most steps the scales may only grow (f8_block_grow): only the rows
//     that change are read and written, straight from and to device memory,
//     and a column whose new values no longer fit takes a larger power of
//     two (kF8Headroom binades above the smallest fitting one), with the
//     block's other rows re-encoded in that column alone;
//   * on one step in kF8FullEvery (staggered over the blocks: iteration +
//     block a multiple of it) the block's full pass recomputes every scale
//     from all 256 rows, staged in shared memory, and shrinks it when the
//     smallest fitting power of two is more than kF8Headroom binades below:
//       0. the largest code magnitude per column over the rows that stay as
//          they are (a bytewise integer max: e4m3 magnitudes order as their
//          codes);
//       1. the new values of the rows that change (visible rows: the update;
//          StSS-sampled rows: the RSR scaling), into the column maxima;
//       2. the new scales, then the same values again: attributes written
//          for visible rows, the changed values encoded with the new scales;
//       3. the kept rows re-encoded in the columns whose scale moved.
// m rounds to nearest, v stochastically, and a positive v never becomes
// zero; import sets the smallest fitting scales.  All arithmetic is FP32
// (the step_element of the other formats).

#include <cuda_fp8.h>

#include "step_common.cuh"

namespace gs {
namespace {

constexpr int kF8Tile = 256;                 // rows per block scale = rows per CTA
constexpr int kF8Cols = 59;
constexpr int kF8Row = 64;                   // bytes per code row
constexpr int kF8TWord = 15;                 // 32-bit word of the m row holding t
constexpr int kF8MinBlocks = 4;
// A block recomputes its scales from all of its rows (and may shrink them)
// on one step in kF8FullEvery, staggered over the blocks; on the others
// they may only grow.
constexpr uint32_t kF8FullEvery = 128;
// Binades above the smallest fitting power of two that a scale takes when it
// moves (except from zero): a block's moments rise over many steps while v
// builds up, and each move re-encodes the column in the block's other rows.
// 0, 1, 2, 3 and 4 binades gave the same 1000-step error on the 3 M
// workload; 3 was the fastest.
constexpr int kF8Headroom = 3;
static_assert(kF8Tile == kThreads, "one row per thread in phase A");

__device__ __forceinline__ float f8_dec(uint32_t code)
{
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)code, __NV_E4M3);
    return __half2float(__half(h));
}

__device__ __forceinline__ uint32_t f8_rn(float x) { return __nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3); }

__device__ __forceinline__ uint32_t f8_rn_floor(float x)
{
    uint32_t c = f8_rn(x);
    if ((c & 0x7fu) == 0u && x > 0.f) c = 1u;
    return c;
}

// Exponent e of the block scale 2^e for a column whose largest magnitude
// has FP32 bits b > 0: amax = M 2^k (1 <= M < 2) fits 448 = 1.75 2^8 under
// 2^(k-8) when M <= 1.75, else under 2^(k-7).  Clamped to [-126, 126] so
// that 2^e and 2^-e are normal FP32 numbers.
__device__ __forceinline__ int f8_scale_exp(uint32_t b)
{
    const int k = (int)(b >> 23) - 127;
    const int e = k - 8 + ((b & 0x7fffffu) > 0x600000u ? 1 : 0);
    return min(max(e, -126), 126);
}
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

// Slot of canonical column c (xyz 0-2, scale 3-5, rot 6-9, opacity 10,
// SH 11-58) in a code row.
__device__ __forceinline__ int f8_slot(int c)
{
    return c < 3 ? 52 + c : c < 6 ? 56 + (c - 3) : c < 10 ? 48 + (c - 6) : c == 10 ? 55 : c - 11;
}

constexpr int kF8Chunks = 15;                // 12 SH, rotation, xyz + opacity, scale

// The 4 values of a code word, times their slots' scales.
__device__ __forceinline__ void f8_dec4(uint32_t w, const float *s, float *x)
{
    const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xffffu), __NV_E4M3);
    const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
    const float2 a = __half22float2(__half2(lo)), b = __half22float2(__half2(hi));
    x[0] = a.x * s[0];
    x[1] = a.y * s[1];
    x[2] = b.x * s[2];
    x[3] = b.y * s[3];
}

__device__ __forceinline__ uint32_t f8_pack4(float y0, float y1, float y2, float y3)
{
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(y0, y1), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(y2, y3), __NV_SATFINITE, __NV_E4M3);
    return (lo & 0xffffu) | (hi << 16);
}

// First moments of a chunk, to nearest under the inverse scales inv.
__device__ __forceinline__ uint32_t f8_enc4_rn(const float *x, const float *inv)
{
    return f8_pack4(x[0] * inv[0], x[1] * inv[1], x[2] * inv[2], x[3] * inv[3]);
}

// Second moments of a chunk: each value dithered by +-1/2 e4m3 ulp (20
// random bits from the chunk's hash times a distinct odd constant, centred,
// below the 3 mantissa bits kept), then to nearest; a positive value keeps
// at least the smallest subnormal code.
__device__ __forceinline__ uint32_t f8_enc4_sr(const float *x, const float *inv, uint32_t h)
{
    constexpr uint32_t kOdd[4] = {1u, 0x9e3779b1u, 0x85ebca77u, 0xc2b2ae3du};
    float y[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        uint32_t u = __float_as_uint(x[e] * inv[e]);
        const uint32_t ex = u & 0x7f800000u;
        u += (ex != 0u && ex != 0x7f800000u) ? ((h * kOdd[e]) & 0xfffffu) - 0x80000u : 0u;
        y[e] = __uint_as_float(u);
    }
    uint32_t w = f8_pack4(y[0], y[1], y[2], y[3]);
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (((w >> (8 * e)) & 0x7fu) == 0u && x[e] > 0.f) w |= 1u << (8 * e);
    return w;
}

// Random bits of a chunk's stochastic rounding.
__device__ __forceinline__ uint32_t f8_rnd(const StepArgs &a, int64_t row, int k)
{
    return fmix32((uint32_t)row * 0x9e3779b1u ^ (uint32_t)k * 0x85ebca77u ^ (uint32_t)a.k_ctr * 0xc2b2ae3du ^
                  (uint32_t)a.seed ^ 0x165667b1u);
}

// Attributes and gradients of chunk k of row r (n = 3 for the scale chunk;
// th[3] = g[3] = 0 there).
__device__ __forceinline__ void f8_load_chunk(const StepArgs &a, const int64_t r, const int k, float *th, float *g)
{
    if (k < 12 || k == 12) {
        const float *pt = k < 12 ? a.a_sh + r * 48 + 4 * k : a.a_rot + r * 4;
        const float *pg = k < 12 ? a.g_sh + r * 48 + 4 * k : a.g_rot + r * 4;
        const float4 x = ld4(pt), y = ldg4_stream(pg);
        th[0] = x.x; th[1] = x.y; th[2] = x.z; th[3] = x.w;
        g[0] = y.x; g[1] = y.y; g[2] = y.z; g[3] = y.w;
    } else if (k == 13) {
        const float *pt = a.a_xyz + r * 3, *pg = a.g_xyz + r * 3;
        th[0] = pt[0]; th[1] = pt[1]; th[2] = pt[2]; th[3] = a.a_op[r];
        g[0] = __ldcs(pg); g[1] = __ldcs(pg + 1); g[2] = __ldcs(pg + 2); g[3] = __ldcs(a.g_op + r);
    } else {
        const float *pt = a.a_scale + r * 3, *pg = a.g_scale + r * 3;
        th[0] = pt[0]; th[1] = pt[1]; th[2] = pt[2]; th[3] = 0.f;
        g[0] = __ldcs(pg); g[1] = __ldcs(pg + 1); g[2] = __ldcs(pg + 2); g[3] = 0.f;
    }
}

__device__ __forceinline__ void f8_store_chunk(const StepArgs &a, const int64_t r, const int k, const float *th)
{
    if (k < 12 || k == 12) {
        st4(k < 12 ? a.a_sh + r * 48 + 4 * k : a.a_rot + r * 4, make_float4(th[0], th[1], th[2], th[3]));
    } else if (k == 13) {
        float *pt = a.a_xyz + r * 3;
        __stcs(pt, th[0]); __stcs(pt + 1, th[1]); __stcs(pt + 2, th[2]);
        __stcs(a.a_op + r, th[3]);
    } else {
        float *pt = a.a_scale + r * 3;
        __stcs(pt, th[0]); __stcs(pt + 1, th[1]); __stcs(pt + 2, th[2]);
    }
}

// The update of chunk k's values in place on their FP32 moments (attributes
// th in place too).  Visible rows take the Sparse Adam step with each
// column's learning rate and regulariser (opacity: sig'(tau), scale:
// exp(kappa), as the other formats' items), then the RSR post-scale when
// sampled; invisible sampled rows take the RSR scaling alone
// (Eq. meth::restate).
__device__ __forceinline__ void f8_apply_chunk(const StepArgs &a, const int k, const bool vis, const bool smp,
                                               const float2 f, float *th, const float *g, float *m, float *v)
{
    const int n = k == 14 ? 3 : 4;
    if (vis) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (e >= n) break;
            float lr;
            bool has = false;
            float gr = 0.f, lam = 0.f, clip = 0.f;
            if (k < 12) {
                lr = (k == 0 && e < 3) ? a.lr[4] : a.lr[5];
            } else if (k == 12) {
                lr = a.lr[2];
            } else if (k == 13) {
                lr = e < 3 ? a.lr[0] : a.lr[3];
                if (e == 3 && a.dar_o) { has = true; gr = dsigmoid(th[e]); lam = a.lam_o; clip = a.clip_o; }
            } else {
                lr = a.lr[1];
                if (a.dar_s) { has = true; gr = expf(th[e]); lam = a.lam_s; clip = a.clip_s; }
            }
            th[e] = step_element(th[e], g[e], m[e], v[e], f.x, f.y, a, lr, has, gr, lam, clip);
        }
    }
    if (smp) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            m[e] *= a.alpha1;
            v[e] *= a.alpha2;
        }
    }
}

// Shared arrays of a block on a grow-only step.
struct F8GrowShared {
    __align__(16) float s_old[2][64], s_inv[2][64];
    uint32_t s_max[2][64];
    uint8_t flg[kF8Tile];                     // bit 0 visible, bit 1 StSS-sampled
    int16_t clist[kF8Tile];                   // rows that change
    float2 fac[kF8Tile];
    uint16_t dmask[kF8Tile];                  // per row: the chunks deferred to pass 2
    uint16_t dlist[kF8Tile * kF8Chunks];      // deferred chunks: list index << 4 | chunk
    int nv, nc, nd, moved;
    uint8_t mov[2 * 64];                      // moment << 6 | slot
};

// A block on a step where its scales may only grow (all but one step in
// kF8FullEvery; the full pass recomputes them from every row and may shrink
// them).  Only the rows that change are read, straight from and to device
// memory, in one pass: a chunk whose new moments fit the range of the
// current scales (448 s) is stored at once; a chunk with a value outside it
// is left as it was and listed.  A column with such a value then takes the
// smallest power of two that fits it (kF8Headroom binades above that when
// the column already had a scale, so that a moment still rising does not
// move it again on the next steps), the block's other chunks are
// re-encoded in that column,
// byte by byte in place (a changed row's new value is then rounded twice),
// and the listed chunks are updated from their stored moments and encoded
// under the grown scales.
__device__ __forceinline__ void f8_block_grow(const StepArgs &a, const int vis_src, const int tile, const int nrow,
                                              F8GrowShared &S)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t r0 = (int64_t)tile * kF8Tile;
    uint8_t *gm = static_cast<uint8_t *>(a.m), *gv = static_cast<uint8_t *>(a.v);
    if (tid < 64) {
        const float sm = tid < kF8Cols ? a.msc[tile * 64 + tid] : 0.f;
        const float sv = tid < kF8Cols ? a.vsc[tile * 64 + tid] : 0.f;
        S.s_old[0][tid] = sm;
        S.s_old[1][tid] = sv;
        S.s_inv[0][tid] = sm > 0.f ? __frcp_rn(sm) : 0.f;     // exact: powers of two
        S.s_inv[1][tid] = sv > 0.f ? __frcp_rn(sv) : 0.f;
        S.s_max[0][tid] = S.s_max[1][tid] = 0u;
    }
    if (tid == 0) S.nv = S.nc = S.nd = S.moved = 0;
    if (tid < kF8Tile) S.dmask[tid] = 0;
    const int64_t row = r0 + tid;
    bool vis = false, smp = false;
    uint32_t t_old = 0;
    if (tid < nrow) {
        if (vis_src == kVisCamera) {
            const float *p = a.a_xyz + row * 3;
            vis = frustum_visible(p[0], p[1], p[2], a.cam);
        } else if (vis_src == kVisMask) {
            vis = a.mask_in[row] != 0;
        } else {
            vis = true;
        }
        if (vis) t_old = reinterpret_cast<const uint32_t *>(gm + row * kF8Row)[kF8TWord];
        if (a.mask_out) a.mask_out[row] = vis ? 1 : 0;
        if (a.restate) smp = stss_sampled(a, (int32_t)row);
    }
    const unsigned bal_v = __ballot_sync(0xffffffffu, vis), bal_c = __ballot_sync(0xffffffffu, vis || smp);
    __syncthreads();                          // scales and counters ready
    if (lane == 0 && bal_v) atomicAdd(&S.nv, __popc(bal_v));
    int base = 0;
    if (lane == 0 && bal_c) base = atomicAdd(&S.nc, __popc(bal_c));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (vis || smp) S.clist[base + __popc(bal_c & ((1u << lane) - 1u))] = (int16_t)tid;
    if (tid < nrow) {
        const uint32_t tb = a.bias_mode ? a.k_bias : t_old + 1u;
        S.fac[tid] = (vis && tb < (uint32_t)a.fac_len) ? a.fac[tb] : make_float2(1.0f, 1.0f);
        S.flg[tid] = (vis ? 1 : 0) | (smp ? 2 : 0);
    }
    __syncthreads();
    if (tid == 0 && a.n_visible && S.nv) atomicAdd(a.n_visible, (unsigned long long)S.nv);
    const int nc = S.nc, e_sh = 12 * nc, total = kF8Chunks * nc;
    // one pass over the changed rows' chunks
    for (int w = tid; w < total; w += kThreads) {
        int j, k;
        if (w < e_sh) { j = w / 12; k = w - 12 * j; }
        else { const int q = w - e_sh; k = 12 + q / nc; j = q - (k - 12) * nc; }
        const int lr = S.clist[j], fl = S.flg[lr];
        const int64_t r = r0 + lr;
        float th[4], g[4], m[4], v[4];
        if (fl & 1) f8_load_chunk(a, r, k, th, g);
        uint32_t *pm = reinterpret_cast<uint32_t *>(gm + r * kF8Row) + k;
        uint32_t *pv = reinterpret_cast<uint32_t *>(gv + r * kF8Row) + k;
        f8_dec4(*pm, &S.s_old[0][4 * k], m);
        f8_dec4(*pv, &S.s_old[1][4 * k], v);
        f8_apply_chunk(a, k, fl & 1, fl & 2, S.fac[lr], th, g, m, v);
        const int n = k == 14 ? 3 : 4;
        bool out = false;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (e >= n) break;
            const int c = 4 * k + e;
            if (fabsf(m[e]) > 448.f * S.s_old[0][c]) { atomicMax(&S.s_max[0][c], __float_as_uint(fabsf(m[e]))); out = true; }
            if (fabsf(v[e]) > 448.f * S.s_old[1][c]) { atomicMax(&S.s_max[1][c], __float_as_uint(fabsf(v[e]))); out = true; }
        }
        if (out) {                            // stored as it was; pass 2 redoes it
            S.dlist[atomicAdd(&S.nd, 1)] = (uint16_t)(j << 4 | k);
            atomicOr(reinterpret_cast<unsigned *>(&S.dmask[lr & ~1]), (1u << k) << (16 * (lr & 1)));
            continue;
        }
        if (fl & 1) f8_store_chunk(a, r, k, th);
        if (k == 14) m[3] = v[3] = 0.f;       // the padding slot
        __stcs(pm, f8_enc4_rn(m, &S.s_inv[0][4 * k]));
        __stcs(pv, f8_enc4_sr(v, &S.s_inv[1][4 * k], f8_rnd(a, r, k)));
    }
    __syncthreads();
    if (tid < 2 * kF8Cols) {                  // grow only
        const int w = tid / kF8Cols, c = tid - w * kF8Cols;
        const uint32_t b = S.s_max[w][c];
        const float so = S.s_old[w][c];
        if (b) {
            const float s = fmaxf(so, pow2f(min(f8_scale_exp(b) + (so > 0.f ? kF8Headroom : 0), 126)));
            if (s != so) {
                S.s_inv[w][c] = __frcp_rn(s);
                (w ? a.vsc : a.msc)[tile * 64 + c] = s;
                S.mov[atomicAdd(&S.moved, 1)] = (uint8_t)(w << 6 | c);
            }
        }
    }
    __syncthreads();
    // the chunks not listed, re-encoded in the columns whose scale grew
    const int nmov = S.moved;
    for (int idx = tid; idx < nrow * nmov; idx += kThreads) {
        const int lr = idx / nmov, q = S.mov[idx - lr * nmov], w = q >> 6, c = q & 63;
        if ((S.dmask[lr] >> (c >> 2)) & 1u) continue;
        uint8_t *pb = (w ? gv : gm) + (r0 + lr) * kF8Row + c;
        const float x = f8_dec(*pb) * S.s_old[w][c] * S.s_inv[w][c];
        *pb = (uint8_t)(w ? f8_rn_floor(x) : f8_rn(x));
    }
    // pass 2: the listed chunks from their stored moments, under the grown scales
    const int nd = S.nd;
    for (int d = tid; d < nd; d += kThreads) {
        const int j = S.dlist[d] >> 4, k = S.dlist[d] & 15;
        const int lr = S.clist[j], fl = S.flg[lr];
        const int64_t r = r0 + lr;
        float th[4], g[4], m[4], v[4];
        if (fl & 1) f8_load_chunk(a, r, k, th, g);
        uint32_t *pm = reinterpret_cast<uint32_t *>(gm + r * kF8Row) + k;
        uint32_t *pv = reinterpret_cast<uint32_t *>(gv + r * kF8Row) + k;
        f8_dec4(*pm, &S.s_old[0][4 * k], m);
        f8_dec4(*pv, &S.s_old[1][4 * k], v);
        f8_apply_chunk(a, k, fl & 1, fl & 2, S.fac[lr], th, g, m, v);
        if (fl & 1) f8_store_chunk(a, r, k, th);
        if (k == 14) m[3] = v[3] = 0.f;
        __stcs(pm, f8_enc4_rn(m, &S.s_inv[0][4 * k]));
        __stcs(pv, f8_enc4_sr(v, &S.s_inv[1][4 * k], f8_rnd(a, r, k)));
    }
    if (tid < nrow && vis) reinterpret_cast<uint32_t *>(gm + row * kF8Row)[kF8TWord] = t_old + 1u;   // Sec. 3.2
}

// Shared arrays of a block on its full pass.
struct F8FullShared {
    uint32_t cm[kF8Tile * kF8Row / 4], cv[kF8Tile * kF8Row / 4];
    __align__(16) float s_old[2][64], s_inv[2][64];
    float s_new[2][64];
    uint32_t s_max[2][64];
    uint32_t s_wmax[kThreads / 32][2][kF8Row / 4 - 1];
    uint8_t flg[kF8Tile];                     // bit 0 visible, bit 1 StSS-sampled
    int16_t clist[kF8Tile];                   // rows that change (visible or sampled)
    float2 fac[kF8Tile];
    int s_nv, s_nc, s_moved;                  // s_moved: slots whose scale changed, listed in s_mov
    uint8_t s_mov[2 * 64];                    // moment << 6 | slot
};

// The block one wave of resident CTAs ahead of `tile`: its means (or mask
// bytes) asked of L2, as the other formats' steps do.
__device__ __forceinline__ void f8_prefetch_ahead(const StepArgs &a, const int vis_src, const int tile)
{
    if (threadIdx.x != 0 || a.tile_ahead <= 0) return;
    const int64_t q = ((int64_t)tile + a.tile_ahead) * kF8Tile;
    if (q + kF8Tile > (int64_t)a.n_rows) return;
    if (vis_src == kVisCamera && ((uintptr_t)a.a_xyz & 15u) == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.a_xyz + q * 3), "n"(kF8Tile * 12) : "memory");
    else if (vis_src == kVisMask && ((uintptr_t)a.mask_in & 15u) == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.mask_in + q), "n"(kF8Tile) : "memory");
}

// A block on its full pass: its scales recomputed from every row.
__device__ __forceinline__ void f8_block_full(const StepArgs &a, const int vis_src, const int tile, F8FullShared &F)
{
    constexpr int kWords = kF8Row / 4 - 1;    // code words of a row (the last holds t)
    constexpr int kWarps = kThreads / 32;
    auto &cm = F.cm;
    auto &cv = F.cv;
    auto &s_old = F.s_old;
    auto &s_inv = F.s_inv;
    auto &s_new = F.s_new;
    auto &s_max = F.s_max;
    auto &s_wmax = F.s_wmax;
    auto &flg = F.flg;
    auto &clist = F.clist;
    auto &fac = F.fac;
    int &s_nv = F.s_nv, &s_nc = F.s_nc, &s_moved = F.s_moved;
    auto &s_mov = F.s_mov;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = (int64_t)tile * kF8Tile;
    const int nrow = (int)min((int64_t)kF8Tile, (int64_t)a.n_rows - r0);

    const uint4 *gm = reinterpret_cast<const uint4 *>(static_cast<const char *>(a.m) + r0 * kF8Row);
    const uint4 *gv = reinterpret_cast<const uint4 *>(static_cast<const char *>(a.v) + r0 * kF8Row);
    for (int q = tid; q < nrow * (kF8Row / 16); q += kThreads) {
        reinterpret_cast<uint4 *>(cm)[q] = __ldcs(gm + q);
        reinterpret_cast<uint4 *>(cv)[q] = __ldcs(gv + q);
    }
    if (tid < 64) {
        s_old[0][tid] = tid < kF8Cols ? a.msc[tile * 64 + tid] : 0.f;
        s_old[1][tid] = tid < kF8Cols ? a.vsc[tile * 64 + tid] : 0.f;
    }
    if (tid == 0) s_nv = s_nc = s_moved = 0;

    // phase A: one row per thread; the rows that change are listed
    const int64_t row = r0 + tid;
    bool vis = false, smp = false;
    if (tid < nrow) {
        if (vis_src == kVisCamera) {
            const float *p = a.a_xyz + row * 3;
            vis = frustum_visible(p[0], p[1], p[2], a.cam);
        } else if (vis_src == kVisMask) {
            vis = a.mask_in[row] != 0;
        } else {
            vis = true;
        }
        if (a.mask_out) a.mask_out[row] = vis ? 1 : 0;
        if (a.restate) smp = stss_sampled(a, (int32_t)row);
    }
    const unsigned bal_v = __ballot_sync(0xffffffffu, vis), bal_c = __ballot_sync(0xffffffffu, vis || smp);
    __syncthreads();                          // codes, scales and counters ready
    if (lane == 0 && bal_v) atomicAdd(&s_nv, __popc(bal_v));
    int base = 0;
    if (lane == 0 && bal_c) base = atomicAdd(&s_nc, __popc(bal_c));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (vis || smp) clist[base + __popc(bal_c & ((1u << lane) - 1u))] = (int16_t)tid;
    if (tid < nrow) {
        const uint32_t t_old = cm[tid * (kF8Row / 4) + kF8TWord];
        const uint32_t tb = a.bias_mode ? a.k_bias : t_old + 1u;
        fac[tid] = (vis && tb < (uint32_t)a.fac_len) ? a.fac[tb] : make_float2(1.0f, 1.0f);
        flg[tid] = (vis ? 1 : 0) | (smp ? 2 : 0);
    }
    // pass 0: largest code magnitude per slot over the rows that stay as
    // they are (e4m3 magnitudes order as their 7-bit codes), bytewise
    {
        const bool keep = tid < nrow && !(vis || smp);
        const uint32_t *rm = cm + tid * (kF8Row / 4), *rv = cv + tid * (kF8Row / 4);
#pragma unroll
        for (int w = 0; w < kWords; ++w) {
            uint32_t xm = keep ? rm[w] & 0x7f7f7f7fu : 0u, xv = keep ? rv[w] & 0x7f7f7f7fu : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                xm = __vmaxu4(xm, __shfl_xor_sync(0xffffffffu, xm, o));
                xv = __vmaxu4(xv, __shfl_xor_sync(0xffffffffu, xv, o));
            }
            if (lane == 0) {
                s_wmax[warp][0][w] = xm;
                s_wmax[warp][1][w] = xv;
            }
        }
    }
    __syncthreads();
    if (tid == 0 && a.n_visible && s_nv) atomicAdd(a.n_visible, (unsigned long long)s_nv);
    if (tid < 2 * 64) {                       // the kept rows' maxima as values: the starting maxima
        const int w = tid >> 6, c = tid & 63;
        uint32_t b = 0u;
        if (c < kF8Cols) {
            uint32_t x = 0u;
            for (int q = 0; q < kWarps; ++q) x = __vmaxu4(x, s_wmax[q][w][c >> 2]);
            const uint32_t code = (x >> (8 * (c & 3))) & 0x7fu;
            b = __float_as_uint(f8_dec(code) * s_old[w][c]);
        }
        s_max[w][c] = b;
    }
    __syncthreads();

    // work items: the changed rows' chunks, kind-major (all SH chunks, then
    // rotation, xyz + opacity, scale) so warps stay convergent
    const int nc = s_nc, e_sh = 12 * nc, total = kF8Chunks * nc;
    // pass 1: the changed rows' new values, into the slot maxima
    for (int w = tid; w < total; w += kThreads) {
        int j, k;
        if (w < e_sh) { j = w / 12; k = w - 12 * j; }
        else { const int q = w - e_sh; k = 12 + q / nc; j = q - (k - 12) * nc; }
        const int lr = clist[j], fl = flg[lr];
        float th[4], g[4], m[4], v[4];
        if (fl & 1) f8_load_chunk(a, r0 + lr, k, th, g);
        f8_dec4(cm[lr * (kF8Row / 4) + k], &s_old[0][4 * k], m);
        f8_dec4(cv[lr * (kF8Row / 4) + k], &s_old[1][4 * k], v);
        f8_apply_chunk(a, k, fl & 1, fl & 2, fac[lr], th, g, m, v);
        const int n = k == 14 ? 3 : 4;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (e >= n) break;
            atomicMax(&s_max[0][4 * k + e], __float_as_uint(fabsf(m[e])));
            atomicMax(&s_max[1][4 * k + e], __float_as_uint(fabsf(v[e])));
        }
    }
    __syncthreads();
    if (tid < 2 * kF8Cols) {
        // the new scale: grows at once when the slot's largest magnitude no
        // longer fits, shrinks when the smallest fitting power of two is more
        // than kF8Headroom binades below; a move (except from zero) lands
        // kF8Headroom binades above the smallest fitting one (a scale change
        // re-encodes the slot in all 256 rows; each binade of slack costs at
        // most one bit at the bottom of e4m3's range)
        const int w = tid / kF8Cols, c = tid - w * kF8Cols;
        const uint32_t b = s_max[w][c];
        const float so = s_old[w][c];
        float s = so;
        if (b) {
            const int e = f8_scale_exp(b);
            const int eo = so > 0.f ? (int)(__float_as_uint(so) >> 23) - 127 : -1000;
            if (e > eo) s = pow2f(so > 0.f ? min(e + kF8Headroom, 126) : e);
            else if (e <= eo - kF8Headroom - 1) s = pow2f(min(e + kF8Headroom, 126));
        }
        s_new[w][c] = s;
        s_inv[w][c] = s > 0.f ? __frcp_rn(s) : 0.f;      // exact: s is a power of two
        if (s != so) {
            (w ? a.vsc : a.msc)[tile * 64 + c] = s;
            s_mov[atomicAdd(&s_moved, 1)] = (uint8_t)(w << 6 | c);
        }
    } else if (tid < 2 * kF8Cols + 2) {
        const int w = tid - 2 * kF8Cols;     // the padding slot: encodes 0
        s_new[w][kF8Cols] = 0.f;
        s_inv[w][kF8Cols] = 0.f;
    }
    __syncthreads();

    // pass 2: attributes of visible rows, the changed rows' codes under the
    // new scales
    for (int w = tid; w < total; w += kThreads) {
        int j, k;
        if (w < e_sh) { j = w / 12; k = w - 12 * j; }
        else { const int q = w - e_sh; k = 12 + q / nc; j = q - (k - 12) * nc; }
        const int lr = clist[j], fl = flg[lr];
        float th[4], g[4], m[4], v[4];
        if (fl & 1) f8_load_chunk(a, r0 + lr, k, th, g);
        uint32_t *pm = cm + lr * (kF8Row / 4) + k, *pv = cv + lr * (kF8Row / 4) + k;
        f8_dec4(*pm, &s_old[0][4 * k], m);
        f8_dec4(*pv, &s_old[1][4 * k], v);
        f8_apply_chunk(a, k, fl & 1, fl & 2, fac[lr], th, g, m, v);
        if (fl & 1) f8_store_chunk(a, r0 + lr, k, th);
        if (k == 14) m[3] = v[3] = 0.f;       // the padding slot
        *pm = f8_enc4_rn(m, &s_inv[0][4 * k]);
        *pv = f8_enc4_sr(v, &s_inv[1][4 * k], f8_rnd(a, r0 + lr, k));
    }
    // the kept rows, re-encoded in the slots whose scale moved
    const int nmov = s_moved;
    for (int idx = tid; idx < nrow * nmov; idx += kThreads) {
        const int lr = idx / nmov, q = s_mov[idx - lr * nmov], w = q >> 6, c = q & 63;
        if (flg[lr]) continue;
        uint8_t *pb = reinterpret_cast<uint8_t *>(w ? cv : cm) + lr * kF8Row + c;
        const float x = f8_dec(*pb) * s_old[w][c] * s_inv[w][c];
        *pb = (uint8_t)(w ? f8_rn_floor(x) : f8_rn(x));
    }
    if (tid < nrow && vis) cm[tid * (kF8Row / 4) + kF8TWord] += 1u;   // the row's own step count (Sec. 3.2)
    __syncthreads();
    // write back the rows that changed: all of them when a scale moved
    uint4 *om4 = reinterpret_cast<uint4 *>(static_cast<char *>(a.m) + r0 * kF8Row);
    uint4 *ov4 = reinterpret_cast<uint4 *>(static_cast<char *>(a.v) + r0 * kF8Row);
    const bool all = s_moved != 0;
    for (int q = tid; q < nrow * (kF8Row / 16); q += kThreads) {
        if (!all && !flg[q / (kF8Row / 16)]) continue;
        __stcs(om4 + q, reinterpret_cast<const uint4 *>(cm)[q]);
        __stcs(ov4 + q, reinterpret_cast<const uint4 *>(cv)[q]);
    }
}

// One launch per step: the first n_full CTAs take the blocks on their full
// pass (tile = full0 + kF8FullEvery * i), so that these longer CTAs start
// first; every other CTA takes tile blockIdx.x - n_full on its grow-only
// step (returning at once for the full-pass tiles).
template <int kMinBlocks>
__global__ void __launch_bounds__(kThreads, kMinBlocks) step_fp8(const StepArgs a, const int vis_src, const int full0,
                                                                  const int n_full)
{
    __shared__ union {
        F8FullShared full;
        F8GrowShared grow;
    } sh;
    if ((int)blockIdx.x < n_full) {
        f8_block_full(a, vis_src, full0 + (int)kF8FullEvery * (int)blockIdx.x, sh.full);
        return;
    }
    const int tile = (int)blockIdx.x - n_full;
    if ((uint32_t)tile % kF8FullEvery == (uint32_t)full0) return;
    f8_prefetch_ahead(a, vis_src, tile);
    const int nrow = (int)min((int64_t)kF8Tile, (int64_t)a.n_rows - (int64_t)tile * kF8Tile);
    f8_block_grow(a, vis_src, tile, nrow, sh.grow);
}

// ------------------------------------------------------ export / import

__global__ void export_fp8_kernel(const uint8_t *__restrict__ m, const uint8_t *__restrict__ v,
                                  const float *__restrict__ msc, const float *__restrict__ vsc, int32_t n,
                                  float *__restrict__ m_out, float *__restrict__ v_out, uint32_t *__restrict__ t_out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * kF8Cols) return;
    const int64_t r = idx / kF8Cols;
    const int c = f8_slot((int)(idx - r * kF8Cols));
    const int64_t sb = (r / kF8Tile) * 64 + c;
    if (m_out) m_out[idx] = f8_dec(m[r * kF8Row + c]) * msc[sb];
    if (v_out) v_out[idx] = f8_dec(v[r * kF8Row + c]) * vsc[sb];
    if (t_out && c == 0) t_out[r] = reinterpret_cast<const uint32_t *>(m + r * kF8Row)[kF8TWord];
}

// One CTA per block: the slot maxima of the imported values, the scales,
// then the codes (both moments to nearest, a positive v never to zero).  A
// NULL part keeps the stored one.
__global__ void __launch_bounds__(kThreads) import_fp8_kernel(uint8_t *__restrict__ m, uint8_t *__restrict__ v,
                                                              float *__restrict__ msc, float *__restrict__ vsc,
                                                              int32_t n, const float *__restrict__ m_in,
                                                              const float *__restrict__ v_in,
                                                              const uint32_t *__restrict__ t_in)
{
    __shared__ uint32_t s_max[2][64];
    __shared__ float s_inv[2][64];
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kF8Tile;
    const int nrow = (int)min((int64_t)kF8Tile, (int64_t)n - r0);
    if (tid < 64) s_max[0][tid] = s_max[1][tid] = 0u;
    __syncthreads();
    const int64_t e0 = r0 * kF8Cols;
    for (int q = tid; q < nrow * kF8Cols; q += kThreads) {
        const int c = f8_slot(q % kF8Cols);
        if (m_in) atomicMax(&s_max[0][c], __float_as_uint(fabsf(m_in[e0 + q])));
        if (v_in) atomicMax(&s_max[1][c], __float_as_uint(fabsf(v_in[e0 + q])));
    }
    __syncthreads();
    if (tid < 2 * kF8Cols) {
        const int w = tid / kF8Cols, c = tid - w * kF8Cols;
        if (w ? v_in != nullptr : m_in != nullptr) {
            const uint32_t b = s_max[w][c];
            const int e = b ? f8_scale_exp(b) : 0;
            (w ? vsc : msc)[blockIdx.x * 64 + c] = b ? pow2f(e) : 0.f;
            s_inv[w][c] = b ? pow2f(-e) : 0.f;
        }
    }
    __syncthreads();
    for (int q = tid; q < nrow * kF8Cols; q += kThreads) {
        const int lr = q / kF8Cols, c = f8_slot(q - lr * kF8Cols);
        if (m_in) m[(r0 + lr) * kF8Row + c] = (uint8_t)f8_rn(m_in[e0 + q] * s_inv[0][c]);
        if (v_in) v[(r0 + lr) * kF8Row + c] = (uint8_t)f8_rn_floor(v_in[e0 + q] * s_inv[1][c]);
    }
    if (t_in && tid < nrow) reinterpret_cast<uint32_t *>(m + (r0 + tid) * kF8Row)[kF8TWord] = t_in[r0 + tid];
}

// ------------------------------------------------------------- re-index
// One CTA per output block.  Output row j takes the state of old row
// src[j] (src[j] < 0 or reset[j]: zero moments and t = 0), decoded with the
// old row's block scales and re-encoded under the output block's new
// scales (both moments to nearest, a positive v never to zero), slot by
// slot.  An out-of-range source is not read: the row is zeroed and the
// error word set.
__global__ void __launch_bounds__(kThreads) reindex_fp8_kernel(
    const uint8_t *__restrict__ m_in, const uint8_t *__restrict__ v_in, const float *__restrict__ msc_in,
    const float *__restrict__ vsc_in, int32_t n_in, uint8_t *__restrict__ m_out, uint8_t *__restrict__ v_out,
    float *__restrict__ msc_out, float *__restrict__ vsc_out, int32_t n_out, const int32_t *__restrict__ src,
    const uint8_t *__restrict__ reset, int32_t *err)
{
    __shared__ uint32_t s_max[2][64];
    __shared__ float s_inv[2][64];
    __shared__ int32_t s_src[kF8Tile];
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kF8Tile;
    const int nrow = (int)min((int64_t)kF8Tile, (int64_t)n_out - r0);
    if (tid < 64) s_max[0][tid] = s_max[1][tid] = 0u;
    if (tid < nrow) {
        int32_t s = src[r0 + tid];
        if (s >= n_in) {
            if (err) atomicCAS(err, 0, GS_ERR_INVALID_ARG);
            s = -1;
        }
        if (reset && reset[r0 + tid]) s = -1;
        s_src[tid] = s;
    }
    __syncthreads();
    for (int q = tid; q < nrow * kF8Cols; q += kThreads) {
        const int lr = q / kF8Cols, c = q - lr * kF8Cols;
        const int64_t s = s_src[lr];
        if (s < 0) continue;
        const int64_t sb = (s / kF8Tile) * 64 + c;
        atomicMax(&s_max[0][c], __float_as_uint(fabsf(f8_dec(m_in[s * kF8Row + c]) * msc_in[sb])));
        atomicMax(&s_max[1][c], __float_as_uint(fabsf(f8_dec(v_in[s * kF8Row + c]) * vsc_in[sb])));
    }
    __syncthreads();
    if (tid < 2 * kF8Cols) {
        const int w = tid / kF8Cols, c = tid - w * kF8Cols;
        const uint32_t b = s_max[w][c];
        const int e = b ? f8_scale_exp(b) : 0;
        (w ? vsc_out : msc_out)[blockIdx.x * 64 + c] = b ? pow2f(e) : 0.f;
        s_inv[w][c] = b ? pow2f(-e) : 0.f;
    }
    __syncthreads();
    for (int q = tid; q < nrow * kF8Cols; q += kThreads) {
        const int lr = q / kF8Cols, c = q - lr * kF8Cols;
        const int64_t s = s_src[lr];
        uint32_t cmv = 0u, cvv = 0u;
        if (s >= 0) {
            const int64_t sb = (s / kF8Tile) * 64 + c;
            cmv = f8_rn(f8_dec(m_in[s * kF8Row + c]) * msc_in[sb] * s_inv[0][c]);
            cvv = f8_rn_floor(f8_dec(v_in[s * kF8Row + c]) * vsc_in[sb] * s_inv[1][c]);
        }
        m_out[(r0 + lr) * kF8Row + c] = (uint8_t)cmv;
        v_out[(r0 + lr) * kF8Row + c] = (uint8_t)cvv;
    }
    if (tid < nrow) {
        const int64_t s = s_src[tid];
        const uint32_t t = s >= 0 ? reinterpret_cast<const uint32_t *>(m_in + s * kF8Row)[kF8TWord] : 0u;
        uint32_t *mo = reinterpret_cast<uint32_t *>(m_out + (r0 + tid) * kF8Row);
        mo[kF8TWord] = t;
        reinterpret_cast<uint32_t *>(v_out + (r0 + tid) * kF8Row)[kF8TWord] = 0u;
        m_out[(r0 + tid) * kF8Row + 59] = 0;
        v_out[(r0 + tid) * kF8Row + 59] = 0;
    }
}

}  // namespace

cudaError_t launch_step_fp8(const StepArgs &a, int vis_src, cudaStream_t s)
{
    if (a.n_rows <= 0) return cudaSuccess;
    auto k = step_fp8<kF8MinBlocks>;
    static int s_res[64] = {};
    StepArgs b = a;
    b.tile_ahead = resident_ctas(reinterpret_cast<const void *>(k), s_res);
    const int n_tiles = (int)((a.n_rows + kF8Tile - 1) / kF8Tile);
    // the tiles of this step's full pass: (iteration + tile) % kF8FullEvery == 0
    const int full0 = (int)((kF8FullEvery - (uint32_t)(a.k_ctr % kF8FullEvery)) % kF8FullEvery);
    const int n_full = full0 < n_tiles ? (n_tiles - full0 + (int)kF8FullEvery - 1) / (int)kF8FullEvery : 0;
    k<<<(unsigned)(n_full + n_tiles), kThreads, 0, s>>>(b, vis_src, full0, n_full);
    return cudaGetLastError();
}

cudaError_t launch_export_fp8(const StateView &st, int32_t n, float *m_out, float *v_out, uint32_t *t_out,
                              cudaStream_t s)
{
    if (n <= 0 || (!m_out && !v_out && !t_out)) return cudaSuccess;
    const int64_t total = (int64_t)n * kF8Cols;
    export_fp8_kernel<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        static_cast<const uint8_t *>(st.m), static_cast<const uint8_t *>(st.v), st.msc, st.vsc, n, m_out, v_out,
        t_out);
    return cudaGetLastError();
}

cudaError_t launch_import_fp8(const StateView &st, int32_t n, const float *m_in, const float *v_in,
                              const uint32_t *t_in, cudaStream_t s)
{
    if (n <= 0 || (!m_in && !v_in && !t_in)) return cudaSuccess;
    import_fp8_kernel<<<(unsigned)((n + kF8Tile - 1) / kF8Tile), kThreads, 0, s>>>(
        static_cast<uint8_t *>(st.m), static_cast<uint8_t *>(st.v), st.msc, st.vsc, n, m_in, v_in, t_in);
    return cudaGetLastError();
}

cudaError_t launch_reindex_fp8(const StateView &in, int32_t n_in, const StateView &out, int32_t n_out,
                               const int32_t *src, const uint8_t *reset, int32_t *err, cudaStream_t s)
{
    if (n_out <= 0) return cudaSuccess;
    reindex_fp8_kernel<<<(unsigned)((n_out + kF8Tile - 1) / kF8Tile), kThreads, 0, s>>>(
        static_cast<const uint8_t *>(in.m), static_cast<const uint8_t *>(in.v), in.msc, in.vsc, n_in,
        static_cast<uint8_t *>(out.m), static_cast<uint8_t *>(out.v), out.msc, out.vsc, n_out, src, reset, err);
    return cudaGetLastError();
}

}  // namespace gs
