// FP8 (e4m3) moments with per-256-row block scales.
//
// Storage: m and v rows of 64 bytes (the 59 e4m3 codes in canonical column
// order, xyz 0-2, scale 3-5, rot 6-9, opacity 10, SH 11-58; bytes 60-63 of
// the m row hold the step counter t), and for every block of 256 rows one
// FP32 scale per column for m and one for v (a power of two, 0 for a column
// that is zero throughout the block).  A value is code x scale.
//
// A block's scale is the smallest power of two that puts the largest
// magnitude of its column within e4m3's finite range (448).  Sparse Adam
// updates only the visible rows of a block, but the scale belongs to all
// 256, so one CTA takes one block, with its codes staged in shared memory:
//   0. the largest code magnitude per column over the rows that stay as they
//      are (a bytewise integer max: e4m3 magnitudes order as their codes);
//   1. the new values of the rows that change (visible rows: the update;
//      StSS-sampled rows: the RSR scaling), into the column maxima;
//   2. the new scales, then the same values again: attributes written for
//      visible rows, the changed values encoded with the new scales (m to
//      nearest, v stochastically, a positive v never to zero);
//   3. the kept rows re-encoded in the columns whose scale moved.
// All arithmetic is FP32 (the step_element of the other formats).

#include <cuda_fp8.h>

#include "step_common.cuh"

namespace gs {
namespace {

constexpr int kF8Tile = 256;                 // rows per block scale = rows per CTA
constexpr int kF8Cols = 59;
constexpr int kF8Row = 64;                   // bytes per code row
constexpr int kF8TWord = 15;                 // 32-bit word of the m row holding t
constexpr int kF8MinBlocks = 4;
static_assert(kF8Tile == kThreads, "one row per thread in phase A");

__device__ __forceinline__ float f8_dec(uint32_t code)
{
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)code, __NV_E4M3);
    return __half2float(__half(h));
}

__device__ __forceinline__ uint32_t f8_rn(float x) { return __nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3); }

// Second moment, rounded stochastically: a dither of +-1/2 e4m3 ulp (20
// random bits, centred, below the 3 mantissa bits e4m3 keeps) then nearest.
// In e4m3's subnormal range the dither is below the quantum and the value
// rounds to nearest.  A positive value never becomes zero (the smallest
// subnormal, 2^-9 of the scale, is kept instead), so m != 0 never meets
// v = 0 in the direction m^ / (sqrt(v^) + eps).
__device__ __forceinline__ uint32_t f8_sr(float x, uint32_t rnd)
{
    uint32_t u = __float_as_uint(x);
    const uint32_t e = u & 0x7f800000u;
    u += (e != 0u && e != 0x7f800000u) ? (rnd & 0xfffffu) - 0x80000u : 0u;
    uint32_t c = f8_rn(__uint_as_float(u));
    if ((c & 0x7fu) == 0u && x > 0.f) c = 1u;
    return c;
}

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

// Random bits of the stochastic rounding of element (row, column).
__device__ __forceinline__ uint32_t f8_rnd(const StepArgs &a, int64_t row, int c)
{
    return fmix32((uint32_t)row * 0x9e3779b1u ^ (uint32_t)c * 0x85ebca77u ^ (uint32_t)a.k_ctr * 0xc2b2ae3du ^
                  (uint32_t)a.seed ^ 0x165667b1u);
}

// Attribute and gradient of element (row r, canonical column c), with the
// column's learning rate and regulariser kind (1: scale, 2: opacity).
struct F8Elem {
    float *th;
    const float *g;
    float lr;
    int reg;
};
__device__ __forceinline__ F8Elem f8_elem(const StepArgs &a, const int64_t r, const int c)
{
    if (c < 3) return {a.a_xyz + r * 3 + c, a.g_xyz + r * 3 + c, a.lr[0], 0};
    if (c < 6) return {a.a_scale + r * 3 + (c - 3), a.g_scale + r * 3 + (c - 3), a.lr[1], 1};
    if (c < 10) return {a.a_rot + r * 4 + (c - 6), a.g_rot + r * 4 + (c - 6), a.lr[2], 0};
    if (c == 10) return {a.a_op + r, a.g_op + r, a.lr[3], 2};
    return {a.a_sh + r * 48 + (c - 11), a.g_sh + r * 48 + (c - 11), c < 14 ? a.lr[4] : a.lr[5], 0};
}

// The update of one element in place on its FP32 moments, from its loaded
// attribute t0 and gradient gv; returns the new attribute.  Visible rows take
// the Sparse Adam step with the column's learning rate and regulariser
// (opacity: sig'(tau), scale: exp(kappa), as the other formats' items), then
// the RSR post-scale when sampled; invisible sampled rows take the RSR
// scaling alone (Eq. meth::restate).
__device__ __forceinline__ float f8_apply(const StepArgs &a, const F8Elem &e, const bool vis, const bool smp,
                                          const float2 f, const float t0, const float gv, float &m, float &v)
{
    float t1 = t0;
    if (vis) {
        bool has = false;
        float gr = 0.f, lam = 0.f, clip = 0.f;
        if (e.reg == 1 && a.dar_s) { has = true; gr = expf(t0); lam = a.lam_s; clip = a.clip_s; }
        else if (e.reg == 2 && a.dar_o) { has = true; gr = dsigmoid(t0); lam = a.lam_o; clip = a.clip_o; }
        t1 = step_element(t0, gv, m, v, f.x, f.y, a, e.lr, has, gr, lam, clip);
    }
    if (smp) {
        m *= a.alpha1;
        v *= a.alpha2;
    }
    return t1;
}

// Elements per thread whose loads are issued together in the two passes.
constexpr int kF8Unroll = 4;

template <int kMinBlocks>
__global__ void __launch_bounds__(kThreads, kMinBlocks) step_fp8(const StepArgs a, const int vis_src)
{
    constexpr int kWords = kF8Row / 4 - 1;    // code words of a row (the last holds t)
    constexpr int kWarps = kThreads / 32;
    __shared__ uint4 cm[kF8Tile * kF8Row / 16], cv[kF8Tile * kF8Row / 16];
    __shared__ float s_old[2][64], s_new[2][64], s_inv[2][64];
    __shared__ uint32_t s_max[2][64];
    __shared__ uint32_t s_wmax[kWarps][2][kWords];
    __shared__ uint8_t flg[kF8Tile];          // bit 0 visible, bit 1 StSS-sampled
    __shared__ int16_t clist[kF8Tile];        // rows that change (visible or sampled)
    __shared__ float2 fac[kF8Tile];
    __shared__ int s_nv, s_nc, s_moved;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * kF8Tile;
    const int nrow = (int)min((int64_t)kF8Tile, (int64_t)a.n_rows - r0);
    prefetch_tile_ahead<kF8Tile>(a, vis_src);

    const uint4 *gm = reinterpret_cast<const uint4 *>(static_cast<const char *>(a.m) + r0 * kF8Row);
    const uint4 *gv = reinterpret_cast<const uint4 *>(static_cast<const char *>(a.v) + r0 * kF8Row);
    for (int q = tid; q < nrow * (kF8Row / 16); q += kThreads) {
        cm[q] = __ldcs(gm + q);
        cv[q] = __ldcs(gv + q);
    }
    if (tid < 64) {
        s_old[0][tid] = tid < kF8Cols ? a.msc[blockIdx.x * 64 + tid] : 0.f;
        s_old[1][tid] = tid < kF8Cols ? a.vsc[blockIdx.x * 64 + tid] : 0.f;
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
        const uint32_t t_old = reinterpret_cast<const uint32_t *>(cm)[tid * (kF8Row / 4) + kF8TWord];
        const uint32_t tb = a.bias_mode ? a.k_bias : t_old + 1u;
        fac[tid] = (vis && tb < (uint32_t)a.fac_len) ? a.fac[tb] : make_float2(1.0f, 1.0f);
        flg[tid] = (vis ? 1 : 0) | (smp ? 2 : 0);
    }
    // pass 0: largest code magnitude per column over the rows that stay as
    // they are (e4m3 magnitudes order as their 7-bit codes), bytewise
    {
        const bool keep = tid < nrow && !(vis || smp);
        const uint32_t *rm = reinterpret_cast<const uint32_t *>(cm) + tid * (kF8Row / 4);
        const uint32_t *rv = reinterpret_cast<const uint32_t *>(cv) + tid * (kF8Row / 4);
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

    // pass 1: the changed rows' new values, into the column maxima
    const uint8_t *bm = reinterpret_cast<const uint8_t *>(cm), *bv = reinterpret_cast<const uint8_t *>(cv);
    const int nc = s_nc, total = nc * kF8Cols;
    for (int b0 = tid; b0 < total; b0 += kF8Unroll * kThreads) {
        float t0[kF8Unroll], gv[kF8Unroll];
#pragma unroll
        for (int u = 0; u < kF8Unroll; ++u) {          // the visible elements' loads, all in flight
            const int idx = b0 + u * kThreads;
            t0[u] = gv[u] = 0.f;
            if (idx < total) {
                const int j = idx / kF8Cols, lr = clist[j];
                if (flg[lr] & 1) {
                    const F8Elem e = f8_elem(a, r0 + lr, idx - j * kF8Cols);
                    t0[u] = *e.th;
                    gv[u] = *e.g;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kF8Unroll; ++u) {
            const int idx = b0 + u * kThreads;
            if (idx >= total) continue;
            const int j = idx / kF8Cols, c = idx - j * kF8Cols, lr = clist[j];
            const int fl = flg[lr];
            float m = f8_dec(bm[lr * kF8Row + c]) * s_old[0][c], v = f8_dec(bv[lr * kF8Row + c]) * s_old[1][c];
            f8_apply(a, f8_elem(a, r0 + lr, c), fl & 1, fl & 2, fac[lr], t0[u], gv[u], m, v);
            atomicMax(&s_max[0][c], __float_as_uint(fabsf(m)));
            atomicMax(&s_max[1][c], __float_as_uint(fabsf(v)));
        }
    }
    __syncthreads();
    if (tid < 2 * kF8Cols) {
        const int w = tid / kF8Cols, c = tid - w * kF8Cols;
        const uint32_t b = s_max[w][c];
        float s = 0.f, inv = 0.f;
        if (b) {
            const int e = f8_scale_exp(b);
            s = pow2f(e);
            inv = pow2f(-e);
        }
        s_new[w][c] = s;
        s_inv[w][c] = inv;
        if (s != s_old[w][c]) {
            (w ? a.vsc : a.msc)[blockIdx.x * 64 + c] = s;
            s_moved = 1;
        }
    }
    __syncthreads();

    // pass 2: attributes of visible rows, the changed rows' codes under the
    // new scales
    uint8_t *wm = reinterpret_cast<uint8_t *>(cm), *wvb = reinterpret_cast<uint8_t *>(cv);
    for (int b0 = tid; b0 < total; b0 += kF8Unroll * kThreads) {
        float t0[kF8Unroll], gv[kF8Unroll];
#pragma unroll
        for (int u = 0; u < kF8Unroll; ++u) {
            const int idx = b0 + u * kThreads;
            t0[u] = gv[u] = 0.f;
            if (idx < total) {
                const int j = idx / kF8Cols, lr = clist[j];
                if (flg[lr] & 1) {
                    const F8Elem e = f8_elem(a, r0 + lr, idx - j * kF8Cols);
                    t0[u] = *e.th;
                    gv[u] = *e.g;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kF8Unroll; ++u) {
            const int idx = b0 + u * kThreads;
            if (idx >= total) continue;
            const int j = idx / kF8Cols, c = idx - j * kF8Cols, lr = clist[j];
            const int fl = flg[lr];
            float m = f8_dec(wm[lr * kF8Row + c]) * s_old[0][c], v = f8_dec(wvb[lr * kF8Row + c]) * s_old[1][c];
            const F8Elem e = f8_elem(a, r0 + lr, c);
            const float t1 = f8_apply(a, e, fl & 1, fl & 2, fac[lr], t0[u], gv[u], m, v);
            if (fl & 1) __stcs(e.th, t1);
            wm[lr * kF8Row + c] = (uint8_t)f8_rn(m * s_inv[0][c]);
            wvb[lr * kF8Row + c] = (uint8_t)f8_sr(v * s_inv[1][c], f8_rnd(a, r0 + lr, c));
        }
    }
    // the kept rows, re-encoded in the columns whose scale moved
    if (s_moved) {
        for (int idx = tid; idx < nrow * kF8Cols; idx += kThreads) {
            const int lr = idx / kF8Cols, c = idx - lr * kF8Cols;
            if (flg[lr]) continue;
            if (s_new[0][c] != s_old[0][c])
                wm[lr * kF8Row + c] = (uint8_t)f8_rn(f8_dec(wm[lr * kF8Row + c]) * s_old[0][c] * s_inv[0][c]);
            if (s_new[1][c] != s_old[1][c])
                wvb[lr * kF8Row + c] = (uint8_t)f8_rn_floor(f8_dec(wvb[lr * kF8Row + c]) * s_old[1][c] * s_inv[1][c]);
        }
    }
    if (tid < nrow && vis) {                  // the row's own step count (Sec. 3.2)
        uint32_t *tw = reinterpret_cast<uint32_t *>(cm) + tid * (kF8Row / 4) + kF8TWord;
        *tw = *tw + 1u;
    }
    __syncthreads();
    // write back the rows that changed: all of them when a scale moved
    uint4 *om4 = reinterpret_cast<uint4 *>(static_cast<char *>(a.m) + r0 * kF8Row);
    uint4 *ov4 = reinterpret_cast<uint4 *>(static_cast<char *>(a.v) + r0 * kF8Row);
    const bool all = s_moved != 0;
    for (int q = tid; q < nrow * (kF8Row / 16); q += kThreads) {
        if (!all && !flg[q / (kF8Row / 16)]) continue;
        __stcs(om4 + q, cm[q]);
        __stcs(ov4 + q, cv[q]);
    }
}

// ------------------------------------------------------ export / import

__global__ void export_fp8_kernel(const uint8_t *__restrict__ m, const uint8_t *__restrict__ v,
                                  const float *__restrict__ msc, const float *__restrict__ vsc, int32_t n,
                                  float *__restrict__ m_out, float *__restrict__ v_out, uint32_t *__restrict__ t_out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * kF8Cols) return;
    const int64_t r = idx / kF8Cols;
    const int c = (int)(idx - r * kF8Cols);
    const int64_t sb = (r / kF8Tile) * 64 + c;
    if (m_out) m_out[idx] = f8_dec(m[r * kF8Row + c]) * msc[sb];
    if (v_out) v_out[idx] = f8_dec(v[r * kF8Row + c]) * vsc[sb];
    if (t_out && c == 0) t_out[r] = reinterpret_cast<const uint32_t *>(m + r * kF8Row)[kF8TWord];
}

// One CTA per block: the column maxima of the imported values, the scales,
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
        const int c = q % kF8Cols;
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
        const int lr = q / kF8Cols, c = q - lr * kF8Cols;
        if (m_in) m[(r0 + lr) * kF8Row + c] = (uint8_t)f8_rn(m_in[e0 + q] * s_inv[0][c]);
        if (v_in) v[(r0 + lr) * kF8Row + c] = (uint8_t)f8_rn_floor(v_in[e0 + q] * s_inv[1][c]);
    }
    if (t_in && tid < nrow) reinterpret_cast<uint32_t *>(m + (r0 + tid) * kF8Row)[kF8TWord] = t_in[r0 + tid];
}

// ------------------------------------------------------------- re-index
// One CTA per output block.  Output row j takes the state of old row
// src[j] (src[j] < 0 or reset[j]: zero moments and t = 0), decoded with the
// old row's block scales and re-encoded under the output block's new
// scales (both moments to nearest, a positive v never to zero).  An
// out-of-range source is not read: the row is zeroed and the error word set.
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
    const unsigned grid = (unsigned)((a.n_rows + kF8Tile - 1) / kF8Tile);
    k<<<grid, kThreads, 0, s>>>(b, vis_src);
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
