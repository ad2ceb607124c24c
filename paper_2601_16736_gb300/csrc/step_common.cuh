// Device pieces shared by the step kernels (step_kernels.cu) and the
// extended step (step_ext.cu): load/store helpers, the moment storage
// formats State<kPrec>, and the per-row work items of a visible row and
// of an invisible StSS-sampled row.  Every function is inline and file-local
// to the translation unit that includes it.
#pragma once

#include <algorithm>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float4 ldg4_stream(const float *p)
{
    return __ldcs(reinterpret_cast<const float4 *>(p));
}
// results are not read again in this step: store them evict-first
__device__ __forceinline__ void st4(float *p, float4 x) { __stcs(reinterpret_cast<float4 *>(p), x); }

__device__ __forceinline__ void unpack_bf16x2(uint32_t u, float &x, float &y)
{
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
    x = f.x;
    y = f.y;
}
__device__ __forceinline__ uint32_t pack_bf16x2(float x, float y)
{
    const __nv_bfloat162 p = __floats2bfloat162_rn(x, y);
    return *reinterpret_cast<const uint32_t *>(&p);
}

// MurmurHash3's 32-bit finaliser (Appleby, public domain): the random bits of
// stochastic rounding, a function of (seed, iteration, row, column) only.
__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// FP32 -> BF16 bits rounded stochastically: add 16 random bits below the kept
// mantissa and truncate (rounds up with probability equal to the discarded
// fraction, so the rounding is unbiased).  Inf / NaN round to nearest.
__device__ __forceinline__ uint32_t bf16_bits_sr(float x, uint32_t rnd16)
{
    const uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) == 0x7f800000u) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return (u + (rnd16 & 0xffffu)) >> 16;
}
__device__ __forceinline__ uint32_t pack_bf16x2_sr(float x, float y, uint32_t h)
{
    return bf16_bits_sr(x, h) | (bf16_bits_sr(y, h >> 16) << 16);
}

// kW values as BF16 at p, rounded stochastically: one counter hash of (seed,
// iteration, row, first column) per 4 values, 16 random bits per value.
// col0 is the state slot of x[0], so every stored value draws its own bits.
template <int kW>
__device__ __forceinline__ void store_bf16_sr(char *p, const float *x, const StepArgs &a, int32_t r, int col0)
{
    uint32_t w[kW / 2];
#pragma unroll
    for (int q = 0; q < kW / 2; q += 2) {
        const uint32_t h = fmix32((uint32_t)r * 0x9e3779b1u ^ (uint32_t)(col0 + 2 * q) * 0x85ebca77u ^
                                  (uint32_t)a.k_ctr * 0xc2b2ae3du ^ (uint32_t)a.seed);
        const uint32_t h2 = fmix32(h ^ 0x27d4eb2fu);
        w[q] = pack_bf16x2_sr(x[2 * q], x[2 * q + 1], h);
        w[q + 1] = pack_bf16x2_sr(x[2 * q + 2], x[2 * q + 3], h2);
    }
    if (kW == 4)
        __stcs(reinterpret_cast<uint2 *>(p), make_uint2(w[0], w[1]));
    else
        __stcs(reinterpret_cast<uint4 *>(p), make_uint4(w[0], w[1], w[kW > 4 ? 2 : 0], w[kW > 4 ? 3 : 0]));
}

// ------------------------------------------------------------ state formats
// A small chunk (small item c = 12, 13, 14): 4 moments of m and of v as FP32,
// plus t where the format keeps it in chunk 14.
struct Chunk {
    float4 m, v;
    uint32_t t;
};

// Every format provides
//   kRowBytes, kTByte   row size and byte offset of t in the m row
//   kTInSh              t is carried by SH item 0 (else by small chunk 14)
//   load_sh / store_sh  the moments of SH columns kW*i .. kW*i+kW-1 (+ t)
//   load_small / store_small  small chunk c in 12..14 (rotation; xyz +
//                       scale0; scale1, scale2, opacity, [t or unused])
template <int kPrec>
struct State;

template <>
struct State<GS_MOM_FP32> {
    static constexpr int kRowBytes = kRowBytesF32, kTByte = kTByteF32;
    static constexpr bool kTInSh = false;
    static __device__ __forceinline__ float *row(void *base, int32_t r)
    {
        return static_cast<float *>(base) + (size_t)r * kSlots;
    }
    template <int kW>
    static __device__ __forceinline__ void load_sh(const StepArgs &a, int32_t r, int i, float *m, float *v, uint32_t &)
    {
#pragma unroll
        for (int q = 0; q < kW / 4; ++q) {
            const float4 x = ld4(row(a.m, r) + kW * i + 4 * q), y = ld4(row(a.v, r) + kW * i + 4 * q);
            m[4 * q] = x.x; m[4 * q + 1] = x.y; m[4 * q + 2] = x.z; m[4 * q + 3] = x.w;
            v[4 * q] = y.x; v[4 * q + 1] = y.y; v[4 * q + 2] = y.z; v[4 * q + 3] = y.w;
        }
    }
    template <int kW>
    static __device__ __forceinline__ void store_sh(const StepArgs &a, int32_t r, int i, const float *m,
                                                    const float *v, uint32_t)
    {
#pragma unroll
        for (int q = 0; q < kW / 4; ++q) {
            st4(row(a.m, r) + kW * i + 4 * q, make_float4(m[4 * q], m[4 * q + 1], m[4 * q + 2], m[4 * q + 3]));
            st4(row(a.v, r) + kW * i + 4 * q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
        }
    }
    static __device__ __forceinline__ Chunk load_small(const StepArgs &a, int32_t r, int c)
    {
        Chunk k;
        k.m = ld4(row(a.m, r) + 4 * c);
        k.v = ld4(row(a.v, r) + 4 * c);
        k.t = __float_as_uint(k.m.w);           // slot 59 of m (meaningful for c == 14)
        return k;
    }
    static __device__ __forceinline__ void store_small(const StepArgs &a, int32_t r, int c, Chunk k)
    {
        if (c == 14) k.m.w = __uint_as_float(k.t);
        st4(row(a.m, r) + 4 * c, k.m);
        st4(row(a.v, r) + 4 * c, k.v);
    }
};

// kW BF16 values at p (kW = 4: one uint2, 8: one uint4) <-> FP32
template <int kW>
__device__ __forceinline__ void load_bf16(const char *p, float *x)
{
    if (kW == 4) {
        const uint2 u = *reinterpret_cast<const uint2 *>(p);
        unpack_bf16x2(u.x, x[0], x[1]);
        unpack_bf16x2(u.y, x[2], x[3]);
    } else {
        const uint4 u = *reinterpret_cast<const uint4 *>(p);
        unpack_bf16x2(u.x, x[0], x[1]);
        unpack_bf16x2(u.y, x[2], x[3]);
        unpack_bf16x2(u.z, x[kW > 4 ? 4 : 0], x[kW > 4 ? 5 : 0]);
        unpack_bf16x2(u.w, x[kW > 4 ? 6 : 0], x[kW > 4 ? 7 : 0]);
    }
}
template <int kW>
__device__ __forceinline__ void store_bf16_rn(char *p, const float *x)
{
    if (kW == 4)
        __stcs(reinterpret_cast<uint2 *>(p), make_uint2(pack_bf16x2(x[0], x[1]), pack_bf16x2(x[2], x[3])));
    else
        __stcs(reinterpret_cast<uint4 *>(p),
               make_uint4(pack_bf16x2(x[0], x[1]), pack_bf16x2(x[2], x[3]), pack_bf16x2(x[kW > 4 ? 4 : 0], x[kW > 4 ? 5 : 0]),
                          pack_bf16x2(x[kW > 4 ? 6 : 0], x[kW > 4 ? 7 : 0])));
}

// BF16 rows of 64 slots (128 B): SH column j at byte 2j; small chunk c at byte
// 8c; t = uint32 at byte 120, loaded and stored with chunk 14 as one 16-B
// access (slots 56-63).  m is rounded to nearest; v is rounded
// stochastically (its ~0.1 % per-step EMA increment is below BF16's
// resolution, and round-to-nearest would freeze it).
template <>
struct State<GS_MOM_BF16> {
    static constexpr int kRowBytes = kRowBytesBf16, kTByte = kTByteBf16;
    static constexpr bool kTInSh = false;
    static __device__ __forceinline__ char *row(void *base, int32_t r)
    {
        return static_cast<char *>(base) + (size_t)r * kRowBytes;
    }
    template <int kW>
    static __device__ __forceinline__ void load_sh(const StepArgs &a, int32_t r, int i, float *m, float *v, uint32_t &)
    {
        load_bf16<kW>(row(a.m, r) + 2 * kW * i, m);
        load_bf16<kW>(row(a.v, r) + 2 * kW * i, v);
    }
    template <int kW>
    static __device__ __forceinline__ void store_sh(const StepArgs &a, int32_t r, int i, const float *m,
                                                    const float *v, uint32_t)
    {
        store_bf16_rn<kW>(row(a.m, r) + 2 * kW * i, m);
        store_bf16_sr<kW>(row(a.v, r) + 2 * kW * i, v, a, r, kW * i);
    }
    static __device__ __forceinline__ Chunk load_small(const StepArgs &a, int32_t r, int c)
    {
        Chunk k;
        float x[4];
        if (c < 14) {
            load_bf16<4>(row(a.m, r) + 8 * c, x);
            k.t = 0;
        } else {
            const uint4 um = *reinterpret_cast<const uint4 *>(row(a.m, r) + 112);
            unpack_bf16x2(um.x, x[0], x[1]);
            unpack_bf16x2(um.y, x[2], x[3]);
            k.t = um.z;
        }
        k.m = make_float4(x[0], x[1], x[2], x[3]);
        load_bf16<4>(row(a.v, r) + 8 * c, x);
        k.v = make_float4(x[0], x[1], x[2], x[3]);
        return k;
    }
    static __device__ __forceinline__ void store_small(const StepArgs &a, int32_t r, int c, const Chunk &k)
    {
        if (c < 14) {
            __stcs(reinterpret_cast<uint2 *>(row(a.m, r) + 8 * c),
                   make_uint2(pack_bf16x2(k.m.x, k.m.y), pack_bf16x2(k.m.z, k.m.w)));
        } else {
            __stcs(reinterpret_cast<uint4 *>(row(a.m, r) + 112),
                   make_uint4(pack_bf16x2(k.m.x, k.m.y), pack_bf16x2(k.m.z, k.m.w), k.t, 0u));
        }
        const float vv[4] = {k.v.x, k.v.y, k.v.z, k.v.w};
        store_bf16_sr<4>(row(a.v, r) + 8 * c, vv, a, r, 4 * c);
    }
};

// BF16 hybrid rows (160 B): FP32 part of 16 slots — [0-2] SH DC, [3] t,
// [4-7] rotation, [8-10] xyz, [11-13] scale, [14] opacity — then the 48 SH
// columns as BF16 at byte 64 (slots 0-2 unused).  SH item 0 takes the DC
// moments and t from the FP32 part.  m is rounded to nearest; v is rounded
// stochastically: its ~0.1 % per-step EMA increment is below BF16 resolution,
// and round-to-nearest would freeze it.
template <>
struct State<GS_MOM_BF16_HYBRID> {
    static constexpr int kRowBytes = kRowBytesHyb, kTByte = kTByteHyb;
    static constexpr bool kTInSh = true;
    static __device__ __forceinline__ char *row(void *base, int32_t r)
    {
        return static_cast<char *>(base) + (size_t)r * kRowBytes;
    }
    template <int kW>
    static __device__ __forceinline__ void load_sh(const StepArgs &a, int32_t r, int i, float *m, float *v,
                                                   uint32_t &t)
    {
        load_bf16<kW>(row(a.m, r) + kHybShByte + 2 * kW * i, m);
        load_bf16<kW>(row(a.v, r) + kHybShByte + 2 * kW * i, v);
        if (i == 0) {
            const float4 fm = *reinterpret_cast<const float4 *>(row(a.m, r));
            const float4 fv = *reinterpret_cast<const float4 *>(row(a.v, r));
            m[0] = fm.x; m[1] = fm.y; m[2] = fm.z;
            v[0] = fv.x; v[1] = fv.y; v[2] = fv.z;
            t = __float_as_uint(fm.w);
        }
    }
    template <int kW>
    static __device__ __forceinline__ void store_sh(const StepArgs &a, int32_t r, int i, const float *m,
                                                    const float *v, uint32_t t)
    {
        float mm[kW], vv[kW];
#pragma unroll
        for (int e = 0; e < kW; ++e) {
            mm[e] = m[e];
            vv[e] = v[e];
        }
        if (i == 0) {
            st4(reinterpret_cast<float *>(row(a.m, r)), make_float4(m[0], m[1], m[2], __uint_as_float(t)));
            st4(reinterpret_cast<float *>(row(a.v, r)), make_float4(v[0], v[1], v[2], 0.f));
            mm[0] = mm[1] = mm[2] = vv[0] = vv[1] = vv[2] = 0.f;   // BF16 DC slots are unused
        }
        store_bf16_rn<kW>(row(a.m, r) + kHybShByte + 2 * kW * i, mm);
        store_bf16_sr<kW>(row(a.v, r) + kHybShByte + 2 * kW * i, vv, a, r, kW * i);
    }
    static __device__ __forceinline__ Chunk load_small(const StepArgs &a, int32_t r, int c)
    {
        Chunk k;
        k.m = *reinterpret_cast<const float4 *>(row(a.m, r) + 16 * (c - 11));
        k.v = *reinterpret_cast<const float4 *>(row(a.v, r) + 16 * (c - 11));
        k.t = 0;
        return k;
    }
    static __device__ __forceinline__ void store_small(const StepArgs &a, int32_t r, int c, const Chunk &k)
    {
        st4(reinterpret_cast<float *>(row(a.m, r) + 16 * (c - 11)), k.m);
        st4(reinterpret_cast<float *>(row(a.v, r) + 16 * (c - 11)), k.v);
    }
};

// ------------------------------------------------------- FP16 with block exponents
// Each work item's group of columns shares one exponent byte: the largest
// biased FP32 exponent e among the group's values.  Values are stored as
// FP16 of x * 2^(141 - e), which puts the largest magnitude in [2^14, 2^15);
// every value within 2^29 of it is an FP16 normal with a 10-bit mantissa.
// e < 15 (all magnitudes below 2^-112) stores zeros and e = 0.

// Packed FP16 words: value 2k in the low half of word k, value 2k+1 in the high half.

// Two values scaled by s, to nearest.
__device__ __forceinline__ uint32_t h2_rn(float x, float y)
{
    const __half2 h = __floats2half2_rn(x, y);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Two second-moment values rounded stochastically: each is dithered by a
// uniform offset of +-1/2 FP16 ulp (13 random bits, centred, added below the
// 10 mantissa bits FP16 keeps), then both are rounded to nearest by one
// conversion.  For FP16 normals (values within 2^29 of the group's largest)
// that rounds up with probability equal to the discarded fraction; in FP16's
// subnormal range the dither is below the quantum and values round to
// nearest.  A positive value never becomes zero: v spans the square of m's
// range, so a column with a gradient ~10^6 below its group's largest would
// otherwise keep m != 0 beside v = 0, and a step that reuses the stored
// moments (AIU) would divide by eps; it keeps the smallest subnormal
// instead.  Zero, Inf and NaN pass unchanged.
__device__ __forceinline__ uint32_t h2_sr(float x, float y, uint32_t rnd)
{
    uint32_t ux = __float_as_uint(x), uy = __float_as_uint(y);
    const uint32_t ex = ux & 0x7f800000u, ey = uy & 0x7f800000u;
    ux += (ex != 0u && ex != 0x7f800000u) ? (rnd & 0x1fffu) - 0x1000u : 0u;
    uy += (ey != 0u && ey != 0x7f800000u) ? ((rnd >> 16) & 0x1fffu) - 0x1000u : 0u;
    uint32_t w = h2_rn(__uint_as_float(ux), __uint_as_float(uy));
    if ((w & 0x7fffu) == 0u && x > 0.f) w |= 1u;
    if ((w & 0x7fff0000u) == 0u && y > 0.f) w |= 1u << 16;
    return w;
}

// n values -> (n + 1) / 2 packed words and the group exponent; m to nearest,
// v stochastically.  The random bits: one hash of (seed, iteration, row,
// first column) per group, times a distinct odd constant for each pair of
// values (multiplying by an odd constant permutes the low bits, so each
// pair's two 13-bit dither fields stay uniform and each value's rounding
// unbiased; one hash instead of one per pair is 2 % of the step at 3 M rows).
// An odd n leaves the last word's high half zero.
template <int n>
__device__ __forceinline__ uint32_t encode_rn_w(const float *x, uint32_t *w)
{
    const uint32_t e = group_exponent(x, n);
    const float s = e ? enc_scale(e) : 0.f;
#pragma unroll
    for (int q = 0; q < n; q += 2) w[q / 2] = h2_rn(x[q] * s, q + 1 < n ? x[q + 1] * s : 0.f);
    return e;
}
template <int n>
__device__ __forceinline__ uint32_t encode_sr_w(const float *x, uint32_t *w, const StepArgs &a, int32_t r, int col0)
{
    const uint32_t e = group_exponent(x, n);
    const float s = e ? enc_scale(e) : 0.f;
    const uint32_t h = fmix32((uint32_t)r * 0x9e3779b1u ^ (uint32_t)col0 * 0x85ebca77u ^
                               (uint32_t)a.k_ctr * 0xc2b2ae3du ^ (uint32_t)a.seed ^ 0x165667b1u);
    constexpr uint32_t kOdd[4] = {1u, 0x9e3779b1u, 0x85ebca77u, 0xc2b2ae3du};
    static_assert(n <= 8, "one odd constant per pair of a group");
#pragma unroll
    for (int q = 0; q < n; q += 2) {
        w[q / 2] = h2_sr(x[q] * s, q + 1 < n ? x[q + 1] * s : 0.f, h * kOdd[q / 2]);
    }
    return e;
}
// n values from packed words, times the group's decode scale d.
template <int n>
__device__ __forceinline__ void decode_w(const uint32_t *w, float d, float *x)
{
#pragma unroll
    for (int q = 0; q < n; q += 2) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[q / 2]));
        x[q] = f.x * d;
        if (q + 1 < n) x[q + 1] = f.y * d;
    }
}

template <>
struct State<GS_MOM_FP16_BLOCK> {
    static constexpr int kRowBytes = kRowBytesF16B, kTByte = kTByteF16B;
    static constexpr bool kTInSh = false;
    static __device__ __forceinline__ char *row(void *base, int32_t r)
    {
        return static_cast<char *>(base) + (size_t)r * kRowBytes;
    }
    template <int kW>
    static __device__ __forceinline__ void load_sh(const StepArgs &a, int32_t r, int i, float *m, float *v, uint32_t &)
    {
        static_assert(kW == 8, "FP16 block items cover 8 SH columns");
        const char *mr = row(a.m, r), *vr = row(a.v, r);
        const uint4 um = *reinterpret_cast<const uint4 *>(mr + 16 * i), uv = *reinterpret_cast<const uint4 *>(vr + 16 * i);
        const uint32_t wm[4] = {um.x, um.y, um.z, um.w}, wv[4] = {uv.x, uv.y, uv.z, uv.w};
        decode_w<8>(wm, dec_scale((uint8_t)mr[kF16BExp + i]), m);
        decode_w<8>(wv, dec_scale((uint8_t)vr[kF16BExp + i]), v);
    }
    template <int kW>
    static __device__ __forceinline__ void store_sh(const StepArgs &a, int32_t r, int i, const float *m,
                                                    const float *v, uint32_t)
    {
        char *mr = row(a.m, r), *vr = row(a.v, r);
        uint32_t wm[4], wv[4];
        const uint32_t em = encode_rn_w<8>(m, wm), ev = encode_sr_w<8>(v, wv, a, r, 11 + 8 * i);
        __stcs(reinterpret_cast<uint4 *>(mr + 16 * i), make_uint4(wm[0], wm[1], wm[2], wm[3]));
        __stcs(reinterpret_cast<uint4 *>(vr + 16 * i), make_uint4(wv[0], wv[1], wv[2], wv[3]));
        mr[kF16BExp + i] = (char)em;
        vr[kF16BExp + i] = (char)ev;
    }
};

// The small columns of an FP16-block row in two items: c = 12 rotation (4
// values at kF16BRot, exponent 6), c = 13 xyz + scale + opacity (7 values at
// kF16BXso, exponent 7) with the step count t (uint16, saturating) in the
// high half of the fourth word.  The visible update as small_item; RSR
// scales the moments afterwards.  kX: item 13 subtracts the row's noise nz
// from xyz and returns whether the row is active after the step.
template <bool kX>
__device__ __forceinline__ bool small_item_f16b(const StepArgs &a, const int32_t row, const int c, const bool sampled,
                                                const float2 f, const float3 nz)
{
    using S = State<GS_MOM_FP16_BLOCK>;
    char *mr = S::row(a.m, row), *vr = S::row(a.v, row);
    const size_t r = (size_t)row;
    if (c == 12) {
        const uint2 um = *reinterpret_cast<const uint2 *>(mr + kF16BRot), uv = *reinterpret_cast<const uint2 *>(vr + kF16BRot);
        const uint32_t wm[2] = {um.x, um.y}, wv[2] = {uv.x, uv.y};
        float m[4], v[4];
        decode_w<4>(wm, dec_scale((uint8_t)mr[kF16BExp + 6]), m);
        decode_w<4>(wv, dec_scale((uint8_t)vr[kF16BExp + 6]), v);
        float *pt = a.a_rot + r * 4;
        float4 th = ld4(pt);
        const float4 g = ldg4_stream(a.g_rot + r * 4);
        const float l = a.lr[2];
        th.x = step_element(th.x, g.x, m[0], v[0], f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
        th.y = step_element(th.y, g.y, m[1], v[1], f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
        th.z = step_element(th.z, g.z, m[2], v[2], f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
        th.w = step_element(th.w, g.w, m[3], v[3], f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
        st4(pt, th);
        if (sampled) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                m[q] *= a.alpha1;
                v[q] *= a.alpha2;
            }
        }
        uint32_t hm[2], hv[2];
        const uint32_t em = encode_rn_w<4>(m, hm), ev = encode_sr_w<4>(v, hv, a, row, 6);
        __stcs(reinterpret_cast<uint2 *>(mr + kF16BRot), make_uint2(hm[0], hm[1]));
        __stcs(reinterpret_cast<uint2 *>(vr + kF16BRot), make_uint2(hv[0], hv[1]));
        mr[kF16BExp + 6] = (char)em;
        vr[kF16BExp + 6] = (char)ev;
        return false;
    } else {
        const uint4 um = *reinterpret_cast<const uint4 *>(mr + kF16BXso), uv = *reinterpret_cast<const uint4 *>(vr + kF16BXso);
        const uint32_t wm[4] = {um.x, um.y, um.z, um.w & 0xffffu}, wv[4] = {uv.x, uv.y, uv.z, uv.w};
        float m[7], v[7];
        decode_w<7>(wm, dec_scale((uint8_t)mr[kF16BExp + 7]), m);
        decode_w<7>(wv, dec_scale((uint8_t)vr[kF16BExp + 7]), v);
        uint32_t t = um.w >> 16;
        float *px = a.a_xyz + r * 3, *ps = a.a_scale + r * 3, *po = a.a_op + r;
        float x0 = px[0], x1 = px[1], x2 = px[2], s0 = ps[0], s1 = ps[1], s2 = ps[2], op = *po;
        const float *gx = a.g_xyz + r * 3, *gs = a.g_scale + r * 3;
        const float g0 = __ldcs(gx), g1 = __ldcs(gx + 1), g2 = __ldcs(gx + 2);
        const float gs0 = __ldcs(gs), gs1 = __ldcs(gs + 1), gs2 = __ldcs(gs + 2), go = __ldcs(a.g_op + r);
        const bool ds = a.dar_s != 0, dop = a.dar_o != 0;
        // regulariser derivatives at the old values (App. Eqs. scale, opacity)
        const float r0s = ds ? expf(s0) : 0.f, r1s = ds ? expf(s1) : 0.f, r2s = ds ? expf(s2) : 0.f;
        const float rop = dop ? dsigmoid(op) : 0.f;
        x0 = step_element(x0, g0, m[0], v[0], f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
        x1 = step_element(x1, g1, m[1], v[1], f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
        x2 = step_element(x2, g2, m[2], v[2], f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
        s0 = step_element(s0, gs0, m[3], v[3], f.x, f.y, a, a.lr[1], ds, r0s, a.lam_s, a.clip_s);
        s1 = step_element(s1, gs1, m[4], v[4], f.x, f.y, a, a.lr[1], ds, r1s, a.lam_s, a.clip_s);
        s2 = step_element(s2, gs2, m[5], v[5], f.x, f.y, a, a.lr[1], ds, r2s, a.lam_s, a.clip_s);
        op = step_element(op, go, m[6], v[6], f.x, f.y, a, a.lr[3], dop, rop, a.lam_o, a.clip_o);
        if constexpr (kX) {
            x0 -= nz.x; x1 -= nz.y; x2 -= nz.z;
        }
        __stcs(px, x0); __stcs(px + 1, x1); __stcs(px + 2, x2);
        __stcs(ps, s0); __stcs(ps + 1, s1); __stcs(ps + 2, s2);
        __stcs(po, op);
        t = min(t + 1u, 65535u);                    // the row's own step count (Sec. 3.2)
        if (sampled) {
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                m[q] *= a.alpha1;
                v[q] *= a.alpha2;
            }
        }
        uint32_t hm[4], hv[4];
        const uint32_t em = encode_rn_w<7>(m, hm), ev = encode_sr_w<7>(v, hv, a, row, 0);
        __stcs(reinterpret_cast<uint4 *>(mr + kF16BXso), make_uint4(hm[0], hm[1], hm[2], hm[3] | t << 16));
        __stcs(reinterpret_cast<uint4 *>(vr + kF16BXso), make_uint4(hv[0], hv[1], hv[2], hv[3]));
        mr[kF16BExp + 7] = (char)em;
        vr[kF16BExp + 7] = (char)ev;
        return kX && op > a.tau_act;
    }
}

// RSR of one small item of an invisible FP16-block row (moments only, t kept).
__device__ __forceinline__ void rsr_small_f16b(const StepArgs &a, const int32_t row, const int c)
{
    using S = State<GS_MOM_FP16_BLOCK>;
    char *mr = S::row(a.m, row), *vr = S::row(a.v, row);
    if (c == 12) {
        const uint2 um = *reinterpret_cast<const uint2 *>(mr + kF16BRot), uv = *reinterpret_cast<const uint2 *>(vr + kF16BRot);
        const uint32_t wm[2] = {um.x, um.y}, wv[2] = {uv.x, uv.y};
        float m[4], v[4];
        decode_w<4>(wm, dec_scale((uint8_t)mr[kF16BExp + 6]) * a.alpha1, m);
        decode_w<4>(wv, dec_scale((uint8_t)vr[kF16BExp + 6]) * a.alpha2, v);
        uint32_t hm[2], hv[2];
        const uint32_t em = encode_rn_w<4>(m, hm), ev = encode_sr_w<4>(v, hv, a, row, 6);
        __stcs(reinterpret_cast<uint2 *>(mr + kF16BRot), make_uint2(hm[0], hm[1]));
        __stcs(reinterpret_cast<uint2 *>(vr + kF16BRot), make_uint2(hv[0], hv[1]));
        mr[kF16BExp + 6] = (char)em;
        vr[kF16BExp + 6] = (char)ev;
    } else {
        const uint4 um = *reinterpret_cast<const uint4 *>(mr + kF16BXso), uv = *reinterpret_cast<const uint4 *>(vr + kF16BXso);
        const uint32_t wm[4] = {um.x, um.y, um.z, um.w & 0xffffu}, wv[4] = {uv.x, uv.y, uv.z, uv.w};
        float m[7], v[7];
        decode_w<7>(wm, dec_scale((uint8_t)mr[kF16BExp + 7]) * a.alpha1, m);
        decode_w<7>(wv, dec_scale((uint8_t)vr[kF16BExp + 7]) * a.alpha2, v);
        const uint32_t t = um.w >> 16;
        uint32_t hm[4], hv[4];
        const uint32_t em = encode_rn_w<7>(m, hm), ev = encode_sr_w<7>(v, hv, a, row, 0);
        __stcs(reinterpret_cast<uint4 *>(mr + kF16BXso), make_uint4(hm[0], hm[1], hm[2], hm[3] | t << 16));
        __stcs(reinterpret_cast<uint4 *>(vr + kF16BXso), make_uint4(hv[0], hv[1], hv[2], hv[3]));
        mr[kF16BExp + 7] = (char)em;
        vr[kF16BExp + 7] = (char)ev;
    }
}

// Ask L2 to fetch the contiguous parts a visible row's items will read (SH
// attributes and gradients, m and v rows; cp.async.bulk.prefetch.L2), as
// soon as the row is known to be visible.  Worth it for sparse tiles: their
// rows are scattered, and the items' later loads then hit L2.  Dense tiles
// already stream well and only pay for the extra requests, so callers skip
// the hint when most of the tile is visible.
template <int kRowBytes>
__device__ __forceinline__ void prefetch_row_l2(const StepArgs &a, int32_t row)
{
    const size_t r = (size_t)row;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], 192;" ::"l"(a.a_sh + r * 48) : "memory");
    if (!a.g_host) asm volatile("cp.async.bulk.prefetch.L2.global [%0], 192;" ::"l"(a.g_sh + r * 48) : "memory");
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_cast<const char *>(a.m) + r * kRowBytes),
                 "n"(kRowBytes) : "memory");
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_cast<const char *>(a.v) + r * kRowBytes),
                 "n"(kRowBytes) : "memory");
}

// Ask L2 for the visibility inputs (means or mask bytes) of the tile one wave
// of resident CTAs ahead: the tile that starts when a slot frees, whose
// phase A then finds them on chip instead of waiting a DRAM round trip.  A
// hint only; nothing waits for it.  Whole tiles only, 16-B aligned sources.
template <int kTile>
__device__ __forceinline__ void prefetch_tile_ahead(const StepArgs &a, const int vis_src)
{
    static_assert((kTile * 12) % 16 == 0 && kTile % 16 == 0, "bulk prefetch sizes are multiples of 16 B");
    if (threadIdx.x != 0 || a.tile_ahead <= 0) return;
    const int64_t q = ((int64_t)blockIdx.x + a.tile_ahead) * kTile;
    if (q + kTile > (int64_t)a.n_rows) return;
    if (vis_src == kVisCamera && ((uintptr_t)a.a_xyz & 15u) == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.a_xyz + q * 3), "n"(kTile * 12) : "memory");
    else if (vis_src == kVisMask && ((uintptr_t)a.mask_in & 15u) == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.mask_in + q), "n"(kTile) : "memory");
}

// CTAs of kernel `fn` (kThreads threads, static shared memory only) resident
// at once on the current device, cached per device in `cache`; 0 if the
// query fails (the caller then launches without the look-ahead).
inline int resident_ctas(const void *fn, int *cache)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    int &c = cache[dev & 63];
    if (!c) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        c = per_sm * sms;
    }
    return c;
}

// Prefetch when at most 60 % of the tile's rows are visible.
// Beside the means: ask L2 for what phase A of the tile one wave ahead reads
// for its rows, so that its loads find them on chip: the opacity logits when
// counting N_a or drawing noise, and the rotations and log-scales for noise.
// A hint only; whole tiles, 16-B aligned sources.
template <int kTile>
__device__ __forceinline__ void prefetch_tile_ahead_x(const StepArgs &a)
{
    if (threadIdx.x != 0 || a.tile_ahead <= 0 || !(a.n_active || a.noise)) return;
    const int64_t q = ((int64_t)blockIdx.x + a.tile_ahead) * kTile;
    if (q + kTile > (int64_t)a.n_rows) return;
    if (((uintptr_t)a.a_op & 15u) == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.a_op + q), "n"(kTile * 4) : "memory");
    if (a.noise) {
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.a_rot + q * 4), "n"(kTile * 16) : "memory");
        if (((uintptr_t)a.a_scale & 15u) == 0)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.a_scale + q * 3), "n"(kTile * 12)
                         : "memory");
    }
}

template <int kTile>
__device__ __forceinline__ bool sparse_tile(int nv) { return 5 * nv <= 3 * kTile; }

// Small items per row: rotation; xyz + scale0; scale1 + scale2 + opacity,
// except FP16-block rows (rotation; xyz + scale + opacity).
template <int kPrec>
constexpr int kSmallItems = kPrec == GS_MOM_FP16_BLOCK ? 2 : 3;

// ---------------------------------------------------------------- the items

// SH item i of a visible row: SH columns kW*i .. kW*i+kW-1 (0-2 are the DC
// term, learning rate lr[4]; the rest lr[5]); no regulariser.
template <int kPrec, int kW>
__device__ __forceinline__ void sh_item(const StepArgs &a, const int32_t row, const int i, const bool sampled,
                                        const float2 f)
{
    using S = State<kPrec>;
    if constexpr (kPrec == GS_MOM_FP16_BLOCK) {
        // Register-lean order, same arithmetic as step_element: the moments
        // and the directions u first (gradients then dead), m and v encoded
        // and stored, and only then the attributes loaded and updated.  24
        // values live at most instead of 32.
        float m[kW], v[kW], u[kW];
        uint32_t t = 0;
        S::template load_sh<kW>(a, row, i, m, v, t);
        const size_t off = (size_t)row * 48 + kW * i;
#pragma unroll
        for (int q = 0; q < kW / 4; ++q) {
            const float4 y = ldg4_stream(a.g_sh + off + 4 * q);
            const float gq[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float &mm = m[4 * q + e], &vv = v[4 * q + e];
                mm = fmaf(a.c1, gq[e] - mm, mm);
                vv = fmaf(a.c2, fmaf(gq[e], gq[e], -vv), vv);
                u[4 * q + e] = __fdividef(mm * f.x, fmaf(sqrt_approx(vv), f.y, a.eps));
            }
        }
        if (sampled) {                     // RSR post-scale (Eq. meth::restate)
#pragma unroll
            for (int e = 0; e < kW; ++e) {
                m[e] *= a.alpha1;
                v[e] *= a.alpha2;
            }
        }
        S::template store_sh<kW>(a, row, i, m, v, t);
#pragma unroll
        for (int q = 0; q < kW / 4; ++q) {
            const float4 x = ld4(a.a_sh + off + 4 * q);
            float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
                xs[e] = fmaf(-((i == 0 && 4 * q + e < 3) ? a.lr[4] : a.lr[5]), u[4 * q + e], xs[e]);
            st4(a.a_sh + off + 4 * q, make_float4(xs[0], xs[1], xs[2], xs[3]));
        }
        return;
    }
    float m[kW], v[kW], th[kW], g[kW];
    uint32_t t = 0;
    S::template load_sh<kW>(a, row, i, m, v, t);
    const size_t off = (size_t)row * 48 + kW * i;
#pragma unroll
    for (int q = 0; q < kW / 4; ++q) {
        const float4 x = ld4(a.a_sh + off + 4 * q), y = ldg4_stream(a.g_sh + off + 4 * q);
        th[4 * q] = x.x; th[4 * q + 1] = x.y; th[4 * q + 2] = x.z; th[4 * q + 3] = x.w;
        g[4 * q] = y.x; g[4 * q + 1] = y.y; g[4 * q + 2] = y.z; g[4 * q + 3] = y.w;
    }
#pragma unroll
    for (int e = 0; e < kW; ++e) {
        const float lr = (i == 0 && e < 3) ? a.lr[4] : a.lr[5];
        th[e] = step_element(th[e], g[e], m[e], v[e], f.x, f.y, a, lr, false, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < kW / 4; ++q)
        st4(a.a_sh + off + 4 * q, make_float4(th[4 * q], th[4 * q + 1], th[4 * q + 2], th[4 * q + 3]));
    if (S::kTInSh && i == 0) t += 1u;      // the row's own step count (Sec. 3.2)
    if (sampled) {                         // RSR post-scale (Eq. meth::restate)
#pragma unroll
        for (int e = 0; e < kW; ++e) {
            m[e] *= a.alpha1;
            v[e] *= a.alpha2;
        }
    }
    S::template store_sh<kW>(a, row, i, m, v, t);
}

// gamma ~ N(0, I_3) by the Box-Muller transform (Box & Muller 1958) on
// 24-bit uniforms from two SplitMix64 words (stream tags 2 and 3):
// ua = (w >> 40 + 1) / 2^24 in (0, 1], ub = bits 16..39 / 2^24 in [0, 1).
__device__ __forceinline__ float3 noise_gamma(const StepArgs &a, int32_t row)
{
    const uint64_t h1 = splitmix64_at(a.seed, draw_counter(2, a.k_ctr, row));
    const uint64_t h2 = splitmix64_at(a.seed, draw_counter(3, a.k_ctr, row));
    const float ua1 = (float)((h1 >> 40) + 1ull) * 0x1p-24f, ub1 = (float)((h1 >> 16) & 0xFFFFFFull) * 0x1p-24f;
    const float ua2 = (float)((h2 >> 40) + 1ull) * 0x1p-24f, ub2 = (float)((h2 >> 16) & 0xFFFFFFull) * 0x1p-24f;
    const float r1 = sqrtf(-2.f * logf(ua1)), r2 = sqrtf(-2.f * logf(ua2));
    float s1, c1;
    sincospif(2.f * ub1, &s1, &c1);
    return make_float3(r1 * c1, r1 * s1, r2 * cospif(2.f * ub2));
}

// Position noise of one primitive from its values before this step (App.
// Eq. disentangled_mu): the amount subtracted from mu,
//   eta_Ro * eta_mu * sigmoid(-lambda_mu (o - lambda_t)) * Sigma gamma,
// Sigma = R diag(exp(2 kappa)) R^T, R the rotation of the normalised
// quaternion q = (w, x, y, z).  Sigma gamma is formed as R (s^2 .* (R^T gamma)).
__device__ __forceinline__ float3 noise_term(const StepArgs &a, int32_t row, float4 q, float k0, float k1, float k2,
                                             float tau)
{
    const float o = 1.f / (1.f + expf(-tau));
    const float gate = 1.f / (1.f + expf(a.noise_k * (o - a.noise_t)));
    const float c = a.noise_scale * gate;
    if (c == 0.f) return make_float3(0.f, 0.f, 0.f);
    const float3 g = noise_gamma(a, row);
    const float nrm = fmaxf(sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w), 1e-12f);
    const float w = q.x / nrm, x = q.y / nrm, y = q.z / nrm, z = q.w / nrm;
    const float r00 = 1.f - 2.f * (y * y + z * z), r01 = 2.f * (x * y - w * z), r02 = 2.f * (x * z + w * y);
    const float r10 = 2.f * (x * y + w * z), r11 = 1.f - 2.f * (x * x + z * z), r12 = 2.f * (y * z - w * x);
    const float r20 = 2.f * (x * z - w * y), r21 = 2.f * (y * z + w * x), r22 = 1.f - 2.f * (x * x + y * y);
    const float p0 = (r00 * g.x + r10 * g.y + r20 * g.z) * expf(2.f * k0);
    const float p1 = (r01 * g.x + r11 * g.y + r21 * g.z) * expf(2.f * k1);
    const float p2 = (r02 * g.x + r12 * g.y + r22 * g.z) * expf(2.f * k2);
    return make_float3(c * (r00 * p0 + r01 * p1 + r02 * p2), c * (r10 * p0 + r11 * p1 + r12 * p2),
                       c * (r20 * p0 + r21 * p1 + r22 * p2));
}

// Small item c of a visible row: 12 rotation, 13 xyz + scale0, 14 scale1 +
// scale2 + opacity (+ t where the format keeps it there).  kX (the step with
// the active count and/or noise on visible rows): the xyz item subtracts the
// row's noise nz, and the opacity item returns whether the row is active
// after the step (opacity logit above tau_act); otherwise nz is unused and
// the result false.
template <int kPrec, bool kX = false>
__device__ __forceinline__ bool small_item(const StepArgs &a, const int32_t row, const int c, const bool sampled,
                                           const float2 f, const float3 nz = float3{0.f, 0.f, 0.f})
{
    if constexpr (kPrec == GS_MOM_FP16_BLOCK) {
        return small_item_f16b<kX>(a, row, c, sampled, f, nz);
    } else {
        bool active = false;
        using S = State<kPrec>;
        Chunk k = S::load_small(a, row, c);
        float4 &m = k.m, &v = k.v;
        const size_t r = (size_t)row;
        if (c == 12) {
            // rotation quaternion
            float *pt = a.a_rot + r * 4;
            float4 th = ld4(pt);
            const float4 g = ldg4_stream(a.g_rot + r * 4);
            const float l = a.lr[2];
            th.x = step_element(th.x, g.x, m.x, v.x, f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
            th.y = step_element(th.y, g.y, m.y, v.y, f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
            th.z = step_element(th.z, g.z, m.z, v.z, f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
            th.w = step_element(th.w, g.w, m.w, v.w, f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
            st4(pt, th);
        } else if (c == 13) {
            // xyz and the first log-scale component
            float *px = a.a_xyz + r * 3;
            float *ps = a.a_scale + r * 3;
            const float *gx = a.g_xyz + r * 3;
            float x0 = px[0], x1 = px[1], x2 = px[2], s0 = ps[0];
            const float g0 = __ldcs(gx), g1 = __ldcs(gx + 1), g2 = __ldcs(gx + 2), gs0 = __ldcs(a.g_scale + r * 3);
            const bool ds = a.dar_s != 0;
            // scale: dR/dkappa = exp(kappa) at the old value (App. Eq. scale)
            const float r0s = ds ? expf(s0) : 0.f;
            x0 = step_element(x0, g0, m.x, v.x, f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
            x1 = step_element(x1, g1, m.y, v.y, f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
            x2 = step_element(x2, g2, m.z, v.z, f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
            s0 = step_element(s0, gs0, m.w, v.w, f.x, f.y, a, a.lr[1], ds, r0s, a.lam_s, a.clip_s);
            if constexpr (kX) {
                x0 -= nz.x; x1 -= nz.y; x2 -= nz.z;
            }
            __stcs(px, x0); __stcs(px + 1, x1); __stcs(px + 2, x2);
            __stcs(ps, s0);
        } else {
            // the other two log-scale components and the opacity logit
            float *ps = a.a_scale + r * 3;
            float *po = a.a_op + r;
            const float *gsp = a.g_scale + r * 3;
            float s1 = ps[1], s2 = ps[2], op = *po;
            const float gs1 = __ldcs(gsp + 1), gs2 = __ldcs(gsp + 2), go = __ldcs(a.g_op + r);
            const bool ds = a.dar_s != 0, dop = a.dar_o != 0;
            const float r1s = ds ? expf(s1) : 0.f, r2s = ds ? expf(s2) : 0.f;
            // opacity: dR/dtau = sig'(tau) at the old value (App. Eq. opacity)
            const float rop = dop ? dsigmoid(op) : 0.f;
            s1 = step_element(s1, gs1, m.x, v.x, f.x, f.y, a, a.lr[1], ds, r1s, a.lam_s, a.clip_s);
            s2 = step_element(s2, gs2, m.y, v.y, f.x, f.y, a, a.lr[1], ds, r2s, a.lam_s, a.clip_s);
            op = step_element(op, go, m.z, v.z, f.x, f.y, a, a.lr[3], dop, rop, a.lam_o, a.clip_o);
            __stcs(ps + 1, s1); __stcs(ps + 2, s2);
            __stcs(po, op);
            if (!S::kTInSh) k.t += 1u;         // the row's own step count (Sec. 3.2)
            if constexpr (kX) active = op > a.tau_act;
        }
        if (sampled) {         // RSR post-scale (chunk 14 holds 3 moments)
            m.x *= a.alpha1; m.y *= a.alpha1; m.z *= a.alpha1;
            v.x *= a.alpha2; v.y *= a.alpha2; v.z *= a.alpha2;
            if (c != 14) { m.w *= a.alpha1; v.w *= a.alpha2; }
        }
        S::store_small(a, row, c, k);
        return active;
    }
}

// RSR (Eq. meth::restate) of an invisible StSS-sampled row: SH item i
// (i < 48/kW) or small chunk c = 12 + (i - 48/kW); t is left unchanged.
template <int kPrec, int kW>
__device__ __forceinline__ void rsr_item(const StepArgs &a, const int32_t row, const int i)
{
    using S = State<kPrec>;
    constexpr int kNsh = 48 / kW;
    if (i < kNsh) {
        float m[kW], v[kW];
        uint32_t t = 0;
        S::template load_sh<kW>(a, row, i, m, v, t);
#pragma unroll
        for (int e = 0; e < kW; ++e) {
            m[e] *= a.alpha1;
            v[e] *= a.alpha2;
        }
        S::template store_sh<kW>(a, row, i, m, v, t);
    } else if constexpr (kPrec == GS_MOM_FP16_BLOCK) {
        rsr_small_f16b(a, row, 12 + (i - kNsh));
    } else {
        const int c = 12 + (i - kNsh);
        Chunk k = S::load_small(a, row, c);
        k.m.x *= a.alpha1; k.m.y *= a.alpha1; k.m.z *= a.alpha1;
        k.v.x *= a.alpha2; k.v.y *= a.alpha2; k.v.z *= a.alpha2;
        if (c != 14) { k.m.w *= a.alpha1; k.v.w *= a.alpha2; }
        S::store_small(a, row, c, k);
    }
}

}  // namespace
}  // namespace gs
