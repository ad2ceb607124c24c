// Fused AdamW-GS step: visibility decision, shared-memory compaction of the
// visible rows of a tile, Sparse Adam + DAR on the visible rows, RSR on the
// StSS-sampled rows — one pass over HBM per step.
//
// One CTA handles one tile of kTile consecutive rows with 256 threads:
//   A. each thread decides visibility (camera frustum test of the mean,
//      caller mask, or all-visible) and StSS membership for kTile/256 rows,
//      issuing the load of a visible row's step counter right away; warp
//      ballots + a per-(chunk, warp) count table place every visible row in a
//      shared-memory list (ascending by row) next to the two bias-correction
//      factors of its new step count.
//   B. a flat loop over work items, each one chunk of 4 state slots (4 moments
//      of m and of v) with the 4 attribute columns that map to it:
//        12 SH items per visible row (slots 0-47: a warp covers 2.7 rows of
//           contiguous 192-B SH rows and state rows),
//        1 rotation item (slots 48-51), 1 xyz + scale0 item (52-55),
//        1 scale1 + scale2 + opacity + t item (56-59) per visible row,
//        15 state-only RSR items per invisible StSS-sampled row.
//      Items are grouped by kind so that warps stay convergent.
// Every row's attributes, moments and counter are read and written by exactly
// one item, once.  The storage format of the moments is a template parameter
// (State<kPrec>): all arithmetic is FP32.

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

// ------------------------------------------------------------ state formats
// A chunk of the state: 4 moments of m and of v as FP32, plus (chunk 14 only)
// the row's step counter t.
struct Chunk {
    float4 m, v;
    uint32_t t;
};

template <int kPrec>
struct State;

template <>
struct State<GS_MOM_FP32> {
    static constexpr int kRowBytes = kRowBytesF32, kTByte = kTByteF32, kTChunk = 14;
    static __device__ __forceinline__ float *row(void *base, int32_t r)
    {
        return static_cast<float *>(base) + (size_t)r * kSlots;
    }
    static __device__ __forceinline__ Chunk load(const StepArgs &a, int32_t r, int c)
    {
        Chunk k;
        k.m = ld4(row(a.m, r) + 4 * c);
        k.v = ld4(row(a.v, r) + 4 * c);
        k.t = __float_as_uint(k.m.w);           // slot 59 of m (meaningful for c == 14)
        return k;
    }
    static __device__ __forceinline__ void store(const StepArgs &a, int32_t r, int c, Chunk k)
    {
        if (c == 14) k.m.w = __uint_as_float(k.t);
        st4(row(a.m, r) + 4 * c, k.m);
        st4(row(a.v, r) + 4 * c, k.v);
    }
};

__device__ __forceinline__ float4 bf16x4_to_f4(uint32_t lo, uint32_t hi)
{
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&lo));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&hi));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ uint32_t pack_bf16x2(float x, float y)
{
    const __nv_bfloat162 p = __floats2bfloat162_rn(x, y);
    return *reinterpret_cast<const uint32_t *>(&p);
}

// BF16 rows of 64 slots (128 B); chunk c = 8 B at byte 8c; t = uint32 at byte
// 120, loaded and stored with chunk 14 as one 16-B access (slots 56-63).
template <>
struct State<GS_MOM_BF16> {
    static constexpr int kRowBytes = kRowBytesBf16, kTByte = kTByteBf16, kTChunk = 14;
    static __device__ __forceinline__ char *row(void *base, int32_t r)
    {
        return static_cast<char *>(base) + (size_t)r * kRowBytes;
    }
    static __device__ __forceinline__ Chunk load(const StepArgs &a, int32_t r, int c)
    {
        Chunk k;
        if (c < 14) {
            const uint2 um = *reinterpret_cast<const uint2 *>(row(a.m, r) + 8 * c);
            k.m = bf16x4_to_f4(um.x, um.y);
            k.t = 0;
        } else {
            const uint4 um = *reinterpret_cast<const uint4 *>(row(a.m, r) + 112);
            k.m = bf16x4_to_f4(um.x, um.y);
            k.t = um.z;
        }
        const uint2 uv = *reinterpret_cast<const uint2 *>(row(a.v, r) + 8 * c);
        k.v = bf16x4_to_f4(uv.x, uv.y);
        return k;
    }
    static __device__ __forceinline__ void store(const StepArgs &a, int32_t r, int c, const Chunk &k)
    {
        if (c < 14) {
            __stcs(reinterpret_cast<uint2 *>(row(a.m, r) + 8 * c),
                   make_uint2(pack_bf16x2(k.m.x, k.m.y), pack_bf16x2(k.m.z, k.m.w)));
        } else {
            __stcs(reinterpret_cast<uint4 *>(row(a.m, r) + 112),
                   make_uint4(pack_bf16x2(k.m.x, k.m.y), pack_bf16x2(k.m.z, k.m.w), k.t, 0u));
        }
        __stcs(reinterpret_cast<uint2 *>(row(a.v, r) + 8 * c),
               make_uint2(pack_bf16x2(k.v.x, k.v.y), pack_bf16x2(k.v.z, k.v.w)));
    }
};

// MurmurHash3's 32-bit finaliser (Appleby, public domain): the random bits of
// stochastic rounding, a function of (seed, iteration, row, slot) only.
__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// FP32 -> BF16 bits, rounded stochastically: add 16 random bits below the
// kept mantissa and truncate (unbiased: rounds up with probability equal to
// the discarded fraction).  Inf / NaN take the round-to-nearest path.
__device__ __forceinline__ uint32_t bf16_bits_sr(float x, uint32_t rnd16)
{
    const uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) == 0x7f800000u) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return (u + (rnd16 & 0xffffu)) >> 16;
}

// BF16 hybrid: FP32 row of 16 slots (64 B) for SH DC, t, rotation, xyz,
// scale, opacity; BF16 row of the 48 SH columns (96 B).  The 15 chunks map to:
//   c = 0      DC0-2 (FP32 slots 0-2) + SH column 3 (BF16 slot 3); t = FP32 slot 3
//   c = 1..11  SH columns 4c..4c+3 (BF16)
//   c = 12..14 FP32 slots 4(c-11)..4(c-11)+3 (rotation; xyz + scale0; scale1-2 + opacity)
// m is rounded to nearest; v stochastically (its ~0.1 % per-step EMA increment
// is below BF16 resolution, and round-to-nearest would freeze it).
template <>
struct State<GS_MOM_BF16_HYBRID> {
    static constexpr int kRowBytes = kRowBytesHyb, kTByte = kTByteHyb, kTChunk = 0;
    static __device__ __forceinline__ float *frow(void *base, int32_t r)
    {
        return static_cast<float *>(base) + (size_t)r * 16;
    }
    static __device__ __forceinline__ char *shrow(void *base, int32_t r)
    {
        return static_cast<char *>(base) + (size_t)r * kRowBytesHybSh;
    }
    static __device__ __forceinline__ Chunk load(const StepArgs &a, int32_t r, int c)
    {
        Chunk k;
        k.t = 0;
        if (c >= 12) {
            k.m = ld4(frow(a.m, r) + 4 * (c - 11));
            k.v = ld4(frow(a.v, r) + 4 * (c - 11));
        } else {
            const uint2 um = *reinterpret_cast<const uint2 *>(shrow(a.m2, r) + 8 * c);
            const uint2 uv = *reinterpret_cast<const uint2 *>(shrow(a.v2, r) + 8 * c);
            k.m = bf16x4_to_f4(um.x, um.y);
            k.v = bf16x4_to_f4(uv.x, uv.y);
            if (c == 0) {
                const float4 fm = ld4(frow(a.m, r)), fv = ld4(frow(a.v, r));
                k.m.x = fm.x; k.m.y = fm.y; k.m.z = fm.z;
                k.v.x = fv.x; k.v.y = fv.y; k.v.z = fv.z;
                k.t = __float_as_uint(fm.w);
            }
        }
        return k;
    }
    static __device__ __forceinline__ void store(const StepArgs &a, int32_t r, int c, const Chunk &k)
    {
        if (c >= 12) {
            st4(frow(a.m, r) + 4 * (c - 11), k.m);
            st4(frow(a.v, r) + 4 * (c - 11), k.v);
            return;
        }
        const uint32_t h1 = fmix32((uint32_t)r * 0x9e3779b1u ^ (uint32_t)c * 0x85ebca77u ^
                                   (uint32_t)a.k_ctr * 0xc2b2ae3du ^ (uint32_t)a.seed);
        const uint32_t h2 = fmix32(h1 ^ 0x27d4eb2fu);
        const uint32_t vlo = bf16_bits_sr(k.v.x, h1) | (bf16_bits_sr(k.v.y, h1 >> 16) << 16);
        const uint32_t vhi = bf16_bits_sr(k.v.z, h2) | (bf16_bits_sr(k.v.w, h2 >> 16) << 16);
        if (c == 0) {
            st4(frow(a.m, r), make_float4(k.m.x, k.m.y, k.m.z, __uint_as_float(k.t)));
            st4(frow(a.v, r), make_float4(k.v.x, k.v.y, k.v.z, 0.f));
            // BF16 slots 0-2 are unused: only SH column 3 lives there
            __stcs(reinterpret_cast<uint2 *>(shrow(a.m2, r)), make_uint2(0u, pack_bf16x2(0.f, k.m.w)));
            __stcs(reinterpret_cast<uint2 *>(shrow(a.v2, r)), make_uint2(0u, vhi & 0xffff0000u));
            return;
        }
        __stcs(reinterpret_cast<uint2 *>(shrow(a.m2, r) + 8 * c),
               make_uint2(pack_bf16x2(k.m.x, k.m.y), pack_bf16x2(k.m.z, k.m.w)));
        __stcs(reinterpret_cast<uint2 *>(shrow(a.v2, r) + 8 * c), make_uint2(vlo, vhi));
    }
};

// ---------------------------------------------------------------- the items

// One visible-row item: state chunk c (0..14) of `row` with its 4 attribute
// columns; `sampled` applies the RSR post-scale; f = the row's bias factors.
template <int kPrec>
__device__ __forceinline__ void visible_item(const StepArgs &a, const int32_t row, const int c, const bool sampled,
                                             const float2 f)
{
    using S = State<kPrec>;
    Chunk k = S::load(a, row, c);
    float4 &m = k.m, &v = k.v;
    const size_t r = (size_t)row;
    if (c < 12) {
        // 4 SH columns (column 4c .. 4c+3; 0-2 are the DC term)
        const size_t off = r * 48 + c * 4;
        float4 th = ld4(a.a_sh + off);
        const float4 g = ldg4_stream(a.g_sh + off);
        const float l0 = c == 0 ? a.lr[4] : a.lr[5], l3 = a.lr[5];
        th.x = step_element(th.x, g.x, m.x, v.x, f.x, f.y, a, l0, false, 0.f, 0.f, 0.f);
        th.y = step_element(th.y, g.y, m.y, v.y, f.x, f.y, a, l0, false, 0.f, 0.f, 0.f);
        th.z = step_element(th.z, g.z, m.z, v.z, f.x, f.y, a, l0, false, 0.f, 0.f, 0.f);
        th.w = step_element(th.w, g.w, m.w, v.w, f.x, f.y, a, l3, false, 0.f, 0.f, 0.f);
        st4(a.a_sh + off, th);
    } else if (c == 12) {
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
        const float *gsp = a.g_scale + r * 3;
        float x0 = px[0], x1 = px[1], x2 = px[2], s0 = ps[0];
        const float g0 = __ldcs(gx), g1 = __ldcs(gx + 1), g2 = __ldcs(gx + 2), gs0 = __ldcs(gsp);
        const bool ds = a.dar_s != 0;
        // scale: dR/dkappa = exp(kappa) at the old value (App. Eq. scale)
        const float r0s = ds ? expf(s0) : 0.f;
        x0 = step_element(x0, g0, m.x, v.x, f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
        x1 = step_element(x1, g1, m.y, v.y, f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
        x2 = step_element(x2, g2, m.z, v.z, f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
        s0 = step_element(s0, gs0, m.w, v.w, f.x, f.y, a, a.lr[1], ds, r0s, a.lam_s, a.clip_s);
        __stcs(px, x0); __stcs(px + 1, x1); __stcs(px + 2, x2);
        __stcs(ps, s0);
    } else {
        // the other two log-scale components, the opacity logit, t
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
    }
    if (c == S::kTChunk) k.t += 1u;     // the row's own step count (Sec. 3.2)
    if (sampled) {         // RSR post-scale of a sampled visible row (chunk 14 has 3 moments)
        m.x *= a.alpha1; m.y *= a.alpha1; m.z *= a.alpha1;
        v.x *= a.alpha2; v.y *= a.alpha2; v.z *= a.alpha2;
        if (c != 14) { m.w *= a.alpha1; v.w *= a.alpha2; }
    }
    S::store(a, row, c, k);
}

// RSR on state chunk c of an invisible StSS-sampled row (Eq. meth::restate).
template <int kPrec>
__device__ __forceinline__ void rsr_item(const StepArgs &a, const int32_t row, const int c)
{
    using S = State<kPrec>;
    Chunk k = S::load(a, row, c);
    k.m.x *= a.alpha1; k.m.y *= a.alpha1; k.m.z *= a.alpha1;
    k.v.x *= a.alpha2; k.v.y *= a.alpha2; k.v.z *= a.alpha2;
    if (c != 14) { k.m.w *= a.alpha1; k.v.w *= a.alpha2; }
    S::store(a, row, c, k);
}

// ---------------------------------------------------------------- phase A

// Shared-memory lists of one tile.
template <int kTile>
struct TileLists {
    int32_t list[kTile];      // visible rows, bit 31 = StSS-sampled
    int32_t rlist[kTile];     // invisible StSS-sampled rows
    float2 fac[kTile];        // bias factors of each visible row
    int32_t cnt[2][kTile / 32];
};

// Decide visibility and StSS membership for the tile's rows, prefetch the
// step counters of visible rows (at byte kTByte of their m row), and compact
// both row sets into `L`.  Returns the visible count in nv and the
// invisible-sampled count in nr.
template <int kTile, int kRowBytes, int kTByte>
__device__ __forceinline__ void tile_decide(const StepArgs &a, const int vis_src, const int64_t r0, TileLists<kTile> &L,
                                            int &nv, int &nr)
{
    constexpr int kRpt = kTile / kThreads;
    constexpr int kWarps = kThreads / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nrow = (int)min((int64_t)kTile, (int64_t)a.n_rows - r0);
    unsigned bal_v[kRpt], bal_r[kRpt], bal_s[kRpt];
    uint32_t t_old[kRpt];
#pragma unroll
    for (int j = 0; j < kRpt; ++j) {
        const int lr = j * kThreads + tid;
        const int64_t row = r0 + lr;
        const bool in = lr < nrow;
        bool vis = false, smp = false;
        t_old[j] = 0;
        if (in) {
            if (vis_src == kVisCamera) {
                const float *p = a.a_xyz + row * 3;
                vis = frustum_visible(p[0], p[1], p[2], a.cam);
            } else if (vis_src == kVisMask) {
                vis = a.mask_in[row] != 0;
            } else {
                vis = true;
            }
            if (vis && !a.bias_mode)
                t_old[j] = *reinterpret_cast<const uint32_t *>(static_cast<const char *>(a.m) +
                                                               (size_t)row * kRowBytes + kTByte);
            if (a.mask_out) a.mask_out[row] = vis ? 1 : 0;
            if (a.restate) smp = stss_sampled(a, (int32_t)row);
        }
        bal_v[j] = __ballot_sync(0xffffffffu, vis);
        bal_s[j] = __ballot_sync(0xffffffffu, smp);
        bal_r[j] = bal_s[j] & ~bal_v[j];
        if (lane == 0) {
            L.cnt[0][j * kWarps + warp] = __popc(bal_v[j]);
            L.cnt[1][j * kWarps + warp] = __popc(bal_r[j]);
        }
    }
    __syncthreads();
    nv = 0;
    nr = 0;
#pragma unroll 4
    for (int q = 0; q < kRpt * kWarps; ++q) {
        nv += L.cnt[0][q];
        nr += L.cnt[1][q];
    }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kRpt; ++j) {
        const int me = j * kWarps + warp;
        int bv = 0, br = 0;
        for (int q = 0; q < me; ++q) {
            bv += L.cnt[0][q];
            br += L.cnt[1][q];
        }
        const int32_t row = (int32_t)(r0 + j * kThreads + tid);
        if (bal_v[j] & (1u << lane)) {
            const bool smp = (bal_s[j] >> lane) & 1u;
            const int pos = bv + __popc(bal_v[j] & lt);
            L.list[pos] = row | (smp ? (int32_t)0x80000000 : 0);
            const uint32_t tb = a.bias_mode ? a.k_bias : t_old[j] + 1u;
            L.fac[pos] = (tb < (uint32_t)a.fac_len) ? a.fac[tb] : make_float2(1.0f, 1.0f);
        }
        if (bal_r[j] & (1u << lane)) L.rlist[br + __popc(bal_r[j] & lt)] = row;
    }
    if (tid == 0 && a.n_visible && nv) atomicAdd(a.n_visible, (unsigned long long)nv);
    __syncthreads();
}

// ---------------------------------------------------------------- the kernel

template <int kTile, int kMinBlocks, int kPrec>
__global__ void __launch_bounds__(kThreads, kMinBlocks) step_tile(const StepArgs a, const int vis_src)
{
    static_assert(kTile % kThreads == 0, "tile must be a multiple of the block");
    using S = State<kPrec>;
    __shared__ TileLists<kTile> L;
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kTile;
    int nv, nr;
    tile_decide<kTile, S::kRowBytes, S::kTByte>(a, vis_src, r0, L, nv, nr);

    // ---- B: flat work loop, items grouped by kind
    const int e_sh = 12 * nv, e_vis = 15 * nv, e_all = e_vis + 15 * nr;
    for (int w = tid; w < e_all; w += kThreads) {
        if (w < e_vis) {
            int j, c;
            if (w < e_sh) {
                j = w / 12;
                c = w - j * 12;
            } else {
                const int q = w - e_sh;
                j = q % nv;
                c = 12 + q / nv;
            }
            const int32_t e = L.list[j];
            visible_item<kPrec>(a, e & 0x7fffffff, c, e < 0, L.fac[j]);
        } else {
            const int q = w - e_vis;
            const int j = q / 15, c = q - j * 15;
            rsr_item<kPrec>(a, L.rlist[j], c);
        }
    }
}

}  // namespace

constexpr int kStepTile = 256;
constexpr int kStepMinBlocks = 4;      // 64 registers: 4 CTAs of 256 threads per SM

cudaError_t launch_step(const StepArgs &a, int prec, int vis_src, cudaStream_t s)
{
    if (a.n_rows <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((a.n_rows + kStepTile - 1) / kStepTile);
    switch (prec) {
    case GS_MOM_FP32:
        step_tile<kStepTile, kStepMinBlocks, GS_MOM_FP32><<<grid, kThreads, 0, s>>>(a, vis_src);
        break;
    case GS_MOM_BF16:
        step_tile<kStepTile, kStepMinBlocks, GS_MOM_BF16><<<grid, kThreads, 0, s>>>(a, vis_src);
        break;
    case GS_MOM_BF16_HYBRID:
        step_tile<kStepTile, kStepMinBlocks, GS_MOM_BF16_HYBRID><<<grid, kThreads, 0, s>>>(a, vis_src);
        break;
    default:
        return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

}  // namespace gs
