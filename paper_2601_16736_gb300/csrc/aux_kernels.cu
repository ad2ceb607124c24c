// Kernels around the fused step: the standalone visibility filter with
// global compaction, the FP64 bias-correction table, optimizer-state
// re-indexing across row-set changes, canonical-layout export/import, and
// the attribute gather that accompanies a re-index.

#include <algorithm>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void record_error(int32_t *err, int32_t code)
{
    if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------- visibility
struct CamArg {
    float c[kCamFloats];
};

// One thread per row decides V (frustum test of the mean); each CTA compacts
// its visible rows with warp ballots, reserves a contiguous range of the
// output list with one atomicAdd, and writes them in ascending row order.
__global__ void __launch_bounds__(kThreads) visibility_kernel(const float *__restrict__ xyz, int32_t n,
                                                              const CamArg cam, uint8_t *__restrict__ mask,
                                                              int32_t *__restrict__ list,
                                                              unsigned long long *__restrict__ count)
{
    __shared__ int32_t s_cnt[kThreads / 32];
    __shared__ unsigned long long s_base;
    pdl_enter();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t row = (int64_t)blockIdx.x * kThreads + tid;
    const float *c = cam.c;
    bool vis = false;
    if (row < n) {
        const float *p = xyz + row * 3;
        vis = frustum_visible(p[0], p[1], p[2], c);
        mask[row] = vis ? 1 : 0;
    }
    if (!count) return;
    const unsigned b = __ballot_sync(0xffffffffu, vis);
    if (lane == 0) s_cnt[warp] = __popc(b);
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        for (int q = 0; q < kThreads / 32; ++q) tot += s_cnt[q];
        s_base = tot ? atomicAdd(count, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    if (list && vis) {
        int off = 0;
        for (int q = 0; q < warp; ++q) off += s_cnt[q];
        off += __popc(b & ((1u << lane) - 1u));
        list[s_base + off] = (int32_t)row;
    }
}

// Eight consecutive rows per thread, for 16-B aligned means: six float4
// loads carry the rows' 24 values, two 32-bit stores their mask bytes.  The
// CTA's visible rows are placed by an exclusive scan of the per-thread
// counts, so the list stays ascending within the CTA's 2048 rows; one
// atomicAdd per CTA reserves its range of the list (8 rows per thread halves
// those atomics against 4, 10 % faster over 6 M means).
constexpr int kVisRpt = 8;

__global__ void __launch_bounds__(kThreads) visibility4_kernel(const float *__restrict__ xyz, int32_t n,
                                                               const CamArg cam, uint8_t *__restrict__ mask,
                                                               int32_t *__restrict__ list,
                                                               unsigned long long *__restrict__ count)
{
    __shared__ int32_t s_warp[kThreads / 32];
    __shared__ unsigned long long s_base;
    pdl_enter();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = ((int64_t)blockIdx.x * kThreads + tid) * kVisRpt;
    const float *c = cam.c;
    unsigned vis = 0;                      // bit j: row r0 + j is visible
    if (r0 + kVisRpt <= n) {
        const float4 *p = reinterpret_cast<const float4 *>(xyz + r0 * 3);
        float4 q4[3 * kVisRpt / 4];
#pragma unroll
        for (int u = 0; u < 3 * kVisRpt / 4; ++u) q4[u] = __ldcs(p + u);
        const float *q = reinterpret_cast<const float *>(q4);
        uint32_t mw[kVisRpt / 4];
#pragma unroll
        for (int u = 0; u < kVisRpt / 4; ++u) mw[u] = 0u;
#pragma unroll
        for (int j = 0; j < kVisRpt; ++j) {
            const bool v = frustum_visible(q[3 * j], q[3 * j + 1], q[3 * j + 2], c);
            vis |= v ? 1u << j : 0u;
            mw[j / 4] |= (v ? 1u : 0u) << (8 * (j % 4));
        }
#pragma unroll
        for (int u = 0; u < kVisRpt / 4; ++u) __stcs(reinterpret_cast<uint32_t *>(mask + r0) + u, mw[u]);
    } else {
        for (int j = 0; j < kVisRpt && r0 + j < n; ++j) {
            const float *q = xyz + (r0 + j) * 3;
            const bool v = frustum_visible(q[0], q[1], q[2], c);
            vis |= v ? 1u << j : 0u;
            mask[r0 + j] = v ? 1 : 0;
        }
    }
    if (!count) return;
    const int mine = __popc(vis);
    int incl = mine;                       // inclusive scan of the counts within the warp
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        for (int q = 0; q < kThreads / 32; ++q) tot += s_warp[q];
        s_base = tot ? atomicAdd(count, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    if (list && vis) {
        int off = incl - mine;
        for (int q = 0; q < warp; ++q) off += s_warp[q];
        int32_t *dst = list + s_base + off;
        for (int j = 0; j < kVisRpt; ++j)
            if (vis & (1u << j)) *dst++ = (int32_t)(r0 + j);
    }
}

// --------------------------------------------------------------- bias table
// 1 - beta^k in FP64 for k = 0 .. len-1 (beta^k by binary exponentiation),
// plus the FP32 factors the step consumes: 1/(1 - b1^k), 1/sqrt(1 - b2^k).
__device__ double pow_int(double b, uint32_t e)
{
    double p = 1.0;
    while (e) {
        if (e & 1u) p *= b;
        b *= b;
        e >>= 1;
    }
    return p;
}

__global__ void bias_table_kernel(double beta1, double beta2, int32_t len, double *t1, double *t2,
                                  float2 *fac)
{
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= len) return;
    const double d1 = 1.0 - pow_int(beta1, (uint32_t)k);
    const double d2 = 1.0 - pow_int(beta2, (uint32_t)k);
    t1[k] = d1;
    t2[k] = d2;
    fac[k] = (k == 0) ? make_float2(0.0f, 0.0f) : make_float2((float)(1.0 / d1), (float)(1.0 / sqrt(d2)));
}

// ------------------------------------------------------------------ reindex
// One thread per (output row, 16-B chunk of its state rows): kChunks chunks
// of the m and v rows (FP32: slots 0-59 incl. the counter; BF16: the whole
// 128-B row incl. the counter at byte 120; hybrid: the whole 160-B row).
// Copied from row src[j], or zeroed for a fresh row.
template <int kChunks, int kRowBytes>
__global__ void reindex_kernel(const StateView in, int32_t n_in, const StateView out, int32_t n_out,
                               const int32_t *__restrict__ src, const uint8_t *__restrict__ reset, int32_t *err)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = gid / kChunks;
    const int c = (int)(gid - j * kChunks);
    if (j >= n_out) return;
    int32_t s = src[j];
    if (s >= n_in) {
        if (c == 0) record_error(err, GS_ERR_INVALID_ARG);
        s = -1;
    }
    const bool fresh = s < 0 || (reset && reset[j]);
    uint4 mv = make_uint4(0u, 0u, 0u, 0u), vv = mv;
    if (!fresh) {      // each row is read once and written once: stream past L2
        mv = __ldcs(reinterpret_cast<const uint4 *>(static_cast<const char *>(in.m) + (size_t)s * kRowBytes + 16 * c));
        vv = __ldcs(reinterpret_cast<const uint4 *>(static_cast<const char *>(in.v) + (size_t)s * kRowBytes + 16 * c));
    }
    __stcs(reinterpret_cast<uint4 *>(static_cast<char *>(out.m) + (size_t)j * kRowBytes + 16 * c), mv);
    __stcs(reinterpret_cast<uint4 *>(static_cast<char *>(out.v) + (size_t)j * kRowBytes + 16 * c), vv);
}

// ------------------------------------------------------------ export/import
// Canonical layout: [n][59] FP32 in the column order xyz, scale, rot,
// opacity, sh; one thread per (row, column).

// Where column c of row r of one moment array lives: a pointer to an FP32
// value, or (through *bf) to a BF16 value.
__device__ __forceinline__ float *locate(const StateView &st, void *base, int64_t r, int c, __nv_bfloat16 **bf)
{
    *bf = nullptr;
    if (st.prec == GS_MOM_FP32) return static_cast<float *>(base) + r * kSlots + slot_of_col(c);
    if (st.prec == GS_MOM_BF16) {
        *bf = reinterpret_cast<__nv_bfloat16 *>(static_cast<char *>(base) + r * kRowBytesBf16) + slot_of_col(c);
        return nullptr;
    }
    // hybrid FP32 part: [0-2] SH DC, [3] t, [4-7] rot, [8-10] xyz, [11-13] scale, [14] opacity
    char *row = static_cast<char *>(base) + r * kRowBytesHyb;
    float *f = reinterpret_cast<float *>(row);
    if (c < 3) return f + 8 + c;
    if (c < 6) return f + 11 + (c - 3);
    if (c < 10) return f + 4 + (c - 6);
    if (c == 10) return f + 14;
    if (c < 14) return f + (c - 11);
    *bf = reinterpret_cast<__nv_bfloat16 *>(row + kHybShByte) + (c - 11);
    return nullptr;
}

__device__ __forceinline__ uint32_t *t_of(const StateView &st, int64_t r)
{
    char *m = static_cast<char *>(st.m);
    if (st.prec == GS_MOM_FP32) return reinterpret_cast<uint32_t *>(m + r * kRowBytesF32 + kTByteF32);
    if (st.prec == GS_MOM_BF16) return reinterpret_cast<uint32_t *>(m + r * kRowBytesBf16 + kTByteBf16);
    return reinterpret_cast<uint32_t *>(m + r * kRowBytesHyb + kTByteHyb);
}

__global__ void export_kernel(const StateView st, int32_t n, float *__restrict__ m_out, float *__restrict__ v_out,
                              uint32_t *__restrict__ t_out)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)n * kNumCols) return;
    const int64_t r = gid / kNumCols;
    const int c = (int)(gid - r * kNumCols);
    __nv_bfloat16 *b;
    if (m_out) {
        const float *p = locate(st, st.m, r, c, &b);
        m_out[gid] = p ? *p : __bfloat162float(*b);
    }
    if (v_out) {
        const float *p = locate(st, st.v, r, c, &b);
        v_out[gid] = p ? *p : __bfloat162float(*b);
    }
    if (t_out && c == 0) t_out[r] = *t_of(st, r);
}

__global__ void import_kernel(const StateView st, int32_t n, const float *__restrict__ m_in,
                              const float *__restrict__ v_in, const uint32_t *__restrict__ t_in)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)n * kNumCols) return;
    const int64_t r = gid / kNumCols;
    const int c = (int)(gid - r * kNumCols);
    __nv_bfloat16 *b;
    if (m_in) {
        float *p = locate(st, st.m, r, c, &b);
        if (p) *p = m_in[gid]; else *b = __float2bfloat16_rn(m_in[gid]);
    }
    if (v_in) {
        float *p = locate(st, st.v, r, c, &b);
        if (p) *p = v_in[gid]; else *b = __float2bfloat16_rn(v_in[gid]);
    }
    if (t_in && c == 0) *t_of(st, r) = t_in[r];
}

// FP16-block rows: export decodes one value per thread (its group exponent
// beside it); import encodes one group per thread (8 SH columns, rotation,
// xyz + scale + opacity) so that the group's shared exponent can be chosen,
// rounding to nearest.  t is a uint16 at kTByteF16B (saturated on import).
__global__ void export_f16b_kernel(const StateView st, int32_t n, float *__restrict__ m_out,
                                   float *__restrict__ v_out, uint32_t *__restrict__ t_out)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)n * kNumCols) return;
    const int64_t r = gid / kNumCols;
    const int c = (int)(gid - r * kNumCols);
    int byte, group;
    f16b_slot(c, byte, group);
    const char *mr = static_cast<const char *>(st.m) + r * kRowBytesF16B;
    const char *vr = static_cast<const char *>(st.v) + r * kRowBytesF16B;
    if (m_out)
        m_out[gid] = __half2float(*reinterpret_cast<const __half *>(mr + byte)) * dec_scale((uint8_t)mr[kF16BExp + group]);
    if (v_out)
        v_out[gid] = __half2float(*reinterpret_cast<const __half *>(vr + byte)) * dec_scale((uint8_t)vr[kF16BExp + group]);
    if (t_out && c == 0) t_out[r] = *reinterpret_cast<const uint16_t *>(mr + kTByteF16B);
}

__global__ void import_f16b_kernel(const StateView st, int32_t n, const float *__restrict__ m_in,
                                   const float *__restrict__ v_in, const uint32_t *__restrict__ t_in)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)n * 8) return;
    const int64_t r = gid / 8;
    const int g = (int)(gid - r * 8);
    int cols[8], cnt;
    if (g < 6) {
        cnt = 8;
        for (int q = 0; q < 8; ++q) cols[q] = 11 + 8 * g + q;
    } else if (g == 6) {
        cnt = 4;
        for (int q = 0; q < 4; ++q) cols[q] = 6 + q;
    } else {
        cnt = 7;
        for (int q = 0; q < 6; ++q) cols[q] = q;
        cols[6] = 10;
    }
    for (int side = 0; side < 2; ++side) {
        const float *in = side ? v_in : m_in;
        if (!in) continue;
        char *row = static_cast<char *>(side ? st.v : st.m) + r * kRowBytesF16B;
        float x[8];
        for (int q = 0; q < cnt; ++q) x[q] = in[r * kNumCols + cols[q]];
        const uint32_t e = group_exponent(x, cnt);
        const float sc = e ? enc_scale(e) : 0.f;
        for (int q = 0; q < cnt; ++q) {
            int byte, group;
            f16b_slot(cols[q], byte, group);
            uint32_t h = e ? h_bits(x[q] * sc) : 0u;
            if (side && (h & 0x7fffu) == 0u && x[q] > 0.f) h = 1u;     // a positive v stays positive
            *reinterpret_cast<uint16_t *>(row + byte) = (uint16_t)h;
        }
        row[kF16BExp + g] = (char)e;
    }
    if (t_in && g == 7)
        *reinterpret_cast<uint16_t *>(static_cast<char *>(st.m) + r * kRowBytesF16B + kTByteF16B) =
            (uint16_t)min(t_in[r], 65535u);
}

// ----------------------------------------------------------- attribute gather
// Two flat index spaces, each walked four items per thread (float4, or
// float) with all loads issued before the stores, so a thread keeps four
// accesses in flight (eight floats per thread measured slower):
// first one item per float4 of the 16-B aligned groups (12 SH float4 and the
// rotation of each row), then one item per float of the small groups (xyz,
// scale, opacity).  Consecutive items write consecutive output addresses, and
// read consecutive input addresses wherever the sources run in order (a prune
// keeps them so).  Nothing is read again, so loads and stores stream past L2.
constexpr int kGatherVec = 13;
constexpr int kGatherU = 4, kGatherSmallU = 4;

__global__ void __launch_bounds__(kThreads) gather_vec_kernel(const gs_attrs in, int32_t n_in, const gs_attrs out,
                                                              const int32_t *__restrict__ src, int32_t n_new,
                                                              int32_t *err)
{
    const int64_t total = (int64_t)kGatherVec * n_new;
    const int64_t base = (int64_t)blockIdx.x * kThreads * kGatherU + threadIdx.x;
    float4 v[kGatherU];
    float4 *dst[kGatherU];
#pragma unroll
    for (int u = 0; u < kGatherU; ++u) {
        const int64_t idx = base + (int64_t)u * kThreads;
        dst[u] = nullptr;
        if (idx >= total) continue;
        const int64_t j = idx / kGatherVec;
        const int k = (int)(idx - kGatherVec * j);
        const int32_t s = src[j];
        if (s < 0) continue;
        if (s >= n_in) {
            if (k == 0) record_error(err, GS_ERR_INVALID_ARG);
            continue;
        }
        if (k < 12) {
            v[u] = __ldcs(reinterpret_cast<const float4 *>(in.sh) + (int64_t)s * 12 + k);
            dst[u] = reinterpret_cast<float4 *>(out.sh) + j * 12 + k;
        } else {
            v[u] = __ldcs(reinterpret_cast<const float4 *>(in.rot) + s);
            dst[u] = reinterpret_cast<float4 *>(out.rot) + j;
        }
    }
#pragma unroll
    for (int u = 0; u < kGatherU; ++u)
        if (dst[u]) __stcs(dst[u], v[u]);
}

// Items 0 .. 3n-1: xyz floats, 3n .. 6n-1: scale floats, 6n .. 7n-1: opacity.
// An out-of-range source is recorded by gather_vec_kernel.
__global__ void __launch_bounds__(kThreads) gather_small_kernel(const gs_attrs in, int32_t n_in, const gs_attrs out,
                                                                const int32_t *__restrict__ src, int32_t n_new)
{
    const int64_t n = n_new, total = 7 * n;
    const int64_t base = (int64_t)blockIdx.x * kThreads * kGatherSmallU + threadIdx.x;
    float v[kGatherSmallU];
    float *dst[kGatherSmallU];
#pragma unroll
    for (int u = 0; u < kGatherSmallU; ++u) {
        const int64_t idx = base + (int64_t)u * kThreads;
        dst[u] = nullptr;
        if (idx >= total) continue;
        const float *a;
        float *o;
        int64_t e, j;
        int c;
        if (idx < 3 * n) {
            e = idx; j = e / 3; c = (int)(e - 3 * j); a = in.xyz; o = out.xyz;
        } else if (idx < 6 * n) {
            e = idx - 3 * n; j = e / 3; c = (int)(e - 3 * j); a = in.scale; o = out.scale;
        } else {
            e = idx - 6 * n; j = e; c = 0; a = in.opacity; o = out.opacity;
        }
        const int32_t s = src[j];
        if (s < 0 || s >= n_in) continue;
        const int w = idx < 6 * n ? 3 : 1;
        v[u] = __ldcs(a + (int64_t)s * w + c);
        dst[u] = o + e;
    }
#pragma unroll
    for (int u = 0; u < kGatherSmallU; ++u)
        if (dst[u]) __stcs(dst[u], v[u]);
}

// ------------------------------------------------------------- row copy
// The memory traffic of a step over listed rows, without the update: each
// byte a visible row's step reads is read, each byte it writes is written
// back with the value read.  Items are kind-major (SH chunks, then
// moment-row chunks, then the four small groups) so warps stay convergent.
struct CopyRowsArgs {
    gs_attrs a;
    gs_grads g;
    char *m, *v;
    int32_t row_bytes, chunks;              // state row stride; 16-B chunks used per row
    const int32_t *rows;
    int64_t nl;
    int32_t n;
    int32_t *err;
    uint32_t zero;                          // 0, passed at run time (see below)
};

// The gradients are read and their bits folded into the stored values
// through a mask that is zero at run time: the stores write back exactly
// what was read, but the compiler cannot prove the gradient loads dead (a
// load whose result is never used is removed, and the copy would then move
// fewer bytes than the step).
__device__ __forceinline__ uint32_t grad_bits4(const float *p, uint32_t zero)
{
    const float4 g = __ldcs(reinterpret_cast<const float4 *>(p));
    return (__float_as_uint(g.x) ^ __float_as_uint(g.y) ^ __float_as_uint(g.z) ^ __float_as_uint(g.w)) & zero;
}
__device__ __forceinline__ float4 xor4(float4 x, uint32_t b)
{
    return make_float4(__uint_as_float(__float_as_uint(x.x) ^ b), __uint_as_float(__float_as_uint(x.y) ^ b),
                       __uint_as_float(__float_as_uint(x.z) ^ b), __uint_as_float(__float_as_uint(x.w) ^ b));
}

__global__ void __launch_bounds__(kThreads) copy_rows_kernel(const CopyRowsArgs c)
{
    pdl_enter();
    const int64_t nl = c.nl, e_sh = 12 * nl, e_m = e_sh + (int64_t)c.chunks * nl, e_st = e_m + (int64_t)c.chunks * nl;
    const int64_t total = e_st + 4 * nl;
    for (int64_t w = (int64_t)blockIdx.x * kThreads + threadIdx.x; w < total; w += (int64_t)gridDim.x * kThreads) {
        int64_t j;
        int i;
        if (w < e_sh) {
            j = w / 12;
            i = (int)(w - 12 * j);
        } else if (w < e_st) {
            const int64_t q = w < e_m ? w - e_sh : w - e_m;   // m rows, then v rows, chunks of a row adjacent
            j = q / c.chunks;
            i = (int)(q - j * c.chunks);
        } else {
            const int64_t q = w - e_st;
            i = (int)(q / nl);                   // 0 xyz, 1 rot, 2 scale, 3 opacity
            j = q - (int64_t)i * nl;
        }
        const int32_t r32 = c.rows[j];
        if (r32 < 0 || r32 >= c.n) {
            if (w < e_sh && i == 0) record_error(c.err, GS_ERR_INVALID_ARG);
            continue;
        }
        const int64_t r = r32;
        if (w < e_sh) {
            float4 *t = reinterpret_cast<float4 *>(c.a.sh + r * 48) + i;
            const uint32_t b = grad_bits4(c.g.sh + r * 48 + 4 * i, c.zero);
            __stcs(t, xor4(*t, b));
        } else if (w < e_st) {
            uint4 *t = reinterpret_cast<uint4 *>((w < e_m ? c.m : c.v) + r * c.row_bytes) + i;
            __stcs(t, *t);
        } else if (i == 1) {
            float4 *t = reinterpret_cast<float4 *>(c.a.rot + r * 4);
            const uint32_t b = grad_bits4(c.g.rot + r * 4, c.zero);
            __stcs(t, xor4(*t, b));
        } else {
            float *t = i == 0 ? c.a.xyz + r * 3 : i == 2 ? c.a.scale + r * 3 : c.a.opacity + r;
            const float *g = i == 0 ? c.g.xyz + r * 3 : i == 2 ? c.g.scale + r * 3 : c.g.opacity + r;
            const int k = i == 3 ? 1 : 3;
            for (int u = 0; u < k; ++u) {
                const uint32_t b = __float_as_uint(__ldcs(g + u)) & c.zero;
                __stcs(t + u, __uint_as_float(__float_as_uint(t[u]) ^ b));
            }
        }
    }
}

// ------------------------------------------------------------ active rows
// The ascending list of rows with tau > tau_act (opacity > 1/255) in two
// passes over blocks of kActRows rows: per-block counts, then the ordered
// write.  In the second pass every block adds up the counts of the blocks
// before it (a few thousand ints, read from L2) to find its offset, so no
// separate scan is needed; the last block also writes the total.  Rows of a
// block are taken as kActRpt strided passes of the CTA (coalesced loads, all
// in flight at once), which is also their ascending order.
constexpr int kActRpt = 16;
constexpr int kActRows = kThreads * kActRpt;
constexpr int kActWarps = kThreads / 32;

__global__ void __launch_bounds__(kThreads) active_count_kernel(const float *__restrict__ tau, int32_t n,
                                                                float tau_act, int32_t *__restrict__ blk)
{
    __shared__ int32_t warp_sum[kActWarps];
    pdl_enter();
    const int64_t r0 = (int64_t)blockIdx.x * kActRows;
    float x[kActRpt];
#pragma unroll
    for (int j = 0; j < kActRpt; ++j) {
        const int64_t r = r0 + j * kThreads + threadIdx.x;
        x[j] = r < n ? __ldg(tau + r) : -INFINITY;      // kept in L2 for the write pass
    }
    int c = 0;
#pragma unroll
    for (int j = 0; j < kActRpt; ++j) c += x[j] > tau_act ? 1 : 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kActWarps; ++w) s += warp_sum[w];
        blk[blockIdx.x] = s;
    }
}

// rows == NULL: count only (only the last block runs, to write the total).
__global__ void __launch_bounds__(kThreads) active_write_kernel(const float *__restrict__ tau, int32_t n,
                                                                float tau_act, const int32_t *__restrict__ blk,
                                                                int32_t *__restrict__ rows, long long *total)
{
    __shared__ int32_t cnt[kActRpt * kActWarps];      // per (pass, warp), then its exclusive offset
    __shared__ int32_t part[kActWarps];
    pdl_enter();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool last = blockIdx.x == gridDim.x - 1;
    if (!rows && !last) return;
    const int64_t r0 = (int64_t)blockIdx.x * kActRows;
    float x[kActRpt];
#pragma unroll
    for (int j = 0; j < kActRpt; ++j) {
        const int64_t r = r0 + j * kThreads + threadIdx.x;
        x[j] = r < n ? __ldcs(tau + r) : -INFINITY;
    }
    int before = 0;                                      // counts of the blocks before this one
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += kThreads) before += blk[b];
    before = __reduce_add_sync(0xffffffffu, before);
    unsigned bal[kActRpt];
#pragma unroll
    for (int j = 0; j < kActRpt; ++j) {
        bal[j] = __ballot_sync(0xffffffffu, x[j] > tau_act);
        if (lane == 0) cnt[j * kActWarps + warp] = __popc(bal[j]);
    }
    if (lane == 0) part[warp] = before;
    __syncthreads();
    if (warp == 0) {                                     // exclusive scan of the kActRpt*kActWarps counts
        constexpr int kPer = kActRpt * kActWarps / 32;
        int v[kPer], sum = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            v[q] = cnt[lane * kPer + q];
            sum += v[q];
        }
        int incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        int base = 0;
        for (int w = 0; w < kActWarps; ++w) base += part[w];
        int run = base + incl - sum;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            cnt[lane * kPer + q] = run;
            run += v[q];
        }
        if (last && lane == 31 && total) *total = run;
    }
    __syncthreads();
    if (!rows) return;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kActRpt; ++j)
        if (bal[j] & (1u << lane))
            rows[cnt[j * kActWarps + warp] + __popc(bal[j] & lt)] = (int32_t)(r0 + j * kThreads + threadIdx.x);
}

unsigned blocks_for(int64_t n_threads) { return (unsigned)((n_threads + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_visibility(const float *xyz, int32_t n, const float cam[kCamFloats], uint8_t *mask, int32_t *list,
                              unsigned long long *count, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    CamArg c;
    memcpy(c.c, cam, sizeof(c.c));
    if (((uintptr_t)xyz & 15u) == 0 && ((uintptr_t)mask & 3u) == 0)
        return launch_pdl(visibility4_kernel, blocks_for(((int64_t)n + kVisRpt - 1) / kVisRpt), kThreads, s, xyz, n, c,
                          mask, list, count);
    return launch_pdl(visibility_kernel, blocks_for(n), kThreads, s, xyz, n, c, mask, list, count);
}

cudaError_t launch_bias_table(double beta1, double beta2, int32_t len, double *t1, double *t2, float2 *fac,
                              cudaStream_t s)
{
    bias_table_kernel<<<blocks_for(len), kThreads, 0, s>>>(beta1, beta2, len, t1, t2, fac);
    return cudaGetLastError();
}

cudaError_t launch_reindex(const StateView &in, int32_t n_in, const StateView &out, int32_t n_out,
                           const int32_t *src, const uint8_t *reset, int32_t *err, cudaStream_t s)
{
    if (n_out <= 0) return cudaSuccess;
    switch (in.prec) {
    case GS_MOM_FP8E4M3: return launch_reindex_fp8(in, n_in, out, n_out, src, reset, err, s);
    case GS_MOM_FP32:      // whole 256-B rows (the last 16 B are padding): a warp moves two rows
        reindex_kernel<16, kRowBytesF32><<<blocks_for((int64_t)n_out * 16), kThreads, 0, s>>>(in, n_in, out, n_out,
                                                                                             src, reset, err);
        break;
    case GS_MOM_BF16:
        reindex_kernel<8, kRowBytesBf16><<<blocks_for((int64_t)n_out * 8), kThreads, 0, s>>>(in, n_in, out, n_out,
                                                                                            src, reset, err);
        break;
    case GS_MOM_BF16_HYBRID:
        reindex_kernel<10, kRowBytesHyb><<<blocks_for((int64_t)n_out * 10), kThreads, 0, s>>>(in, n_in, out, n_out,
                                                                                             src, reset, err);
        break;
    case GS_MOM_FP16_BLOCK:
        reindex_kernel<8, kRowBytesF16B><<<blocks_for((int64_t)n_out * 8), kThreads, 0, s>>>(in, n_in, out, n_out,
                                                                                            src, reset, err);
        break;
    default:
        return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

cudaError_t launch_export(const StateView &st, int32_t n, float *m_out, float *v_out, uint32_t *t_out,
                          cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (st.prec == GS_MOM_FP8E4M3) return launch_export_fp8(st, n, m_out, v_out, t_out, s);
    if (st.prec == GS_MOM_FP16_BLOCK)
        export_f16b_kernel<<<blocks_for((int64_t)n * kNumCols), kThreads, 0, s>>>(st, n, m_out, v_out, t_out);
    else
        export_kernel<<<blocks_for((int64_t)n * kNumCols), kThreads, 0, s>>>(st, n, m_out, v_out, t_out);
    return cudaGetLastError();
}

cudaError_t launch_import(const StateView &st, int32_t n, const float *m_in, const float *v_in,
                          const uint32_t *t_in, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (st.prec == GS_MOM_FP8E4M3) return launch_import_fp8(st, n, m_in, v_in, t_in, s);
    if (st.prec == GS_MOM_FP16_BLOCK)
        import_f16b_kernel<<<blocks_for((int64_t)n * 8), kThreads, 0, s>>>(st, n, m_in, v_in, t_in);
    else
        import_kernel<<<blocks_for((int64_t)n * kNumCols), kThreads, 0, s>>>(st, n, m_in, v_in, t_in);
    return cudaGetLastError();
}

cudaError_t launch_gather_attrs(const gs_attrs &in, int32_t n_in, const gs_attrs &out, const int32_t *src,
                                int32_t n_new, int32_t *err, cudaStream_t s)
{
    if (n_new <= 0) return cudaSuccess;
    const int64_t per_cta = (int64_t)kThreads * kGatherU;
    gather_vec_kernel<<<(unsigned)(((int64_t)kGatherVec * n_new + per_cta - 1) / per_cta), kThreads, 0, s>>>(
        in, n_in, out, src, n_new, err);
    const int64_t per_cta_small = (int64_t)kThreads * kGatherSmallU;
    gather_small_kernel<<<(unsigned)((7 * (int64_t)n_new + per_cta_small - 1) / per_cta_small), kThreads, 0, s>>>(
        in, n_in, out, src, n_new);
    return cudaGetLastError();
}

cudaError_t launch_copy_rows(const gs_attrs &a, const gs_grads &g, void *m, void *v, int32_t row_bytes,
                             int32_t used_bytes, const int32_t *rows, int64_t n_listed, int32_t n, int32_t *err,
                             cudaStream_t s)
{
    if (n_listed <= 0) return cudaSuccess;
    CopyRowsArgs c{a, g, static_cast<char *>(m), static_cast<char *>(v), row_bytes, used_bytes / 16, rows, n_listed,
                   n, err, 0u};
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t items = (16 + 2 * (int64_t)c.chunks) * n_listed;
    const unsigned grid = (unsigned)std::min<int64_t>((items + kThreads - 1) / kThreads, 8 * (int64_t)sms);
    return launch_pdl(copy_rows_kernel, grid, kThreads, s, c);
}

int64_t active_rows_scratch(int64_t n) { return std::max<int64_t>(1, (n + kActRows - 1) / kActRows); }

cudaError_t launch_active_rows(const float *tau, int32_t n, float tau_act, int32_t *blk, int32_t *rows,
                               long long *n_active, cudaStream_t s)
{
    if (n <= 0) return cudaMemsetAsync(n_active, 0, sizeof(long long), s);
    const int32_t nblk = (int32_t)((n + kActRows - 1) / kActRows);
    cudaError_t e = launch_pdl(active_count_kernel, (unsigned)nblk, kThreads, s, tau, n, tau_act, blk);
    if (e != cudaSuccess) return e;
    return launch_pdl(active_write_kernel, (unsigned)nblk, kThreads, s, tau, n, tau_act,
                      static_cast<const int32_t *>(blk), rows, n_active);
}

}  // namespace gs
