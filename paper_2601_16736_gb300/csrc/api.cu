// Host side of libgsopt.so: the extern "C" entry points declared in
// include/gsopt.h.  Validates every argument before launching anything,
// owns the optimizer state and the FP64 bias-correction table, and turns the
// per-step parameters into the kernel argument block.

#include <cuda.h>
#include <math.h>
#include <string.h>

#include <stddef.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include "gs_internal.cuh"

using gs::StepArgs;

struct gs_opt {
    gs_opt_config cfg;
    int device = -1;
    int64_t n_rows = 0;
    int64_t capacity = 0;         // rows the current state buffers hold
    void *m = nullptr, *v = nullptr;
    int64_t capacity2 = 0;        // rows the spare (re-index target) buffers hold
    void *m2 = nullptr, *v2 = nullptr;
    double *tab1 = nullptr, *tab2 = nullptr;
    float2 *fac = nullptr;
    int32_t tab_len = 0;
    int32_t *err = nullptr;       // device error word written by kernel-side checks
    float *staging = nullptr;     // gs_step_host gradient staging, staging_rows rows
    int64_t staging_rows = 0;
    unsigned long long *count = nullptr;   // device counter for gs_step_host
    unsigned long long *count_host = nullptr;  // pinned
    int32_t *act_blk = nullptr;   // gs_active_rows scratch, act_blk_len entries
    int64_t act_blk_len = 0;
    double n_i = 0.0;
    bool latched = false;
    // cache of validated device allocation ranges [base, end)
    static constexpr int kRanges = 32;
    uintptr_t rbase[kRanges] = {}, rend[kRanges] = {};
    int rnext = 0;
};

namespace {

// Device address of gs_step_host_noalloc's fixed staging array on the
// current device (defined at the end of this file).
float *noalloc_scratch(int device);

constexpr int64_t kMaxRows = (int64_t)0x7fffffff - 4096;
constexpr int32_t kMaxTable = 1 << 22;

size_t state_row_bytes(int prec)
{
    return prec == GS_MOM_FP32 ? gs::kRowBytesF32
           : prec == GS_MOM_BF16 ? gs::kRowBytesBf16
           : prec == GS_MOM_FP16_BLOCK ? gs::kRowBytesF16B
           : prec == GS_MOM_FP8E4M3 ? gs::kRowBytesF8
                                   : gs::kRowBytesHyb;
}

// Bytes of one moment's state for `rows` rows: the rows, and for FP8 the
// block scales after them (64 floats per 256 rows, from a 256-B boundary).
size_t fp8_scale_offset(int64_t rows) { return ((size_t)rows * gs::kRowBytesF8 + 255) / 256 * 256; }
size_t state_bytes(int prec, int64_t rows)
{
    if (prec != GS_MOM_FP8E4M3) return state_row_bytes(prec) * (size_t)rows;
    return fp8_scale_offset(rows) + (size_t)((rows + gs::kF8BlockRows - 1) / gs::kF8BlockRows) * 64 * sizeof(float);
}
float *fp8_scales(void *base, int64_t capacity)
{
    return reinterpret_cast<float *>(static_cast<char *>(base) + fp8_scale_offset(capacity));
}

gs_status fail_cuda(gs_opt *o, cudaError_t e)
{
    if (e == cudaSuccess) return GS_OK;
    if (o) o->latched = true;
    return e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA;
}

// The two driver-API queries used for pointer validation, resolved at run
// time through the runtime (the library has no link-time dependency on
// libcuda, so it loads on machines without a driver).
typedef CUresult (*PFN_addr_range)(CUdeviceptr *, size_t *, CUdeviceptr);
typedef CUresult (*PFN_ptr_attr)(void *, CUpointer_attribute, CUdeviceptr);

bool driver_queries(PFN_addr_range *range, PFN_ptr_attr *attr)
{
    static PFN_addr_range s_range = nullptr;
    static PFN_ptr_attr s_attr = nullptr;
    if (!s_range || !s_attr) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f1, 12000, cudaEnableDefault, &q1) !=
                cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f2, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return false;
        s_range = reinterpret_cast<PFN_addr_range>(f1);
        s_attr = reinterpret_cast<PFN_ptr_attr>(f2);
    }
    *range = s_range;
    *attr = s_attr;
    return true;
}

// Is [p, p + bytes) inside one device allocation of the context's device,
// with p aligned to `align`?  NULL with bytes == 0 counts as valid.
bool dev_ok(gs_opt *o, const void *p, size_t bytes, size_t align)
{
    if (!p) return bytes == 0;
    if ((uintptr_t)p % align) return false;
    if (bytes == 0) return true;
    const uintptr_t a = (uintptr_t)p, b = a + bytes;
    if (b < a) return false;
    for (int i = 0; i < gs_opt::kRanges; ++i)
        if (o->rend[i] && a >= o->rbase[i] && b <= o->rend[i]) return true;
    PFN_addr_range range_q;
    PFN_ptr_attr attr_q;
    if (cudaSetDevice(o->device) != cudaSuccess || !driver_queries(&range_q, &attr_q)) return false;
    CUdeviceptr base = 0;
    size_t size = 0;
    if (range_q(&base, &size, (CUdeviceptr)a) != CUDA_SUCCESS) return false;
    int ordinal = -1;
    if (attr_q(&ordinal, CU_POINTER_ATTRIBUTE_DEVICE_ORDINAL, (CUdeviceptr)a) != CUDA_SUCCESS) return false;
    if (ordinal != o->device) return false;
    if (b > (uintptr_t)base + size) return false;
    o->rbase[o->rnext] = (uintptr_t)base;
    o->rend[o->rnext] = (uintptr_t)base + size;
    o->rnext = (o->rnext + 1) % gs_opt::kRanges;
    return true;
}

bool current_device_ok(const gs_opt *o)
{
    int d = -1;
    return cudaGetDevice(&d) == cudaSuccess && d == o->device;
}

gs_status precheck(gs_opt *o)
{
    if (!o) return GS_ERR_INVALID_ARG;
    if (o->latched) return GS_ERR_STATE;
    if (!current_device_ok(o)) return GS_ERR_INVALID_ARG;
    return GS_OK;
}

template <class A>
bool attrs_ok(gs_opt *o, const A &a, int64_t n)
{
    const size_t r = (size_t)n;
    return dev_ok(o, a.xyz, 12 * r, 4) && dev_ok(o, a.scale, 12 * r, 4) && dev_ok(o, a.rot, 16 * r, 16) &&
           dev_ok(o, a.opacity, 4 * r, 4) && dev_ok(o, a.sh, 192 * r, 16) &&
           (n == 0 || (a.xyz && a.scale && a.rot && a.opacity && a.sh));
}

bool finite(float x) { return isfinite(x); }

bool camera_ok(const gs_camera *c)
{
    if (!c) return false;
    const float *f = reinterpret_cast<const float *>(c);
    for (int i = 0; i < 16; ++i)
        if (!finite(f[i])) return false;
    return true;
}

// Paper's N_I rule (App. "DAR"): leading decimal digit kept, then / 10.
double n_i_rule(int64_t n_pixels)
{
    if (n_pixels <= 0) return 0.0;
    int64_t p = 1;
    while (n_pixels / p >= 10) p *= 10;
    return (double)((n_pixels / p) * p) / 10.0;
}

// Length of the factor table: the first k at which both FP32 factors are
// exactly 1 (they stay 1 for larger k), capped at kMaxTable.
int32_t table_length(double b1, double b2)
{
    double p1 = 1.0, p2 = 1.0;
    for (int32_t k = 1; k < kMaxTable; ++k) {
        p1 *= b1;
        p2 *= b2;
        if ((float)(1.0 / (1.0 - p1)) == 1.0f && (float)(1.0 / sqrt(1.0 - p2)) == 1.0f) return k + 1;
    }
    return kMaxTable;
}

// Allocate the m, v rows of `rows` primitives; on failure nothing stays
// allocated.
gs_status alloc_state(gs_opt *o, int64_t rows, void **m, void **v)
{
    const size_t bytes = state_bytes(o->cfg.prec, rows > 0 ? rows : 1);
    *m = *v = nullptr;
    if (cudaMalloc(m, bytes) != cudaSuccess || cudaMalloc(v, bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(*m);
        cudaFree(*v);
        *m = *v = nullptr;
        return GS_ERR_OOM;
    }
    return GS_OK;
}

gs::StateView view_of(const gs_opt *o, void *m, void *v, int64_t capacity)
{
    gs::StateView st{o->cfg.prec, m, v};
    if (o->cfg.prec == GS_MOM_FP8E4M3) {
        st.msc = fp8_scales(m, capacity);
        st.vsc = fp8_scales(v, capacity);
    }
    return st;
}
gs::StateView view(const gs_opt *o) { return view_of(o, o->m, o->v, o->capacity); }

// The optional terms of the extended step are not built for FP8 moments.
bool terms_unsupported(const gs_opt *o, const gs_step_params *p)
{
    return o->cfg.prec == GS_MOM_FP8E4M3 && (p->noise || p->aiu || p->n_active);
}

bool params_ok(gs_opt *o, const gs_step_params *p)
{
    if (!p || p->reserved != 0 || p->reserved2 != 0) return false;
    for (int i = 0; i < 6; ++i)
        if (!finite(p->lr[i])) return false;
    if (p->restate && !(p->restate_ratio >= 0.0 && p->restate_ratio <= 1.0)) return false;
    // k fills bits 32-61 of the draw counters
    if (p->iteration < 1 || p->iteration >= ((int64_t)1 << 30)) return false;
    if (p->noise < GS_NOISE_OFF || p->noise > GS_NOISE_ALL) return false;
    if (p->noise && !(finite(p->noise_lr) && finite(p->noise_k) && finite(p->noise_t))) return false;
    if (p->aiu != 0 && p->aiu != 1) return false;
    if (p->aiu && !(p->aiu_prob >= 0.f && p->aiu_prob <= 1.f && finite(p->aiu_scale))) return false;
    if (!dev_ok(o, p->n_active, p->n_active ? 8 : 0, 8)) return false;
    if (o->cfg.reg_mode == GS_REG_COUPLED && (p->dar_opacity || p->dar_scale) && p->n_visible <= 0) return false;
    return true;
}

// sigmoid(tau) > 1/255  <=>  tau > -ln 254.  For FP32 tau the test
// tau > c with c the largest float below -ln 254 decides it exactly.
float active_threshold()
{
    const double t = -log(254.0);
    float c = (float)t;
    if ((double)c >= t) c = nextafterf(c, -INFINITY);
    return c;
}

void fill_args(const gs_opt *o, const gs_step_params *p, StepArgs *a)
{
    memset(a, 0, sizeof(*a));
    a->m = o->m;
    a->v = o->v;
    if (o->cfg.prec == GS_MOM_FP8E4M3) {
        a->msc = fp8_scales(o->m, o->capacity);
        a->vsc = fp8_scales(o->v, o->capacity);
    }
    a->fac = o->fac;
    a->fac_len = o->tab_len;
    a->n_rows = (int32_t)o->n_rows;
    a->err = o->err;
    for (int i = 0; i < 6; ++i) a->lr[i] = p->lr[i];
    a->c1 = (float)(1.0 - o->cfg.beta1);
    a->c2 = (float)(1.0 - o->cfg.beta2);
    a->eps = o->cfg.eps;
    double lo = o->cfg.lambda_o, ls = o->cfg.lambda_s;
    switch (o->cfg.reg_mode) {
    case GS_REG_DAR: lo /= o->n_i; ls /= o->n_i; break;
    case GS_REG_COUPLED: lo /= (double)p->n_visible; ls /= (double)p->n_visible; break;
    default: break;
    }
    a->lam_o = (float)lo;
    a->lam_s = (float)ls;
    a->clip_o = o->cfg.clip_o;
    a->clip_s = o->cfg.clip_s;
    a->alpha1 = o->cfg.alpha1;
    a->alpha2 = o->cfg.alpha2;
    a->dar_o = p->dar_opacity ? 1 : 0;
    a->dar_s = p->dar_scale ? 1 : 0;
    a->restate = p->restate ? 1 : 0;
    a->bias_mode = o->cfg.bias_mode;
    a->reg_mode = o->cfg.reg_mode;
    a->k_bias = (uint32_t)(p->iteration < o->tab_len ? p->iteration : o->tab_len);
    a->seed = p->seed;
    a->k_ctr = (uint64_t)p->iteration;
    // sampled iff (draw >> 11) * 2^-53 < ratio  <=>  (draw >> 11) < ceil(ratio * 2^53)
    a->rs_thr = p->restate ? (uint64_t)ceil(p->restate_ratio * 9007199254740992.0) : 0ull;
    a->noise = p->noise;
    a->noise_scale = (float)((double)p->noise_lr * (double)p->lr[0]);
    a->noise_k = p->noise_k;
    a->noise_t = p->noise_t;
    a->aiu = p->aiu;
    a->aiu_scale = p->aiu_scale;
    a->aiu_thr = p->aiu ? (uint64_t)ceil((double)p->aiu_prob * 9007199254740992.0) : 0ull;
    a->n_active = reinterpret_cast<unsigned long long *>(p->n_active);
    a->tau_act = active_threshold();
}

template <class A>
void set_attrs(StepArgs *a, const gs_attrs *x, const A *g)
{
    a->a_xyz = x->xyz; a->a_scale = x->scale; a->a_rot = x->rot; a->a_op = x->opacity; a->a_sh = x->sh;
    a->g_xyz = g->xyz; a->g_scale = g->scale; a->g_rot = g->rot; a->g_op = g->opacity; a->g_sh = g->sh;
}

// Pinned host memory the device can address (mapped, unified addressing):
// the device-side address of p, or nullptr.
const float *mapped_host(const float *p, size_t align)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer || (uintptr_t)at.devicePointer % align) return nullptr;
    return static_cast<const float *>(at.devicePointer);
}

}  // namespace

extern "C" {

const char *gs_status_string(gs_status s)
{
    switch (s) {
    case GS_OK: return "GS_OK";
    case GS_ERR_INVALID_ARG: return "GS_ERR_INVALID_ARG";
    case GS_ERR_CUDA: return "GS_ERR_CUDA";
    case GS_ERR_OOM: return "GS_ERR_OOM";
    case GS_ERR_UNSUPPORTED: return "GS_ERR_UNSUPPORTED";
    case GS_ERR_TIMEOUT: return "GS_ERR_TIMEOUT";
    case GS_ERR_STATE: return "GS_ERR_STATE";
    }
    return "GS_ERR_UNKNOWN";
}

int32_t gs_abi_version(void) { return GS_ABI_VERSION; }

double gs_dar_normaliser(int64_t n_pixels) { return n_i_rule(n_pixels); }

int64_t gs_opt_rows(const gs_opt *o) { return o ? o->n_rows : -1; }

gs_status gs_opt_init(gs_opt **out, const gs_opt_config *cfg, int64_t n_rows, void *stream)
{
    if (!out) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || n_rows < 0 || n_rows > kMaxRows) return GS_ERR_INVALID_ARG;
    const gs_opt_config &c = *cfg;
    if (!(c.beta1 >= 0.0 && c.beta1 < 1.0 && c.beta2 >= 0.0 && c.beta2 < 1.0)) return GS_ERR_INVALID_ARG;
    if (!(c.eps >= 0.0f) || !finite(c.eps) || !finite(c.lambda_o) || !finite(c.lambda_s) || !finite(c.clip_o) ||
        !finite(c.clip_s))
        return GS_ERR_INVALID_ARG;
    if (!(c.alpha1 >= 0.0f && c.alpha1 < 1.0f && c.alpha2 >= 0.0f && c.alpha2 < 1.0f)) return GS_ERR_INVALID_ARG;
    if (c.prec < GS_MOM_FP32 || c.prec > GS_MOM_FP16_BLOCK) return GS_ERR_INVALID_ARG;
    if (c.bias_mode != 0 && c.bias_mode != 1) return GS_ERR_INVALID_ARG;
    if (c.reg_mode < GS_REG_DAR || c.reg_mode > GS_REG_ADAMW_CLIP || c.reserved != 0) return GS_ERR_INVALID_ARG;
    if (c.reg_mode == GS_REG_DAR && c.n_pixels <= 0) return GS_ERR_INVALID_ARG;

    gs_opt *o = new (std::nothrow) gs_opt;
    if (!o) return GS_ERR_OOM;
    o->cfg = c;
    o->n_i = n_i_rule(c.n_pixels);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gs_status st = GS_OK;
    cudaError_t e = cudaGetDevice(&o->device);
    if (e != cudaSuccess) {
        delete o;
        return GS_ERR_CUDA;
    }
    o->n_rows = n_rows;
    o->capacity = n_rows > 0 ? n_rows : 1;
    st = alloc_state(o, o->capacity, &o->m, &o->v);
    if (st != GS_OK) {
        gs_opt_destroy(o);
        return st;
    }
    o->tab_len = table_length(c.beta1, c.beta2);
    if (cudaMalloc(&o->tab1, sizeof(double) * o->tab_len) != cudaSuccess ||
        cudaMalloc(&o->tab2, sizeof(double) * o->tab_len) != cudaSuccess ||
        cudaMalloc(&o->fac, sizeof(float2) * o->tab_len) != cudaSuccess ||
        cudaMalloc(&o->err, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        gs_opt_destroy(o);
        return GS_ERR_OOM;
    }
    const size_t sbytes = state_bytes(c.prec, o->capacity);
    if ((e = cudaMemsetAsync(o->m, 0, sbytes, s)) != cudaSuccess || (e = cudaMemsetAsync(o->v, 0, sbytes, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(o->err, 0, sizeof(int32_t), s)) != cudaSuccess ||
        (e = gs::launch_bias_table(c.beta1, c.beta2, o->tab_len, o->tab1, o->tab2, o->fac, s)) != cudaSuccess) {
        gs_opt_destroy(o);
        return GS_ERR_CUDA;
    }
    // Resolve the allocation-free step's staging array now, so that its
    // reservation and the symbol lookup happen at set-up rather than in the
    // first gs_step_host_noalloc; a failure is retried by that call.
    if (!noalloc_scratch(o->device)) cudaGetLastError();
    *out = o;
    return GS_OK;
}

void gs_opt_destroy(gs_opt *o)
{
    if (!o) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (o->device >= 0) cudaSetDevice(o->device);
    cudaDeviceSynchronize();
    cudaFree(o->m);
    cudaFree(o->v);
    cudaFree(o->m2);
    cudaFree(o->v2);
    cudaFree(o->tab1);
    cudaFree(o->tab2);
    cudaFree(o->fac);
    cudaFree(o->err);
    cudaFree(o->staging);
    cudaFree(o->count);
    cudaFree(o->act_blk);
    if (o->count_host) cudaFreeHost(o->count_host);
    cudaGetLastError();
    if (prev >= 0) cudaSetDevice(prev);
    delete o;
}

gs_status gs_visibility(gs_opt *o, const float *xyz, const gs_camera *cam, uint8_t *mask, int32_t *visible_rows,
                        int64_t *n_visible, void *stream)
{
    gs_status st = precheck(o);
    if (st != GS_OK) return st;
    const int64_t n = o->n_rows;
    if (!camera_ok(cam) || !mask || (visible_rows && !n_visible)) return GS_ERR_INVALID_ARG;
    if (!dev_ok(o, xyz, 12 * (size_t)n, 4) || (n && !xyz) || !dev_ok(o, mask, (size_t)n, 1) ||
        !dev_ok(o, visible_rows, visible_rows ? 4 * (size_t)n : 0, 4) ||
        !dev_ok(o, n_visible, n_visible ? 8 : 0, 8))
        return GS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    float c[gs::kCamFloats];
    gs::camera_arg(reinterpret_cast<const float *>(cam), c);
    if (n_visible) e = cudaMemsetAsync(n_visible, 0, 8, s);
    if (e == cudaSuccess)
        e = gs::launch_visibility(xyz, (int32_t)n, c, mask, visible_rows,
                                  reinterpret_cast<unsigned long long *>(n_visible), s);
    return fail_cuda(o, e);
}

gs_status gs_step(gs_opt *o, const gs_attrs *attrs, const gs_grads *grads, const uint8_t *mask,
                  const gs_step_params *params, void *stream)
{
    gs_status st = precheck(o);
    if (st != GS_OK) return st;
    const int64_t n = o->n_rows;
    if (!attrs || !grads || !params_ok(o, params)) return GS_ERR_INVALID_ARG;
    if (terms_unsupported(o, params)) return GS_ERR_UNSUPPORTED;
    if (!attrs_ok(o, *attrs, n) || !attrs_ok(o, *grads, n) || !dev_ok(o, mask, mask ? (size_t)n : 0, 1))
        return GS_ERR_INVALID_ARG;
    StepArgs a;
    fill_args(o, params, &a);
    set_attrs(&a, attrs, grads);
    a.mask_in = mask;
    return fail_cuda(o, gs::launch_step(a, o->cfg.prec, mask ? gs::kVisMask : gs::kVisAll,
                                        static_cast<cudaStream_t>(stream)));
}

gs_status gs_step_camera(gs_opt *o, const gs_attrs *attrs, const gs_grads *grads, const gs_camera *cam,
                         uint8_t *mask_out, int64_t *n_visible, const gs_step_params *params, void *stream)
{
    gs_status st = precheck(o);
    if (st != GS_OK) return st;
    const int64_t n = o->n_rows;
    if (!attrs || !grads || !camera_ok(cam) || !params_ok(o, params)) return GS_ERR_INVALID_ARG;
    if (terms_unsupported(o, params)) return GS_ERR_UNSUPPORTED;
    if (!attrs_ok(o, *attrs, n) || !attrs_ok(o, *grads, n) || !dev_ok(o, mask_out, mask_out ? (size_t)n : 0, 1) ||
        !dev_ok(o, n_visible, n_visible ? 8 : 0, 8))
        return GS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StepArgs a;
    fill_args(o, params, &a);
    set_attrs(&a, attrs, grads);
    gs::camera_arg(reinterpret_cast<const float *>(cam), a.cam);
    a.mask_out = mask_out;
    a.n_visible = reinterpret_cast<unsigned long long *>(n_visible);
    return fail_cuda(o, gs::launch_step(a, o->cfg.prec, gs::kVisCamera, s));
}

gs_status gs_step_host(gs_opt *o, const gs_attrs *attrs, const gs_grads *gh, const gs_camera *cam,
                       const gs_step_params *params, int64_t *n_visible_host, void *stream)
{
    gs_status st = precheck(o);
    if (st != GS_OK) return st;
    const int64_t n = o->n_rows;
    if (!attrs || !gh || !camera_ok(cam) || !params_ok(o, params) || !n_visible_host) return GS_ERR_INVALID_ARG;
    if (terms_unsupported(o, params)) return GS_ERR_UNSUPPORTED;
    if (n && (!gh->xyz || !gh->scale || !gh->rot || !gh->opacity || !gh->sh)) return GS_ERR_INVALID_ARG;
    if (!attrs_ok(o, *attrs, n)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!o->count) {
        if (cudaMalloc(&o->count, sizeof(unsigned long long)) != cudaSuccess ||
            cudaMallocHost(&o->count_host, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return GS_ERR_OOM;
        }
    }
    // Pinned gradients are read in place by the step kernel over the CPU-GPU
    // link, so only the visible rows' gradients cross it; other host memory
    // is copied to device staging first.
    if (n) {
        const float *mx = mapped_host(gh->xyz, 4), *ms = mapped_host(gh->scale, 4), *mr = mapped_host(gh->rot, 16),
                    *mo = mapped_host(gh->opacity, 4), *mh = mapped_host(gh->sh, 16);
        if (mx && ms && mr && mo && mh) {
            gs_grads gd{mx, ms, mr, mo, mh};
            StepArgs a;
            fill_args(o, params, &a);
            set_attrs(&a, attrs, &gd);
            gs::camera_arg(reinterpret_cast<const float *>(cam), a.cam);
            a.n_visible = o->count;
            a.g_host = 1;
            cudaError_t e = cudaMemsetAsync(o->count, 0, sizeof(unsigned long long), s);
            if (e == cudaSuccess) e = gs::launch_step(a, o->cfg.prec, gs::kVisCamera, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(o->count_host, o->count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return fail_cuda(o, e);
            *n_visible_host = (int64_t)*o->count_host;
            return GS_OK;
        }
    }
    // staging: five groups at 256-B aligned offsets
    const int64_t w[5] = {3, 3, 4, 1, 48};
    int64_t off[5], tot = 0;
    for (int i = 0; i < 5; ++i) {
        off[i] = tot;
        tot += ((w[i] * (n > 0 ? n : 1) + 63) / 64) * 64;
    }
    if (o->staging_rows < n || !o->staging) {
        cudaFree(o->staging);
        o->staging = nullptr;
        o->staging_rows = 0;
        if (cudaMalloc(&o->staging, sizeof(float) * (size_t)tot) != cudaSuccess) {
            cudaGetLastError();
            return GS_ERR_OOM;
        }
        o->staging_rows = n > 0 ? n : 1;
    }
    if (!o->count) {
        if (cudaMalloc(&o->count, sizeof(unsigned long long)) != cudaSuccess ||
            cudaMallocHost(&o->count_host, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return GS_ERR_OOM;
        }
    }
    const float *src[5] = {gh->xyz, gh->scale, gh->rot, gh->opacity, gh->sh};
    float *dst[5];
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) {
        dst[i] = o->staging + off[i];
        if (n) e = cudaMemcpyAsync(dst[i], src[i], sizeof(float) * (size_t)(w[i] * n), cudaMemcpyHostToDevice, s);
    }
    gs_grads gd{dst[0], dst[1], dst[2], dst[3], dst[4]};
    StepArgs a;
    fill_args(o, params, &a);
    set_attrs(&a, attrs, &gd);
    gs::camera_arg(reinterpret_cast<const float *>(cam), a.cam);
    a.n_visible = o->count;
    if (e == cudaSuccess) e = cudaMemsetAsync(o->count, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = gs::launch_step(a, o->cfg.prec, gs::kVisCamera, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(o->count_host, o->count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(o, e);
    *n_visible_host = (int64_t)*o->count_host;
    return GS_OK;
}

gs_status gs_reindex_state(gs_opt *o, const int32_t *src_rows, const uint8_t *reset, int64_t n_new, void *stream)
{
    gs_status st = precheck(o);
    if (st != GS_OK) return st;
    if (n_new < 0 || n_new > kMaxRows) return GS_ERR_INVALID_ARG;
    if (!dev_ok(o, src_rows, 4 * (size_t)n_new, 4) || (n_new && !src_rows) ||
        !dev_ok(o, reset, reset ? (size_t)n_new : 0, 1))
        return GS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (o->capacity2 < n_new || !o->m2) {
        // the spare buffers are only read by the previous re-index, which
        // cudaFree waits for
        cudaFree(o->m2);
        cudaFree(o->v2);
        o->m2 = o->v2 = nullptr;
        o->capacity2 = 0;
        const int64_t cap = n_new > 0 ? n_new : 1;
        gs_status a = alloc_state(o, cap, &o->m2, &o->v2);
        if (a != GS_OK) return a;
        o->capacity2 = cap;
    }
    const gs::StateView out = view_of(o, o->m2, o->v2, o->capacity2);
    cudaError_t e = gs::launch_reindex(view(o), (int32_t)o->n_rows, out, (int32_t)n_new, src_rows, reset, o->err, s);
    if (e != cudaSuccess) return fail_cuda(o, e);
    std::swap(o->m, o->m2);
    std::swap(o->v, o->v2);
    const int64_t tc = o->capacity;
    o->capacity = o->capacity2;
    o->capacity2 = tc;
    o->n_rows = n_new;
    return GS_OK;
}

gs_status gs_gather_attrs(gs_opt *o, const gs_attrs *in, int64_t n_in, const gs_attrs *out, const int32_t *src_rows,
                          int64_t n_new, void *stream)
{
    gs_status st = precheck(o);
    if (st != GS_OK) return st;
    if (!in || !out || n_in < 0 || n_in > kMaxRows || n_new < 0 || n_new > kMaxRows) return GS_ERR_INVALID_ARG;
    if (!attrs_ok(o, *in, n_in) || !attrs_ok(o, *out, n_new) || !dev_ok(o, src_rows, 4 * (size_t)n_new, 4) ||
        (n_new && !src_rows))
        return GS_ERR_INVALID_ARG;
    return fail_cuda(o, gs::launch_gather_attrs(*in, (int32_t)n_in, *out, src_rows, (int32_t)n_new, o->err,
                                                static_cast<cudaStream_t>(stream)));
}

gs_status gs_copy_rows(gs_opt *o, const gs_attrs *attrs, const gs_grads *grads, const int32_t *rows,
                       int64_t n_listed, void *stream)
{
    gs_status st = precheck(o);
    if (st != GS_OK) return st;
    const int64_t n = o->n_rows;
    if (!attrs || !grads || n_listed < 0 || n_listed > n) return GS_ERR_INVALID_ARG;
    if (!attrs_ok(o, *attrs, n) || !attrs_ok(o, *grads, n) || !dev_ok(o, rows, 4 * (size_t)n_listed, 4) ||
        (n_listed && !rows))
        return GS_ERR_INVALID_ARG;
    const int32_t row_bytes = (int32_t)state_row_bytes(o->cfg.prec);
    const int32_t used = o->cfg.prec == GS_MOM_FP32 ? 240 : row_bytes;    // FP32: 59 values + t
    return fail_cuda(o, gs::launch_copy_rows(*attrs, *grads, o->m, o->v, row_bytes, used, rows, n_listed,
                                             (int32_t)n, o->err, static_cast<cudaStream_t>(stream)));
}

gs_status gs_active_rows(gs_opt *o, const float *opacity, int32_t *rows, int64_t *n_active, void *stream)
{
    gs_status st = precheck(o);
    if (st != GS_OK) return st;
    const int64_t n = o->n_rows;
    if (!n_active || !dev_ok(o, n_active, 8, 8) || !dev_ok(o, opacity, 4 * (size_t)n, 4) ||
        !dev_ok(o, rows, rows ? 4 * (size_t)n : 0, 4) || (n && !opacity))
        return GS_ERR_INVALID_ARG;
    const int64_t need = gs::active_rows_scratch(n);
    if (need > o->act_blk_len) {
        cudaError_t e = cudaFree(o->act_blk);
        o->act_blk = nullptr;
        o->act_blk_len = 0;
        if (e == cudaSuccess) e = cudaMalloc(&o->act_blk, (size_t)need * sizeof(int32_t));
        if (e != cudaSuccess) return fail_cuda(o, e);
        o->act_blk_len = need;
    }
    return fail_cuda(o, gs::launch_active_rows(opacity, (int32_t)n, active_threshold(), o->act_blk, rows,
                                               reinterpret_cast<long long *>(n_active),
                                               static_cast<cudaStream_t>(stream)));
}

gs_status gs_opt_export_state(gs_opt *o, float *m, float *v, uint32_t *t, void *stream)
{
    gs_status st = precheck(o);
    if (st != GS_OK) return st;
    const size_t n = (size_t)o->n_rows;
    if (!dev_ok(o, m, m ? 4 * 59 * n : 0, 4) || !dev_ok(o, v, v ? 4 * 59 * n : 0, 4) || !dev_ok(o, t, t ? 4 * n : 0, 4))
        return GS_ERR_INVALID_ARG;
    return fail_cuda(o, gs::launch_export(view(o), (int32_t)n, m, v, t, static_cast<cudaStream_t>(stream)));
}

gs_status gs_opt_import_state(gs_opt *o, const float *m, const float *v, const uint32_t *t, void *stream)
{
    gs_status st = precheck(o);
    if (st != GS_OK) return st;
    const size_t n = (size_t)o->n_rows;
    if (!dev_ok(o, m, m ? 4 * 59 * n : 0, 4) || !dev_ok(o, v, v ? 4 * 59 * n : 0, 4) || !dev_ok(o, t, t ? 4 * n : 0, 4))
        return GS_ERR_INVALID_ARG;
    return fail_cuda(o, gs::launch_import(view(o), (int32_t)n, m, v, t, static_cast<cudaStream_t>(stream)));
}

int64_t gs_bias_table_len(const gs_opt *o) { return o ? o->tab_len : -1; }

gs_status gs_bias_table(gs_opt *o, double *b1, double *b2, int64_t len, void *stream)
{
    gs_status st = precheck(o);
    if (st != GS_OK) return st;
    if (len < 0 || len > o->tab_len || !dev_ok(o, b1, b1 ? 8 * (size_t)len : 0, 8) ||
        !dev_ok(o, b2, b2 ? 8 * (size_t)len : 0, 8))
        return GS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (b1 && len) e = cudaMemcpyAsync(b1, o->tab1, 8 * (size_t)len, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && b2 && len) e = cudaMemcpyAsync(b2, o->tab2, 8 * (size_t)len, cudaMemcpyDeviceToDevice, s);
    return fail_cuda(o, e);
}

gs_status gs_opt_sync_errors(gs_opt *o, void *stream)
{
    gs_status st = precheck(o);
    if (st != GS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, o->err, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && h) e = cudaMemsetAsync(o->err, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return fail_cuda(o, e);
    return (gs_status)h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched step (gs_batch_*).

struct gs_batch {
    std::vector<gs_opt *> scenes;
    int prec = 0;
    int device = -1;
    gs::BatchParams *d_params = nullptr;   // device scene table
    unsigned *d_counters = nullptr;        // work, done
    gs::BatchParams *h_slot[2] = {nullptr, nullptr};   // pinned staging
    cudaEvent_t slot_ev[2] = {nullptr, nullptr};
    bool slot_pending[2] = {false, false};
    int next_slot = 0;
    // autotuning
    static constexpr int kReps = 3;
    int n_cand = 0, best = -1, calls = 0;
    std::vector<cudaEvent_t> ev;           // start / stop per tuning call
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t copy_node = nullptr, kern_node = nullptr;
    size_t graph_bytes = 0;
    int graph_grid = 0;
};

namespace {

size_t batch_bytes(int n) { return offsetof(gs::BatchParams, args) + (size_t)n * sizeof(StepArgs); }

gs_status batch_check(gs_batch *b, const gs_attrs *attrs, const gs_grads *grads, const gs_camera *cams,
                      const gs_step_params *params, int64_t *n_visible)
{
    if (!b || !attrs || !grads || !cams || !params) return GS_ERR_INVALID_ARG;
    const int n = (int)b->scenes.size();
    for (int s = 0; s < n; ++s) {
        gs_opt *o = b->scenes[s];
        gs_status st = precheck(o);
        if (st != GS_OK) return st;
        if (!camera_ok(&cams[s]) || !params_ok(o, &params[s])) return GS_ERR_INVALID_ARG;
        if (params[s].noise || params[s].aiu || params[s].n_active) return GS_ERR_UNSUPPORTED;
        if (!attrs_ok(o, attrs[s], o->n_rows) || !attrs_ok(o, grads[s], o->n_rows)) return GS_ERR_INVALID_ARG;
    }
    if (!dev_ok(b->scenes[0], n_visible, n_visible ? 8 * (size_t)n : 0, 8)) return GS_ERR_INVALID_ARG;
    return GS_OK;
}

// Fill the scene table for candidate `cand` into host memory `hp`.
void batch_fill(gs_batch *b, int cand, const gs_attrs *attrs, const gs_grads *grads, const gs_camera *cams,
                const gs_step_params *params, int64_t *n_visible, gs::BatchParams *hp)
{
    int tile = 0, width = 0, mb = 0;
    gs::batch_candidate_info(b->prec, cand, &tile, &width, &mb);
    const int n = (int)b->scenes.size();
    int total = 0;
    for (int s = 0; s < n; ++s) {
        const gs_opt *o = b->scenes[s];
        hp->tile_start[s] = total;
        total += (int)((o->n_rows + tile - 1) / tile);
        StepArgs &a = hp->args[s];
        fill_args(o, &params[s], &a);
        set_attrs(&a, &attrs[s], &grads[s]);
        gs::camera_arg(reinterpret_cast<const float *>(&cams[s]), a.cam);
        a.n_visible = n_visible ? reinterpret_cast<unsigned long long *>(n_visible + s) : nullptr;
    }
    hp->tile_start[n] = total;
    hp->n_scenes = n;
    hp->total_tiles = total;
}

// Take the next pinned slot (waiting until the copy that last read it ran).
cudaError_t batch_slot(gs_batch *b, int *slot)
{
    const int k = b->next_slot;
    b->next_slot ^= 1;
    if (b->slot_pending[k]) {
        const cudaError_t e = cudaEventSynchronize(b->slot_ev[k]);
        if (e != cudaSuccess) return e;
        b->slot_pending[k] = false;
    }
    *slot = k;
    return cudaSuccess;
}

// Candidate for this call: the tuning schedule, then the fastest.
cudaError_t batch_pick(gs_batch *b, int *cand, bool *timed)
{
    *timed = false;
    if (b->best >= 0) {
        *cand = b->best;
        return cudaSuccess;
    }
    const int total = b->n_cand * gs_batch::kReps;
    if (b->calls < total) {
        *cand = b->calls % b->n_cand;
        *timed = true;
        return cudaSuccess;
    }
    // all timings issued: read them and keep the fastest candidate
    cudaError_t e = cudaEventSynchronize(b->ev[2 * total - 1]);
    if (e != cudaSuccess) return e;
    std::vector<float> sum(b->n_cand, 0.f);
    for (int c = 0; c < total; ++c) {
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, b->ev[2 * c], b->ev[2 * c + 1])) != cudaSuccess) return e;
        sum[c % b->n_cand] += ms;
    }
    b->best = (int)(std::min_element(sum.begin(), sum.end()) - sum.begin());
    *cand = b->best;
    return cudaSuccess;
}

gs_status batch_run(gs_batch *b, const gs_attrs *attrs, const gs_grads *grads, const gs_camera *cams,
                    const gs_step_params *params, int64_t *n_visible, void *stream, bool graph)
{
    gs_status st = batch_check(b, attrs, grads, cams, params, n_visible);
    if (st != GS_OK) return st;
    gs_opt *o0 = b->scenes[0];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int cand = 0, slot = 0;
    bool timed = false;
    cudaError_t e = batch_pick(b, &cand, &timed);
    if (e == cudaSuccess) e = batch_slot(b, &slot);
    if (e != cudaSuccess) return fail_cuda(o0, e);
    batch_fill(b, cand, attrs, grads, cams, params, n_visible, b->h_slot[slot]);
    const int total_tiles = b->h_slot[slot]->total_tiles;
    const size_t bytes = batch_bytes((int)b->scenes.size());
    if (graph && b->best >= 0) {
        int grid = 0;
        void *fn = nullptr;
        if ((e = gs::launch_batch(b->d_params, b->d_counters, b->d_counters + 1, total_tiles, b->prec, cand, s, &grid,
                                  &fn)) != cudaSuccess)
            return fail_cuda(o0, e);
        cudaKernelNodeParams kp = {};
        unsigned *work = b->d_counters, *done = b->d_counters + 1;
        void *args[3] = {&b->d_params, &work, &done};
        kp.func = fn;
        kp.gridDim = dim3((unsigned)grid);
        kp.blockDim = dim3(256);
        kp.kernelParams = args;
        if (!b->exec) {
            if ((e = cudaGraphCreate(&b->graph, 0)) != cudaSuccess ||
                (e = cudaGraphAddMemcpyNode1D(&b->copy_node, b->graph, nullptr, 0, b->d_params, b->h_slot[slot], bytes,
                                              cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaGraphAddKernelNode(&b->kern_node, b->graph, &b->copy_node, 1, &kp)) != cudaSuccess ||
                (e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
                return fail_cuda(o0, e);
            b->graph_bytes = bytes;
            b->graph_grid = grid;
        } else {
            if ((e = cudaGraphExecMemcpyNodeSetParams1D(b->exec, b->copy_node, b->d_params, b->h_slot[slot], bytes,
                                                        cudaMemcpyHostToDevice)) != cudaSuccess)
                return fail_cuda(o0, e);
            if (grid != b->graph_grid) {      // the one-CTA-per-tile form follows the scenes' sizes
                if ((e = cudaGraphExecKernelNodeSetParams(b->exec, b->kern_node, &kp)) != cudaSuccess)
                    return fail_cuda(o0, e);
                b->graph_grid = grid;
            }
        }
        e = cudaGraphLaunch(b->exec, s);
        if (e == cudaSuccess) e = cudaEventRecord(b->slot_ev[slot], s);
        if (e != cudaSuccess) return fail_cuda(o0, e);
        b->slot_pending[slot] = true;
        return GS_OK;
    }
    e = cudaMemcpyAsync(b->d_params, b->h_slot[slot], bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->slot_ev[slot], s);
    if (e != cudaSuccess) return fail_cuda(o0, e);
    b->slot_pending[slot] = true;
    if (timed) e = cudaEventRecord(b->ev[2 * b->calls], s);
    if (e == cudaSuccess)
        e = gs::launch_batch(b->d_params, b->d_counters, b->d_counters + 1, total_tiles, b->prec, cand, s, nullptr,
                             nullptr);
    if (e == cudaSuccess && timed) e = cudaEventRecord(b->ev[2 * b->calls + 1], s);
    if (e != cudaSuccess) return fail_cuda(o0, e);
    if (timed) ++b->calls;
    return GS_OK;
}

}  // namespace

extern "C" gs_status gs_batch_create(gs_batch **out, gs_opt *const *scenes, int32_t n_scenes)
{
    if (!out) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!scenes || n_scenes < 1 || n_scenes > GS_MAX_BATCH) return GS_ERR_INVALID_ARG;
    for (int s = 0; s < n_scenes; ++s) {
        gs_status st = precheck(scenes[s]);
        if (st != GS_OK) return st;
        if (scenes[s]->cfg.prec != scenes[0]->cfg.prec || scenes[s]->device != scenes[0]->device)
            return GS_ERR_INVALID_ARG;
    }
    if (scenes[0]->cfg.prec == GS_MOM_FP8E4M3) return GS_ERR_UNSUPPORTED;   // no batched FP8 kernel
    gs_batch *b = new (std::nothrow) gs_batch;
    if (!b) return GS_ERR_OOM;
    b->scenes.assign(scenes, scenes + n_scenes);
    b->prec = scenes[0]->cfg.prec;
    b->device = scenes[0]->device;
    b->n_cand = gs::batch_candidates(b->prec);
    const size_t bytes = sizeof(gs::BatchParams);
    bool ok = b->n_cand > 0 && cudaMalloc(&b->d_params, bytes) == cudaSuccess &&
              cudaMalloc(&b->d_counters, 2 * sizeof(unsigned)) == cudaSuccess &&
              cudaMemset(b->d_counters, 0, 2 * sizeof(unsigned)) == cudaSuccess &&
              cudaMallocHost(&b->h_slot[0], bytes) == cudaSuccess && cudaMallocHost(&b->h_slot[1], bytes) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->slot_ev[0], cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->slot_ev[1], cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
        b->ev.resize(2 * b->n_cand * gs_batch::kReps, nullptr);
        for (auto &e : b->ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        const gs_status st = b->n_cand > 0 ? GS_ERR_OOM : GS_ERR_UNSUPPORTED;
        gs_batch_destroy(b);
        return st;
    }
    *out = b;
    return GS_OK;
}

extern "C" void gs_batch_destroy(gs_batch *b)
{
    if (!b) return;
    if (b->device >= 0) cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto e : b->ev)
        if (e) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k) {
        if (b->slot_ev[k]) cudaEventDestroy(b->slot_ev[k]);
        if (b->h_slot[k]) cudaFreeHost(b->h_slot[k]);
    }
    cudaFree(b->d_params);
    cudaFree(b->d_counters);
    cudaGetLastError();
    delete b;
}

extern "C" gs_status gs_batch_step(gs_batch *b, const gs_attrs *attrs, const gs_grads *grads, const gs_camera *cams,
                                   const gs_step_params *params, int64_t *n_visible, void *stream)
{
    return batch_run(b, attrs, grads, cams, params, n_visible, stream, false);
}

extern "C" gs_status gs_batch_graph_step(gs_batch *b, const gs_attrs *attrs, const gs_grads *grads,
                                         const gs_camera *cams, const gs_step_params *params, int64_t *n_visible,
                                         void *stream)
{
    return batch_run(b, attrs, grads, cams, params, n_visible, stream, true);
}

extern "C" gs_status gs_batch_config(const gs_batch *b, int32_t *tile_rows, int32_t *sh_width,
                                     int32_t *blocks_per_sm, int32_t *tuned)
{
    if (!b) return GS_ERR_INVALID_ARG;
    int tile = 0, width = 0, mb = 0;
    gs::batch_candidate_info(b->prec, b->best >= 0 ? b->best : 0, &tile, &width, &mb);
    if (tile_rows) *tile_rows = tile;
    if (sh_width) *sh_width = width;
    if (blocks_per_sm) *blocks_per_sm = mb;
    if (tuned) *tuned = b->best >= 0 ? 1 : 0;
    return GS_OK;
}

// ---------------------------------------------------------------------------
// gs_step_host_noalloc: the host-gradient step with its staging in a fixed
// device array instead of memory allocated on first use.

namespace {

constexpr size_t kNaRows = GS_NOALLOC_MAX_ROWS;
// staging offsets in floats; every group starts on a 256-B boundary
constexpr size_t kNaOff[5] = {0, 3 * kNaRows, 6 * kNaRows, 10 * kNaRows, 11 * kNaRows};
constexpr size_t kNaCount = 59 * kNaRows;        // the visible counter (8 B)
constexpr size_t kNaFloats = kNaCount + 64;
constexpr int kNaMaxDevices = 64;
static_assert((kNaRows * 4) % 256 == 0, "group offsets must stay 256-B aligned");

std::atomic<float *> g_na_addr[kNaMaxDevices];

}  // namespace

static __device__ __align__(256) float g_noalloc_scratch[kNaFloats];

namespace {

// Device address of the fixed array on `device` (which must be current):
// looked up once per device, normally by gs_opt_init.
float *noalloc_scratch(int device)
{
    if (device < 0 || device >= kNaMaxDevices) return nullptr;
    float *p = g_na_addr[device].load(std::memory_order_acquire);
    if (p) return p;
    void *q = nullptr;
    if (cudaGetSymbolAddress(&q, g_noalloc_scratch) != cudaSuccess || !q) {
        cudaGetLastError();
        return nullptr;
    }
    g_na_addr[device].store(static_cast<float *>(q), std::memory_order_release);
    return static_cast<float *>(q);
}

}  // namespace

extern "C" gs_status gs_step_host_noalloc(gs_opt *o, const gs_attrs *attrs, const gs_grads *gh, const gs_camera *cam,
                                          const gs_step_params *params, int64_t *n_visible_host, void *stream)
{
    gs_status st = precheck(o);
    if (st != GS_OK) return st;
    const int64_t n = o->n_rows;
    if (n > (int64_t)kNaRows) return GS_ERR_INVALID_ARG;
    if (!attrs || !gh || !camera_ok(cam) || !params_ok(o, params) || !n_visible_host) return GS_ERR_INVALID_ARG;
    if (terms_unsupported(o, params)) return GS_ERR_UNSUPPORTED;
    if (n && (!gh->xyz || !gh->scale || !gh->rot || !gh->opacity || !gh->sh)) return GS_ERR_INVALID_ARG;
    if (!attrs_ok(o, *attrs, n)) return GS_ERR_INVALID_ARG;
    float *base = noalloc_scratch(o->device);
    if (!base) return GS_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t w[5] = {3, 3, 4, 1, 48};
    const float *src[5] = {gh->xyz, gh->scale, gh->rot, gh->opacity, gh->sh};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 5 && e == cudaSuccess; ++i)
        if (n) e = cudaMemcpyAsync(base + kNaOff[i], src[i], sizeof(float) * w[i] * (size_t)n, cudaMemcpyHostToDevice, s);
    unsigned long long *count = reinterpret_cast<unsigned long long *>(base + kNaCount);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
    gs_grads gd{base + kNaOff[0], base + kNaOff[1], base + kNaOff[2], base + kNaOff[3], base + kNaOff[4]};
    StepArgs a;
    fill_args(o, params, &a);
    set_attrs(&a, attrs, &gd);
    gs::camera_arg(reinterpret_cast<const float *>(cam), a.cam);
    a.n_visible = count;
    if (e == cudaSuccess) e = gs::launch_step(a, o->cfg.prec, gs::kVisCamera, s);
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, count, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(o, e);
    *n_visible_host = (int64_t)h;
    return GS_OK;
}

