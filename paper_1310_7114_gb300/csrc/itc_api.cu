// itc_api.cu -- host side of libitc.so: argument checks, tap tables, batch plans and launches.
// Every entry point is declared (and documented) in include/itc.h.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "itc_internal.cuh"

using namespace itc;

namespace {

constexpr size_t kFieldsStatusBytes = 256;   // itc_fields scratch: the status word and the tile
                                             // counter of the fields launch

bool finite_pos(float x) { return isfinite(x) && x > 0.f; }

int radius_of(float sigma, float trunc) { return (int)ceil((double)trunc * (double)sigma); }

int check_image(const itc_image* img) {
    if (!img || !img->data) return ITC_ERR_INVALID_ARG;
    if (img->ndim != 2 && img->ndim != 3) return ITC_ERR_INVALID_ARG;
    if (img->H < 1 || img->W < 1 || img->pitch < img->W) return ITC_ERR_INVALID_ARG;
    if (img->ndim == 2) {
        if (img->G != 1 && img->G != 0) return ITC_ERR_INVALID_ARG;
        if (img->dtype != ITC_U8 && img->dtype != ITC_F32) return ITC_ERR_INVALID_ARG;
        if (img->weight) return ITC_ERR_INVALID_ARG;
    } else {
        if (img->G < 1 || img->G > ITC_MAX_GRAY) return ITC_ERR_INVALID_ARG;
        if (img->dtype != ITC_U8) return ITC_ERR_INVALID_ARG;
    }
    if ((long long)img->H * img->pitch > (1LL << 40)) return ITC_ERR_UNSUPPORTED;
    return ITC_OK;
}

// Widths of the codebook overlap (rho) and the data overlap (s); 0 in the struct means sigma.
float pair_width(const itc_params* p, int i) { return p->sigma_pair[i] > 0.f ? p->sigma_pair[i] : p->sigma[i]; }
float self_width(const itc_params* p, int i) { return p->sigma_self[i] > 0.f ? p->sigma_self[i] : p->sigma[i]; }

// True when V(X) needs its own fields pass (s != sigma on some axis).
bool has_self_pass(const itc_params* p, int ndim) {
    for (int i = 0; i < ndim; ++i)
        if (self_width(p, i) != p->sigma[i]) return true;
    return false;
}

int check_params(const itc_params* p, int ndim) {
    if (!p) return ITC_ERR_INVALID_ARG;
    if (!finite_pos(p->trunc)) return ITC_ERR_INVALID_ARG;
    for (int i = 0; i < ndim; ++i)
        if (!finite_pos(p->sigma[i])) return ITC_ERR_INVALID_ARG;
    if (p->iters < 0 || !isfinite(p->step_scale)) return ITC_ERR_INVALID_ARG;
    if (p->flags & ~(ITC_CONTINUOUS | ITC_FIELDS_ABSOLUTE | ITC_STOP_ON_FIXED | ITC_RECURSIVE | ITC_TEST_STALL_WAIT))
        return ITC_ERR_INVALID_ARG;
    if ((p->flags & ITC_RECURSIVE) && ndim != 2) return ITC_ERR_UNSUPPORTED;
    for (int i = 0; i < ndim; ++i) {
        // 0 selects sigma; anything else must be a positive finite width
        if (p->sigma_pair[i] != 0.f && !finite_pos(p->sigma_pair[i])) return ITC_ERR_INVALID_ARG;
        if (p->sigma_self[i] != 0.f && !finite_pos(p->sigma_self[i])) return ITC_ERR_INVALID_ARG;
    }
    if (p->flags & ITC_RECURSIVE) return ITC_OK;   // no masks: no radius limit
    float ws[3];
    for (int pass = 0; pass < 2; ++pass) {   // the fields widths, then the self-overlap widths
        for (int i = 0; i < 3; ++i) ws[i] = pass == 0 ? p->sigma[i] : self_width(p, i);
        const double ru = ceil((double)p->trunc * ws[0]), rv = ceil((double)p->trunc * ws[1]);
        if (ru > ITC_MAX_RADIUS_UV || rv > ITC_MAX_RADIUS_UV) return ITC_ERR_UNSUPPORTED;
        if (ndim == 3 && ceil((double)p->trunc * ws[2]) > ITC_MAX_RADIUS_G) return ITC_ERR_UNSUPPORTED;
        // 3-D tiles hold S, S_g, three row-pass planes and the gray bytes of 32 + 2R rows: 143 KB
        // of shared memory at R = 24, the largest radius accepted for them
        if (ndim == 3 && (ru > ITC_MAX_RADIUS_UV_3D || rv > ITC_MAX_RADIUS_UV_3D)) return ITC_ERR_UNSUPPORTED;
    }
    return ITC_OK;
}

// g[d + R] = exp(-d^2 / (2 sigma^2)) and d g[d + R], computed in double, rounded once.
void fill_taps(float sigma, int R, float* g, float* dg) {
    for (int d = -R; d <= R; ++d) {
        const double v = exp(-((double)d * d) / (2.0 * (double)sigma * sigma));
        g[d + R] = (float)v;
        dg[d + R] = (float)(d * v);
    }
}

// Deriche's damped-sinusoid fit of exp(-x^2/2) (weights alpha, beta; frequencies omega; decays b)
constexpr double kRecAlpha[2] = {1.680, -0.6803}, kRecBeta[2] = {3.735, -0.2598};
constexpr double kRecOmega[2] = {0.6318, 1.997}, kRecDecay[2] = {1.783, 1.723};

void make_rec_coef(const float* sigma, RecCoef* rc) {
    for (int a = 0; a < 2; ++a)
        for (int t = 0; t < 2; ++t) {
            const double mag = exp(-kRecDecay[t] / (double)sigma[a]), ang = kRecOmega[t] / (double)sigma[a];
            rc->zr[a][t] = (float)(mag * cos(ang));
            rc->zi[a][t] = (float)(mag * sin(ang));
        }
    for (int t = 0; t < 2; ++t) {
        rc->cr[t] = (float)kRecAlpha[t];
        rc->ci[t] = (float)(-kRecBeta[t]);
    }
}

void make_taps(const itc_params* p, int ndim, Taps* t, bool self = false) {
    memset(t, 0, sizeof(*t));
    const bool rec = (p->flags & ITC_RECURSIVE) != 0;
    for (int i = 0; i < 3; ++i) {
        const float s = (i < ndim) ? (self ? self_width(p, i) : p->sigma[i]) : 1.f;
        t->sigma[i] = s;
        t->inv2s2[i] = (i < ndim) ? (float)(1.0 / (2.0 * (double)s * s)) : 0.f;
        t->R[i] = (i < ndim && !rec) ? radius_of(s, p->trunc) : 0;
    }
    if (rec) return;   // no masks
    fill_taps(t->sigma[0], t->R[0], t->gu, t->dgu);
    fill_taps(t->sigma[1], t->R[1], t->gv, t->dgv);
    if (ndim == 3) fill_taps(t->sigma[2], t->R[2], t->gg, t->dgg);
    float a = 0.f, b = 0.f;
    for (int d = 0; d <= 2 * t->R[1]; ++d) {
        a = fmaf(t->gv[d], 1.f, a);
        b = fmaf(t->dgv[d], 1.f, b);
    }
    t->ones_gv = a;
    t->ones_dgv = b;
}

int tile_h_of(int ndim) { return ndim == 3 ? kGridTileH3 : kGridTileH2; }

void fill_desc(const itc_image* img, const itc_params* p, int M, ImageDesc* d) {
    memset(d, 0, sizeof(*d));
    d->data = img->data;
    d->weight = img->weight;
    d->ndim = img->ndim;
    d->H = img->H;
    d->W = img->W;
    d->G = img->ndim == 3 ? img->G : 1;
    d->pitch = img->pitch;
    d->dtype = img->dtype;
    d->fpitch = itc_field_pitch(img->W);
    d->M = M;
    d->iters = p->iters;
    d->flags = p->flags;
    d->step_scale = p->step_scale;
    const int th = tile_h_of(img->ndim);
    d->tiles_u = (img->H + th - 1) / th;
    d->tiles_v = (img->W + kTileW - 1) / kTileW;
    if (p->flags & ITC_RECURSIVE) {   // one S_XX partial per 32 columns
        d->tiles_u = 1;
        d->tiles_v = (img->W + 31) / 32;
    }
    d->tiles_g = img->ndim == 3 ? d->G : 1;   // 3-D tiles: one gray slice each
    d->plane_floats = (long long)d->G * img->H * d->fpitch;
    d->bwd_tiles_u = (img->H + kBwdTileH - 1) / kBwdTileH;
    d->bwd_tiles_v = (img->W + kBwdTileW - 1) / kBwdTileW;
    double k = 0;
    for (int i = 0; i < 3; ++i) {
        const bool on = i < img->ndim;
        const float s = on ? p->sigma[i] : 1.f;
        const double r = on ? (double)pair_width(p, i) : 1.0, ss = on ? (double)self_width(p, i) : 1.0;
        d->sigma[i] = s;
        d->inv2s2[i] = on ? (float)(1.0 / (2.0 * (double)s * s)) : 0.f;
        d->R[i] = on && !(p->flags & ITC_RECURSIVE) ? radius_of(s, p->trunc) : 0;
        d->rho[i] = (float)r;
        d->pinv2s2[i] = on ? (float)(1.0 / (2.0 * r * r)) : 0.f;
        d->kappa[i] = on ? (float)(((double)s * s) / (r * r)) : 0.f;
        if (on) k += 0.5 * log(pow((double)s, 4) / (r * r * ss * ss));
    }
    d->dcs_const = k;
    if (p->flags & ITC_RECURSIVE) {
        float sw[3];
        for (int i = 0; i < 3; ++i) sw[i] = i < img->ndim ? self_width(p, i) : 1.f;
        make_rec_coef(p->sigma, &d->rc);
        make_rec_coef(sw, &d->rc_self);
    }
    d->self_tiles_u = d->tiles_u;
    d->self_off = -1;
    d->self_cls = -1;
    d->sxx_off = 0;
    d->sxx_tiles = (int)((long long)d->tiles_u * d->tiles_v * d->tiles_g);
}

long long tiles_of(const ImageDesc& d) { return (long long)d.tiles_u * d.tiles_v * d.tiles_g; }

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

int cuda_status(cudaError_t e) { return e == cudaSuccess ? ITC_OK : ITC_ERR_CUDA; }

size_t plan_layout(int B, size_t* desc_off, size_t* ints_off, size_t* tmap_off = nullptr) {
    const size_t h = align_up(sizeof(PlanHeader), 256);
    const size_t d = align_up((size_t)B * sizeof(ImageDesc), 256);
    // per class an image list and a tile prefix (an image is in at most two classes: its
    // fields class and its self-overlap class), then the backward image order
    const size_t n = align_up((size_t)((5 + kGroupInts) * (size_t)B + kMaxClasses + 2) * sizeof(int), 256);
    const size_t m = align_up((size_t)B * sizeof(CUtensorMap), 256);
    if (desc_off) *desc_off = h;
    if (ints_off) *ints_off = h + d;
    if (tmap_off) *tmap_off = h + d + n;
    return h + d + n + m;
}

// cuTensorMapEncodeTiled from the CUDA driver API, looked up once; null when no CUDA driver is present (then
// every image takes the non-TMA fields path).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of an image's input for the TMA fields tiles; false if the image's rows are not
// 16-byte aligned or no encoder is available.
bool encode_input_map(const void* data, int H, int W, int pitch, int dtype, int R, int tile_h, CUtensorMap* out) {
    const int es = dtype == ITC_U8 ? 1 : 4;
    if (((uintptr_t)data % 16) != 0 || ((size_t)pitch * es) % 16 != 0) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    int bw = 0, bh = 0;
    fields_tma_box(dtype, R, tile_h, &bw, &bh);
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * es};
    const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(out, dtype == ITC_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                           2, const_cast<void*>(data), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}
bool encode_input_map(const itc_image* img, int R, CUtensorMap* out) {
    return encode_input_map(img->data, img->H, img->W, img->pitch, img->dtype, R, 64, out);
}

// Tile grid, class tile prefixes and S_XX partial offsets of a plan from each class's tile
// height; per-image tensor maps follow the tile height.  The int area keeps its size.
int relayout(PlanHeader* h, ImageDesc* descs, int* ints, CUtensorMap* tmaps) {
    for (int c = 0; c < h->ncls; ++c) {
        ClassInfo& ci = h->cls[c];
        if (ci.tma && !ci.use_plain)
            for (int i = 0; i < ci.nimg && ci.tma; ++i) {
                const ImageDesc& d = descs[ints[ci.list_off + i]];
                if (!encode_input_map(d.data, d.H, d.W, d.pitch, d.dtype, ci.taps.R[0], ci.tile_h,
                                      tmaps + ints[ci.list_off + i]))
                    ci.tma = 0;
            }
        // the plain-load kernel has one tile height per lattice dimension
        if (!ci.tma || ci.use_plain) ci.tile_h = tile_h_of(ci.ndim);
    }
    for (int b = 0; b < h->B; ++b) {
        ImageDesc& d = descs[b];
        const ClassInfo& ci = h->cls[d.cls];
        if (!ci.recursive) d.tiles_u = (d.H + ci.tile_h - 1) / ci.tile_h;
    }
    long long pbase = 0;
    for (int c = 0; c < h->ncls; ++c) {
        ClassInfo& ci = h->cls[c];
        long long t = 0;
        ci.partial_base = pbase;
        for (int i = 0; i < ci.nimg; ++i) {
            ImageDesc& d = descs[ints[ci.list_off + i]];
            ints[ci.prefix_off + i] = (int)t;
            if (ci.self) {
                // the self-overlap pass: its own tiles and partials, which S_XX then sums
                const long long nt = (long long)d.self_tiles_u * d.tiles_v * d.tiles_g;
                d.sxx_off = pbase + t;
                d.sxx_tiles = (int)nt;
                t += nt;
            } else {
                d.tile_begin = (int)t;
                d.partial_off = pbase + t;
                if (d.self_cls < 0) {
                    d.sxx_off = d.partial_off;
                    d.sxx_tiles = (int)tiles_of(d);
                }
                t += tiles_of(d);
            }
            if (t > 0x7fffffffLL) return ITC_ERR_UNSUPPORTED;
        }
        ints[ci.prefix_off + ci.nimg] = (int)t;
        ci.ntiles = (int)t;
        pbase += t;
    }
    h->total_tiles = pbase;
    return ITC_OK;
}

// Tiles [begin, end) of one class (L.tile_base is set to begin here).
cudaError_t launch_fields_any(FieldsLaunch& L, bool tma, int begin, int end, int Ru, int Rv, int ndim, int dtype,
                              cudaStream_t s) {
    L.tile_base = begin;
    if (end <= begin) return cudaSuccess;
    if (tma && fields_tma_supported(ndim, Ru, Rv)) return launch_fields_tma(L, end, Ru, dtype, s);
    if (ndim == 3) return launch_fields3d(L, end, Ru, Rv, s);
    return launch_fields(L, end - begin, Ru, Rv, ndim, dtype, s);
}

// First position in a class image list (ascending image indices) whose image is >= b.
int lower_pos(const int* list, int n, int b) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (list[mid] < b) lo = mid + 1; else hi = mid;
    }
    return lo;
}

const PlanHeader* plan_of(const void* plan_host) {
    const PlanHeader* h = reinterpret_cast<const PlanHeader*>(plan_host);
    if (!h || h->magic != kPlanMagic) return nullptr;
    return h;
}

// Where a plan's kernels find their scratch: the base from which every image's field_off (and
// self_off) counts, the S_XX partials, the backward scalars and the per-image status words.
struct WsView {
    float* fields;
    double* partials;
    double* scal;
    int* status;
    int* counters;
};

// The full workspace: [fields of every image][partials][scalars][status words].
WsView full_view(const PlanHeader* h, void* ws) {
    unsigned char* w = reinterpret_cast<unsigned char*>(ws);
    return {reinterpret_cast<float*>(w + h->ws_fields_off), reinterpret_cast<double*>(w + h->ws_partials_off),
            reinterpret_cast<double*>(w + h->ws_scal_off), reinterpret_cast<int*>(w + h->ws_status_off),
            reinterpret_cast<int*>(w + h->ws_count_off)};
}

// The budgeted workspace: the tail of the full layout ([partials][scalars][status words], for the
// whole batch) and then a window that holds the fields of one image range at a time.
size_t budget_tail_bytes(const PlanHeader* h) { return (size_t)(h->ws_bytes - h->ws_partials_off); }

// Floats of image b's fields span (its planes, scratch planes and A_s plane).
long long field_span(const PlanHeader* h, const ImageDesc* d, int b) {
    return (b + 1 < h->B ? d[b + 1].field_off : h->fields_floats) - d[b].field_off;
}

// The view of a budgeted workspace while the window holds the fields of the images from b0 on:
// the fields base is the window moved back by image b0's offset, so that base + field_off of
// those images lands inside the window (integer arithmetic; the kernels add the offsets back).
WsView budget_view(const PlanHeader* h, void* ws, const ImageDesc* hdescs, int b0) {
    unsigned char* w = reinterpret_cast<unsigned char*>(ws);
    const size_t tail = budget_tail_bytes(h);
    const uintptr_t window = reinterpret_cast<uintptr_t>(w + tail);
    const uintptr_t shift = (uintptr_t)hdescs[b0].field_off * sizeof(float);
    return {reinterpret_cast<float*>(window - shift), reinterpret_cast<double*>(w),
            reinterpret_cast<double*>(w + (h->ws_scal_off - h->ws_partials_off)),
            reinterpret_cast<int*>(w + (h->ws_status_off - h->ws_partials_off)),
            reinterpret_cast<int*>(w + (h->ws_count_off - h->ws_partials_off))};
}

}  // namespace

extern "C" {

int itc_field_pitch(int W) { return W <= 0 ? 0 : (W + 3) & ~3; }

size_t itc_fields_bytes(const itc_image* img) {
    if (check_image(img) != ITC_OK) return 0;
    const int G = img->ndim == 3 ? img->G : 1;
    return (size_t)(img->ndim + 1) * G * img->H * itc_field_pitch(img->W) * sizeof(float);
}

size_t itc_fields_workspace_bytes(const itc_image* img) {
    if (check_image(img) != ITC_OK) return 0;
    itc_params p;
    memset(&p, 0, sizeof(p));
    p.sigma[0] = p.sigma[1] = p.sigma[2] = 1.f;
    p.trunc = 1.f;
    ImageDesc d;
    fill_desc(img, &p, 1, &d);
    // the call's device status word (first 256 bytes), then one S_XX partial per tile
    return kFieldsStatusBytes + align_up((size_t)tiles_of(d) * sizeof(double), 256);
}

const char* itc_status_string(int code) {
    switch (code) {
        case ITC_OK: return "ok";
        case ITC_WARN_EMPTY_SUPPORT: return "warning: a codebook vector has no data within its mask (kept in place)";
        case ITC_ERR_INVALID_ARG: return "invalid argument";
        case ITC_ERR_CUDA: return "CUDA launch or query failed";
        case ITC_ERR_TIMEOUT: return "a bounded device wait gave up";
        case ITC_ERR_NONFINITE: return "S_XW is zero or a value is not finite";
        case ITC_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
        case ITC_ERR_UNSUPPORTED: return "request outside the library's compiled limits";
        default: return "unknown status";
    }
}

int itc_fields(const itc_image* img, const itc_params* p, float* fields, double* sxx, void* ws,
               size_t ws_bytes, void* stream) {
    int rc = check_image(img);
    if (rc) return rc;
    if ((rc = check_params(p, img->ndim))) return rc;
    if (!fields || !aligned(fields, 16)) return ITC_ERR_INVALID_ARG;
    if (p->flags & ITC_RECURSIVE) return ITC_ERR_UNSUPPORTED;   // recursive fields need a plan's scratch planes
    const size_t need = itc_fields_workspace_bytes(img);
    if (!ws || ws_bytes < need || !aligned(ws, 16)) return ITC_ERR_WORKSPACE;
    FieldsLaunch L;
    memset(&L, 0, sizeof(L));
    make_taps(p, img->ndim, &L.taps);
    fill_desc(img, p, 1, &L.one);
    L.fields = fields;
    L.status = reinterpret_cast<int*>(ws);
    L.counter = L.status + 1;
    L.partials = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(ws) + kFieldsStatusBytes);
    L.tile_h = tile_h_of(img->ndim);
    L.absolute = (p->flags & ITC_FIELDS_ABSOLUTE) ? 1 : 0;
    L.test_stall = (p->flags & ITC_TEST_STALL_WAIT) ? 1 : 0;
    const long long nt = tiles_of(L.one);
    if (nt > 0x7fffffffLL) return ITC_ERR_UNSUPPORTED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool tma = fields_tma_supported(img->ndim, L.taps.R[0], L.taps.R[1]) &&
                     encode_input_map(img, L.taps.R[0], &L.tmap_one);
    // status ITC_OK unless a wait gives up; no tiles handed out yet
    rc = cuda_status(cudaMemsetAsync(L.status, 0, 2 * sizeof(int), s));
    if (rc) return rc;
    rc = cuda_status(launch_fields_any(L, tma, 0, (int)nt, L.taps.R[0], L.taps.R[1], img->ndim, img->dtype, s));
    if (rc) return rc;
    if (sxx && has_self_pass(p, img->ndim)) {
        // V(X) at its own width: the same tiles again (plain staging), S_XX partials only
        make_taps(p, img->ndim, &L.taps, true);
        L.mode = 2;
        L.absolute = 0;
        L.test_stall = 0;
        rc = cuda_status(launch_fields_any(L, false, 0, (int)nt, L.taps.R[0], L.taps.R[1], img->ndim, img->dtype, s));
        if (rc) return rc;
    }
    if (sxx) rc = cuda_status(launch_reduce_sxx(L.partials, (int)nt, sxx, s));
    return rc;
}

int itc_step(const itc_image* img, const itc_params* p, const float* fields, const double* sxx, int M,
             const float* W_in, float* W_out, int* W_lattice, itc_stats* stats, void* stream) {
    int rc = check_image(img);
    if (rc) return rc;
    if ((rc = check_params(p, img->ndim))) return rc;
    if (M < 1 || M > ITC_MAX_M) return ITC_ERR_INVALID_ARG;
    if (!fields || !W_in || !W_out || !sxx) return ITC_ERR_INVALID_ARG;
    RunLaunch L;
    memset(&L, 0, sizeof(L));
    fill_desc(img, p, M, &L.one);
    L.one.iters = 1;
    L.fields = fields;
    L.sxx_single = sxx;
    L.W_in = W_in;
    L.W_out = W_out;
    L.W_lattice = W_lattice;
    L.stats = stats;
    L.absolute = (p->flags & ITC_FIELDS_ABSOLUTE) ? 1 : 0;
    L.final_eval = 0;
    const int dims[3] = {img->H, img->W, img->ndim == 3 ? img->G : 1};
    return cuda_status(launch_run(L, 1, M, dims, reinterpret_cast<cudaStream_t>(stream), img->ndim));
}

size_t itc_plan_bytes(int B) {
    if (B < 1) return 0;
    return plan_layout(B, nullptr, nullptr);
}

int itc_plan(int B, const itc_image* imgs, const int* M, const itc_params* p, int p_stride,
             void* plan, size_t plan_bytes, size_t* ws_bytes_out) {
    if (B < 1 || !imgs || !M || !p || !plan) return ITC_ERR_INVALID_ARG;
    size_t desc_off, ints_off, tmap_off;
    const size_t need = plan_layout(B, &desc_off, &ints_off, &tmap_off);
    if (plan_bytes < need) return ITC_ERR_INVALID_ARG;
    for (int b = 0; b < B; ++b) {
        int rc = check_image(imgs + b);
        if (rc) return rc;
        const itc_params* pb = p_stride ? p + b : p;
        if ((rc = check_params(pb, imgs[b].ndim))) return rc;
        if (M[b] < 1 || M[b] > ITC_MAX_M) return ITC_ERR_INVALID_ARG;
    }
    std::vector<unsigned char> buf(need, 0);
    PlanHeader* h = reinterpret_cast<PlanHeader*>(buf.data());
    ImageDesc* descs = reinterpret_cast<ImageDesc*>(buf.data() + desc_off);
    int* ints = reinterpret_cast<int*>(buf.data() + ints_off);
    h->magic = kPlanMagic;
    h->B = B;
    h->desc_off = (long long)desc_off;
    h->ints_off = (long long)ints_off;
    h->tmap_off = (long long)tmap_off;
    CUtensorMap* tmaps = reinterpret_cast<CUtensorMap*>(buf.data() + tmap_off);

    // parameter classes: (ndim, dtype, sigma, trunc)
    struct Key { int ndim, dtype; float s0, s1, s2, trunc; int self, rec; };
    std::vector<Key> keys;
    std::vector<int> cls_of(B), self_of(B, -1);
    // the class of (image b, pass): fields classes by (ndim, dtype, sigma, trunc); images whose
    // V(X) width differs from sigma also join a self-overlap class keyed by that width
    auto class_of = [&](int b, const itc_params* pb, bool self) -> int {
        const int nd = imgs[b].ndim;
        float w[3];
        for (int i = 0; i < 3; ++i) w[i] = i < nd ? (self ? self_width(pb, i) : pb->sigma[i]) : 0.f;
        const int rec = (pb->flags & ITC_RECURSIVE) ? 1 : 0;
        // recursive fields take their widths from each image: one class for all of them
        if (rec) w[0] = w[1] = w[2] = 0.f;
        Key k{nd, imgs[b].dtype, w[0], w[1], w[2], rec ? 0.f : pb->trunc, self ? 1 : 0, rec};
        for (size_t i = 0; i < keys.size(); ++i)
            if (memcmp(&keys[i], &k, sizeof(Key)) == 0) return (int)i;
        if ((int)keys.size() == kMaxClasses) return -1;
        keys.push_back(k);
        const int c = (int)keys.size() - 1;
        ClassInfo& ci = h->cls[c];
        make_taps(pb, nd, &ci.taps, self);
        ci.ndim = nd;
        ci.dtype = imgs[b].dtype;
        ci.absolute = 0;
        ci.self = self ? 1 : 0;
        ci.tile_h = tile_h_of(nd);
        ci.recursive = rec;
        ci.tma = !self && !rec && fields_tma_supported(ci.ndim, ci.taps.R[0], ci.taps.R[1]) ? 1 : 0;
        return c;
    };
    for (int b = 0; b < B; ++b) {
        const itc_params* pb = p_stride ? p + b : p;
        const int c = class_of(b, pb, false);
        if (c < 0) return ITC_ERR_UNSUPPORTED;
        cls_of[b] = c;
        fill_desc(imgs + b, pb, M[b], descs + b);
        descs[b].cls = c;
        if (has_self_pass(pb, imgs[b].ndim)) {
            const int sc = class_of(b, pb, true);
            if (sc < 0) return ITC_ERR_UNSUPPORTED;
            self_of[b] = sc;
            descs[b].self_cls = sc;
        }
    }
    h->ncls = (int)keys.size();

    // fields, codebook and pixel offsets
    long long foff = 0, woff = 0, ghoff = 0, maxM = 0, padoff = 0;
    int bwd = 0;
    for (int b = 0; b < B; ++b) {
        ImageDesc& d = descs[b];
        d.pad_off = padoff;
        padoff += (long long)d.H * d.fpitch;
        d.field_off = foff;
        // recursive fields keep two scratch planes (the along-v results) after the field planes
        const bool rec = (d.flags & ITC_RECURSIVE) != 0;
        foff += (long long)align_up((size_t)(d.ndim + 1 + (rec ? 2 : 0)) * d.plane_floats, 64);
        if (rec) h->has_recursive = 1;
        // then the A_s plane of an image with a self-overlap pass (plus one scratch plane for
        // recursive fields): every image's scratch is one contiguous span, so the spans of an
        // image range are contiguous too (the budgeted calls recompute them range by range)
        if (d.self_cls >= 0) {
            d.self_off = foff;
            foff += (long long)align_up((size_t)(rec ? 2 : 1) * d.plane_floats, 64);
        }
        d.w_off = woff;
        woff += (long long)d.M * d.ndim;
        d.gh_off = ghoff;
        ghoff += (long long)d.H * d.W;
        d.bwd_tile_begin = bwd;
        bwd += d.bwd_tiles_u * d.bwd_tiles_v;
        h->max_bwd_tiles = std::max(h->max_bwd_tiles, d.bwd_tiles_u * d.bwd_tiles_v);
        if (d.M > maxM) maxM = d.M;
        h->max_dim[0] = d.H > h->max_dim[0] ? d.H : h->max_dim[0];
        h->max_dim[1] = d.W > h->max_dim[1] ? d.W : h->max_dim[1];
        h->max_dim[2] = d.G > h->max_dim[2] ? d.G : h->max_dim[2];
        h->ndim_mask |= 1 << d.ndim;
    }
    h->fields_floats = foff;
    h->total_pixels = ghoff;
    h->pad_floats = padoff;
    h->max_M = (int)maxM;

    // per class: image list (ascending image index) and the place of its tile prefix
    int io = 0;
    for (int c = 0; c < h->ncls; ++c) {
        ClassInfo& ci = h->cls[c];
        ci.list_off = io;
        int n = 0;
        for (int b = 0; b < B; ++b)
            if ((ci.self ? self_of[b] : cls_of[b]) == c) ints[io + n++] = b;
        ci.nimg = n;
        io += n;
        ci.prefix_off = io;
        io += n + 1;
    }
    // S_XX partials: room for the most tiles any tunable tile height can give (32-row tiles)
    long long pcap = 0;
    {
        // the largest count over "every class at its smallest tile height" bounds any tuning
        for (int c = 0; c < h->ncls; ++c)
            if (h->cls[c].tma) h->cls[c].tile_h = 32;
        int rc = relayout(h, descs, ints, tmaps);
        if (rc) return rc;
        pcap = h->total_tiles;
        for (int c = 0; c < h->ncls; ++c) h->cls[c].tile_h = tile_h_of(h->cls[c].ndim);
        rc = relayout(h, descs, ints, tmaps);
        if (rc) return rc;
    }
    long long pbase = pcap;
    // backward pixel pass: one CTA per image, images with the most tiles first
    const int bwd_off = io;
    {
        std::vector<int> order(B);
        for (int b = 0; b < B; ++b) order[b] = b;
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
            return descs[a].bwd_tiles_u * descs[a].bwd_tiles_v > descs[c].bwd_tiles_u * descs[c].bwd_tiles_v;
        });
        for (int b = 0; b < B; ++b) ints[io++] = order[b];
    }
    // iterations: images with up to 16, 32 or 64 codebook vectors share a CTA (8, 4 or 2 of them,
    // 16, 32 or 64 threads each), larger ones have a CTA each; per dimension, the groups are
    // listed by the pair work (iters x M^2) of their costliest image, largest first, so that the
    // long ones do not start last
    const int run_off = io;
    for (int nd = 2; nd <= 3; ++nd) {
        std::vector<int> order;
        for (int b = 0; b < B; ++b)
            if (descs[b].ndim == nd) order.push_back(b);
        auto cost = [&](int b) { return (double)(descs[b].iters + 1) * descs[b].M * descs[b].M; };
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost(a) > cost(c); });
        int open[4] = {-1, -1, -1, -1};   // the group each span class is filling (int offset)
        int ng = 0;
        for (int b : order) {
            const int M = descs[b].M;
            const int cl = M <= 16 ? 0 : (M <= 32 ? 1 : (M <= 64 ? 2 : 3));
            const int span = 16 << cl, cap = cl == 3 ? 1 : kRunThreads / span;
            if (open[cl] < 0 || ints[open[cl]] == cap) {
                open[cl] = io;
                ints[io] = 0;
                ints[io + 1] = span;
                for (int i = 0; i < kGroupMax; ++i) ints[io + 2 + i] = -1;
                io += kGroupInts;
                ++ng;
            }
            int* g = ints + open[cl];
            g[2 + g[0]++] = b;
        }
        h->run_ngroups[nd - 2] = ng;
    }
    h->nints = io;
    h->bwd_order_off = bwd_off;
    h->run_groups_off = run_off;
    h->bwd_tiles = bwd;

    // workspace: [fields][S_XX partials][per-image backward scalars][per-image status words]
    // [tile counters]
    size_t off = 0;
    h->ws_fields_off = 0;
    off = align_up((size_t)foff * sizeof(float), 256);
    h->ws_partials_off = (long long)off;
    off = align_up(off + (size_t)pbase * sizeof(double), 256);
    h->ws_scal_off = (long long)off;
    off = align_up(off + (size_t)B * 4 * sizeof(double), 256);
    h->ws_status_off = (long long)off;
    off = align_up(off + (size_t)B * sizeof(int), 256);
    h->ws_count_off = (long long)off;
    off = align_up(off + (size_t)io * sizeof(int), 256);   // io: every class list position fits
    h->ws_bytes = (long long)off;
    if (ws_bytes_out) *ws_bytes_out = off;
    memcpy(plan, buf.data(), need);
    return ITC_OK;
}

size_t itc_plan_pixels(const void* plan_host) {
    const PlanHeader* h = plan_of(plan_host);
    return h ? (size_t)h->total_pixels : 0;
}

int itc_plan_offsets(const void* plan_host, int b, size_t* field_off, size_t* w_off, size_t* gh_off) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h || b < 0 || b >= h->B) return ITC_ERR_INVALID_ARG;
    const ImageDesc& d = reinterpret_cast<const ImageDesc*>(reinterpret_cast<const unsigned char*>(plan_host) + h->desc_off)[b];
    if (field_off) *field_off = (size_t)h->ws_fields_off + (size_t)d.field_off * sizeof(float);
    if (w_off) *w_off = (size_t)d.w_off;
    if (gh_off) *gh_off = (size_t)d.gh_off;
    return ITC_OK;
}

// The fields pass (every class) of images [b0, b1) into the scratch of view v.
static int fields_range(const PlanHeader* h, const void* plan_host, const void* plan_dev, int b0, int b1,
                        const WsView& v, cudaStream_t s) {
    const unsigned char* pd = reinterpret_cast<const unsigned char*>(plan_dev);
    const int* hints = reinterpret_cast<const int*>(reinterpret_cast<const unsigned char*>(plan_host) + h->ints_off);
    const ImageDesc* descs = reinterpret_cast<const ImageDesc*>(pd + h->desc_off);
    const int* ints = reinterpret_cast<const int*>(pd + h->ints_off);
    const ImageDesc* hdescs = reinterpret_cast<const ImageDesc*>(reinterpret_cast<const unsigned char*>(plan_host) +
                                                                 h->desc_off);
    // the images' status words start at ITC_OK; a fields CTA whose bounded wait gives up sets them
    if (b1 > b0 && cudaMemsetAsync(v.status + b0, 0, (size_t)(b1 - b0) * sizeof(int), s) != cudaSuccess)
        return ITC_ERR_CUDA;
    for (int c = 0; c < h->ncls; ++c) {
        const ClassInfo& ci = h->cls[c];
        const int p0 = lower_pos(hints + ci.list_off, ci.nimg, b0), p1 = lower_pos(hints + ci.list_off, ci.nimg, b1);
        const int t0 = hints[ci.prefix_off + p0], t1 = hints[ci.prefix_off + p1];
        if (t1 <= t0) continue;
        // test hook: an image of the launch asks for the stalled first copy (tensor tiles only)
        int stall = 0;
        for (int q = p0; q < p1 && !stall; ++q) stall = (hdescs[hints[ci.list_off + q]].flags & ITC_TEST_STALL_WAIT) != 0;
        FieldsLaunch L;
        memset(&L, 0, sizeof(L));
        L.taps = ci.taps;
        L.descs = descs;
        L.img_list = ints + ci.list_off;
        L.tile_prefix = ints + ci.prefix_off;
        L.nimg = ci.nimg;
        L.fields = v.fields;
        L.partials = v.partials;
        L.tile_h = ci.tile_h;
        L.absolute = 0;
        L.tmaps = reinterpret_cast<const CUtensorMap*>(pd + h->tmap_off);
        L.grid_per_sm = ci.grid_per_sm;
        L.mode = ci.self ? 1 : 0;
        L.status = v.status;
        L.test_stall = stall;
        // this launch's tile counter (unique per class and first image, so that range calls on
        // other streams do not share it), zeroed first
        L.counter = v.counters + ci.list_off + p0;
        if (cudaMemsetAsync(L.counter, 0, sizeof(int), s) != cudaSuccess) return ITC_ERR_CUDA;
        int rc;
        if (ci.recursive) {
            RecursiveLaunch R;
            R.descs = L.descs;
            R.fields = L.fields;
            R.partials = L.partials;
            R.img_list = L.img_list;
            R.pos_base = p0;
            R.mode = L.mode;
            rc = cuda_status(launch_recursive(R, p1 - p0, h->max_dim[0], h->max_dim[1], s));
        } else {
            rc = cuda_status(launch_fields_any(L, ci.tma != 0 && !ci.use_plain && !ci.self, t0, t1, ci.taps.R[0],
                                               ci.taps.R[1], ci.ndim, ci.dtype, s));
        }
        if (rc) return rc;
    }
    return ITC_OK;
}

int itc_run_fields_range(const void* plan_host, const void* plan_dev, int b0, int b1, void* ws, size_t ws_bytes,
                         void* stream) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h || !plan_dev || !aligned(plan_dev, 16)) return ITC_ERR_INVALID_ARG;
    if (b0 < 0 || b1 > h->B || b0 > b1) return ITC_ERR_INVALID_ARG;
    if (!ws || ws_bytes < (size_t)h->ws_bytes || !aligned(ws, 256)) return ITC_ERR_WORKSPACE;
    return fields_range(h, plan_host, plan_dev, b0, b1, full_view(h, ws), reinterpret_cast<cudaStream_t>(stream));
}

int itc_autotune(void* plan_host, void* plan_dev, void* ws, size_t ws_bytes, int reps, void* stream) {
    PlanHeader* h = const_cast<PlanHeader*>(plan_of(plan_host));
    if (!h || !plan_dev || !aligned(plan_dev, 16) || reps < 1 || reps > 1000) return ITC_ERR_INVALID_ARG;
    if (!ws || ws_bytes < (size_t)h->ws_bytes || !aligned(ws, 256)) return ITC_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* ph = reinterpret_cast<unsigned char*>(plan_host);
    ImageDesc* descs = reinterpret_cast<ImageDesc*>(ph + h->desc_off);
    int* ints = reinterpret_cast<int*>(ph + h->ints_off);
    CUtensorMap* tmaps = reinterpret_cast<CUtensorMap*>(ph + h->tmap_off);
    const size_t nbytes = plan_layout(h->B, nullptr, nullptr);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return ITC_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return ITC_ERR_CUDA; }
    int rc = ITC_OK;
    // Apply the current choices to both plan copies, then time one class's fields launches.
    auto time_class = [&](int c, float* ms) -> int {
        int r = relayout(h, descs, ints, tmaps);
        if (r) return r;
        if (cudaMemcpyAsync(plan_dev, plan_host, nbytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return ITC_ERR_CUDA;
        const ClassInfo& ci = h->cls[c];
        FieldsLaunch L;
        memset(&L, 0, sizeof(L));
        const unsigned char* pd = reinterpret_cast<const unsigned char*>(plan_dev);
        L.taps = ci.taps;
        L.descs = reinterpret_cast<const ImageDesc*>(pd + h->desc_off);
        L.img_list = reinterpret_cast<const int*>(pd + h->ints_off) + ci.list_off;
        L.tile_prefix = reinterpret_cast<const int*>(pd + h->ints_off) + ci.prefix_off;
        L.nimg = ci.nimg;
        unsigned char* w = reinterpret_cast<unsigned char*>(ws);
        L.fields = reinterpret_cast<float*>(w + h->ws_fields_off);
        L.partials = reinterpret_cast<double*>(w + h->ws_partials_off);
        L.tile_h = ci.tile_h;
        L.tmaps = reinterpret_cast<const CUtensorMap*>(pd + h->tmap_off);
        L.grid_per_sm = ci.grid_per_sm;
        L.mode = ci.self ? 1 : 0;
        L.status = reinterpret_cast<int*>(w + h->ws_status_off);
        L.counter = reinterpret_cast<int*>(w + h->ws_count_off) + ci.list_off;
        const bool tma = ci.tma && !ci.use_plain;
        for (int i = 0; i <= reps; ++i) {   // the first launch warms caches and is not timed
            if (i == 1 && cudaEventRecord(e0, s) != cudaSuccess) return ITC_ERR_CUDA;
            if (cudaMemsetAsync(L.counter, 0, sizeof(int), s) != cudaSuccess) return ITC_ERR_CUDA;
            r = cuda_status(launch_fields_any(L, tma, 0, ci.ntiles, ci.taps.R[0], ci.taps.R[1], ci.ndim, ci.dtype, s));
            if (r) return r;
        }
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return ITC_ERR_CUDA;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return ITC_ERR_CUDA;
        *ms = t / reps;
        return ITC_OK;
    };
    for (int c = 0; c < h->ncls && !rc; ++c) {
        ClassInfo& ci = h->cls[c];
        if (ci.ndim != 2 || ci.self || ci.recursive) continue;   // one configuration for these
        struct Cand { int plain, tile_h, grid; };
        Cand cands[6];
        int nc = 0;
        if (ci.tma) {
            cands[nc++] = {0, 64, 0};
            cands[nc++] = {0, 64, 1};
            cands[nc++] = {0, 32, 0};
            cands[nc++] = {0, 32, 1};
            cands[nc++] = {0, 128, 0};
        }
        cands[nc++] = {1, 64, 0};
        float best = 3.4e38f;
        Cand pick = cands[0];
        for (int i = 0; i < nc && !rc; ++i) {
            ci.use_plain = cands[i].plain;
            ci.tile_h = cands[i].tile_h;
            ci.grid_per_sm = cands[i].grid;
            float ms = 0.f;
            rc = time_class(c, &ms);
            if (!rc && ms < best) { best = ms; pick = cands[i]; }
        }
        ci.use_plain = pick.plain;
        ci.tile_h = pick.tile_h;
        ci.grid_per_sm = pick.grid;
        ci.tuned_ms = best;
    }
    if (!rc) rc = relayout(h, descs, ints, tmaps);
    if (!rc && cudaMemcpyAsync(plan_dev, plan_host, nbytes, cudaMemcpyHostToDevice, s) != cudaSuccess) rc = ITC_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = ITC_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int itc_plan_class(const void* plan_host, int c, int* ndim, float* sigma, int* tile_h, int* grid_per_sm,
                   int* staging, int* images, float* tuned_ms) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h || c < 0 || c >= h->ncls) return ITC_ERR_INVALID_ARG;
    const ClassInfo& ci = h->cls[c];
    if (ndim) *ndim = ci.ndim;
    if (sigma) for (int i = 0; i < 3; ++i) sigma[i] = ci.taps.sigma[i];
    if (tile_h) *tile_h = ci.tile_h;
    if (grid_per_sm) *grid_per_sm = ci.grid_per_sm;
    if (staging) *staging = ci.recursive ? 3 : (ci.self ? 2 : ((ci.tma && !ci.use_plain) ? 1 : 0));
    if (images) *images = ci.nimg;
    if (tuned_ms) *tuned_ms = ci.tuned_ms;
    return ITC_OK;
}

int itc_plan_configure(void* plan_host, void* plan_dev, int c, int tile_h, int grid_per_sm, int staging,
                       void* stream) {
    PlanHeader* h = const_cast<PlanHeader*>(plan_of(plan_host));
    if (!h || !plan_dev || !aligned(plan_dev, 16) || c < 0 || c >= h->ncls) return ITC_ERR_INVALID_ARG;
    if (grid_per_sm < 0 || grid_per_sm > 64 || (staging != 0 && staging != 1)) return ITC_ERR_INVALID_ARG;
    ClassInfo& ci = h->cls[c];
    if (ci.self || ci.recursive) return ITC_ERR_UNSUPPORTED;   // one configuration for these
    if (staging == 1 && !ci.tma) return ITC_ERR_UNSUPPORTED;
    if (staging == 1 ? (tile_h != 32 && tile_h != 64 && tile_h != 128) : tile_h != tile_h_of(ci.ndim))
        return ITC_ERR_INVALID_ARG;
    ci.use_plain = staging ? 0 : 1;
    ci.tile_h = tile_h;
    ci.grid_per_sm = grid_per_sm;
    unsigned char* ph = reinterpret_cast<unsigned char*>(plan_host);
    int rc = relayout(h, reinterpret_cast<ImageDesc*>(ph + h->desc_off), reinterpret_cast<int*>(ph + h->ints_off),
                      reinterpret_cast<CUtensorMap*>(ph + h->tmap_off));
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(plan_dev, plan_host, plan_layout(h->B, nullptr, nullptr), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ITC_ERR_CUDA;
    return ITC_OK;
}

int itc_params_parzen(int ndim, const float* xi, const float* omega, double mass, int M, float trunc,
                      int iters, int form, int flags, itc_params* out) {
    if (!out || (ndim != 2 && ndim != 3) || (form != 0 && form != 1)) return ITC_ERR_INVALID_ARG;
    double x[3], o[3];
    const bool schedule = mass > 0.0 && M > 0;
    for (int i = 0; i < ndim; ++i) {
        if (schedule) {
            // Sec. 4: omega = sqrt(N / M) / 2, xi = omega / 2
            o[i] = sqrt(mass / M) / 2.0;
            x[i] = o[i] / 2.0;
        } else {
            if (!xi || !omega) return ITC_ERR_INVALID_ARG;
            x[i] = xi[i];
            o[i] = omega[i];
        }
        if (!(x[i] > 0.0) || !(o[i] > 0.0) || !isfinite(x[i]) || !isfinite(o[i])) return ITC_ERR_INVALID_ARG;
    }
    itc_params p;
    memset(&p, 0, sizeof(p));
    double step = 1.0;
    for (int i = 0; i < ndim; ++i) {
        const double t2 = x[i] * x[i] + o[i] * o[i];
        p.sigma[i] = (float)sqrt(t2);
        p.sigma_pair[i] = (float)(sqrt(2.0) * o[i]);
        p.sigma_self[i] = (float)(sqrt(2.0) * x[i]);
        const double si = o[i] * o[i] / t2;
        if (form == 1) {
            if (i > 0 && fabs(si - step) > 1e-12 * step) return ITC_ERR_INVALID_ARG;
            step = si;
        }
    }
    p.trunc = trunc;
    p.iters = iters;
    p.step_scale = (float)step;
    p.flags = flags;
    *out = p;
    return ITC_OK;
}

long long itc_plan_padded_offset(const void* plan_host, int b) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h || b < 0 || b > h->B) return ITC_ERR_INVALID_ARG;
    if (b == h->B) return h->pad_floats;
    const ImageDesc* descs = reinterpret_cast<const ImageDesc*>(reinterpret_cast<const unsigned char*>(plan_host) +
                                                                h->desc_off);
    return descs[b].pad_off;
}

int itc_chamfer(const void* plan_host, const void* plan_dev, float* out, void* stream) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h || !plan_dev || !aligned(plan_dev, 16) || !out || !aligned(out, 16)) return ITC_ERR_INVALID_ARG;
    const ImageDesc* descs = reinterpret_cast<const ImageDesc*>(reinterpret_cast<const unsigned char*>(plan_host) +
                                                                h->desc_off);
    for (int b = 0; b < h->B; ++b) {
        if (descs[b].ndim != 2 || descs[b].dtype != ITC_U8) return ITC_ERR_INVALID_ARG;
        if (descs[b].W > kChamferMaxW) return ITC_ERR_UNSUPPORTED;
    }
    const unsigned char* pd = reinterpret_cast<const unsigned char*>(plan_dev);
    ChamferLaunch L;
    L.descs = reinterpret_cast<const ImageDesc*>(pd + h->desc_off);
    L.out = out;
    L.order = reinterpret_cast<const int*>(pd + h->ints_off) + h->bwd_order_off;
    L.B = h->B;
    return cuda_status(launch_chamfer(L, h->max_dim[1], reinterpret_cast<cudaStream_t>(stream)));
}

int itc_segment(const void* plan_host, const void* plan_dev, const float* W, short* labels, void* stream) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h || !plan_dev || !aligned(plan_dev, 16) || !W || !labels) return ITC_ERR_INVALID_ARG;
    if (!aligned(W, 4) || !aligned(labels, 2)) return ITC_ERR_INVALID_ARG;
    const unsigned char* pd = reinterpret_cast<const unsigned char*>(plan_dev);
    SegmentLaunch L;
    L.descs = reinterpret_cast<const ImageDesc*>(pd + h->desc_off);
    L.W = W;
    L.labels = labels;
    L.order = reinterpret_cast<const int*>(pd + h->ints_off) + h->bwd_order_off;
    return cuda_status(launch_segment(L, h->B, h->max_M, reinterpret_cast<cudaStream_t>(stream)));
}

int itc_plan_classes(const void* plan_host) {
    const PlanHeader* h = plan_of(plan_host);
    return h ? h->ncls : ITC_ERR_INVALID_ARG;
}

static int run_iterate_images(const void* plan_host, const void* plan_dev, int b0, int b1, bool whole, float* W,
                              itc_stats* stats, void* ws, size_t ws_bytes, void* stream);

int itc_run_iterate_range(const void* plan_host, const void* plan_dev, int b0, int b1, float* W, itc_stats* stats,
                          void* ws, size_t ws_bytes, void* stream) {
    return run_iterate_images(plan_host, plan_dev, b0, b1, false, W, stats, ws, ws_bytes, stream);
}

// The iterations of images [b0, b1) in order (one image per CTA), or (whole) of every image of the
// plan in the plan's iteration order (grouped CTAs), on the fields of view v.
static int iterate_images(const PlanHeader* h, const void* plan_dev, int b0, int b1, bool whole, float* W,
                          itc_stats* stats, const WsView& v, cudaStream_t s) {
    if (b1 == b0) return ITC_OK;
    const unsigned char* pd = reinterpret_cast<const unsigned char*>(plan_dev);
    RunLaunch R;
    memset(&R, 0, sizeof(R));
    R.descs = reinterpret_cast<const ImageDesc*>(pd + h->desc_off);
    R.fields = v.fields;
    R.partials = v.partials;
    R.W_in = W;
    R.W_out = W;
    R.stats = stats;
    R.absolute = 0;
    R.final_eval = 1;
    R.img_base = b0;
    R.img_status = v.status;
    const bool grouped = whole && b0 == 0 && b1 == h->B;
    const int* groups = reinterpret_cast<const int*>(pd + h->ints_off) + h->run_groups_off;
    for (int nd = 2; nd <= 3; ++nd) {
        if (!(h->ndim_mask & (1 << nd))) continue;
        int ctas = b1 - b0;
        if (grouped) {
            // the 3-D groups follow the 2-D ones
            R.groups = groups + (nd == 3 ? (size_t)h->run_ngroups[0] * kGroupInts : 0);
            ctas = h->run_ngroups[nd - 2];
        }
        const int rc = cuda_status(launch_run(R, ctas, h->max_M, h->max_dim, s, nd));
        if (rc) return rc;
    }
    return ITC_OK;
}

static int run_iterate_images(const void* plan_host, const void* plan_dev, int b0, int b1, bool whole, float* W,
                              itc_stats* stats, void* ws, size_t ws_bytes, void* stream) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h || !plan_dev || !W || !aligned(plan_dev, 16)) return ITC_ERR_INVALID_ARG;
    if (b0 < 0 || b1 > h->B || b0 > b1) return ITC_ERR_INVALID_ARG;
    if (!ws || ws_bytes < (size_t)h->ws_bytes || !aligned(ws, 256)) return ITC_ERR_WORKSPACE;
    return iterate_images(h, plan_dev, b0, b1, whole, W, stats, full_view(h, ws), reinterpret_cast<cudaStream_t>(stream));
}

int itc_run_fields(const void* plan_host, const void* plan_dev, void* ws, size_t ws_bytes, void* stream) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h) return ITC_ERR_INVALID_ARG;
    return itc_run_fields_range(plan_host, plan_dev, 0, h->B, ws, ws_bytes, stream);
}

int itc_run_iterate(const void* plan_host, const void* plan_dev, float* W, itc_stats* stats, void* ws,
                    size_t ws_bytes, void* stream) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h) return ITC_ERR_INVALID_ARG;
    return run_iterate_images(plan_host, plan_dev, 0, h->B, true, W, stats, ws, ws_bytes, stream);
}

int itc_run_pipelined(const void* plan_host, const void* plan_dev, float* W, itc_stats* stats, void* ws,
                      size_t ws_bytes, void* stream, void* stream2, int chunks) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h || !plan_dev || !W || chunks < 1 || chunks > 64) return ITC_ERR_INVALID_ARG;
    if (!ws || ws_bytes < (size_t)h->ws_bytes || !aligned(ws, 256)) return ITC_ERR_WORKSPACE;
    if (chunks == 1 || !stream2 || stream2 == stream) return itc_run(plan_host, plan_dev, W, stats, ws, ws_bytes, stream);
    cudaStream_t s1 = reinterpret_cast<cudaStream_t>(stream), s2 = reinterpret_cast<cudaStream_t>(stream2);
    const int n = chunks < h->B ? chunks : h->B;
    cudaEvent_t ev[65];
    int made = 0, rc = ITC_OK;
    for (; made <= n; ++made)
        if (cudaEventCreateWithFlags(&ev[made], cudaEventDisableTiming) != cudaSuccess) { rc = ITC_ERR_CUDA; break; }
    // the second stream starts after everything the caller queued on the first
    if (!rc) rc = cuda_status(cudaEventRecord(ev[n], s1));
    if (!rc) rc = cuda_status(cudaStreamWaitEvent(s2, ev[n], 0));
    for (int k = 0; k < n && !rc; ++k) {
        const int b0 = (int)((long long)h->B * k / n), b1 = (int)((long long)h->B * (k + 1) / n);
        rc = itc_run_fields_range(plan_host, plan_dev, b0, b1, ws, ws_bytes, s1);
        if (!rc) rc = cuda_status(cudaEventRecord(ev[k], s1));
        if (!rc) rc = cuda_status(cudaStreamWaitEvent(s2, ev[k], 0));
        if (!rc) rc = itc_run_iterate_range(plan_host, plan_dev, b0, b1, W, stats, ws, ws_bytes, s2);
    }
    // join: the first stream continues after the last iterations
    if (!rc) rc = cuda_status(cudaEventRecord(ev[n], s2));
    if (!rc) rc = cuda_status(cudaStreamWaitEvent(s1, ev[n], 0));
    for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);   // released once the work has run
    return rc;
}

// Bytes [lo, hi) of the device image buffer that images [b0, b1) occupy (data and weights).
static bool image_extent(const ImageDesc* d, int b0, int b1, const unsigned char* base, size_t bytes, size_t* lo,
                         size_t* hi) {
    size_t a = bytes, z = 0;
    for (int b = b0; b < b1; ++b) {
        const size_t es = d[b].dtype == ITC_F32 ? 4 : 1;
        const size_t ext = ((size_t)(d[b].H - 1) * d[b].pitch + d[b].W);
        const void* ptrs[2] = {d[b].data, d[b].weight};
        const size_t sz[2] = {ext * es, ext * 4};
        for (int q = 0; q < 2; ++q) {
            if (!ptrs[q]) continue;
            const unsigned char* p = reinterpret_cast<const unsigned char*>(ptrs[q]);
            if (p < base || (size_t)(p - base) + sz[q] > bytes) return false;
            a = std::min(a, (size_t)(p - base));
            z = std::max(z, (size_t)(p - base) + sz[q]);
        }
    }
    *lo = a < z ? a : 0;
    *hi = a < z ? z : 0;
    return true;
}

int itc_run_staged(const void* plan_host, const void* plan_dev, const void* host_base, void* dev_base, size_t bytes,
                   float* W, itc_stats* stats, void* ws, size_t ws_bytes, int chunks, void* stream, void* copy_stream) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h || !plan_dev || !W || !host_base || !dev_base || chunks < 1 || chunks > 64) return ITC_ERR_INVALID_ARG;
    if (!ws || ws_bytes < (size_t)h->ws_bytes || !aligned(ws, 256)) return ITC_ERR_WORKSPACE;
    const ImageDesc* descs = reinterpret_cast<const ImageDesc*>(reinterpret_cast<const unsigned char*>(plan_host) +
                                                                h->desc_off);
    const unsigned char* base = reinterpret_cast<const unsigned char*>(dev_base);
    const int n = chunks < h->B ? chunks : h->B;
    std::vector<size_t> lo(n), hi(n);
    for (int k = 0; k < n; ++k) {
        const int b0 = (int)((long long)h->B * k / n), b1 = (int)((long long)h->B * (k + 1) / n);
        if (!image_extent(descs, b0, b1, base, bytes, &lo[k], &hi[k])) return ITC_ERR_INVALID_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaStream_t cs = copy_stream ? reinterpret_cast<cudaStream_t>(copy_stream) : s;
    cudaEvent_t ev[65];
    int made = 0, rc = ITC_OK;
    for (; made <= n; ++made)
        if (cudaEventCreateWithFlags(&ev[made], cudaEventDisableTiming) != cudaSuccess) { rc = ITC_ERR_CUDA; break; }
    // the copies start after the work already queued on `stream` (it may still read the buffer)
    if (!rc && cs != s) rc = cuda_status(cudaEventRecord(ev[n], s));
    if (!rc && cs != s) rc = cuda_status(cudaStreamWaitEvent(cs, ev[n], 0));
    for (int k = 0; k < n && !rc; ++k) {
        if (hi[k] > lo[k])
            rc = cuda_status(cudaMemcpyAsync(const_cast<unsigned char*>(base) + lo[k],
                                             reinterpret_cast<const unsigned char*>(host_base) + lo[k], hi[k] - lo[k],
                                             cudaMemcpyHostToDevice, cs));
        if (!rc && cs != s) rc = cuda_status(cudaEventRecord(ev[k], cs));
    }
    // the fields of each range as soon as its bytes have landed; then the iterations of the whole
    // batch in one launch (one CTA per image needs the whole batch to fill the GPU)
    for (int k = 0; k < n && !rc; ++k) {
        const int b0 = (int)((long long)h->B * k / n), b1 = (int)((long long)h->B * (k + 1) / n);
        if (cs != s) rc = cuda_status(cudaStreamWaitEvent(s, ev[k], 0));
        if (!rc) rc = itc_run_fields_range(plan_host, plan_dev, b0, b1, ws, ws_bytes, s);
    }
    if (!rc) rc = itc_run_iterate(plan_host, plan_dev, W, stats, ws, ws_bytes, s);
    for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);   // released once the work has run
    return rc;
}

int itc_run(const void* plan_host, const void* plan_dev, float* W, itc_stats* stats, void* ws,
            size_t ws_bytes, void* stream) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h || !plan_dev || !W || !aligned(plan_dev, 16)) return ITC_ERR_INVALID_ARG;
    int rc = itc_run_fields(plan_host, plan_dev, ws, ws_bytes, stream);
    if (rc) return rc;
    return itc_run_iterate(plan_host, plan_dev, W, stats, ws, ws_bytes, stream);
}

// The backward of images [b0, b1) (whole: every image, in the plan's backward order) on the
// fields and S_XX partials of view v.
static int backward_images(const PlanHeader* h, const void* plan_host, const void* plan_dev, int b0, int b1,
                           bool whole, const float* W, const float* grad_dcs, float* grad_W, float* grad_h,
                           itc_stats* stats, const WsView& v, cudaStream_t s) {
    if (b1 == b0) return ITC_OK;
    const unsigned char* pd = reinterpret_cast<const unsigned char*>(plan_dev);
    BackwardLaunch L;
    memset(&L, 0, sizeof(L));
    L.descs = reinterpret_cast<const ImageDesc*>(pd + h->desc_off);
    L.fields = v.fields;
    L.partials = v.partials;
    L.W = W;
    L.grad_dcs = grad_dcs;
    L.grad_W = grad_W;
    L.grad_h = grad_h;
    L.stats = stats;
    L.scal = v.scal;
    L.B = h->B;
    L.img_status = v.status;
    if (whole) {
        L.bwd_order = reinterpret_cast<const int*>(pd + h->ints_off) + h->bwd_order_off;
        return cuda_status(launch_backward(L, h->B, h->max_M, h->bwd_tiles, h->max_bwd_tiles, s));
    }
    // an image range: its CTAs in image order
    const ImageDesc* hd = reinterpret_cast<const ImageDesc*>(reinterpret_cast<const unsigned char*>(plan_host) +
                                                             h->desc_off);
    long long tiles = 0;
    int max_tiles = 0, max_M = 0;
    for (int b = b0; b < b1; ++b) {
        const int t = hd[b].bwd_tiles_u * hd[b].bwd_tiles_v;
        tiles += t;
        max_tiles = std::max(max_tiles, t);
        max_M = std::max(max_M, hd[b].M);
    }
    L.bwd_order = nullptr;
    L.img_base = b0;
    return cuda_status(launch_backward(L, b1 - b0, max_M, tiles, max_tiles, s));
}

int itc_backward(const void* plan_host, const void* plan_dev, const float* W, const float* grad_dcs,
                 float* grad_W, float* grad_h, itc_stats* stats, void* ws, size_t ws_bytes, void* stream) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h || !plan_dev || !W || !aligned(plan_dev, 16)) return ITC_ERR_INVALID_ARG;
    if (!ws || ws_bytes < (size_t)h->ws_bytes || !aligned(ws, 256)) return ITC_ERR_WORKSPACE;
    // the adjoint stamps truncated kernel boxes; recursive fields have none
    if (h->has_recursive) return ITC_ERR_UNSUPPORTED;
    return backward_images(h, plan_host, plan_dev, 0, h->B, true, W, grad_dcs, grad_W, grad_h, stats,
                           full_view(h, ws), reinterpret_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------------ budgeted (recomputing) calls

size_t itc_plan_budget_bytes(const void* plan_host, size_t budget_bytes) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h) return 0;
    const ImageDesc* d = reinterpret_cast<const ImageDesc*>(reinterpret_cast<const unsigned char*>(plan_host) +
                                                            h->desc_off);
    long long largest = 0;
    for (int b = 0; b < h->B; ++b) largest = std::max(largest, field_span(h, d, b));
    const size_t least = budget_tail_bytes(h) + align_up((size_t)largest * sizeof(float), 256);
    return std::max(budget_bytes / 256 * 256, least);
}

// Cuts the plan into image ranges whose fields fit the window of a budgeted workspace of
// ws_bytes; ITC_ERR_WORKSPACE if it is smaller than itc_plan_budget_bytes(plan, 0).
static int budget_ranges(const PlanHeader* h, const ImageDesc* d, size_t ws_bytes, std::vector<int>* cuts) {
    const size_t tail = budget_tail_bytes(h);
    if (ws_bytes < tail) return ITC_ERR_WORKSPACE;
    const long long window = (long long)((ws_bytes - tail) / sizeof(float));
    cuts->assign(1, 0);
    long long used = 0;
    for (int b = 0; b < h->B; ++b) {
        const long long span = field_span(h, d, b);
        if (span > window) return ITC_ERR_WORKSPACE;
        if (used + span > window) {
            cuts->push_back(b);
            used = 0;
        }
        used += span;
    }
    cuts->push_back(h->B);
    return ITC_OK;
}

int itc_run_budget(const void* plan_host, const void* plan_dev, float* W, itc_stats* stats, void* ws,
                   size_t ws_bytes, void* stream) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h || !plan_dev || !W || !aligned(plan_dev, 16)) return ITC_ERR_INVALID_ARG;
    if (!ws || !aligned(ws, 256)) return ITC_ERR_WORKSPACE;
    const ImageDesc* hd = reinterpret_cast<const ImageDesc*>(reinterpret_cast<const unsigned char*>(plan_host) +
                                                             h->desc_off);
    std::vector<int> cuts;
    int rc = budget_ranges(h, hd, ws_bytes, &cuts);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (size_t r = 0; r + 1 < cuts.size() && !rc; ++r) {
        const WsView v = budget_view(h, ws, hd, cuts[r]);
        rc = fields_range(h, plan_host, plan_dev, cuts[r], cuts[r + 1], v, s);
        if (!rc) rc = iterate_images(h, plan_dev, cuts[r], cuts[r + 1], false, W, stats, v, s);
    }
    return rc;
}

int itc_backward_budget(const void* plan_host, const void* plan_dev, const float* W, const float* grad_dcs,
                        float* grad_W, float* grad_h, itc_stats* stats, void* ws, size_t ws_bytes, void* stream) {
    const PlanHeader* h = plan_of(plan_host);
    if (!h || !plan_dev || !W || !aligned(plan_dev, 16)) return ITC_ERR_INVALID_ARG;
    if (!ws || !aligned(ws, 256)) return ITC_ERR_WORKSPACE;
    if (h->has_recursive) return ITC_ERR_UNSUPPORTED;
    const ImageDesc* hd = reinterpret_cast<const ImageDesc*>(reinterpret_cast<const unsigned char*>(plan_host) +
                                                             h->desc_off);
    std::vector<int> cuts;
    int rc = budget_ranges(h, hd, ws_bytes, &cuts);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (size_t r = 0; r + 1 < cuts.size() && !rc; ++r) {
        const WsView v = budget_view(h, ws, hd, cuts[r]);
        rc = fields_range(h, plan_host, plan_dev, cuts[r], cuts[r + 1], v, s);
        if (!rc)
            rc = backward_images(h, plan_host, plan_dev, cuts[r], cuts[r + 1], false, W, grad_dcs, grad_W, grad_h,
                                 stats, v, s);
    }
    return rc;
}

}  // extern "C"
