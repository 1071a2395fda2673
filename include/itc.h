/*
 * itc.h -- C ABI of libitc.so: lattice information-theoretic clustering on one GPU
 * (C. Bauckhage, K. Kersting, "Efficient Information Theoretic Clustering on Discrete Lattices",
 * arXiv:1310.7114).
 *
 * Problem (Sec. 2.1): given data on a lattice -- a binary image X (Sec. 3.2), a per-pixel weight
 * image h (Sec. 5) or a gray image read as a 3-D [u, v, g] occupancy lattice (Sec. 1 (ii)) -- and
 * an initial codebook W = {w_1..w_M}, move W to minimise the Cauchy-Schwarz divergence of
 * Eq. (1) between the Parzen densities p = h * G and q = W * G (Eq. (dens1), (dens2)).
 * Following Sec. 3.1 the data sums are read from precomputed, truncated, separable Gaussian
 * fields; Algorithm 1 iterates the fixed-point update of Eq. (origupdate) with those fields.
 *
 * Conventions shared by every entry point
 *   - Coordinates: u = row (slow axis), v = column (fast axis), g = gray level.  A codebook
 *     vector is stored as (u, v) or (u, v, g) floats; W arrays are [M][ndim] row-major.
 *   - Kernel: g(d) = prod_i exp(-d_i^2 / (2 sigma_i^2)) (unnormalised).  sigma is the width of
 *     the product kernels tau = rho of Sec. 2.1 (xi = omega = sigma / sqrt 2), so the three
 *     overlap integrals of Eq. (1) share one kernel and D_cs = log S_WW + log S_XX - 2 log S_XW.
 *   - Truncation (Sec. 3.1, finite filter masks): data sums run over the box
 *     |x_i - y_i| <= R_i, R_i = ceil(trunc * sigma_i); taps are not renormalised; sites
 *     outside the lattice hold no data.  Codebook-codebook sums are not truncated.
 *   - Fields: planar FP32, plane p of an image is [G][H][fpitch] floats with
 *     fpitch = itc_field_pitch(W) (a multiple of 4); planes are A, F_u, F_v (, F_g):
 *       A(y)   = sum_x h(x) g(x - y)
 *       F_i(y) = sum_x h(x) g(x - y) (x_i - y_i)   (centred moments, default)
 *       F_i(y) = sum_x h(x) g(x - y) x_i           (ITC_FIELDS_ABSOLUTE: the convolution of the
 *                                                   coordinate-weighted image u.X, v.X, g.X)
 *   - Memory: every data pointer is a DEVICE pointer unless its comment says "host".  The caller
 *     owns every buffer; the library allocates no device memory and keeps no global state.
 *     Scratch memory is caller-provided `ws` of at least the size the matching *_bytes query
 *     returns.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Every call only
 *     enqueues work and returns; results are valid once the stream has reached them.
 *   - Errors: 0 = success; negative = error (nothing was launched unless ITC_ERR_CUDA says a
 *     launch failed); positive = warning.  Per-image device status goes to itc_stats.status.
 */
#ifndef ITC_H
#define ITC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------- status codes */
#define ITC_OK 0
#define ITC_WARN_EMPTY_SUPPORT 1   /* device status: some w_k had no data in its window (kept) */
#define ITC_ERR_INVALID_ARG (-1)   /* bad pointer, size, sigma, flag or layout */
#define ITC_ERR_CUDA (-2)          /* a CUDA launch or query failed */
#define ITC_ERR_TIMEOUT (-3)       /* a bounded device wait gave up */
#define ITC_ERR_NONFINITE (-4)     /* device status: S_XW = 0 or a non-finite value appeared */
#define ITC_ERR_WORKSPACE (-5)     /* workspace missing, too small or misaligned */
#define ITC_ERR_UNSUPPORTED (-6)   /* valid request outside the library's compiled limits */

/* --------------------------------------------------------------------------- data types */
#define ITC_U8 0   /* 2-D: occupancy 0/1 (binary image X of Sec. 3.2); 3-D: gray level */
#define ITC_F32 1  /* 2-D: weights h >= 0 (weighted ITC, Sec. 5) */

/* -------------------------------------------------------------------------------- flags */
#define ITC_CONTINUOUS 1       /* keep W real (lookups at the rounded site); default snaps W to
                                  the lattice after every update (W as an image, Sec. 3.2) */
#define ITC_FIELDS_ABSOLUTE 2  /* itc_fields writes u.X, v.X (, g.X) convolutions, not centred */
#define ITC_STOP_ON_FIXED 4    /* stop when an iteration moves no codebook (theta = 0 test of
                                  Algorithm 1) */
#define ITC_RECURSIVE 8        /* 2-D plans only: fields by recursive filtering instead of masks
                                  (Sec. 3.1, for large widths): Deriche's fit of the Gaussian by
                                  two damped sinusoids, untruncated, cost independent of sigma;
                                  no radius limit.  itc_fields rejects it (ITC_ERR_UNSUPPORTED);
                                  itc_backward rejects plans that use it */
#define ITC_TEST_STALL_WAIT 256 /* test hook (tensor-tile fields path only): the first tile copy
                                  of the first CTA of the fields launch is never started, so that
                                  CTA's bounded wait (about one second) runs out.  itc_fields then
                                  reports ITC_ERR_TIMEOUT in its workspace status word and
                                  S_XX = NaN; in a plan (any image of a fields launch carrying the
                                  flag arms it) the images of that CTA's tiles get the status
                                  ITC_ERR_TIMEOUT in itc_stats.  Nothing else is affected and the
                                  GPU stays usable.  Never set otherwise. */

/* Compiled limits of the library. */
#define ITC_MAX_RADIUS_UV 32   /* R_u, R_v */
#define ITC_MAX_RADIUS_UV_3D 24 /* R_u, R_v of 3-D gray lattices */
#define ITC_MAX_RADIUS_G 64    /* R_g */
#define ITC_MAX_M 2048         /* codebook vectors per image */
#define ITC_MAX_GRAY 256       /* G */

/* One lattice image.  `data` and `weight` are device pointers. */
typedef struct {
    int ndim;            /* 2: binary or weighted image; 3: gray image as [u, v, g] lattice */
    int H, W;            /* rows (u) and columns (v) */
    int G;               /* ndim 3: gray levels (lattice depth along g, <= 256); ndim 2: 1 */
    int pitch;           /* elements between consecutive rows of `data` and `weight` (>= W) */
    int dtype;           /* ITC_U8 or ITC_F32 (ITC_F32 only for ndim 2) */
    const void* data;    /* H rows of `pitch` elements */
    const float* weight; /* ndim 3 only: per-pixel weight h(u, v) >= 0, or NULL for 1 */
} itc_image;

/* Method parameters (host struct, passed by pointer, read during the call). */
typedef struct {
    float sigma[3];      /* kernel width per axis (u, v, g), lattice units, > 0: the width tau of
                            the data-codebook overlap V(X;W) (tau^2 = xi^2 + omega^2, Sec. 2.1);
                            the fields are convolutions with it */
    float trunc;         /* mask half width in sigmas: R_i = ceil(trunc * sigma_i); paper: small
                            masks (Sec. 3.1); 3 is the usual choice */
    int iters;           /* fixed-point iterations (Algorithm 1 loop), >= 0 */
    float step_scale;    /* 1: the fixed-point form of Eq. (origupdate); Eq. (accupdate)
                            evaluated exactly moves by omega^2 / tau^2 of that step (0.5 when
                            xi = omega) */
    int flags;           /* ITC_CONTINUOUS | ITC_FIELDS_ABSOLUTE | ITC_STOP_ON_FIXED */
    float sigma_pair[3]; /* width rho of the codebook overlap V(W) (rho^2 = 2 omega^2); 0 = sigma.
                            The pair terms of the update carry tau^2 / rho^2 per axis, the factor
                            that differentiating Eq. (1) gives (Eq. (origupdate) as printed omits
                            it; the two agree when tau = rho) */
    float sigma_self[3]; /* width s of the data overlap V(X) (s^2 = 2 xi^2); 0 = sigma.  A width
                            other than sigma costs one more fields pass (A only) per call */
} itc_params;

/* Per-image results, written by the device. */
typedef struct {
    double dcs;          /* D_cs of Eq. (1) at the reported W (+inf if S_XW == 0) */
    double sxw, sww, sxx;/* the three sums of Eq. (1) */
    double c;            /* S_XW / S_WW, the constant c of Eq. (origupdate) */
    int empty;           /* codebooks with no data in their window in the last evaluation */
    int moved;           /* codebooks moved by the last update */
    int iters_done;      /* updates applied */
    int status;          /* ITC_OK, ITC_WARN_EMPTY_SUPPORT, ITC_ERR_NONFINITE, or ITC_ERR_TIMEOUT
                            when a bounded wait of the image's fields pass gave up (its fields are
                            then incomplete and S_XX is NaN) */
} itc_stats;

/* --------------------------------------------------------------- parameters from xi, omega */

/*
 * itc_params_parzen -- method parameters from the Parzen widths of Eq. (dens1) (xi, data) and
 * Eq. (dens2) (omega, codebook), per axis (ndim values each), by the Gaussian product theorem of
 * Sec. 2.1: sigma = tau = sqrt(xi^2 + omega^2), sigma_pair = rho = sqrt(2) omega,
 * sigma_self = sqrt(2) xi; step_scale = 1 (form 0, the fixed point of Eq. (origupdate)) or
 * omega^2 / tau^2 (form 1, Eq. (accupdate) evaluated exactly; it must then be the same on every
 * axis).  D_cs then includes the normalising constant 1/2 sum_i log(tau_i^4 / (rho_i^2 s_i^2)).
 * When mass > 0 and M > 0 the widths are instead the paper's schedule of Sec. 4,
 * omega = sqrt(mass / M) / 2 and xi = omega / 2 on every axis (mass = number of foreground
 * pixels, or the total weight), and xi, omega are ignored (may be NULL).
 * Errors: ITC_ERR_INVALID_ARG (non-positive width, ndim not 2 or 3, form 1 with axis-dependent
 * omega^2 / tau^2).  Host-only.
 */
int itc_params_parzen(int ndim, const float* xi, const float* omega, double mass, int M,
                      float trunc, int iters, int form, int flags, itc_params* out);

/* ------------------------------------------------------------------------------ queries */

/* Row pitch (floats) of every field plane of an image W columns wide: W rounded up to 4. */
int itc_field_pitch(int W);

/* Bytes of the field planes of `img` (ndim+1 planes of G*H*itc_field_pitch(W) floats);
 * 0 if img is invalid. */
size_t itc_fields_bytes(const itc_image* img);

/* Scratch bytes itc_fields needs for `img` (a 256-byte status slot, then per-tile S_XX partial
 * sums); 0 if invalid. */
size_t itc_fields_workspace_bytes(const itc_image* img);

/* Message for a status code (static string). */
const char* itc_status_string(int code);

/* ------------------------------------------------------------------------------ fields */
/*
 * itc_fields -- step 2 of Algorithm 1, P = X * G (Sec. 3.1; weighted P = h * G, Sec. 5):
 * the truncated separable Gaussian fields of one image and S_XX = sum_x h(x) A(x) (the V(X)
 * term of Eq. (1)).
 *   img    : the image (host struct; data on device)
 *   p      : sigma, trunc and ITC_FIELDS_ABSOLUTE are used
 *   fields : device, itc_fields_bytes(img) bytes, 16-byte aligned; written
 *   sxx    : device double, written (may be NULL)
 *   ws     : device scratch of itc_fields_workspace_bytes(img) bytes, 16-byte aligned.  Its first
 *            int is the call's device status, written on the stream: ITC_OK, or ITC_ERR_TIMEOUT
 *            when a bounded wait of the fields pass gave up (the fields of the tiles its CTA still
 *            owned are then not written, and S_XX is NaN).  It is the only signal when sxx is
 *            NULL; read it after the stream has reached the call.
 * Errors: ITC_ERR_INVALID_ARG (bad image/params/pointer), ITC_ERR_WORKSPACE, ITC_ERR_CUDA.
 */
int itc_fields(const itc_image* img, const itc_params* p, float* fields, double* sxx,
               void* ws, size_t ws_bytes, void* stream);

/*
 * itc_fields_noalloc -- itc_fields for callers that cannot allocate device memory.  The paper
 * has no counterpart: this is a deployment variant.  Some hosts give a library only the input
 * and output buffers and forbid any allocation while they run (plugin and real-time hosts with
 * a fixed memory budget, or code that must not call cudaMalloc while it records work); they
 * cannot provide itc_fields' scratch.  This entry point keeps that scratch (a status slot and
 * one double per fields tile) in a fixed device array inside the library, 256 bytes plus
 * ITC_NOALLOC_MAX_TILES doubles (512 KiB), which every GPU that loads the library holds until
 * the process exits.  A bounded wait that gives up shows here only as S_XX = NaN (pass sxx).
 *   Same arguments and results as itc_fields, without ws / ws_bytes.  Allocates nothing.
 *   The first call on each device looks up the array's device address (cudaGetSymbolAddress,
 *   with that device current); make that first call before any stream capture.
 *   All calls share the one array: calls whose work overlaps on a GPU (other streams, other
 *   host threads) race on it and must be serialised by the caller.  The array keeps the last
 *   call's partial sums; each call sets its status word to ITC_OK first and overwrites every
 *   partial it reads, so nothing else is cleared.
 * Errors: ITC_ERR_UNSUPPORTED if the image needs more than ITC_NOALLOC_MAX_TILES tiles (2-D:
 * ceil(H/64) ceil(W/64); 3-D: ceil(H/32) ceil(W/64) G, one tile per gray slice); otherwise as itc_fields.
 */
#define ITC_NOALLOC_MAX_TILES 65536
int itc_fields_noalloc(const itc_image* img, const itc_params* p, float* fields, double* sxx,
                       void* stream);

/* ---------------------------------------------------------------------- one update step */
/*
 * itc_step -- one iteration of Algorithm 1 (steps 4-10): gather A and the moments at the
 * lattice-rounded codebook sites, add the M x M codebook interaction sums, apply Eq. (origupdate)
 * in the centred form w_k' = w_k + step_scale (D_k - c E_k) / a_k with c = S_XW / S_WW, then
 * (default) round w_k' to the lattice, floor(x + 0.5) clamped to the image.  All codebooks read
 * the same old W (Jacobi).  A codebook with a_k = 0 keeps its position (status warning).
 *   fields    : device, from itc_fields with the same img/p (centred or absolute, per p->flags)
 *   sxx       : device double from itc_fields (required; used for the D_cs in stats)
 *   W_in      : device [M][ndim]; W_out: device [M][ndim] (may alias W_in)
 *   W_lattice : device int [M][ndim] = rounded W_out, or NULL
 *   stats     : device, 1 record: D_cs, sums and c at W_in; moved/empty of this update; or NULL
 * Errors: ITC_ERR_INVALID_ARG, ITC_ERR_CUDA.
 */
int itc_step(const itc_image* img, const itc_params* p, const float* fields, const double* sxx,
             int M, const float* W_in, float* W_out, int* W_lattice, itc_stats* stats,
             void* stream);

/* ------------------------------------------------------------------- batched runs (plan) */
/*
 * A plan describes a batch of B images (ragged sizes, codebook counts and parameters) for
 * itc_run and itc_backward.  It is a byte blob built on the host by itc_plan; the caller copies
 * the same bytes to device memory (16-byte aligned) and passes both copies.  The plan picks the
 * tile shape per parameter class (itc_autotune may refine it) and lays out the workspace:
 * the fields of every image, per-tile partial sums and the ragged W / grad_h offsets.
 *
 * Ragged arrays: W and grad_W are [sum_b M_b][ndim_b] floats, image b starting at codebook
 * offset w_off(b) = sum_{b' < b} M_b' (times ndim); grad_h is one float per pixel, image b at
 * offset gh_off(b) = sum_{b' < b} H_b' W_b', rows of W_b floats.
 */

/* Host bytes of a plan for B images. */
size_t itc_plan_bytes(int B);

/*
 * itc_plan -- build a batch plan.
 *   imgs   : host array of B image descriptors (data on device; 2-D images only in a batch
 *            with ndim 3 images is allowed, each image keeps its own ndim)
 *   M      : host int[B], codebook count per image (1..ITC_MAX_M)
 *   p      : host itc_params[B] (per image) -- or one record if p_stride == 0
 *   plan   : host buffer of itc_plan_bytes(B) bytes, written
 *   ws_bytes_out : workspace bytes itc_run / itc_backward need for this plan
 * Errors: ITC_ERR_INVALID_ARG (any invalid image, M or params; nothing written).
 */
int itc_plan(int B, const itc_image* imgs, const int* M, const itc_params* p, int p_stride,
             void* plan, size_t plan_bytes, size_t* ws_bytes_out);

/* Total floats of the ragged grad_h layout of a plan (sum of H_b W_b). */
size_t itc_plan_pixels(const void* plan_host);

/*
 * itc_plan_offsets -- where image b of a plan lives (host-only query):
 *   field_off : byte offset of the image's field planes inside `ws` (planes as for itc_fields,
 *               plane stride = G * H * itc_field_pitch(W) floats), valid after itc_run
 *   w_off     : offset in floats of the image's codebooks in the ragged W / grad_W arrays
 *   gh_off    : offset in floats of the image's pixels in the ragged grad_h array
 * Any output pointer may be NULL.  Errors: ITC_ERR_INVALID_ARG (bad plan or b out of range).
 */
int itc_plan_offsets(const void* plan_host, int b, size_t* field_off, size_t* w_off, size_t* gh_off);

/*
 * itc_run -- Algorithm 1 for every image of a plan: fields (step 2) for all images in one
 * launch per parameter class, then all images' iterations (steps 3-11) in one launch per
 * lattice dimension: a CTA per image with more than 64 codebook vectors, smaller images 2, 4 or
 * 8 to a CTA, each stopping on its own (the results equal those of one image per CTA bit for
 * bit).  W is read as the initial codebooks (step 1 is done by the caller) and overwritten
 * with the result.  The fields stay in `ws` for a following itc_backward with the same plan.
 *   plan_host, plan_dev : the same plan bytes on host and on device
 *   W      : device ragged [sum M][ndim], in/out
 *   stats  : device itc_stats[B]: D_cs and sums at the returned W; or NULL
 *   ws     : device scratch, >= ws_bytes from itc_plan, 256-byte aligned
 * The enqueued work is stream-capturable (CUDA graphs).
 * Errors: ITC_ERR_INVALID_ARG, ITC_ERR_WORKSPACE, ITC_ERR_CUDA.
 */
int itc_run(const void* plan_host, const void* plan_dev, float* W, itc_stats* stats, void* ws,
            size_t ws_bytes, void* stream);

/*
 * itc_run_fields / itc_run_iterate -- the two phases of itc_run as separate calls (same
 * arguments, same results when called in this order): step 2 of Algorithm 1 for every image
 * (fields and S_XX partials into `ws`), then steps 3-11 on those fields.  Useful to time or
 * overlap the phases; itc_run_iterate requires the fields of the same plan in `ws`.
 */
int itc_run_fields(const void* plan_host, const void* plan_dev, void* ws, size_t ws_bytes,
                   void* stream);
int itc_run_iterate(const void* plan_host, const void* plan_dev, float* W, itc_stats* stats,
                    void* ws, size_t ws_bytes, void* stream);

/*
 * The two phases for the images [b0, b1) of a plan only (0 <= b0 <= b1 <= B).  The fields of
 * an image must be done before its iterations start; different image ranges are independent.
 * Errors: ITC_ERR_INVALID_ARG (bad plan or range), ITC_ERR_WORKSPACE, ITC_ERR_CUDA.
 */
int itc_run_fields_range(const void* plan_host, const void* plan_dev, int b0, int b1, void* ws,
                         size_t ws_bytes, void* stream);
int itc_run_iterate_range(const void* plan_host, const void* plan_dev, int b0, int b1, float* W,
                          itc_stats* stats, void* ws, size_t ws_bytes, void* stream);

/*
 * itc_run_pipelined -- itc_run with the batch cut into `chunks` image ranges: the fields of
 * range k+1 run on `stream` while the iterations of range k run on `stream2`, so the
 * latency-bound iterations overlap the bandwidth- and FMA-bound fields.  Same results as
 * itc_run.  `stream2` starts after the work already queued on `stream`, and `stream` waits
 * for all of `stream2`'s work before anything queued after this call (events joined inside;
 * the enqueued work is stream-capturable with both streams).  chunks in 1..64; chunks == 1 or
 * stream2 == stream is plain itc_run.
 * Errors: as itc_run.
 */
int itc_run_pipelined(const void* plan_host, const void* plan_dev, float* W, itc_stats* stats,
                      void* ws, size_t ws_bytes, void* stream, void* stream2, int chunks);

/*
 * itc_run_staged -- itc_run for images that are still in host memory: the images' bytes are
 * copied to the device range by range (`chunks` image ranges, one cudaMemcpyAsync each) on
 * `copy_stream`, and the fields of each range run on `stream` as soon as its bytes have landed,
 * so the copy of range k+1 overlaps the fields of range k; the iterations of the whole batch
 * follow in one launch.
 * host_base / dev_base: a host copy and the device buffer that the plan's image pointers (data
 * and weights) point into, same layout, `bytes` long; every image must lie inside the device
 * buffer.  The host copy should be page-locked for the copies to overlap.  The copies start
 * after the work already queued on `stream`; the results are those of itc_run.  copy_stream NULL
 * or equal to stream: copies and work in order on one stream.  chunks in 1..64.
 * Errors: ITC_ERR_INVALID_ARG (an image outside the buffer, bad sizes), ITC_ERR_WORKSPACE,
 * ITC_ERR_CUDA; as itc_run.
 */
int itc_run_staged(const void* plan_host, const void* plan_dev, const void* host_base,
                   void* dev_base, size_t bytes, float* W, itc_stats* stats, void* ws,
                   size_t ws_bytes, int chunks, void* stream, void* copy_stream);

/*
 * itc_autotune -- pick, per parameter class of a plan, the fields-pass configuration that runs
 * fastest on this GPU for this batch: the rows of output per tile (128, 64 or 32, i.e. how much
 * of the R-wide halo the row pass recomputes), the number of persistent CTAs per SM (1 or as many
 * as fit), and the input staging (tensor-memory-accelerator tiles, where the image rows are
 * 16-byte aligned, or plain loads).  Each candidate is timed with CUDA events over `reps`
 * launches (after one untimed launch) on `stream`; the choice is stored in the host plan and
 * the updated plan is copied to plan_dev (synchronously).  Results of later calls do not
 * depend on the choice except for the summation order of S_XX (fields are identical).
 * `ws` is overwritten.  Errors: ITC_ERR_INVALID_ARG, ITC_ERR_WORKSPACE, ITC_ERR_CUDA.
 */
int itc_autotune(void* plan_host, void* plan_dev, void* ws, size_t ws_bytes, int reps,
                 void* stream);

/*
 * itc_plan_configure -- set the fields-pass configuration of class c by hand (what itc_autotune
 * chooses): staging 1 = tensor tiles with tile_h 32, 64 or 128 output rows, staging 0 = plain loads
 * with the fixed tile height of the lattice dimension (64 in 2-D, 32 in 3-D; pass it);
 * grid_per_sm = persistent CTAs per SM (0 = as many as fit, else 1..64).  Updates the host
 * plan and copies it to plan_dev (synchronously on `stream`).  Errors: ITC_ERR_INVALID_ARG,
 * ITC_ERR_UNSUPPORTED (tensor tiles for a class whose images cannot use them, or a
 * self-overlap class), ITC_ERR_CUDA.
 */
int itc_plan_configure(void* plan_host, void* plan_dev, int c, int tile_h, int grid_per_sm,
                       int staging, void* stream);

/* Number of parameter classes of a plan (host-only); negative on error. */
int itc_plan_classes(const void* plan_host);

/*
 * itc_plan_class -- the configuration of class c (host-only): lattice dimension, sigma, output
 * rows per fields tile, persistent CTAs per SM (0 = as many as fit), staging (1 = tensor tiles,
 * 0 = plain loads, 2 = the extra pass that computes the field of h at the width of V(X) for
 * images whose sigma_self differs from sigma: plain loads, A only, 3 = recursive filtering,
 * ITC_RECURSIVE), number of images and the
 * tuned fields time in ms (0 if not tuned).  Any output pointer may be NULL.
 * Errors: ITC_ERR_INVALID_ARG.
 */
int itc_plan_class(const void* plan_host, int c, int* ndim, float* sigma, int* tile_h,
                   int* grid_per_sm, int* staging, int* images, float* tuned_ms);

/*
 * itc_plan_padded_offset -- offset (in elements) of image b in the plan's padded per-pixel
 * layout: every image as H rows of itc_field_pitch(W) elements (16-byte aligned rows), images
 * one after another.  b = B gives the total.  Host-only; negative on error.
 */
long long itc_plan_padded_offset(const void* plan_host, int b);

/*
 * itc_chamfer -- the pixel weights T(X) of weighted ITC, Sec. 5: for every binary image of a
 * plan (all images must be 2-D ITC_U8; nonzero = foreground) the 3-4 chamfer distance transform
 * (Borgefors) of the foreground, i.e. the length of the shortest 8-connected path to the nearest
 * background pixel with axial steps costing 3 and diagonal steps 4; the outside of the image
 * counts as background (reading); background pixels get 0.  Values are exact integers stored as
 * floats.  out: device, the padded per-pixel layout (itc_plan_padded_offset; the padding columns
 * are not written), 16-byte aligned, caller-owned; a plan over these weights (ITC_F32 images of
 * pitch itc_field_pitch(W)) gives the chamfer-weighted clustering P = T(X) * G of Sec. 5.
 * Errors: ITC_ERR_INVALID_ARG, ITC_ERR_UNSUPPORTED (an image wider than 1024), ITC_ERR_CUDA.
 */
int itc_chamfer(const void* plan_host, const void* plan_dev, float* out, void* stream);

/*
 * itc_segment -- the segments of Figs. 3 and 6 for every image of a plan: each pixel with data
 * (h != 0; in 3-D the voxel (u, v, gray(u, v))) gets the index k of the codebook vector whose
 * lattice site r_k = round(w_k) (clamped to the lattice) gives the largest kernel value
 * g_tau(x - r_k), i.e. the smallest sum_i (x_i - r_{k,i})^2 / tau_i^2 (tau = the plan's sigma).
 * The paper does not state the rule; this is the reading, evaluated in single precision term
 * by term (q_i = 1/tau_i^2 rounded once to float, each product and sum rounded, axis order, no
 * fused multiply-add), lowest k on ties.  Pixels without data get -1.
 * W: the plan's codebook layout (device, as for itc_run).  labels: device, one int16 per pixel,
 * image b at the pixel offset of itc_plan_offsets, rows of W entries (caller-owned).
 * Errors: ITC_ERR_INVALID_ARG, ITC_ERR_CUDA.
 */
int itc_segment(const void* plan_host, const void* plan_dev, const float* W, short* labels,
                void* stream);

/*
 * itc_backward -- gradient of Eq. (1) for every image of a plan, scaled by an upstream gradient:
 *   dD/dw_{k,i} = (2 / sigma_i^2) (E_{k,i} / S_WW - D_{k,i} / S_XW)
 *   dD/dh(x)    = 2 A(x) / S_XX - (2 / S_XW) sum_k g(x - w_k) [x in the box of round(w_k)]
 * D_k = sum_x h g(x - w_k)(x - w_k) over the box around round(w_k) (kernel at the real w_k),
 * E_k = sum_j g(w_j - w_k)(w_j - w_k).  dD/dh is the derivative with respect to the per-pixel
 * weight of weighted ITC (Sec. 5); its second term is a transposed Gaussian stamp of the
 * codebook (q = W * G, Sec. 3.1).  A and S_XX are read from the fields that itc_run (or
 * itc_run_fields) left in `ws` for the same plan and images; D_k and the sums are recomputed
 * at W, so W may differ from the forward's.
 *   W       : device ragged codebooks at which to differentiate
 *   grad_dcs: device float[B] upstream gradient (NULL = 1)
 *   grad_W  : device ragged [sum M][ndim], written (or NULL)
 *   grad_h  : device ragged pixels (itc_plan_pixels floats), written (or NULL); 2-D images get
 *             dD/dh(u,v); 3-D images get dD/dh of the weight of pixel (u,v) (voxel at its gray)
 *   stats   : device itc_stats[B], D_cs and sums at W (or NULL)
 *   ws      : as for itc_run
 * Errors: ITC_ERR_INVALID_ARG, ITC_ERR_WORKSPACE, ITC_ERR_CUDA.
 */
int itc_backward(const void* plan_host, const void* plan_dev, const float* W,
                 const float* grad_dcs, float* grad_W, float* grad_h, itc_stats* stats, void* ws,
                 size_t ws_bytes, void* stream);

/* ----------------------------------------------------- fields recomputed under a memory budget */
/*
 * When the fields of a whole batch do not fit in device memory (every image's ndim+1 FP32 planes:
 * 12 bytes per pixel of a 2-D batch, e.g. about 4 GB for 4096 images of up to 512 x 512), the
 * budgeted calls keep no fields between calls.  Their workspace holds the batch's S_XX partials,
 * per-image scalars and status words (a few bytes per image and per tile) plus a window of any
 * size that holds the fields of at least the largest image; the batch is cut into consecutive
 * image ranges whose fields fit the window, and each range's fields (step 2 of Algorithm 1,
 * Sec. 3.1) are computed into the window just before they are used.  The results are those of
 * the stored-fields calls bit for bit: the same fields kernels, tile configuration and
 * summation order, range by range.
 */

/* Workspace bytes for the budgeted calls within a total of budget_bytes: budget_bytes rounded
 * down to a multiple of 256, raised to the smallest workspace they accept (the batch's partials,
 * scalars and status words plus the fields of its largest image); 0 gives that smallest
 * workspace.  The window is what the workspace holds beyond that fixed part: the larger it is,
 * the fewer and larger the ranges.  0 if the plan is invalid. */
size_t itc_plan_budget_bytes(const void* plan_host, size_t budget_bytes);

/*
 * itc_run_budget -- itc_run with the fields recomputed range by range in the window: per range,
 * the fields pass and then the iterations of its images (one image per CTA).  Same arguments
 * and results as itc_run; ws of ws_bytes >= itc_plan_budget_bytes(plan, 0), 256-byte aligned.
 * The fields are not left in ws: follow it with itc_backward_budget, not itc_backward.
 * Errors: ITC_ERR_INVALID_ARG, ITC_ERR_WORKSPACE (smaller than the smallest budget), ITC_ERR_CUDA.
 */
int itc_run_budget(const void* plan_host, const void* plan_dev, float* W, itc_stats* stats, void* ws,
                   size_t ws_bytes, void* stream);

/*
 * itc_backward_budget -- itc_backward (the gradient of Eq. (1), weighted ITC of Sec. 5) with A
 * and S_XX recomputed range by range in the window instead of read from a stored fields pass:
 * per range, the fields pass, then the codebook and pixel kernels of the backward for its
 * images.  Same arguments and results as itc_backward (bit for bit); ws as for itc_run_budget.
 * It needs no earlier call: everything it reads is computed inside it.
 * Errors: as itc_run_budget; ITC_ERR_UNSUPPORTED for plans with recursive fields.
 */
int itc_backward_budget(const void* plan_host, const void* plan_dev, const float* W,
                        const float* grad_dcs, float* grad_W, float* grad_h, itc_stats* stats,
                        void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ITC_H */
