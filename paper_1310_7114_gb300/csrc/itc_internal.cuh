// itc_internal.cuh -- layouts shared by the kernels and the host side of libitc.so.
// Nothing here is part of the public ABI (include/itc.h is).
#pragma once

#include <cuda.h>   // CUtensorMap (type only; the encoder is fetched from the CUDA driver API at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include "itc.h"

namespace itc {

constexpr int kMaxTapsUV = 2 * ITC_MAX_RADIUS_UV + 1;
constexpr int kMaxTapsG = 2 * ITC_MAX_RADIUS_G + 1;
constexpr int kMaxClasses = 16;     // distinct (sigma, trunc, flags, ndim, dtype) classes per plan
constexpr int kThreads = 256;       // fields / backward CTA size
constexpr int kTileW = 64;          // output columns per fields tile
constexpr int kRunThreads = 128;    // codebook-iteration CTA size
// Iteration group record: image count n, span (threads per image: 16, 32, 64 or 128), then up to
// kRunThreads / 16 image indices.  Images with M <= span share one CTA, span threads each.
constexpr int kGroupMax = 8;
constexpr int kGroupInts = 2 + kGroupMax;
// Dynamic shared floats per codebook vector of the iteration and backward-codebook kernels:
// w (3), a (1), D (3), s (1), E (3).
constexpr int kCodebookSmemFloats = 11;

// Truncated, unnormalised 1-D Gaussian taps of one parameter class, computed on the host in
// double and rounded once to float:  g[d + R] = exp(-d^2 / (2 sigma^2)),  dg[d + R] = d g[d + R].
struct Taps {
    float gu[kMaxTapsUV], dgu[kMaxTapsUV];
    float gv[kMaxTapsUV], dgv[kMaxTapsUV];
    float gg[kMaxTapsG], dgg[kMaxTapsG];
    float sigma[3];
    float inv2s2[3];   // 1 / (2 sigma_i^2)
    int R[3];
    // the row pass of a window whose inputs are all 1: the FP32 FMA chains of the v taps in
    // kernel order, acc = fma(g[d], 1, acc) for d = 0 .. 2R (the same value as the arithmetic)
    float ones_gv, ones_dgv;
};

// Deriche's recursive Gaussian for one width: per axis (u, v) and term t the complex pole
// z = exp((-b_t + i omega_t) / sigma) and per term the complex weight c_t.
struct RecCoef {
    float zr[2][2], zi[2][2];
    float cr[2], ci[2];
};

// One image as the kernels see it (device-resident inside a plan, or passed by value).
struct ImageDesc {
    const void* data;
    const float* weight;
    int ndim, H, W, G, pitch, dtype;
    int fpitch;                 // field row pitch in floats
    int M;
    int cls;                    // parameter class
    int iters, flags;
    float step_scale;
    int tiles_u, tiles_v, tiles_g;   // fields tile grid of this image
    int tile_begin;             // first tile of this image inside its class launch
    long long partial_off;      // first S_XX partial (doubles) of this image
    long long field_off;        // offset of plane 0 in floats (from the fields base)
    long long plane_floats;     // floats per plane = G * H * fpitch
    long long w_off;            // offset of the image's codebooks, in floats (codebook * ndim)
    long long gh_off;           // offset of the image's grad_h, in floats
    int bwd_tile_begin;         // first tile of this image in the backward pixel pass
    int bwd_tiles_u, bwd_tiles_v;
    float sigma[3];
    float inv2s2[3];            // 1 / (2 sigma_i^2)
    int R[3];
    float rho[3];               // width of the codebook pair sums (rho = sigma unless set)
    float pinv2s2[3];           // 1 / (2 rho_i^2)
    float kappa[3];             // tau_i^2 / rho_i^2: factor of the pair term in the update
    double dcs_const;           // normalisers of Eq. (1): 1/2 sum log(tau^4 / (rho^2 s^2))
    long long sxx_off;          // first S_XX partial summed for S_XX (partial_off unless a
    int sxx_tiles;              //   separate self-overlap pass holds them), and their count
    int self_tiles_u;           // tile rows of the self-overlap pass (plain tiles)
    long long self_off;         // offset of the A_s plane (field of h at width s), -1: s = sigma
    int self_cls;               // class of the self-overlap pass, -1: none
    long long pad_off;          // offset (floats) of the image in the padded per-pixel layout
                                // (H rows of fpitch floats; chamfer weights)
    RecCoef rc, rc_self;        // ITC_RECURSIVE: the recursions at sigma and at the V(X) width
};


struct ClassInfo {
    Taps taps;
    int ndim, dtype, absolute, tile_h;
    int nimg, ntiles;
    int tma;                    // every image of the class has a tensor map (TMA fields path)
    int use_plain;              // tuned: take the plain-staged kernel even though TMA is possible
    int grid_per_sm;            // tuned persistent CTAs per SM (0: as many as fit)
    float tuned_ms;             // fields time of the class under the chosen configuration (0: untuned)
    int self;                   // self-overlap class: A at width s only, plain tiles
    int recursive;              // fields by recursive filtering (ITC_RECURSIVE); widths per image
    int list_off;               // offset (ints) of this class's image list in the plan int area
    int prefix_off;             // offset (ints) of the class tile prefix (nimg + 1 ints)
    long long partial_base;     // first partial of the class
};

struct PlanHeader {
    uint32_t magic;
    int B;
    int ncls;
    int max_M;
    int max_dim[3];             // largest H, W, G over the plan's images
    int ndim_mask;              // bit 2: the plan has 2-D images; bit 3: it has 3-D images
    long long total_pixels;     // sum H*W (grad_h layout)
    long long fields_floats;    // sum of every image's field planes
    long long total_tiles;
    long long ws_fields_off;    // bytes
    long long ws_partials_off;  // bytes
    long long ws_bytes;
    long long desc_off;         // bytes from plan start to ImageDesc[B]
    long long ints_off;         // bytes from plan start to the int area
    long long nints;
    long long ws_scal_off;      // bytes: per-image backward scalars (4 doubles each)
    long long ws_status_off;    // bytes: per-image device status words of the fields pass (B ints)
    long long ws_count_off;     // bytes: tile counters of the fields launches, one per class list
                                // position (the launch of class c from list position p uses
                                // list_off(c) + p)
    long long bwd_tiles;        // backward pixel tiles over all images
    int max_bwd_tiles;          // most backward pixel tiles of one image
    int bwd_order_off;          // offset (ints) of the backward image order (B ints, most tiles first)
    int run_groups_off;         // offset (ints) of the iteration groups (kGroupInts ints each)
    int run_ngroups[2];         // iteration groups of the 2-D images, then of the 3-D images
    long long tmap_off;         // bytes from plan start to CUtensorMap[B] (input tiles)
    long long pad_floats;       // sum H*fpitch (padded per-pixel layout)
    int has_recursive;          // some class computes its fields by recursion
    ClassInfo cls[kMaxClasses];
};

constexpr uint32_t kPlanMagic = 0x49544350u;  // "ITCP"

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Tile height of the fields kernels for a given radius (rows of outputs per CTA).
inline int default_tile_h(int ndim, int Ru) {
    if (ndim == 3) return 32;
    return Ru <= 6 ? 64 : 64;
}

// Kernel launch records (passed by value as __grid_constant__ parameters).
struct FieldsLaunch {
    CUtensorMap tmap_one;       // input tiles of the single image (TMA path)
    const CUtensorMap* tmaps;   // per-image maps in the plan (batched TMA path)
    Taps taps;
    const ImageDesc* descs;     // plan descriptors (batched) or nullptr (single image)
    ImageDesc one;              // the single image when descs == nullptr
    const int* img_list;        // class image list (batched)
    const int* tile_prefix;     // class tile prefix (batched, nimg + 1)
    int nimg;
    float* fields;              // fields base
    double* partials;           // S_XX partial base
    int tile_h;
    int absolute;
    int tile_base;              // first tile of this launch within the class (image sub-ranges)
    int test_stall;             // ITC_TEST_STALL_WAIT: CTA 0 waits for a phase that never completes
    int grid_per_sm;            // persistent CTAs per SM (0: as many as fit)
    int mode;                   // 0: every field plane; 1: A only, into the A_s plane, S_XX
                                // partials at sxx_off (self-overlap pass); 2: S_XX partials only
    int* counter;               // tensor-tile path: chunks of tiles handed out so far (0 at launch)
    int* status;                // device status words: one per image of the plan (batched) or one
                                // for the call (single image); a CTA whose bounded wait gives up
                                // writes ITC_ERR_TIMEOUT for every image it still owned tiles of
};

struct RunLaunch {
    const ImageDesc* descs;
    ImageDesc one;
    const float* fields;
    const double* partials;
    const double* sxx_single;   // single-image S_XX (itc_step) or nullptr
    const float* W_in;
    float* W_out;
    int* W_lattice;
    itc_stats* stats;
    int absolute;
    int final_eval;             // 1: stats at the final W (itc_run); 0: stats at W_in (itc_step)
    int img_base;               // image of blockIdx.x == 0 (image sub-ranges)
    const int* groups;          // whole batch: the images of each CTA (kGroupInts ints a CTA), else
                                // one image a CTA, img_base + blockIdx.x
    const int* img_status;      // per-image status words of the fields pass (plans) or nullptr
};

struct BackwardLaunch {
    const ImageDesc* descs;
    const float* fields;
    const double* partials;
    const float* W;
    const float* grad_dcs;
    float* grad_W;
    float* grad_h;
    itc_stats* stats;
    double* scal;               // per-image scalars in workspace: S_XW, S_WW, S_XX, gD
    const int* bwd_order;       // image of each backward pixel CTA (B ints, most tiles first), or
                                // nullptr: images img_base, img_base + 1, ... in order
    int B;
    int split;                  // pixel-pass CTAs per image (set at launch)
    int img_base;               // image of the first CTA (image ranges)
    const int* img_status;      // per-image status words of the fields pass, or nullptr
};

constexpr int kChamferMaxW = 1024;   // chamfer rows: 32 lanes x 4 columns x 8 chunks

struct RecursiveLaunch {
    const ImageDesc* descs;
    float* fields;              // fields base (the images' planes and scratch planes)
    double* partials;
    const int* img_list;        // class image list
    int pos_base;               // first list position of this launch
    int mode;                   // 0: A, F_u, F_v and S_XX; 1: A_s and S_XX (self-overlap pass)
};

struct ChamferLaunch {
    const ImageDesc* descs;
    float* out;                 // padded per-pixel layout (pad_off, rows of fpitch floats)
    const int* order;           // image of each warp (B ints, most pixels first)
    int B;
};

struct SegmentLaunch {
    const ImageDesc* descs;
    const float* W;
    short* labels;              // per image H x W at gh_off
    const int* order;           // image of each CTA (B ints, most pixels first)
};

constexpr int kBwdTileH = 64;   // backward pixel tile: 64 rows x 64 columns
constexpr int kBwdTileW = 64;
constexpr int kGridTileH2 = 64;   // fields tile height, 2-D (plain staging)
constexpr int kGridTileH3 = 32;   // fields tile height, 3-D (one gray slice per tile)

}  // namespace itc

// Kernel entry points (defined in the .cu files, launched from itc_api.cu).
namespace itc {
cudaError_t launch_fields(const FieldsLaunch& L, int nblocks, int R_u, int R_v, int ndim, int dtype,
                          cudaStream_t s);
cudaError_t launch_reduce_sxx(const double* partials, int n, double* out, cudaStream_t s);
// 3-D fields (itc_fields3d.cu): tiles [L.tile_base, ntiles) of the launch's images
cudaError_t launch_fields3d(const FieldsLaunch& L, int ntiles, int R_u, int R_v, cudaStream_t s);
// TMA-staged 2-D fields (itc_fields_tma.cu): the radii it is compiled for, its box per radius
// and data type, and its launch.
bool fields_tma_supported(int ndim, int Ru, int Rv);
int fields_tma_box(int dtype, int R, int tile_h, int* box_w, int* box_h);
cudaError_t launch_fields_tma(const FieldsLaunch& L, int ntiles, int R, int dtype, cudaStream_t s);
// ndim: the lattice dimension of every image of the launch (2 or 3)
cudaError_t launch_run(const RunLaunch& L, int nimg, int max_M, const int* max_dim, cudaStream_t s, int ndim);
cudaError_t launch_recursive(const RecursiveLaunch& L, int nimg, int max_H, int max_W, cudaStream_t s);
cudaError_t launch_chamfer(const ChamferLaunch& L, int max_W, cudaStream_t s);
cudaError_t launch_segment(const SegmentLaunch& L, int B, int max_M, cudaStream_t s);
cudaError_t launch_backward(const BackwardLaunch& L, int B, int max_M, long long pixel_tiles, int max_image_tiles,
                            cudaStream_t s);
}  // namespace itc
