// itc_fields.cu -- truncated separable Gaussian fields of 2-D lattice images (Sec. 3.1, Sec. 5)
// with plain staging (rows that are not on 16-byte boundaries, radii without a compiled TMA
// kernel); gray images as [u, v, g] lattices are in itc_fields3d.cu.
//
// One CTA computes a TH x 64 tile of output sites:
//   1. the input tile plus an R-wide halo is staged in shared memory as float (zero outside the
//      lattice: sites outside hold no data);
//   2. pass along v (Sec. 3.1: two 1-D masks): T = g_v * X and T_v = (d g_v) * X (centred) or
//      g_v * (v X) (absolute), for every staged row;
//   3. pass along u over the staged rows: A = g_u * T, F_u = (d g_u) * T or g_u * (u T),
//      F_v = g_u * T_v, written with 128-bit stores;
//   4. epilogue: the tile's share of S_XX = sum_x h(x) A(x) (V(X) of Eq. (1)) as one double.
// Tiles whose staged input is all zero only write zeros.  For the radii the parameter sets use
// (6, 9, 12) both passes are fully unrolled with the taps in the constant bank; other radii
// run the same passes with runtime loops.
#include "itc_internal.cuh"

namespace itc {
namespace {

__device__ __forceinline__ double block_sum_double(double v, double* red) {
    // Fixed-order block reduction (deterministic): warp xor-shuffles, then warp 0 over warps.
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0;
    if (wid == 0) {
        t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

__device__ __forceinline__ double block_sum_tile(float v, double* red) {
    // S_XX share of one tile (deterministic): FP32 xor-shuffles within each warp (the FP64 rate
    // of the part is a small fraction of its FP32 rate), then the warp sums in FP64 by warp 0.
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = (double)v;
    __syncthreads();
    double t = 0;
    if (wid == 0) {
        t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

__device__ __forceinline__ int find_image(const int* __restrict__ prefix, int n, int b) {
    // largest p with prefix[p] <= b
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

template <int RU, int RV, bool ABS, int DTYPE, int TH>
__global__ void __launch_bounds__(kThreads, 2) fields_kernel(const __grid_constant__ FieldsLaunch L)
{
    constexpr int TW = kTileW;
    constexpr int K = TH / 16;                 // output rows per thread in the u pass
    constexpr int NR = 2;                      // row-pass outputs: T, T_v
    constexpr int NC = 3;                      // column-pass outputs: A, F_u, F_v
    const Taps& tp = L.taps;
    const int Ru = RU > 0 ? RU : tp.R[0];
    const int Rv = RV > 0 ? RV : tp.R[1];
    const int ROWS = TH + 2 * Ru;
    const int SW = ((TW + 2 * Rv + 3) & ~3) + 4;   // staged row length (floats)

    // ---- which image / tile
    int b = blockIdx.x + L.tile_base;
    const ImageDesc* dp;
    if (L.descs) {
        const int p = find_image(L.tile_prefix, L.nimg + 1, b);
        dp = L.descs + __ldg(L.img_list + p);
        b -= __ldg(L.tile_prefix + p);
    } else {
        dp = &L.one;
    }
    const int H = dp->H, W = dp->W, pitch = dp->pitch, fpitch = dp->fpitch;
    // mode 0: every plane of the fields; 1: A only, into the A_s plane (self-overlap pass);
    // 2: the S_XX partials only
    const int mode = L.mode;
    const int nstore = mode == 0 ? NC : (mode == 1 ? 1 : 0);
    const int tiles_v = dp->tiles_v, tiles_u = mode ? dp->self_tiles_u : dp->tiles_u;
    const int tv = b % tiles_v;
    const int tu = (b / tiles_v) % tiles_u;
    const int u0 = tu * TH, v0 = tv * TW;
    float* const fbase = L.fields + (mode == 1 ? dp->self_off : dp->field_off);
    const long long plane = dp->plane_floats;

    extern __shared__ __align__(16) float smem[];
    float* s_in = smem;                                 // ROWS x SW: input
    float* sT = s_in + ROWS * SW;                       // NR planes of ROWS x TW
    __shared__ double red[32];
    const int tid = threadIdx.x;

    // ---- stage the input tile with its halo
    int nonzero = 0;
    {
        const int wid = tid >> 5, lane = tid & 31;
        for (int r = wid; r < ROWS; r += kThreads / 32) {
            const int gu = u0 - Ru + r;
            const bool row_in = (gu >= 0) && (gu < H);
            for (int c = lane; c < SW; c += 32) {
                const int gv = v0 - Rv + c;
                const bool in = row_in && gv >= 0 && gv < W && c < TW + 2 * Rv;
                float x = 0.f;
                if (in) {
                    if (DTYPE == ITC_U8)
                        x = (float)__ldg(reinterpret_cast<const unsigned char*>(dp->data) + (size_t)gu * pitch + gv);
                    else
                        x = __ldg(reinterpret_cast<const float*>(dp->data) + (size_t)gu * pitch + gv);
                }
                nonzero |= (x != 0.f);
                s_in[r * SW + c] = x;
            }
        }
    }

    // Column-pass ownership (also used for zero stores): rows k0..k0+K-1, columns c0..c0+3.
    const int kb = tid >> 4, cg = tid & 15;
    const int k0 = kb * K, c0 = cg * 4;
    const bool col_active = (u0 + k0 < H) && (v0 + c0 < W);

    float part = 0.f;

    if (!__syncthreads_or(nonzero)) {
        if (col_active) {
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const int u = u0 + k0 + kk;
                if (u >= H) break;
                float* o = fbase + (long long)u * fpitch + v0 + c0;
#pragma unroll
                for (int f = 0; f < NC; ++f)
                    if (f < nstore) st4(o + f * plane, 0.f, 0.f, 0.f, 0.f);
            }
        }
    } else {
        // ---- pass along v
        for (int item = tid; item < ROWS * 16; item += kThreads) {
            const int r = item >> 4, c = (item & 15) * 4;
            float* o0 = sT + r * TW + c;
            const int gu = u0 - Ru + r;
            if (v0 + c >= W) continue;
            if (gu < 0 || gu >= H) {
#pragma unroll
                for (int f = 0; f < NR; ++f) st4(o0 + f * ROWS * TW, 0.f, 0.f, 0.f, 0.f);
                continue;
            }
            float t[NR][4];
#pragma unroll
            for (int f = 0; f < NR; ++f)
#pragma unroll
                for (int j = 0; j < 4; ++j) t[f][j] = 0.f;
            const float* src = s_in + r * SW + c;
            const float vbase = (float)(v0 - Rv + c);
            if constexpr (RV > 0) {
                constexpr int NWIN = ((4 + 2 * RV) + 3) & ~3;
                float x[NWIN];
#pragma unroll
                for (int q = 0; q < NWIN / 4; ++q) {
                    const float4 f4 = ld4(src + 4 * q);
                    x[4 * q] = f4.x; x[4 * q + 1] = f4.y; x[4 * q + 2] = f4.z; x[4 * q + 3] = f4.w;
                }
                float xv[ABS ? NWIN : 1];
                if constexpr (ABS) {
#pragma unroll
                    for (int i = 0; i < NWIN; ++i) xv[i] = x[i] * (vbase + (float)i);
                }
#pragma unroll
                for (int d = 0; d <= 2 * RV; ++d) {
                    const float g = tp.gv[d];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        t[0][j] = fmaf(g, x[j + d], t[0][j]);
                        if constexpr (ABS) t[1][j] = fmaf(g, xv[j + d], t[1][j]);
                        else t[1][j] = fmaf(tp.dgv[d], x[j + d], t[1][j]);
                    }
                }
            } else {
                for (int d = 0; d <= 2 * Rv; ++d) {
                    const float g = tp.gv[d], dg = tp.dgv[d];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float x = src[j + d];
                        t[0][j] = fmaf(g, x, t[0][j]);
                        if (ABS) t[1][j] = fmaf(g, x * (vbase + (float)(j + d)), t[1][j]);
                        else t[1][j] = fmaf(dg, x, t[1][j]);
                    }
                }
            }
#pragma unroll
            for (int f = 0; f < NR; ++f) st4(o0 + f * ROWS * TW, t[f][0], t[f][1], t[f][2], t[f][3]);
        }
        __syncthreads();

        // ---- pass along u, stores and S_XX share
        if (col_active) {
            float acc[NC][K][4];
#pragma unroll
            for (int f = 0; f < NC; ++f)
#pragma unroll
                for (int kk = 0; kk < K; ++kk)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[f][kk][j] = 0.f;
            const float* Tp = sT + k0 * TW + c0;
            const float ubase = (float)(u0 - Ru + k0);
            const int NI = K + 2 * Ru;
#pragma unroll
            for (int i = 0; i < (RU > 0 ? K + 2 * RU : 1); ++i) {
                // compile-time radius: fully unrolled (the runtime case is handled below)
                if constexpr (RU > 0) {
                    float t[NR][4];
#pragma unroll
                    for (int f = 0; f < NR; ++f) {
                        const float4 f4 = ld4(Tp + f * ROWS * TW + i * TW);
                        t[f][0] = f4.x; t[f][1] = f4.y; t[f][2] = f4.z; t[f][3] = f4.w;
                    }
                    float tu[4];
                    if constexpr (ABS) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) tu[j] = t[0][j] * (ubase + (float)i);
                    }
#pragma unroll
                    for (int kk = 0; kk < K; ++kk) {
                        const int e = i - kk;
                        if (e >= 0 && e <= 2 * RU) {
                            const float g = tp.gu[e];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                acc[0][kk][j] = fmaf(g, t[0][j], acc[0][kk][j]);
                                if constexpr (ABS) acc[1][kk][j] = fmaf(g, tu[j], acc[1][kk][j]);
                                else acc[1][kk][j] = fmaf(tp.dgu[e], t[0][j], acc[1][kk][j]);
                                acc[2][kk][j] = fmaf(g, t[1][j], acc[2][kk][j]);
                            }
                        }
                    }
                }
            }
            if constexpr (RU == 0) {
                for (int i = 0; i < NI; ++i) {
                    float t[NR][4];
#pragma unroll
                    for (int f = 0; f < NR; ++f) {
                        const float4 f4 = ld4(Tp + f * ROWS * TW + i * TW);
                        t[f][0] = f4.x; t[f][1] = f4.y; t[f][2] = f4.z; t[f][3] = f4.w;
                    }
#pragma unroll
                    for (int kk = 0; kk < K; ++kk) {
                        const int e = i - kk;
                        if (e >= 0 && e <= 2 * Ru) {
                            const float g = tp.gu[e], dg = tp.dgu[e];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                acc[0][kk][j] = fmaf(g, t[0][j], acc[0][kk][j]);
                                if (ABS) acc[1][kk][j] = fmaf(g, t[0][j] * (ubase + (float)i), acc[1][kk][j]);
                                else acc[1][kk][j] = fmaf(dg, t[0][j], acc[1][kk][j]);
                                acc[2][kk][j] = fmaf(g, t[1][j], acc[2][kk][j]);
                            }
                        }
                    }
                }
            }
            float ps = 0.f;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const int u = u0 + k0 + kk;
                if (u < H) {
                    float* o = fbase + (long long)u * fpitch + v0 + c0;
#pragma unroll
                    for (int f = 0; f < NC; ++f)
                        if (f < nstore) st4(o + f * plane, acc[f][kk][0], acc[f][kk][1], acc[f][kk][2], acc[f][kk][3]);
                    const int si = (k0 + kk + Ru) * SW + c0 + Rv;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (v0 + c0 + j < W) {
                            ps = fmaf(s_in[si + j], acc[0][kk][j], ps);
                        }
                    }
                }
            }
            part += ps;
        }
    }

    const double tot = block_sum_tile(part, red);
    // b = tile index within the image
    if (tid == 0) L.partials[(mode ? dp->sxx_off : dp->partial_off) + b] = tot;
}

template <int RU, int RV, bool ABS, int DTYPE, int TH>
cudaError_t launch_one(const FieldsLaunch& L, int nblocks, int Ru, int Rv, cudaStream_t s) {
    const int rows = TH + 2 * Ru;
    const int SW = ((kTileW + 2 * Rv + 3) & ~3) + 4;
    const size_t smem = (size_t)rows * SW * sizeof(float) + (size_t)2 * rows * kTileW * sizeof(float);
    auto k = fields_kernel<RU, RV, ABS, DTYPE, TH>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<nblocks, kThreads, smem, s>>>(L);
    return cudaGetLastError();
}

template <bool ABS, int DTYPE, int TH>
cudaError_t dispatch_radius(const FieldsLaunch& L, int nblocks, int Ru, int Rv, cudaStream_t s) {
    if (Ru == Rv) {
        if (Ru == 6) return launch_one<6, 6, ABS, DTYPE, TH>(L, nblocks, Ru, Rv, s);
        if (Ru == 9) return launch_one<9, 9, ABS, DTYPE, TH>(L, nblocks, Ru, Rv, s);
        if (Ru == 12) return launch_one<12, 12, ABS, DTYPE, TH>(L, nblocks, Ru, Rv, s);
    }
    return launch_one<0, 0, ABS, DTYPE, TH>(L, nblocks, Ru, Rv, s);
}

__global__ void reduce_sxx_kernel(const double* __restrict__ partials, int n, double* out) {
    __shared__ double red[32];
    double v = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += partials[i];
    const double t = block_sum_double(v, red);
    if (threadIdx.x == 0) *out = t;
}

}  // namespace

cudaError_t launch_fields(const FieldsLaunch& L, int nblocks, int Ru, int Rv, int ndim, int dtype,
                          cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    const bool abs_ = L.absolute != 0;
    if (ndim == 3) return launch_fields3d(L, L.tile_base + nblocks, Ru, Rv, s);
    if (dtype == ITC_U8)
        return abs_ ? dispatch_radius<true, ITC_U8, kGridTileH2>(L, nblocks, Ru, Rv, s)
                    : dispatch_radius<false, ITC_U8, kGridTileH2>(L, nblocks, Ru, Rv, s);
    return abs_ ? dispatch_radius<true, ITC_F32, kGridTileH2>(L, nblocks, Ru, Rv, s)
                : dispatch_radius<false, ITC_F32, kGridTileH2>(L, nblocks, Ru, Rv, s);
}

cudaError_t launch_reduce_sxx(const double* partials, int n, double* out, cudaStream_t s) {
    reduce_sxx_kernel<<<1, 256, 0, s>>>(partials, n, out);
    return cudaGetLastError();
}

}  // namespace itc
