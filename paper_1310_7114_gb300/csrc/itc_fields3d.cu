// itc_fields3d.cu -- fields of gray images as [u, v, g] lattices (Sec. 1 (ii)): the truncated
// separable Gaussian of Sec. 3.1 along u, v and the gray axis g.
//
// The input of a gray image is one lattice point per pixel, at (u, v, I(u, v)) with the pixel's
// weight.  The convolution along g is analytic: on gray slice g a pixel carries
//   S = w g_g(g - I) and S_g = S (I - g) (centred moments; S I for absolute ones),
// and the slice's fields are the 2-D passes over S and S_g:
//   T = g_v * S, T_v = (d g_v) * S or g_v * (v S), T_g = g_v * S_g                (along v)
//   A = g_u * T, F_u = (d g_u) * T or g_u * (u T), F_v = g_u * T_v, F_g = g_u * T_g (along u).
//
// One tile is TH x 64 sites of one gray slice.  The CTAs are persistent: each takes a contiguous
// run of the class's tiles, which are ordered slice-fastest within an image, so consecutive tiles
// share their (u, v) window and the pixels' gray levels are staged once per window and run.  Each tile's share of S_XX is its own partial (FP32 within warps, FP64 across them).
// Tiles whose slice holds no data write zeros.
#include "itc_internal.cuh"

namespace itc {
namespace {

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
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

template <int RU, int RV, bool ABS, int TH>
__global__ void __launch_bounds__(kThreads, (RU > 0 && RU <= 9) ? 3 : 2) fields3d_kernel(const __grid_constant__ FieldsLaunch L, int ntiles)
{
    constexpr int TW = kTileW;
    constexpr int K = TH / 16;                 // rows per thread of the zero stores
    static_assert(TH == 32 && kThreads == 256, "the pass along u maps 4 x 8 rows x 64 columns");
    const Taps& tp = L.taps;
    const int Ru = RU > 0 ? RU : tp.R[0];
    const int Rv = RV > 0 ? RV : tp.R[1];
    const int Rg = tp.R[2];
    const int ROWS = TH + 2 * Ru;
    const int SW = (TW + 2 * Rv + 3) & ~3;   // staged row length (sites, a multiple of 4)
    // mode 0: every plane of the fields; 1: A only, into the A_s plane (self-overlap pass);
    // 2: the S_XX partials only
    const int mode = L.mode;
    const int nstore = mode == 0 ? 4 : (mode == 1 ? 1 : 0);

    // 76 KB at R = 9, so that three CTAs share an SM (two at larger radii): the gray levels are
    // staged as bytes and the weights of weighted images are read from global memory (L1) where
    // they are needed
    extern __shared__ __align__(16) float smem[];
    float* s_S = smem;                    // ROWS x SW: S of the slice
    float* s_Sg = s_S + ROWS * SW;        // S_g
    float* sT = s_Sg + ROWS * SW;         // T, T_v, T_g: ROWS x TW each
    float* s_gg = sT + 3 * ROWS * TW;     // g_g taps (indexed per site), 2 Rg + 1 of them
    unsigned char* s_gray = reinterpret_cast<unsigned char*>(s_gg + ((2 * Rg + 4) & ~3));   // ROWS x SW
    __shared__ double red[2][kThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i <= 2 * Rg; i += kThreads) s_gg[i] = tp.gg[i];

    // this CTA's run of tiles
    const long long n = ntiles - L.tile_base;
    const int t_begin = L.tile_base + (int)(n * blockIdx.x / gridDim.x);
    const int t_end = L.tile_base + (int)(n * (blockIdx.x + 1) / gridDim.x);
    if (t_begin >= t_end) return;

    // zero stores of a tile without data: rows k0..k0+K-1, columns c0..c0+3
    const int k0 = (tid >> 4) * K, c0 = (tid & 15) * 4;

    // a tile's image and its index within the image (tiles are visited in order)
    int img_p = 0;
    auto locate = [&](int t, int& b) -> const ImageDesc* {
        b = t;
        if (!L.descs) return &L.one;
        if (t == t_begin || t >= __ldg(L.tile_prefix + img_p + 1)) img_p = find_image(L.tile_prefix, L.nimg + 1, t);
        b -= __ldg(L.tile_prefix + img_p);
        return L.descs + __ldg(L.img_list + img_p);
    };
    // stage the gray levels of the (u, v) window at u0, v0 as bytes (0 outside the image; the S
    // pass tests the sites' coordinates).  With rows on 16-byte boundaries: 16-byte loads of the
    // row chunks [v0 - 16, v0 + 80), which cover the staged columns v0 - Rv .. v0 + 63 + Rv
    // (Rv <= 16); a chunk that starts inside the row ends inside its 16-byte pitch
    auto stage = [&](const ImageDesc* dp, int u0, int v0) {
        const int H = dp->H, W = dp->W, pitch = dp->pitch;
        const unsigned char* data = reinterpret_cast<const unsigned char*>(dp->data);
        if ((pitch & 15) == 0 && (reinterpret_cast<uintptr_t>(data) & 15) == 0 && Rv <= 16) {
            for (int e = tid; e < ROWS * 6; e += kThreads) {
                const int r = e / 6, q = e - 6 * r;
                const int gu = u0 - Ru + r, col = v0 - 16 + 16 * q;
                const bool row_in = gu >= 0 && gu < H;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (row_in && col >= 0 && col < W)
                    v = __ldg(reinterpret_cast<const uint4*>(data + (size_t)gu * pitch + col));
                const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int c = col - (v0 - Rv) + k;   // staged column of byte k
                    if (c >= 0 && c < SW) s_gray[r * SW + c] = (unsigned char)(wv[k >> 2] >> (8 * (k & 3)));
                }
            }
        } else {
            for (int e = tid; e < ROWS * SW; e += kThreads) {
                const int r = e / SW, c = e - r * SW;
                const int gu = u0 - Ru + r, gv = v0 - Rv + c;
                s_gray[e] = (gu >= 0 && gu < H && gv >= 0 && gv < W) ? __ldg(data + (size_t)gu * pitch + gv) : 0;
            }
        }
    };
    // S and S_g of slice yg over the staged window, four sites per step; nonzero if any S is.
    // Staged columns [clo, chi) of rows inside the image hold its sites; the others hold no data.
    // The four gray levels of a step are tested at once (byte-wise |I - g| <= Rg), and images
    // without weights take a loop of their own (a tested weight load costs its address
    // arithmetic in every step).
    auto s_pass = [&](const ImageDesc* dp, int u0, int v0, int yg) -> int {
        const int H = dp->H, pitch = dp->pitch;
        const float* wimg = dp->weight;
        const int clo = Rv - v0 > 0 ? Rv - v0 : 0;
        const int chi = min(dp->W - (v0 - Rv), TW + 2 * Rv);
        const uint32_t yg4 = (uint32_t)yg * 0x01010101u, rg4 = (uint32_t)min(Rg, 255) * 0x01010101u;
        const float fb = 8388608.f + (float)yg;   // (2^23 + I) - (2^23 + g) = I - g, exactly
        const int QW = SW / 4;
        int nonzero = 0;
        // per step: 0xff in each byte whose site is in the image and within the slice's band
        auto band = [&](int q, int& r, int& c, int& gu, uint32_t& g4) -> uint32_t {
            r = q / QW;
            c = 4 * (q - r * QW);
            gu = u0 - Ru + r;
            g4 = *reinterpret_cast<const uint32_t*>(s_gray + r * SW + c);
            uint32_t m = (unsigned)gu < (unsigned)H ? __vcmpleu4(__vabsdiffu4(g4, yg4), rg4) : 0u;
            if (c < clo || c + 3 >= chi) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (c + j < clo || c + j >= chi) m &= ~(0xffu << (8 * j));
            }
            return m;
        };
        if (!wimg) {
#pragma unroll 4   // 0.186 -> 0.183 ms on C5 against 2 (1: 0.195 ms): the steps' loads overlap
            for (int q = tid; q < ROWS * QW; q += kThreads) {
                int r, c, gu;
                uint32_t g4;
                const uint32_t m = band(q, r, c, gu, g4);
                float sv[4], sa[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int gl = (int)((g4 >> (8 * j)) & 0xffu);
                    const bool in = (m >> (8 * j)) & 1u;
                    const float gg = s_gg[in ? gl - yg + Rg : 0];
                    const float v = in ? gg : 0.f;
                    sv[j] = v;
                    sa[j] = ABS ? v * (float)gl : v * (__int_as_float(0x4B000000 | gl) - fb);
                }
                nonzero |= (m != 0u);
                st4(s_S + 4 * q, sv[0], sv[1], sv[2], sv[3]);
                st4(s_Sg + 4 * q, sa[0], sa[1], sa[2], sa[3]);
            }
        } else {
            for (int q = tid; q < ROWS * QW; q += kThreads) {
                int r, c, gu;
                uint32_t g4;
                const uint32_t m = band(q, r, c, gu, g4);
                float sv[4], sa[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int gl = (int)((g4 >> (8 * j)) & 0xffu);
                    float v = 0.f;
                    if ((m >> (8 * j)) & 1u)
                        v = __ldg(wimg + (size_t)gu * pitch + (v0 - Rv + c + j)) * s_gg[gl - yg + Rg];
                    sv[j] = v;
                    sa[j] = ABS ? v * (float)gl : v * (__int_as_float(0x4B000000 | gl) - fb);
                    nonzero |= (v != 0.f);
                }
                st4(s_S + 4 * q, sv[0], sv[1], sv[2], sv[3]);
                st4(s_Sg + 4 * q, sa[0], sa[1], sa[2], sa[3]);
            }
        }
        return nonzero;
    };

    // Pipeline per tile: [pass along v] barrier [pass along u; then S of the next tile] barrier.
    // The next tile's S overwrites S only after the pass along v has read it, and the pass along
    // u reads the staged window, so a window change stages between two extra barriers.
    int b = 0;
    const ImageDesc* dp = locate(t_begin, b);
    int yg = b % dp->tiles_g, sp = b / dp->tiles_g;   // slice; (u, v) window
    stage(dp, (sp / dp->tiles_v) * TH, (sp % dp->tiles_v) * TW);
    __syncthreads();
    int any = __syncthreads_or(s_pass(dp, (sp / dp->tiles_v) * TH, (sp % dp->tiles_v) * TW, yg));

    for (int t = t_begin; t < t_end; ++t) {
        const int H = dp->H, W = dp->W, fpitch = dp->fpitch, ipitch = dp->pitch;
        const float* const wimg = dp->weight;
        const int u0 = (sp / dp->tiles_v) * TH, v0 = (sp % dp->tiles_v) * TW;
        float* const fbase = L.fields + (mode == 1 ? dp->self_off : dp->field_off);
        const long long plane = dp->plane_floats;
        const long long slice_off = (long long)yg * H * fpitch;
        const bool col_active = (u0 + k0 < H) && (v0 + c0 < W);
        float part = 0.f;
        if (!any) {
            if (col_active) {
                for (int kk = 0; kk < K; ++kk) {
                    const int u = u0 + k0 + kk;
                    if (u >= H) break;
                    float* o = fbase + slice_off + (long long)u * fpitch + v0 + c0;
                    for (int f = 0; f < nstore; ++f) st4(o + f * plane, 0.f, 0.f, 0.f, 0.f);
                }
            }
        } else {
            // ---- pass along v: 8 outputs of one staged row per item (a window of 8 + 2 Rv
            // inputs read once for the 8); T and T_v first, then T_g, to bound the live registers
            for (int item = tid; item < ROWS * 8; item += kThreads) {
                const int r = item >> 3, c = (item & 7) * 8;
                if (v0 + c >= W) continue;
                const float* src = s_S + r * SW + c;
                const float* srca = s_Sg + r * SW + c;
                const float vbase = (float)(v0 - Rv + c);
                float* o0 = sT + r * TW + c;
                float ta[8], tb[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) { ta[j] = 0.f; tb[j] = 0.f; }
                if constexpr (RV > 0) {
                    constexpr int NWIN = ((8 + 2 * RV) + 3) & ~3;   // within the staged row: SW >= 68 + 2 RV
                    float x[NWIN];
#pragma unroll
                    for (int q = 0; q < NWIN / 4; ++q) {
                        const float4 f4 = ld4(src + 4 * q);
                        x[4 * q] = f4.x; x[4 * q + 1] = f4.y; x[4 * q + 2] = f4.z; x[4 * q + 3] = f4.w;
                    }
#pragma unroll
                    for (int d = 0; d <= 2 * RV; ++d) {
                        const float g = tp.gv[d];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            ta[j] = fmaf(g, x[j + d], ta[j]);
                            if constexpr (ABS) tb[j] = fmaf(g, x[j + d] * (vbase + (float)(j + d)), tb[j]);
                            else tb[j] = fmaf(tp.dgv[d], x[j + d], tb[j]);
                        }
                    }
                    st4(o0, ta[0], ta[1], ta[2], ta[3]); st4(o0 + 4, ta[4], ta[5], ta[6], ta[7]);
                    st4(o0 + ROWS * TW, tb[0], tb[1], tb[2], tb[3]); st4(o0 + ROWS * TW + 4, tb[4], tb[5], tb[6], tb[7]);
#pragma unroll
                    for (int q = 0; q < NWIN / 4; ++q) {
                        const float4 f4 = ld4(srca + 4 * q);
                        x[4 * q] = f4.x; x[4 * q + 1] = f4.y; x[4 * q + 2] = f4.z; x[4 * q + 3] = f4.w;
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) ta[j] = 0.f;
#pragma unroll
                    for (int d = 0; d <= 2 * RV; ++d) {
                        const float g = tp.gv[d];
#pragma unroll
                        for (int j = 0; j < 8; ++j) ta[j] = fmaf(g, x[j + d], ta[j]);
                    }
                    st4(o0 + 2 * ROWS * TW, ta[0], ta[1], ta[2], ta[3]); st4(o0 + 2 * ROWS * TW + 4, ta[4], ta[5], ta[6], ta[7]);
                } else {
                    for (int d = 0; d <= 2 * Rv; ++d) {
                        const float g = tp.gv[d], dg = tp.dgv[d];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float x = src[j + d];
                            ta[j] = fmaf(g, x, ta[j]);
                            if (ABS) tb[j] = fmaf(g, x * (vbase + (float)(j + d)), tb[j]);
                            else tb[j] = fmaf(dg, x, tb[j]);
                        }
                    }
                    st4(o0, ta[0], ta[1], ta[2], ta[3]); st4(o0 + 4, ta[4], ta[5], ta[6], ta[7]);
                    st4(o0 + ROWS * TW, tb[0], tb[1], tb[2], tb[3]); st4(o0 + ROWS * TW + 4, tb[4], tb[5], tb[6], tb[7]);
#pragma unroll
                    for (int j = 0; j < 8; ++j) ta[j] = 0.f;
                    for (int d = 0; d <= 2 * Rv; ++d) {
                        const float g = tp.gv[d];
#pragma unroll
                        for (int j = 0; j < 8; ++j) ta[j] = fmaf(g, srca[j + d], ta[j]);
                    }
                    st4(o0 + 2 * ROWS * TW, ta[0], ta[1], ta[2], ta[3]); st4(o0 + 2 * ROWS * TW + 4, ta[4], ta[5], ta[6], ta[7]);
                }
            }
            __syncthreads();

            // ---- pass along u: 8 rows of one column per thread (each staged T value read once
            // for the 8), stores and the tile's S_XX share
            const int kr = (tid >> 6) * 8, cc = tid & 63;   // rows kr..kr+7 (TH = 32), column cc
            if (u0 + kr < H && v0 + cc < W) {
                float acc[4][8];
#pragma unroll
                for (int f = 0; f < 4; ++f)
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) acc[f][kk] = 0.f;
                const float* Tp = sT + kr * TW + cc;
                const float ubase = (float)(u0 - Ru + kr);
                if constexpr (RU > 0 && !ABS) {
                    // two fields per packed FMA, tap-outer over the unit's inputs in registers (a
                    // tap pair is formed once for the 8 rows): (A, F_u) += (g_u, d g_u) (T, T), then
                    // (F_v, F_g) += (g_u, g_u) (T_v, T_g); the same products in the same order as
                    // the scalar loop below (0.183 -> 0.181 ms on C5)
                    constexpr int NI = 8 + 2 * RU;
                    float2 pa[8], pb[8];
                    {
                        float2 x[NI];
#pragma unroll
                        for (int i = 0; i < NI; ++i) {
                            const float t0 = Tp[i * TW];
                            x[i] = make_float2(t0, t0);
                        }
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) pa[kk] = make_float2(0.f, 0.f);
#pragma unroll
                        for (int e = 0; e <= 2 * RU; ++e) {
                            const float2 gp = make_float2(tp.gu[e], tp.dgu[e]);
#pragma unroll
                            for (int kk = 0; kk < 8; ++kk) pa[kk] = __ffma2_rn(gp, x[kk + e], pa[kk]);
                        }
                    }
                    {
                        float2 x[NI];
#pragma unroll
                        for (int i = 0; i < NI; ++i) x[i] = make_float2(Tp[ROWS * TW + i * TW], Tp[2 * ROWS * TW + i * TW]);
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) pb[kk] = make_float2(0.f, 0.f);
#pragma unroll
                        for (int e = 0; e <= 2 * RU; ++e) {
                            const float2 gp = make_float2(tp.gu[e], tp.gu[e]);
#pragma unroll
                            for (int kk = 0; kk < 8; ++kk) pb[kk] = __ffma2_rn(gp, x[kk + e], pb[kk]);
                        }
                    }
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        acc[0][kk] = pa[kk].x; acc[1][kk] = pa[kk].y;
                        acc[2][kk] = pb[kk].x; acc[3][kk] = pb[kk].y;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < (RU > 0 ? 8 + 2 * RU : 8 + 2 * Ru); ++i) {
                        const float t0 = Tp[i * TW], t1 = Tp[ROWS * TW + i * TW], t2 = Tp[2 * ROWS * TW + i * TW];
                        const float tu = ABS ? t0 * (ubase + (float)i) : 0.f;
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) {
                            const int e = i - kk;
                            if (e >= 0 && e <= 2 * Ru) {
                                const float g = tp.gu[e];
                                acc[0][kk] = fmaf(g, t0, acc[0][kk]);
                                if constexpr (ABS) acc[1][kk] = fmaf(g, tu, acc[1][kk]);
                                else acc[1][kk] = fmaf(tp.dgu[e], t0, acc[1][kk]);
                                acc[2][kk] = fmaf(g, t1, acc[2][kk]);
                                acc[3][kk] = fmaf(g, t2, acc[3][kk]);
                            }
                        }
                    }
                }
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const int u = u0 + kr + kk;
                    if (u < H) {
                        float* o = fbase + slice_off + (long long)u * fpitch + v0 + cc;
#pragma unroll
                        for (int f = 0; f < 4; ++f)
                            if (f < nstore) o[f * plane] = acc[f][kk];
                        // h at the output: the pixel's weight on its own gray slice
                        const int si = (kr + kk + Ru) * SW + cc + Rv;
                        const float hx = s_gray[si] != yg ? 0.f : (wimg ? __ldg(wimg + (size_t)u * ipitch + v0 + cc) : 1.f);
                        part = fmaf(hx, acc[0][kk], part);
                    }
                }
            }
        }
        // the tile's S_XX share: FP32 within the warp now, FP64 over the warps by thread 0 after
        // the next barrier (two buffers, so a tile without data cannot overwrite them early)
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) red[t & 1][tid >> 5] = (double)part;
        const long long pidx = (mode ? dp->sxx_off : dp->partial_off) + b;

        // ---- the next tile: its window (staged anew if it changes) and its S
        int nonzero = 0;
        if (t + 1 < t_end) {
            int bn = 0;
            const ImageDesc* dn = locate(t + 1, bn);
            const int ygn = bn % dn->tiles_g, spn = bn / dn->tiles_g;
            if (dn != dp || spn != sp) {
                __syncthreads();   // the pass along u is done with the staged window
                stage(dn, (spn / dn->tiles_v) * TH, (spn % dn->tiles_v) * TW);
                __syncthreads();
            }
            nonzero = s_pass(dn, (spn / dn->tiles_v) * TH, (spn % dn->tiles_v) * TW, ygn);
            dp = dn;
            b = bn;
            yg = ygn;
            sp = spn;
        }
        any = __syncthreads_or(nonzero);
        if (tid == 0) {
            double tot = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) tot += red[t & 1][w];
            L.partials[pidx] = tot;
        }
    }
}

template <int RU, int RV, bool ABS, int TH>
cudaError_t launch_3d(const FieldsLaunch& L, int ntiles, int Ru, int Rv, cudaStream_t s) {
    const int rows = TH + 2 * Ru;
    const int SW = (kTileW + 2 * Rv + 3) & ~3;
    const size_t smem = ((size_t)2 * rows * SW + (size_t)3 * rows * kTileW + ((2 * L.taps.R[2] + 4) & ~3)) * sizeof(float) +
                        (size_t)rows * SW;   // S, S_g, T, T_v, T_g, the g taps, the gray bytes
    auto k = fields3d_kernel<RU, RV, ABS, TH>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem)) != cudaSuccess) return e;
    const int n = ntiles - L.tile_base;
    const int cap = sms * (per_sm > 0 ? per_sm : 1);
    k<<<n < cap ? n : cap, kThreads, smem, s>>>(L, ntiles);
    return cudaGetLastError();
}

template <bool ABS>
cudaError_t dispatch_3d(const FieldsLaunch& L, int ntiles, int Ru, int Rv, cudaStream_t s) {
    if (Ru == Rv) {
        if (Ru == 6) return launch_3d<6, 6, ABS, kGridTileH3>(L, ntiles, Ru, Rv, s);
        if (Ru == 9) return launch_3d<9, 9, ABS, kGridTileH3>(L, ntiles, Ru, Rv, s);
        if (Ru == 12) return launch_3d<12, 12, ABS, kGridTileH3>(L, ntiles, Ru, Rv, s);
    }
    return launch_3d<0, 0, ABS, kGridTileH3>(L, ntiles, Ru, Rv, s);
}

}  // namespace

cudaError_t launch_fields3d(const FieldsLaunch& L, int ntiles, int Ru, int Rv, cudaStream_t s) {
    if (ntiles - L.tile_base <= 0) return cudaSuccess;
    return L.absolute ? dispatch_3d<true>(L, ntiles, Ru, Rv, s) : dispatch_3d<false>(L, ntiles, Ru, Rv, s);
}

}  // namespace itc
