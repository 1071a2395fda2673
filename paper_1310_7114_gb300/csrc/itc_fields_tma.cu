// itc_fields_tma.cu -- 2-D fields (Sec. 3.1, Sec. 5) with TMA-staged input tiles.
//
// Same arithmetic as fields_kernel in itc_fields.cu (the results are bit for bit the same: every
// output accumulates the same products in the same order), reorganised for throughput:
//   * persistent CTAs each walk a contiguous run of the tile list, image lookups loaded ahead;
//   * the input tile plus its halo arrives by one cp.async.bulk.tensor (TMA) per tile into one
//     of two staging buffers (one for 4-byte inputs), so copies run ahead of the tile being
//     computed;
//   * both passes use packed FP32 FMAs (fma.rn.f32x2) over pairs of neighbouring columns.
// Used for 2-D images whose rows start on 16-byte boundaries (the tensor map needs it) and for
// the compiled radii 6, 9 and 12; everything else goes through fields_kernel.
#include <cuda.h>

#include "itc_internal.cuh"

namespace itc {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        "  .reg .pred p;\n"
        "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "  selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

// The class-list position p of the image holding tile t of this launch, found by the whole
// calling warp: a 32-ary search over the class tile prefix (largest p with prefix[p] <= t),
// three dependent loads for 4096 images instead of twelve for a binary search.
__device__ __forceinline__ int locate_pos(const FieldsLaunch& L, int t) {
    const int lane = threadIdx.x & 31;
    const int* prefix = L.tile_prefix;
    int lo = 0, hi = L.nimg - 1;   // prefix[lo] <= t always holds (prefix[0] = 0)
    while (hi - lo >= 32) {
        const int step = (hi - lo + 32) / 32;
        const int idx = lo + lane * step;
        const bool ok = idx <= hi && __ldg(prefix + idx) <= t;
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        const int best = 31 - __clz(m);   // lane 0 always qualifies
        const int nlo = lo + best * step;
        hi = min(hi, nlo + step - 1);
        lo = nlo;
    }
    const int idx = lo + lane;
    const bool ok = idx <= hi && __ldg(prefix + idx) <= t;
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    return lo + 31 - __clz(m);
}

// The image and tile-local index of tile t (whole warp).
__device__ __forceinline__ void locate_warp(const FieldsLaunch& L, int t, int& img, int& local) {
    if (!L.descs) {
        img = 0;
        local = t;
        return;
    }
    const int p = locate_pos(L, t);
    img = __ldg(L.img_list + p);
    local = t - __ldg(L.tile_prefix + p);
}

// Walks the tiles of one CTA's contiguous run in order (warp 0, every lane the same values).
// The image changes only at image boundaries; the next image's entry, first tile and tiles per
// row are loaded one boundary ahead and the list entry of the image after it two ahead, so no
// load issued at a boundary depends on another and no tile waits on a lookup.
struct TileCursor {
    int t, p, img, local, next, tv;   // tile, list position, image, tile in image, first tile of
                                      // the next image, tiles per row of the image
    int n_img, n_next, n_tv;          // the same for position p + 1
    int nn_img;                       // image at position p + 2
    __device__ void start(const FieldsLaunch& L, int t0) {
        t = t0;
        if (!L.descs) {
            p = 0; img = 0; local = t0; next = 0x7fffffff; tv = L.one.tiles_v;
            return;
        }
        p = locate_pos(L, t0);
        img = __ldg(L.img_list + p);
        local = t0 - __ldg(L.tile_prefix + p);
        next = __ldg(L.tile_prefix + p + 1);
        tv = L.descs[img].tiles_v;
        if (p + 1 < L.nimg) {
            n_img = __ldg(L.img_list + p + 1);
            n_next = __ldg(L.tile_prefix + p + 2);
            n_tv = L.descs[n_img].tiles_v;
        }
        if (p + 2 < L.nimg) nn_img = __ldg(L.img_list + p + 2);
    }
    __device__ void advance(const FieldsLaunch& L) {
        ++t;
        ++local;
        if (t == next && L.descs && p + 1 < L.nimg) {
            ++p;
            img = n_img; next = n_next; tv = n_tv; local = 0;
            if (p + 1 < L.nimg) {
                n_img = nn_img;
                n_next = __ldg(L.tile_prefix + p + 2);
                n_tv = L.descs[nn_img].tiles_v;
            }
            if (p + 2 < L.nimg) nn_img = __ldg(L.img_list + p + 2);
        }
    }
};

// Bounded wait for a staged tile: gives up after about one second (2^31 SM clocks); false means
// the copy never landed.
__device__ __forceinline__ bool wait_stage(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1LL << 31)) return false;
    return true;
}

template <int R, bool ABS, int DTYPE, int TH>
__global__ void __launch_bounds__(kThreads, 2) fields_tma_kernel(const __grid_constant__ FieldsLaunch L, int ntiles) {
    constexpr int TW = kTileW, K = TH / 16;
    constexpr int ROWS = TH + 2 * R;
    constexpr int SW = ((TW + 2 * R + 3) & ~3) + 4;
    constexpr int ES = DTYPE == ITC_U8 ? 1 : 4;
    constexpr int RA = DTYPE == ITC_U8 ? 16 : ((R + 3) & ~3);   // box starts 16-byte aligned
    constexpr int BW = TW + 2 * RA;                              // box width in elements
    constexpr int BOX_BYTES = BW * ROWS * ES;
    constexpr int STAGE_BYTES = (BOX_BYTES + 127) & ~127;
    constexpr int NST = STAGE_BYTES <= 16384 ? 2 : 1;           // staging buffers (copies in flight)
    constexpr int NWIN = ((8 + 2 * R) + 3) & ~3;                 // window of 8 row-pass outputs

    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the TMA destination must be 128-byte aligned: round the base up (128 spare bytes reserved)
    unsigned char* stage0 = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);   // NST stages
    float* s_in = reinterpret_cast<float*>(stage0 + NST * STAGE_BYTES);  // ROWS x SW
    float* sT = s_in + ROWS * SW;                                     // T then T_v: ROWS x TW each
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ double red[32];
    __shared__ int s_abort;
    // Zero tracking: rowmask[r] bit q = staged row r has a nonzero in its 4-column group q;
    // colbits[b] = bits over staged rows whose T (8-column block b) is not known to be zero.
    __shared__ uint32_t rowmask[ROWS];
    __shared__ uint32_t colbits[TW / 8][4];
    __shared__ int s_img[2], s_local[2];   // image and local tile of the copy in each stage
    const Taps& tp = L.taps;
    const int tid = threadIdx.x;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
        s_abort = 0;
    }
    __syncthreads();

    // This CTA's tiles: the contiguous run [t_lo, t_hi) of the launch's tiles [tile_base, ntiles),
    // split evenly over the grid, so that neighbouring tiles share their image lookups.
    const long long count = ntiles - L.tile_base;
    const int t_lo = L.tile_base + (int)(count * blockIdx.x / gridDim.x);
    const int t_hi = L.tile_base + (int)(count * (blockIdx.x + 1) / gridDim.x);

    // tile copies run NST tiles ahead: the n-th tile of this CTA lands in stage n % NST
    // called by all of warp 0: remember the cursor's tile for its stage, lane 0 starts the copy
    uint32_t inflight = 0;   // (thread 0) bit b: a copy into stage b has been started, not yet waited for
    TileCursor cur = {};
    auto issue = [&](int buf, bool copy) {
        if (tid == 0) {
            const int tv = cur.local % cur.tv, tu = cur.local / cur.tv;
            const CUtensorMap* map = L.descs ? L.tmaps + cur.img : &L.tmap_one;
            s_img[buf] = cur.img;
            s_local[buf] = cur.local;
            if (copy) {
                mbar_expect_tx(&bar[buf], BOX_BYTES);
                tma_load_2d(stage0 + buf * STAGE_BYTES, map, tv * TW - RA, tu * TH - R, &bar[buf]);
                inflight |= 1u << buf;
            }
        }
        cur.advance(L);
    };

    int t = t_lo;
    if (tid < 32 && t_lo < t_hi) {
        cur.start(L, t_lo);
        for (int b = 0; b < NST; ++b)
            if (t + b < t_hi)
                // the test hook starts no copy for the first tile of CTA 0: its wait cannot end
                issue(b, !(L.test_stall && blockIdx.x == 0 && b == 0));
    }
    uint32_t phase = 0;   // bit b: parity of the next completion of bar[b]
    int n = 0;            // tiles of this CTA so far
    const int kb = tid >> 4, cg = tid & 15;
    const int k0 = kb * K, c0 = cg * 4;
    // S_XX share of the previous tile: its warps leave their sums in red[]; thread 0 adds them
    // (warp order) after the next barrier, so no tile needs a barrier of its own for it
    long long pending = -1;
    auto flush = [&]() {
        if (pending >= 0) {
            static_assert(kThreads / 32 == 8, "eight warp sums");
            // the xor-butterfly order of the block reduction in fields_kernel, so both kernels
            // give bit-identical partials
            const double tot = ((red[0] + red[4]) + (red[2] + red[6])) + ((red[1] + red[5]) + (red[3] + red[7]));
            L.partials[pending] = tot;
            pending = -1;
        }
    };

    for (; t < t_hi; ++t) {
        const int buf = NST == 2 ? (n & 1) : 0;
        const unsigned char* stage = stage0 + buf * STAGE_BYTES;
        if (tid == 0) {
            if (wait_stage(&bar[buf], (phase >> buf) & 1u)) inflight &= ~(1u << buf);
            else s_abort = 1;
        }
        __syncthreads();   // the staged tile has landed; the previous tile's passes are done
        if (tid == 0) flush();
        if (s_abort) {
            // every tile this CTA still owns gets a NaN S_XX share, so each affected image
            // reports a non-finite status; then the copies still in flight land (bounded waits)
            if (tid < 32) {
                for (int tt = t; tt < t_hi; ++tt) {
                    int im, lc;
                    locate_warp(L, tt, im, lc);
                    const ImageDesc* d2 = L.descs ? L.descs + im : &L.one;
                    if (tid == 0) L.partials[d2->partial_off + lc] = __longlong_as_double(0x7ff8000000000000LL);
                }
                if (tid == 0)
                    for (int b = 0; b < NST; ++b)
                        if ((inflight >> b) & 1u) wait_stage(&bar[b], (phase >> b) & 1u);
            }
            __syncthreads();
            return;
        }
        phase ^= 1u << buf;
        ++n;
        const int img = s_img[buf], local = s_local[buf];
        const ImageDesc* dp = L.descs ? L.descs + img : &L.one;
        const int H = dp->H, W = dp->W, fpitch = dp->fpitch;
        const int u0 = (local / dp->tiles_v) * TH, v0 = (local % dp->tiles_v) * TW;
        float* const fbase = L.fields + dp->field_off;
        const long long plane = dp->plane_floats;

        // staged box -> float input tile, columns shifted so that s_in column 0 is v0 - R; one
        // warp per staged row, one 4-column group per lane, a ballot gives the row's zero mask
        int nonzero = 0;
        {
            constexpr int NG = SW / 4;
            static_assert(NG <= 32, "one lane per 4-column group");
            const int wid = tid >> 5, lane = tid & 31;
            for (int r = wid; r < ROWS; r += kThreads / 32) {
                int nz = 0;
                if (lane < NG) {
                    const int c = lane * 4;
                    float x[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int cc = c + j;
                        float v = 0.f;
                        if (cc < TW + 2 * R) {
                            const int sc = r * BW + cc + (RA - R);
                            // byte -> float exactly: 2^23 + b as a float, minus 2^23
                            if (DTYPE == ITC_U8) v = __int_as_float(0x4B000000 | (int)stage[sc]) - 8388608.f;
                            else v = reinterpret_cast<const float*>(stage)[sc];
                        }
                        x[j] = v;
                        nz |= (v != 0.f);
                    }
                    st4(s_in + r * SW + c, x[0], x[1], x[2], x[3]);
                }
                const unsigned m = __ballot_sync(0xffffffffu, nz);
                if (lane == 0) rowmask[r] = m;
                nonzero |= nz;
            }
            if (tid < 32) colbits[tid >> 2][tid & 3] = 0u;
        }
        const int any = __syncthreads_or(nonzero);   // the stage is free from here on
        if (tid < 32 && t + NST < t_hi) issue(buf, true);

        const bool col_active = (u0 + k0 < H) && (v0 + c0 < W);
        if (!any) {
            if (col_active) {
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    const int u = u0 + k0 + kk;
                    if (u >= H) break;
                    float* o = fbase + (long long)u * fpitch + v0 + c0;
#pragma unroll
                    for (int f = 0; f < 3; ++f) st4(o + f * plane, 0.f, 0.f, 0.f, 0.f);
                }
            }
            if (tid == 0) L.partials[dp->partial_off + local] = 0.0;
            continue;
        }

        // ---- pass along v: 8 outputs per item, pairs of neighbouring columns per packed FMA
        for (int item = tid; item < ROWS * 8; item += kThreads) {
            const int r = item >> 3, c = (item & 7) * 8;
            const int gu = u0 - R + r;
            if (v0 + c >= W) continue;
            float* oT = sT + r * TW + c;
            float* oV = oT + ROWS * TW;
            if (gu < 0 || gu >= H) {
                st4(oT, 0.f, 0.f, 0.f, 0.f); st4(oT + 4, 0.f, 0.f, 0.f, 0.f);
                st4(oV, 0.f, 0.f, 0.f, 0.f); st4(oV + 4, 0.f, 0.f, 0.f, 0.f);
                continue;
            }
            constexpr uint32_t WMASK = (1u << (NWIN / 4)) - 1u;
            if (((rowmask[r] >> (c >> 2)) & WMASK) == 0u) {   // every input of the window is zero
                st4(oT, 0.f, 0.f, 0.f, 0.f); st4(oT + 4, 0.f, 0.f, 0.f, 0.f);
                st4(oV, 0.f, 0.f, 0.f, 0.f); st4(oV + 4, 0.f, 0.f, 0.f, 0.f);
                continue;
            }
            atomicOr(&colbits[item & 7][r >> 5], 1u << (r & 31));
            float x[NWIN];
            const float* src = s_in + r * SW + c;
#pragma unroll
            for (int q = 0; q < NWIN / 4; ++q) {
                const float4 f = *reinterpret_cast<const float4*>(src + 4 * q);
                x[4 * q] = f.x; x[4 * q + 1] = f.y; x[4 * q + 2] = f.z; x[4 * q + 3] = f.w;
            }
            float xv[ABS ? NWIN : 1];
            if constexpr (ABS) {
                const float vb = (float)(v0 - R + c);
#pragma unroll
                for (int i = 0; i < NWIN; ++i) xv[i] = x[i] * (vb + (float)i);
            }
            float2 aT[4], aV[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) { aT[p] = f2(0.f, 0.f); aV[p] = f2(0.f, 0.f); }
#pragma unroll
            for (int d = 0; d <= 2 * R; ++d) {
                const float2 g2 = f2(tp.gv[d], tp.gv[d]);
                const float2 dg2 = f2(tp.dgv[d], tp.dgv[d]);
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const float2 xx = f2(x[2 * p + d], x[2 * p + 1 + d]);
                    aT[p] = __ffma2_rn(g2, xx, aT[p]);
                    if constexpr (ABS) aV[p] = __ffma2_rn(g2, f2(xv[2 * p + d], xv[2 * p + 1 + d]), aV[p]);
                    else aV[p] = __ffma2_rn(dg2, xx, aV[p]);
                }
            }
            st4(oT, aT[0].x, aT[0].y, aT[1].x, aT[1].y); st4(oT + 4, aT[2].x, aT[2].y, aT[3].x, aT[3].y);
            st4(oV, aV[0].x, aV[0].y, aV[1].x, aV[1].y); st4(oV + 4, aV[2].x, aV[2].y, aV[3].x, aV[3].y);
        }
        __syncthreads();

        // ---- pass along u: K rows x 4 columns per thread, column pairs per packed FMA
        // T rows k0 .. k0 + K + 2R - 1 of this thread's 8-column block all zero -> outputs are zero
        bool t_any = false;
        if (col_active) {
            const uint32_t* cb = colbits[cg >> 1];
            const int rlo = k0, w0 = rlo >> 5;
            const unsigned long long both = ((unsigned long long)cb[w0 + 1] << 32) | cb[w0];
            const unsigned long long need = (K + 2 * R >= 64) ? ~0ull : ((1ull << (K + 2 * R)) - 1ull);
            t_any = ((both >> (rlo & 31)) & need) != 0ull;
            if (!t_any) {
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    const int u = u0 + k0 + kk;
                    if (u >= H) break;
                    float* o = fbase + (long long)u * fpitch + v0 + c0;
#pragma unroll
                    for (int f = 0; f < 3; ++f) st4(o + f * plane, 0.f, 0.f, 0.f, 0.f);
                }
            }
        }
        float part = 0.f;
        if (col_active && t_any) {
            float2 aA[K][2], aU[K][2], aV[K][2];
#pragma unroll
            for (int kk = 0; kk < K; ++kk)
#pragma unroll
                for (int p = 0; p < 2; ++p) { aA[kk][p] = f2(0.f, 0.f); aU[kk][p] = f2(0.f, 0.f); aV[kk][p] = f2(0.f, 0.f); }
            const float* Tp = sT + k0 * TW + c0;
            const float ub = (float)(u0 - R + k0);
#pragma unroll
            for (int i = 0; i < K + 2 * R; ++i) {
                const float4 t4 = *reinterpret_cast<const float4*>(Tp + i * TW);
                const float4 v4 = *reinterpret_cast<const float4*>(Tp + ROWS * TW + i * TW);
                const float2 t01 = f2(t4.x, t4.y), t23 = f2(t4.z, t4.w);
                const float2 v01 = f2(v4.x, v4.y), v23 = f2(v4.z, v4.w);
                float2 tu01, tu23;
                if constexpr (ABS) {
                    const float uc = ub + (float)i;
                    tu01 = f2(t4.x * uc, t4.y * uc);
                    tu23 = f2(t4.z * uc, t4.w * uc);
                }
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    const int e = i - kk;
                    if (e >= 0 && e <= 2 * R) {
                        const float2 g2 = f2(tp.gu[e], tp.gu[e]);
                        aA[kk][0] = __ffma2_rn(g2, t01, aA[kk][0]);
                        aA[kk][1] = __ffma2_rn(g2, t23, aA[kk][1]);
                        if constexpr (ABS) {
                            aU[kk][0] = __ffma2_rn(g2, tu01, aU[kk][0]);
                            aU[kk][1] = __ffma2_rn(g2, tu23, aU[kk][1]);
                        } else {
                            const float2 dg2 = f2(tp.dgu[e], tp.dgu[e]);
                            aU[kk][0] = __ffma2_rn(dg2, t01, aU[kk][0]);
                            aU[kk][1] = __ffma2_rn(dg2, t23, aU[kk][1]);
                        }
                        aV[kk][0] = __ffma2_rn(g2, v01, aV[kk][0]);
                        aV[kk][1] = __ffma2_rn(g2, v23, aV[kk][1]);
                    }
                }
            }
            float ps = 0.f;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const int u = u0 + k0 + kk;
                if (u < H) {
                    float* o = fbase + (long long)u * fpitch + v0 + c0;
                    st4(o, aA[kk][0].x, aA[kk][0].y, aA[kk][1].x, aA[kk][1].y);
                    st4(o + plane, aU[kk][0].x, aU[kk][0].y, aU[kk][1].x, aU[kk][1].y);
                    st4(o + 2 * plane, aV[kk][0].x, aV[kk][0].y, aV[kk][1].x, aV[kk][1].y);
                    const float* hrow = s_in + (k0 + kk + R) * SW + c0 + R;
                    const float a4[4] = {aA[kk][0].x, aA[kk][0].y, aA[kk][1].x, aA[kk][1].y};
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (v0 + c0 + j < W) ps = fmaf(hrow[j], a4[j], ps);
                }
            }
            part = ps;
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((tid & 31) == 0) red[tid >> 5] = (double)part;   // FP32 within a warp, FP64 across warps
        if (tid == 0) pending = dp->partial_off + local;
    }
    __syncthreads();
    if (tid == 0) flush();
}

template <int R, bool ABS, int DTYPE, int TH>
cudaError_t launch_tma(const FieldsLaunch& L, int ntiles, cudaStream_t s) {
    constexpr int TW = kTileW;
    constexpr int ROWS = TH + 2 * R;
    constexpr int SW = ((TW + 2 * R + 3) & ~3) + 4;
    constexpr int ES = DTYPE == ITC_U8 ? 1 : 4;
    constexpr int RA = DTYPE == ITC_U8 ? 16 : ((R + 3) & ~3);
    constexpr int BOX_BYTES = (TW + 2 * RA) * ROWS * ES;
    constexpr int STAGE_BYTES = (BOX_BYTES + 127) & ~127;
    constexpr int NST = STAGE_BYTES <= 16384 ? 2 : 1;
    const size_t smem = 128 + NST * (size_t)STAGE_BYTES + (size_t)ROWS * SW * 4 + 2 * (size_t)ROWS * TW * 4;
    auto k = fields_tma_kernel<R, ABS, DTYPE, TH>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem)) != cudaSuccess) return e;
    if (L.grid_per_sm > 0 && L.grid_per_sm < per_sm) per_sm = L.grid_per_sm;   // tuned persistent grid
    const int count = ntiles - L.tile_base;
    const int grid = count < sms * (per_sm > 0 ? per_sm : 1) ? count : sms * (per_sm > 0 ? per_sm : 1);
    k<<<grid, kThreads, smem, s>>>(L, ntiles);
    return cudaGetLastError();
}

template <bool ABS, int DTYPE>
cudaError_t dispatch(const FieldsLaunch& L, int ntiles, int R, cudaStream_t s) {
    if (L.tile_h == 32) {
        if (R == 6) return launch_tma<6, ABS, DTYPE, 32>(L, ntiles, s);
        if (R == 9) return launch_tma<9, ABS, DTYPE, 32>(L, ntiles, s);
        return launch_tma<12, ABS, DTYPE, 32>(L, ntiles, s);
    }
    if (R == 6) return launch_tma<6, ABS, DTYPE, 64>(L, ntiles, s);
    if (R == 9) return launch_tma<9, ABS, DTYPE, 64>(L, ntiles, s);
    return launch_tma<12, ABS, DTYPE, 64>(L, ntiles, s);
}

}  // namespace

bool fields_tma_supported(int ndim, int Ru, int Rv) {
    return ndim == 2 && Ru == Rv && (Ru == 6 || Ru == 9 || Ru == 12);
}

int fields_tma_box(int dtype, int R, int tile_h, int* box_w, int* box_h) {
    const int ra = dtype == ITC_U8 ? 16 : ((R + 3) & ~3);
    *box_w = kTileW + 2 * ra;
    *box_h = tile_h + 2 * R;
    return 0;
}

cudaError_t launch_fields_tma(const FieldsLaunch& L, int ntiles, int R, int dtype, cudaStream_t s) {
    if (ntiles - L.tile_base <= 0) return cudaSuccess;
    const bool abs_ = L.absolute != 0;
    if (dtype == ITC_U8) return abs_ ? dispatch<true, ITC_U8>(L, ntiles, R, s) : dispatch<false, ITC_U8>(L, ntiles, R, s);
    return abs_ ? dispatch<true, ITC_F32>(L, ntiles, R, s) : dispatch<false, ITC_F32>(L, ntiles, R, s);
}

}  // namespace itc
