// itc_fields_tma.cu -- 2-D fields (Sec. 3.1, Sec. 5) with TMA-staged input tiles.
//
// Same arithmetic as fields_kernel in itc_fields.cu (the results are bit for bit the same: every
// output accumulates the same products in the same order), reorganised for throughput:
//   * persistent CTAs take chunks of consecutive tiles from a per-launch counter, image lookups
//     loaded ahead;
//   * the input tile plus its halo arrives by one cp.async.bulk.tensor (TMA) per tile into one
//     of three staging buffers (two for 4-byte inputs and for 64-row byte tiles at R = 12), so
//     copies run ahead of the tile being computed;
//   * byte inputs skip the arithmetic of windows without data, store precomputed chains for
//     windows of ones, take windows that are one run of 0/1 inputs from a table of chains, and
//     run the rest of the row pass warp-compacted;
//   * the row pass reads its input windows straight from the staged box (bytes are turned into
//     floats in registers), so a tile needs two barriers and no float copy of its input, and three
//     CTAs fit on an SM for byte inputs;
//   * both passes use packed FP32 FMAs (fma.rn.f32x2): the row pass of byte inputs over pairs of
//     neighbouring rows (each packed operand holds the same column of two rows, so no pair is
//     realigned), the row pass of float inputs and the column pass over pairs of neighbouring
//     columns.
// Used for 2-D images whose rows start on 16-byte boundaries (the tensor map needs it) and for
// the compiled radii 6, 9 and 12; other 2-D images go through fields_kernel, gray images through
// fields3d_kernel (itc_fields3d.cu).
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

// Bytes of 4-byte word q that lie in the window [OFF, OFF + N) of a row pass item.
template <int OFF, int N>
__device__ __forceinline__ constexpr uint32_t window_mask(int q) {
    uint32_t m = 0u;
    for (int k = 0; k < 4; ++k) {
        const int b = 4 * q + k;
        if (b >= OFF && b < OFF + N) m |= 0xffu << (8 * k);
    }
    return m;
}

// Tiles a persistent CTA takes from the launch's counter at a time.
constexpr int kFieldsChunk = 4;
// Row-pass items start at (tid + kItemRotate) mod kThreads: the threads of warps 0 and 1 take the
// last item numbers of each round, so when a tile's items do not fill the last round those warps
// have one item fewer -- thread 0 also adds up the previous tile's S_XX share before its items.
constexpr int kItemRotate = kThreads - 64;

// Bounded wait for a staged tile: gives up after about one second (2^31 SM clocks); false means
// the copy never landed.
__device__ __forceinline__ bool wait_stage(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1LL << 31)) return false;
    return true;
}

// Compile-time shape of one tile (rows TH + 2R of the staged box, stages in flight).
template <int R, bool ABS, int DTYPE, int TH>
struct TmaTile {
    static constexpr int TW = kTileW, K = TH / 16;
    static constexpr int ROWS = TH + 2 * R;
    static constexpr int ES = DTYPE == ITC_U8 ? 1 : 4;
    static constexpr int RA = DTYPE == ITC_U8 ? 16 : ((R + 3) & ~3);   // box starts 16-byte aligned
    static constexpr int BW = TW + 2 * RA;                              // box width in elements
    static constexpr int BOX_BYTES = BW * ROWS * ES;
    static constexpr int STAGE_BYTES = (BOX_BYTES + 127) & ~127;
    static constexpr int NST = STAGE_BYTES <= 8192 ? 3 : 2;            // staging buffers
    // byte inputs with centred moments and R >= 9 take row windows that are one run of 0/1 inputs
    // from a table (below); it does not fit beside 128-row tiles at R = 12
    static constexpr bool RUNS = DTYPE == ITC_U8 && !ABS && R >= 9 && !(TH == 128 && R == 12);
    static constexpr int NTAP = 2 * R + 1;
    static constexpr int T2 = (NTAP + 1) * (NTAP + 2) / 2;             // runs [a, b), 0 <= a <= b <= NTAP
    static constexpr size_t TAB_BYTES = RUNS ? 2 * (size_t)T2 * 8 : 0;
    static constexpr size_t SMEM = 128 + (size_t)NST * STAGE_BYTES + 2 * (size_t)ROWS * TW * 4 + TAB_BYTES;
    static constexpr int MIN_CTAS = (DTYPE == ITC_U8 && TH == 64) ? 3 : 2;
};

template <int R, bool ABS, int DTYPE, int TH>
__global__ void __launch_bounds__(kThreads, (TmaTile<R, ABS, DTYPE, TH>::MIN_CTAS))
    fields_tma_kernel(const __grid_constant__ FieldsLaunch L, int ntiles) {
    using TT = TmaTile<R, ABS, DTYPE, TH>;
    constexpr int TW = TT::TW, K = TT::K, ROWS = TT::ROWS, RA = TT::RA, BW = TT::BW;
    constexpr int BOX_BYTES = TT::BOX_BYTES, STAGE_BYTES = TT::STAGE_BYTES, NST = TT::NST;
    constexpr int OFF = (RA - R) & 3;                // a window's first input within its 4-group
    constexpr int NWIN = 8 + 2 * R;                  // inputs of 8 neighbouring outputs (one-row pass)
    constexpr int NQ = (OFF + NWIN + 3) / 4;         // 4-element groups covering that window

    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the TMA destination must be 128-byte aligned: round the base up (128 spare bytes reserved)
    unsigned char* stage0 = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);   // NST stages
    float* sT = reinterpret_cast<float*>(stage0 + NST * STAGE_BYTES);   // T then T_v: ROWS x TW each
    // (T, T_v) of every window of 0/1 inputs that is one run: ones on [a, b) at entry
    // b (b + 1) / 2 + a, ones outside [a, b) at T2 + that entry
    float2* s_run = reinterpret_cast<float2*>(sT + 2 * ROWS * TW);
    __shared__ __align__(8) uint64_t bar[NST];
    __shared__ double red[32];
    __shared__ int s_abort;
    // colbits[p][b] (tile parity p): bits over staged rows whose T in 8-column block b is not
    // known to be zero; the buffer of the next tile is cleared while this one is read
    constexpr int CBW = (ROWS + 31) / 32 + 1;   // words per block and parity (one spare for 64-bit reads)
    __shared__ uint32_t colbits[2][TW / 8][CBW];
    __shared__ int s_img[NST], s_local[NST];   // image and local tile of the copy in each stage
    const Taps& tp = L.taps;
    const int tid = threadIdx.x;

    if (tid == 0) {
        for (int b = 0; b < NST; ++b) mbar_init(&bar[b], 1);
        mbar_init_fence();
        s_abort = 0;
    }
    for (int i = tid; i < 2 * (TW / 8) * CBW; i += kThreads) (&colbits[0][0][0])[i] = 0u;
    if constexpr (TT::RUNS) {
        // each entry is the row pass's own FMA chain over the taps with inputs 1 on the run and 0
        // elsewhere, so a window that is such a run gets the bits the FMAs would give
        for (int e = tid; e < 2 * TT::T2; e += kThreads) {
            const bool outside = e >= TT::T2;
            const int t = outside ? e - TT::T2 : e;
            int b = 0;
            while ((b + 1) * (b + 2) / 2 <= t) ++b;
            const int a = t - b * (b + 1) / 2;
            float accT = 0.f, accV = 0.f;
#pragma unroll
            for (int d = 0; d < TT::NTAP; ++d) {
                const float x = ((d >= a && d < b) != outside) ? 1.f : 0.f;
                accT = fmaf(tp.gv[d], x, accT);
                accV = fmaf(tp.dgv[d], x, accV);
            }
            s_run[e] = make_float2(accT, accV);
        }
    }
    __syncthreads();

    // Tiles are handed out dynamically, kFieldsChunk consecutive tiles at a time, from the launch's
    // counter (zero at launch), so that CTAs whose tiles hold more data do not finish last: a
    // persistent CTA takes a new chunk whenever it has issued the copies of its last one.  Warp 0
    // walks the chunk's tiles with a cursor (image lookups loaded ahead within the chunk) and
    // takes the next chunk's index one chunk ahead, so the atomic's latency is hidden.
    // tile copies run up to NST - 1 tiles ahead: the n-th tile of this CTA lands in stage n % NST,
    // whose previous tile (n - NST) has finished both passes by the time the copy is started
    uint32_t inflight = 0;   // (thread 0) bit b: a copy into stage b has been started, not yet waited for
    // the cursor lives in shared memory and is advanced by thread 0 alone (it costs the other
    // threads no registers)
    __shared__ TileCursor s_cur;
    __shared__ int s_chunk_end;    // first tile past the cursor's chunk; -1 once the tiles are exhausted
    __shared__ int s_valid[NST];   // the stage holds a tile of this CTA
    int next_chunk = 0;            // (lane 0 of warp 0) index of the chunk after the current one
    // called by all of warp 0: the next tile of this CTA goes to stage `buf` (or none is left)
    auto issue = [&](int buf, bool copy) {
        __syncwarp();
        if (s_chunk_end >= 0 && s_cur.t >= s_chunk_end) {   // warp-uniform: start the next chunk
            const int c = __shfl_sync(0xffffffffu, next_chunk, 0);
            const long long t0 = (long long)L.tile_base + (long long)c * kFieldsChunk;
            if (t0 >= ntiles) {
                if (tid == 0) s_chunk_end = -1;
            } else {
                if (tid == 0) next_chunk = atomicAdd(L.counter, 1);   // consumed one chunk later
                TileCursor c0 = {};
                c0.start(L, (int)t0);   // the whole warp: a warp search
                if (tid == 0) {
                    s_cur = c0;
                    s_chunk_end = (int)(t0 + kFieldsChunk < ntiles ? t0 + kFieldsChunk : ntiles);
                }
            }
            __syncwarp();
        }
        if (tid == 0) {
            s_valid[buf] = s_chunk_end >= 0;
            if (s_chunk_end >= 0) {
                const int tv = s_cur.local % s_cur.tv, tu = s_cur.local / s_cur.tv;
                const CUtensorMap* map = L.descs ? L.tmaps + s_cur.img : &L.tmap_one;
                s_img[buf] = s_cur.img;
                s_local[buf] = s_cur.local;
                if (copy) {
                    mbar_expect_tx(&bar[buf], BOX_BYTES);
                    tma_load_2d(stage0 + buf * STAGE_BYTES, map, tv * TW - RA, tu * TH - R, &bar[buf]);
                    inflight |= 1u << buf;
                }
                s_cur.advance(L);
            }
        }
    };

    if (tid < 32) {
        if (tid == 0) {
            next_chunk = atomicAdd(L.counter, 1);
            s_cur.t = 0;
            s_chunk_end = 0;   // no chunk yet: the first issue takes one
        }
        for (int b = 0; b < NST; ++b)
            // the test hook starts no copy for the first tile of CTA 0: its wait cannot end
            issue(b, !(L.test_stall && blockIdx.x == 0 && b == 0));
    }
    __syncthreads();   // s_valid of the first stages
    uint32_t phase = 0;   // bit b: parity of the next completion of bar[b]
    int n = 0;            // tiles of this CTA so far
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

    // element i of a staged 4-group q: bytes -> float exactly (2^23 + b as a float, minus 2^23)
    auto elem = [&](const uint32_t (&w)[NQ > 0 ? NQ * (DTYPE == ITC_U8) + 1 : 1], const float4 (&f)[NQ], int i) -> float {
        if constexpr (DTYPE == ITC_U8)
            return __int_as_float((int)__byte_perm(w[i >> 2], 0x4B000000u, 0x7540u | (unsigned)(i & 3))) - 8388608.f;
        else {
            const float4 g = f[i >> 2];
            return (i & 3) == 0 ? g.x : ((i & 3) == 1 ? g.y : ((i & 3) == 2 ? g.z : g.w));
        }
    };

    // Byte inputs (binary images: most windows hold no data) with the widest masks compact the row
    // pass per warp: each warp first lists those of its items whose windows hold data (the others
    // store their zeros meanwhile), then runs the listed items on consecutive lanes, so that its
    // packed FMAs run on full lanes (a warp whose lanes diverge keeps the FMA pipe busy for its
    // idle lanes too).  An item computes the same products in the same order whichever lane takes
    // it.  Items whose two windows are all ones are not listed either (their outputs are
    // constants).  On the ragged binary batch this pays at every radius: 0.382 / 0.499 / 0.570 ms
    // at R = 6 / 9 / 12 against 0.384 / 0.509 / 0.571 ms with the items run in place.  A listed
    // item of 0/1 inputs whose row windows are one run each (98-99 % of them on that batch) takes
    // its outputs from the run table instead of the FMAs (R >= 9: 0.497 / 0.541 ms at R = 9 / 12
    // with two stages at R = 12; at R = 6 the FMAs cost no more than the table's index arithmetic).
    constexpr bool COMPACT = DTYPE == ITC_U8;
    constexpr int NITEMS = ROWS * 8;                 // row-pass items of a tile (8 per staged row)
    constexpr int NROUNDS = (NITEMS + kThreads - 1) / kThreads;
    __shared__ short s_items[COMPACT ? kThreads / 32 : 1][COMPACT ? NROUNDS * 32 : 1];   // per warp
    const int lane = tid & 31;
    const unsigned lanes_below = (1u << lane) - 1u;
    const int rot = (tid + kItemRotate) & (kThreads - 1);   // first item of this thread

    // the column unit (K rows x 4 columns at rows k0.., columns c0..): A, F_u, F_v with packed FMAs
    // over column pairs, stored; returns the unit's share of S_XX (h from the staged box)
    auto column_unit = [&](const unsigned char* stage, int k0, int c0, int u0, int v0, int H, int W, int fpitch,
                           float* fbase, long long plane) -> float {
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
                // h at the four outputs, from the staged box (row k0 + kk + R, columns RA + c0 ..)
                float h4[4];
                if constexpr (DTYPE == ITC_U8) {
                    const uint32_t hw = *reinterpret_cast<const uint32_t*>(stage + (k0 + kk + R) * BW + RA + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        h4[j] = __int_as_float((int)__byte_perm(hw, 0x4B000000u, 0x7540u | (unsigned)j)) - 8388608.f;
                } else {
                    const float4 hf = *reinterpret_cast<const float4*>(stage + ((size_t)(k0 + kk + R) * BW + RA + c0) * 4);
                    h4[0] = hf.x; h4[1] = hf.y; h4[2] = hf.z; h4[3] = hf.w;
                }
                const float a4[4] = {aA[kk][0].x, aA[kk][0].y, aA[kk][1].x, aA[kk][1].y};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (v0 + c0 + j < W) ps = fmaf(h4[j], a4[j], ps);
            }
        }
        return ps;
    };
    // the column unit of thread tid: inside the image, and any T row of its window nonzero
    auto unit_state = [&](int k0, int c0, int cgb, int par, int u0, int v0, int H, int W, bool* active) -> bool {
        const bool col_active = (u0 + k0 < H) && (v0 + c0 < W);
        bool t_any = false;
        if (col_active) {
            const uint32_t* cb = colbits[par][cgb];
            const int w0 = k0 >> 5;
            const unsigned long long both = ((unsigned long long)cb[w0 + 1] << 32) | cb[w0];
            const unsigned long long need = (K + 2 * R >= 64) ? ~0ull : ((1ull << (K + 2 * R)) - 1ull);
            t_any = ((both >> (k0 & 31)) & need) != 0ull;
        }
        *active = col_active && t_any;
        return col_active;
    };
    auto zero_unit = [&](int k0, int c0, int u0, int v0, int H, int fpitch, float* fbase, long long plane) {
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            const int u = u0 + k0 + kk;
            if (u >= H) break;
            float* o = fbase + (long long)u * fpitch + v0 + c0;
#pragma unroll
            for (int ff = 0; ff < 3; ++ff) st4(o + ff * plane, 0.f, 0.f, 0.f, 0.f);
        }
    };

    for (;;) {
        const int buf = n % NST;
        const unsigned char* stage = stage0 + buf * STAGE_BYTES;
        if (tid == 0 && s_valid[buf]) {
            if (wait_stage(&bar[buf], (phase >> buf) & 1u)) inflight &= ~(1u << buf);
            else s_abort = 1;
        }
        __syncthreads();   // the staged tile has landed; the previous tile's passes are done
        if (tid == 0) flush();
        if (!s_valid[buf]) break;   // no tiles left for this CTA (uniform: read after the barrier)
        if (s_abort) {
            // every tile this CTA still owns -- this one, those staged ahead and the rest of its
            // chunk -- gets a NaN S_XX share and its image the status ITC_ERR_TIMEOUT (their fields
            // stay unwritten); then the copies still in flight land (bounded waits)
            if (tid < 32) {
                auto mark = [&](int im, int lc) {
                    const ImageDesc* d2 = L.descs ? L.descs + im : &L.one;
                    L.partials[d2->partial_off + lc] = __longlong_as_double(0x7ff8000000000000LL);
                    if (L.status) L.status[L.descs ? im : 0] = ITC_ERR_TIMEOUT;
                };
                // staged: tiles n .. n + NST - 1 before the first tile's wait, n .. n + NST - 2 later
                // (the last stage still holds tile n - 1, whose share is already written)
                if (tid == 0)
                    for (int b = 0; b < (n == 0 ? NST : NST - 1); ++b)
                        if (s_valid[(buf + b) % NST]) mark(s_img[(buf + b) % NST], s_local[(buf + b) % NST]);
                for (int tt = s_cur.t; s_chunk_end >= 0 && tt < s_chunk_end; ++tt) {
                    int im, lc;
                    locate_warp(L, tt, im, lc);
                    if (tid == 0) mark(im, lc);
                }
                // and the chunk taken ahead, which no other CTA will take
                const long long tn = (long long)L.tile_base + (long long)__shfl_sync(0xffffffffu, next_chunk, 0) * kFieldsChunk;
                for (long long tt = tn; s_chunk_end >= 0 && tt < tn + kFieldsChunk && tt < ntiles; ++tt) {
                    int im, lc;
                    locate_warp(L, (int)tt, im, lc);
                    if (tid == 0) mark(im, lc);
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
        const int par = n & 1;
        if (tid < (TW / 8) * CBW) (&colbits[par ^ 1][0][0])[tid] = 0u;   // for the next tile
        const int img = s_img[buf], local = s_local[buf];
        const ImageDesc* dp = L.descs ? L.descs + img : &L.one;
        const int H = dp->H, W = dp->W, fpitch = dp->fpitch;
        const int u0 = (local / dp->tiles_v) * TH, v0 = (local % dp->tiles_v) * TW;
        float* const fbase = L.fields + dp->field_off;
        const long long plane = dp->plane_floats;

        if constexpr (DTYPE == ITC_U8) {
            // ---- pass along v, read straight from the staged box.  An item is 4 outputs in each of
            // two neighbouring rows: the two rows' inputs are the halves of every packed operand, so
            // the packed FMAs need no realigned pairs
            constexpr int NW4 = 4 + 2 * R;                   // inputs of 4 neighbouring outputs
            constexpr int NQ4 = (OFF + NW4 + 3) / 4;         // 4-element groups covering the window
            // the item's input words (box columns c - R + RA - OFF .., a multiple of 4) of its two
            // rows; the staged box holds zeros outside the image (the copy's fill beyond the tensor
            // map's bounds), so rows and columns outside need no test (1.385 -> 1.353 ms on C3)
            auto load_item = [&](int item, uint32_t (&w0)[NQ4], uint32_t (&w1)[NQ4]) {
                const int r0 = (item >> 4) * 2, c = (item & 15) * 4;
                const int g0 = (c - R + RA - OFF) >> 2;
                const uint32_t* row0 = reinterpret_cast<const uint32_t*>(stage + r0 * BW);
                const uint32_t* row1 = row0 + BW / 4;
#pragma unroll
                for (int q = 0; q < NQ4; ++q) {
                    w0[q] = row0[g0 + q];
                    w1[q] = row1[g0 + q];
                }
            };
            // one item from its input words: inputs as (row r0, row r0 + 1) pairs, bytes -> floats
            // exactly (2^23 + b, minus 2^23), the two masks' FMAs, T and T_v stored
            auto compute_item = [&](int item, const uint32_t (&w0)[NQ4], const uint32_t (&w1)[NQ4]) {
                const int r0 = (item >> 4) * 2, c = (item & 15) * 4;
                float2 X[NW4];
#pragma unroll
                for (int i = 0; i < NW4; ++i) {
                    const int e = OFF + i;
                    const float a0 = __int_as_float((int)__byte_perm(w0[e >> 2], 0x4B000000u, 0x7540u | (unsigned)(e & 3)));
                    const float a1 = __int_as_float((int)__byte_perm(w1[e >> 2], 0x4B000000u, 0x7540u | (unsigned)(e & 3)));
                    X[i] = __fadd2_rn(f2(a0, a1), f2(-8388608.f, -8388608.f));
                }
                float2 XV[ABS ? NW4 : 1];
                if constexpr (ABS) {
                    const float vb = (float)(v0 - R + c);
#pragma unroll
                    for (int i = 0; i < NW4; ++i) {
                        const float pv = vb + (float)i;
                        XV[i] = f2(X[i].x * pv, X[i].y * pv);
                    }
                }
                float2 aT[4], aV[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) { aT[jj] = f2(0.f, 0.f); aV[jj] = f2(0.f, 0.f); }
#pragma unroll
                for (int d = 0; d <= 2 * R; ++d) {
                    const float2 g2 = f2(tp.gv[d], tp.gv[d]);
                    const float2 dg2 = f2(tp.dgv[d], tp.dgv[d]);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        aT[jj] = __ffma2_rn(g2, X[jj + d], aT[jj]);
                        if constexpr (ABS) aV[jj] = __ffma2_rn(g2, XV[jj + d], aV[jj]);
                        else aV[jj] = __ffma2_rn(dg2, X[jj + d], aV[jj]);
                    }
                }
                float* oT = sT + r0 * TW + c;
                float* oV = oT + ROWS * TW;
                st4(oT, aT[0].x, aT[1].x, aT[2].x, aT[3].x); st4(oT + TW, aT[0].y, aT[1].y, aT[2].y, aT[3].y);
                st4(oV, aV[0].x, aV[1].x, aV[2].x, aV[3].x); st4(oV + TW, aV[0].y, aV[1].y, aV[2].y, aV[3].y);
            };
            // one item from the run table when both of its row windows (4 + 2R inputs) hold only 0
            // and 1 with at most two changes along the row, i.e. one run of ones or one run of
            // zeros; each output's window then holds that run clipped to its 2R + 1 taps.  False
            // (nothing stored) for any other item.  Binary shapes give such windows almost always.
            auto run_item = [&](int item, const uint32_t (&w0)[NQ4], const uint32_t (&w1)[NQ4]) -> bool {
                if constexpr (!TT::RUNS) {
                    return false;
                } else {
                    constexpr int N = TT::NTAP;
                    constexpr uint32_t FULL = (1u << NW4) - 1u;     // NW4 <= 28
                    constexpr uint32_t EDGES = (1u << (NW4 - 1)) - 1u;
                    uint32_t high = 0u, m0 = 0u, m1 = 0u;
#pragma unroll
                    for (int q = 0; q < NQ4; ++q) {
                        high |= (w0[q] | w1[q]) & (0xfefefefeu & window_mask<OFF, NW4>(q));
                        // the low bits of the 4 bytes gathered into 4 bits (no carries: the 16
                        // partial products land on distinct bits)
                        m0 |= (((w0[q] & 0x01010101u) * 0x01020408u) >> 24) << (4 * q);
                        m1 |= (((w1[q] & 0x01010101u) * 0x01020408u) >> 24) << (4 * q);
                    }
                    m0 = (m0 >> OFF) & FULL;   // bit i: input at column c - R + i
                    m1 = (m1 >> OFF) & FULL;
                    if (high != 0u || __popc((m0 ^ (m0 >> 1)) & EDGES) > 2 || __popc((m1 ^ (m1 >> 1)) & EDGES) > 2)
                        return false;
                    const int r0 = (item >> 4) * 2, c = (item & 15) * 4;
                    float tv[2][2][4];   // [T or T_v][row][output]
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t m = h ? m1 : m0;
                        const bool zeros = (m & 1u) != 0u;            // starts with a one: a run of zeros
                        const uint32_t run = zeros ? (~m & FULL) : m;
                        const int a = run ? __ffs((int)run) - 1 : 0, b = a + __popc(run);
                        const int base = zeros ? TT::T2 : 0;
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const int aa = min(max(a - jj, 0), N), bb = min(max(b - jj, 0), N);
                            const float2 e = s_run[base + (bb * (bb + 1) >> 1) + aa];
                            tv[0][h][jj] = e.x;
                            tv[1][h][jj] = e.y;
                        }
                    }
                    float* oT = sT + r0 * TW + c;
                    float* oV = oT + ROWS * TW;
                    st4(oT, tv[0][0][0], tv[0][0][1], tv[0][0][2], tv[0][0][3]);
                    st4(oT + TW, tv[0][1][0], tv[0][1][1], tv[0][1][2], tv[0][1][3]);
                    st4(oV, tv[1][0][0], tv[1][0][1], tv[1][0][2], tv[1][0][3]);
                    st4(oV + TW, tv[1][1][0], tv[1][1][1], tv[1][1][2], tv[1][1][3]);
                    return true;
                }
            };
            // every item of this thread: windows without data store zeros; with COMPACT the items
            // with data are listed per warp and run afterwards on consecutive lanes, otherwise
            // they run in place
            short* wl = s_items[COMPACT ? (tid >> 5) : 0];
            int cnt = 0;   // warp-uniform
            // the rounds unrolled (their window loads overlap): 1.345 -> 1.330 ms on C3; absolute
            // moments keep one round at a time (unrolled, they spill at 80 registers)
            constexpr int ROUND_UNROLL = ABS ? 1 : NROUNDS;
#pragma unroll ROUND_UNROLL
            for (int k = 0; k < NROUNDS; ++k) {
                const int item = rot + k * kThreads;
                const int r0 = (item >> 4) * 2, c = (item & 15) * 4;
                bool nz0 = false, nz1 = false, ones = false;
                if (item < NITEMS && v0 + c < W) {
                    uint32_t w0[NQ4], w1[NQ4];
                    load_item(item, w0, w1);
#pragma unroll
                    for (int q = 0; q < NQ4; ++q) {
                        nz0 |= w0[q] != 0u;
                        nz1 |= w1[q] != 0u;
                    }
                    if (!(nz0 | nz1)) {
                        float* oT = sT + r0 * TW + c;
                        float* oV = oT + ROWS * TW;
                        st4(oT, 0.f, 0.f, 0.f, 0.f); st4(oT + TW, 0.f, 0.f, 0.f, 0.f);
                        st4(oV, 0.f, 0.f, 0.f, 0.f); st4(oV + TW, 0.f, 0.f, 0.f, 0.f);
                    }
                    // rows r0 and r0 + 1 (r0 even) share a word of the column bits
                    const uint32_t rb = (nz0 ? 1u : 0u) | (nz1 ? 2u : 0u);
                    if (rb) atomicOr(&colbits[par][c >> 3][r0 >> 5], rb << (r0 & 31));
                    // both windows all ones (shape interiors; centred moments): T and T_v are the
                    // FMA chains of the taps, prepared on the host
                    if constexpr (!ABS) {
                        if (nz0 & nz1) {
                            uint32_t diff = 0u;
#pragma unroll
                            for (int q = 0; q < NQ4; ++q)
                                diff |= ((w0[q] ^ 0x01010101u) | (w1[q] ^ 0x01010101u)) & window_mask<OFF, NW4>(q);
                            ones = diff == 0u;
                        }
                    }
                    if (ones) {
                        float* oT = sT + r0 * TW + c;
                        float* oV = oT + ROWS * TW;
                        const float a = tp.ones_gv, b = tp.ones_dgv;
                        st4(oT, a, a, a, a); st4(oT + TW, a, a, a, a);
                        st4(oV, b, b, b, b); st4(oV + TW, b, b, b, b);
                    }
                    if constexpr (!COMPACT)
                        if ((nz0 | nz1) && !ones) compute_item(item, w0, w1);
                }
                if constexpr (COMPACT) {
                    const bool mixed = (nz0 | nz1) && !ones;
                    const unsigned ba = __ballot_sync(0xffffffffu, mixed);
                    if (mixed) wl[cnt + __popc(ba & lanes_below)] = (short)item;
                    cnt += __popc(ba);
                }
            }
            if constexpr (COMPACT) {
                __syncwarp();
                for (int j = lane; j < cnt; j += 32) {
                    const int item = wl[j];
                    uint32_t w0[NQ4], w1[NQ4];
                    load_item(item, w0, w1);
                    if (!run_item(item, w0, w1)) compute_item(item, w0, w1);
                }
            }
        } else {
            // 4-byte inputs: 8 outputs of one row per item, pairs of neighbouring columns per packed
            // FMA (the pairs of rows of byte inputs would need register moves here)
            // ---- pass along v, read straight from the staged box: 8 outputs per item, pairs of
            // neighbouring columns per packed FMA; windows without data store zeros
            for (int item = rot; item < ROWS * 8; item += kThreads) {
                const int r = item >> 3, c = (item & 7) * 8;
                const int gu = u0 - R + r;
                if (v0 + c >= W) continue;
                float* oT = sT + r * TW + c;
                float* oV = oT + ROWS * TW;
                // the window's 4-groups: box columns c - R + RA - OFF ... (a multiple of 4)
                const int g0 = (c - R + RA - OFF) >> 2;
                uint32_t w[NQ * (DTYPE == ITC_U8) + 1];
                float4 f[NQ];
                bool nz = false;
                if (gu >= 0 && gu < H) {
                    const float4* row = reinterpret_cast<const float4*>(stage + (size_t)r * BW * 4);
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        f[q] = row[g0 + q];
                        nz |= (f[q].x != 0.f) | (f[q].y != 0.f) | (f[q].z != 0.f) | (f[q].w != 0.f);
                    }
                }
                if (!nz) {
                    st4(oT, 0.f, 0.f, 0.f, 0.f); st4(oT + 4, 0.f, 0.f, 0.f, 0.f);
                    st4(oV, 0.f, 0.f, 0.f, 0.f); st4(oV + 4, 0.f, 0.f, 0.f, 0.f);
                    continue;
                }
                atomicOr(&colbits[par][item & 7][r >> 5], 1u << (r & 31));
                float x[NWIN];
#pragma unroll
                for (int i = 0; i < NWIN; ++i) x[i] = elem(w, f, OFF + i);
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
        }
        __syncthreads();
        // the stage of the previous tile is free: start the copy NST - 1 tiles ahead into it.
        // Warp 0 does this here rather than before its row items: every warp waits at the barrier
        // above for the last one to finish its row items (1.386 against 1.408 ms on the C3 batch)
        if (tid < 32 && n > 1) issue((n - 2) % NST, true);
        // ---- pass along u: K rows x 4 columns per thread, column pairs per packed FMA; a unit
        // whose T rows k0 .. k0 + K + 2R - 1 of its 8-column block are all zero stores zeros
        const int k0 = (tid >> 4) * K, c0 = (tid & 15) * 4;
        bool active;
        const bool inside = unit_state(k0, c0, (tid & 15) >> 1, par, u0, v0, H, W, &active);
        if (inside && !active) zero_unit(k0, c0, u0, v0, H, fpitch, fbase, plane);
        float part = active ? column_unit(stage, k0, c0, u0, v0, H, W, fpitch, fbase, plane) : 0.f;
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) red[tid >> 5] = (double)part;   // FP32 within a warp, FP64 across warps
        if (tid == 0) pending = dp->partial_off + local;
    }
    __syncthreads();
    if (tid == 0) flush();
}

template <int R, bool ABS, int DTYPE, int TH>
cudaError_t launch_tma(const FieldsLaunch& L, int ntiles, cudaStream_t s) {
    const size_t smem = TmaTile<R, ABS, DTYPE, TH>::SMEM;
    auto k = fields_tma_kernel<R, ABS, DTYPE, TH>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem)) != cudaSuccess) return e;
    if (L.grid_per_sm > 0 && L.grid_per_sm < per_sm) per_sm = L.grid_per_sm;   // tuned persistent grid
    const int chunks = (ntiles - L.tile_base + kFieldsChunk - 1) / kFieldsChunk;
    const int cap = sms * (per_sm > 0 ? per_sm : 1);
    k<<<chunks < cap ? chunks : cap, kThreads, smem, s>>>(L, ntiles);
    return cudaGetLastError();
}

template <bool ABS, int DTYPE>
cudaError_t dispatch(const FieldsLaunch& L, int ntiles, int R, cudaStream_t s) {
    if (L.tile_h == 128) {
        if (R == 6) return launch_tma<6, ABS, DTYPE, 128>(L, ntiles, s);
        if (R == 9) return launch_tma<9, ABS, DTYPE, 128>(L, ntiles, s);
        return launch_tma<12, ABS, DTYPE, 128>(L, ntiles, s);
    }
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
    if (!L.counter) return cudaErrorInvalidValue;   // the tile counter is required (zeroed by the caller)
    const bool abs_ = L.absolute != 0;
    if (dtype == ITC_U8) return abs_ ? dispatch<true, ITC_U8>(L, ntiles, R, s) : dispatch<false, ITC_U8>(L, ntiles, R, s);
    return abs_ ? dispatch<true, ITC_F32>(L, ntiles, R, s) : dispatch<false, ITC_F32>(L, ntiles, R, s);
}

}  // namespace itc
