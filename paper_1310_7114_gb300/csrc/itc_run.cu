// itc_run.cu -- the fixed-point iterations of Algorithm 1 (steps 3-11) on precomputed fields.
//
// A CTA owns its images for all of their iterations: one image with more than 64 codebook
// vectors, else 2, 4 or 8 images of up to 64, 32 or 16 vectors, each on as many threads, in
// lockstep.  W, the gathered field values and the codebook sums stay in shared memory, the
// fields are read from L2/HBM by gathers.  Per iteration:
//   gather   a_k = A(r_k), D_k = F(r_k) (- r_k a_k if absolute) + (r_k - w_k) a_k,
//            r_k = round(w_k) clamped to the lattice                  (Eq. (accupdate) data terms)
//   pairs    s_k = sum_j g_rho(w_j - w_k),  E_k = sum_j g_rho(w_j - w_k)(w_j - w_k)   (Eq. (origupdate))
//            one thread per k loops over every j in order (positions are broadcast from shared
//            memory), so the per-k sums need no reduction; g = 2^(-sum_i d_i^2 c_i) (ex2.approx.ftz) with
//            log2(e) folded into c_i.
//   sums     S_XW = sum_k a_k, S_WW = sum_k s_k (FP32 shuffle trees, then the image's warps in order),
//            c = S_XW / S_WW, D_cs of Eq. (1) in double at the reported W
//   update   w_k' = w_k + step_scale (D_k - kappa c E_k) / a_k, kappa_i = tau_i^2 / rho_i^2 (the
//            factor differentiating Eq. (1) gives the pair term; 1 when tau = rho), rounded to the
//            lattice unless ITC_CONTINUOUS (floor(w) + round(w - floor(w) + delta), exact in FP32
//            up to the one sum of the fraction and delta; a real-valued W lands on the lattice
//            after its first update); a_k = 0 keeps w_k.  Jacobi: every k reads the old W.
#include <math.h>

#include <type_traits>

#include "itc_internal.cuh"

namespace itc {
namespace {

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// 2^x by the PTX instruction ex2.approx.ftz.f32 (relative error about 2^-22; results below the
// smallest normal float flush to zero, which for the pair kernel means a weight under 1e-38)
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float lattice_round(float x, int n) {
    float r = floorf(x + 0.5f);
    return fminf(fmaxf(r, 0.f), (float)(n - 1));
}

struct Sums {
    float sxw, sww;
    int empty;
};

// dev_status: the image's status word from the fields pass (ITC_ERR_TIMEOUT when a bounded wait
// there gave up; its S_XX is then NaN)
__device__ void write_stats(itc_stats* st, const Sums& s, double sxx, int moved, int iters_done,
                            double dcs_const, int dev_status) {
    itc_stats r;
    r.sxw = s.sxw;
    r.sww = s.sww;
    r.sxx = sxx;
    r.c = (double)s.sxw / (double)s.sww;
    r.dcs = s.sxw > 0 ? log((double)s.sww) + log(sxx) - 2.0 * log((double)s.sxw) + dcs_const : INFINITY;
    r.empty = s.empty;
    r.moved = moved;
    r.iters_done = iters_done;
    r.status = dev_status == ITC_ERR_TIMEOUT ? ITC_ERR_TIMEOUT
               : (!(s.sxw > 0) || !isfinite(r.dcs) ? ITC_ERR_NONFINITE
                  : (s.empty > 0 ? ITC_WARN_EMPTY_SUPPORT : ITC_OK));
    *st = r;
}

// The image fields the iteration needs, copied to registers once.
struct Img {
    const float* A;
    long long plane;
    int H, W, G, fpitch, M, iters, flags;
    float step;
};

// Sums over the codebook vectors of each image of the CTA: an image owns `span` consecutive
// threads (16, 32, 64 or 128; the threads past its M contribute zeros).  A shuffle tree over the
// image's lanes (over the whole warp from span 32 up), then, for images over several warps, the
// warp sums in warp order through shared memory (one barrier, taken by the whole CTA).  Zeros
// added to a sum leave it unchanged, so the result is the same for any span that holds the image.
__device__ __forceinline__ void group_sums(float a, float s, int e, int span, bool warp_has, float* red, Sums* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (warp_has) {   // a warp without images only takes the barrier below
        for (int o = span >= 32 ? 16 : span >> 1; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            s += __shfl_xor_sync(0xffffffffu, s, o);
            e += __shfl_xor_sync(0xffffffffu, e, o);
        }
    }
    if (span <= 32) {
        __syncwarp();   // the image's pair reads are done before any of its lanes updates W
        out->sxw = a;
        out->sww = s;
        out->empty = e;
        return;
    }
    if (lane == 0) {
        red[wid * 3] = a;
        red[wid * 3 + 1] = s;
        red[wid * 3 + 2] = __int_as_float(e);
    }
    __syncthreads();
    const int w0 = (threadIdx.x / span) * (span >> 5);
    float x = 0.f, y = 0.f;
    int z = 0;
    for (int w = w0; w < w0 + (span >> 5); ++w) {
        x += red[w * 3];
        y += red[w * 3 + 1];
        z += __float_as_int(red[w * 3 + 2]);
    }
    out->sxw = x;
    out->sww = y;
    out->empty = z;
}

// NPER: codebooks owned per thread (compile-time so the per-codebook state stays in registers).
// ND: lattice dimension (2 or 3).
// A CTA runs a group of images of one span class in lockstep (the same iteration index t); each
// image stops on its own test and its threads then idle to the end of the group.
// Register budget: 7 CTAs per SM in 2-D and 6 in 3-D leave the per-iteration state in registers
// (8 CTAs per SM spilled it and lengthened every iteration: 50 iterations of 4096 ragged binary
// shapes 0.469 -> 0.441 ms, 100 of one 256^3 gray lattice with M 64 0.306 -> 0.233 ms).
template <int NPER, int ND>
__global__ void __launch_bounds__(kRunThreads, ND == 3 ? 6 : 7) run_kernel(const __grid_constant__ RunLaunch L) {
    using P = typename std::conditional<ND == 2, float2, float4>::type;
    const int tid = threadIdx.x, wid = tid >> 5;
    const int* grp = L.groups ? L.groups + (size_t)blockIdx.x * kGroupInts : nullptr;
    const int n = grp ? __ldg(grp) : 1;
    const int span = grp ? __ldg(grp + 1) : kRunThreads;
    const int sub = tid / span, kl = tid - sub * span;   // the thread's image in the group, its lane there
    const int img = grp ? (sub < n ? __ldg(grp + 2 + sub) : -1) : L.img_base + blockIdx.x;
    const ImageDesc& Dg = L.descs ? L.descs[img < 0 ? __ldg(grp + 2) : img] : L.one;
    if (!grp && Dg.ndim != ND) return;   // a mixed range launches once per dimension (CTA-uniform)
    const bool has = img >= 0;
    const bool warp_has = __any_sync(0xffffffffu, has);   // warp-uniform
    Img D;
    D.A = L.fields + Dg.field_off;
    D.plane = Dg.plane_floats;
    D.H = Dg.H; D.W = Dg.W; D.G = Dg.G; D.fpitch = Dg.fpitch; D.M = has ? Dg.M : 0; D.iters = Dg.iters;
    D.flags = Dg.flags; D.step = Dg.step_scale;
    // pair kernel g_rho(d) = exp(-sum_i d_i^2 / (2 rho_i^2)) = 2^(-sum_i d_i^2 c_i),
    // c_i = log2(e) / (2 rho_i^2); rho = sigma unless the codebook width is set apart
    const float c0 = (float)(1.4426950408889634 * (double)Dg.pinv2s2[0]);
    const float c1 = (float)(1.4426950408889634 * (double)Dg.pinv2s2[1]);
    const float c2 = ND == 3 ? (float)(1.4426950408889634 * (double)Dg.pinv2s2[2]) : 0.f;
    const bool iso = ND == 2 && c0 == c1;
    const int M = D.M;
    extern __shared__ __align__(16) unsigned char smraw[];
    // positions, then the same regrouped so that the pair sums read two j at a time with one
    // 16-byte load, (x_j, x_j+1, y_j, y_j+1) per even j, and z by itself; room for
    // NPER * kRunThreads vectors, the image of lane group `sub` at offset sub * span
    constexpr int CAP = NPER * kRunThreads;
    const int base = sub * span;
    P* sw = reinterpret_cast<P*>(smraw) + base;
    float* sxy = reinterpret_cast<float*>(smraw + (size_t)CAP * sizeof(P)) + 2 * base;
    float* sz = sxy + 2 * CAP - 2 * base + base;
    __shared__ float red[3 * (kRunThreads / 32)];
    __shared__ int mvred[kRunThreads / 32];
    __shared__ double s_sxx[kGroupMax];
    __shared__ double s_part[kRunThreads / 32];   // S_XX partial sums of the warps
    __shared__ float s_kap[kGroupMax][3];   // tau_i^2 / rho_i^2 of each image of the group

    if (L.sxx_single) {
        if (tid == 0) s_sxx[0] = *L.sxx_single;
    } else {
        // S_XX of each image from its tile partials, one warp per image; gray images (a partial
        // per slice tile) split the warps evenly over the group's images, eight loads in flight
        // per lane; a fixed order throughout
        constexpr int NW = kRunThreads / 32;
        const int wpi = (ND == 3 && n < NW) ? NW / n : 1;   // warps per image
        const int lane = tid & 31;
        for (int g = wid / wpi; g < n; g += NW / wpi) {
            const ImageDesc& ds = grp ? L.descs[__ldg(grp + 2 + g)] : Dg;
            const long long nt = ds.sxx_tiles, po = ds.sxx_off, step = 32LL * wpi;
            double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            long long i = (long long)(wid % wpi) * 32 + lane;
            for (; i + 7 * step < nt; i += 8 * step)
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] += L.partials[po + i + q * step];
            for (; i < nt; i += step) v[0] += L.partials[po + i];
            double t = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
            t = warp_sum_d(t);
            if (lane == 0) {
                if (wpi == 1) s_sxx[g] = t;
                else s_part[wid] = t;
            }
        }
        if (wpi > 1) {
            __syncthreads();
            if (tid < n) {
                double t = 0;
                for (int q = 0; q < wpi; ++q) t += s_part[tid * wpi + q];
                s_sxx[tid] = t;
            }
        }
    }
    if (has && kl == 0)
        for (int i = 0; i < 3; ++i) s_kap[sub][i] = Dg.kappa[i];
    const float* Win = L.W_in + Dg.w_off;
    for (int k = kl; k < M; k += span) {
        P w;
        w.x = Win[k * ND];
        w.y = Win[k * ND + 1];
        if constexpr (ND == 3) { w.z = Win[k * ND + 2]; w.w = 0.f; }
        sw[k] = w;
        sxy[(k >> 1) * 4 + (k & 1)] = w.x;
        sxy[(k >> 1) * 4 + 2 + (k & 1)] = w.y;
        if constexpr (ND == 3) sz[k] = w.z;
    }
    __syncthreads();
    const bool snap = !(D.flags & ITC_CONTINUOUS);
    const bool stop_fixed = (D.flags & ITC_STOP_ON_FIXED) != 0;

    Sums s = {0.f, 0.f, 0};
    int moved = 0, done = 0;
    bool stop = false, live = has;   // live: the image still iterates
    for (int t = 0;; ++t) {
        if (!L.final_eval && t == D.iters) live = false;
        float a[NPER], Dm[NPER][ND], Ek[NPER][ND];
        float pa = 0.f, ps = 0.f;
        int pe = 0;
#pragma unroll
        for (int q = 0; q < NPER; ++q) {
            const int k = kl + q * span;
            a[q] = 0.f;
            if (!live || k >= M) continue;
            const P wk = sw[k];
            // gather first (its latency overlaps the pair sums)
            float r[3], wv[3];
            wv[0] = wk.x; wv[1] = wk.y;
            r[0] = lattice_round(wk.x, D.H);
            r[1] = lattice_round(wk.y, D.W);
            if constexpr (ND == 3) { wv[2] = wk.z; r[2] = lattice_round(wk.z, D.G); }
            const long long o = ((long long)(ND == 3 ? (int)r[2] : 0) * D.H + (int)r[0]) * D.fpitch + (int)r[1];
            const float ak = __ldg(D.A + o);
            float f[ND];
#pragma unroll
            for (int i = 0; i < ND; ++i) f[i] = __ldg(D.A + (i + 1) * D.plane + o);
            // pair sums over every j in order, two j per packed FP32 operation (the .x lanes take the
            // even j, the .y lanes the odd j; summed at the end)
            const float2 nk0 = f2(-wk.x, -wk.x), nk1 = f2(-wk.y, -wk.y);
            const float2 cc0 = f2(c0, c0), cc1 = f2(c1, c1), cc2 = f2(c2, c2);
            float2 nk2 = f2(0.f, 0.f);
            if constexpr (ND == 3) nk2 = f2(-wk.z, -wk.z);
            float2 sp = f2(0.f, 0.f), ep0 = f2(0.f, 0.f), ep1 = f2(0.f, 0.f), ep2 = f2(0.f, 0.f);
            int j = 0;
            if (iso) {
                // equal widths (2-D): c (d0^2 + d1^2), one product fewer per pair; on the lattice
                // d0^2 + d1^2 is an exact integer, rounded once by the product with c
#pragma unroll 16
                for (; j + 1 < M; j += 2) {
                    const float4 q4 = *reinterpret_cast<const float4*>(sxy + 2 * j);
                    const float2 d0 = __fadd2_rn(f2(q4.x, q4.y), nk0);
                    const float2 d1 = __fadd2_rn(f2(q4.z, q4.w), nk1);
                    float2 x = __fmul2_rn(__ffma2_rn(d1, d1, __fmul2_rn(d0, d0)), cc0);
                    float2 d2 = f2(0.f, 0.f);
                    if constexpr (ND == 3) {
                        d2 = __fadd2_rn(*reinterpret_cast<const float2*>(sz + j), nk2);
                        x = __ffma2_rn(__fmul2_rn(d2, d2), cc2, x);
                    }
                    const float2 g = f2(ex2_ftz(-x.x), ex2_ftz(-x.y));
                    sp = __fadd2_rn(sp, g);
                    ep0 = __ffma2_rn(g, d0, ep0);
                    ep1 = __ffma2_rn(g, d1, ep1);
                    if constexpr (ND == 3) ep2 = __ffma2_rn(g, d2, ep2);
                }
            } else {
#pragma unroll 16
                for (; j + 1 < M; j += 2) {
                    const float4 q4 = *reinterpret_cast<const float4*>(sxy + 2 * j);
                    const float2 d0 = __fadd2_rn(f2(q4.x, q4.y), nk0);
                    const float2 d1 = __fadd2_rn(f2(q4.z, q4.w), nk1);
                    float2 x = __fmul2_rn(__fmul2_rn(d0, d0), cc0);
                    x = __ffma2_rn(__fmul2_rn(d1, d1), cc1, x);
                    float2 d2 = f2(0.f, 0.f);
                    if constexpr (ND == 3) {
                        d2 = __fadd2_rn(*reinterpret_cast<const float2*>(sz + j), nk2);
                        x = __ffma2_rn(__fmul2_rn(d2, d2), cc2, x);
                    }
                    const float2 g = f2(ex2_ftz(-x.x), ex2_ftz(-x.y));
                    sp = __fadd2_rn(sp, g);
                    ep0 = __ffma2_rn(g, d0, ep0);
                    ep1 = __ffma2_rn(g, d1, ep1);
                    if constexpr (ND == 3) ep2 = __ffma2_rn(g, d2, ep2);
                }
            }
            if (j < M) {   // odd M: the last j in the .x lanes
                const float d0 = sxy[2 * j] - wk.x, d1 = sxy[2 * j + 2] - wk.y;
                float x = (d0 * d0) * c0;
                x = fmaf(d1 * d1, c1, x);
                float d2 = 0.f;
                if constexpr (ND == 3) { d2 = sz[j] - wk.z; x = fmaf(d2 * d2, c2, x); }
                const float g = ex2_ftz(-x);
                sp.x += g;
                ep0.x = fmaf(g, d0, ep0.x);
                ep1.x = fmaf(g, d1, ep1.x);
                if constexpr (ND == 3) ep2.x = fmaf(g, d2, ep2.x);
            }
            const float s0 = sp.x, s1 = sp.y;
            float e0[ND], e1[ND];
            e0[0] = ep0.x; e1[0] = ep0.y;
            e0[1] = ep1.x; e1[1] = ep1.y;
            if constexpr (ND == 3) { e0[2] = ep2.x; e1[2] = ep2.y; }
            a[q] = ak;
#pragma unroll
            for (int i = 0; i < ND; ++i) {
                // centred moment about the real w_k: F(r) (- r a if absolute) + (r - w) a
                const float fi = L.absolute ? f[i] - r[i] * ak : f[i];
                Dm[q][i] = fmaf(r[i] - wv[i], ak, fi);
                Ek[q][i] = e0[i] + e1[i];
            }
            pa += ak;
            ps += s0 + s1;
            pe += !(ak > 0.f);
        }
        Sums r;
        group_sums(pa, ps, pe, span, warp_has, red, &r);
        if (live) s = r;
        if (live && !L.final_eval && t == 0 && L.stats && kl == 0)
            write_stats(L.stats + img, s, s_sxx[sub], 0, 0, Dg.dcs_const, L.img_status ? L.img_status[img] : ITC_OK);
        const bool upd = live && t != D.iters && !stop;
        if (!upd) live = false;
        // update (Jacobi: every k above read the old W; the barrier in group_sums, or the image's
        // warp for spans up to 32, separates them)
        // only threads that update divide (an idle thread's 0 / 0 would take the slow division
        // path and hold its image's warps at the next barrier)
        const float c = upd ? s.sxw / s.sww : 0.f;
        float kap[ND];   // from shared memory where it is used (it need not hold registers)
#pragma unroll
        for (int i = 0; i < ND; ++i) kap[i] = upd ? s_kap[sub][i] : 0.f;
        int mv = 0;
#pragma unroll
        for (int q = 0; q < NPER; ++q) {
            const int k = kl + q * span;
            if (!upd || k >= M || !(a[q] > 0.f)) continue;
            P w = sw[k];
            float nw[3];
            nw[0] = w.x; nw[1] = w.y;
            if constexpr (ND == 3) nw[2] = w.z;
            bool kmoved = false;
#pragma unroll
            for (int i = 0; i < ND; ++i) {
                const int ni = i == 0 ? D.H : (i == 1 ? D.W : D.G);
                // tau^2 / rho^2 on the pair term: 1 (exact) when tau = rho
                const float delta = D.step * (Dm[q][i] - (c * kap[i]) * Ek[q][i]) / a[q];
                float nv;
                if (snap) {
                    // round(w + delta) = fl + round(fr + delta) with w = fl + fr, fl = floor(w):
                    // fl and fr are exact in FP32, and on the lattice (fr = 0, the state after
                    // the first update) this is w + round(delta) with the one rounding of delta
                    // + 0.5.  A real-valued initial W (from a continuous run, or optimised by
                    // gradients) is rounded onto the lattice by its first update.
                    const float fl = floorf(nw[i]);
                    nv = fminf(fmaxf(fl + floorf((nw[i] - fl) + delta + 0.5f), 0.f), (float)(ni - 1));
                } else {
                    nv = fminf(fmaxf(nw[i] + delta, 0.f), (float)(ni - 1));
                }
                kmoved |= (nv != nw[i]);
                nw[i] = nv;
            }
            w.x = nw[0]; w.y = nw[1];
            if constexpr (ND == 3) w.z = nw[2];
            sw[k] = w;
            sxy[(k >> 1) * 4 + (k & 1)] = w.x;
            sxy[(k >> 1) * 4 + 2 + (k & 1)] = w.y;
            if constexpr (ND == 3) sz[k] = w.z;
            mv += kmoved;
        }
        // vectors moved per image (same trees as the sums) where it is used: by the stopping test,
        // and for the stats after an image's last update; whether any image goes on.  The
        // barrier also orders this update before the next pair sums.  (The count is decided per
        // warp, the same for every warp of an image.)
        const bool count = __any_sync(0xffffffffu, upd && (stop_fixed || t + 1 == D.iters));
        if (count) {
            for (int o = span >= 32 ? 16 : span >> 1; o > 0; o >>= 1) mv += __shfl_xor_sync(0xffffffffu, mv, o);
            if (span > 32 && (tid & 31) == 0) mvred[wid] = mv;
        }
        const bool any = __syncthreads_or(live);
        if (count && span > 32) {
            const int w0 = sub * (span >> 5);
            mv = 0;
            for (int w = w0; w < w0 + (span >> 5); ++w) mv += mvred[w];
        }
        if (upd) {
            if (count) moved = mv;
            ++done;
            if (stop_fixed && moved == 0) stop = true;
        }
        if (!any) break;
    }
    if (has && L.final_eval && L.stats && kl == 0)
        write_stats(L.stats + img, s, s_sxx[sub], moved, done, Dg.dcs_const, L.img_status ? L.img_status[img] : ITC_OK);
    if (has && !L.final_eval && L.stats && kl == 0) {
        L.stats[img].moved = moved;
        L.stats[img].iters_done = done;
    }
    float* Wout = L.W_out + Dg.w_off;
    const long long w_off = Dg.w_off;
    for (int k = kl; k < M; k += span) {
        const P w = sw[k];
        float ww[3];
        ww[0] = w.x; ww[1] = w.y;
        if constexpr (ND == 3) ww[2] = w.z;
#pragma unroll
        for (int i = 0; i < ND; ++i) {
            const int ni = i == 0 ? D.H : (i == 1 ? D.W : D.G);
            Wout[k * ND + i] = ww[i];
            if (L.W_lattice) L.W_lattice[w_off + k * ND + i] = (int)lattice_round(ww[i], ni);
        }
    }
}

template <int ND>
cudaError_t launch_nd(const RunLaunch& L, int nimg, int max_M, cudaStream_t s) {
    const int nper = (max_M + kRunThreads - 1) / kRunThreads;
    // positions (AoS) and the same regrouped by pairs of j, room for NPER * kRunThreads vectors
    const int np2 = nper <= 1 ? 1 : nper <= 2 ? 2 : nper <= 4 ? 4 : nper <= 8 ? 8 : nper <= 16 ? 16 : 32;
    const size_t cap = (size_t)np2 * kRunThreads;
    const size_t smem = cap * (ND == 2 ? sizeof(float2) : sizeof(float4)) + (size_t)ND * cap * sizeof(float);
    static_assert(ITC_MAX_M <= 32 * kRunThreads, "codebooks per thread cover ITC_MAX_M");
    auto k = nper <= 1 ? run_kernel<1, ND> : nper <= 2 ? run_kernel<2, ND> : nper <= 4 ? run_kernel<4, ND>
           : nper <= 8 ? run_kernel<8, ND> : nper <= 16 ? run_kernel<16, ND> : run_kernel<32, ND>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<nimg, kRunThreads, smem, s>>>(L);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_run(const RunLaunch& L, int nimg, int max_M, const int* max_dim, cudaStream_t s, int ndim) {
    (void)max_dim;
    if (nimg <= 0) return cudaSuccess;
    return ndim == 3 ? launch_nd<3>(L, nimg, max_M, s) : launch_nd<2>(L, nimg, max_M, s);
}

}  // namespace itc
