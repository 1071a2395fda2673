// itc_backward.cu -- gradient of the Cauchy-Schwarz divergence, Eq. (1), with respect to the
// codebook and to the per-pixel weights of weighted ITC (Sec. 5).
//
//   dD/dw_{k,i} = (2 / rho_i^2) E_{k,i} / S_WW - (2 / tau_i^2) D_{k,i} / S_XW
//   dD/dh(x)    = 2 A_s(x) / S_XX - (2 / S_XW) sum_k g_tau(x - w_k) [x in box(round(w_k))]
// (tau = sigma: the data kernel and its fields; rho: the codebook pair kernel; A_s: the field of h
// at the width s of V(X); rho = s = tau unless set apart, and then A_s = A.)
//
// Kernel 1 (one CTA per image): window sums a_k, D_k around round(w_k) read directly from the
// image (kernel evaluated at the real w_k, one warp per k), the M x M sums s_k, E_k (one warp
// per k, xor-shuffle reduction), S_XW, S_WW, grad_W and two per-image scalars for kernel 2.
// Kernel 2 (one CTA per image, over its 64 x 64 pixel tiles): the codebooks whose box meets a
// tile are listed in k order (ballot compaction), their Gaussians are stamped onto the tile in
// that order -- the transposed form of the gather in the forward update -- and every pixel
// combines the stored field A with the stamp.
#include <math.h>

#include "itc_internal.cuh"

namespace itc {
namespace {

__device__ __forceinline__ float warp_sum_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// 2^x by the PTX instruction ex2.approx.ftz.f32 (relative error about 2^-22; results below the
// smallest normal float flush to zero)
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ int lattice_round_i(float x, int n) {
    float r = floorf(x + 0.5f);
    return (int)fminf(fmaxf(r, 0.f), (float)(n - 1));
}
__device__ __forceinline__ float pixel_weight(const ImageDesc& D, int u, int v) {
    const size_t o = (size_t)u * D.pitch + v;
    if (D.ndim == 3) return D.weight ? __ldg(D.weight + o) : 1.f;
    if (D.dtype == ITC_U8) return (float)__ldg(reinterpret_cast<const unsigned char*>(D.data) + o);
    return __ldg(reinterpret_cast<const float*>(D.data) + o);
}
__device__ __forceinline__ int pixel_gray(const ImageDesc& D, int u, int v) {
    return (int)__ldg(reinterpret_cast<const unsigned char*>(D.data) + (size_t)u * D.pitch + v);
}

__global__ void __launch_bounds__(kRunThreads) bwd_codebook_kernel(const __grid_constant__ BackwardLaunch L) {
    const int img = L.img_base + blockIdx.x;
    const ImageDesc& D = L.descs[img];
    const int M = D.M, nd = D.ndim, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nw = blockDim.x >> 5;
    extern __shared__ __align__(16) float sm[];
    float* sw = sm;
    float* sa = sw + 3 * M;
    float* sD = sa + M;
    float* ss = sD + 3 * M;
    float* sE = ss + M;
    __shared__ double red[4];

    // S_XX from the image's tile partials: warp 0 alone, or for a gray image (a partial per
    // slice tile) every warp a strided share with eight loads in flight per lane, the warp sums
    // added in warp order
    __shared__ double s_px[32];
    const int nws = nd == 3 ? nw : 1;
    if (wid < nws) {
        const long long nt = D.sxx_tiles, step = 32LL * nws;
        double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        long long i = tid;
        for (; i + 7 * step < nt; i += 8 * step)
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] += L.partials[D.sxx_off + i + q * step];
        for (; i < nt; i += step) v[0] += L.partials[D.sxx_off + i];
        const double t = warp_sum_d(((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])));
        if (lane == 0) s_px[wid] = t;
    }
    const float* Wk = L.W + D.w_off;
    for (int k = tid; k < M; k += blockDim.x)
        for (int i = 0; i < 3; ++i) sw[k * 3 + i] = i < nd ? Wk[k * nd + i] : 0.f;
    __syncthreads();
    double sxx = 0;
    for (int q = 0; q < nws; ++q) sxx += s_px[q];
    const float c0 = D.inv2s2[0], c1 = D.inv2s2[1], c2 = D.inv2s2[2];
    const int Ru = D.R[0], Rv = D.R[1], Rg = D.R[2];

    // a_k and D_k: on the lattice (every w_k integral and inside it) they are the stored field
    // values at w_k; otherwise window sums around round(w_k) with the kernel at the real w_k
    int off_lattice = 0;
    for (int k = tid; k < M; k += blockDim.x)
        for (int i = 0; i < nd; ++i) {
            const float w = sw[k * 3 + i];
            const int ni = i == 0 ? D.H : (i == 1 ? D.W : D.G);
            off_lattice |= (w != rintf(w)) || !(w >= 0.f) || !(w <= (float)(ni - 1));
        }
    const bool gather = !__syncthreads_or(off_lattice);
    if (gather) {
        const float* A = L.fields + D.field_off;
        for (int k = tid; k < M; k += blockDim.x) {
            const int r0 = (int)sw[k * 3], r1 = (int)sw[k * 3 + 1], r2 = nd == 3 ? (int)sw[k * 3 + 2] : 0;
            const long long o = ((long long)r2 * D.H + r0) * D.fpitch + r1;
            sa[k] = __ldg(A + o);
            for (int i = 0; i < 3; ++i) sD[k * 3 + i] = i < nd ? __ldg(A + (i + 1) * D.plane_floats + o) : 0.f;
        }
    } else {
        for (int k = wid; k < M; k += nw) {
            const float w0 = sw[k * 3], w1 = sw[k * 3 + 1], w2 = sw[k * 3 + 2];
            const int r0 = lattice_round_i(w0, D.H), r1 = lattice_round_i(w1, D.W);
            const int r2 = nd == 3 ? lattice_round_i(w2, D.G) : 0;
            const int ua = max(0, r0 - Ru), ub = min(D.H - 1, r0 + Ru);
            const int va = max(0, r1 - Rv), vb = min(D.W - 1, r1 + Rv);
            const int nv = vb - va + 1, npos = (ub - ua + 1) * nv;
            float a = 0.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
            for (int p = lane; p < npos; p += 32) {
                const int u = ua + p / nv, v = va + p % nv;
                const float h = pixel_weight(D, u, v);
                if (h == 0.f) continue;
                const float du = (float)u - w0, dv = (float)v - w1;
                float dg = 0.f;
                if (nd == 3) {
                    const int gl = pixel_gray(D, u, v);
                    if (abs(gl - r2) > Rg) continue;
                    dg = (float)gl - w2;
                }
                const float g = h * expf(-(du * du * c0 + dv * dv * c1 + dg * dg * c2));
                a += g;
                d0 = fmaf(g, du, d0);
                d1 = fmaf(g, dv, d1);
                d2 = fmaf(g, dg, d2);
            }
            a = warp_sum_f(a);
            d0 = warp_sum_f(d0);
            d1 = warp_sum_f(d1);
            d2 = warp_sum_f(d2);
            if (lane == 0) {
                sa[k] = a;
                sD[k * 3] = d0;
                sD[k * 3 + 1] = d1;
                sD[k * 3 + 2] = d2;
            }
        }
    }
    // codebook interaction sums: one thread per k, every j in order
    {
        const float q0 = (float)(1.4426950408889634 * (double)D.pinv2s2[0]);
        const float q1 = (float)(1.4426950408889634 * (double)D.pinv2s2[1]);
        const float q2 = (float)(1.4426950408889634 * (double)D.pinv2s2[2]);
        for (int k = tid; k < M; k += blockDim.x) {
            const float wk0 = sw[k * 3], wk1 = sw[k * 3 + 1], wk2 = sw[k * 3 + 2];
            float s_ = 0.f, e0 = 0.f, e1 = 0.f, e2 = 0.f;
            for (int j = 0; j < M; ++j) {
                const float d0 = sw[j * 3] - wk0, d1 = sw[j * 3 + 1] - wk1, d2 = sw[j * 3 + 2] - wk2;
                const float g = exp2f(-(d0 * d0 * q0 + d1 * d1 * q1 + d2 * d2 * q2));
                s_ += g;
                e0 = fmaf(g, d0, e0);
                e1 = fmaf(g, d1, e1);
                e2 = fmaf(g, d2, e2);
            }
            ss[k] = s_;
            sE[k * 3] = e0;
            sE[k * 3 + 1] = e1;
            sE[k * 3 + 2] = e2;
        }
    }
    __syncthreads();
    if (wid == 0) {
        double x = 0, y = 0;
        int e = 0;
        for (int k = lane; k < M; k += 32) {
            x += (double)sa[k];
            y += (double)ss[k];
            e += !(sa[k] > 0.f);
        }
        x = warp_sum_d(x);
        y = warp_sum_d(y);
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (lane == 0) {
            red[0] = x;
            red[1] = y;
            red[2] = (double)e;
        }
    }
    __syncthreads();
    const double sxw = red[0], sww = red[1];
    const double gD = L.grad_dcs ? (double)L.grad_dcs[img] : 1.0;
    if (L.grad_W) {
        float* gW = L.grad_W + D.w_off;
        for (int k = tid; k < M; k += blockDim.x)
            for (int i = 0; i < nd; ++i) {
                const double t2 = (double)D.sigma[i] * (double)D.sigma[i];
                const double r2 = (double)D.rho[i] * (double)D.rho[i];
                gW[k * nd + i] = (float)(gD * 2.0 * ((double)sE[k * 3 + i] / (r2 * sww) -
                                                     (double)sD[k * 3 + i] / (t2 * sxw)));
            }
    }
    if (tid == 0) {
        L.scal[img * 4 + 0] = 2.0 * gD / sxx;
        L.scal[img * 4 + 1] = 2.0 * gD / sxw;
        if (L.stats) {
            itc_stats r;
            r.sxw = sxw;
            r.sww = sww;
            r.sxx = sxx;
            r.c = sxw / sww;
            r.dcs = sxw > 0 ? log(sww) + log(sxx) - 2.0 * log(sxw) + D.dcs_const : INFINITY;
            r.empty = (int)red[2];
            r.moved = 0;
            r.iters_done = 0;
            const int dev_status = L.img_status ? L.img_status[img] : ITC_OK;
            r.status = dev_status == ITC_ERR_TIMEOUT ? ITC_ERR_TIMEOUT
                       : (!(sxw > 0) || !isfinite(r.dcs) ? ITC_ERR_NONFINITE
                          : (r.empty > 0 ? ITC_WARN_EMPTY_SUPPORT : ITC_OK));
            L.stats[img] = r;
        }
    }
}

constexpr int kChunk = 64;   // codebooks staged per round in the pixel kernel

// Pixel pass: one CTA per image walks the image's 64 x 64 tiles (images with the most tiles
// are launched first).  The stamp S(x) = sum_k g(x - w_k) [x in box(round(w_k))] is separable
// in 2-D: g(x - w) = g_u(x_u - w_u) g_v(x_v - w_v) and the box is a product of two intervals,
// so for the codebooks whose box meets a tile (listed in k order)
//   S(r, c) = sum_l a_l(r) b_l(c),  a_l(r) = g_u(u0 + r - w_lu) [|u0 + r - r_lu| <= R_u], ...
// Chunks of 64 listed codebooks are staged as a (64 x 64) and b (64 x 64) in shared memory and
// every thread accumulates a 4 x 4 block of pixels in l order (deterministic, no atomics), with
// packed FMAs over pairs of columns.  In 3-D the g factor depends on each pixel's gray level and
// is applied per pixel and codebook.
__global__ void __launch_bounds__(kThreads, 3) bwd_pixels_kernel(const __grid_constant__ BackwardLaunch L) {
    // split CTAs per image (few large images): CTA s of an image takes its tiles s, s + split, ...
    const int split = L.split;
    const int img = L.bwd_order ? __ldg(L.bwd_order + blockIdx.x / split) : L.img_base + (int)(blockIdx.x / split);
    const int part = blockIdx.x % split;
    const ImageDesc& D = L.descs[img];
    const int M = D.M, nd = D.ndim, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int H = D.H, Wd = D.W, G = D.G, fpitch = D.fpitch, tiles_v = D.bwd_tiles_v;
    const int ntiles = D.bwd_tiles_u * D.bwd_tiles_v;
    const int Ru = D.R[0], Rv = D.R[1], Rg = D.R[2];
    const float c0 = D.inv2s2[0], c1 = D.inv2s2[1], c2 = D.inv2s2[2];
    // the separable factors exp(-d^2 c) = 2^(-d^2 c log2 e), log2 e folded into the widths
    const float l0 = (float)(1.4426950408889634 * (double)c0), l1 = (float)(1.4426950408889634 * (double)c1);
    // the S_XX term uses the field of h at the width of V(X): A itself unless set apart
    const float* A = L.fields + (D.self_off >= 0 ? D.self_off : D.field_off);
    float* gh = L.grad_h + D.gh_off;
    const float s1 = (float)L.scal[img * 4 + 0], s2 = (float)L.scal[img * 4 + 1];
    // every row of this image's dD/dh starts on a 16-byte boundary (width and offset multiples of
    // 4 floats, aligned base): the results go out as 16-byte row pieces, else through shared
    // memory as whole row segments
    const bool rows16 = ((Wd & 3) == 0) && ((reinterpret_cast<size_t>(gh) & 15) == 0);

    extern __shared__ __align__(16) unsigned char bsm[];
    // per listed codebook of the current tile one 16-byte record (position and site along u
    // and v), then the codebooks' positions, sites and the list itself
    float4* lc = reinterpret_cast<float4*>(bsm);
    float* cw = reinterpret_cast<float*>(lc + M);       // M x 3 codebook positions
    int* cr = reinterpret_cast<int*>(cw + 3 * M);       // M x 3 rounded lattice sites
    int* lk = cr + 3 * M;                               // listed codebooks of the current tile
    __shared__ __align__(16) float sa[kChunk][kBwdTileH];
    __shared__ __align__(16) float sb[kChunk][kBwdTileW];
    __shared__ __align__(16) int wcount[kThreads / 32];

    const float* Wk = L.W + D.w_off;
    for (int k = tid; k < M; k += blockDim.x) {
        const float w0 = Wk[k * nd], w1 = Wk[k * nd + 1], w2 = nd == 3 ? Wk[k * nd + 2] : 0.f;
        cw[k * 3] = w0;
        cw[k * 3 + 1] = w1;
        cw[k * 3 + 2] = w2;
        cr[k * 3] = lattice_round_i(w0, H);
        cr[k * 3 + 1] = lattice_round_i(w1, Wd);
        cr[k * 3 + 2] = nd == 3 ? lattice_round_i(w2, G) : 0;
    }
    __syncthreads();

    const int pr = (tid >> 4) * 4, pc = (tid & 15) * 4;   // this thread's 4 x 4 block
    if (part >= ntiles) return;
    for (int t = part; t < ntiles; t += split) {
        const int u0 = (t / tiles_v) * kBwdTileH, v0 = (t % tiles_v) * kBwdTileW;
        // field values of this thread's block, loaded first so their latency overlaps the stamp
        float4 a4[4];
        int gray[4][4];
        const bool cols_in = v0 + pc < Wd;
        if (nd == 2) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int u = min(u0 + pr + i, H - 1);
                a4[i] = cols_in ? __ldg(reinterpret_cast<const float4*>(A + (long long)u * fpitch + v0 + pc))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int u = u0 + pr + i, v = v0 + pc + j;
                    gray[i][j] = (u < H && v < Wd) ? pixel_gray(D, u, v) : 0;
                }
        }

        // stable compaction of the codebooks whose box meets this tile
        int nl = 0;
        for (int base = 0; base < M; base += blockDim.x) {
            const int k = base + tid;
            bool hit = false;
            if (k < M) {
                const int r0 = cr[k * 3], r1 = cr[k * 3 + 1];
                hit = (r0 + Ru >= u0) && (r0 - Ru <= u0 + kBwdTileH - 1) &&
                      (r1 + Rv >= v0) && (r1 - Rv <= v0 + kBwdTileW - 1);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            if (lane == 0) wcount[wid] = __popc(bal);
            __syncthreads();
            static_assert(kThreads / 32 == 8, "eight warp counts");
            const int4 wc0 = *reinterpret_cast<const int4*>(wcount), wc1 = *reinterpret_cast<const int4*>(wcount + 4);
            const int cnt[8] = {wc0.x, wc0.y, wc0.z, wc0.w, wc1.x, wc1.y, wc1.z, wc1.w};
            int off = nl, tot = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                off += q < wid ? cnt[q] : 0;
                tot += cnt[q];
            }
            if (hit) {
                const int pos = off + __popc(bal & ((1u << lane) - 1u));
                lk[pos] = k;
                lc[pos] = make_float4(cw[k * 3], cw[k * 3 + 1], __int_as_float(cr[k * 3]), __int_as_float(cr[k * 3 + 1]));
            }
            nl += tot;
            __syncthreads();
        }

        // accumulators as column pairs (j = 0, 1 and 2, 3) of each row, the packed FMA operands
        float2 acc2[4][2];
#pragma unroll
        for (int i = 0; i < 4; ++i) { acc2[i][0] = make_float2(0.f, 0.f); acc2[i][1] = make_float2(0.f, 0.f); }
        // factor staging: each thread fills one row / column r of the factors for every fourth l
        const int sr = tid & (kBwdTileH - 1), sl = tid / kBwdTileH;
        static_assert(kBwdTileH == kBwdTileW && kThreads % kBwdTileH == 0, "square tiles, whole rows of threads");
        constexpr int kStageStep = kThreads / kBwdTileH;
        const int su = u0 + sr, sv = v0 + sr;
        const bool su_in = su < H, sv_in = sv < Wd;
        const float fu = (float)su, fv = (float)sv;
        for (int base = 0; base < nl; base += kChunk) {
            const int nc = min(kChunk, nl - base);
            for (int l = sl; l < nc; l += kStageStep) {
                const float4 rec = lc[base + l];
                float av = 0.f, bv = 0.f;
                if (su_in && abs(su - __float_as_int(rec.z)) <= Ru) { const float d = fu - rec.x; av = ex2_ftz(-(d * d) * l0); }
                if (sv_in && abs(sv - __float_as_int(rec.w)) <= Rv) { const float d = fv - rec.y; bv = ex2_ftz(-(d * d) * l1); }
                sa[l][sr] = av;
                sb[l][sr] = bv;
            }
            __syncthreads();
            if (nd == 2) {
#pragma unroll 1   // unrolled, the loop spills at the 80-register budget of 3 CTAs per SM
                for (int l = 0; l < nc; ++l) {
                    const float4 av4 = *reinterpret_cast<const float4*>(&sa[l][pr]);
                    const float4 bv4 = *reinterpret_cast<const float4*>(&sb[l][pc]);
                    const float av[4] = {av4.x, av4.y, av4.z, av4.w};
                    const float2 b01 = make_float2(bv4.x, bv4.y), b23 = make_float2(bv4.z, bv4.w);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 ai = make_float2(av[i], av[i]);
                        acc2[i][0] = __ffma2_rn(ai, b01, acc2[i][0]);
                        acc2[i][1] = __ffma2_rn(ai, b23, acc2[i][1]);
                    }
                }
            } else {
                for (int l = 0; l < nc; ++l) {
                    const float4 av4 = *reinterpret_cast<const float4*>(&sa[l][pr]);
                    const float4 bv4 = *reinterpret_cast<const float4*>(&sb[l][pc]);
                    const float av[4] = {av4.x, av4.y, av4.z, av4.w}, bv[4] = {bv4.x, bv4.y, bv4.z, bv4.w};
                    const int k = lk[base + l];
                    const float wg = cw[k * 3 + 2];
                    const int rg = cr[k * 3 + 2];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int gl = gray[i][j];
                            if (abs(gl - rg) <= Rg) {
                                const float d = (float)gl - wg;
                                float& aij = (j & 1) ? acc2[i][j >> 1].y : acc2[i][j >> 1].x;
                                aij = fmaf(av[i] * bv[j], expf(-d * d * c2), aij);
                            }
                        }
                }
            }
            __syncthreads();   // sa / sb are rewritten by the next chunk or tile
        }
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            acc[i][0] = acc2[i][0].x; acc[i][1] = acc2[i][0].y; acc[i][2] = acc2[i][1].x; acc[i][3] = acc2[i][1].y;
        }

        if (nd == 2 && rows16) {
            // rows of dD/dh start on 16-byte boundaries: one 16-byte store per row of the block
            // (a warp writes two full 256-byte row segments per instruction)
            if (cols_in) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int u = u0 + pr + i;
                    if (u >= H) break;
                    float* out = gh + (long long)u * Wd + v0 + pc;
                    const float r4[4] = {s1 * a4[i].x - s2 * acc[i][0], s1 * a4[i].y - s2 * acc[i][1],
                                         s1 * a4[i].z - s2 * acc[i][2], s1 * a4[i].w - s2 * acc[i][3]};
                    if (v0 + pc + 3 < Wd) {
                        *reinterpret_cast<float4*>(out) = make_float4(r4[0], r4[1], r4[2], r4[3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (v0 + pc + j < Wd) out[j] = r4[j];
                    }
                }
            }
            continue;
        }
        if (nd == 2) {
            // the thread's 4 x 4 results go through shared memory (sa is free after the last
            // chunk's barrier), so that each warp writes 32 consecutive pixels of a row
#pragma unroll
            for (int i = 0; i < 4; ++i)
                *reinterpret_cast<float4*>(&sa[pr + i][pc]) =
                    make_float4(s1 * a4[i].x - s2 * acc[i][0], s1 * a4[i].y - s2 * acc[i][1],
                                s1 * a4[i].z - s2 * acc[i][2], s1 * a4[i].w - s2 * acc[i][3]);
            __syncthreads();
            const int r0 = tid >> 6, c = tid & 63;   // rows r0, r0 + 4, ..., column c
            if (v0 + c < Wd) {
                const int nrow = min(16, max(0, (H - u0 - r0 + 3) >> 2));
                float* gp = gh + (long long)(u0 + r0) * Wd + v0 + c;
#pragma unroll
                for (int m = 0; m < 16; ++m)
                    if (m < nrow) gp[4 * m * Wd] = sa[r0 + 4 * m][c];
            }
            continue;   // the next tile's list building passes two barriers before sa is rewritten
        }
        if (!cols_in) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int u = u0 + pr + i;
            if (u >= H) break;
            float* out = gh + (long long)u * Wd + v0 + pc;
            {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int v = v0 + pc + j;
                    if (v >= Wd) break;
                    if (gray[i][j] >= G) {   // a voxel outside the lattice: no field value
                        out[j] = 0.f;
                        continue;
                    }
                    const long long o = ((long long)gray[i][j] * H + u) * fpitch + v;
                    out[j] = s1 * __ldg(A + o) - s2 * acc[i][j];
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_backward(const BackwardLaunch& L, int B, int max_M, long long pixel_tiles, int max_image_tiles,
                            cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    const size_t smem1 = (size_t)max_M * kCodebookSmemFloats * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(bwd_codebook_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
    if (e != cudaSuccess) return e;
    bwd_codebook_kernel<<<B, kRunThreads, smem1, s>>>(L);
    e = cudaGetLastError();
    if (e != cudaSuccess || !L.grad_h || pixel_tiles <= 0) return e;
    const size_t smem2 = (size_t)max_M * (16 + 7 * sizeof(int));   // list records, positions, sites, tile list
    e = cudaFuncSetAttribute(bwd_pixels_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    if (e != cudaSuccess) return e;
    // one CTA per image when the batch fills the GPU; otherwise each image's tiles are shared out
    // over `split` CTAs (a single large image would else run on one SM)
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bwd_pixels_kernel, kThreads, smem2)) != cudaSuccess)
        return e;
    const long long slots = (long long)sms * (per_sm > 0 ? per_sm : 1);
    long long split = (slots + B - 1) / B;
    if (split > max_image_tiles) split = max_image_tiles;
    if (split < 1) split = 1;
    BackwardLaunch L2 = L;
    L2.split = (int)split;
    bwd_pixels_kernel<<<(unsigned)(B * split), kThreads, smem2, s>>>(L2);
    return cudaGetLastError();
}

}  // namespace itc
