// itc_recursive.cu -- 2-D fields for large widths by recursive filtering (Sec. 3.1 points to
// recursive filters, citing Deriche 1992): the cost per pixel does not grow with sigma.
//
// Deriche's recursive Gaussian fits the kernel by two damped sinusoids,
//     exp(-x^2/2) ~ sum_t Re(c_t exp((-b_t + i omega_t) x)),  x >= 0,
// so with z_t = exp((-b_t + i omega_t) / sigma) the sampled kernel is g(j) ~ Re sum_t c_t z_t^j and
// a convolution along one axis is four first-order complex recursions per signal:
//   causal       s0[n] = x[n] + z s0[n-1],          s1[n] = z (s1[n-1] + s0[n-1])
//   anticausal   r0[n] = z (r0[n+1] + x[n+1]),      r1[n] = z (r1[n+1] + r0[n+1] + x[n+1])
//   g * x  = Re sum_t c_t (s0 + r0),     (d g) * x = Re sum_t c_t (r1 - s1)     (d = offset)
// with zero states at the ends (no data outside the image), so the kernel is untruncated.
//
// Pass along v (one lane per row, rows staged through shared memory in 32 x 32 tiles so that
// global accesses are coalesced; a warp per 32-row block, the blocks of an image spread over the
// grid's y dimension): T = g_v * h, T_v = (d g)_v * h into two scratch planes (the causal part is
// stored, the anticausal part added).  Pass along u (one thread per column, 128 columns per CTA,
// so warps read and write whole row segments; rows in prefetched chunks): A = g_u * T,
// F_u = (d g)_u * T, F_v = g_u * T_v into the field planes, same order; the column pass also sums
// h A per column (FP64) and each warp's 32 columns into one S_XX partial, in a fixed order.  The
// self-overlap pass (mode 1) computes A alone into the A_s plane with one scratch plane.
#include "itc_internal.cuh"

namespace itc {
namespace {

struct Cplx {
    float r, i;
};
__device__ __forceinline__ Cplx cmul(Cplx a, Cplx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ Cplx cadd(Cplx a, Cplx b) { return {a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ float re_mul(Cplx c, Cplx s) { return c.r * s.r - c.i * s.i; }

__device__ __forceinline__ float pixel(const ImageDesc& D, int u, int v) {
    const size_t o = (size_t)u * D.pitch + v;
    if (D.dtype == ITC_U8) return (float)__ldg(reinterpret_cast<const unsigned char*>(D.data) + o);
    return __ldg(reinterpret_cast<const float*>(D.data) + o);
}

// the image of the CTA: the class list entry of position base + blockIdx.x (blockIdx.y picks the
// CTA's block of rows or columns within it)
__device__ __forceinline__ const ImageDesc& rec_image(const RecursiveLaunch& L) {
    return L.descs[__ldg(L.img_list + L.pos_base + blockIdx.x)];
}

// Along v: a warp takes 32 rows, one lane per row, and walks them in 32 x 32 tiles staged in
// shared memory (rows of 33 floats), so every global load and store is a coalesced row segment
// while each lane runs its row's recursion on the staged tile.
constexpr int kRecRowWarps = 4;                        // row blocks per CTA
constexpr int kRecTileFloats = 3 * 32 * 33;            // a warp's three 32 x 33 tiles
constexpr int kRecCh = 8;                              // rows per prefetched chunk in the column pass
constexpr int kRecColThreads = 128;                    // columns per CTA in the column pass

__global__ void __launch_bounds__(32 * kRecRowWarps) rec_rows_kernel(const __grid_constant__ RecursiveLaunch L) {
    const ImageDesc& D = rec_image(L);
    const int H = D.H, W = D.W, fp = D.fpitch;
    const bool moments = L.mode == 0;
    float* P0 = L.fields + (moments ? D.field_off + 3 * D.plane_floats : D.self_off + D.plane_floats);
    float* P1 = P0 + D.plane_floats;   // T_v (moments only)
    const RecCoef& rc = moments ? D.rc : D.rc_self;
    const Cplx z0 = {rc.zr[1][0], rc.zi[1][0]}, z1 = {rc.zr[1][1], rc.zi[1][1]};
    const Cplx c0 = {rc.cr[0], rc.ci[0]}, c1 = {rc.cr[1], rc.ci[1]};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    extern __shared__ float rsm[];
    float (*X)[33] = reinterpret_cast<float (*)[33]>(rsm + wid * kRecTileFloats);
    float (*O0)[33] = X + 32;
    float (*O1)[33] = X + 64;
    const int ntc = (W + 31) / 32;
    // this warp's block of 32 rows (warps past the image's last row have nothing to do; the
    // kernel takes no block-wide barrier)
    {
        const int r0 = (blockIdx.y * kRecRowWarps + wid) * 32;
        if (r0 >= H) return;
        const int nr = min(32, H - r0);
        auto load_x = [&](int cb) {   // input tile: rows r0.., columns cb.. (8 loads in flight at a time)
            const int v = cb + lane;
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr)
                if (rr < nr) X[rr][lane] = v < W ? pixel(D, r0 + rr, v) : 0.f;
            __syncwarp();
        };
        // causal: tiles left to right
        Cplx a0 = {0.f, 0.f}, a1 = {0.f, 0.f}, m0 = {0.f, 0.f}, m1 = {0.f, 0.f};   // s0, s1 per term
        for (int tc = 0; tc < ntc; ++tc) {
            const int cb = tc * 32, nc = min(32, W - cb);
            load_x(cb);
            if (lane < nr) {
                for (int cc = 0; cc < nc; ++cc) {
                    const float x = X[lane][cc];
                    m0 = cmul(z0, cadd(m0, a0));
                    m1 = cmul(z1, cadd(m1, a1));
                    a0 = cmul(z0, a0); a0.r += x;
                    a1 = cmul(z1, a1); a1.r += x;
                    O0[lane][cc] = re_mul(c0, a0) + re_mul(c1, a1);
                    if (moments) O1[lane][cc] = -(re_mul(c0, m0) + re_mul(c1, m1));
                }
            }
            __syncwarp();
            for (int rr = 0; rr < nr; ++rr) {
                if (lane < nc) {
                    P0[(size_t)(r0 + rr) * fp + cb + lane] = O0[rr][lane];
                    if (moments) P1[(size_t)(r0 + rr) * fp + cb + lane] = O1[rr][lane];
                }
            }
            __syncwarp();
        }
        // anticausal: tiles right to left; x[v + 1] of a tile's last column is the first column
        // of the tile to its right
        a0 = a1 = m0 = m1 = Cplx{0.f, 0.f};   // r0, r1 per term
        float xnext = 0.f;
        for (int tc = ntc - 1; tc >= 0; --tc) {
            const int cb = tc * 32, nc = min(32, W - cb);
            load_x(cb);
            if (lane < nc) {
#pragma unroll 4
                for (int rr = 0; rr < 32; ++rr) {
                    if (rr < nr) {
                        O0[rr][lane] = P0[(size_t)(r0 + rr) * fp + cb + lane];
                        if (moments) O1[rr][lane] = P1[(size_t)(r0 + rr) * fp + cb + lane];
                    }
                }
            }
            __syncwarp();
            if (lane < nr) {
                for (int cc = nc - 1; cc >= 0; --cc) {
                    const float xn = cc + 1 < nc ? X[lane][cc + 1] : xnext;
                    m0 = cmul(z0, cadd(cadd(m0, a0), Cplx{xn, 0.f}));
                    m1 = cmul(z1, cadd(cadd(m1, a1), Cplx{xn, 0.f}));
                    a0 = cmul(z0, cadd(a0, Cplx{xn, 0.f}));
                    a1 = cmul(z1, cadd(a1, Cplx{xn, 0.f}));
                    O0[lane][cc] += re_mul(c0, a0) + re_mul(c1, a1);
                    if (moments) O1[lane][cc] += re_mul(c0, m0) + re_mul(c1, m1);
                }
                xnext = X[lane][0];
            }
            __syncwarp();
            for (int rr = 0; rr < nr; ++rr) {
                if (lane < nc) {
                    P0[(size_t)(r0 + rr) * fp + cb + lane] = O0[rr][lane];
                    if (moments) P1[(size_t)(r0 + rr) * fp + cb + lane] = O1[rr][lane];
                }
            }
            __syncwarp();
        }
    }
}

__global__ void __launch_bounds__(kRecColThreads) rec_cols_kernel(const __grid_constant__ RecursiveLaunch L) {
    const ImageDesc& D = rec_image(L);
    const int H = D.H, W = D.W, fp = D.fpitch;
    const bool moments = L.mode == 0;
    const long long pl = D.plane_floats;
    const float* T = L.fields + (moments ? D.field_off + 3 * pl : D.self_off + pl);
    const float* Tv = T + pl;
    float* A = L.fields + (moments ? D.field_off : D.self_off);
    float* Fu = A + pl;
    float* Fv = A + 2 * pl;
    const RecCoef& rc = moments ? D.rc : D.rc_self;
    const Cplx z0 = {rc.zr[0][0], rc.zi[0][0]}, z1 = {rc.zr[0][1], rc.zi[0][1]};
    const Cplx c0 = {rc.cr[0], rc.ci[0]}, c1 = {rc.cr[1], rc.ci[1]};
    const int lane = threadIdx.x & 31;
    const long long poff = moments ? D.partial_off : D.sxx_off;
    // whole warps walk the columns so that each warp's partial covers 32 consecutive columns;
    // this CTA takes columns blockIdx.y * kRecColThreads ..
    const int wcols = (W + 31) & ~31;
    const int vb = blockIdx.y * kRecColThreads;
    if (vb + (threadIdx.x & ~31) >= wcols) return;   // whole warps past the image
    // rows go in chunks of kRecCh: a chunk's loads are all issued before its recursion steps,
    // so the sequential walk waits on one memory round trip per chunk, not per row
    constexpr int CH = kRecCh;
    {
        const int v = vb + threadIdx.x;
        const bool on = v < W;
        double hs = 0.0;
        if (on) {
            Cplx a0 = {0.f, 0.f}, a1 = {0.f, 0.f}, m0 = {0.f, 0.f}, m1 = {0.f, 0.f}, b0 = {0.f, 0.f}, b1 = {0.f, 0.f};
            for (int ub = 0; ub < H; ub += CH) {
                float xs[CH], ys[CH];
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const int u = ub + c;
                    xs[c] = u < H ? T[(size_t)u * fp + v] : 0.f;
                    ys[c] = (moments && u < H) ? Tv[(size_t)u * fp + v] : 0.f;
                }
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const int u = ub + c;
                    if (u >= H) break;
                    const size_t o = (size_t)u * fp + v;
                    const float x = xs[c];
                    m0 = cmul(z0, cadd(m0, a0));
                    m1 = cmul(z1, cadd(m1, a1));
                    a0 = cmul(z0, a0); a0.r += x;
                    a1 = cmul(z1, a1); a1.r += x;
                    A[o] = re_mul(c0, a0) + re_mul(c1, a1);
                    if (moments) {
                        const float y = ys[c];
                        b0 = cmul(z0, b0); b0.r += y;
                        b1 = cmul(z1, b1); b1.r += y;
                        Fu[o] = -(re_mul(c0, m0) + re_mul(c1, m1));
                        Fv[o] = re_mul(c0, b0) + re_mul(c1, b1);
                    }
                }
            }
            a0 = a1 = m0 = m1 = b0 = b1 = Cplx{0.f, 0.f};
            for (int ue = H - 1; ue >= 0; ue -= CH) {
                // this chunk's inputs (the row below each row) and the causal parts it adds to
                float xn[CH], yn[CH], ao[CH], fu[CH], fv[CH], hv[CH];
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const int u = ue - c;
                    xn[c] = yn[c] = ao[c] = fu[c] = fv[c] = hv[c] = 0.f;
                    if (u >= 0) {
                        const size_t o = (size_t)u * fp + v;
                        xn[c] = u + 1 < H ? T[o + fp] : 0.f;
                        ao[c] = A[o];
                        hv[c] = pixel(D, u, v);
                        if (moments) {
                            yn[c] = u + 1 < H ? Tv[o + fp] : 0.f;
                            fu[c] = Fu[o];
                            fv[c] = Fv[o];
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const int u = ue - c;
                    if (u < 0) break;
                    const size_t o = (size_t)u * fp + v;
                    m0 = cmul(z0, cadd(cadd(m0, a0), Cplx{xn[c], 0.f}));
                    m1 = cmul(z1, cadd(cadd(m1, a1), Cplx{xn[c], 0.f}));
                    a0 = cmul(z0, cadd(a0, Cplx{xn[c], 0.f}));
                    a1 = cmul(z1, cadd(a1, Cplx{xn[c], 0.f}));
                    const float a = ao[c] + re_mul(c0, a0) + re_mul(c1, a1);
                    A[o] = a;
                    if (moments) {
                        b0 = cmul(z0, cadd(b0, Cplx{yn[c], 0.f}));
                        b1 = cmul(z1, cadd(b1, Cplx{yn[c], 0.f}));
                        Fu[o] = fu[c] + (re_mul(c0, m0) + re_mul(c1, m1));
                        Fv[o] = fv[c] + (re_mul(c0, b0) + re_mul(c1, b1));
                    }
                    hs += (double)hv[c] * (double)a;
                }
            }
        }
        // S_XX share of these 32 columns: a fixed-order shuffle tree
        for (int o = 16; o > 0; o >>= 1) hs += __shfl_xor_sync(0xffffffffu, hs, o);
        if (lane == 0) L.partials[poff + (v >> 5)] = hs;
    }
}

}  // namespace

cudaError_t launch_recursive(const RecursiveLaunch& L, int nimg, int max_H, int max_W, cudaStream_t s) {
    if (nimg <= 0 || max_H <= 0 || max_W <= 0) return cudaSuccess;
    const size_t smem = (size_t)kRecRowWarps * kRecTileFloats * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(rec_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grow((unsigned)nimg, (unsigned)((max_H + 32 * kRecRowWarps - 1) / (32 * kRecRowWarps)));
    rec_rows_kernel<<<grow, 32 * kRecRowWarps, smem, s>>>(L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const dim3 gcol((unsigned)nimg, (unsigned)((max_W + kRecColThreads - 1) / kRecColThreads));
    rec_cols_kernel<<<gcol, kRecColThreads, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace itc
