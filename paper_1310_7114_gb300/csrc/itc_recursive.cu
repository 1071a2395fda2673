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

template <bool MOM>   // MOM: the moment fields too (else the self-overlap pass: A alone)
__global__ void __launch_bounds__(32 * kRecRowWarps) rec_rows_kernel(const __grid_constant__ RecursiveLaunch L) {
    const ImageDesc& D = rec_image(L);
    const int H = D.H, W = D.W, fp = D.fpitch, pitch = D.pitch;
    float* P0 = L.fields + (MOM ? D.field_off + 3 * D.plane_floats : D.self_off + D.plane_floats);
    float* P1 = P0 + D.plane_floats;   // T_v (moments only)
    const RecCoef& rc = MOM ? D.rc : D.rc_self;
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
    const int r0 = (blockIdx.y * kRecRowWarps + wid) * 32;
    if (r0 >= H) return;
    const int nr = min(32, H - r0);
    float* const q0 = P0 + (size_t)r0 * fp;   // row r0 of the scratch planes
    float* const q1 = P1 + (size_t)r0 * fp;
    const bool u8 = D.dtype == ITC_U8;
    const unsigned char* const xb = reinterpret_cast<const unsigned char*>(D.data) + (size_t)r0 * pitch;
    const float* const xf = reinterpret_cast<const float*>(D.data) + (size_t)r0 * pitch;
    auto load_x = [&](int cb) {   // input tile: rows r0.., columns cb.. (8 loads in flight at a time)
        const int v = cb + lane;
        if (v < W && u8) {
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr)
                if (rr < nr) X[rr][lane] = (float)__ldg(xb + rr * pitch + v);
        } else if (v < W) {
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr)
                if (rr < nr) X[rr][lane] = __ldg(xf + rr * pitch + v);
        } else {
            for (int rr = 0; rr < nr; ++rr) X[rr][lane] = 0.f;
        }
        __syncwarp();
    };
    auto store_tile = [&](int cb, int nc) {   // the staged outputs back, one coalesced row segment per row
        if (lane < nc) {
            for (int rr = 0; rr < nr; ++rr) {
                q0[rr * fp + cb + lane] = O0[rr][lane];
                if (MOM) q1[rr * fp + cb + lane] = O1[rr][lane];
            }
        }
        __syncwarp();
    };
    // causal: tiles left to right
    Cplx a0 = {0.f, 0.f}, a1 = {0.f, 0.f}, m0 = {0.f, 0.f}, m1 = {0.f, 0.f};   // s0, s1 per term
    auto causal = [&](int cc) {
        const float x = X[lane][cc];
        m0 = cmul(z0, cadd(m0, a0));
        m1 = cmul(z1, cadd(m1, a1));
        a0 = cmul(z0, a0); a0.r += x;
        a1 = cmul(z1, a1); a1.r += x;
        O0[lane][cc] = re_mul(c0, a0) + re_mul(c1, a1);
        if (MOM) O1[lane][cc] = -(re_mul(c0, m0) + re_mul(c1, m1));
    };
    for (int tc = 0; tc < ntc; ++tc) {
        const int cb = tc * 32, nc = min(32, W - cb);
        load_x(cb);
        if (lane < nr) {
            if (nc == 32) {
#pragma unroll 8
                for (int cc = 0; cc < 32; ++cc) causal(cc);
            } else {
                for (int cc = 0; cc < nc; ++cc) causal(cc);
            }
        }
        __syncwarp();
        store_tile(cb, nc);
    }
    // anticausal: tiles right to left; x[v + 1] of a tile's last column is the first column
    // of the tile to its right
    a0 = a1 = m0 = m1 = Cplx{0.f, 0.f};   // r0, r1 per term
    float xnext = 0.f;
    auto anticausal = [&](int cc, float xn) {
        m0 = cmul(z0, cadd(cadd(m0, a0), Cplx{xn, 0.f}));
        m1 = cmul(z1, cadd(cadd(m1, a1), Cplx{xn, 0.f}));
        a0 = cmul(z0, cadd(a0, Cplx{xn, 0.f}));
        a1 = cmul(z1, cadd(a1, Cplx{xn, 0.f}));
        O0[lane][cc] += re_mul(c0, a0) + re_mul(c1, a1);
        if (MOM) O1[lane][cc] += re_mul(c0, m0) + re_mul(c1, m1);
    };
    for (int tc = ntc - 1; tc >= 0; --tc) {
        const int cb = tc * 32, nc = min(32, W - cb);
        load_x(cb);
        if (lane < nc) {
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) {
                if (rr < nr) {
                    O0[rr][lane] = q0[rr * fp + cb + lane];
                    if (MOM) O1[rr][lane] = q1[rr * fp + cb + lane];
                }
            }
        }
        __syncwarp();
        if (lane < nr) {
            if (nc == 32) {
                anticausal(31, xnext);
#pragma unroll 8
                for (int cc = 30; cc >= 0; --cc) anticausal(cc, X[lane][cc + 1]);
            } else {
                for (int cc = nc - 1; cc >= 0; --cc) anticausal(cc, cc + 1 < nc ? X[lane][cc + 1] : xnext);
            }
            xnext = X[lane][0];
        }
        __syncwarp();
        store_tile(cb, nc);
    }
}

template <bool MOM>
__global__ void __launch_bounds__(kRecColThreads) rec_cols_kernel(const __grid_constant__ RecursiveLaunch L) {
    const ImageDesc& D = rec_image(L);
    const int H = D.H, W = D.W, fp = D.fpitch;
    const long long pl = D.plane_floats;
    const float* T = L.fields + (MOM ? D.field_off + 3 * pl : D.self_off + pl);
    const float* Tv = T + pl;
    float* A = L.fields + (MOM ? D.field_off : D.self_off);
    float* Fu = A + pl;
    float* Fv = A + 2 * pl;
    const RecCoef& rc = MOM ? D.rc : D.rc_self;
    const Cplx z0 = {rc.zr[0][0], rc.zi[0][0]}, z1 = {rc.zr[0][1], rc.zi[0][1]};
    const Cplx c0 = {rc.cr[0], rc.ci[0]}, c1 = {rc.cr[1], rc.ci[1]};
    const int lane = threadIdx.x & 31;
    const long long poff = MOM ? D.partial_off : D.sxx_off;
    // whole warps walk the columns so that each warp's partial covers 32 consecutive columns;
    // this CTA takes columns blockIdx.y * kRecColThreads ..
    const int wcols = (W + 31) & ~31;
    const int vb = blockIdx.y * kRecColThreads;
    if (vb + (threadIdx.x & ~31) >= wcols) return;   // whole warps past the image
    // rows go in chunks of kRecCh: a chunk's loads are all issued before its recursion steps,
    // so the sequential walk waits on one memory round trip per chunk, not per row.  S_XX of the
    // column: FP32 within a chunk (at most kRecCh non-negative products), FP64 across chunks.
    constexpr int CH = kRecCh;
    const int v = vb + threadIdx.x;
    double hs = 0.0;
    if (v < W) {
        const bool u8 = D.dtype == ITC_U8;
        const unsigned char* const hb = reinterpret_cast<const unsigned char*>(D.data) + v;
        const float* const hf = reinterpret_cast<const float*>(D.data) + v;
        const int pitch = D.pitch;
        Cplx a0 = {0.f, 0.f}, a1 = {0.f, 0.f}, m0 = {0.f, 0.f}, m1 = {0.f, 0.f}, b0 = {0.f, 0.f}, b1 = {0.f, 0.f};
        for (int ub = 0; ub < H; ub += CH) {
            float xs[CH], ys[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int u = ub + c;
                xs[c] = u < H ? T[(size_t)u * fp + v] : 0.f;
                ys[c] = (MOM && u < H) ? Tv[(size_t)u * fp + v] : 0.f;
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
                if (MOM) {
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
                    hv[c] = u8 ? (float)__ldg(hb + (size_t)u * pitch) : __ldg(hf + (size_t)u * pitch);
                    if (MOM) {
                        yn[c] = u + 1 < H ? Tv[o + fp] : 0.f;
                        fu[c] = Fu[o];
                        fv[c] = Fv[o];
                    }
                }
            }
            float hc = 0.f;
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
                if (MOM) {
                    b0 = cmul(z0, cadd(b0, Cplx{yn[c], 0.f}));
                    b1 = cmul(z1, cadd(b1, Cplx{yn[c], 0.f}));
                    Fu[o] = fu[c] + (re_mul(c0, m0) + re_mul(c1, m1));
                    Fv[o] = fv[c] + (re_mul(c0, b0) + re_mul(c1, b1));
                }
                hc = fmaf(hv[c], a, hc);
            }
            hs += (double)hc;
        }
    }
    // S_XX share of these 32 columns: a fixed-order shuffle tree
    for (int o = 16; o > 0; o >>= 1) hs += __shfl_xor_sync(0xffffffffu, hs, o);
    if (lane == 0) L.partials[poff + (v >> 5)] = hs;
}

}  // namespace

cudaError_t launch_recursive(const RecursiveLaunch& L, int nimg, int max_H, int max_W, cudaStream_t s) {
    if (nimg <= 0 || max_H <= 0 || max_W <= 0) return cudaSuccess;
    const size_t smem = (size_t)kRecRowWarps * kRecTileFloats * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(rec_rows_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(rec_rows_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grow((unsigned)nimg, (unsigned)((max_H + 32 * kRecRowWarps - 1) / (32 * kRecRowWarps)));
    const dim3 gcol((unsigned)nimg, (unsigned)((max_W + kRecColThreads - 1) / kRecColThreads));
    if (L.mode == 0) {
        rec_rows_kernel<true><<<grow, 32 * kRecRowWarps, smem, s>>>(L);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        rec_cols_kernel<true><<<gcol, kRecColThreads, 0, s>>>(L);
    } else {
        rec_rows_kernel<false><<<grow, 32 * kRecRowWarps, smem, s>>>(L);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        rec_cols_kernel<false><<<gcol, kRecColThreads, 0, s>>>(L);
    }
    return cudaGetLastError();
}

}  // namespace itc
