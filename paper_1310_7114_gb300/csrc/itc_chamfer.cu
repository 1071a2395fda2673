// itc_chamfer.cu -- the chamfer distance transform that weights the pixels of a binary shape for
// weighted ITC (Sec. 5): T(x) = 3-4 chamfer distance of a foreground pixel to the nearest
// background pixel, the outside of the image counted as background; 0 on the background.
//
// The two raster passes of the 3 x 3 chamfer mask, with each row done in parallel: one warp per
// image walks the rows; lane l holds columns 128 q + 4 l + t (t = 0..3) of each 128-column chunk q.
//   forward (top to bottom):   c(u,j) = min(T(u-1,j-1) + 4, T(u-1,j) + 3, T(u-1,j+1) + 4)
//                              T(u,j) = min(c(u,j), T(u,j-1) + 3)
//     and the row recursion is a prefix minimum,  T(u,j) = 3j + min_{k <= j} (e(k) - 3k),  with
//     e = c on the shape, 0 on the background and at the frame column k = -1;
//   backward (bottom to top):  c(u,j) = min(T_f(u,j), T(u+1,j+1) + 4, T(u+1,j) + 3, T(u+1,j-1) + 4)
//                              T(u,j) = min(c(u,j), T(u,j+1) + 3) = -3j + min_{k >= j} (e(k) + 3k),
//     e = c on the shape, 0 on the background and at the frame column k = W.
// Each prefix (suffix) minimum is a running minimum over a lane's 4 columns, a warp scan of the
// lane minima, and the running minimum of the chunks before it, so the result equals the
// sequential passes exactly (integer arithmetic).  The previous row is kept in shared memory
// (two buffers per warp); input bytes come 4 at a time with 32-bit loads, one row ahead, and the
// forward values 4 at a time with 64-bit loads.  The forward result of row u is kept as 16-bit
// values in the first half of output row u, where the backward pass reads it before it
// overwrites the row with the final floats.
#include "itc_internal.cuh"

namespace itc {
namespace {

constexpr unsigned kFull = 0xffffffffu;

constexpr int kBig = 0x3fffffff;   // +infinity for the prefix minima

// 32-bit loads of 4 input bytes need 4-byte aligned rows
__device__ __forceinline__ uint32_t load_bytes4(const unsigned char* row, int j0, int W, bool aligned) {
    if (aligned && j0 + 3 < W) return __ldg(reinterpret_cast<const uint32_t*>(row + j0));
    uint32_t w = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (j0 + t < W) w |= (uint32_t)__ldg(row + j0 + t) << (8 * t);
    return w;
}

// NCH chunks of 128 columns per row; lane l holds columns 128 q + 4 l + t, t = 0..3.  The previous
// row lives in shared memory (two buffers per warp, alternating by row; columns past W hold 0).
template <int NCH>
__global__ void __launch_bounds__(128) chamfer_kernel(const __grid_constant__ ChamferLaunch L) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int slot = blockIdx.x * 4 + wid;
    extern __shared__ __align__(16) int csm[];
    constexpr int RW = 128 * NCH + 4;                   // a row plus the zero column past the last chunk
    int* rows = csm + wid * 2 * RW;
    if (slot >= L.B) return;
    const ImageDesc& D = L.descs[__ldg(L.order + slot)];
    const int H = D.H, W = D.W, pitch = D.pitch, fp = D.fpitch;
    const int nch = (W + 127) >> 7;
    const unsigned char* X = reinterpret_cast<const unsigned char*>(D.data);
    const bool aligned = ((pitch & 3) == 0) && ((reinterpret_cast<size_t>(X) & 3) == 0);
    float* T = L.out + D.pad_off;
    unsigned short* Tf = reinterpret_cast<unsigned short*>(T);   // row u: Tf + 2 u fp

    for (int i = lane; i < 2 * RW; i += 32) rows[i] = 0;   // the frame row (zeros), both buffers
    __syncwarp();
    // ---- forward pass: T(u, j) = min(c(u, j), T(u, j - 1) + 3) = 3 j + min_{k <= j} (e(k) - 3 k)
    uint32_t nx[NCH];
#pragma unroll
    for (int q = 0; q < NCH; ++q) nx[q] = (q < nch && H > 0) ? load_bytes4(X, 128 * q + 4 * lane, W, aligned) : 0u;
    for (int u = 0; u < H; ++u) {
        const int* Pr = rows + (u & 1) * RW;            // row u - 1
        int* Cr = rows + ((u + 1) & 1) * RW;            // row u
        uint32_t xw[NCH];
#pragma unroll
        for (int q = 0; q < NCH; ++q) {
            xw[q] = nx[q];
            if (u + 1 < H && q < nch) nx[q] = load_bytes4(X + (size_t)(u + 1) * pitch, 128 * q + 4 * lane, W, aligned);
        }
        int carry = 3;   // frame column -1: e = 0 at k = -1
#pragma unroll
        for (int q = 0; q < NCH; ++q) {
            if (q >= nch) break;
            const int j0 = 128 * q + 4 * lane;
            const int4 p = *reinterpret_cast<const int4*>(Pr + j0);
            const int pl = j0 > 0 ? Pr[j0 - 1] : 0, pr = Pr[j0 + 4];
            const int pv[6] = {pl, p.x, p.y, p.z, p.w, pr};
            int m[4], run = kBig;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int c = min(min(pv[t] + 4, pv[t + 1] + 3), pv[t + 2] + 4);
                const int e = (j0 + t < W && ((xw[q] >> (8 * t)) & 0xffu) != 0u) ? c : 0;
                run = min(run, e - 3 * (j0 + t));
                m[t] = run;
            }
            // minimum over the lanes before this one (exclusive scan of the lane minima)
            int incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl = min(incl, y);
            }
            int excl = __shfl_up_sync(kFull, incl, 1);
            if (lane == 0) excl = kBig;
            const int cin = min(carry, excl);
            carry = min(carry, __shfl_sync(kFull, incl, 31));
            int tv[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) tv[t] = j0 + t < W ? min(m[t], cin) + 3 * (j0 + t) : 0;
            *reinterpret_cast<int4*>(Cr + j0) = make_int4(tv[0], tv[1], tv[2], tv[3]);
            unsigned short* o = Tf + (size_t)u * 2 * fp + j0;
            if (j0 + 3 < W) {
                *reinterpret_cast<uint2*>(o) = make_uint2((uint32_t)tv[0] | ((uint32_t)tv[1] << 16),
                                                          (uint32_t)tv[2] | ((uint32_t)tv[3] << 16));
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (j0 + t < W) o[t] = (unsigned short)tv[t];
            }
        }
        __syncwarp();   // row u complete before it is read as the previous row
    }
    __syncwarp();   // the forward rows are read back by other lanes below
    // ---- backward pass: T(u, j) = min(c(u, j), T(u, j + 1) + 3) = -3 j + min_{k >= j} (e(k) + 3 k)
    for (int i = lane; i < 2 * RW; i += 32) rows[i] = 0;   // the frame row below the image
    __syncwarp();
    auto load_f = [&](int u, int j0) -> uint2 {   // forward values of row u, columns j0 .. j0 + 3
        const unsigned short* r = Tf + (size_t)u * 2 * fp + j0;
        if (j0 + 3 < W) return *reinterpret_cast<const uint2*>(r);
        uint32_t a = 0, b = 0;
        if (j0 < W) a |= r[0];
        if (j0 + 1 < W) a |= (uint32_t)r[1] << 16;
        if (j0 + 2 < W) b |= r[2];
        if (j0 + 3 < W) b |= (uint32_t)r[3] << 16;
        return make_uint2(a, b);
    };
    uint2 nf[NCH];
#pragma unroll
    for (int q = 0; q < NCH; ++q) nf[q] = (q < nch && H > 0) ? load_f(H - 1, 128 * q + 4 * lane) : make_uint2(0u, 0u);
    for (int u = H - 1; u >= 0; --u) {
        const int* Pr = rows + (u & 1) * RW;            // row u + 1 (final values)
        int* Cr = rows + ((u + 1) & 1) * RW;            // row u
        uint2 fw[NCH];
#pragma unroll
        for (int q = 0; q < NCH; ++q) {
            fw[q] = nf[q];
            if (u > 0 && q < nch) nf[q] = load_f(u - 1, 128 * q + 4 * lane);
        }
        __syncwarp();   // every lane has read row u's forward values before it is overwritten
        int carry = 3 * W;   // frame column W: e = 0 at k = W
#pragma unroll
        for (int qq = NCH - 1; qq >= 0; --qq) {
            if (qq >= nch) continue;
            const int q = qq, j0 = 128 * q + 4 * lane;
            const int4 p = *reinterpret_cast<const int4*>(Pr + j0);
            const int pl = j0 > 0 ? Pr[j0 - 1] : 0, pr = Pr[j0 + 4];
            const int pv[6] = {pl, p.x, p.y, p.z, p.w, pr};
            const int fv[4] = {(int)(fw[q].x & 0xffffu), (int)(fw[q].x >> 16), (int)(fw[q].y & 0xffffu),
                               (int)(fw[q].y >> 16)};
            int n[4], run = kBig;
#pragma unroll
            for (int t = 3; t >= 0; --t) {
                const int c = min(min(fv[t], pv[t] + 4), min(pv[t + 1] + 3, pv[t + 2] + 4));
                const int e = (j0 + t < W && fv[t] != 0) ? c : 0;
                run = min(run, e + 3 * (j0 + t));
                n[t] = run;
            }
            // minimum over the lanes after this one
            int incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_down_sync(kFull, incl, o);
                if (lane + o < 32) incl = min(incl, y);
            }
            int excl = __shfl_down_sync(kFull, incl, 1);
            if (lane == 31) excl = kBig;
            const int cin = min(carry, excl);
            carry = min(carry, __shfl_sync(kFull, incl, 0));
            int tv[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) tv[t] = j0 + t < W ? min(n[t], cin) - 3 * (j0 + t) : 0;
            *reinterpret_cast<int4*>(Cr + j0) = make_int4(tv[0], tv[1], tv[2], tv[3]);
            float* o = T + (size_t)u * fp + j0;
            if (j0 + 3 < W) {
                *reinterpret_cast<float4*>(o) = make_float4((float)tv[0], (float)tv[1], (float)tv[2], (float)tv[3]);
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (j0 + t < W) o[t] = (float)tv[t];
            }
        }
        __syncwarp();   // row u complete before it is read as the next row's neighbour
    }
}

}  // namespace

cudaError_t launch_chamfer(const ChamferLaunch& L, int max_W, cudaStream_t s) {
    if (L.B <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((L.B + 3) / 4);
    auto go = [&](auto k, int nch) -> cudaError_t {
        const size_t smem = (size_t)4 * 2 * (128 * nch + 4) * sizeof(int);   // two rows per warp
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<grid, 128, smem, s>>>(L);
        return cudaGetLastError();
    };
    if (max_W <= 128) return go(chamfer_kernel<1>, 1);
    if (max_W <= 256) return go(chamfer_kernel<2>, 2);
    if (max_W <= 512) return go(chamfer_kernel<4>, 4);
    return go(chamfer_kernel<8>, 8);
}

}  // namespace itc
