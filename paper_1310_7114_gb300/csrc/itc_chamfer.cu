// itc_chamfer.cu -- the chamfer distance transform that weights the pixels of a binary shape for
// weighted ITC (Sec. 5): T(x) = 3-4 chamfer distance of a foreground pixel to the nearest
// background pixel, the outside of the image counted as background; 0 on the background.
//
// The two raster passes of the 3 x 3 chamfer mask, with each row done in parallel: one warp per
// image walks the rows; lane l holds the columns 32 s + l of the row (s < NSEG segments).
//   forward (top to bottom):   c(u,j) = min(T(u-1,j-1) + 4, T(u-1,j) + 3, T(u-1,j+1) + 4)
//                              T(u,j) = min(c(u,j), T(u,j-1) + 3)
//     and the row recursion is a prefix minimum,  T(u,j) = 3j + min_{k <= j} (e(k) - 3k),  with
//     e = c on the shape, 0 on the background and at the frame column k = -1;
//   backward (bottom to top):  c(u,j) = min(T_f(u,j), T(u+1,j+1) + 4, T(u+1,j) + 3, T(u+1,j-1) + 4)
//                              T(u,j) = min(c(u,j), T(u,j+1) + 3) = -3j + min_{k >= j} (e(k) + 3k),
//     e = c on the shape, 0 on the background and at the frame column k = W.
// Each prefix (suffix) minimum is a warp scan of the 32 columns of a segment (all segments of a
// row scanned independently) plus the running minimum of the segments before it, so the result
// equals the sequential passes exactly (integer arithmetic).  The previous row stays in
// registers; the next input row is loaded one row ahead.  The forward result of row u is kept as
// 16-bit values in the first half of output row u, where the backward pass reads it before it
// overwrites the row with the final floats.
#include "itc_internal.cuh"

namespace itc {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int warp_prefix_min(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v = min(v, t);
    }
    return v;
}

__device__ __forceinline__ int warp_suffix_min(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_down_sync(kFull, v, o);
        if (lane + o < 32) v = min(v, t);
    }
    return v;
}

// Neighbours j - 1 and j + 1 of column j = 32 s + lane in the register row P (frame: 0).
template <int NSEG>
__device__ __forceinline__ void neighbours(const int (&P)[NSEG], int s, int nseg, int lane, int& left, int& right) {
    const int prev_last = __shfl_sync(kFull, s > 0 ? P[s > 0 ? s - 1 : 0] : 0, 31);
    const int next_first = __shfl_sync(kFull, s + 1 < nseg ? P[s + 1 < NSEG ? s + 1 : s] : 0, 0);
    left = __shfl_up_sync(kFull, P[s], 1);
    right = __shfl_down_sync(kFull, P[s], 1);
    if (lane == 0) left = prev_last;
    if (lane == 31) right = next_first;
}

template <int NSEG>
__global__ void __launch_bounds__(128) chamfer_kernel(const __grid_constant__ ChamferLaunch L) {
    const int lane = threadIdx.x & 31;
    const int slot = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (slot >= L.B) return;
    const ImageDesc& D = L.descs[__ldg(L.order + slot)];
    const int H = D.H, W = D.W, pitch = D.pitch, fp = D.fpitch;
    const int nseg = (W + 31) >> 5;
    const unsigned char* X = reinterpret_cast<const unsigned char*>(D.data);
    float* T = L.out + D.pad_off;
    unsigned short* Tf = reinterpret_cast<unsigned short*>(T);   // row u: Tf + 2 u fp

    int P[NSEG], cur[NSEG], nx[NSEG];
    // ---- forward pass
#pragma unroll
    for (int s = 0; s < NSEG; ++s) {
        P[s] = 0;
        const int j = 32 * s + lane;
        nx[s] = (s < nseg && j < W) ? (int)__ldg(X + j) : 0;
    }
    for (int u = 0; u < H; ++u) {
        int x[NSEG];
#pragma unroll
        for (int s = 0; s < NSEG; ++s) {
            x[s] = nx[s];
            const int j = 32 * s + lane;
            if (u + 1 < H && s < nseg && j < W) nx[s] = (int)__ldg(X + (size_t)(u + 1) * pitch + j);
        }
        // every segment's scan first (independent, so they overlap), then the running minimum of
        // the segments to the left, which only needs each segment's last value
        int v[NSEG], tot[NSEG];
#pragma unroll
        for (int s = 0; s < NSEG; ++s) {
            if (s >= nseg) break;
            const int j = 32 * s + lane;
            int left, right;
            neighbours<NSEG>(P, s, nseg, lane, left, right);
            const int c = min(min(left + 4, P[s] + 3), right + 4);
            const int e = (j < W && x[s] != 0) ? c : 0;
            v[s] = warp_prefix_min(e - 3 * j, lane);
            tot[s] = __shfl_sync(kFull, v[s], 31);
        }
        int carry = 3;   // frame column -1: e = 0 at k = -1
#pragma unroll
        for (int s = 0; s < NSEG; ++s) {
            if (s >= nseg) break;
            const int j = 32 * s + lane;
            cur[s] = j < W ? min(v[s], carry) + 3 * j : 0;
            carry = min(carry, tot[s]);
        }
#pragma unroll
        for (int s = 0; s < NSEG; ++s) {
            if (s >= nseg) break;
            const int j = 32 * s + lane;
            if (j < W) Tf[(size_t)u * 2 * fp + j] = (unsigned short)cur[s];
            P[s] = cur[s];
        }
    }
    __syncwarp();   // the forward rows are read back by other lanes below
    // ---- backward pass
#pragma unroll
    for (int s = 0; s < NSEG; ++s) {
        P[s] = 0;
        const int j = 32 * s + lane;
        nx[s] = (H > 0 && s < nseg && j < W) ? (int)Tf[(size_t)(H - 1) * 2 * fp + j] : 0;
    }
    for (int u = H - 1; u >= 0; --u) {
        int f[NSEG];
#pragma unroll
        for (int s = 0; s < NSEG; ++s) {
            f[s] = nx[s];
            const int j = 32 * s + lane;
            if (u > 0 && s < nseg && j < W) nx[s] = (int)Tf[(size_t)(u - 1) * 2 * fp + j];
        }
        int v[NSEG], tot[NSEG];
#pragma unroll
        for (int s = 0; s < NSEG; ++s) {
            if (s >= nseg) break;
            const int j = 32 * s + lane;
            int left, right;
            neighbours<NSEG>(P, s, nseg, lane, left, right);
            const int c = min(min(f[s], left + 4), min(P[s] + 3, right + 4));
            const int e = (j < W && f[s] != 0) ? c : 0;
            v[s] = warp_suffix_min(e + 3 * j, lane);
            tot[s] = __shfl_sync(kFull, v[s], 0);
        }
        int carry = 3 * W;   // frame column W: e = 0 at k = W
#pragma unroll
        for (int s = NSEG - 1; s >= 0; --s) {
            if (s >= nseg) continue;
            const int j = 32 * s + lane;
            cur[s] = j < W ? min(v[s], carry) - 3 * j : 0;
            carry = min(carry, tot[s]);
        }
        __syncwarp();   // every lane has read row u's forward values before it is overwritten
#pragma unroll
        for (int s = 0; s < NSEG; ++s) {
            if (s >= nseg) break;
            const int j = 32 * s + lane;
            if (j < W) T[(size_t)u * fp + j] = (float)cur[s];
            P[s] = cur[s];
        }
    }
}

}  // namespace

cudaError_t launch_chamfer(const ChamferLaunch& L, int max_W, cudaStream_t s) {
    if (L.B <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((L.B + 3) / 4);
    if (max_W <= 128) chamfer_kernel<4><<<grid, 128, 0, s>>>(L);
    else if (max_W <= 256) chamfer_kernel<8><<<grid, 128, 0, s>>>(L);
    else if (max_W <= 512) chamfer_kernel<16><<<grid, 128, 0, s>>>(L);
    else chamfer_kernel<32><<<grid, 128, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace itc
