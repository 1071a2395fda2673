// itc_segment.cu -- segmentation of the data pixels by the codebook (the segments of Figs. 3 and 6).
//
// Every pixel with data (h != 0; in 3-D the voxel (u, v, gray(u, v))) gets the index of the
// codebook vector whose lattice site r_k = round(w_k) gives the largest kernel value
// g_tau(x - r_k), i.e. the smallest
//     D_k(x) = sum_i d_i^2 q_i,   d_i = x_i - r_{k,i},  q_i = 1 / tau_i^2 (rounded once to float),
// evaluated in single precision term by term (each product rounded, the terms added in axis
// order with one rounding each, no fused multiply-add), lowest k on ties; pixels without data
// get -1.
//
// One CTA per image (largest images first); its warps take the image's 16 x 16 pixel tiles in
// turn, each on its own (no block-wide barrier after the codebook is staged).  The small tile
// keeps the candidate list short: on a batch of 4096 ragged binary shapes (sides 64 to 512,
// M up to 128) 16 x 16 tiles take 1.21 ms against 1.51 ms for 32 x 32 (the lists cost more than
// they save at 8 x 8).  Per tile the
// codebooks that can win somewhere in it are listed first: with dmin_k / dmax_k the metric of
// the nearest / farthest point of the tile's box, every k with dmin_k <= min_j dmax_j (the same
// rounded arithmetic, which is monotone in each |d_i|, so the bounds hold for every pixel).  The
// list keeps k order, so the first strict minimum over it is the lowest index on ties.
#include "itc_internal.cuh"

namespace itc {
namespace {

constexpr int kSegTile = 16;

__device__ __forceinline__ int site_round(float x, int n) {
    const float r = floorf(x + 0.5f);
    return (int)fminf(fmaxf(r, 0.f), (float)(n - 1));
}

// sum_i d_i^2 q_i with every product and sum rounded separately (axis order)
__device__ __forceinline__ float metric(int nd, int d0, int d1, int d2, float q0, float q1, float q2) {
    float m = __fadd_rn(__fmul_rn((float)(d0 * d0), q0), __fmul_rn((float)(d1 * d1), q1));
    if (nd == 3) m = __fadd_rn(m, __fmul_rn((float)(d2 * d2), q2));
    return m;
}

__device__ __forceinline__ int gap(int r, int lo, int hi) {   // distance of r to [lo, hi]
    return r < lo ? lo - r : (r > hi ? r - hi : 0);
}

__global__ void __launch_bounds__(kThreads) segment_kernel(const __grid_constant__ SegmentLaunch L) {
    const int img = __ldg(L.order + blockIdx.x);
    const ImageDesc& D = L.descs[img];
    const int M = D.M, nd = D.ndim, H = D.H, Wd = D.W, G = D.G;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    // q_i = 1 / tau_i^2: the square of the float width in double (exact), one division, one
    // rounding to float
    const float q0 = (float)(1.0 / ((double)D.sigma[0] * (double)D.sigma[0]));
    const float q1 = (float)(1.0 / ((double)D.sigma[1] * (double)D.sigma[1]));
    const float q2 = nd == 3 ? (float)(1.0 / ((double)D.sigma[2] * (double)D.sigma[2])) : 0.f;
    short* out = L.labels + D.gh_off;

    extern __shared__ __align__(16) int ssm[];
    int* cr = ssm;                   // M x 3 lattice sites
    int* lk = cr + 3 * M + wid * M;  // this warp's list for its current tile, ascending k

    const float* Wk = L.W + D.w_off;
    for (int k = tid; k < M; k += blockDim.x) {
        cr[k * 3] = site_round(Wk[k * nd], H);
        cr[k * 3 + 1] = site_round(Wk[k * nd + 1], Wd);
        cr[k * 3 + 2] = nd == 3 ? site_round(Wk[k * nd + 2], G) : 0;
    }
    __syncthreads();

    // every warp walks its own tiles: no block-wide barrier below
    const int tiles_v = (Wd + kSegTile - 1) / kSegTile, ntiles = tiles_v * ((H + kSegTile - 1) / kSegTile);
    for (int t = wid; t < ntiles; t += nw) {
        const int u0 = (t / tiles_v) * kSegTile, v0 = (t % tiles_v) * kSegTile;
        const int u1 = min(u0 + kSegTile, H) - 1, v1 = min(v0 + kSegTile, Wd) - 1;
        // the least farthest-point metric over the codebooks bounds the winner at every pixel
        float bound = __int_as_float(0x7f800000);
        for (int k = lane; k < M; k += 32) {
            const int r0 = cr[k * 3], r1 = cr[k * 3 + 1], r2 = cr[k * 3 + 2];
            const int a0 = max(abs(u0 - r0), abs(u1 - r0)), a1 = max(abs(v0 - r1), abs(v1 - r1));
            const int a2 = nd == 3 ? max(r2, G - 1 - r2) : 0;
            bound = fminf(bound, metric(nd, a0, a1, a2, q0, q1, q2));
        }
        for (int o = 16; o > 0; o >>= 1) bound = fminf(bound, __shfl_xor_sync(0xffffffffu, bound, o));
        // stable compaction of the codebooks whose nearest-point metric does not exceed it
        int nl = 0;
        for (int base = 0; base < M; base += 32) {
            const int k = base + lane;
            bool hit = false;
            if (k < M) hit = metric(nd, gap(cr[k * 3], u0, u1), gap(cr[k * 3 + 1], v0, v1), 0, q0, q1, q2) <= bound;
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            if (hit) lk[nl + __popc(bal & ((1u << lane) - 1u))] = k;
            nl += __popc(bal);
        }
        __syncwarp();
        // pixels: two tile rows per step (half a warp each), 32-byte label stores
        for (int r = lane >> 4; r < kSegTile; r += 2) {
            const int u = u0 + r, v = v0 + (lane & 15);
            if (u > u1) break;
            if (v > v1) continue;
            const size_t o = (size_t)u * D.pitch + v;
            float h;
            int gl = 0;
            if (nd == 3) {
                h = D.weight ? __ldg(D.weight + o) : 1.f;
                gl = (int)__ldg(reinterpret_cast<const unsigned char*>(D.data) + o);
            } else if (D.dtype == ITC_U8) {
                h = (float)__ldg(reinterpret_cast<const unsigned char*>(D.data) + o);
            } else {
                h = __ldg(reinterpret_cast<const float*>(D.data) + o);
            }
            int best = -1;
            if (h != 0.f) {
                float bd = 0.f;
                for (int l = 0; l < nl; ++l) {
                    const int k = lk[l];
                    const float m = metric(nd, u - cr[k * 3], v - cr[k * 3 + 1], gl - cr[k * 3 + 2], q0, q1, q2);
                    if (best < 0 || m < bd) {
                        best = k;
                        bd = m;
                    }
                }
            }
            out[(size_t)u * Wd + v] = (short)best;
        }
        __syncwarp();   // the list is rewritten for the warp's next tile
    }
}

}  // namespace

cudaError_t launch_segment(const SegmentLaunch& L, int B, int max_M, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    const size_t smem = (size_t)max_M * (3 + kThreads / 32) * sizeof(int);   // sites, one list per warp
    cudaError_t e = cudaFuncSetAttribute(segment_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    segment_kernel<<<(unsigned)B, kThreads, smem, s>>>(L);
    return cudaGetLastError();
}

}  // namespace itc
