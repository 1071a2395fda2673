// itc_run.cu -- the fixed-point iterations of Algorithm 1 (steps 3-11) on precomputed fields.
//
// One CTA owns one image for all of its iterations; W, the gathered field values and the
// codebook sums stay in shared memory, the fields are read from L2/HBM by gathers.  Per
// iteration:
//   gather   a_k = A(r_k), D_k = F(r_k) (- r_k a_k if absolute) + (r_k - w_k) a_k,
//            r_k = round(w_k) clamped to the lattice                  (Eq. (accupdate) data terms)
//   pairs    s_k = sum_j g(w_j - w_k),  E_k = sum_j g(w_j - w_k)(w_j - w_k)   (Eq. (origupdate))
//            one thread per k loops over every j in order (positions are broadcast from shared
//            memory), so the per-k sums need no reduction; g = exp2f(-sum_i d_i^2 c_i) with
//            log2(e) folded into c_i.
//   sums     S_XW = sum_k a_k, S_WW = sum_k s_k in double (lanes, then warps, fixed order),
//            c = S_XW / S_WW, D_cs of Eq. (1)
//   update   w_k' = w_k + step_scale (D_k - c E_k) / a_k (double), rounded to the lattice
//            unless ITC_CONTINUOUS; a_k = 0 keeps w_k.  Jacobi: every k reads the old W.
#include <math.h>

#include "itc_internal.cuh"

namespace itc {
namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float lattice_round(float x, int n) {
    float r = floorf(x + 0.5f);
    return fminf(fmaxf(r, 0.f), (float)(n - 1));
}

__device__ __forceinline__ double lattice_round_d(double x, int n) {
    double r = floor(x + 0.5);
    return fmin(fmax(r, 0.0), (double)(n - 1));
}

struct Sums {
    double sxw, sww;
    int empty;
};

// Block sums of (a, s, empty) in a fixed order: lanes, then warps.
__device__ __forceinline__ void block_sums(double a, double s, int e, double* red, Sums* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_sum_d(a);
    s = warp_sum_d(s);
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) {
        red[wid * 3] = a;
        red[wid * 3 + 1] = s;
        red[wid * 3 + 2] = (double)e;
    }
    __syncthreads();
    double x = 0, y = 0, z = 0;
    for (int w = 0; w < nw; ++w) {
        x += red[w * 3];
        y += red[w * 3 + 1];
        z += red[w * 3 + 2];
    }
    out->sxw = x;
    out->sww = y;
    out->empty = (int)z;
    __syncthreads();   // red is reused by the next call
}

__device__ void write_stats(itc_stats* st, const Sums& s, double sxx, int moved, int iters_done) {
    itc_stats r;
    r.sxw = s.sxw;
    r.sww = s.sww;
    r.sxx = sxx;
    r.c = s.sxw / s.sww;
    r.dcs = s.sxw > 0 ? log(s.sww) + log(sxx) - 2.0 * log(s.sxw) : INFINITY;
    r.empty = s.empty;
    r.moved = moved;
    r.iters_done = iters_done;
    r.status = !(s.sxw > 0) || !isfinite(r.dcs) ? ITC_ERR_NONFINITE
               : (s.empty > 0 ? ITC_WARN_EMPTY_SUPPORT : ITC_OK);
    *st = r;
}

// NPER: codebooks owned per thread (compile-time so the per-codebook state stays in registers).
template <int NPER>
__global__ void __launch_bounds__(kRunThreads, 4) run_kernel(const __grid_constant__ RunLaunch L) {
    const ImageDesc& D = L.descs ? L.descs[blockIdx.x] : L.one;
    const int M = D.M, nd = D.ndim, tid = threadIdx.x;
    extern __shared__ __align__(16) float4 sw[];   // M positions (u, v, g, 0)
    __shared__ double red[3 * (kRunThreads / 32)];
    __shared__ double s_sxx;

    if (L.sxx_single) {
        if (tid == 0) s_sxx = *L.sxx_single;
    } else if (tid < 32) {
        const long long nt = (long long)D.tiles_u * D.tiles_v * D.tiles_g;
        double v = 0;
        for (long long i = tid; i < nt; i += 32) v += L.partials[D.partial_off + i];
        v = warp_sum_d(v);
        if (tid == 0) s_sxx = v;
    }
    const float* Win = L.W_in + D.w_off;
    for (int k = tid; k < M; k += blockDim.x)
        sw[k] = make_float4(Win[k * nd], Win[k * nd + 1], nd == 3 ? Win[k * nd + 2] : 0.f, 0.f);
    __syncthreads();
    const double sxx = s_sxx;

    const float* A = L.fields + D.field_off;
    const long long plane = D.plane_floats;
    const bool snap = !(D.flags & ITC_CONTINUOUS);
    const bool stop_fixed = (D.flags & ITC_STOP_ON_FIXED) != 0;
    // g(d) = exp(-sum_i d_i^2 / (2 sigma_i^2)) = 2^(-sum_i d_i^2 c_i), c_i = log2(e) / (2 sigma_i^2)
    const float c0 = (float)(1.4426950408889634 * (double)D.inv2s2[0]);
    const float c1 = (float)(1.4426950408889634 * (double)D.inv2s2[1]);
    const float c2 = (float)(1.4426950408889634 * (double)D.inv2s2[2]);

    Sums s;
    int moved = 0, done = 0;
    bool stop = false;
    for (int t = 0;; ++t) {
        if (!L.final_eval && t == D.iters) break;
        // gather (issued first, consumed after the pair sums), then pair sums, per owned k
        float a[NPER], Dm[NPER][3], Ek[NPER][3];
        double pa = 0.0, ps = 0.0;
        int pe = 0;
#pragma unroll
        for (int q = 0; q < NPER; ++q) {
            const int k = tid + q * blockDim.x;
            if (k >= M) break;
            const float4 wk = sw[k];
            const float r0 = lattice_round(wk.x, D.H), r1 = lattice_round(wk.y, D.W);
            const float r2 = nd == 3 ? lattice_round(wk.z, D.G) : 0.f;
            const long long o = ((long long)(int)r2 * D.H + (int)r0) * D.fpitch + (int)r1;
            const float ak = __ldg(A + o);
            const float f0 = __ldg(A + plane + o), f1 = __ldg(A + 2 * plane + o);
            const float f2 = nd == 3 ? __ldg(A + 3 * plane + o) : 0.f;
            float s_ = 0.f, e0 = 0.f, e1 = 0.f, e2 = 0.f;
            for (int j = 0; j < M; ++j) {
                const float4 wj = sw[j];
                const float d0 = wj.x - wk.x, d1 = wj.y - wk.y, d2 = wj.z - wk.z;
                const float g = exp2f(-(d0 * d0 * c0 + d1 * d1 * c1 + d2 * d2 * c2));
                s_ += g;
                e0 = fmaf(g, d0, e0);
                e1 = fmaf(g, d1, e1);
                e2 = fmaf(g, d2, e2);
            }
            a[q] = ak;
            const float rr[3] = {r0, r1, r2}, ww[3] = {wk.x, wk.y, wk.z}, ff[3] = {f0, f1, f2};
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double m = (double)ff[i] - (L.absolute ? (double)rr[i] * ak : 0.0) + ((double)rr[i] - (double)ww[i]) * ak;
                Dm[q][i] = i < nd ? (float)m : 0.f;
            }
            Ek[q][0] = e0;
            Ek[q][1] = e1;
            Ek[q][2] = e2;
            pa += (double)ak;
            ps += (double)s_;
            pe += !(ak > 0.f);
        }
        block_sums(pa, ps, pe, red, &s);
        if (!L.final_eval && t == 0 && L.stats && tid == 0) write_stats(L.stats + blockIdx.x, s, sxx, 0, 0);
        if (t == D.iters || stop) break;
        // update (Jacobi: every k above read the old W; the barrier in block_sums separates them)
        const double c = s.sxw / s.sww;
        int mv = 0;
#pragma unroll
        for (int q = 0; q < NPER; ++q) {
            const int k = tid + q * blockDim.x;
            if (k >= M) break;
            if (!(a[q] > 0.f)) continue;
            float4 w = sw[k];
            float nw[3] = {w.x, w.y, w.z};
            bool kmoved = false;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (i >= nd) break;
                const int ni = i == 0 ? D.H : (i == 1 ? D.W : D.G);
                const double raw = (double)nw[i] + (double)D.step_scale * ((double)Dm[q][i] - c * (double)Ek[q][i]) / (double)a[q];
                const double nwv = snap ? lattice_round_d(raw, ni) : fmin(fmax(raw, 0.0), (double)(ni - 1));
                const float nf = (float)nwv;
                kmoved |= (nf != nw[i]);
                nw[i] = nf;
            }
            sw[k] = make_float4(nw[0], nw[1], nw[2], 0.f);
            mv += kmoved;
        }
        moved = __syncthreads_count(mv);
        ++done;
        if (stop_fixed && moved == 0) stop = true;
    }
    if (L.final_eval && L.stats && tid == 0) write_stats(L.stats + blockIdx.x, s, sxx, moved, done);
    if (!L.final_eval && L.stats && tid == 0) {
        L.stats[blockIdx.x].moved = moved;
        L.stats[blockIdx.x].iters_done = done;
    }
    float* Wout = L.W_out + D.w_off;
    for (int k = tid; k < M; k += blockDim.x) {
        const float4 w = sw[k];
        const float ww[3] = {w.x, w.y, w.z};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (i >= nd) break;
            const int ni = i == 0 ? D.H : (i == 1 ? D.W : D.G);
            Wout[k * nd + i] = ww[i];
            if (L.W_lattice) L.W_lattice[D.w_off + k * nd + i] = (int)lattice_round(ww[i], ni);
        }
    }
}

}  // namespace

cudaError_t launch_run(const RunLaunch& L, int nimg, int max_M, const int* max_dim, cudaStream_t s) {
    (void)max_dim;
    if (nimg <= 0) return cudaSuccess;
    const size_t smem = (size_t)max_M * sizeof(float4);
    const int nper = (max_M + kRunThreads - 1) / kRunThreads;
    auto k = nper <= 1 ? run_kernel<1> : nper <= 2 ? run_kernel<2> : nper <= 4 ? run_kernel<4> : run_kernel<16>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<nimg, kRunThreads, smem, s>>>(L);
    return cudaGetLastError();
}

}  // namespace itc
