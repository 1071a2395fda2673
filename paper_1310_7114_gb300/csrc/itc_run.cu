// itc_run.cu -- the fixed-point iterations of Algorithm 1 (steps 3-11) on precomputed fields.
//
// One CTA owns one image for all of its iterations; W, the gathered field values and the
// codebook sums stay in shared memory, the fields are read from L2/HBM by gathers.  Per
// iteration:
//   gather   a_k = A(r_k), D_k = F(r_k) (- r_k a_k if absolute) + (r_k - w_k) a_k,
//            r_k = round(w_k) clamped to the lattice                  (Eq. (accupdate) data terms)
//   pairs    s_k = sum_j g(w_j - w_k),  E_k = sum_j g(w_j - w_k)(w_j - w_k)   (Eq. (origupdate))
//            one warp per k, lanes stride over j, xor-shuffle reduction (fixed order)
//   sums     S_XW = sum_k a_k, S_WW = sum_k s_k in double, c = S_XW / S_WW, D_cs of Eq. (1)
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
__device__ __forceinline__ float warp_sum_f(float v) {
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

// Gather, pair sums and block sums at the current W (in shared memory).
__device__ void evaluate(const ImageDesc& D, const float* __restrict__ A, long long plane,
                         int absolute, const float* sw, float* sa, float* sD, float* ss, float* sE,
                         double* red, Sums* out) {
    const int M = D.M, nd = D.ndim, tid = threadIdx.x;
    for (int k = tid; k < M; k += blockDim.x) {
        float r[3];
        r[0] = lattice_round(sw[k * 3], D.H);
        r[1] = lattice_round(sw[k * 3 + 1], D.W);
        r[2] = nd == 3 ? lattice_round(sw[k * 3 + 2], D.G) : 0.f;
        const long long o = ((long long)(int)r[2] * D.H + (int)r[0]) * D.fpitch + (int)r[1];
        const float a = __ldg(A + o);
        sa[k] = a;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (i < nd) {
                const double f = (double)__ldg(A + (i + 1) * plane + o);
                const double m = f - (absolute ? (double)r[i] * a : 0.0) + ((double)r[i] - (double)sw[k * 3 + i]) * a;
                sD[k * 3 + i] = (float)m;
            } else {
                sD[k * 3 + i] = 0.f;
            }
        }
    }
    const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const float c0 = D.inv2s2[0], c1 = D.inv2s2[1], c2 = D.inv2s2[2];
    for (int k = wid; k < M; k += nw) {
        const float wk0 = sw[k * 3], wk1 = sw[k * 3 + 1], wk2 = sw[k * 3 + 2];
        float s = 0.f, e0 = 0.f, e1 = 0.f, e2 = 0.f;
        for (int j = lane; j < M; j += 32) {
            const float d0 = sw[j * 3] - wk0, d1 = sw[j * 3 + 1] - wk1;
            const float d2 = nd == 3 ? sw[j * 3 + 2] - wk2 : 0.f;
            const float g = expf(-(d0 * d0 * c0 + d1 * d1 * c1 + d2 * d2 * c2));
            s += g;
            e0 = fmaf(g, d0, e0);
            e1 = fmaf(g, d1, e1);
            e2 = fmaf(g, d2, e2);
        }
        s = warp_sum_f(s);
        e0 = warp_sum_f(e0);
        e1 = warp_sum_f(e1);
        e2 = warp_sum_f(e2);
        if (lane == 0) {
            ss[k] = s;
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
    out->sxw = red[0];
    out->sww = red[1];
    out->empty = (int)red[2];
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

__global__ void __launch_bounds__(kRunThreads) run_kernel(const __grid_constant__ RunLaunch L) {
    const ImageDesc& D = L.descs ? L.descs[blockIdx.x] : L.one;
    const int M = D.M, nd = D.ndim, tid = threadIdx.x;
    extern __shared__ __align__(16) float sm[];
    float* sw = sm;             // M x 3 positions
    float* sa = sw + 3 * M;     // M
    float* sD = sa + M;         // M x 3
    float* ss = sD + 3 * M;     // M
    float* sE = ss + M;         // M x 3
    __shared__ double red[4];

    // S_XX from the tile partials of this image, fixed order
    double sxx = 0;
    if (L.sxx_single) {
        sxx = *L.sxx_single;
    } else {
        const long long nt = (long long)D.tiles_u * D.tiles_v * D.tiles_g;
        if (tid < 32) {
            double v = 0;
            for (long long i = tid; i < nt; i += 32) v += L.partials[D.partial_off + i];
            v = warp_sum_d(v);
            if (tid == 0) red[3] = v;
        }
        __syncthreads();
        sxx = red[3];
    }

    const float* Win = L.W_in + D.w_off;
    for (int k = tid; k < M; k += blockDim.x) {
        for (int i = 0; i < 3; ++i) sw[k * 3 + i] = i < nd ? Win[k * nd + i] : 0.f;
    }
    __syncthreads();

    const float* A = L.fields + D.field_off;
    const long long plane = D.plane_floats;
    const bool snap = !(D.flags & ITC_CONTINUOUS);
    const bool stop_fixed = (D.flags & ITC_STOP_ON_FIXED) != 0;
    const int iters = D.iters;
    Sums s;
    int moved = 0, done = 0;
    bool stop = false;
    for (int t = 0;; ++t) {
        if (!L.final_eval && t == iters) break;
        evaluate(D, A, plane, L.absolute, sw, sa, sD, ss, sE, red, &s);
        if (!L.final_eval && t == 0 && L.stats && tid == 0) write_stats(L.stats + blockIdx.x, s, sxx, 0, 0);
        if (t == iters || stop) {
            break;
        }
        const double c = s.sxw / s.sww;
        int mv = 0;
        for (int k = tid; k < M; k += blockDim.x) {
            const float a = sa[k];
            if (!(a > 0.f)) continue;
            bool kmoved = false;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (i >= nd) break;
                const int ni = i == 0 ? D.H : (i == 1 ? D.W : D.G);
                const double w = sw[k * 3 + i];
                const double raw = w + (double)D.step_scale * ((double)sD[k * 3 + i] - c * (double)sE[k * 3 + i]) / (double)a;
                double nwv;
                if (snap) nwv = lattice_round_d(raw, ni);
                else nwv = fmin(fmax(raw, 0.0), (double)(ni - 1));
                const float nf = (float)nwv;
                kmoved |= (nf != sw[k * 3 + i]);
                sw[k * 3 + i] = nf;   // only thread k touches w_k in this phase
            }
            mv += kmoved;
        }
        moved = __syncthreads_count(mv);
        ++done;
        if (stop_fixed && moved == 0) stop = true;
        // the next pass re-reads W (evaluate syncs before the pair sums; sw writes are complete)
    }
    if (L.final_eval && L.stats && tid == 0) write_stats(L.stats + blockIdx.x, s, sxx, moved, done);
    if (!L.final_eval && L.stats && tid == 0) {
        L.stats[blockIdx.x].moved = moved;
        L.stats[blockIdx.x].iters_done = done;
    }
    float* Wout = L.W_out + D.w_off;
    for (int k = tid; k < M; k += blockDim.x) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (i >= nd) break;
            const int ni = i == 0 ? D.H : (i == 1 ? D.W : D.G);
            Wout[k * nd + i] = sw[k * 3 + i];
            if (L.W_lattice) L.W_lattice[D.w_off + k * nd + i] = (int)lattice_round(sw[k * 3 + i], ni);
        }
    }
}

}  // namespace

cudaError_t launch_run(const RunLaunch& L, int nimg, int max_M, int iters_cap, cudaStream_t s) {
    (void)iters_cap;
    if (nimg <= 0) return cudaSuccess;
    const size_t smem = (size_t)max_M * kCodebookSmemFloats * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(run_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    run_kernel<<<nimg, kRunThreads, smem, s>>>(L);
    return cudaGetLastError();
}

}  // namespace itc
