/*
 * itc_oracle.c -- FP64 CPU oracle for lattice information-theoretic clustering
 * (C. Bauckhage, K. Kersting, "Efficient Information Theoretic Clustering on Discrete
 * Lattices", arXiv:1310.7114).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct statement of what
 * the CUDA library computes.  Only the test suite, the package smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header, table or constant with the CUDA
 * path, and the product path never calls it.
 *
 * Notation (Sec. 2.1, Sec. 3.1):
 *   lattice sites x with weights h(x) >= 0 (binary image: h = X in {0,1}, Sec. 3.2; weighted
 *   image: h, Sec. 5; gray image: one voxel (u, v, gray(u,v)) per pixel with weight h(u,v),
 *   Sec. 1 case (ii));  codebook W = {w_1..w_M}.
 *   Kernel g(d) = prod_i exp(-d_i^2 / (2 sigma_i^2)), unnormalised.
 *
 * Kernel widths (the paper has xi, omega, tau, rho, Sec. 2.1).  By the Gaussian product theorem
 * the three overlap integrals of Eq. (1) are Gaussian sums of three widths:
 *     V(X;W) ~ S_XW = sum_k sum_x h(x) g_tau(x - w_k),      tau^2 = xi^2 + omega^2
 *     V(W)   ~ S_WW = sum_j sum_k g_rho(w_j - w_k),         rho^2 = 2 omega^2
 *     V(X)   ~ S_XX = sum_x sum_y h(x) h(y) g_s(x - y),     s^2   = 2 xi^2
 * and D_cs = log S_WW + log S_XX - 2 log S_XW + K with K = 1/2 sum_i log(tau_i^4 / (rho_i^2 s_i^2))
 * collecting the normalisers (K = 0 when xi = omega, the default reading: one width sigma =
 * tau = rho = s).  Functions take sigma (= tau) and optional rho and s (NULL = sigma).
 * Truncation (Sec. 3.1, finite filter masks): data sums run over the box |x_i - r_i| <= R_i
 * around the lattice site r they are centred on, R_i = ceil(trunc * sigma_i); the codebook
 * interaction sums S_WW, s_k, E_k are not truncated.  Sites outside the lattice hold no data.
 *
 * Parity status of every function is given in its comment; all of them are pinned by the
 * not-gpu tests (brute force, library convolutions, closed forms, the mean-shift special case,
 * numerical overlap integrals, finite differences).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- kernel and truncation */

/* One axis of the Gaussian, exp(-d^2 / (2 s^2)).  Sec. 2.1 Eq. (dens1)/(dens2). */
static double gauss1(double d, double s) { return exp(-(d * d) / (2.0 * s * s)); }

/* Truncation radius of the finite filter mask, Sec. 3.1: R = ceil(trunc * sigma). */
int orc_radius(double sigma, double trunc)
{
    return (int)ceil(trunc * sigma);
}

/* Lattice rounding used for codebook vectors on the grid (Sec. 3.2, Fig. 2 text):
 * floor(x + 0.5), clamped to [0, n-1]. */
static double lattice_round(double x, int n)
{
    double r = floor(x + 0.5);
    if (r < 0) r = 0;
    if (r > n - 1) r = n - 1;
    return r;
}

/* -------------------------------------------------------------- 2-D fields (Sec. 3.1) */
/*
 * The data density p = h * G (Sec. 3.1, Sec. 5) and its first moments, sampled on the lattice
 * and truncated to the box |x - y|_inf <= R:
 *   A(y)   = sum_x h(x) g(x - y)
 *   F_i(y) = sum_x h(x) g(x - y) (x_i - y_i)   (centred moments, absolute == 0)
 *   F_i(y) = sum_x h(x) g(x - y) x_i           (coordinate-weighted images u.X, v.X, absolute == 1)
 * Layout: h, A, Fu, Fv are H x W row-major (u = row, v = column).
 */

/* Direct windowed sum over the (2R+1)^2 box around every site.  Definition, written out. */
void orc_fields2d_direct(const double *h, int H, int W, double su, double sv, int Ru, int Rv,
                         int absolute, double *A, double *Fu, double *Fv)
{
    for (int yu = 0; yu < H; ++yu)
        for (int yv = 0; yv < W; ++yv) {
            double a = 0, fu = 0, fv = 0;
            for (int xu = yu - Ru; xu <= yu + Ru; ++xu) {
                if (xu < 0 || xu >= H) continue;
                for (int xv = yv - Rv; xv <= yv + Rv; ++xv) {
                    if (xv < 0 || xv >= W) continue;
                    double hx = h[(size_t)xu * W + xv];
                    if (hx == 0) continue;
                    double k = hx * gauss1(xu - yu, su) * gauss1(xv - yv, sv);
                    a += k;
                    fu += k * (absolute ? xu : (xu - yu));
                    fv += k * (absolute ? xv : (xv - yv));
                }
            }
            A[(size_t)yu * W + yv] = a;
            Fu[(size_t)yu * W + yv] = fu;
            Fv[(size_t)yu * W + yv] = fv;
        }
}

/* The same fields at a list of sites only (sites[2*s] = u, sites[2*s+1] = v). */
void orc_fields2d_sites(const double *h, int H, int W, double su, double sv, int Ru, int Rv,
                        int absolute, int nsites, const int *sites, double *A, double *Fu, double *Fv)
{
    for (int s = 0; s < nsites; ++s) {
        int yu = sites[2 * s], yv = sites[2 * s + 1];
        double a = 0, fu = 0, fv = 0;
        for (int xu = yu - Ru; xu <= yu + Ru; ++xu) {
            if (xu < 0 || xu >= H) continue;
            for (int xv = yv - Rv; xv <= yv + Rv; ++xv) {
                if (xv < 0 || xv >= W) continue;
                double hx = h[(size_t)xu * W + xv];
                if (hx == 0) continue;
                double k = hx * gauss1(xu - yu, su) * gauss1(xv - yv, sv);
                a += k;
                fu += k * (absolute ? xu : (xu - yu));
                fv += k * (absolute ? xv : (xv - yv));
            }
        }
        A[s] = a;
        Fu[s] = fu;
        Fv[s] = fv;
    }
}

/* Separable evaluation: a 1-D pass along v then a 1-D pass along u (Sec. 3.1, "two 1D
 * convolution kernels").  Independent second implementation of orc_fields2d_direct. */
void orc_fields2d_separable(const double *h, int H, int W, double su, double sv, int Ru, int Rv,
                            int absolute, double *A, double *Fu, double *Fv)
{
    double *T = (double *)calloc((size_t)H * W, sizeof(double));
    double *Tv = (double *)calloc((size_t)H * W, sizeof(double));
    /* pass along v: T(x_u, y_v) = sum_dv g(dv) h(x_u, y_v+dv), Tv with the v moment */
    for (int xu = 0; xu < H; ++xu)
        for (int yv = 0; yv < W; ++yv) {
            double t = 0, tv = 0;
            for (int dv = -Rv; dv <= Rv; ++dv) {
                int xv = yv + dv;
                if (xv < 0 || xv >= W) continue;
                double k = gauss1(dv, sv) * h[(size_t)xu * W + xv];
                t += k;
                tv += k * (absolute ? xv : dv);
            }
            T[(size_t)xu * W + yv] = t;
            Tv[(size_t)xu * W + yv] = tv;
        }
    /* pass along u */
    for (int yu = 0; yu < H; ++yu)
        for (int yv = 0; yv < W; ++yv) {
            double a = 0, fu = 0, fv = 0;
            for (int du = -Ru; du <= Ru; ++du) {
                int xu = yu + du;
                if (xu < 0 || xu >= H) continue;
                double k = gauss1(du, su);
                a += k * T[(size_t)xu * W + yv];
                fu += k * (absolute ? xu : du) * T[(size_t)xu * W + yv];
                fv += k * Tv[(size_t)xu * W + yv];
            }
            A[(size_t)yu * W + yv] = a;
            Fu[(size_t)yu * W + yv] = fu;
            Fv[(size_t)yu * W + yv] = fv;
        }
    free(T);
    free(Tv);
}

/* S_XX = sum_x h(x) A(x): the V(X) term of Eq. (1) on the truncated lattice. */
double orc_sxx(const double *h, const double *A, size_t n)
{
    double s = 0;
    for (size_t i = 0; i < n; ++i) s += h[i] * A[i];
    return s;
}

/* -------------------------------------------------- 3-D gray-value lattice (Sec. 1 (ii)) */
/*
 * A gray image is the occupancy volume X(u, v, g) = [gray(u,v) == g] on the [u, v, g] lattice,
 * G gray levels; pixel (u,v) carries weight h(u,v) (NULL means 1).  Fields are 4 volumes
 * A, F_u, F_v, F_g laid out [g][u][v].
 */
void orc_fields3d_direct(const int *gray, const double *hw, int H, int W, int G,
                         const double *sigma, const int *R, int absolute,
                         double *A, double *Fu, double *Fv, double *Fg)
{
    for (int yg = 0; yg < G; ++yg)
        for (int yu = 0; yu < H; ++yu)
            for (int yv = 0; yv < W; ++yv) {
                double a = 0, fu = 0, fv = 0, fg = 0;
                for (int xu = yu - R[0]; xu <= yu + R[0]; ++xu) {
                    if (xu < 0 || xu >= H) continue;
                    for (int xv = yv - R[1]; xv <= yv + R[1]; ++xv) {
                        if (xv < 0 || xv >= W) continue;
                        size_t p = (size_t)xu * W + xv;
                        int xg = gray[p];
                        if (xg - yg > R[2] || yg - xg > R[2]) continue;
                        double hx = hw ? hw[p] : 1.0;
                        if (hx == 0) continue;
                        double k = hx * gauss1(xu - yu, sigma[0]) * gauss1(xv - yv, sigma[1]) *
                                   gauss1(xg - yg, sigma[2]);
                        a += k;
                        fu += k * (absolute ? xu : (xu - yu));
                        fv += k * (absolute ? xv : (xv - yv));
                        fg += k * (absolute ? xg : (xg - yg));
                    }
                }
                size_t o = ((size_t)yg * H + yu) * W + yv;
                A[o] = a;
                Fu[o] = fu;
                Fv[o] = fv;
                Fg[o] = fg;
            }
}

/* Fields of the 3-D lattice at listed sites (sites[3*s..] = u, v, g). */
void orc_fields3d_sites(const int *gray, const double *hw, int H, int W, int G,
                        const double *sigma, const int *R, int absolute, int nsites,
                        const int *sites, double *A, double *Fu, double *Fv, double *Fg)
{
    (void)G;
    for (int s = 0; s < nsites; ++s) {
        int yu = sites[3 * s], yv = sites[3 * s + 1], yg = sites[3 * s + 2];
        double a = 0, fu = 0, fv = 0, fg = 0;
        for (int xu = yu - R[0]; xu <= yu + R[0]; ++xu) {
            if (xu < 0 || xu >= H) continue;
            for (int xv = yv - R[1]; xv <= yv + R[1]; ++xv) {
                if (xv < 0 || xv >= W) continue;
                size_t p = (size_t)xu * W + xv;
                int xg = gray[p];
                if (xg - yg > R[2] || yg - xg > R[2]) continue;
                double hx = hw ? hw[p] : 1.0;
                if (hx == 0) continue;
                double k = hx * gauss1(xu - yu, sigma[0]) * gauss1(xv - yv, sigma[1]) *
                           gauss1(xg - yg, sigma[2]);
                a += k;
                fu += k * (absolute ? xu : (xu - yu));
                fv += k * (absolute ? xv : (xv - yv));
                fg += k * (absolute ? xg : (xg - yg));
            }
        }
        A[s] = a;
        Fu[s] = fu;
        Fv[s] = fv;
        Fg[s] = fg;
    }
}

/* Separable 3-D evaluation: the pass along g is read off the gray value (each pixel occupies
 * exactly one voxel of its column), then the v and u passes run per g-slice. */
void orc_fields3d_separable(const int *gray, const double *hw, int H, int W, int G,
                            const double *sigma, const int *R, int absolute,
                            double *A, double *Fu, double *Fv, double *Fg)
{
    size_t n = (size_t)H * W;
    double *S = (double *)malloc(n * sizeof(double));
    double *Sg = (double *)malloc(n * sizeof(double));
    double *T = (double *)malloc(n * sizeof(double));
    double *Tv = (double *)malloc(n * sizeof(double));
    double *Tg = (double *)malloc(n * sizeof(double));
    for (int yg = 0; yg < G; ++yg) {
        for (size_t p = 0; p < n; ++p) {
            int dg = gray[p] - yg;
            double hx = hw ? hw[p] : 1.0;
            double k = (dg > R[2] || -dg > R[2]) ? 0.0 : hx * gauss1(dg, sigma[2]);
            S[p] = k;
            Sg[p] = k * (absolute ? gray[p] : dg);
        }
        for (int xu = 0; xu < H; ++xu)
            for (int yv = 0; yv < W; ++yv) {
                double t = 0, tv = 0, tg = 0;
                for (int dv = -R[1]; dv <= R[1]; ++dv) {
                    int xv = yv + dv;
                    if (xv < 0 || xv >= W) continue;
                    double k = gauss1(dv, sigma[1]);
                    size_t p = (size_t)xu * W + xv;
                    t += k * S[p];
                    tv += k * (absolute ? xv : dv) * S[p];
                    tg += k * Sg[p];
                }
                T[(size_t)xu * W + yv] = t;
                Tv[(size_t)xu * W + yv] = tv;
                Tg[(size_t)xu * W + yv] = tg;
            }
        for (int yu = 0; yu < H; ++yu)
            for (int yv = 0; yv < W; ++yv) {
                double a = 0, fu = 0, fv = 0, fg = 0;
                for (int du = -R[0]; du <= R[0]; ++du) {
                    int xu = yu + du;
                    if (xu < 0 || xu >= H) continue;
                    double k = gauss1(du, sigma[0]);
                    size_t p = (size_t)xu * W + yv;
                    a += k * T[p];
                    fu += k * (absolute ? xu : du) * T[p];
                    fv += k * Tv[p];
                    fg += k * Tg[p];
                }
                size_t o = ((size_t)yg * H + yu) * W + yv;
                A[o] = a;
                Fu[o] = fu;
                Fv[o] = fv;
                Fg[o] = fg;
            }
    }
    free(S);
    free(Sg);
    free(T);
    free(Tv);
    free(Tg);
}

/* ------------------------------------------------ fixed-point update (Sec. 2.1, Sec. 3.1) */
/*
 * One lattice ITC iteration, Algorithm 1 steps 4-9 with the data integrals of Eq. (accupdate)
 * read from the precomputed fields and the codebook integrals written as the M x M interaction
 * sums of Eq. (origupdate):
 *   r_k  = lattice_round(w_k)                      (the filter mask is centred on the grid)
 *   a_k  = A(r_k)                                  (sum_x h g(x - w_k): denominator)
 *   D_k  = F(r_k) [- r_k a_k if absolute] + (r_k - w_k) a_k
 *                                                  (sum_x h g(x - w_k)(x - w_k))
 *   s_k  = sum_j g(w_j - w_k),  E_k = sum_j g(w_j - w_k)(w_j - w_k)
 *   c    = S_XW / S_WW = sum_k a_k / sum_k s_k     (the constant c of Eq. (origupdate))
 *   w_k' = w_k + step_scale (D_k - c E_k) / a_k
 * With step_scale = 1 this is Eq. (origupdate) term by term: its first term is (D_k + w_k a_k)/a_k,
 * its second and third terms combine to -c E_k / a_k.  All codebooks are updated from the same
 * old W (Algorithm 1 step 10 replaces W as a whole).  A codebook whose window holds no data
 * (a_k = 0) keeps its position and is counted.  snap != 0 keeps W on the lattice:
 * w_k' = lattice_round(w_k').  Otherwise w_k' is only clamped to [0, n_i - 1].
 *
 * ndim 2: shape = {H, W}, fields [u][v]; ndim 3: shape = {H, W, G}, fields [g][u][v];
 * F holds ndim pointers.  W_in / W_out / W_raw are M x ndim (u, v[, g]).
 * stats[0..4] = c, S_XW, S_WW, number of empty-support codebooks, number of moved codebooks.
 */
static size_t site_index(int ndim, const int *shape, const double *r)
{
    if (ndim == 2) return (size_t)r[0] * shape[1] + (size_t)r[1];
    return ((size_t)r[2] * shape[0] + (size_t)r[0]) * shape[1] + (size_t)r[1];
}

void orc_lattice_step(int ndim, const int *shape, const double *A, const double *const *F,
                      int absolute, const double *sigma, const double *rho, int M, const double *W_in,
                      double step_scale, int snap, double *W_out, double *W_raw, double *stats)
{
    if (!rho) rho = sigma;
    /* the stationarity condition of Eq. (1) in w_k: D_k / tau^2 = c E_k / rho^2 per axis, so the
       pair term carries kappa = tau^2 / rho^2 (1 when tau = rho) */
    double kappa[3];
    for (int i = 0; i < ndim; ++i) kappa[i] = (sigma[i] * sigma[i]) / (rho[i] * rho[i]);
    double *a = (double *)malloc(M * sizeof(double));
    double *D = (double *)malloc((size_t)M * ndim * sizeof(double));
    double *s = (double *)malloc(M * sizeof(double));
    double *E = (double *)malloc((size_t)M * ndim * sizeof(double));
    double sxw = 0, sww = 0;
    for (int k = 0; k < M; ++k) {
        double r[3];
        for (int i = 0; i < ndim; ++i) r[i] = lattice_round(W_in[k * ndim + i], shape[i]);
        size_t o = site_index(ndim, shape, r);
        a[k] = A[o];
        for (int i = 0; i < ndim; ++i)
            D[k * ndim + i] = F[i][o] - (absolute ? r[i] * a[k] : 0.0) +
                              (r[i] - W_in[k * ndim + i]) * a[k];
        s[k] = 0;
        for (int i = 0; i < ndim; ++i) E[k * ndim + i] = 0;
        for (int j = 0; j < M; ++j) {
            double gk = 1.0;
            for (int i = 0; i < ndim; ++i)
                gk *= gauss1(W_in[j * ndim + i] - W_in[k * ndim + i], rho[i]);
            s[k] += gk;
            for (int i = 0; i < ndim; ++i)
                E[k * ndim + i] += gk * (W_in[j * ndim + i] - W_in[k * ndim + i]);
        }
        sxw += a[k];
        sww += s[k];
    }
    double c = sxw / sww;
    int empty = 0, moved = 0;
    for (int k = 0; k < M; ++k) {
        int mv = 0;
        for (int i = 0; i < ndim; ++i) {
            double w = W_in[k * ndim + i], nw;
            if (a[k] > 0) {
                double raw = w + step_scale * (D[k * ndim + i] - kappa[i] * c * E[k * ndim + i]) / a[k];
                W_raw[k * ndim + i] = raw;
                if (snap) nw = lattice_round(raw, shape[i]);
                else nw = raw < 0 ? 0 : (raw > shape[i] - 1 ? shape[i] - 1 : raw);
            } else {
                W_raw[k * ndim + i] = w;
                nw = w;
            }
            if (nw != w) mv = 1;
            W_out[k * ndim + i] = nw;
        }
        if (!(a[k] > 0)) ++empty;
        moved += mv;
    }
    stats[0] = c;
    stats[1] = sxw;
    stats[2] = sww;
    stats[3] = empty;
    stats[4] = moved;
    free(a);
    free(D);
    free(s);
    free(E);
}

/* Algorithm 1 loop: iterate orc_lattice_step `iters` times (steps 3-11); with stop_on_fixed
 * the loop ends when an iteration moves no codebook (the theta = 0 test of step 11).
 * dcs[t] = D_cs at the W entering iteration t, for t < iters_done, and dcs[iters_done] at the
 * returned W.  tie[t] = distance of the closest unrounded coordinate of iteration t to a
 * half-integer (snap mode).  Returns the number of iterations run. */
int orc_lattice_run(int ndim, const int *shape, const double *A, const double *const *F,
                    int absolute, double sxx, const double *sigma, const double *rho, double dcs_const,
                    int M, double *W, double step_scale, int snap, int iters, int stop_on_fixed,
                    double *dcs, double *tie)
{
    double *Wn = (double *)malloc((size_t)M * ndim * sizeof(double));
    double *raw = (double *)malloc((size_t)M * ndim * sizeof(double));
    double st[5];
    int t = 0;
    for (; t < iters; ++t) {
        orc_lattice_step(ndim, shape, A, F, absolute, sigma, rho, M, W, step_scale, snap, Wn, raw, st);
        if (dcs) dcs[t] = log(st[2]) + log(sxx) - 2.0 * log(st[1]) + dcs_const;
        if (tie) {
            double m = 1e300;
            for (int i = 0; i < M * ndim; ++i) {
                double f = raw[i] - floor(raw[i]);
                double d = fabs(f - 0.5);
                if (d < m) m = d;
            }
            tie[t] = m;
        }
        memcpy(W, Wn, (size_t)M * ndim * sizeof(double));
        if (stop_on_fixed && st[4] == 0) { ++t; break; }
    }
    if (dcs) {
        orc_lattice_step(ndim, shape, A, F, absolute, sigma, rho, M, W, step_scale, snap, Wn, raw, st);
        dcs[t] = log(st[2]) + log(sxx) - 2.0 * log(st[1]) + dcs_const;
    }
    free(Wn);
    free(raw);
    return t;
}

/* ------------------------------------------------ original ITC (Sec. 2.1, Eq. (origupdate)) */
/*
 * Continuous, untruncated update over an explicit point list X (N x ndim) with weights hx
 * (NULL = 1), evaluated as the three terms of Eq. (origupdate):
 *   w_k' = sum_i g(x_i - w_k) x_i / den_k - c sum_j g(w_j - w_k) w_j / den_k
 *          + c sum_j g(w_j - w_k) w_k / den_k,   den_k = sum_i g(x_i - w_k)
 * with the data sums over g_tau (sigma) and the codebook sums over g_rho (rho; NULL = sigma).
 * Written out with normalised Gaussians, c = (N/M) V(X;W)/V(W) times the ratio of the
 * normalisers of the two sums is S_XW / S_WW.  As printed, Eq. (origupdate) has no further
 * factor (kappa_from_widths = 0); differentiating Eq. (1) gives the pair terms an extra
 * tau^2/rho^2 per axis (kappa_from_widths = 1).  The two agree when tau = rho.
 * Cost O(N M) exponentials per iteration (Sec. 2.2).
 */
void orc_original_step(int ndim, int N, const double *X, const double *hx, const double *sigma,
                       const double *rho, int kappa_from_widths, int M, const double *W_in,
                       double *W_out)
{
    if (!rho) rho = sigma;
    double *den = (double *)malloc(M * sizeof(double));
    double *num = (double *)malloc((size_t)M * ndim * sizeof(double));
    double *s = (double *)malloc(M * sizeof(double));
    double *mw = (double *)malloc((size_t)M * ndim * sizeof(double));
    double sxw = 0, sww = 0;
    for (int k = 0; k < M; ++k) {
        den[k] = 0;
        for (int i = 0; i < ndim; ++i) num[k * ndim + i] = 0;
        for (int p = 0; p < N; ++p) {
            double gk = hx ? hx[p] : 1.0;
            for (int i = 0; i < ndim; ++i) gk *= gauss1(X[p * ndim + i] - W_in[k * ndim + i], sigma[i]);
            den[k] += gk;
            for (int i = 0; i < ndim; ++i) num[k * ndim + i] += gk * X[p * ndim + i];
        }
        s[k] = 0;
        for (int i = 0; i < ndim; ++i) mw[k * ndim + i] = 0;
        for (int j = 0; j < M; ++j) {
            double gk = 1.0;
            for (int i = 0; i < ndim; ++i) gk *= gauss1(W_in[j * ndim + i] - W_in[k * ndim + i], rho[i]);
            s[k] += gk;
            for (int i = 0; i < ndim; ++i) mw[k * ndim + i] += gk * W_in[j * ndim + i];
        }
        sxw += den[k];
        sww += s[k];
    }
    double c = sxw / sww;
    for (int k = 0; k < M; ++k)
        for (int i = 0; i < ndim; ++i) {
            const double ck = kappa_from_widths ? c * (sigma[i] * sigma[i]) / (rho[i] * rho[i]) : c;
            W_out[k * ndim + i] = num[k * ndim + i] / den[k] - ck * mw[k * ndim + i] / den[k] +
                                  ck * s[k] / den[k] * W_in[k * ndim + i];
        }
    free(den);
    free(num);
    free(s);
    free(mw);
}

/* ------------------------------------------------ divergence and its gradient (Eq. (1)) */
/*
 * Lattice data enters as a point list: N sites X (N x ndim, integer coordinates) with weights
 * hx, and per-axis lattice sizes `shape` (used to round w_k onto the grid).  Truncated data
 * sums use the box |x - lattice_round(w_k)|_inf <= R around each codebook's grid site and the
 * box |x - y|_inf <= R for S_XX; the kernel itself is evaluated at the real w_k, so D_cs is a
 * smooth function of w inside each lattice cell.
 */
static int in_box(int ndim, const double *x, const double *c, const int *R)
{
    for (int i = 0; i < ndim; ++i)
        if (fabs(x[i] - c[i]) > R[i]) return 0;
    return 1;
}

/* sums[0..2] = S_XW, S_WW, S_XX, evaluated directly from their definitions: S_XW with g_sigma
 * over the box R, S_WW with g_rho (untruncated), S_XX with g_s over the box Rs (rho, s, Rs may
 * be NULL: sigma, sigma, R). */
void orc_dcs_sums(int ndim, const int *shape, int N, const double *X, const double *hx,
                  const double *sigma, const int *R, const double *rho, const double *ss,
                  const int *Rs, int M, const double *W, double *sums)
{
    if (!rho) rho = sigma;
    if (!ss) ss = sigma;
    if (!Rs) Rs = R;
    double sxw = 0, sww = 0, sxx = 0;
    for (int k = 0; k < M; ++k) {
        double r[3];
        for (int i = 0; i < ndim; ++i) r[i] = lattice_round(W[k * ndim + i], shape[i]);
        for (int p = 0; p < N; ++p) {
            if (!in_box(ndim, X + (size_t)p * ndim, r, R)) continue;
            double gk = hx[p];
            for (int i = 0; i < ndim; ++i) gk *= gauss1(X[(size_t)p * ndim + i] - W[k * ndim + i], sigma[i]);
            sxw += gk;
        }
        for (int j = 0; j < M; ++j) {
            double gk = 1.0;
            for (int i = 0; i < ndim; ++i) gk *= gauss1(W[j * ndim + i] - W[k * ndim + i], rho[i]);
            sww += gk;
        }
    }
    for (int p = 0; p < N; ++p)
        for (int q = 0; q < N; ++q) {
            if (!in_box(ndim, X + (size_t)p * ndim, X + (size_t)q * ndim, Rs)) continue;
            double gk = hx[p] * hx[q];
            for (int i = 0; i < ndim; ++i)
                gk *= gauss1(X[(size_t)p * ndim + i] - X[(size_t)q * ndim + i], ss[i]);
            sxx += gk;
        }
    sums[0] = sxw;
    sums[1] = sww;
    sums[2] = sxx;
}

/* The normalisers of Eq. (1): K = log(n_rho n_s / n_tau^2) for the normalised Gaussians
 * n_t = prod_i (2 pi t_i^2)^(-1/2), i.e. 1/2 sum_i log(tau_i^4 / (rho_i^2 s_i^2)). */
double orc_dcs_const(int ndim, const double *sigma, const double *rho, const double *ss)
{
    if (!rho) rho = sigma;
    if (!ss) ss = sigma;
    double k = 0;
    for (int i = 0; i < ndim; ++i)
        k += 0.5 * log(pow(sigma[i], 4) / (rho[i] * rho[i] * ss[i] * ss[i]));
    return k;
}

/* D_cs = 2H(X;W) - H(W) - H(X) = log S_WW + log S_XX - 2 log S_XW + K, Eq. (1). */
double orc_dcs(int ndim, const int *shape, int N, const double *X, const double *hx,
               const double *sigma, const int *R, const double *rho, const double *ss, const int *Rs,
               int M, const double *W)
{
    double s[3];
    orc_dcs_sums(ndim, shape, N, X, hx, sigma, R, rho, ss, Rs, M, W, s);
    return log(s[1]) + log(s[2]) - 2.0 * log(s[0]) + orc_dcs_const(ndim, sigma, rho, ss);
}

/*
 * Analytic gradient of orc_dcs (Eq. (1) differentiated; dq/dw_k of Sec. 3.1 with the sign and
 * factor of d/dw exp(-|x-w|^2/(2 s^2)) = exp(.) (x - w)/s^2):
 *   dD/dw_{k,i} = (2/rho_i^2) E_{k,i}/S_WW - (2/tau_i^2) D_{k,i}/S_XW,
 *        D_k = sum_{x in box(r_k)} h g_tau(x - w_k)(x - w_k),  E_k = sum_j g_rho(w_j - w_k)(w_j - w_k)
 *   dD/dh(x)    = 2 A_s(x)/S_XX - (2/S_XW) sum_k g_tau(x - w_k) [x in box(r_k)],
 *        A_s(x) = sum_{y in box_s(x)} h(y) g_s(x - y).
 * (tau = sigma; rho, s, Rs NULL = sigma, sigma, R.)  gW is M x ndim; gh has one entry per point.
 */
void orc_dcs_grad(int ndim, const int *shape, int N, const double *X, const double *hx,
                  const double *sigma, const int *R, const double *rho, const double *ss,
                  const int *Rs, int M, const double *W, double *gW, double *gh)
{
    if (!rho) rho = sigma;
    if (!ss) ss = sigma;
    if (!Rs) Rs = R;
    double sums[3];
    orc_dcs_sums(ndim, shape, N, X, hx, sigma, R, rho, ss, Rs, M, W, sums);
    double sxw = sums[0], sww = sums[1], sxx = sums[2];
    for (int k = 0; k < M; ++k) {
        double r[3], D[3] = {0, 0, 0}, E[3] = {0, 0, 0};
        for (int i = 0; i < ndim; ++i) r[i] = lattice_round(W[k * ndim + i], shape[i]);
        for (int p = 0; p < N; ++p) {
            if (!in_box(ndim, X + (size_t)p * ndim, r, R)) continue;
            double gk = hx[p];
            for (int i = 0; i < ndim; ++i) gk *= gauss1(X[(size_t)p * ndim + i] - W[k * ndim + i], sigma[i]);
            for (int i = 0; i < ndim; ++i) D[i] += gk * (X[(size_t)p * ndim + i] - W[k * ndim + i]);
        }
        for (int j = 0; j < M; ++j) {
            double gk = 1.0;
            for (int i = 0; i < ndim; ++i) gk *= gauss1(W[j * ndim + i] - W[k * ndim + i], rho[i]);
            for (int i = 0; i < ndim; ++i) E[i] += gk * (W[j * ndim + i] - W[k * ndim + i]);
        }
        for (int i = 0; i < ndim; ++i)
            gW[k * ndim + i] = 2.0 / (rho[i] * rho[i]) * E[i] / sww - 2.0 / (sigma[i] * sigma[i]) * D[i] / sxw;
    }
    if (!gh) return;
    for (int p = 0; p < N; ++p) {
        const double *x = X + (size_t)p * ndim;
        double a = 0, st = 0;
        for (int q = 0; q < N; ++q) {
            if (!in_box(ndim, x, X + (size_t)q * ndim, Rs)) continue;
            double gk = hx[q];
            for (int i = 0; i < ndim; ++i) gk *= gauss1(x[i] - X[(size_t)q * ndim + i], ss[i]);
            a += gk;
        }
        for (int k = 0; k < M; ++k) {
            double r[3];
            for (int i = 0; i < ndim; ++i) r[i] = lattice_round(W[k * ndim + i], shape[i]);
            if (!in_box(ndim, x, r, R)) continue;
            double gk = 1.0;
            for (int i = 0; i < ndim; ++i) gk *= gauss1(x[i] - W[k * ndim + i], sigma[i]);
            st += gk;
        }
        gh[p] = 2.0 * a / sxx - 2.0 / sxw * st;
    }
}

/*
 * Gradient on a dense lattice image, evaluated from precomputed oracle fields (for sizes where
 * the O(N^2) point-list form is too slow).  ndim 2 only.  A is the field of h (same layout),
 * sxx = sum h A.  gh (H x W) gets dD/dh at every site, gW (M x 2) dD/dw at lattice W.  The
 * window sums at w_k are taken directly from h.
 */
void orc_dcs_grad2d_dense(const double *h, const double *A, int H, int W, double su, double sv,
                          int Ru, int Rv, double pu, double pv, double sxx, int M, const double *Wc,
                          double *gW, double *gh, double *sums_out)
{
    /* (su, sv) = tau, (pu, pv) = rho of the pair sums; A is the field of h at the width of
       S_XX, so that sxx = sum h A */
    double sxw = 0, sww = 0;
    double *D = (double *)malloc((size_t)M * 2 * sizeof(double));
    double *E = (double *)malloc((size_t)M * 2 * sizeof(double));
    for (int k = 0; k < M; ++k) {
        double wu = Wc[2 * k], wv = Wc[2 * k + 1];
        int ru = (int)lattice_round(wu, H), rv = (int)lattice_round(wv, W);
        double a = 0, du = 0, dv = 0;
        for (int xu = ru - Ru; xu <= ru + Ru; ++xu) {
            if (xu < 0 || xu >= H) continue;
            for (int xv = rv - Rv; xv <= rv + Rv; ++xv) {
                if (xv < 0 || xv >= W) continue;
                double gk = h[(size_t)xu * W + xv] * gauss1(xu - wu, su) * gauss1(xv - wv, sv);
                a += gk;
                du += gk * (xu - wu);
                dv += gk * (xv - wv);
            }
        }
        sxw += a;
        D[2 * k] = du;
        D[2 * k + 1] = dv;
        double eu = 0, ev = 0;
        for (int j = 0; j < M; ++j) {
            double gk = gauss1(Wc[2 * j] - wu, pu) * gauss1(Wc[2 * j + 1] - wv, pv);
            sww += gk;
            eu += gk * (Wc[2 * j] - wu);
            ev += gk * (Wc[2 * j + 1] - wv);
        }
        E[2 * k] = eu;
        E[2 * k + 1] = ev;
    }
    for (int k = 0; k < M; ++k) {
        gW[2 * k] = 2.0 / (pu * pu) * E[2 * k] / sww - 2.0 / (su * su) * D[2 * k] / sxw;
        gW[2 * k + 1] = 2.0 / (pv * pv) * E[2 * k + 1] / sww - 2.0 / (sv * sv) * D[2 * k + 1] / sxw;
    }
    if (gh) {
        for (int u = 0; u < H; ++u)
            for (int v = 0; v < W; ++v) {
                double st = 0;
                for (int k = 0; k < M; ++k) {
                    double wu = Wc[2 * k], wv = Wc[2 * k + 1];
                    double ru = lattice_round(wu, H), rv = lattice_round(wv, W);
                    if (fabs(u - ru) > Ru || fabs(v - rv) > Rv) continue;
                    st += gauss1(u - wu, su) * gauss1(v - wv, sv);
                }
                gh[(size_t)u * W + v] = 2.0 * A[(size_t)u * W + v] / sxx - 2.0 / sxw * st;
            }
    }
    if (sums_out) {
        sums_out[0] = sxw;
        sums_out[1] = sww;
        sums_out[2] = sxx;
    }
    free(D);
    free(E);
}

/* ------------------------------------------------------------- segmentation (Figs. 3 and 6) */
/*
 * The segments of Figs. 3 and 6 assign every pixel of the shape to one codebook vector; the
 * paper does not state the rule.  Reading: the codebook vector of largest kernel value
 * g_tau(x - r_k) at the pixel, i.e. the smallest
 *     D_k(x) = sum_i d_i^2 q_i,   d_i = x_i - r_{k,i},  r_k = lattice_round(w_k),  q_i = 1/tau_i^2,
 * evaluated in single precision exactly as written: each d_i^2 q_i rounded to float, the terms
 * added in axis order (u, v[, g]) with one rounding each (no fused multiply-add), lowest k on
 * ties.  q (float, ndim values) is given by the caller.  Sites without data (h = 0) get -1.
 * labels has one entry per pixel (H x W, row major); in 3-D the pixel (u, v) is the voxel
 * (u, v, gray(u, v)) with weight hw(u, v).
 */
static int nearest_codebook(int ndim, const int *x, const float *q, int M, const int *r)
{
    int best = -1;
    float bd = 0.f;
    for (int k = 0; k < M; ++k) {
        float d = 0.f;
        for (int i = 0; i < ndim; ++i) {
            const int di = x[i] - r[k * ndim + i];
            const float t = (float)(di * di) * q[i];
            d = (i == 0) ? t : d + t;
        }
        if (best < 0 || d < bd) {
            best = k;
            bd = d;
        }
    }
    return best;
}

static int *codebook_sites(int ndim, const int *shape, int M, const double *Wc)
{
    int *r = (int *)malloc((size_t)M * ndim * sizeof(int));
    for (int k = 0; k < M; ++k)
        for (int i = 0; i < ndim; ++i) r[k * ndim + i] = (int)lattice_round(Wc[k * ndim + i], shape[i]);
    return r;
}

void orc_segment2d(const double *h, int H, int W, const float *q, int M, const double *Wc, int *labels)
{
    const int shape[2] = {H, W};
    int *r = codebook_sites(2, shape, M, Wc);
    for (int u = 0; u < H; ++u)
        for (int v = 0; v < W; ++v) {
            const int x[2] = {u, v};
            labels[(size_t)u * W + v] = h[(size_t)u * W + v] != 0.0 ? nearest_codebook(2, x, q, M, r) : -1;
        }
    free(r);
}

void orc_segment3d(const int *gray, const double *hw, int H, int W, int G, const float *q, int M,
                   const double *Wc, int *labels)
{
    const int shape[3] = {H, W, G};
    int *r = codebook_sites(3, shape, M, Wc);
    for (int u = 0; u < H; ++u)
        for (int v = 0; v < W; ++v) {
            const size_t o = (size_t)u * W + v;
            const int x[3] = {u, v, gray[o]};
            labels[o] = (hw ? hw[o] : 1.0) != 0.0 ? nearest_codebook(3, x, q, M, r) : -1;
        }
    free(r);
}

/* -------------------------------------------- chamfer distance transform (Sec. 5 weighting) */
/*
 * Sec. 5 weights the pixels of a binary shape by a distance transform T(X) (Borgefors' chamfer
 * transform), so that interior pixels count more.  Reading: the 3-4 chamfer distance of every
 * foreground pixel to the nearest background pixel, with the outside of the image counted as
 * background (a one-pixel background frame); background pixels get 0.  Unit steps cost 3 along
 * an axis and 4 along a diagonal.  Computed here by the two raster passes of the 3 x 3 mask:
 * forward (rows top to bottom, columns left to right) over the upper-left half of the mask,
 * then backward (bottom to top, right to left) over the lower-right half.  X: H x W bytes
 * (nonzero = foreground); T: H x W ints.
 */
static int chamfer_at(const int *T, int H, int W, int u, int v)
{
    return (u < 0 || u >= H || v < 0 || v >= W) ? 0 : T[(size_t)u * W + v];   /* frame: 0 */
}

static int min2(int a, int b) { return a < b ? a : b; }

void orc_chamfer34(const unsigned char *X, int H, int W, int *T)
{
    for (int u = 0; u < H; ++u)
        for (int v = 0; v < W; ++v) {
            if (!X[(size_t)u * W + v]) {
                T[(size_t)u * W + v] = 0;
                continue;
            }
            int d = chamfer_at(T, H, W, u - 1, v - 1) + 4;
            d = min2(d, chamfer_at(T, H, W, u - 1, v) + 3);
            d = min2(d, chamfer_at(T, H, W, u - 1, v + 1) + 4);
            d = min2(d, chamfer_at(T, H, W, u, v - 1) + 3);
            T[(size_t)u * W + v] = d;
        }
    for (int u = H - 1; u >= 0; --u)
        for (int v = W - 1; v >= 0; --v) {
            int d = T[(size_t)u * W + v];
            if (d == 0) continue;
            d = min2(d, chamfer_at(T, H, W, u + 1, v + 1) + 4);
            d = min2(d, chamfer_at(T, H, W, u + 1, v) + 3);
            d = min2(d, chamfer_at(T, H, W, u + 1, v - 1) + 4);
            d = min2(d, chamfer_at(T, H, W, u, v + 1) + 3);
            T[(size_t)u * W + v] = d;
        }
}

/* --------------------------------------------- recursive Gaussian fields (large sigma, Sec. 3.1) */
/*
 * For large widths Sec. 3.1 points to recursive filters (it cites Deriche 1992).  Deriche's
 * recursive Gaussian fits the kernel by two damped sinusoids,
 *     exp(-x^2/2) ~ k(x) = sum_t (alpha_t cos(omega_t x) + beta_t sin(omega_t x)) exp(-b_t x),  x >= 0,
 * (the published fit: alpha = 1.680, -0.6803; beta = 3.735, -0.2598; omega = 0.6318, 1.997;
 * b = 1.783, 1.723), and the convolution with the sampled kernel g(d) ~ k(|d| / sigma) is then
 * exact by recursion: with z_t = exp((-b_t + i omega_t) / sigma) and c_t = alpha_t - i beta_t,
 * k(j / sigma) = Re sum_t c_t z_t^j, so for a signal x[0..n)
 *     y[n]  = sum_m x[m] g(m - n)            = Re sum_t c_t (s0_t[n] + r0_t[n])
 *     yd[n] = sum_m x[m] g(m - n) (m - n)    = Re sum_t c_t (r1_t[n] - s1_t[n])
 * with the first-order complex recursions (zero outside the signal: zero start states)
 *     s0[n] = x[n] + z s0[n-1],           s1[n] = z (s1[n-1] + s0[n-1])        (causal, j >= 0)
 *     r0[n] = z (x[n+1] + r0[n+1]),       r1[n] = z (r1[n+1] + r0[n+1]) + z x[n+1]   (anticausal, j >= 1)
 * where s1 = sum_j j z^j x[n-j] and r1 = sum_{j>=1} j z^j x[n+j].  The kernel is untruncated; the
 * approximation is only the fit.  Written with explicit complex arithmetic in double.
 */
static const double kDericheAlpha[2] = {1.680, -0.6803};
static const double kDericheBeta[2] = {3.735, -0.2598};
static const double kDericheOmega[2] = {0.6318, 1.997};
static const double kDericheB[2] = {1.783, 1.723};

/* the fitted kernel k(x), x >= 0 */
double orc_deriche_kernel(double x)
{
    double k = 0;
    for (int t = 0; t < 2; ++t)
        k += (kDericheAlpha[t] * cos(kDericheOmega[t] * x) + kDericheBeta[t] * sin(kDericheOmega[t] * x)) *
             exp(-kDericheB[t] * x);
    return k;
}

/* y = sum_m x[m] g(m - n), yd = sum_m x[m] g(m - n)(m - n) (either may be NULL) */
void orc_deriche_filter(const double *x, int n, double sigma, double *y, double *yd)
{
    for (int i = 0; i < n; ++i) {
        if (y) y[i] = 0;
        if (yd) yd[i] = 0;
    }
    for (int t = 0; t < 2; ++t) {
        const double mag = exp(-kDericheB[t] / sigma), ang = kDericheOmega[t] / sigma;
        const double zr = mag * cos(ang), zi = mag * sin(ang);
        const double cr = kDericheAlpha[t], ci = -kDericheBeta[t];
        /* causal */
        double s0r = 0, s0i = 0, s1r = 0, s1i = 0;
        for (int i = 0; i < n; ++i) {
            /* s1[i] = z (s1[i-1] + s0[i-1]) uses the previous s0 */
            const double ar = s1r + s0r, ai = s1i + s0i;
            s1r = zr * ar - zi * ai;
            s1i = zr * ai + zi * ar;
            const double pr = zr * s0r - zi * s0i, pi = zr * s0i + zi * s0r;
            s0r = x[i] + pr;
            s0i = pi;
            if (y) y[i] += cr * s0r - ci * s0i;
            if (yd) yd[i] -= cr * s1r - ci * s1i;
        }
        /* anticausal */
        double r0r = 0, r0i = 0, r1r = 0, r1i = 0;
        for (int i = n - 1; i >= 0; --i) {
            const double xn = i + 1 < n ? x[i + 1] : 0.0;
            /* r1[i] = z (r1[i+1] + r0[i+1] + x[i+1]),  r0[i] = z (r0[i+1] + x[i+1]) */
            const double ar = r1r + r0r + xn, ai = r1i + r0i;
            const double br = r0r + xn, bi = r0i;
            r1r = zr * ar - zi * ai;
            r1i = zr * ai + zi * ar;
            r0r = zr * br - zi * bi;
            r0i = zr * bi + zi * br;
            if (y) y[i] += cr * r0r - ci * r0i;
            if (yd) yd[i] += cr * r1r - ci * r1i;
        }
    }
}

/*
 * 2-D fields by recursion along v, then along u (separable):  T = g_v * h, T_v = (d g)_v * h, then
 * A = g_u * T, F_u = (d g)_u * T, F_v = g_u * T_v (centred moments, as for the mask fields);
 * absolute: F_i + y_i A.
 */
void orc_fields2d_recursive(const double *h, int H, int W, double su, double sv, int absolute,
                            double *A, double *Fu, double *Fv)
{
    double *T = (double *)malloc((size_t)H * W * sizeof(double));
    double *Tv = (double *)malloc((size_t)H * W * sizeof(double));
    const int L = H > W ? H : W;
    double *in = (double *)malloc((size_t)L * sizeof(double));
    double *o0 = (double *)malloc((size_t)L * sizeof(double));
    double *o1 = (double *)malloc((size_t)L * sizeof(double));
    for (int u = 0; u < H; ++u) orc_deriche_filter(h + (size_t)u * W, W, sv, T + (size_t)u * W, Tv + (size_t)u * W);
    for (int v = 0; v < W; ++v) {
        for (int u = 0; u < H; ++u) in[u] = T[(size_t)u * W + v];
        orc_deriche_filter(in, H, su, o0, o1);
        for (int u = 0; u < H; ++u) {
            A[(size_t)u * W + v] = o0[u];
            Fu[(size_t)u * W + v] = o1[u] + (absolute ? u * o0[u] : 0.0);
        }
        for (int u = 0; u < H; ++u) in[u] = Tv[(size_t)u * W + v];
        orc_deriche_filter(in, H, su, o0, NULL);
        for (int u = 0; u < H; ++u) Fv[(size_t)u * W + v] = o0[u] + (absolute ? v * A[(size_t)u * W + v] : 0.0);
    }
    free(T);
    free(Tv);
    free(in);
    free(o0);
    free(o1);
}
