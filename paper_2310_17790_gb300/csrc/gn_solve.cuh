// Gauss-Newton normal equations of the network inversion (§5.3, Eq. 9), in
// float64, finished by the last CTA of the Jacobian kernel that produced the
// per-CTA partial sums of an iteration.
//
// Partial layout per CTA (stride gn_partial_stride(r)):
//   [0, T)            sum_p J_p^T J_p, upper triangle (i <= j), T = r (r + 1) / 2
//   [T, T + r)        sum_p J_p^T res_p
//   [T + r]           sum_p |res_p|^2
// The system (A + damping I) dz = -b is solved by a column-parallel Cholesky
// factorisation and two triangular solves; z_new = z + dz.  Dependent float64
// operations are slow on this part, so every step keeps the chain short: the
// CTA reduction is a tree, each pivot costs one reciprocal square root
// (float32 estimate + Newton steps) and no division is used.  A non-positive
// or non-finite pivot sets NSF_ERR_SINGULAR and leaves z unchanged for that
// iteration.
#pragma once

#include "device_common.cuh"

namespace nsf {

// 1 / sqrt(d) for d > 0 in float64: Newton-Raphson on f(y) = y^-2 - d,
// y <- y (3 - d y^2) / 2, from the float32 reciprocal square root (relative
// error ~1e-7).  One step squares the error (~1e-14, far below what the
// Gauss-Newton step needs).  Values outside the float32 range start from the
// float64 library square root instead.
__device__ __forceinline__ double rsqrt_newton(double d) {
    const float df = (float)d;
    double y;
    if (df > 1e-30f && df < 1e30f) y = (double)rsqrtf(df);
    else y = 1.0 / sqrt(d);
    const double hd = -0.5 * d;
    return y * fma(hd * y, y, 1.5);
}

struct GnShared {
    double sum[kMaxR * (kMaxR + 1) / 2 + kMaxR + 1];
    double red[1024];
    double A[kMaxR * kMaxR];
    double y[kMaxR];
    double inv[kMaxR];
    int singular;
    int is_last;
};

// z used by iteration `it` of a Gauss-Newton run.
__host__ __device__ __forceinline__ const double *gn_z_in(const GnArgs &g, int it) {
    return it == 0 ? g.z_start : g.z_buf;
}

// Called by every thread of every CTA after the CTA wrote its partials of
// iteration `it`.  The last CTA to arrive solves the system and writes the new
// z; the function returns true in that CTA only, after the new z is written.
// Other CTAs return false at once.  blockDim.x must be <= 1024.
__device__ inline bool gn_arrive_and_solve(const GnArgs &g, int r, int it, int *status,
                                           GnShared &sh) {
    const int tid = threadIdx.x;
    const int nthreads = blockDim.x;
    const int T = r * (r + 1) / 2;
    const int stride = T + r + 1;
    const int nblk = (int)gridDim.x;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        int ticket = atomicAdd(g.counter, 1);
        sh.is_last = (ticket == nblk - 1);
        sh.singular = 0;
    }
    __syncthreads();
    if (!sh.is_last) return false;
    __threadfence();

    // Tree reduction over CTAs: thread t sums CTAs c, c + C, ... of entry
    // e = t % stride (c = t / stride), then the C values of each entry are
    // combined pairwise in a fixed order (deterministic).
    const int C = nthreads / stride;
    const int e_t = tid % stride, c_t = tid / stride;
    if (c_t < C) {
        double s = 0.0;
        for (int b = c_t; b < nblk; b += C) s += __ldcg(&g.partials[(size_t)b * stride + e_t]);
        sh.red[c_t * stride + e_t] = s;
    }
    __syncthreads();
    for (int half = 1; half < C; half <<= 1) {
        if (c_t < C && (c_t % (2 * half)) == 0 && c_t + half < C)
            sh.red[c_t * stride + e_t] += sh.red[(c_t + half) * stride + e_t];
        __syncthreads();
    }
    for (int idx = tid; idx < r * r; idx += nthreads) {
        int i = idx / r, j = idx - i * r;
        int e = i <= j ? tri_index(i, j, r) : tri_index(j, i, r);
        sh.A[idx] = sh.red[e] + (i == j ? g.damping : 0.0);
    }
    for (int k = tid; k < r; k += nthreads) sh.y[k] = -sh.red[T + k];
    __syncthreads();

    // Right-looking Cholesky A = L L^T (L in the lower triangle of A) and the
    // two triangular solves, by warp 0: lane i owns row i, so the steps need
    // only warp-level synchronisation (r <= 16 <= 32 lanes).
    if (tid < 32) {
        const int lane = tid;
        int singular = 0;
        for (int j = 0; j < r; ++j) {
            if (lane == 0) {
                const double d = sh.A[j * r + j];
                if (!(d > 0.0) || !isfinite(d)) {
                    sh.singular = 1;
                } else {
                    const double rs = rsqrt_newton(d);
                    sh.inv[j] = rs;
                    sh.A[j * r + j] = d * rs;
                }
            }
            __syncwarp();
            if (sh.singular) {
                singular = 1;
                break;
            }
            const int i = lane;
            if (i > j && i < r) sh.A[i * r + j] *= sh.inv[j];
            __syncwarp();
            if (i > j && i < r) {
                const double lij = sh.A[i * r + j];
                for (int k = j + 1; k <= i; ++k)
                    sh.A[i * r + k] = fma(-lij, sh.A[k * r + j], sh.A[i * r + k]);
            }
            __syncwarp();
        }
        if (!singular) {
            double yi = lane < r ? sh.y[lane] : 0.0;      // -b
            for (int k = 0; k < r; ++k) {                 // L y = -b
                const double yk = __shfl_sync(0xffffffffu, yi, k) * sh.inv[k];
                if (lane == k) yi = yk;
                else if (lane > k && lane < r) yi = fma(-sh.A[lane * r + k], yk, yi);
            }
            for (int k = r - 1; k >= 0; --k) {            // L^T dz = y
                const double yk = __shfl_sync(0xffffffffu, yi, k) * sh.inv[k];
                if (lane == k) yi = yk;
                else if (lane < k) yi = fma(-sh.A[k * r + lane], yk, yi);
            }
            if (lane < r) sh.y[lane] = yi;
        } else if (lane == 0) {
            set_status(status, NSF_ERR_SINGULAR);
        }
    }
    __syncthreads();
    const bool singular = sh.singular != 0;

    const bool fin = it == g.iters - 1;
    const double *zin = gn_z_in(g, it);
    double *zout = fin ? g.z_out : g.z_buf;
    for (int k = tid; k < r; k += nthreads) {
        const double z0 = __ldcg(&zin[k]);
        double zn = singular ? z0 : z0 + sh.y[k];
        if (!isfinite(zn)) {
            set_status(status, NSF_ERR_NONFINITE);
            zn = z0;
        }
        if (fin && g.z_prev_out) g.z_prev_out[k] = __ldcg(&g.z_start[k]);
        zout[k] = zn;
        if (g.z_taps) g.z_taps[(size_t)it * r + k] = zn;
    }
    if (tid == 0) *g.counter = 0;
    __threadfence();
    __syncthreads();
    return true;
}

}  // namespace nsf
