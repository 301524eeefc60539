// Gauss-Newton normal equations of the network inversion (§5.3, Eq. 9), in
// float64, from the per-CTA partial sums of the Jacobian kernel.
//
// Partial layout (stride gn_partial_stride(r)):
//   [0, T)            sum_p J_p^T J_p, upper triangle (i <= j), T = r (r + 1) / 2
//   [T, T + r)        sum_p J_p^T res_p
//   [T + r]           sum_p |res_p|^2
// CTAs add their partial sums into a float64 accumulator with atomics.  The
// system (A + damping I) dz = -b is solved by gn_solve_warp and z_new = z + dz.
// A non-positive or non-finite pivot sets NSF_ERR_SINGULAR and leaves z
// unchanged for that iteration.
//
// This file serves the one-launch-per-iteration path of the FP32 Jacobian
// kernel: the last CTA to arrive solves and writes z to global memory.  The
// cooperative tensor-core kernel runs all iterations in one launch with the
// float-float variant in gn_ff.cuh.
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
    double sum[kGnStrideMax];
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

// float64 solve of A x = y (A: r x r SPD in sh.A, right-hand side in sh.y) by
// warp 0, lane i owning row i: Cholesky factorisation A = L L^T and the two
// triangular solves, with warp-level synchronisation only.  Each pivot costs
// one reciprocal square root (float32 estimate + one Newton step) and no
// division is used; dependent float64 operations are slow on this part, so
// the chain is kept to a few operations per column.  Writes x to sh.y;
// returns 1 if A is not positive definite.
__device__ inline int gn_solve_warp(GnShared &sh, int r) {
    const int lane = threadIdx.x & 31;
    int singular = 0;
    for (int j = 0; j < r; ++j) {
        const double d = sh.A[j * r + j];
        if (!(d > 0.0) || !isfinite(d)) { singular = 1; break; }
        const double rs = rsqrt_newton(d);
        if (lane == 0) {
            sh.inv[j] = rs;
            sh.A[j * r + j] = d * rs;
        }
        if (lane > j && lane < r) sh.A[lane * r + j] *= rs;
        __syncwarp();
        if (lane > j && lane < r) {
            const double lij = sh.A[lane * r + j];
            for (int k = j + 1; k <= lane; ++k)
                sh.A[lane * r + k] = fma(-lij, sh.A[k * r + j], sh.A[lane * r + k]);
        }
        __syncwarp();
    }
    if (singular) return 1;
    double yi = lane < r ? sh.y[lane] : 0.0;
    for (int k = 0; k < r; ++k) {                         // L u = y
        const double yk = __shfl_sync(0xffffffffu, yi, k) * sh.inv[k];
        if (lane == k) yi = yk;
        else if (lane > k && lane < r) yi = fma(-sh.A[lane * r + k], yk, yi);
    }
    for (int k = r - 1; k >= 0; --k) {                    // L^T x = u
        const double yk = __shfl_sync(0xffffffffu, yi, k) * sh.inv[k];
        if (lane == k) yi = yk;
        else if (lane < k) yi = fma(-sh.A[k * r + lane], yk, yi);
    }
    if (lane < r) sh.y[lane] = yi;
    __syncwarp();
    return 0;
}

// Builds A + damping I and y = -b from the sums in sh.sum and solves in
// warp 0; leaves dz in sh.y and the outcome in sh.singular.
__device__ inline void gn_build_and_solve(const GnArgs &g, int r, int *status, GnShared &sh) {
    const int tid = threadIdx.x;
    const int T = r * (r + 1) / 2;
    for (int idx = tid; idx < r * r; idx += blockDim.x) {
        const int i = idx / r, j = idx - i * r;
        const int e = i <= j ? tri_index(i, j, r) : tri_index(j, i, r);
        sh.A[idx] = sh.sum[e] + (i == j ? g.damping : 0.0);
    }
    for (int k = tid; k < r; k += blockDim.x) sh.y[k] = -sh.sum[T + k];
    __syncthreads();
    if (tid < 32) {
        const int sing = gn_solve_warp(sh, r);
        if (tid == 0) {
            sh.singular = sing;
            if (sing) set_status(status, NSF_ERR_SINGULAR);
        }
    }
    __syncthreads();
}

// Called by every thread of every CTA with the CTA's float64 partial sums of
// iteration `it` in `part` (shared memory, gn_partial_stride(r) values).  The
// partials are added into g.gsum with float64 atomics; the last CTA to arrive
// reads the sums, clears them, solves the system and writes the new z.  The
// function returns true in that CTA only, after the new z is written; other
// CTAs return false at once.
__device__ inline bool gn_arrive_and_solve(const GnArgs &g, int r, int it, int *status,
                                           GnShared &sh, const double *part) {
    const int tid = threadIdx.x;
    const int nthreads = blockDim.x;
    const int T = r * (r + 1) / 2;
    const int stride = T + r + 1;
    const int nblk = (int)gridDim.x;
    for (int e = tid; e < stride; e += nthreads) atomicAdd(&g.gsum[e], part[e]);
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
    for (int e = tid; e < stride; e += nthreads) {
        sh.sum[e] = __ldcg(&g.gsum[e]);
        g.gsum[e] = 0.0;                   // ready for the next iteration / launch
    }
    __syncthreads();
    gn_build_and_solve(g, r, status, sh);
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
