// Gauss-Newton normal equations of the network inversion (§5.3, Eq. 9), in
// float64, finished by the last CTA of the Jacobian kernel that produced the
// per-CTA partial sums.
//
// Partial layout per CTA (stride gn_partial_stride(r)):
//   [0, T)            sum_p J_p^T J_p, upper triangle (i <= j), T = r (r + 1) / 2
//   [T, T + r)        sum_p J_p^T res_p
//   [T + r]           sum_p |res_p|^2
// The system (A + damping I) dz = -b is solved by a right-looking Cholesky
// factorisation with one thread per entry, then column-oriented triangular
// solves; z_out = z_in + dz.  A non-positive or non-finite pivot sets
// NSF_ERR_SINGULAR and leaves z unchanged.
#pragma once

#include "device_common.cuh"

namespace nsf {

struct GnShared {
    double sum[kMaxR * (kMaxR + 1) / 2 + kMaxR + 1];
    double A[kMaxR * kMaxR];
    double y[kMaxR];
    int singular;
    int is_last;
};

// Called by every thread of every CTA after the CTA wrote its partials.
// Returns after the last CTA has finished the solve (others return at once).
__device__ inline void gn_arrive_and_finish(const GnArgs &g, int r, int *status,
                                     GnShared &sh) {
    const int tid = threadIdx.x;
    const int nthreads = blockDim.x;
    const int T = r * (r + 1) / 2;
    const int stride = T + r + 1;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        int ticket = atomicAdd(g.counter, 1);
        sh.is_last = (ticket == (int)gridDim.x - 1);
        sh.singular = 0;
    }
    __syncthreads();
    if (!sh.is_last) return;
    __threadfence();

    // Deterministic reduction over CTAs in index order.
    for (int e = tid; e < stride; e += nthreads) {
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(&g.partials[(size_t)b * stride + e]);
        sh.sum[e] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < r * r; idx += nthreads) {
        int i = idx / r, j = idx - i * r;
        int e = i <= j ? tri_index(i, j, r) : tri_index(j, i, r);
        sh.A[idx] = sh.sum[e] + (i == j ? g.damping : 0.0);
    }
    for (int k = tid; k < r; k += nthreads) sh.y[k] = -sh.sum[T + k];
    __syncthreads();

    // Cholesky A = L L^T, L stored in the lower triangle of A.
    for (int j = 0; j < r; ++j) {
        if (tid == 0) {
            double d = sh.A[j * r + j];
            if (!(d > 0.0) || !isfinite(d)) {
                sh.singular = 1;
                sh.A[j * r + j] = 1.0;
            } else {
                sh.A[j * r + j] = sqrt(d);
            }
        }
        __syncthreads();
        if (sh.singular) break;
        for (int i = j + 1 + tid; i < r; i += nthreads) sh.A[i * r + j] /= sh.A[j * r + j];
        __syncthreads();
        const int m = r - j - 1;
        for (int idx = tid; idx < m * m; idx += nthreads) {
            int i = j + 1 + idx / m, k = j + 1 + idx % m;
            if (k <= i) sh.A[i * r + k] -= sh.A[i * r + j] * sh.A[k * r + j];
        }
        __syncthreads();
    }
    const bool singular = sh.singular != 0;
    if (!singular) {
        // Forward solve L y = -b (column oriented).
        for (int k = 0; k < r; ++k) {
            if (tid == 0) sh.y[k] /= sh.A[k * r + k];
            __syncthreads();
            for (int i = k + 1 + tid; i < r; i += nthreads) sh.y[i] -= sh.A[i * r + k] * sh.y[k];
            __syncthreads();
        }
        // Back solve L^T dz = y.
        for (int k = r - 1; k >= 0; --k) {
            if (tid == 0) sh.y[k] /= sh.A[k * r + k];
            __syncthreads();
            for (int i = tid; i < k; i += nthreads) sh.y[i] -= sh.A[k * r + i] * sh.y[k];
            __syncthreads();
        }
    } else if (tid == 0) {
        set_status(status, NSF_ERR_SINGULAR);
    }
    for (int k = tid; k < r; k += nthreads) {
        double z0 = __ldcg(&g.z_in[k]);
        double zn = singular ? z0 : z0 + sh.y[k];
        if (!isfinite(zn)) {
            set_status(status, NSF_ERR_NONFINITE);
            zn = z0;
        }
        if (g.z_prev_out) g.z_prev_out[k] = __ldcg(&g.z_first[k]);
        g.z_out[k] = zn;
        if (g.z_tap) g.z_tap[k] = zn;
    }
    if (tid == 0) *g.counter = 0;
}

}  // namespace nsf
