// Device helpers shared by the kernels of libnsf.
#pragma once

#include "internal.h"

namespace nsf {

// Bound on every spin-wait of the library's kernels (barriers, mbarriers):
// a wait that runs out records an error status and returns.
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may be scheduled while the kernel before it
// in the stream is still finishing; griddepcontrol.wait then blocks until that
// kernel has completed and its memory is visible (a no-op for a normal
// launch).  The kernels that are launched this way call it before touching
// global memory at all, so only their launch and CTA set-up overlap the
// previous kernel.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// First error wins: the status word only moves away from NSF_OK once.
__device__ __forceinline__ void set_status(int *status, int code) {
    if (status) atomicCAS(status, NSF_OK, code);
}

// ELU of the field networks (App. E): a for a > 0, exp(a) - 1 otherwise.
__device__ __forceinline__ float elu(float a) { return a > 0.f ? a : expm1f(a); }
// Its derivative, from the pre-activation: 1 for a > 0, exp(a) otherwise.
__device__ __forceinline__ float elu_grad(float a) { return a > 0.f ? 1.f : expf(a); }

// Grid-wide barrier of a cooperative launch (all CTAs co-resident) on one
// arrival word that is zero before the launch's first barrier.  CTA 0 adds
// 2^31 - (gridDim.x - 1), every other CTA adds 1: the low bits count the
// arrivals and carry into the top bit exactly when the last CTA arrives, after
// which they are back at zero, so the word is ready for the next barrier with
// no reset.  Every thread of every CTA calls it.  Returns false after
// recording NSF_ERR_ITER_CAP if the wait ran out; the word is then undefined.
//
// group_barrier is the same over the `size` CTAs of a group that share `word`,
// the CTA of rank 0 taking the part of CTA 0.
__device__ inline bool group_barrier(unsigned *word, int rank, int size, int *status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        const unsigned inc = rank == 0 ? 0x80000000u - (unsigned)(size - 1) : 1u;
        __threadfence();
        const unsigned old = atomicAdd(word, inc);
        volatile unsigned *w = word;
        const unsigned long long t0 = global_ns();
        while (((*w ^ old) & 0x80000000u) == 0u) {
            if (global_ns() - t0 > kWaitNs) {
                set_status(status, NSF_ERR_ITER_CAP);
                s_ok = 0;
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ inline bool grid_barrier(unsigned *word, int *status) {
    return group_barrier(word, (int)blockIdx.x, (int)gridDim.x, status);
}

// Upper-triangle (i <= j) packed index of an r x r symmetric matrix.
__host__ __device__ __forceinline__ int tri_index(int i, int j, int r) {
    // rows 0 .. i-1 hold r, r-1, ..., r-i+1 entries
    return i * r - (i * (i - 1)) / 2 + (j - i);
}

// Quadratic B-spline stencil along one axis (§3.2, b = 2):
// base = floor(s - 0.5) with s = x / dx, fx = s - base in [0.5, 1.5).
// s and s - 0.5 are rounded explicitly (no multiply-add contraction), so every
// kernel that bins, scatters or gathers a particle finds the same base node.
struct Axis {
    int base;
    float fx;
    float w[3];
};

__device__ __forceinline__ Axis bspline_axis(float x, float inv_dx) {
    Axis a;
    const float s = __fmul_rn(x, inv_dx);
    a.base = __float2int_rd(__fsub_rn(s, 0.5f));
    a.fx = __fsub_rn(s, (float)a.base);
    float t0 = 1.5f - a.fx, t1 = a.fx - 1.0f, t2 = a.fx - 0.5f;
    a.w[0] = 0.5f * t0 * t0;
    a.w[1] = 0.75f - t1 * t1;
    a.w[2] = 0.5f * t2 * t2;
    return a;
}

// Block-linear address of node (i, j, k) of the workspace grid.
__device__ __forceinline__ int node_addr(const GridWs &g, int i, int j, int k) {
    int b = ((i >> 2) * g.nb1 + (j >> 2)) * g.nb2 + (k >> 2);
    return b * 64 + (((i & 3) * 4 + (j & 3)) * 4 + (k & 3));
}

__device__ __forceinline__ bool finite3(float a, float b, float c) {
    return isfinite(a) && isfinite(b) && isfinite(c);
}

}  // namespace nsf
