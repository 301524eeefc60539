// Sample and integration particles (paper §5.4): with the particle positions
// x_p = g(X_p, z) at the current latent code,
//   I = grid nodes in the quadratic B-spline stencil of some sample particle,
//   N = every particle whose stencil contains a node of I,
// listed S first (in the caller's order), then the other members of N in
// increasing particle index.  For the quadratic B-spline a particle's stencil
// is the 3^3 nodes base + {0, 1, 2}^3, base = floor(x / dx - 0.5) (the same
// float32 arithmetic as the MPM kernels).
//
// Kernels: mark the sample stencils in a node bitmap, flag the particles whose
// stencil meets it (per-block counts), scan the counts in one CTA, scatter the
// flagged indices, gather their reference positions.
#include "device_common.cuh"

namespace nsf {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ bool position(const SubsetArgs &a, int p, float x[3]) {
    x[0] = a.u[p];
    x[1] = a.u[a.n + p];
    x[2] = a.u[2 * a.n + p];
    if (a.residual) {
        x[0] = a.X[p] + x[0];
        x[1] = a.X[a.n + p] + x[1];
        x[2] = a.X[2 * a.n + p] + x[2];
    }
    return finite3(x[0], x[1], x[2]);
}

// Stencil base of x (the base node of the MPM kernels' bspline_axis, with
// x / dx and the shift by 0.5 each rounded to float32), false if the stencil
// leaves the grid.
__device__ __forceinline__ bool stencil_base(const SubsetArgs &a, const float x[3], int b[3]) {
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        b[d] = bspline_axis(x[d], a.inv_dx).base;
        ok &= b[d] >= 0 && b[d] + 2 <= a.dims[d] - 1;
    }
    return ok;
}

__device__ __forceinline__ int node_bit(const SubsetArgs &a, int i, int j, int k) {
    return (i * a.dims[1] + j) * a.dims[2] + k;
}

// Step a: the nodes of every sample particle's stencil; marks S membership.
__global__ void __launch_bounds__(kThreads) k_mark(SubsetArgs a, int *status) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n_S) return;
    const int p = a.sample[s];
    if (p < 0 || p >= a.n) {
        set_status(status, NSF_ERR_INVALID_ARG);
        return;
    }
    a.in_S[p] = 1;
    float x[3];
    int b[3];
    if (!position(a, p, x)) {
        set_status(status, NSF_ERR_NONFINITE);
        return;
    }
    if (!stencil_base(a, x, b)) {
        set_status(status, NSF_ERR_OUT_OF_GRID);
        return;
    }
    for (int q = 0; q < 27; ++q) {
        const int bit = node_bit(a, b[0] + q / 9, b[1] + (q / 3) % 3, b[2] + q % 3);
        atomicOr(&a.bitmap[bit >> 5], 1u << (bit & 31));
    }
}

// Whether particle p (not a sample particle) belongs to N.
__device__ __forceinline__ bool member(const SubsetArgs &a, int p) {
    if (p >= a.n || a.in_S[p]) return false;
    float x[3];
    int b[3];
    if (!position(a, p, x) || !stencil_base(a, x, b)) return false;
    for (int q = 0; q < 27; ++q) {
        const int bit = node_bit(a, b[0] + q / 9, b[1] + (q / 3) % 3, b[2] + q % 3);
        if (__ldg(&a.bitmap[bit >> 5]) & (1u << (bit & 31))) return true;
    }
    return false;
}

// Rank of this thread's flag among the CTA's set flags (ascending thread
// order) and the CTA's count.
__device__ __forceinline__ int block_rank(bool f, int &count) {
    __shared__ int wcount[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcount[warp] = __popc(bal);
    __syncthreads();
    int before = 0;
    count = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
        if (w < warp) before += wcount[w];
        count += wcount[w];
    }
    __syncthreads();
    return before + __popc(bal & ((1u << lane) - 1u));
}

// Step b, first pass: members per CTA.
__global__ void __launch_bounds__(kThreads) k_count(SubsetArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    int count;
    block_rank(member(a, p), count);
    if (threadIdx.x == 0) a.block_count[blockIdx.x] = count;
}

// Exclusive scan of the CTA counts (one CTA, in chunks), |N| = n_S + total.
__global__ void __launch_bounds__(1024) k_scan(SubsetArgs a, int nblocks, int *count_out) {
    __shared__ int part[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nblocks; c0 += 1024) {
        const int i = c0 + (int)threadIdx.x;
        const int v = i < nblocks ? a.block_count[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {          // inclusive Hillis-Steele
            const int t = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nblocks) a.block_off[i] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *count_out = a.n_S + carry;
}

// Step b, second pass: S first, then the members in increasing index.
__global__ void __launch_bounds__(kThreads) k_scatter(SubsetArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < a.n_S) a.index_out[p] = a.sample[p];
    const bool f = member(a, p);
    int count;
    const int rank = block_rank(f, count);
    if (f) a.index_out[a.n_S + a.block_off[blockIdx.x] + rank] = p;
}

// Reference positions of N in the order of index_out.
__global__ void __launch_bounds__(kThreads) k_gather(SubsetArgs a, const int *count,
                                                     float *X_out, int ld_out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= __ldg(count)) return;
    const int p = a.index_out[k];
    if (p < 0 || p >= a.n) return;
    X_out[k] = a.X[p];
    X_out[ld_out + k] = a.X[a.n + p];
    X_out[2 * ld_out + k] = a.X[2 * a.n + p];
}

}  // namespace

cudaError_t launch_subset(const SubsetArgs &a, int *count_out, float *X_out, int ld_out,
                          int *status, cudaStream_t s) {
    const int nb = (a.n + kThreads - 1) / kThreads;
    if (a.n_S > 0) k_mark<<<(a.n_S + kThreads - 1) / kThreads, kThreads, 0, s>>>(a, status);
    k_count<<<nb, kThreads, 0, s>>>(a);
    k_scan<<<1, 1024, 0, s>>>(a, nb, count_out);
    k_scatter<<<nb, kThreads, 0, s>>>(a);
    if (X_out) k_gather<<<nb, kThreads, 0, s>>>(a, count_out, X_out, ld_out);
    return cudaGetLastError();
}

}  // namespace nsf
