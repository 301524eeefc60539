// BF16 field networks on the tcgen05 tensor cores (precision NSF_PREC_BF16):
// value evaluation of g, h and l (paper §5.1, inference on the integration
// particles; App. E, fields are ELU MLPs on [X; z]).  The Jacobian and the
// Gauss-Newton iterations run in jacobian_tc.cu.
//
// One CTA = eight warpgroups (1024 threads) on a 128-point tile; point i is
// tile row i and TMEM lane i, which only the warps with (warp index % 4) ==
// i / 32 can read.  Warpgroup w owns the column eighth [w W / 8, (w + 1) W / 8)
// of every layer.  Per tile:
//   layer 0 (K = 3 + r)  on the CUDA cores in FP32, written as bf16 into the
//                        shared-memory A operand;
//   hidden layers        tcgen05.mma M = 128, N = width, K = width (16 per
//                        instruction), FP32 accumulator in tensor memory; the
//                        epilogue reads it with tcgen05.ld, adds the FP32 bias,
//                        applies ELU, rounds to bf16 and rewrites A in place;
//   output layer         the same MMA with N = 16 (out_dim padded with zero
//                        rows), bias added when the outputs are read.
// All weights of the CTA's field stay resident in shared memory (one bulk copy
// per CTA on an mbarrier with a transaction count); persistent CTAs loop over
// tiles.  Every wait on an mbarrier is bounded by time: on expiry the kernel
// records NSF_ERR_ITER_CAP, waits (bounded) for its outstanding operations,
// frees its tensor memory and returns.
//
// Weight operands (B here, A in the Jacobian kernel) and the activation tile
// are K-major with the 128-byte swizzle (tc_common.cuh).
#include "tc_common.cuh"

namespace nsf {

using namespace tc;

// ------------------------------------------------------------ packing ----
size_t tc_layer_elems(int rows_pad, int k) { return (size_t)rows_pad * k; }

// One layer [rows][k] (fp32 host values, rows zero-padded to rows_pad, k a
// multiple of 64) as a K-major, 128-byte-swizzled bf16 operand.
void tc_pack_layer(const float *W, int rows, int rows_pad, int k, __nv_bfloat16 *dst) {
    for (int n = 0; n < rows_pad; ++n)
        for (int c = 0; c < k; ++c)
            dst[sw128_kmajor_offset(n, c, rows_pad) / 2] =
                __float2bfloat16_rn(n < rows ? W[(size_t)n * k + c] : 0.f);
}

size_t jac_tc_smem_bytes(int r, int width, int depth);   // jacobian_tc.cu

namespace {

// Shared-memory carve of one CTA (byte offsets from a 1024-aligned base).
struct TcLayout {
    int a, blob, w0v, bias, bars, tmem, total;
};

__host__ __device__ inline TcLayout tc_layout(int W, int D) {
    TcLayout L;
    int o = 0;
    L.a = o;    o = align_to(o + kM * W * 2, 1024);
    L.blob = o; o = align_to(o + (D - 1) * W * W * 2 + kMaxOut * W * 2, 1024);
    L.w0v = o;  o = align_to(o + W * 16, 16);                 // float4 {w_x, w_y, w_z, c0}
    L.bias = o; o = align_to(o + D * W * 4, 16);              // hidden biases, then output bias
    L.bars = o; o = align_to(o + 2 * 8, 16);
    L.tmem = o; o = align_to(o + 16, 16);
    L.total = o + 1024;   // room to align the dynamic base to 1024 bytes
    return L;
}

// Byte offset of the 16-byte chunk holding columns c .. c + 7 (c % 8 == 0) of
// row m in the 128-row A tile.
__device__ __forceinline__ int a_chunk(int m, int c) {
    return (c >> 6) * (kM * 128) + (m >> 3) * 1024 + (m & 7) * 128 +
           ((((c >> 3) & 7) ^ (m & 7)) << 4);
}

__device__ __forceinline__ void store_a8(uint8_t *A, int m, int c, const float *h) {
    *reinterpret_cast<uint4 *>(A + a_chunk(m, c)) = pack_bf16x8(h);
}

struct TcJobs {
    int njobs;
    FieldJob job[4];
};

__global__ void __launch_bounds__(kThreads, 1)
k_fields_tc(const __grid_constant__ FieldsDev fd, const float *__restrict__ X, int n, int ld,
            const __grid_constant__ TcJobs jobs, int *status) {
    extern __shared__ uint8_t smem_dyn[];
    __shared__ int s_abort;
    uint8_t *base = aligned_smem(smem_dyn);

    const FieldJob &job = jobs.job[blockIdx.y];
    const FieldDev &F = fd.f[job.field];
    const int W = F.width, D = F.depth, r = fd.r;
    const int tiles = (n + kM - 1) / kM;
    const int tid = threadIdx.x;
    const int wg = tid >> 7;                 // warpgroup: column eighth
    const int row = tid & (kM - 1);          // tile row == TMEM lane
    const int wq = row >> 5;                 // lane quarter of this warp
    const int cw = W / kWG;                  // columns per warpgroup (multiple of 8)
    const int cbeg = wg * cw;
    const TcLayout L = tc_layout(W, D);
    uint8_t *A = base + L.a;
    uint8_t *blob = base + L.blob;
    float4 *W0v = reinterpret_cast<float4 *>(base + L.w0v); // [W] {W0[j][0..2], c0[j]}
    float *bias = reinterpret_cast<float *>(base + L.bias);  // [D][W]
    uint64_t *bar_w = reinterpret_cast<uint64_t *>(base + L.bars);
    uint64_t *bar_mma = bar_w + 1;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(base + L.tmem);
    uint32_t ncols = 32;
    while ((int)ncols < W) ncols <<= 1;

    if (tid == 0) {
        s_abort = 0;
        mbar_init(bar_w, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) tmem_alloc(tmem_holder, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    // weights: one bulk copy, landing while the CTA prepares the input layer
    if (tid == 0) bulk_load(blob, F.tc_blob, (uint32_t)F.tc_blob_bytes, bar_w);
    const int in0 = 3 + r;
    for (int j = tid; j < W; j += kThreads) {
        // z-part of the input layer folded into its bias: c0 = b0 + W0[:, 3:] z
        const float *w = F.W0 + (size_t)j * in0;
        float c0 = F.b[0][j];
        for (int k = 0; k < r; ++k) c0 = fmaf(w[3 + k], (float)__ldcg(&job.z[k]), c0);
        W0v[j] = make_float4(w[0], w[1], w[2], c0);
    }
    for (int l = 1; l <= D; ++l) {
        const int o = l == D ? F.out_dim : W;
        for (int j = tid; j < o; j += kThreads) bias[(l - 1) * W + j] = F.b[l][j];
    }
    bool weights_ready = false;
    const uint32_t a_addr = smem_u32(A);
    const uint32_t b_addr = smem_u32(blob);
    const uint32_t idesc_h = idesc_bf16(kM, W);
    const uint32_t idesc_o = idesc_bf16(kM, kMaxOut);
    const uint32_t tlane = tmem + ((uint32_t)(wq * 32) << 16);
    uint32_t phase = 0;
    __syncthreads();

    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int p = tile * kM + row;
        const bool valid = p < n;
        // ---- layer 0 on the CUDA cores
        float x0 = 0.f, x1 = 0.f, x2 = 0.f;
        if (valid) {
            x0 = X[p];
            x1 = X[ld + p];
            x2 = X[2 * ld + p];
        }
        for (int cc = cbeg; cc < cbeg + cw; cc += kGroup) {
            float v[kGroup];
#pragma unroll
            for (int i = 0; i < kGroup; ++i) {
                const float4 w = W0v[cc + i];
                float g;
                v[i] = elu_fast(fmaf(w.x, x0, fmaf(w.y, x1, fmaf(w.z, x2, w.w))), g);
            }
            store_a8(A, row, cc, v);
        }
        fence_proxy_async();
        __syncthreads();
        if (!weights_ready) {
            if (!__syncthreads_and(mbar_wait(bar_w, 0))) {
                if (tid == 0) set_status(status, NSF_ERR_ITER_CAP);
                mbar_wait(bar_w, 0);      // bounded: let the copy land before leaving
                goto teardown;
            }
            weights_ready = true;
        }

        // ---- hidden layers, then the output layer (l == D)
        for (int l = 1; l <= D; ++l) {
            const bool out_layer = l == D;
            if (tid == 0) {
                tc_fence_after();
                const uint32_t boff = (uint32_t)((l - 1) * W * W * 2);
                const int nrows = out_layer ? kMaxOut : W;
                const uint32_t idesc = out_layer ? idesc_o : idesc_h;
                for (int ks = 0; ks < W / 16; ++ks) {
                    const uint32_t koff = (uint32_t)((ks & 3) * 32);
                    const uint32_t atom = (uint32_t)(ks >> 2);
                    mma_bf16(tmem, sw128_desc(a_addr + atom * (kM * 128) + koff),
                             sw128_desc(b_addr + boff + atom * (nrows * 128) + koff), idesc,
                             ks > 0 ? 1u : 0u);
                }
                mma_commit(bar_mma);
                // the issuing thread alone waits (polling by every thread would
                // take issue slots from the others); the rest sleep at the barrier
                if (!mbar_wait(bar_mma, phase)) s_abort = 1;
                tc_fence_before();
            }
            phase ^= 1u;
            __syncthreads();
            tc_fence_after();
            if (s_abort) goto mma_timeout;
            if (!out_layer) {
                const float *bl = bias + (l - 1) * W;
                for (int cc = cbeg; cc < cbeg + cw; cc += 2 * kGroup) {
                    const bool two = cc + kGroup < cbeg + cw;
                    float v[kGroup], w[kGroup];
                    tmem_ld8(tlane + cc, v);
                    if (two) tmem_ld8(tlane + cc + kGroup, w);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < kGroup; ++i) {
                        float g;
                        v[i] = elu_fast(v[i] + bl[cc + i], g);
                    }
                    store_a8(A, row, cc, v);
                    if (two) {
#pragma unroll
                        for (int i = 0; i < kGroup; ++i) {
                            float g;
                            w[i] = elu_fast(w[i] + bl[cc + kGroup + i], g);
                        }
                        store_a8(A, row, cc + kGroup, w);
                    }
                }
                tc_fence_before();
                fence_proxy_async();
                __syncthreads();
            } else {
                bool bad = false;
                if (wg == 0) {
                    float v[16];
                    tmem_ld8(tlane, v);
                    tmem_ld8(tlane + 8, v + 8);
                    tmem_wait_ld();
                    const float *bo = bias + (D - 1) * W;
                    if (valid) {
#pragma unroll
                        for (int o = 0; o < 9; ++o) {
                            if (o < F.out_dim) {
                                const float y = fmaf(F.scale[o], v[o] + bo[o], F.shift[o]);
                                bad |= !isfinite(y);
                                job.out[(size_t)o * ld + p] = y;
                            }
                        }
                    }
                }
                tc_fence_before();
                if (bad) set_status(status, NSF_ERR_NONFINITE);
                __syncthreads();
            }
        }
    }
    goto teardown;

mma_timeout:
    if (tid == 0) set_status(status, NSF_ERR_ITER_CAP);
    // bounded: let the outstanding MMA finish before the memory is released
    mbar_wait(bar_mma, phase ^ 1u);

teardown:
    // a CTA must not leave while its weight copy may still be landing
    if (!weights_ready) mbar_wait(bar_w, 0);
    __syncthreads();
    if (tid < 32) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

size_t value_smem_bytes(int width, int depth) {
    TcLayout L = tc_layout(width, depth);
    if ((size_t)L.total + 64 > (size_t)kMaxSmem) return 0;
    return (size_t)L.total;
}

}  // namespace

// Shared memory a field needs on the tensor-core path (value and Jacobian
// kernels); 0 if it does not fit or the width is not supported.
size_t tc_smem_bytes(int r, int width, int depth) {
    if (width % 64 || width > 256 || depth < 2) return 0;
    const size_t v = value_smem_bytes(width, depth);
    const size_t j = jac_tc_smem_bytes(r, width, depth);
    if (v == 0 || j == 0) return 0;
    return v > j ? v : j;
}

cudaError_t launch_fields_tc(const FieldsDev &fd, const float *X, int n, int ld, int njobs,
                             const FieldJob *jobs, int *status, cudaStream_t s) {
    TcJobs tj;
    tj.njobs = njobs;
    size_t sm = 0;
    for (int i = 0; i < njobs; ++i) {
        tj.job[i] = jobs[i];
        const FieldDev &F = fd.f[jobs[i].field];
        const size_t b = value_smem_bytes(F.width, F.depth);
        if (b == 0) return cudaErrorInvalidValue;
        sm = b > sm ? b : sm;
    }
    static bool attr_done = false;
    set_max_dynamic_smem(k_fields_tc, attr_done);
    const int tiles = (n + kM - 1) / kM;
    int per_job = sm_count() / njobs;
    if (per_job < 1) per_job = 1;
    if (per_job > tiles) per_job = tiles;
    dim3 grid(per_job, njobs);
    k_fields_tc<<<grid, kThreads, sm, s>>>(fd, X, n, ld, tj, status);
    return cudaGetLastError();
}

}  // namespace nsf
