// BF16 field networks on the tcgen05 tensor cores (precision NSF_PREC_BF16).
//
// Paper §4.2-§4.4, App. E (fields are ELU MLPs on [X; z]), §5.1 (inference on
// the integration particles) and §5.3 (g and dg/dz on the sample particles).
//
// One CTA = one warpgroup (128 threads); thread t owns row t of a 128-row tile
// and TMEM lane t.  Per tile:
//   layer 0 (K = 3 + r)  on the CUDA cores in FP32, written as bf16 into the
//                        shared-memory A operand;
//   hidden layers        tcgen05.mma M = 128, N = width, K = 16 steps, FP32
//                        accumulator in tensor memory; the epilogue (bias, ELU,
//                        bf16 convert) reads it with tcgen05.ld and rewrites the
//                        A operand in place for the next layer;
//   output layer         the same MMA with N = 16 (out_dim padded with zero rows).
// All weights of the CTA's field stay resident in shared memory (one bulk copy
// per CTA, an mbarrier with a transaction count); persistent CTAs loop over
// tiles.  Every wait on an mbarrier is bounded by time: on expiry the kernel
// records NSF_ERR_ITER_CAP, waits (bounded) for its outstanding operations,
// frees its tensor memory and returns.
//
// Jacobian mode (Gauss-Newton): each point owns S = 1 + r rows, its value row
// and one forward-mode tangent row per latent component.  Tangent rows share
// the GEMMs (without bias); their activation is ELU'(a_value) * t, where the
// value row publishes ELU'(a_value) through shared memory, so only value rows
// evaluate exp().
//
// Operand layout (K-major, no swizzle): 8-row x 16-byte core matrices stored as
// contiguous 128-byte blocks.  A (activations, 128 x width): core (m8, k8) at
// (k8 * 16 + m8) * 128 bytes, i.e. stride 128 B between 8-row groups (SBO) and
// 2048 B between K-adjacent cores (LBO).  B (weights, N x width): core (n8, k8)
// at (k8 * N / 8 + n8) * 128 bytes: SBO 128 B, LBO 16 N bytes.
#include "device_common.cuh"
#include "gn_solve.cuh"

namespace nsf {

// ------------------------------------------------------------ packing ----
void tc_pack_matrix(const float *W, int rows, int rows_pad, int k, __nv_bfloat16 *dst) {
    const int g = rows_pad / 8;
    for (int n = 0; n < rows_pad; ++n)
        for (int c = 0; c < k; ++c) {
            size_t core = (size_t)(c / 8) * g + (n / 8);
            size_t idx = core * 64 + (n % 8) * 8 + (c % 8);
            float v = n < rows ? W[(size_t)n * k + c] : 0.f;
            dst[idx] = __float2bfloat16_rn(v);
        }
}

namespace {

constexpr int kM = 128;
constexpr int kThreads = 128;
constexpr int kChunkCols = 32;
constexpr int kMaxSmem = 227 * 1024;
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s bound on any wait

// Shared-memory carve of one CTA (byte offsets from a 1024-aligned base).
struct TcLayout {
    int a, blob, w0, c0, bias, dv, o3, part, bars, tmem, total;
};

__host__ __device__ inline int align_to(int v, int a) { return (v + a - 1) / a * a; }

__host__ __device__ inline TcLayout tc_layout(int r, int W, int D) {
    TcLayout L;
    int o = 0;
    L.a = o;    o = align_to(o + kM * W * 2, 128);
    L.blob = o; o = align_to(o + (D - 1) * W * W * 2 + 16 * W * 2, 128);
    L.w0 = o;   o = align_to(o + (3 + r) * W * 4, 16);
    L.c0 = o;   o = align_to(o + W * 4, 16);
    L.bias = o; o = align_to(o + ((D - 1) * W + 16) * 4, 16);
    L.dv = o;   o = align_to(o + (kM / 2) * kChunkCols * 4, 16);
    L.o3 = o;   o = align_to(o + kM * 3 * 4, 16);
    L.part = o; o = align_to(o + (kMaxR * (kMaxR + 1) / 2 + kMaxR + 1) * 8, 16);
    L.bars = o; o = align_to(o + 2 * 8, 16);
    L.tmem = o; o = align_to(o + 16, 16);
    L.total = o + 1024;   // room to align the dynamic base to 1024 bytes
    return L;
}

// ------------------------------------------------------------ PTX ---------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait for the given phase parity; false if it did not complete in time.
__device__ bool mbar_wait(uint64_t *bar, uint32_t phase) {
    if (mbar_try_wait(bar, phase)) return true;
    const unsigned long long t0 = now_ns();
    while (!mbar_try_wait(bar, phase))
        if (now_ns() - t0 > kWaitNs) return false;
    return true;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(holder)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;          // descriptor version of the tcgen05 family
    return d;                        // base offset 0, swizzle none
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 D, both K-major.
__host__ __device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
    return (1u << 4)                 // D format F32
           | (1u << 7)               // A format BF16
           | (1u << 10)              // B format BF16
           | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void named_sync(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kThreads) : "memory");
}

// Store 32 activations of row m (columns c0 .. c0 + 31) as bf16 into the A tile.
__device__ __forceinline__ void store_a_chunk(uint8_t *A, int m, int c0, const float (&h)[32]) {
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const int k8 = (c0 >> 3) + g;
        uint4 q;
        __nv_bfloat162 b0 = __floats2bfloat162_rn(h[8 * g + 0], h[8 * g + 1]);
        __nv_bfloat162 b1 = __floats2bfloat162_rn(h[8 * g + 2], h[8 * g + 3]);
        __nv_bfloat162 b2 = __floats2bfloat162_rn(h[8 * g + 4], h[8 * g + 5]);
        __nv_bfloat162 b3 = __floats2bfloat162_rn(h[8 * g + 6], h[8 * g + 7]);
        q.x = *reinterpret_cast<uint32_t *>(&b0);
        q.y = *reinterpret_cast<uint32_t *>(&b1);
        q.z = *reinterpret_cast<uint32_t *>(&b2);
        q.w = *reinterpret_cast<uint32_t *>(&b3);
        *reinterpret_cast<uint4 *>(A + ((k8 * (kM / 8) + (m >> 3)) * 128 + (m & 7) * 16)) = q;
    }
}

struct TcJobs {
    int njobs;
    FieldJob job[4];
};

// ELU on the BF16 path: one exponential per element (the result is rounded to
// bf16 right after, so exp(a) - 1 is as good as expm1 here).
__device__ __forceinline__ float elu_fast(float a, float &grad) {
    const float e = __expf(fminf(a, 0.f));
    grad = a > 0.f ? 1.f : e;
    return a > 0.f ? a : e - 1.f;
}

// Activation of one 32-column chunk for all rows: value rows h = ELU(pre),
// tangent rows h = ELU'(pre of the point's value row) * pre.  In Jacobian mode
// the value rows publish ELU'(pre) through DV[column][point] (two named
// barriers; consecutive points are consecutive words, so no bank conflicts).
template <int MODE>
__device__ __forceinline__ void activate_chunk(float (&v)[32], bool value_row, int lp,
                                               float *DV) {
    float g;
    if (MODE == 0) {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = elu_fast(v[i], g);
        return;
    }
    if (value_row) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            v[i] = elu_fast(v[i], g);
            DV[i * (kM / 2) + lp] = g;
        }
    }
    named_sync(1);
    if (!value_row) {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] *= DV[i * (kM / 2) + lp];
    }
    named_sync(1);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_mlp_tc(const __grid_constant__ FieldsDev fd, const float *__restrict__ X, int n, int ld,
         const __grid_constant__ TcJobs jobs, const double *zj, float *u, float *dudz,
         const __grid_constant__ GnArgs gn, int gn_on, int *status) {
    extern __shared__ uint8_t smem_dyn[];
    __shared__ GnShared gsh;
    __shared__ int s_fail;
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);

    const int fidx = MODE == 0 ? jobs.job[blockIdx.y].field : NSF_FIELD_G;
    const double *z = MODE == 0 ? jobs.job[blockIdx.y].z : zj;
    const FieldDev &F = fd.f[fidx];
    const int W = F.width, D = F.depth, r = fd.r;
    const int S = MODE == 0 ? 1 : 1 + r;
    const int P = kM / S;
    const int tiles = (n + P - 1) / P;
    const int tid = threadIdx.x, warp = tid >> 5;
    const TcLayout L = tc_layout(r, W, D);
    uint8_t *A = base + L.a;
    uint8_t *blob = base + L.blob;
    float *W0s = reinterpret_cast<float *>(base + L.w0);     // [3 + r][W]
    float *c0 = reinterpret_cast<float *>(base + L.c0);      // [W]
    float *bias = reinterpret_cast<float *>(base + L.bias);  // [D - 1][W], then out [16]
    float *DV = reinterpret_cast<float *>(base + L.dv);
    float *O3 = reinterpret_cast<float *>(base + L.o3);      // [128][3]
    double *part = reinterpret_cast<double *>(base + L.part);
    uint64_t *bar_w = reinterpret_cast<uint64_t *>(base + L.bars);
    uint64_t *bar_mma = bar_w + 1;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(base + L.tmem);
    uint32_t ncols = 32;
    while ((int)ncols < W) ncols <<= 1;

    if (tid == 0) {
        s_fail = 0;
        mbar_init(bar_w, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_holder, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    // Weights: one bulk copy of the packed blob, issued by thread 0.
    if (tid == 0) {
        const uint32_t bytes = (uint32_t)F.tc_blob_bytes;
        mbar_expect_tx(bar_w, bytes);
        const uint8_t *src = reinterpret_cast<const uint8_t *>(F.tc_blob);
        for (uint32_t off = 0; off < bytes; off += 32768u) {
            uint32_t len = bytes - off < 32768u ? bytes - off : 32768u;
            bulk_g2s(blob + off, src + off, len, bar_w);
        }
    }
    // FP32 side data while the copy is in flight.
    const int in0 = 3 + r;
    for (int idx = tid; idx < in0 * W; idx += kThreads) {
        int d = idx / W, j = idx - d * W;
        W0s[idx] = F.W0[(size_t)j * in0 + d];
    }
    for (int l = 1; l < D; ++l)
        for (int j = tid; j < W; j += kThreads) bias[(l - 1) * W + j] = F.b[l][j];
    for (int o = tid; o < 16; o += kThreads) bias[(D - 1) * W + o] = o < F.out_dim ? F.b[D][o] : 0.f;
    const int T = r * (r + 1) / 2, stride = T + r + 1;
    if (MODE == 1)
        for (int e = tid; e < stride; e += kThreads) part[e] = 0.0;
    __syncthreads();
    for (int j = tid; j < W; j += kThreads) {
        float a = F.b[0][j];
        for (int k = 0; k < r; ++k) a = fmaf(W0s[(3 + k) * W + j], (float)z[k], a);
        c0[j] = a;
    }
    bool ok = true;
    bool weights_ready = false;
    __syncthreads();

    {
        const uint32_t a_addr = smem_u32(A);
        const uint32_t b_addr = smem_u32(blob);
        const uint32_t lbo_a = (kM / 8) * 128;
        const uint32_t lbo_w = (uint32_t)(W / 8) * 128;
        const uint32_t idesc_h = idesc_bf16(kM, W);
        const uint32_t idesc_o = idesc_bf16(kM, 16);
        const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);
        uint32_t phase = 0;
        const int row = tid;
        const int lp = row / S, slot = row - lp * S;
        const bool value_row = slot == 0;

        for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
            const int p0 = tile * P;
            const int p = p0 + lp;
            const bool valid = lp < P && p < n;
            // ---- layer 0 on the CUDA cores
            float x0 = 0.f, x1 = 0.f, x2 = 0.f;
            if (valid && value_row) {
                x0 = X[p];
                x1 = X[ld + p];
                x2 = X[2 * ld + p];
            }
            for (int cc = 0; cc < W; cc += kChunkCols) {
                float v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int j = cc + i;
                    if (value_row)
                        v[i] = fmaf(W0s[j], x0, fmaf(W0s[W + j], x1, fmaf(W0s[2 * W + j], x2, c0[j])));
                    else
                        v[i] = W0s[(3 + slot - 1) * W + j];
                }
                activate_chunk<MODE>(v, value_row, lp, DV);
                store_a_chunk(A, row, cc, v);
            }
            fence_proxy_async();
            __syncthreads();
            if (!weights_ready) {
                // the weight copy overlapped the first tile's input layer
                ok = mbar_wait(bar_w, 0);
                if (!__syncthreads_and(ok)) {
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
                    const uint32_t lbo_b = out_layer ? 2u * 128u : lbo_w;
                    const uint32_t idesc = out_layer ? idesc_o : idesc_h;
                    for (int ks = 0; ks < W / 16; ++ks) {
                        uint64_t ad = smem_desc(a_addr + ks * 2 * lbo_a, lbo_a, 128);
                        uint64_t bd = smem_desc(b_addr + boff + ks * 2 * lbo_b, lbo_b, 128);
                        mma_bf16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
                    }
                    mma_commit(bar_mma);
                }
                ok = mbar_wait(bar_mma, phase);
                phase ^= 1u;
                if (!__syncthreads_and(ok)) {
                    if (tid == 0) set_status(status, NSF_ERR_ITER_CAP);
                    mbar_wait(bar_mma, phase ^ 1u);
                    goto teardown;
                }
                tc_fence_after();
                if (!out_layer) {
                    const float *bl = bias + (l - 1) * W;
                    for (int cc = 0; cc < W; cc += kChunkCols) {
                        float v[32];
                        tmem_ld32(tlane + cc, v);
                        if (value_row) {
#pragma unroll
                            for (int i = 0; i < 32; ++i) v[i] += bl[cc + i];
                        }
                        activate_chunk<MODE>(v, value_row, lp, DV);
                        store_a_chunk(A, row, cc, v);
                    }
                    tc_fence_before();
                    fence_proxy_async();
                    __syncthreads();
                } else {
                    float v[16];
                    tmem_ld16(tlane, v);
                    tc_fence_before();
                    const float *bo = bias + (D - 1) * W;
                    bool bad = false;
                    if (MODE == 0) {
                        const FieldJob &job = jobs.job[blockIdx.y];
                        if (valid) {
                            for (int o = 0; o < F.out_dim; ++o) {
                                float y = fmaf(F.scale[o], v[o] + bo[o], F.shift[o]);
                                bad |= !isfinite(y);
                                job.out[(size_t)o * ld + p] = y;
                            }
                        }
                    } else {
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            float y = value_row ? fmaf(F.scale[a], v[a] + bo[a], F.shift[a])
                                                : F.scale[a] * v[a];
                            if (valid) bad |= !isfinite(y);
                            if (valid && value_row) {
                                if (u) u[(size_t)a * ld + p] = y;
                                if (gn_on) y -= gn.target[(size_t)a * gn.target_ld + p];
                            }
                            if (valid && !value_row && dudz)
                                dudz[(size_t)(a * r + slot - 1) * ld + p] = y;
                            O3[row * 3 + a] = valid ? y : 0.f;
                        }
                    }
                    if (bad) set_status(status, NSF_ERR_NONFINITE);
                    __syncthreads();
                    if (MODE == 1 && gn_on) {
                        // float64 partial normal equations of this tile's points
                        const int npts = max(0, min(P, n - p0));
                        for (int e = tid; e < stride; e += kThreads) {
                            double s = 0.0;
                            if (e < T) {
                                int i = 0, off = 0;
                                while (e >= off + (r - i)) { off += r - i; ++i; }
                                const int j = i + (e - off);
                                for (int q = 0; q < npts; ++q)
                                    for (int a = 0; a < 3; ++a)
                                        s = fma((double)O3[(q * S + 1 + i) * 3 + a],
                                                (double)O3[(q * S + 1 + j) * 3 + a], s);
                            } else if (e < T + r) {
                                const int k = e - T;
                                for (int q = 0; q < npts; ++q)
                                    for (int a = 0; a < 3; ++a)
                                        s = fma((double)O3[(q * S + 1 + k) * 3 + a],
                                                (double)O3[(q * S) * 3 + a], s);
                            } else {
                                for (int q = 0; q < npts; ++q)
                                    for (int a = 0; a < 3; ++a)
                                        s = fma((double)O3[(q * S) * 3 + a],
                                                (double)O3[(q * S) * 3 + a], s);
                            }
                            part[e] += s;
                        }
                    }
                    __syncthreads();
                }
            }
        }
    }

teardown:
    // a CTA must not leave while its weight copy may still be landing
    if (!weights_ready) mbar_wait(bar_w, 0);
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
    if (MODE == 1 && gn_on) {
        for (int e = tid; e < stride; e += kThreads)
            gn.partials[(size_t)blockIdx.x * stride + e] = part[e];
        gn_arrive_and_finish(gn, r, status, gsh);
    }
}

int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

template <int MODE>
void set_smem_attr() {
    static bool done = false;
    if (!done) {
        cudaFuncAttributes fa;
        int stat = 0;
        if (cudaFuncGetAttributes(&fa, k_mlp_tc<MODE>) == cudaSuccess) stat = (int)fa.sharedSizeBytes;
        cudaFuncSetAttribute(k_mlp_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMaxSmem - stat);
        done = true;
    }
}

}  // namespace

size_t tc_smem_bytes(int r, int width, int depth) {
    TcLayout L = tc_layout(r, width, depth);
    const size_t static_bytes = sizeof(GnShared) + 64;
    if ((size_t)L.total + static_bytes > (size_t)kMaxSmem) return 0;
    if (width % 32 || width > 256) return 0;
    return (size_t)L.total;
}

int jac_grid_size_tc(const FieldsDev &fd, int n) {
    const int P = kM / (1 + fd.r);
    const int tiles = (n + P - 1) / P;
    return tiles < sm_count() ? tiles : sm_count();
}

cudaError_t launch_fields_tc(const FieldsDev &fd, const float *X, int n, int ld, int njobs,
                             const FieldJob *jobs, int *status, cudaStream_t s) {
    TcJobs tj;
    tj.njobs = njobs;
    size_t sm = 0;
    for (int i = 0; i < njobs; ++i) {
        tj.job[i] = jobs[i];
        const FieldDev &F = fd.f[jobs[i].field];
        size_t b = tc_smem_bytes(fd.r, F.width, F.depth);
        if (b == 0) return cudaErrorInvalidValue;
        sm = b > sm ? b : sm;
    }
    set_smem_attr<0>();
    const int tiles = (n + kM - 1) / kM;
    int per_job = sm_count() / njobs;
    if (per_job < 1) per_job = 1;
    if (per_job > tiles) per_job = tiles;
    GnArgs none{};
    dim3 grid(per_job, njobs);
    k_mlp_tc<0><<<grid, kThreads, sm, s>>>(fd, X, n, ld, tj, nullptr, nullptr, nullptr, none, 0,
                                           status);
    return cudaGetLastError();
}

cudaError_t launch_jacobian_tc(const FieldsDev &fd, const float *X, int n, int ld,
                               const double *z, float *u, float *dudz, const GnArgs *gn,
                               int *status, cudaStream_t s) {
    const FieldDev &F = fd.f[NSF_FIELD_G];
    size_t sm = tc_smem_bytes(fd.r, F.width, F.depth);
    if (sm == 0) return cudaErrorInvalidValue;
    set_smem_attr<1>();
    TcJobs tj{};
    GnArgs g{};
    if (gn) g = *gn;
    const int grid = jac_grid_size_tc(fd, n);
    k_mlp_tc<1><<<grid, kThreads, sm, s>>>(fd, X, n, ld, tj, z, u, dudz, g, gn ? 1 : 0, status);
    return cudaGetLastError();
}

}  // namespace nsf
