// BF16 field networks on the tcgen05 tensor cores (precision NSF_PREC_BF16).
//
// Paper §4.2-§4.4, App. E (fields are ELU MLPs on [X; z]), §5.1 (inference on
// the integration particles) and §5.3 (g and dg/dz on the sample particles).
//
// One CTA = eight warpgroups (1024 threads).  Thread t owns row t % 128 of a
// 128-row tile (TMEM lane t % 128) and the column eighth t / 128 of every
// layer, so each scheduler keeps eight warps to hide latency.  Per tile:
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
// Biases of the hidden and output layers ride in the MMA: the A operand carries
// 16 extra K columns, two of them 1 on value rows (0 on tangent rows), and the
// weight operand holds each bias split into a bf16 head and a bf16 tail there,
// so the bias keeps ~16 significant bits and the epilogue needs no bias add.
//
// Jacobian mode (Gauss-Newton): each point owns L consecutive rows (L the
// smallest power of two >= 1 + r, so they sit in one warp): its value row and
// one forward-mode tangent row per latent component.  Tangent rows share the
// GEMMs (and get no bias); their activation is ELU'(a_value) * t, which they
// take from their value row by a warp shuffle, so all rows run the same code.
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
// One layer [rows][k] (fp32 host values) and its bias [rows] in the bf16
// tensor-core operand order, K-major no-swizzle core matrices, with 16 extra K
// columns: column k holds bf16(b), column k + 1 holds bf16(b - bf16(b)), the
// rest zero; rows are zero-padded to rows_pad.  Core (n / 8, c / 8) sits at
// ((c / 8) * rows_pad / 8 + n / 8) * 64 elements.
size_t tc_layer_elems(int rows_pad, int k) { return (size_t)rows_pad * (k + 16); }

void tc_pack_layer(const float *W, const float *b, int rows, int rows_pad, int k,
                   __nv_bfloat16 *dst) {
    const int g = rows_pad / 8;
    const int ka = k + 16;
    for (int n = 0; n < rows_pad; ++n) {
        const float bias = n < rows ? b[n] : 0.f;
        const __nv_bfloat16 head = __float2bfloat16_rn(bias);
        const __nv_bfloat16 tail = __float2bfloat16_rn(bias - __bfloat162float(head));
        for (int c = 0; c < ka; ++c) {
            __nv_bfloat16 v;
            if (c < k) v = __float2bfloat16_rn(n < rows ? W[(size_t)n * k + c] : 0.f);
            else if (c == k) v = head;
            else if (c == k + 1) v = tail;
            else v = __float2bfloat16_rn(0.f);
            const size_t core = (size_t)(c / 8) * g + (n / 8);
            dst[core * 64 + (n % 8) * 8 + (c % 8)] = v;
        }
    }
}

namespace {

constexpr int kM = 128;
constexpr int kWG = 8;                    // warpgroups; each owns an eighth of the columns
constexpr int kWgThreads = 128;
constexpr int kThreads = kWG * kWgThreads;
constexpr int kGroup = 8;                 // columns per epilogue group (one core-matrix row)
constexpr int kMaxSmem = 227 * 1024;

// Shared-memory carve of one CTA (byte offsets from a 1024-aligned base).
struct TcLayout {
    int a, blob, w0v, w0t, o3, part, pe, bars, tmem, total;
};

__host__ __device__ inline int align_to(int v, int a) { return (v + a - 1) / a * a; }

// Operand sizes: A is 128 x (W + 16) bf16; each hidden layer W x (W + 16);
// the output layer 16 x (W + 16).
__host__ __device__ inline TcLayout tc_layout(int r, int W, int D) {
    TcLayout L;
    int o = 0;
    L.a = o;    o = align_to(o + kM * (W + 16) * 2, 128);
    L.blob = o; o = align_to(o + (D - 1) * W * (W + 16) * 2 + 16 * (W + 16) * 2, 128);
    L.w0v = o;  o = align_to(o + W * 16, 16);                 // float4 {w_x, w_y, w_z, c0}
    L.w0t = o;  o = align_to(o + r * (W + 1) * 4, 16);        // tangent inputs W0[:, 3 + k]
    L.o3 = o;   o = align_to(o + kM * 3 * 4, 16);
    L.part = o; o = align_to(o + (kGnStrideMax) * 8, 16);
    L.pe = o;   o = align_to(o + kThreads * 8, 16);
    L.bars = o; o = align_to(o + 2 * 8, 16);
    L.tmem = o; o = align_to(o + 16, 16);
    L.total = o + 1024;   // room to align the dynamic base to 1024 bytes
    return L;
}

// ------------------------------------------------------------ PTX ---------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
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
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, phase))
        if (global_ns() - t0 > kWaitNs) return false;
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

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}


// Store 8 activations of row m (columns c .. c + 7, c a multiple of 8) as bf16
// into the A tile: one 16-byte row of one core matrix.
__device__ __forceinline__ void store_a8(uint8_t *A, int m, int c, const float *h) {
    uint4 q;
    __nv_bfloat162 b0 = __floats2bfloat162_rn(h[0], h[1]);
    __nv_bfloat162 b1 = __floats2bfloat162_rn(h[2], h[3]);
    __nv_bfloat162 b2 = __floats2bfloat162_rn(h[4], h[5]);
    __nv_bfloat162 b3 = __floats2bfloat162_rn(h[6], h[7]);
    q.x = *reinterpret_cast<uint32_t *>(&b0);
    q.y = *reinterpret_cast<uint32_t *>(&b1);
    q.z = *reinterpret_cast<uint32_t *>(&b2);
    q.w = *reinterpret_cast<uint32_t *>(&b3);
    *reinterpret_cast<uint4 *>(A + (((c >> 3) * (kM / 8) + (m >> 3)) * 128 + (m & 7) * 16)) = q;
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

// Activation of kGroup pre-activations of one row.  Value rows: ELU.  Tangent
// rows (Jacobian mode): ELU'(pre-activation of the point's value row) * t, the
// derivative taken from the value lane `vlane` of the same warp by a shuffle.
// Every lane runs the same instructions.
template <int MODE>
__device__ __forceinline__ void activate_group(float *v, bool value_row, int vlane) {
#pragma unroll
    for (int i = 0; i < kGroup; ++i) {
        float g;
        const float h = elu_fast(v[i], g);
        if (MODE == 0) {
            v[i] = h;
        } else {
            const float gv = __shfl_sync(0xffffffffu, g, vlane);
            v[i] = value_row ? h : gv * v[i];
        }
    }
}

// Rows per point: 1 in value mode; in Jacobian mode the smallest power of two
// >= 1 + r, so that a point's rows (value row first) share one warp.
__host__ __device__ __forceinline__ int rows_per_point(int mode, int r) {
    if (mode == 0) return 1;
    int L = 2;
    while (L < 1 + r) L <<= 1;
    return L;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_mlp_tc(const __grid_constant__ FieldsDev fd, const float *__restrict__ X, int n, int ld,
         const __grid_constant__ TcJobs jobs, const double *zj, float *u, float *dudz,
         const __grid_constant__ GnArgs gn, int gn_on, int pts_per_tile, int *status) {
    extern __shared__ uint8_t smem_dyn[];
    __shared__ GnShared gsh;
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);

    const int fidx = MODE == 0 ? jobs.job[blockIdx.y].field : NSF_FIELD_G;
    const FieldDev &F = fd.f[fidx];
    const int W = F.width, D = F.depth, r = fd.r;
    const int KA = W + 16;                   // K of every tensor-core product
    const int Lp = rows_per_point(MODE, r);
    // points per tile: all 128 rows in value mode; in Jacobian mode the host
    // may use fewer rows per tile to spread a small point set over more SMs
    const int P = pts_per_tile;
    const int tiles = (n + P - 1) / P;
    const int tid = threadIdx.x;
    const int wg = tid >> 7;                 // warpgroup: column quarter
    const int row = tid & (kM - 1);          // tile row == TMEM lane
    const int wq = (tid >> 5) & 3;           // warp within the warpgroup
    const int cw = W / kWG;                  // columns per warpgroup (multiple of 8)
    const int cbeg = wg * cw;
    const int ldt = W + 1;                   // padded row of the tangent inputs
    const TcLayout L = tc_layout(r, W, D);
    uint8_t *A = base + L.a;
    uint8_t *blob = base + L.blob;
    float4 *W0v = reinterpret_cast<float4 *>(base + L.w0v); // [W] {W0[j][0..2], c0[j]}
    float *W0t = reinterpret_cast<float *>(base + L.w0t);    // [r][W + 1]: W0[j][3 + k]
    float *O3 = reinterpret_cast<float *>(base + L.o3);      // [128][3]
    double *part = reinterpret_cast<double *>(base + L.part);
    double *pe = reinterpret_cast<double *>(base + L.pe);    // [kThreads]
    uint64_t *bar_w = reinterpret_cast<uint64_t *>(base + L.bars);
    uint64_t *bar_mma = bar_w + 1;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(base + L.tmem);
    uint32_t ncols = 32;
    while ((int)ncols < W) ncols <<= 1;
    const int n_iter = (MODE == 1 && gn_on) ? gn.iters : 1;

    if (tid == 0) {
        mbar_init(bar_w, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) tmem_alloc(tmem_holder, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    // Weights: one bulk copy of the packed blob, issued by thread 0; it lands
    // while the CTA prepares its FP32 data and the first tile's input layer.
    if (tid == 0) {
        const uint32_t bytes = (uint32_t)F.tc_blob_bytes;
        mbar_expect_tx(bar_w, bytes);
        const uint8_t *src = reinterpret_cast<const uint8_t *>(F.tc_blob);
        for (uint32_t off = 0; off < bytes; off += 32768u) {
            uint32_t len = bytes - off < 32768u ? bytes - off : 32768u;
            bulk_g2s(blob + off, src + off, len, bar_w);
        }
    }
    const int in0 = 3 + r;
    for (int j = tid; j < W; j += kThreads) {
        const float *w = F.W0 + (size_t)j * in0;
        W0v[j] = make_float4(w[0], w[1], w[2], 0.f);
        for (int k = 0; k < r; ++k) W0t[k * ldt + j] = w[3 + k];
    }
    for (int idx = tid; idx < kM * KA / 8; idx += kThreads)
        reinterpret_cast<uint4 *>(A)[idx] = make_uint4(0u, 0u, 0u, 0u);
    const int T = r * (r + 1) / 2, stride = T + r + 1;
    bool ok = true;
    bool weights_ready = false;

    const uint32_t a_addr = smem_u32(A);
    const uint32_t b_addr = smem_u32(blob);
    const uint32_t lbo_a = (kM / 8) * 128;
    const uint32_t lbo_w = (uint32_t)(W / 8) * 128;
    const uint32_t idesc_h = idesc_bf16(kM, W);
    const uint32_t idesc_o = idesc_bf16(kM, 16);
    const uint32_t tlane = tmem + ((uint32_t)(wq * 32) << 16);
    uint32_t phase = 0;
    // this thread's point and slot
    const int slot = row & (Lp - 1);
    const int lp = row / Lp;
    const bool value_row = slot == 0;
    const bool live_row = slot < 1 + r && lp < P;   // padding rows stay zero
    const bool live_warp = (row & ~31) < P * Lp;     // warps with no tile row skip the epilogue
    const int vlane = (row & 31) & ~(Lp - 1);

    // Gauss-Newton: every CTA carries z in shared memory from iteration to
    // iteration (it solves each iteration's system itself)
    if (MODE == 1 && gn_on && tid < r) gsh.z[tid] = gsh.z0[tid] = __ldcg(&gn.z_start[tid]);

    for (int it = 0; it < n_iter; ++it) {
        const double *z = MODE == 0 ? jobs.job[blockIdx.y].z : zj;
        __syncthreads();
        for (int j = tid; j < W; j += kThreads) {
            float a = F.b[0][j];
            for (int k = 0; k < r; ++k) {
                const double zk = (MODE == 1 && gn_on) ? gsh.z[k] : __ldcg(&z[k]);
                a = fmaf(W0t[k * ldt + j], (float)zk, a);
            }
            W0v[j].w = a;
        }
        if (MODE == 1)
            for (int e = tid; e < stride; e += kThreads) part[e] = 0.0;
        __syncthreads();

        for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
            const int p0 = tile * P;
            const int p = p0 + lp;
            const bool valid = live_row && p < n;
            // ---- layer 0 on the CUDA cores (this thread: its row, its columns)
            float x0 = 0.f, x1 = 0.f, x2 = 0.f;
            if (valid && value_row) {
                x0 = X[p];
                x1 = X[ld + p];
                x2 = X[2 * ld + p];
            }
            const float *w0t = W0t + (live_row && !value_row ? (slot - 1) * ldt : 0);
            for (int cc = cbeg; live_warp && cc < cbeg + cw; cc += kGroup) {
                float v[kGroup];
#pragma unroll
                for (int i = 0; i < kGroup; ++i) {
                    const int j = cc + i;
                    if (value_row) {
                        const float4 w = W0v[j];
                        v[i] = fmaf(w.x, x0, fmaf(w.y, x1, fmaf(w.z, x2, w.w)));
                    } else {
                        v[i] = live_row ? w0t[j] : 0.f;
                    }
                }
                activate_group<MODE>(v, value_row, vlane);
                store_a8(A, row, cc, v);
            }
            if (wg == 0 && live_warp) {
                // bias columns of the A operand: 1, 1 on value rows, 0 elsewhere
                float ones[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                ones[0] = ones[1] = value_row ? 1.f : 0.f;
                store_a8(A, row, W, ones);
                ones[0] = ones[1] = 0.f;
                store_a8(A, row, W + 8, ones);
            }
            fence_proxy_async();
            __syncthreads();
            if (!weights_ready) {
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
                    const uint32_t boff = (uint32_t)((l - 1) * W * KA * 2);
                    const uint32_t lbo_b = out_layer ? 2u * 128u : lbo_w;
                    const uint32_t idesc = out_layer ? idesc_o : idesc_h;
                    for (int ks = 0; ks < KA / 16; ++ks) {
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
                    for (int cc = cbeg; live_warp && cc < cbeg + cw; cc += kGroup) {
                        float v[kGroup];
                        tmem_ld8(tlane + cc, v);
                        tmem_wait_ld();
                        activate_group<MODE>(v, value_row, vlane);
                        store_a8(A, row, cc, v);
                    }
                    tc_fence_before();
                    fence_proxy_async();
                    __syncthreads();
                } else {
                    bool bad = false;
                    if (wg == 0 && live_warp) {
                        float v[16];
                        tmem_ld8(tlane, v);
                        tmem_ld8(tlane + 8, v + 8);
                        tmem_wait_ld();
                        if (MODE == 0) {
                            const FieldJob &job = jobs.job[blockIdx.y];
                            if (valid) {
#pragma unroll
                                for (int o = 0; o < 9; ++o) {
                                    if (o < F.out_dim) {
                                        float y = fmaf(F.scale[o], v[o], F.shift[o]);
                                        bad |= !isfinite(y);
                                        job.out[(size_t)o * ld + p] = y;
                                    }
                                }
                            }
                        } else {
#pragma unroll
                            for (int a = 0; a < 3; ++a) {
                                float y = value_row ? fmaf(F.scale[a], v[a], F.shift[a])
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
                    }
                    tc_fence_before();
                    if (bad) set_status(status, NSF_ERR_NONFINITE);
                    __syncthreads();
                    if (MODE == 1 && gn_on) {
                        // float64 partial normal equations of this tile's points:
                        // thread t takes entry e = t % stride for the points
                        // q = t / stride, + G, ... (G = threads per entry), then
                        // one thread per entry sums the G partial values in order
                        const int npts = max(0, min(P, n - p0));
                        const int G = kThreads / stride;
                        const int e = tid % stride, g0 = tid / stride;
                        if (g0 < G) {
                            int ii = -1, jj = -1;
                            if (e < T) {
                                int i = 0, off = 0;
                                while (e >= off + (r - i)) { off += r - i; ++i; }
                                ii = i;
                                jj = i + (e - off);
                            } else if (e < T + r) {
                                ii = e - T;
                            }
                            double s = 0.0;
                            for (int q = g0; q < npts; q += G) {
                                const float *vr = O3 + (q * Lp) * 3;
                                if (e < T) {
                                    const float *ri = O3 + (q * Lp + 1 + ii) * 3;
                                    const float *rj = O3 + (q * Lp + 1 + jj) * 3;
                                    s = fma((double)ri[0], (double)rj[0], s);
                                    s = fma((double)ri[1], (double)rj[1], s);
                                    s = fma((double)ri[2], (double)rj[2], s);
                                } else if (e < T + r) {
                                    const float *ri = O3 + (q * Lp + 1 + ii) * 3;
                                    s = fma((double)ri[0], (double)vr[0], s);
                                    s = fma((double)ri[1], (double)vr[1], s);
                                    s = fma((double)ri[2], (double)vr[2], s);
                                } else {
                                    s = fma((double)vr[0], (double)vr[0], s);
                                    s = fma((double)vr[1], (double)vr[1], s);
                                    s = fma((double)vr[2], (double)vr[2], s);
                                }
                            }
                            pe[g0 * stride + e] = s;
                        }
                        __syncthreads();
                        if (tid < stride) {
                            double s = part[tid];
                            for (int g = 0; g < G; ++g) s += pe[g * stride + tid];
                            part[tid] = s;
                        }
                    }
                    __syncthreads();
                }
            }
        }

        if (MODE == 1 && gn_on) {
            // Gauss-Newton iteration `it`: all CTAs' partials summed behind a
            // grid barrier (cooperative launch), then every CTA solves
            __syncthreads();
            if (!gn_allreduce_solve(gn, r, it, status, gsh, part)) goto teardown;
        }
    }

teardown:
    // a CTA must not leave while its weight copy may still be landing
    if (!weights_ready) mbar_wait(bar_w, 0);
    __syncthreads();
    if (tid < 32) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
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
    if (width % 64 || width > 256) return 0;
    return (size_t)L.total;
}

// Jacobian mode: points per tile.  A full tile holds 128 / L points; for
// small point sets fewer points per tile (whole warps of rows) spread the work
// over more SMs, which shortens the latency of a Gauss-Newton iteration.
int jac_points_per_tile(const FieldsDev &fd, int n) {
    const int Lp = rows_per_point(1, fd.r);
    const int pmax = kM / Lp;
    const int per_warp = 32 / Lp > 0 ? 32 / Lp : 1;      // points per 32 rows
    int P = (n + sm_count() - 1) / sm_count();
    P = (P + per_warp - 1) / per_warp * per_warp;
    if (P > pmax) P = pmax;
    if (P < 1) P = 1;
    return P;
}

int jac_grid_size_tc(const FieldsDev &fd, int n) {
    const int P = jac_points_per_tile(fd, n);
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
                                           kM, status);
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
    int gn_on = gn ? 1 : 0;
    const int grid = jac_grid_size_tc(fd, n);
    // The Gauss-Newton run waits between iterations on a grid barrier, so all
    // CTAs must be co-resident: cooperative launch (one CTA per SM).
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = gn_on ? 1 : 0;
    const int P = jac_points_per_tile(fd, n);
    return cudaLaunchKernelEx(&cfg, k_mlp_tc<1>, fd, X, n, ld, tj, z, u, dudz, g, gn_on, P, status);
}

}  // namespace nsf
