// BF16 field networks on the tcgen05 tensor cores (precision NSF_PREC_BF16).
//
// Paper §4.2-§4.4, App. E (fields are ELU MLPs on [X; z]), §5.1 (inference on
// the integration particles) and §5.3 (g and dg/dz on the sample particles).
//
// One CTA = eight warpgroups (1024 threads) on a 128-row tile; row i of the
// tile is TMEM lane i, which only the warps with (warp index % 4) == i / 32
// can read.  Warpgroup w owns the column eighth [w W / 8, (w + 1) W / 8) of
// every layer.  Per tile:
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
// Value mode (inference): row i of a tile is point i; every thread handles its
// row and its warpgroup's columns.
//
// Jacobian mode (Gauss-Newton): a tile holds P points (P <= 32, r P <= 96).
// Value rows sit in lane quarter 0 (row p), forward-mode tangent rows in
// quarters 1-3 (row 32 + k P + p for latent component k).  Tangent rows share
// the GEMMs (no bias); their activation is ELU'(a_value) * t.  In each
// warpgroup, the quarter-0 warp publishes the value rows' pre-activations of
// the warpgroup's columns in shared memory, all 128 threads of the warpgroup
// turn them into ELU values (for A) and derivatives, and the tangent warps
// scale their rows by those derivatives, with a named barrier per warpgroup
// between the steps.  So the exponentials are spread over the whole
// warpgroup rather than computed in every lane.
//
// Operand layout: K-major with the 128-byte swizzle.  A K-atom is 64 bf16
// columns; within an atom, row n's 128 bytes sit at (n / 8) * 1024 + (n % 8) *
// 128 and its 16-byte chunk c at chunk position c ^ (n % 8).  Atoms of A
// (128 rows) are 16 KB apart, atoms of a weight matrix with N rows N * 128
// bytes apart; every atom starts on a 1024-byte boundary.
#include "device_common.cuh"
#include "gn_ff.cuh"

namespace nsf {

// ------------------------------------------------------------ packing ----
// Byte offset of element (n, k) of a K-major, 128-byte-swizzled operand with
// rows_pad rows.
static size_t sw128_offset(int n, int k, int rows_pad) {
    const int atom = k / 64, kk = k % 64, chunk = kk / 8;
    return (size_t)atom * rows_pad * 128 + (size_t)(n / 8) * 1024 + (n % 8) * 128 +
           ((chunk ^ (n % 8)) * 16) + (kk % 8) * 2;
}

size_t tc_layer_elems(int rows_pad, int k) { return (size_t)rows_pad * k; }

// One layer [rows][k] (fp32 host values, rows zero-padded to rows_pad, k a
// multiple of 64) in the bf16 operand order above.
void tc_pack_layer(const float *W, int rows, int rows_pad, int k, __nv_bfloat16 *dst) {
    for (int n = 0; n < rows_pad; ++n)
        for (int c = 0; c < k; ++c)
            dst[sw128_offset(n, c, rows_pad) / 2] =
                __float2bfloat16_rn(n < rows ? W[(size_t)n * k + c] : 0.f);
}

namespace {

constexpr int kM = 128;
constexpr int kWG = 8;                    // warpgroups; each owns an eighth of the columns
constexpr int kWgThreads = 128;
constexpr int kThreads = kWG * kWgThreads;
constexpr int kGroup = 8;                 // columns per bf16 store (one 16-byte chunk)
constexpr int kMaxSmem = 227 * 1024;
constexpr int kMaxOut = 16;               // output rows of the last MMA (out_dim padded)

// Jacobian mode: points per tile.
__host__ __device__ inline int jac_tile_points(int r) {
    const int p = 96 / r;
    return p < 32 ? p : 32;
}

// Shared-memory carve of one CTA (byte offsets from a 1024-aligned base).
struct TcLayout {
    int a, blob, w0v, w0t, b0, bias, xs, xbuf, o3, bars, tmem, total;
};

__host__ __device__ inline int align_to(int v, int a) { return (v + a - 1) / a * a; }

__host__ __device__ inline TcLayout tc_layout(int r, int W, int D) {
    TcLayout L;
    int o = 0;
    L.a = o;    o = align_to(o + kM * W * 2, 1024);
    L.blob = o; o = align_to(o + (D - 1) * W * W * 2 + kMaxOut * W * 2, 1024);
    L.w0v = o;  o = align_to(o + W * 16, 16);                 // float4 {w_x, w_y, w_z, c0}
    L.w0t = o;  o = align_to(o + r * (W + 1) * 4, 16);        // tangent inputs W0[:, 3 + k]
    L.b0 = o;   o = align_to(o + W * 4, 16);                  // input-layer bias
    L.bias = o; o = align_to(o + D * W * 4, 16);              // hidden biases, then output bias
    L.xs = o;   o = align_to(o + 32 * 16, 16);                // Jacobian tile positions
    L.xbuf = o; o = align_to(o + jac_tile_points(r) * (W + 4) * 4, 16);  // value-row exchange
    L.o3 = o;   o = align_to(o + kM * 3 * 4, 16);
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

// Named barrier of one warpgroup (ids 1 .. 8; id 0 is __syncthreads).
__device__ __forceinline__ void wg_sync(int wg) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + wg), "r"(kWgThreads) : "memory");
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

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset); the leading byte offset is not used
// by this layout (set to 16 bytes).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;          // descriptor version of the tcgen05 family
    d |= (uint64_t)2 << 61;          // swizzle mode: 128 bytes
    return d;
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

// Byte offset of the 16-byte chunk holding columns c .. c + 7 (c % 8 == 0) of
// row m in the A tile.
__device__ __forceinline__ int a_chunk(int m, int c) {
    return (c >> 6) * (kM * 128) + (m >> 3) * 1024 + (m & 7) * 128 +
           ((((c >> 3) & 7) ^ (m & 7)) << 4);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Store 8 activations of row m (columns c .. c + 7) as bf16 into A.
__device__ __forceinline__ void store_a8(uint8_t *A, int m, int c, const float *h) {
    uint4 q;
    q.x = pack_bf16x2(h[0], h[1]);
    q.y = pack_bf16x2(h[2], h[3]);
    q.z = pack_bf16x2(h[4], h[5]);
    q.w = pack_bf16x2(h[6], h[7]);
    *reinterpret_cast<uint4 *>(A + a_chunk(m, c)) = q;
}

// Store 2 activations of row m (columns c, c + 1; c even) as bf16 into A.
__device__ __forceinline__ void store_a2(uint8_t *A, int m, int c, float h0, float h1) {
    *reinterpret_cast<uint32_t *>(A + a_chunk(m, c & ~7) + (c & 7) * 2) = pack_bf16x2(h0, h1);
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

// Jacobian mode, one warpgroup: the value rows' pre-activations of the
// warpgroup's columns are in xbuf[p * XS + c] (p < P, row stride XS = W + 4
// floats, so that rows start in different banks); every thread of the
// warpgroup takes column pairs (point index fastest), writes ELU(a) into A
// (row p) and replaces a by ELU'(a) in xbuf.
// e / P for 0 <= e < 2048 and 1 <= P <= 32, with pinv = ceil(2^16 / P): the
// error of pinv is below 1, times e < 2^16 / P, so the quotient is exact.
__device__ __forceinline__ int div_small(int e, uint32_t pinv) { return (int)(((uint32_t)e * pinv) >> 16); }

__device__ __forceinline__ void wg_value_activation(uint8_t *A, float *xbuf, int XS, int P,
                                                    uint32_t pinv, int cbeg, int cw, int tw) {
    const int pairs = cw >> 1;
    for (int e = tw; e < P * pairs; e += kWgThreads) {
        const int pr = div_small(e, pinv);
        const int p = e - pr * P;
        const int c = cbeg + 2 * pr;
        float2 *x = reinterpret_cast<float2 *>(xbuf + p * XS + c);
        const float2 a = *x;
        float g0, g1;
        const float h0 = elu_fast(a.x, g0), h1 = elu_fast(a.y, g1);
        store_a2(A, p, c, h0, h1);
        *x = make_float2(g0, g1);
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_mlp_tc(const __grid_constant__ FieldsDev fd, const float *__restrict__ X, int n, int ld,
         const __grid_constant__ TcJobs jobs, const double *zj, float *u, float *dudz,
         const __grid_constant__ GnArgs gn, int gn_on, int pts_per_tile, int *status) {
    extern __shared__ uint8_t smem_dyn[];
    __shared__ GnFF gff;
    __shared__ int s_abort;
    // 1024-byte aligned base by pointer arithmetic on the shared array (an
    // integer round trip would hide the address space from the compiler and
    // turn every shared access below into a generic one)
    uint8_t *base = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);

    const int fidx = MODE == 0 ? jobs.job[blockIdx.y].field : NSF_FIELD_G;
    const FieldDev &F = fd.f[fidx];
    const int W = F.width, D = F.depth, r = fd.r;
    const int P = MODE == 0 ? kM : pts_per_tile;   // points per tile
    const uint32_t pinv = (65536u + (uint32_t)P - 1u) / (uint32_t)P;
    const int tiles = (n + P - 1) / P;
    const int tid = threadIdx.x;
    const int wg = tid >> 7;                 // warpgroup: column eighth
    const int tw = tid & (kWgThreads - 1);   // thread within the warpgroup
    const int wq = tw >> 5;                  // lane quarter of this warp
    const int lane = tid & 31;
    const int row = tw;                      // tile row == TMEM lane
    const int cw = W / kWG;                  // columns per warpgroup (multiple of 8)
    const int cbeg = wg * cw;
    const int ldt = W + 1;                   // padded row of the tangent inputs
    const int XS = W + 4;                    // padded row of the value-row exchange
    const TcLayout L = tc_layout(r, W, D);
    uint8_t *A = base + L.a;
    uint8_t *blob = base + L.blob;
    float4 *W0v = reinterpret_cast<float4 *>(base + L.w0v); // [W] {W0[j][0..2], c0[j]}
    float *W0t = reinterpret_cast<float *>(base + L.w0t);    // [r][W + 1]: W0[j][3 + k]
    float *b0s = reinterpret_cast<float *>(base + L.b0);     // [W]
    float *bias = reinterpret_cast<float *>(base + L.bias);  // [D][W]
    float4 *xs = reinterpret_cast<float4 *>(base + L.xs);    // [32] Jacobian tile positions
    float *xbuf = reinterpret_cast<float *>(base + L.xbuf);  // [P][W + 4]
    float *O3 = reinterpret_cast<float *>(base + L.o3);      // [128][3]
    uint64_t *bar_w = reinterpret_cast<uint64_t *>(base + L.bars);
    uint64_t *bar_mma = bar_w + 1;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(base + L.tmem);
    uint32_t ncols = 32;
    while ((int)ncols < W) ncols <<= 1;
    const int n_iter = (MODE == 1 && gn_on) ? gn.iters : 1;

    // role of this thread's row
    //   value mode: point `row` of the tile
    //   Jacobian mode: quarter 0 -> value row of point `lane` (live if lane < P);
    //   quarters 1-3 -> tangent row kt of point lp
    int lp = row, kt = -1;
    bool live = true;
    if (MODE == 1) {
        if (wq == 0) {
            lp = lane;
            live = lane < P;
        } else {
            const int t = row - 32;
            kt = t / P;
            lp = t - kt * P;
            live = kt < r;
        }
    }
    const bool value_row = MODE == 0 || wq == 0;
    const bool live_warp = MODE == 0 || wq == 0 || 32 * (wq - 1) < r * P;

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
        b0s[j] = F.b[0][j];
        for (int k = 0; k < r; ++k) W0t[k * ldt + j] = w[3 + k];
    }
    for (int l = 1; l <= D; ++l) {
        const int o = l == D ? F.out_dim : W;
        for (int j = tid; j < o; j += kThreads) bias[(l - 1) * W + j] = F.b[l][j];
    }
    for (int idx = tid; idx < kM * W / 8; idx += kThreads)
        reinterpret_cast<uint4 *>(A)[idx] = make_uint4(0u, 0u, 0u, 0u);
    // positions of this CTA's first tile, loaded once: a Gauss-Newton run
    // revisits the same tile in every iteration
    float xf0 = 0.f, xf1 = 0.f, xf2 = 0.f;
    if (MODE == 0) {
        const int p = blockIdx.x * P + row;
        if (p < n) {
            xf0 = X[p];
            xf1 = X[ld + p];
            xf2 = X[2 * ld + p];
        }
    } else if (tid < P) {
        const int p = blockIdx.x * P + tid;
        xs[tid] = p < n ? make_float4(X[p], X[ld + p], X[2 * ld + p], 0.f)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    bool ok = true;
    bool weights_ready = false;

    const uint32_t a_addr = smem_u32(A);
    const uint32_t b_addr = smem_u32(blob);
    const uint32_t idesc_h = idesc_bf16(kM, W);
    const uint32_t idesc_o = idesc_bf16(kM, kMaxOut);
    const uint32_t tlane = tmem + ((uint32_t)(wq * 32) << 16);
    uint32_t phase = 0;

    // Gauss-Newton: every CTA carries z in shared memory from iteration to
    // iteration (it solves each iteration's system itself)
    if (MODE == 1 && gn_on) gn_ff_begin(gn, r, gff);

    for (int it = 0; it < n_iter; ++it) {
        const double *z = MODE == 0 ? jobs.job[blockIdx.y].z : zj;
        __syncthreads();
        for (int j = tid; j < W; j += kThreads) {
            float a = b0s[j];
            for (int k = 0; k < r; ++k) {
                const float zk = (MODE == 1 && gn_on) ? gff.z[k].hi : (float)__ldcg(&z[k]);
                a = fmaf(W0t[k * ldt + j], zk, a);
            }
            W0v[j].w = a;
        }
        __syncthreads();

        for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
            const int p0 = tile * P;
            const int p = p0 + lp;
            const bool valid = live && p < n;
            // ---- layer 0 on the CUDA cores
            if (MODE == 0) {
                float x0 = xf0, x1 = xf1, x2 = xf2;
                if (tile != (int)blockIdx.x) {
                    x0 = x1 = x2 = 0.f;
                    if (p < n) {
                        x0 = X[p];
                        x1 = X[ld + p];
                        x2 = X[2 * ld + p];
                    }
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
            } else {
                if (tile != (int)blockIdx.x) {
                    __syncthreads();
                    if (tid < P) {
                        const int q = p0 + tid;
                        xs[tid] = q < n ? make_float4(X[q], X[ld + q], X[2 * ld + q], 0.f)
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    __syncthreads();
                }
                // value rows: pre-activations of the warpgroup's columns
                const int pairs = cw >> 1;
                for (int e = tw; e < P * pairs; e += kWgThreads) {
                    const int pr = div_small(e, pinv);
                    const int q = e - pr * P;
                    const int c = cbeg + 2 * pr;
                    const float4 x = xs[q];
                    const float4 w0 = W0v[c], w1 = W0v[c + 1];
                    *reinterpret_cast<float2 *>(xbuf + q * XS + c) =
                        make_float2(fmaf(w0.x, x.x, fmaf(w0.y, x.y, fmaf(w0.z, x.z, w0.w))),
                                    fmaf(w1.x, x.x, fmaf(w1.y, x.y, fmaf(w1.z, x.z, w1.w))));
                }
                wg_sync(wg);
                wg_value_activation(A, xbuf, XS, P, pinv, cbeg, cw, tw);
                wg_sync(wg);
                // tangent rows: ELU'(a_value) * W0[:, 3 + k]
                if (!value_row && live) {
                    const float *w0t = W0t + kt * ldt;
                    for (int cc = cbeg; cc < cbeg + cw; cc += kGroup) {
                        const float4 g0 = *reinterpret_cast<const float4 *>(xbuf + lp * XS + cc);
                        const float4 g1 = *reinterpret_cast<const float4 *>(xbuf + lp * XS + cc + 4);
                        float v[kGroup] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
                        for (int i = 0; i < kGroup; ++i) v[i] *= w0t[cc + i];
                        store_a8(A, row, cc, v);
                    }
                }
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
                    const uint32_t boff = (uint32_t)((l - 1) * W * W * 2);
                    const int nrows = out_layer ? kMaxOut : W;
                    const uint32_t idesc = out_layer ? idesc_o : idesc_h;
                    for (int ks = 0; ks < W / 16; ++ks) {
                        const uint32_t koff = (uint32_t)((ks & 3) * 32);
                        const uint32_t atom = (uint32_t)(ks >> 2);
                        const uint64_t ad = sw128_desc(a_addr + atom * (kM * 128) + koff);
                        const uint64_t bd = sw128_desc(b_addr + boff + atom * (nrows * 128) + koff);
                        mma_bf16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
                    }
                    mma_commit(bar_mma);
                    // the issuing thread alone waits for the MMA (polling by
                    // every thread would take issue slots from the others);
                    // the rest of the CTA sleeps at the barrier below
                    if (!mbar_wait(bar_mma, phase)) s_abort = 1;
                    tc_fence_before();
                }
                phase ^= 1u;
                __syncthreads();
                tc_fence_after();
                if (s_abort) goto mma_timeout;
                if (!out_layer) {
                    const float *bl = bias + (l - 1) * W;
                    if (MODE == 0) {
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
                    } else {
                        // the value warp hands its rows' pre-activations to
                        // the warpgroup; the tangent warps read their first 16
                        // columns meanwhile (further columns after the
                        // exchange: the accumulator stays valid until the next
                        // MMA, which waits for the barrier closing the layer)
                        float v[16];
                        const int c16n = cw < 16 ? cw : 16;
                        if (live_warp) {
                            tmem_ld8(tlane + cbeg, v);
                            if (c16n > 8) tmem_ld8(tlane + cbeg + 8, v + 8);
                            tmem_wait_ld();
                        }
                        if (value_row) {
                            for (int c16 = 0; c16 < cw; c16 += 16) {
                                if (c16 > 0) {
                                    tmem_ld8(tlane + cbeg + c16, v);
                                    if (c16 + 8 < cw) tmem_ld8(tlane + cbeg + c16 + 8, v + 8);
                                    tmem_wait_ld();
                                }
                                if (live) {
                                    const int nq = (cw - c16 < 16 ? cw - c16 : 16) >> 2;
#pragma unroll
                                    for (int q4 = 0; q4 < 4; ++q4) {
                                        if (q4 < nq) {
                                            const int c = cbeg + c16 + 4 * q4;
                                            *reinterpret_cast<float4 *>(xbuf + lp * XS + c) =
                                                make_float4(v[4 * q4] + bl[c], v[4 * q4 + 1] + bl[c + 1],
                                                            v[4 * q4 + 2] + bl[c + 2], v[4 * q4 + 3] + bl[c + 3]);
                                        }
                                    }
                                }
                            }
                        }
                        wg_sync(wg);
                        wg_value_activation(A, xbuf, XS, P, pinv, cbeg, cw, tw);
                        wg_sync(wg);
                        if (!value_row && live_warp) {
                            for (int c16 = 0; c16 < cw; c16 += 16) {
                                if (c16 > 0) {
                                    tmem_ld8(tlane + cbeg + c16, v);
                                    if (c16 + 8 < cw) tmem_ld8(tlane + cbeg + c16 + 8, v + 8);
                                    tmem_wait_ld();
                                }
                                if (live) {
#pragma unroll
                                    for (int g8 = 0; g8 < 2; ++g8) {
                                        const int cc = cbeg + c16 + g8 * kGroup;
                                        if (cc < cbeg + cw) {
                                            const float4 g0 = *reinterpret_cast<const float4 *>(xbuf + lp * XS + cc);
                                            const float4 g1 = *reinterpret_cast<const float4 *>(xbuf + lp * XS + cc + 4);
                                            float t[kGroup] = {g0.x * v[g8 * 8], g0.y * v[g8 * 8 + 1],
                                                               g0.z * v[g8 * 8 + 2], g0.w * v[g8 * 8 + 3],
                                                               g1.x * v[g8 * 8 + 4], g1.y * v[g8 * 8 + 5],
                                                               g1.z * v[g8 * 8 + 6], g1.w * v[g8 * 8 + 7]};
                                            store_a8(A, row, cc, t);
                                        }
                                    }
                                }
                            }
                        }
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
                        const float *bo = bias + (D - 1) * W;
                        if (MODE == 0) {
                            const FieldJob &job = jobs.job[blockIdx.y];
                            if (valid) {
#pragma unroll
                                for (int o = 0; o < 9; ++o) {
                                    if (o < F.out_dim) {
                                        float y = fmaf(F.scale[o], v[o] + bo[o], F.shift[o]);
                                        bad |= !isfinite(y);
                                        job.out[(size_t)o * ld + p] = y;
                                    }
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
                                    dudz[(size_t)(a * r + kt) * ld + p] = y;
                                O3[row * 3 + a] = valid ? y : 0.f;
                            }
                        }
                    }
                    tc_fence_before();
                    if (bad) set_status(status, NSF_ERR_NONFINITE);
                    __syncthreads();
                    if (MODE == 1 && gn_on) {
                        // this tile's share of the normal equations
                        gn_ff_tile_partials(O3, P, max(0, min(P, n - p0)), r, gff);
                    }
                    __syncthreads();
                }
            }
        }

        if (MODE == 1 && gn_on) {
            // Gauss-Newton iteration `it`: all CTAs' partials summed behind a
            // grid barrier (cooperative launch), then every CTA solves
            __syncthreads();
            if (!gn_ff_finish_iteration(gn, r, it, status, gff)) goto teardown;
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
    const size_t static_bytes = sizeof(GnFF) + 64;
    if ((size_t)L.total + static_bytes > (size_t)kMaxSmem) return 0;
    if (width % 64 || width > 256) return 0;
    return (size_t)L.total;
}

// Jacobian mode: every tile holds the most points it can (value rows in one
// lane quarter, tangent rows in the other three); the latency of a layer does
// not depend on how many of those rows are live, so fuller tiles only mean
// fewer CTAs to combine in each Gauss-Newton iteration.
int jac_points_per_tile(const FieldsDev &fd, int n) {
    (void)n;
    return jac_tile_points(fd.r);
}

int jac_grid_size_tc(const FieldsDev &fd, int n) {
    const int P = jac_points_per_tile(fd, n);
    const int tiles = (n + P - 1) / P;
    const int cap = sm_count() < kGnMaxCtas ? sm_count() : kGnMaxCtas;
    return tiles < cap ? tiles : cap;
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
