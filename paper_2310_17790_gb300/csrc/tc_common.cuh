// Shared pieces of the tcgen05 tensor-core kernels (BF16 field evaluation in
// fields_tc.cu, Jacobian and Gauss-Newton in jacobian_tc.cu): PTX wrappers for
// mbarriers, bulk copies, tensor memory and tcgen05.mma, the shared-memory
// operand descriptors, and the BF16-path activation.
//
// Operand layouts use the 128-byte swizzle.
//   K-major (rows of K contiguous): a K-atom is 64 bf16 columns; row n's 128
//   bytes sit at (n / 8) * 1024 + (n % 8) * 128 in the atom and its 16-byte
//   chunk c at chunk position c ^ (n % 8); 8-row groups are 1024 bytes apart.
//   MN-major (rows of MN contiguous, one row per k): an atom is 8 k-rows of
//   64 bf16 MN-elements (1024 bytes), chunk c of k-row kr at position
//   c ^ kr; atoms are tiled along MN (leading byte offset) and along K in
//   8-row steps (stride byte offset).
// Every atom starts on a 1024-byte boundary.
#pragma once

#include <cuda_bf16.h>

#include "device_common.cuh"

namespace nsf {
namespace tc {

constexpr int kM = 128;                   // tile rows (TMEM lanes)
constexpr int kWG = 8;                    // warpgroups per CTA
constexpr int kWgThreads = 128;
constexpr int kThreads = kWG * kWgThreads;
constexpr int kGroup = 8;                 // bf16 values per 16-byte chunk
constexpr int kMaxSmem = 227 * 1024;
constexpr int kMaxOut = 16;               // output rows of the last layer (out_dim padded)

__host__ __device__ inline int align_to(int v, int a) { return (v + a - 1) / a * a; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// 1024-byte aligned base inside the dynamic shared array, by pointer
// arithmetic on the shared array itself (an integer round trip would hide the
// address space and turn every shared access into a generic one).
__device__ __forceinline__ uint8_t *aligned_smem(uint8_t *dyn) {
    return dyn + ((1024u - (smem_u32(dyn) & 1023u)) & 1023u);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Ends an mbarrier's life before its shared memory is used for anything else.
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
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
__device__ inline bool mbar_wait(uint64_t *bar, uint32_t phase) {
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

// One bulk copy of `bytes` (a multiple of 16) in 32 KB pieces, all completing
// on `bar` (which expects the whole transaction count).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    mbar_expect_tx(bar, bytes);
    for (uint32_t off = 0; off < bytes; off += 32768u) {
        const uint32_t len = bytes - off < 32768u ? bytes - off : 32768u;
        bulk_g2s(static_cast<uint8_t *>(dst) + off, static_cast<const uint8_t *>(src) + off, len,
                 bar);
    }
}

// Plain arrival (count 1) on an mbarrier.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One tiled TMA load of a 2-D box at coordinates (x innermost, y) of the
// tensor map into shared memory at dst, completing on bar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
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

// Allocates ncols tensor-memory columns (one warp calls).  A CTA that will
// allocate again later (a batched launch running several problems) keeps its
// allocation permit; otherwise it gives the permit up so that other CTAs on
// the SM need not wait for it.
__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols,
                                           bool relinquish = true) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(holder)),
                 "r"(ncols)
                 : "memory");
    if (relinquish)
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// Shared-memory matrix descriptor with the 128-byte swizzle.  K-major: the
// stride byte offset is the 1024-byte step between 8-row groups and the
// leading byte offset is not used (16).  MN-major: lbo = step between
// 64-element MN blocks, sbo = step between 8-row K blocks.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr, uint32_t lbo = 16,
                                               uint32_t sbo = 1024) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;          // descriptor version of the tcgen05 family
    d |= (uint64_t)2 << 61;          // swizzle mode: 128 bytes
    return d;
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 D; A K-major, B
// K-major or (b_mn) MN-major.
__host__ __device__ __forceinline__ uint32_t idesc_bf16(int M, int N, bool b_mn = false) {
    return (1u << 4)                 // D format F32
           | (1u << 7)               // A format BF16
           | (1u << 10)              // B format BF16
           | ((b_mn ? 1u : 0u) << 16)
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

// The same product with the A operand in tensor memory (M rows in lanes, two
// bf16 K-values per 32-bit column, K-slice ks at column offset 8 ks).
__device__ __forceinline__ void mma_bf16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// 8 consecutive 32-bit columns of this warp's 32 TMEM lanes (one per thread).
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

// 16 consecutive 32-bit columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive 32-bit columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive 32-bit columns of this warp's 32 TMEM lanes from registers.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15])
        : "memory");
}

// 8 consecutive 32-bit columns of this warp's 32 TMEM lanes from registers.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t *r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ uint4 pack_bf16x8(const float *h) {
    return make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]), pack_bf16x2(h[4], h[5]),
                      pack_bf16x2(h[6], h[7]));
}

// ELU on the BF16 path: one exponential per element (the result is rounded to
// bf16 right after, so exp(a) - 1 is as good as expm1 here); grad = ELU'(a).
__device__ __forceinline__ float elu_fast(float a, float &grad) {
    const float e = __expf(fminf(a, 0.f));
    grad = a > 0.f ? 1.f : e;
    return a > 0.f ? a : e - 1.f;
}

// 2^t on the special-function unit (PTX ex2.approx.ftz: +inf for large t,
// +0 for very negative t).
__device__ __forceinline__ float ex2_approx(float t) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(t));
    return y;
}

// ELU of two accumulator values plus their biases, with packed f32x2
// arithmetic: a = acc + b, e = 2^(a log2(e)) on the special-function unit,
// ELU = a (a > 0) or e - 1.  For large positive a, e is +inf and unused.
__device__ __forceinline__ float2 elu2(float2 acc, float2 b) {
    const float2 a = __fadd2_rn(acc, b);
    const float2 t = __fmul2_rn(a, make_float2(1.4426950408889634f, 1.4426950408889634f));
    const float2 em1 = __fadd2_rn(make_float2(ex2_approx(t.x), ex2_approx(t.y)),
                                  make_float2(-1.f, -1.f));
    return make_float2(a.x > 0.f ? a.x : em1.x, a.y > 0.f ? a.y : em1.y);
}

// Barrier over the nthreads threads of one named barrier id (1 .. 15).
__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Byte offset of element (n, k) of a K-major, 128-byte-swizzled operand whose
// K-atoms hold rows_pad rows.
__host__ __device__ inline size_t sw128_kmajor_offset(int n, int k, int rows_pad) {
    const int atom = k / 64, kk = k % 64, chunk = kk / 8;
    return (size_t)atom * rows_pad * 128 + (size_t)(n / 8) * 1024 + (n % 8) * 128 +
           ((chunk ^ (n % 8)) * 16) + (kk % 8) * 2;
}

inline int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// Dynamic shared memory limit of a kernel: the opt-in maximum minus its
// static shared memory; set once per kernel, before any stream capture.
template <class K>
inline void set_max_dynamic_smem(K kernel, bool &done) {
    if (done) return;
    cudaFuncAttributes fa;
    int stat = 0;
    if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) stat = (int)fa.sharedSizeBytes;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem - stat);
    done = true;
}

}  // namespace tc
}  // namespace nsf
