// Dense products of field training (paper App. D): the forward layer
// products, the backward products W^T delta and the weight gradients
// delta H^T, written for this library (no BLAS).
//
//   D(m, n) = sum_k A(m, k) B(n, k),  m < M, n < N, k < K,
//
// with each operand read through a strided view (element (row, k) at
// ptr[row * s_row + k * s_k], float or bf16), so every product of the
// training chain -- whatever the transposition of its factors in the
// column-per-point activation layout -- is the same kernel.  Epilogues fuse
// the elementwise work of the chain: bias + ELU (with the pre-activation and
// the bf16 copy the next product reads), multiplication by ELU'(a), or a
// per-K-slice slab for split-K weight gradients (summed in a fixed order by
// reduce_slabs).
//
// k_gemm_tc (BF16 fields, the width x width layers): 128 x 128 output tiles on
// the tcgen05 tensor cores, FP32 accumulator in tensor memory.  Per K-chunk of
// 64 every thread stages 8-element row pieces of both operands from their
// views into shared memory as bf16, K-major with the 128-byte swizzle; one
// thread issues four M = 128, N = 128, K = 16 tcgen05.mma per chunk and
// commits them to the chunk's buffer barrier; two buffers, so the staging of
// chunk c + 1 overlaps the products of chunk c.  A "split" operand is staged
// as two bf16 tiles, hi = bf16(v) and lo = bf16(v - hi), and both are
// multiplied: the backward products keep ~16 significant bits of the FP32
// cotangents against the exact bf16 weights and activations.
//
// k_gemm_simt (FP32 fields, and the thin input and output layers of every
// field): 64 x 64 tiles, 4 x 4 outputs per thread, FP32 FMA.
#include "tc_common.cuh"

namespace nsf {

using namespace tc;

namespace {

// ---------------------------------------------------------- operands ----
__device__ __forceinline__ float view_at(const MatView &v, long long row, long long k) {
    const long long i = row * v.s_row + k * v.s_k;
    return v.bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(v.ptr)[i])
                  : reinterpret_cast<const float *>(v.ptr)[i];
}

// ELU and its derivative (App. E), FP32.
__device__ __forceinline__ float elu_f(float a) { return a > 0.f ? a : expm1f(a); }
__device__ __forceinline__ float elu_grad_f(float a) { return a > 0.f ? 1.f : expf(a); }

// The epilogue of output (m, n) of K-slice z with accumulated value d.
__device__ __forceinline__ void epilogue(const GemmEpilogue &e, int M, int N, int z, int m, int n,
                                         float d) {
    const size_t i = (size_t)n * e.ld + m;
    switch (e.mode) {
        case kEpiStore: e.out[i] = d; break;
        case kEpiBiasElu: {
            const float a = d + e.bias[m];
            e.pre[i] = a;
            float h = elu_f(a);
            const __nv_bfloat16 hb = __float2bfloat16_rn(h);
            if (e.round_bf16) h = __bfloat162float(hb);
            if (e.h32) e.h32[i] = h;
            if (e.h16) e.h16[i] = hb;
            break;
        }
        case kEpiEluGrad: {
            const float o = d * elu_grad_f(e.apre[i]);
            e.out[i] = o;
            if (e.dhi) {
                const __nv_bfloat16 hb = __float2bfloat16_rn(o);
                e.dhi[i] = hb;
                e.dlo[i] = __float2bfloat16_rn(o - __bfloat162float(hb));
            }
            break;
        }
        default: e.out[(size_t)z * M * N + (size_t)m * N + n] = d; break;
    }
}

// ------------------------------------------------------------- SIMT ----
constexpr int kSt = 64, kSk = 16, kSThreads = 256;

__global__ void __launch_bounds__(kSThreads)
k_gemm_simt(int M, int N, int K, int kper, const MatView A, const MatView B,
            const GemmEpilogue e) {
    __shared__ float As[kSk][kSt + 4], Bs[kSk][kSt + 4];
    const int m0 = blockIdx.y * kSt, n0 = blockIdx.x * kSt, z = blockIdx.z;
    const int k_beg = z * kper, k_end = min(K, k_beg + kper);
    const int tid = threadIdx.x, tm = (tid % 16) * 4, tn = (tid / 16) * 4;
    float acc[4][4] = {};
    for (int k0 = k_beg; k0 < k_end; k0 += kSk) {
        // 64 x 16 elements of each operand: row-fastest, so that a view with
        // contiguous rows (s_row = 1) reads coalesced
#pragma unroll
        for (int u = 0; u < (kSt * kSk) / kSThreads; ++u) {
            const int q = tid + u * kSThreads, r = q % kSt, kk = q / kSt;
            const int k = k0 + kk;
            As[kk][r] = (m0 + r < M && k < k_end) ? view_at(A, m0 + r, k) : 0.f;
            Bs[kk][r] = (n0 + r < N && k < k_end) ? view_at(B, n0 + r, k) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kSk; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][tm + i];
                b[i] = Bs[kk][tn + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = m0 + tm + i, n = n0 + tn + j;
            if (m < M && n < N) epilogue(e, M, N, z, m, n, acc[i][j]);
        }
}

// ------------------------------------------------------------ tcgen05 ----
constexpr int kTM = 128, kTN = 128, kTK = 64, kTThreads = 256, kMaxStages = 3;
// Copy stages: three without a split operand (96 KB of tiles), two with one
// (also 96 KB): two CTAs share an SM either way.
__host__ __device__ constexpr int tc_stages(bool split) { return split ? 2 : 3; }
constexpr int kTileBytes = kTM * kTK * 2;           // one bf16 operand tile: 16 KB

// Shared-memory carve (offsets from a 1024-aligned base): per stage s the A
// tile, the B tile and, with a split operand, the tile of its lo parts; then
// the stages' barriers and the tensor-memory address.
struct TcGemmLayout {
    int tile[kMaxStages][3];
    int bars, tmem, total;
};
__host__ __device__ inline TcGemmLayout tc_gemm_layout(bool split) {
    TcGemmLayout L;
    int o = 0;
    for (int st = 0; st < kMaxStages; ++st)
        for (int t = 0; t < 3; ++t) {
            L.tile[st][t] = o;
            if (st < tc_stages(split) && (t < 2 || split)) o += kTileBytes;
        }
    L.bars = o;
    o += kMaxStages * 8;
    L.tmem = align_to(o, 16);
    o = L.tmem + 16;
    L.total = o + 1024;
    return L;
}

// Byte offset of the 16-byte chunk holding rows r .. r + 7 (r % 8 == 0) at k
// of an MN-major, 128-byte-swizzled tile of 128 rows: two 64-row atoms 1024
// bytes apart (leading byte offset), 8-k-row groups 2048 bytes apart (stride
// byte offset).
constexpr uint32_t kMnSbo = 2048;
__device__ __forceinline__ int mn_chunk(int k, int r) {
    return (k >> 3) * (int)kMnSbo + (r >> 6) * 1024 + (k & 7) * 128 +
           ((((r >> 3) & 7) ^ (k & 7)) << 4);
}

// 16-byte asynchronous copy global -> shared; src_bytes = 0 fills zeros.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Issues the copies of rows [r0, r0 + 128) x k-chunk [k0, k0 + 64) of a bf16
// view into its swizzled tile at `hi` (and the lo parts at `lo`).  A unit is
// one 16-byte chunk: 8 consecutive k of one row (K-major, MN = false) or 8
// consecutive rows at one k (MN-major); out-of-range units are zero-filled.
template <bool MN>
__device__ __forceinline__ void load_tile(const MatView &V, int rows, int K, int r0, int k0,
                                          uint32_t hi, uint32_t lo, bool with_lo) {
    const __nv_bfloat16 *ph = reinterpret_cast<const __nv_bfloat16 *>(V.ptr);
    const __nv_bfloat16 *pl = reinterpret_cast<const __nv_bfloat16 *>(V.lo);
#pragma unroll
    for (int u = 0; u < (kTM * kTK / 8) / kTThreads; ++u) {
        const int q = threadIdx.x + u * kTThreads;
        int r, kk;
        if (MN) { r = 8 * (q % (kTM / 8)); kk = q / (kTM / 8); }
        else { r = q % kTM; kk = 8 * (q / kTM); }
        const int row = r0 + r, k = k0 + kk;
        // the whole chunk is in range or none of it: rows and K are multiples
        // of 8 where it matters (checked by the launcher)
        const bool in = MN ? (row < rows && k < K) : (row < rows && k < K);
        const size_t e0 = in ? (size_t)row * V.s_row + (size_t)k * V.s_k : 0;
        const uint32_t off = MN ? (uint32_t)mn_chunk(kk, r) : (uint32_t)sw128_kmajor_offset(r, kk, kTM);
        cp_async16(hi + off, ph + e0, in ? 16 : 0);
        if (with_lo) cp_async16(lo + off, pl + e0, in ? 16 : 0);
    }
}

// Tile products of one K-chunk from the tiles at a_addr and b_addr.
template <bool AMN, bool BMN>
__device__ __forceinline__ void chunk_mma(uint32_t tmem, uint32_t a_addr, uint32_t b_addr,
                                          uint32_t idesc, bool first) {
#pragma unroll
    for (int ks = 0; ks < kTK / 16; ++ks) {
        const uint64_t ad = AMN ? sw128_desc(a_addr + 2u * ks * kMnSbo, 1024u, kMnSbo)
                                : sw128_desc(a_addr + 32u * ks);
        const uint64_t bd = BMN ? sw128_desc(b_addr + 2u * ks * kMnSbo, 1024u, kMnSbo)
                                : sw128_desc(b_addr + 32u * ks);
        mma_bf16(tmem, ad, bd, idesc, (!first || ks > 0) ? 1u : 0u);
    }
}

// D = A B^T over the CTA's K-slice for a 128 x 128 output tile, then the
// epilogue EPI.  AMN / BMN: operand with contiguous rows (staged MN-major)
// instead of contiguous k (K-major); SPLIT: 1 (2) also multiplies A's (B's)
// lo parts.  kStages stages of copies in flight: the copies of chunk c + 2
// overlap the products of chunk c.
template <bool AMN, bool BMN, int SPLIT, int EPI>
__global__ void __launch_bounds__(kTThreads)
k_gemm_tc(int M, int N, int K, int kper, const MatView A, const MatView B,
          const GemmEpilogue e, int *status) {
    extern __shared__ uint8_t smem_dyn[];
    uint8_t *base = aligned_smem(smem_dyn);
    constexpr bool split_a = SPLIT == 1, split_b = SPLIT == 2;
    const TcGemmLayout L = tc_gemm_layout(SPLIT != 0);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + L.bars);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(base + L.tmem);
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN, z = blockIdx.z;
    const int k_beg = z * kper, k_end = min(K, k_beg + kper);
    const int nchunks = k_end > k_beg ? (k_end - k_beg + kTK - 1) / kTK : 0;
    constexpr int kStages = tc_stages(SPLIT != 0);

    if (tid == 0) {
        s_ok = 1;
        for (int st = 0; st < kStages; ++st) mbar_init(&bar[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) tmem_alloc(tmem_holder, kTN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    const uint32_t idesc = idesc_bf16(kTM, kTN, BMN) | (AMN ? (1u << 15) : 0u);
    const uint32_t sb = smem_u32(base);
    auto issue = [&](int c) {           // the copies of chunk c into stage c % kStages
        const int st = c % kStages, k0 = k_beg + c * kTK;
        load_tile<AMN>(A, M, k_end, m0, k0, sb + L.tile[st][0], sb + L.tile[st][2], split_a);
        load_tile<BMN>(B, N, k_end, n0, k0, sb + L.tile[st][1], sb + L.tile[st][2], split_b);
    };
    for (int c = 0; c < kStages - 1; ++c) {
        if (c < nchunks) issue(c);
        cp_async_commit();
    }
    uint32_t phase_bits = 0u;          // bit st: parity of stage st's next product completion
    for (int c = 0; c < nchunks; ++c) {
        // stage (c + kStages - 1) % kStages last held chunk c - 1: its products
        // must be done before the copies of chunk c + kStages - 1 land there
        const int cn = c + kStages - 1;
        if (cn < nchunks) {
            if (c >= 1) {
                const int st = (c - 1) % kStages;
                if (!mbar_wait(&bar[st], (phase_bits >> st) & 1u)) s_ok = 0;
                phase_bits ^= 1u << st;
            }
            issue(cn);
        }
        cp_async_commit();
        cp_async_wait<kStages - 1>();   // this thread's copies of chunk c have landed
        fence_proxy_async();
        __syncthreads();                // ... and every thread's
        if (!s_ok) break;
        if (tid == 0) {
            tc_fence_after();
            const int st = c % kStages;
            const uint32_t a_hi = sb + L.tile[st][0], b_hi = sb + L.tile[st][1];
            const uint32_t lo = sb + L.tile[st][2];
            chunk_mma<AMN, BMN>(tmem, a_hi, b_hi, idesc, c == 0);
            if (split_a) chunk_mma<AMN, BMN>(tmem, lo, b_hi, idesc, false);
            if (split_b) chunk_mma<AMN, BMN>(tmem, a_hi, lo, idesc, false);
            mma_commit(&bar[st]);
        }
    }
    cp_async_wait<0>();
    // the products of the last chunks (those not yet waited for)
    for (int c = nchunks - kStages + 1 > 1 ? nchunks - kStages + 1 : 1; c <= nchunks; ++c) {
        const int st = (c - 1) % kStages;
        if (c - 1 < 0 || c - 1 >= nchunks) continue;
        // chunk c - 1 was waited for in-loop only if a later chunk reused its stage
        if (c - 1 + kStages < nchunks) continue;
        if (!mbar_wait(&bar[st], (phase_bits >> st) & 1u)) s_ok = 0;
        phase_bits ^= 1u << st;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int w = tid >> 5, lane = tid & 31, half = w >> 2;
    const int m = m0 + (w & 3) * 32 + lane;
    const uint32_t tq = tmem + ((uint32_t)((w & 3) * 32) << 16);
    float csum = 0.f;
    if (!s_ok) {
        if (tid == 0) set_status(status, NSF_ERR_ITER_CAP);
    } else {
        // warp w reads lanes 32 (w % 4) .. + 31 (rows m) and columns
        // 64 (w / 4) .. + 63 (n), 16 at a time
#pragma unroll 1
        for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 16) {
            float v[16];
            tmem_ld16(tq + (uint32_t)c0, v);
            tmem_wait_ld();
            if (nchunks == 0)
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = 0.f;
            if (m >= M) continue;
            const int nb = n0 + c0;
            if (EPI == kEpiBiasElu) {
                const float bm = e.bias[m];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (nb + j >= N) break;
                    const size_t i = (size_t)(nb + j) * e.ld + m;
                    const float a = v[j] + bm;
                    e.pre[i] = a;
                    float h = elu_f(a);
                    const __nv_bfloat16 hb = __float2bfloat16_rn(h);
                    if (e.round_bf16) h = __bfloat162float(hb);
                    if (e.h32) e.h32[i] = h;
                    if (e.h16) e.h16[i] = hb;
                }
            } else if (EPI == kEpiEluGrad) {
                float ap[16];
#pragma unroll
                for (int j = 0; j < 16; ++j)       // all the loads first
                    ap[j] = nb + j < N ? __ldg(e.apre + (size_t)(nb + j) * e.ld + m) : 0.f;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (nb + j >= N) break;
                    const size_t i = (size_t)(nb + j) * e.ld + m;
                    const float o = v[j] * elu_grad_f(ap[j]);
                    if (e.out) e.out[i] = o;
                    if (e.dhi) {
                        const __nv_bfloat16 hb = __float2bfloat16_rn(o);
                        e.dhi[i] = hb;
                        e.dlo[i] = __float2bfloat16_rn(o - __bfloat162float(hb));
                    }
                    csum += o;
                }
            } else if (EPI == kEpiSlab) {
                float *o = e.out + (size_t)z * M * N + (size_t)m * N + nb;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (nb + j < N) o[j] = v[j];
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (nb + j < N) e.out[(size_t)(nb + j) * e.ld + m] = v[j];
            }
        }
        if (EPI == kEpiEluGrad && e.colsum && m < M)
            e.colsum[((size_t)blockIdx.x * 2 + half) * M + m] = csum;
    }
    tc_fence_before();
    __syncthreads();
    if (tid < 32) {
        tc_fence_after();
        tmem_dealloc(tmem, kTN);
    }
}

__global__ void k_reduce_slabs(const float *__restrict__ slab, int slices, long long count,
                               float *out) {
    // 32 outputs a CTA, 8 groups of slices per output, then a shared sum
    __shared__ float part[8][33];
    const int ix = threadIdx.x & 31, g = threadIdx.x >> 5;
    const long long i = (long long)blockIdx.x * 32 + ix;
    float s = 0.f;
    if (i < count)
        for (int z = g; z < slices; z += 8) s += slab[(size_t)z * count + i];
    part[g][ix] = s;
    __syncthreads();
    if (g == 0 && i < count) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += part[q][ix];
        out[i] = t;
    }
}

int slice_len(int K, int slices, int multiple) {
    const int per = (K + slices - 1) / slices;
    return (per + multiple - 1) / multiple * multiple;
}

// ------------------------------------------------------- thin shapes ----
// out(a, c) = sum_k U(a, k) V(c, k) for a < A (<= kThinA), c < C, the k range
// of slice blockIdx.y into slab[y][a C + c]: weight gradients of the thin
// input and output layers and (U = ones) the bias gradients.  Thread c keeps
// A accumulators; the U values of a chunk of k are staged in shared memory
// and read by every thread; V is read once, coalesced when its rows are
// contiguous.
constexpr int kThinA = 32, kThinK = 32, kThinThreads = 256;

template <int NA>
__global__ void __launch_bounds__(kThinThreads)
k_thin_outer(int A, int C, int K, int kper, const MatView U, const MatView V, float *slab) {
    __shared__ float us[kThinK][NA];
    const int c = blockIdx.x * kThinThreads + threadIdx.x, z = blockIdx.y;
    const int k_beg = z * kper, k_end = min(K, k_beg + kper);
    float acc[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) acc[a] = 0.f;
    for (int k0 = k_beg; k0 < k_end; k0 += kThinK) {
        for (int q = threadIdx.x; q < kThinK * NA; q += kThinThreads) {
            const int kk = q / NA, a = q % NA;
            us[kk][a] = (a < A && k0 + kk < k_end) ? view_at(U, a, k0 + kk) : 0.f;
        }
        __syncthreads();
        if (c < C) {
            // the chunk's V values first (independent loads), then the sums
            float v[kThinK];
#pragma unroll
            for (int kk = 0; kk < kThinK; ++kk)
                v[kk] = k0 + kk < k_end ? view_at(V, c, k0 + kk) : 0.f;
#pragma unroll
            for (int kk = 0; kk < kThinK; ++kk)
#pragma unroll
                for (int a = 0; a < NA; ++a) acc[a] = fmaf(us[kk][a], v[kk], acc[a]);
        }
        __syncthreads();
    }
    if (c < C)
#pragma unroll
        for (int a = 0; a < NA; ++a)
            if (a < A) slab[(size_t)z * A * C + (size_t)a * C + c] = acc[a];
}

// D(m, n) = sum_k A(m, k) B(n, k) for few rows M (<= kThinA) and K <= kThinMaxK:
// thread n keeps M accumulators, A sits in shared memory.  Store epilogue.
constexpr int kThinMaxK = 256;

template <int NM>
__global__ void __launch_bounds__(kThinThreads)
k_thin_m(int M, int N, int K, const MatView A, const MatView B, float *out, long long ld) {
    __shared__ float as[kThinMaxK][NM];
    for (int q = threadIdx.x; q < K * NM; q += kThinThreads) {
        const int k = q / NM, m = q % NM;
        as[k][m] = m < M ? view_at(A, m, k) : 0.f;
    }
    __syncthreads();
    const int n = blockIdx.x * kThinThreads + threadIdx.x;
    if (n >= N) return;
    float acc[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc[m] = 0.f;
    if (B.s_k == 1 && B.bf16 && (K & 7) == 0 &&
        ((((size_t)B.ptr) + 2 * (size_t)n * B.s_row) & 15) == 0) {
        const uint4 *row = reinterpret_cast<const uint4 *>(
            reinterpret_cast<const __nv_bfloat16 *>(B.ptr) + (size_t)n * B.s_row);
        for (int k8 = 0; k8 < K / 8; ++k8) {
            const uint4 q = __ldg(row + k8);
            const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&q);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float b = __bfloat162float(h[j]);
#pragma unroll
                for (int m = 0; m < NM; ++m) acc[m] = fmaf(as[8 * k8 + j][m], b, acc[m]);
            }
        }
    } else if (B.s_k == 1 && !B.bf16 && (K & 3) == 0 &&
        ((((size_t)B.ptr) + 4 * (size_t)n * B.s_row) & 15) == 0) {
        const float4 *row = reinterpret_cast<const float4 *>(
            reinterpret_cast<const float *>(B.ptr) + (size_t)n * B.s_row);
        for (int k4 = 0; k4 < K / 4; ++k4) {
            const float4 b = __ldg(row + k4);
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int m = 0; m < NM; ++m) acc[m] = fmaf(as[4 * k4 + j][m], bv[j], acc[m]);
        }
    } else {
        for (int k = 0; k < K; ++k) {
            const float b = view_at(B, n, k);
#pragma unroll
            for (int m = 0; m < NM; ++m) acc[m] = fmaf(as[k][m], b, acc[m]);
        }
    }
#pragma unroll
    for (int m = 0; m < NM; ++m)
        if (m < M) out[(size_t)n * ld + m] = acc[m];
}

__global__ void k_reduce_slabs_t(const float *__restrict__ slab, int slices, int A, int C,
                                 float *out) {
    __shared__ float part[8][33];
    const int ix = threadIdx.x & 31, g = threadIdx.x >> 5;
    const long long i = (long long)blockIdx.x * 32 + ix, count = (long long)A * C;
    float s = 0.f;
    if (i < count)
        for (int z = g; z < slices; z += 8) s += slab[(size_t)z * count + i];
    part[g][ix] = s;
    __syncthreads();
    if (g == 0 && i < count) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += part[q][ix];
        out[(size_t)(i % C) * A + (i / C)] = t;
    }
}

}  // namespace

cudaError_t gemm_simt(int M, int N, int K, const MatView &A, const MatView &B,
                      const GemmEpilogue &e, int kslices, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (kslices < 1 || (kslices > 1 && e.mode != kEpiSlab)) return cudaErrorInvalidValue;
    const int kper = slice_len(K, kslices, kSk);
    dim3 grid((N + kSt - 1) / kSt, (M + kSt - 1) / kSt, e.mode == kEpiSlab ? kslices : 1);
    k_gemm_simt<<<grid, kSThreads, 0, s>>>(M, N, K, kper, A, B, e);
    return cudaGetLastError();
}

namespace {
template <bool AMN, bool BMN, int SPLIT, int EPI>
cudaError_t launch_tc(int M, int N, int K, int kper, dim3 grid, const MatView &A,
                      const MatView &B, const GemmEpilogue &e, int *status, cudaStream_t s) {
    static bool attr = false;
    set_max_dynamic_smem(k_gemm_tc<AMN, BMN, SPLIT, EPI>, attr);
    k_gemm_tc<AMN, BMN, SPLIT, EPI><<<grid, kTThreads, tc_gemm_layout(SPLIT != 0).total, s>>>(
        M, N, K, kper, A, B, e, status);
    return cudaGetLastError();
}
}  // namespace

// The three product shapes of training: forward (bf16 weights and
// activations, both with contiguous k, bias + ELU), backward data (weights
// transposed and the cotangent's hi/lo pairs, both with contiguous k,
// * ELU'), weight gradient (cotangent pairs and activations, both with
// contiguous rows, slabs).
cudaError_t gemm_tc(int M, int N, int K, const MatView &A, const MatView &B, int split,
                    const GemmEpilogue &e, int kslices, int *status, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (kslices < 1 || (kslices > 1 && e.mode != kEpiSlab)) return cudaErrorInvalidValue;
    const int kper = slice_len(K, kslices, kTK);
    dim3 grid((N + kTN - 1) / kTN, (M + kTM - 1) / kTM, e.mode == kEpiSlab ? kslices : 1);
    const bool a_mn = A.s_row == 1 && A.s_k != 1, b_mn = B.s_row == 1 && B.s_k != 1;
    // bf16 operands whose 16-byte chunks are aligned and lie wholly in or out
    // of range
    auto ok = [&](const MatView &V, bool mn, int rows, bool lo) {
        if (!V.bf16 || (lo && !V.lo)) return false;
        const long long stride = mn ? V.s_k : V.s_row;
        if ((mn ? V.s_row : V.s_k) != 1 || stride % 8) return false;
        if ((((size_t)V.ptr) & 15) || (lo && (((size_t)V.lo) & 15))) return false;
        return mn ? rows % 8 == 0 : K % 8 == 0;
    };
    if (!ok(A, a_mn, M, split == 1) || !ok(B, b_mn, N, split == 2)) return cudaErrorInvalidValue;
    if (!a_mn && !b_mn && split == 0 && e.mode == kEpiBiasElu)
        return launch_tc<false, false, 0, kEpiBiasElu>(M, N, K, kper, grid, A, B, e, status, s);
    if (!a_mn && !b_mn && split == 2 && e.mode == kEpiEluGrad)
        return launch_tc<false, false, 2, kEpiEluGrad>(M, N, K, kper, grid, A, B, e, status, s);
    if (a_mn && b_mn && split == 1 && e.mode == kEpiSlab)
        return launch_tc<true, true, 1, kEpiSlab>(M, N, K, kper, grid, A, B, e, status, s);
    return cudaErrorInvalidValue;   // a shape training does not use
}

cudaError_t thin_outer(int A, int C, int K, const MatView &U, const MatView &V, float *slab,
                       int slices, float *out, bool transposed, cudaStream_t s) {
    if (A <= 0 || C <= 0) return cudaSuccess;
    if (A > kThinA || slices < 1) return cudaErrorInvalidValue;
    const int kper = slice_len(K, slices, kThinK);
    dim3 grid((C + kThinThreads - 1) / kThinThreads, slices);
    if (A == 1) k_thin_outer<1><<<grid, kThinThreads, 0, s>>>(A, C, K, kper, U, V, slab);
    else if (A <= 4) k_thin_outer<4><<<grid, kThinThreads, 0, s>>>(A, C, K, kper, U, V, slab);
    else if (A <= 16) k_thin_outer<16><<<grid, kThinThreads, 0, s>>>(A, C, K, kper, U, V, slab);
    else k_thin_outer<32><<<grid, kThinThreads, 0, s>>>(A, C, K, kper, U, V, slab);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long count = (long long)A * C;
    if (transposed)
        k_reduce_slabs_t<<<(int)((count + 31) / 32), 256, 0, s>>>(slab, slices, A, C, out);
    else
        k_reduce_slabs<<<(int)((count + 31) / 32), 256, 0, s>>>(slab, slices, count, out);
    return cudaGetLastError();
}

cudaError_t thin_m(int M, int N, int K, const MatView &A, const MatView &B, float *out,
                   long long ld, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (M > kThinA || K > kThinMaxK) return cudaErrorInvalidValue;
    const int g = (N + kThinThreads - 1) / kThinThreads;
    if (M <= 4) k_thin_m<4><<<g, kThinThreads, 0, s>>>(M, N, K, A, B, out, ld);
    else if (M <= 16) k_thin_m<16><<<g, kThinThreads, 0, s>>>(M, N, K, A, B, out, ld);
    else k_thin_m<32><<<g, kThinThreads, 0, s>>>(M, N, K, A, B, out, ld);
    return cudaGetLastError();
}

cudaError_t reduce_slabs(const float *slab, int slices, long long count, float *out,
                         cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    k_reduce_slabs<<<(int)((count + 31) / 32), 256, 0, s>>>(slab, slices, count, out);
    return cudaGetLastError();
}

}  // namespace nsf
