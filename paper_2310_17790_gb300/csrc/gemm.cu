// Dense products of field training (paper App. D): the forward layer
// products, the backward products W^T delta and the weight gradients
// delta H^T, written for this library (no BLAS).
//
//   D(m, n) = sum_k A(m, k) B(n, k),  m < M, n < N, k < K,
//
// Epilogues fuse the elementwise work of the chain: bias + ELU (with the
// ELU' code and the bf16 copy the next product reads), multiplication by
// ELU'(a), or a per-K-slice slab for split-K weight gradients (summed in a
// fixed order by reduce_slabs / reduce_dw).  BF16 fields:
//
//   k_layer_tc   the hidden W x W layers with the points as the M dimension,
//                persistent and warp-specialised (TMA producer warp, MMA warp,
//                16 epilogue warps), the unit's weight rows resident in shared
//                memory, four TMEM accumulators, coalesced staged stores;
//   k_gemm_tc    the weight gradients delta H^T (and, from a tile of ones, the
//                bias sums): persistent, warp-specialised, 128 x 128 tiles over
//                K-slices of points, both operands MN-major through TMA;
//   k_thin_k     the input layer forward (K = 3 + r) and the output layer
//                backward with its weight gradient, on the CUDA cores;
//   k_thin_m_warp  the output layer forward (few output rows);
//   k_input_bwd  the input layer backward: dinp, dW0 and db0 in one pass.
//
// The backward products multiply the FP32 cotangent split into two bf16
// parts, hi = bf16(v) and lo = bf16(v - hi), against the exact bf16 weights
// and activations (~16 significant bits).  FP32 fields run every product in
// FP32 on the CUDA cores (k_gemm_simt: 64 x 64 tiles, 4 x 4 outputs per
// thread; k_thin_outer, k_thin_m), each operand read through a strided view
// (element (row, k) at ptr[row * s_row + k * s_k], float or bf16).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <type_traits>

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

// ELU and ELU' on the BF16 path, where the activation is rounded to bf16 right
// after: e = 2^(a log2 e) on the special-function unit, ELU = e - 1, except
// for -1/32 < a <= 0, where the series a (1 + a/2 (1 + a/3)) (relative error
// < 1.3e-6) keeps small activations accurate.  Both stay far inside half a
// bf16 ulp of the exact value.  Large a gives e = inf, unused.
__device__ __forceinline__ float elu_bf16_path(float a, float &grad) {
    const float e = ex2_approx(a * 1.4426950408889634f);
    grad = a > 0.f ? 1.f : e;
    const float series = a * fmaf(a, fmaf(a, 0.16666667f, 0.5f), 1.f);
    return a > 0.f ? a : (a > -0.03125f ? series : e - 1.f);
}

// ELU' on the BF16 path is kept as a 16-bit fixed-point code q = rint(ELU'
// 2^15) (ELU' lies in (0, 1], and 1 codes as 32768 exactly; absolute error
// <= 2^-16), two bytes a value instead of the four of the pre-activation.
// Encoding: the low 16 bits of the float ELU' 2^15 + 2^23 (the addition
// rounds to the nearest integer); decoding: 0x4B000000 | q read as a float is
// 2^23 + q.
__device__ __forceinline__ unsigned short dact_code(float g) {
    return (unsigned short)(__float_as_uint(fmaf(g, 32768.f, 8388608.f)) & 0xFFFFu);
}
__device__ __forceinline__ float dact_value(unsigned q) {
    return (__uint_as_float(0x4B000000u | q) - 8388608.f) * 3.0517578125e-05f;
}

// The split of a cotangent value into bf16 hi + lo.
__device__ __forceinline__ void split_bf16(float o, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(o);
    lo = __float2bfloat16_rn(o - __bfloat162float(hi));
}

// The epilogue of output (m, n) of K-slice z with accumulated value d.
__device__ __forceinline__ void epilogue(const GemmEpilogue &e, int M, int N, int z, int m, int n,
                                         float d) {
    const size_t i = (size_t)n * e.ld + m;
    switch (e.mode) {
        case kEpiStore: e.out[i] = d; break;
        case kEpiBiasElu: {
            const float a = d + e.bias[m];
            if (e.dact) {                      // BF16 path
                float g;
                const float h = elu_bf16_path(a, g);
                e.dact[i] = dact_code(g);
                e.h16[i] = __float2bfloat16_rn(h);
                break;
            }
            e.pre[i] = a;
            const float h = elu_f(a);
            if (e.h32) e.h32[i] = h;
            if (e.h16) e.h16[i] = __float2bfloat16_rn(h);
            break;
        }
        case kEpiEluGrad: {
            const float o = d * (e.dact ? dact_value(e.dact[i]) : elu_grad_f(e.apre[i]));
            if (e.out) e.out[i] = o;
            if (e.dhi) split_bf16(o, e.dhi[i], e.dlo[i]);
            break;
        }
        default: e.out[(size_t)z * M * N + (size_t)n * M + m] = d; break;
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
// Persistent, warp-specialised: one CTA per SM walks the work units (a
// 128 x 128 output tile and a K-slice) u = blockIdx.x, + gridDim.x, ...;
// units with the same output columns and K-slice are adjacent, so the CTAs
// that share an operand tile fetch it at about the same time (one HBM read,
// the rest from L2).
//   warp 0      one thread issues the TMA copies of each K-chunk (64) of
//               both operands (and the lo parts of a split operand) into a
//               ring of shared-memory stages, each completing on the stage's
//               `full` barrier;
//   warp 1      owns the tensor memory; one thread issues the tcgen05.mma of
//               each chunk (four M = 128, N = 128, K = 16 products, eight with
//               a split operand) into one of two FP32 accumulators and commits
//               them to the stage's `empty` barrier, and after a unit's last
//               chunk to the accumulator's `tfull` barrier;
//   warps 2-9   the epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its
//               output rows) and 64 of the 128 columns, hands the accumulator
//               back (`tempty`), then applies the epilogue and stores.
// So the copies of the next chunks, the products of the next unit and the
// epilogue of this one overlap.  Every wait is bounded in time.
constexpr int kTM = 128, kTN = 128, kTK = 64;
constexpr int kWsThreads = 320, kWsEpiWarps = 8;
constexpr int kTileBytes = kTM * kTK * 2;           // one bf16 operand tile: 16 KB
// Stages of the copy ring: 6 x 32 KB, or 4 x 48 KB with a split operand.
__host__ __device__ constexpr int ws_stages(bool split) { return split ? 4 : 6; }
__host__ __device__ constexpr int ws_stage_bytes(bool split) {
    return (split ? 3 : 2) * kTileBytes;
}
// After the stages: the barriers, the TMEM holder, then (1024-aligned) a
// 16 x 64 tile of bf16 ones, the B operand of the column sums.
__host__ __device__ constexpr int ws_ones_offset(bool split) {
    return (ws_stages(split) * ws_stage_bytes(split) + (2 * ws_stages(split) + 5) * 8 + 16 + 1023) /
           1024 * 1024;
}
__host__ __device__ constexpr int ws_smem_bytes(bool split) {
    return ws_ones_offset(split) + 2048 + 1024;
}
// MN-major operand tiles as the TMA writes them: two 64-row blocks (8 KB
// apart, the leading byte offset), each 64 k-rows of 128 bytes in 8-row
// atoms 1024 bytes apart (the stride byte offset).
constexpr uint32_t kMnLbo = 8192, kMnSbo = 1024;

struct WsShape {
    int M, N, K, kper, tiles_m, tiles_n, units;
};

// Tile products of one K-chunk from the tiles at a_addr and b_addr.
template <bool AMN, bool BMN>
__device__ __forceinline__ void chunk_mma(uint32_t tmem, uint32_t a_addr, uint32_t b_addr,
                                          uint32_t idesc, bool first) {
#pragma unroll
    for (int ks = 0; ks < kTK / 16; ++ks) {
        const uint64_t ad = AMN ? sw128_desc(a_addr + 2048u * ks, kMnLbo, kMnSbo)
                                : sw128_desc(a_addr + 32u * ks);
        const uint64_t bd = BMN ? sw128_desc(b_addr + 2048u * ks, kMnLbo, kMnSbo)
                                : sw128_desc(b_addr + 32u * ks);
        mma_bf16(tmem, ad, bd, idesc, (!first || ks > 0) ? 1u : 0u);
    }
}

// The copies of rows [r0, r0 + 128) x k [k0, k0 + 64) of one operand: one box
// of 64 k x 128 rows (K-major) or two of 64 rows x 64 k (MN-major).
template <bool MN>
__device__ __forceinline__ void load_operand(const CUtensorMap *map, uint32_t dst, int r0, int k0,
                                             uint64_t *bar) {
    if (MN) {
        tma_load_2d(dst, map, r0, k0, bar);
        tma_load_2d(dst + kMnLbo, map, r0 + 64, k0, bar);
    } else {
        tma_load_2d(dst, map, k0, r0, bar);
    }
}

__device__ __forceinline__ void unit_coords(const WsShape &g, int u, int &m0, int &n0, int &tn,
                                            int &z, int &k_beg, int &nch) {
    const int tm = u % g.tiles_m, r = u / g.tiles_m;
    tn = r % g.tiles_n;
    z = r / g.tiles_n;
    m0 = tm * kTM;
    n0 = tn * kTN;
    k_beg = z * g.kper;
    const int k_end = min(g.K, k_beg + g.kper);
    nch = k_end > k_beg ? (k_end - k_beg + kTK - 1) / kTK : 0;
}

// D = A B^T by units, then the epilogue EPI.  AMN / BMN: operand with
// contiguous rows (MN-major) instead of contiguous k (K-major); SPLIT: 1 (2)
// also multiplies A's (B's) lo parts, whose tensor map is mLo.  K-slices are
// whole chunks (kper % 64 == 0): a chunk past K reads the TMA's zero fill.
template <bool AMN, bool BMN, int SPLIT, int EPI>
__global__ void __launch_bounds__(kWsThreads, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
          const __grid_constant__ CUtensorMap mLo, const WsShape g, const GemmEpilogue e,
          int *status) {
    extern __shared__ uint8_t smem_dyn[];
    uint8_t *base = aligned_smem(smem_dyn);
    constexpr bool split = SPLIT != 0;
    constexpr int S = ws_stages(split), SB = ws_stage_bytes(split);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + S * SB);
    uint64_t *empty = full + S, *tfull = empty + S, *tempty = tfull + 2, *done = tempty + 2;
    uint32_t *holder = reinterpret_cast<uint32_t *>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], kWsEpiWarps);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // With colsum: TMEM columns 256 + 16 acc hold the sums of A's rows over the
    // unit's k (A times a tile of ones), computed by the units of column tile 0.
    const bool sums = e.colsum != nullptr;
    const uint32_t tcols = sums ? 4 * kTN : 2 * kTN;
    if (sums) {
        uint4 *ones = reinterpret_cast<uint4 *>(base + ws_ones_offset(split));
        for (int i = threadIdx.x; i < 2048 / 16; i += kWsThreads)
            ones[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
        fence_proxy_async();         // visible to the tensor cores
    }
    if (warp == 1) tmem_alloc(holder, tcols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;
    const uint32_t sb = smem_u32(base);
    int m0, n0, tn, z, k_beg, nch;

    if (warp == 0) {
        if (lane == 0) {
            int st = 0;
            uint32_t ph = 0, filled = 0, last_ph = 0;   // per stage: ever filled, parity
            bool ok = true;
            for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
                unit_coords(g, u, m0, n0, tn, z, k_beg, nch);
                for (int c = 0; c < nch; ++c) {
                    if (!mbar_wait(&empty[st], ph ^ 1u)) { ok = false; break; }
                    const uint32_t dst = sb + (uint32_t)(st * SB);
                    const int k0 = k_beg + c * kTK;
                    mbar_expect_tx(&full[st], (uint32_t)SB);
                    load_operand<AMN>(&mA, dst, m0, k0, &full[st]);
                    load_operand<BMN>(&mB, dst + kTileBytes, n0, k0, &full[st]);
                    if (SPLIT == 1) load_operand<AMN>(&mLo, dst + 2 * kTileBytes, m0, k0, &full[st]);
                    if (SPLIT == 2) load_operand<BMN>(&mLo, dst + 2 * kTileBytes, n0, k0, &full[st]);
                    filled |= 1u << st;
                    last_ph = (last_ph & ~(1u << st)) | (ph << st);
                    if (++st == S) { st = 0; ph ^= 1u; }
                }
            }
            if (!ok) {
                set_status(status, NSF_ERR_ITER_CAP);
                // the copies already issued land before the CTA ends
                for (int i = 0; i < S; ++i)
                    if (filled >> i & 1u) mbar_wait(&full[i], (last_ph >> i) & 1u);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kTM, kTN, BMN) | (AMN ? (1u << 15) : 0u);
            const uint32_t idesc1 = idesc_bf16(kTM, 16, false) | (AMN ? (1u << 15) : 0u);
            const uint32_t ones = sb + (uint32_t)ws_ones_offset(split);
            int st = 0, it = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
                unit_coords(g, u, m0, n0, tn, z, k_beg, nch);
                if (nch == 0) continue;
                const int acc = it & 1;
                if (!mbar_wait(&tempty[acc], ((it >> 1) & 1) ^ 1)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * kTN);
                for (int c = 0; c < nch; ++c) {
                    if (!mbar_wait(&full[st], ph)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a_hi = sb + (uint32_t)(st * SB), b_hi = a_hi + kTileBytes;
                    const uint32_t lo = a_hi + 2 * kTileBytes;
                    chunk_mma<AMN, BMN>(d, a_hi, b_hi, idesc, c == 0);
                    if (SPLIT == 1) chunk_mma<AMN, BMN>(d, lo, b_hi, idesc, false);
                    if (SPLIT == 2) chunk_mma<AMN, BMN>(d, a_hi, lo, idesc, false);
                    if (sums && tn == 0) {
                        const uint32_t d1 = tmem + (uint32_t)(2 * kTN + 16 * acc);
                        chunk_mma<AMN, false>(d1, a_hi, ones, idesc1, c == 0);
                        if (SPLIT == 1) chunk_mma<AMN, false>(d1, lo, ones, idesc1, false);
                    }
                    mma_commit(&empty[st]);
                    if (++st == S) { st = 0; ph ^= 1u; }
                }
                if (!ok) break;
                mma_commit(&tfull[acc]);
                ++it;
            }
            if (!ok) set_status(status, NSF_ERR_ITER_CAP);
            // every product issued has completed before the tensor memory is freed
            mma_commit(done);
            mbar_wait(done, 0);
        }
    } else {
        const int q = warp & 3, half = (warp - 2) >> 2;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        int it = 0;
        for (int u = blockIdx.x; u < g.units; u += gridDim.x) {
            unit_coords(g, u, m0, n0, tn, z, k_beg, nch);
            const int m = m0 + q * 32 + lane, nb = n0 + half * 64;
            const bool row_in = m < g.M;
            float v[64];
            if (nch > 0) {
                const int acc = it & 1;
                if (!mbar_wait(&tfull[acc], (it >> 1) & 1)) {
                    set_status(status, NSF_ERR_ITER_CAP);
                    break;
                }
                tc_fence_after();
                const uint32_t ta = tmem + (uint32_t)(acc * kTN + half * 64) + lane_off;
                tmem_ld32(ta, v);
                tmem_ld32(ta + 32, v + 32);
                if (sums && tn == 0 && half == 0) {
                    float r[8];
                    tmem_ld8(tmem + (uint32_t)(2 * kTN + 16 * acc) + lane_off, r);
                    tmem_wait_ld();
                    if (row_in) e.colsum[(size_t)z * g.M + m] = r[0];
                }
                tmem_wait_ld();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[acc]);
                ++it;
            } else {
#pragma unroll
                for (int j = 0; j < 64; ++j) v[j] = 0.f;
                if (sums && tn == 0 && half == 0 && row_in) e.colsum[(size_t)z * g.M + m] = 0.f;
            }
            if (!row_in) continue;
            if (EPI == kEpiSlab) {
                float *o = e.out + (size_t)z * g.M * g.N + m;
#pragma unroll
                for (int j = 0; j < 64; ++j)
                    if (nb + j < g.N) o[(size_t)(nb + j) * g.M] = v[j];
            } else {
#pragma unroll
                for (int j = 0; j < 64; ++j)
                    if (nb + j < g.N) e.out[(size_t)(nb + j) * e.ld + m] = v[j];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, tcols);
    }
}

// ------------------------------------------------ hidden-layer products ----
// The W x W products of the hidden layers with the points as the M dimension:
//   Y(p, c) = sum_k X(p, k) Wt(c, k),
// forward: X = H_{l-1} (bf16 [p][k]), Wt = W_l ([c][k]), epilogue bias + ELU
// -> ELU' code and bf16 activation; backward: X = delta_l as hi + lo pairs,
// Wt = W_l^T ([c][o]), epilogue * ELU' -> delta_{l-1} as hi + lo pairs (and
// FP32 when asked), with the column sums (the bias gradient) when asked.
// A unit is 128 points x 128 output channels (column tile tn of the
// ceil(W / 128)).  The grid is a multiple of the column-tile count, so a CTA
// always has the same tn and keeps those 128 rows of Wt in shared memory for
// the whole launch (ceil(K / 64) K-atoms of 16 KB); only X streams through
// the stage ring (the CTAs of one point tile fetch it at the same time: one
// HBM read).  TMEM: four 128 x 128 FP32 accumulators, so the products run up
// to three units ahead of the epilogue.  Roles as in k_gemm_tc,
// with 16 epilogue warps: warp w holds points 32 (w % 4) .. + 31 (TMEM lanes)
// and channels 32 ((w - 2) / 4) .. + 31 of the unit, one point per lane.
// Rows of an [p][c] array are 2 W bytes apart, so a lane's own row is a poor
// access pattern: every global load and store goes through a 32 x 64-byte
// staging block of the warp (rows 80 bytes apart: no bank conflicts when a
// lane writes its row), read back and written as 8 rows x 64 bytes per
// instruction.
constexpr int kLP = 128, kLN = 128;
constexpr int kLStagesMax = 8, kLEpiWarps = 16, kLThreads = 32 * (2 + kLEpiWarps);
constexpr int kLAcc = 4;            // TMEM accumulators (all 512 columns)
constexpr int kLRow = 80, kLStaging = 32 * kLRow;   // staging block of one warp
struct LayerShape {
    int n, W, K, tiles_n, units, stages;
    long long ld;
};
__host__ __device__ inline int layer_katoms(int K) { return (K + kTK - 1) / kTK; }
__host__ __device__ inline int layer_stage_bytes(bool split) { return (split ? 2 : 1) * kTileBytes; }
// weights, stages, staging blocks, bias (128 floats), barriers, TMEM holder,
// 1024 alignment slack
__host__ __device__ inline int layer_smem_bytes(int K, bool split, int stages) {
    return layer_katoms(K) * kLN * 128 + stages * layer_stage_bytes(split) +
           kLEpiWarps * kLStaging + kLN * 4 + (2 * kLStagesMax + 2 * kLAcc + 2) * 8 + 16 + 1024;
}

// Sum over the warp's lanes of each of 32 values, lane l ending with the sum
// of x[l]: five exchange steps, each halving the values a lane keeps (a fixed
// order, so the result is reproducible).
__device__ __forceinline__ float lane_column_sum(float (&x)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < s; ++i) {
            const float send = upper ? x[i] : x[i + s];
            const float keep = upper ? x[i + s] : x[i];
            x[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return x[0];
}

// Two channels of the forward epilogue with packed f32x2 arithmetic: a = acc
// + bias, e = 2^(a log2 e) on the special-function unit, ELU = a (a > 0) or
// e - 1 (absolute error ~1e-7: below half a bf16 ulp of every activation
// larger than 2^-14 in magnitude, negligible below), ELU' = 1 or e.  Returns
// the two ELU' codes (low half: the first channel) and the two bf16 values.
__device__ __forceinline__ void elu2_codes(float2 acc, float2 bias, uint32_t &codes,
                                           uint32_t &hb) {
    const float2 a = __fadd2_rn(acc, bias);
    const float2 t = __fmul2_rn(a, make_float2(1.4426950408889634f, 1.4426950408889634f));
    const float2 e = make_float2(ex2_approx(t.x), ex2_approx(t.y));
    const float2 em1 = __fadd2_rn(e, make_float2(-1.f, -1.f));
    const bool px = a.x > 0.f, py = a.y > 0.f;
    const float2 g = make_float2(px ? 1.f : e.x, py ? 1.f : e.y);
    const float2 c = __ffma2_rn(g, make_float2(32768.f, 32768.f), make_float2(8388608.f, 8388608.f));
    codes = __byte_perm(__float_as_uint(c.x), __float_as_uint(c.y), 0x5410);
    hb = pack_bf16x2(px ? a.x : em1.x, py ? a.y : em1.y);
}

// Two channels of the backward epilogue: o = acc * ELU' from the two codes
// of `codes` (the same decoding as dact_value, packed).
__device__ __forceinline__ float2 mul_codes2(float2 acc, uint32_t codes) {
    const float2 q = make_float2(__uint_as_float(__byte_perm(codes, 0x4B000000u, 0x7610)),
                                 __uint_as_float(__byte_perm(codes, 0x4B000000u, 0x7632)));
    const float2 d = __fadd2_rn(q, make_float2(-8388608.f, -8388608.f));
    return __fmul2_rn(__fmul2_rn(acc, d), make_float2(3.0517578125e-05f, 3.0517578125e-05f));
}

// The staging block: lane l's own row (four 16-byte chunks) and the chunk of
// instruction i of a coalesced pass (row 8 i + l / 4, chunk l % 4).
__device__ __forceinline__ void stage_own_row(uint8_t *st, const uint32_t (&w)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        *reinterpret_cast<uint4 *>(st + lane * kLRow + 16 * c) =
            make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
}
__device__ __forceinline__ uint4 staged_chunk(const uint8_t *st, int i) {
    const int lane = threadIdx.x & 31;
    return *reinterpret_cast<const uint4 *>(st + (8 * i + (lane >> 2)) * kLRow + 16 * (lane & 3));
}

// Writes the warp's 32 rows x 32 16-bit values (lane l: row l in w) to
// dst[(row0 + r) ld + 8 chunk ...]: through the staging block, 8 rows a store.
__device__ __forceinline__ void store_rows16(uint8_t *st, const uint32_t (&w)[16], uint16_t *dst,
                                             long long ld, int row0, int n, int cw) {
    const int lane = threadIdx.x & 31;
    stage_own_row(st, w);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = 8 * i + (lane >> 2), ck = lane & 3;
        const uint4 v = staged_chunk(st, i);
        if (row0 + r < n && 8 * ck < cw)
            *reinterpret_cast<uint4 *>(dst + (size_t)(row0 + r) * ld + 8 * ck) = v;
    }
    __syncwarp();
}

template <bool SPLIT, int EPI>
__global__ void __launch_bounds__(kLThreads, 1)
k_layer_tc(const __grid_constant__ CUtensorMap mX, const __grid_constant__ CUtensorMap mXlo,
           const __grid_constant__ CUtensorMap mW, const LayerShape g, const GemmEpilogue e,
           int *status) {
    extern __shared__ uint8_t smem_dyn[];
    uint8_t *base = aligned_smem(smem_dyn);
    const int katoms = layer_katoms(g.K), S = g.stages, SB = layer_stage_bytes(SPLIT);
    const int tn = blockIdx.x % g.tiles_n;          // this CTA's column tile
    const uint32_t sb = smem_u32(base);
    const uint32_t sW = sb, sX = sb + (uint32_t)(katoms * kLN * 128);
    uint8_t *staging = base + katoms * kLN * 128 + S * SB;
    float *sbias = reinterpret_cast<float *>(staging + kLEpiWarps * kLStaging);
    uint64_t *full = reinterpret_cast<uint64_t *>(sbias + kLN);
    uint64_t *empty = full + kLStagesMax, *tfull = empty + kLStagesMax, *tempty = tfull + kLAcc;
    uint64_t *wbar = tempty + kLAcc, *done = wbar + 1;
    uint32_t *holder = reinterpret_cast<uint32_t *>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < kLAcc; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], kLEpiWarps);
        }
        mbar_init(wbar, 1);
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (EPI == kEpiBiasElu)
        for (int c = threadIdx.x; c < kLN; c += kLThreads)
            sbias[c] = tn * kLN + c < g.W ? e.bias[tn * kLN + c] : 0.f;
    if (warp == 1) tmem_alloc(holder, kLAcc * kLN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;

    if (warp == 0) {
        if (lane == 0) {
            mbar_expect_tx(wbar, (uint32_t)(katoms * kLN * 128));
            for (int a = 0; a < katoms; ++a)
                tma_load_2d(sW + (uint32_t)(a * kLN * 128), &mW, a * kTK, tn * kLN, wbar);
            int st = 0;
            uint32_t ph = 0, filled = 0, last_ph = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
                const int p0 = (u / g.tiles_n) * kLP;
                for (int c = 0; c < katoms; ++c) {
                    if (!mbar_wait(&empty[st], ph ^ 1u)) { ok = false; break; }
                    const uint32_t dst = sX + (uint32_t)(st * SB);
                    mbar_expect_tx(&full[st], (uint32_t)SB);
                    tma_load_2d(dst, &mX, c * kTK, p0, &full[st]);
                    if (SPLIT) tma_load_2d(dst + kTileBytes, &mXlo, c * kTK, p0, &full[st]);
                    filled |= 1u << st;
                    last_ph = (last_ph & ~(1u << st)) | (ph << st);
                    if (++st == S) { st = 0; ph ^= 1u; }
                }
            }
            if (!ok) {
                set_status(status, NSF_ERR_ITER_CAP);
                for (int i = 0; i < S; ++i)
                    if (filled >> i & 1u) mbar_wait(&full[i], (last_ph >> i) & 1u);
            }
            mbar_wait(wbar, 0);          // the weights have landed before the CTA ends
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kLP, kLN);
            int st = 0, it = 0;
            uint32_t ph = 0;
            bool ok = mbar_wait(wbar, 0);
            for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
                const int acc = it % kLAcc;
                if (!mbar_wait(&tempty[acc], ((it / kLAcc) & 1) ^ 1)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * kLN);
                for (int c = 0; c < katoms; ++c) {
                    if (!mbar_wait(&full[st], ph)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t x = sX + (uint32_t)(st * SB), w = sW + (uint32_t)(c * kLN * 128);
#pragma unroll
                    for (int ks = 0; ks < kTK / 16; ++ks) {
                        const uint64_t bd = sw128_desc(w + 32u * ks);
                        mma_bf16(d, sw128_desc(x + 32u * ks), bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                        if (SPLIT) mma_bf16(d, sw128_desc(x + kTileBytes + 32u * ks), bd, idesc, 1u);
                    }
                    mma_commit(&empty[st]);
                    if (++st == S) { st = 0; ph ^= 1u; }
                }
                if (!ok) break;
                mma_commit(&tfull[acc]);
                ++it;
            }
            if (!ok) set_status(status, NSF_ERR_ITER_CAP);
            mma_commit(done);
            mbar_wait(done, 0);
        }
    } else {
        const int q = warp & 3, bt = (warp - 2) >> 2;
        const int c_loc = 32 * bt, chan0 = tn * kLN + c_loc;
        const int cw = g.W - chan0;                  // valid channels of this warp (may be <= 0)
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        uint8_t *st = staging + (warp - 2) * kLStaging;
        float csum = 0.f;
        int it = 0;
        for (int u = blockIdx.x; u < g.units; u += gridDim.x) {
            const int row0 = (u / g.tiles_n) * kLP + q * 32;   // the warp's first point
            uint4 pf[EPI == kEpiEluGrad ? 4 : 1];
            if (EPI == kEpiEluGrad) {
                // the ELU' codes, coalesced, before the accumulator is ready
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = 8 * i + (lane >> 2), ck = lane & 3;
                    pf[i] = (row0 + r < g.n && 8 * ck < cw)
                                ? __ldg(reinterpret_cast<const uint4 *>(
                                      e.dact + (size_t)(row0 + r) * g.ld + chan0 + 8 * ck))
                                : make_uint4(0u, 0u, 0u, 0u);
                }
            }
            const int acc = it % kLAcc;
            if (!mbar_wait(&tfull[acc], (it / kLAcc) & 1)) {
                set_status(status, NSF_ERR_ITER_CAP);
                break;
            }
            tc_fence_after();
            float v[32];
            tmem_ld32(tmem + (uint32_t)(acc * kLN + c_loc) + lane_off, v);
            tmem_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);   // free for a later unit
            ++it;
            if (EPI == kEpiBiasElu) {
                uint32_t code[16], hb[16];
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    const float4 b4 = *reinterpret_cast<const float4 *>(sbias + c_loc + j);
                    elu2_codes(make_float2(v[j], v[j + 1]), make_float2(b4.x, b4.y), code[j / 2],
                               hb[j / 2]);
                    elu2_codes(make_float2(v[j + 2], v[j + 3]), make_float2(b4.z, b4.w),
                               code[j / 2 + 1], hb[j / 2 + 1]);
                }
                store_rows16(st, code, e.dact + chan0, g.ld, row0, g.n, cw);
                store_rows16(st, hb, reinterpret_cast<uint16_t *>(e.h16) + chan0, g.ld, row0, g.n,
                             cw);
            } else {
                // the codes of this lane's row, from the coalesced loads
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    *reinterpret_cast<uint4 *>(st + (8 * i + (lane >> 2)) * kLRow + 16 * (lane & 3)) =
                        pf[i];
                __syncwarp();
                uint32_t code[16];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const uint4 w4 = *reinterpret_cast<const uint4 *>(st + lane * kLRow + 16 * c);
                    code[4 * c] = w4.x;
                    code[4 * c + 1] = w4.y;
                    code[4 * c + 2] = w4.z;
                    code[4 * c + 3] = w4.w;
                }
                __syncwarp();
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const float2 o = mul_codes2(make_float2(v[2 * t], v[2 * t + 1]), code[t]);
                    v[2 * t] = o.x;
                    v[2 * t + 1] = o.y;
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(o.x, o.y);
                    hi[t] = *reinterpret_cast<const uint32_t *>(&h2);
                    const float2 r = __fadd2_rn(o, make_float2(-__low2float(h2), -__high2float(h2)));
                    lo[t] = pack_bf16x2(r.x, r.y);
                }
                store_rows16(st, hi, reinterpret_cast<uint16_t *>(e.dhi) + chan0, g.ld, row0, g.n,
                             cw);
                store_rows16(st, lo, reinterpret_cast<uint16_t *>(e.dlo) + chan0, g.ld, row0, g.n,
                             cw);
                const int p = row0 + lane;
                if (e.out && p < g.n)
#pragma unroll
                    for (int k4 = 0; k4 < 8; ++k4)
                        if (4 * k4 < cw)
                            *reinterpret_cast<float4 *>(e.out + (size_t)p * g.ld + chan0 + 4 * k4) =
                                make_float4(v[4 * k4], v[4 * k4 + 1], v[4 * k4 + 2], v[4 * k4 + 3]);
                // points past n have zero products and zero codes: o = 0
                if (e.colsum) csum += lane_column_sum(v);
            }
        }
        if (EPI == kEpiEluGrad && e.colsum && lane < cw)
            e.colsum[((size_t)(blockIdx.x / g.tiles_n) * 4 + q) * g.W + chan0 + lane] = csum;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kLAcc * kLN);
    }
}

// Sums rows z in [y per, min(slices, (y + 1) per)) of the slabs (row z at
// slab + z step) for y = blockIdx.y into out + y out_step: 32 outputs a CTA,
// 8 groups of rows per output, then a shared sum, all in a fixed order.
// With out = slab and out_step = per step, a CTA overwrites only the first
// row of its own range, after all its reads: the first pass of a two-pass sum.
__global__ void k_reduce_slabs(const float *slab, int slices, int per, long long step,
                               long long count, float *out, long long out_step) {
    __shared__ float part[8][33];
    const int ix = threadIdx.x & 31, g = threadIdx.x >> 5;
    const long long i = (long long)blockIdx.x * 32 + ix;
    const int z0 = blockIdx.y * per, z1 = min(slices, z0 + per);
    float s = 0.f;
    if (i < count) {
        int z = z0 + g;
        // four independent loads in flight per thread, summed in row order
        for (; z + 24 < z1; z += 32) {
            const float a = slab[(size_t)z * step + i], b = slab[(size_t)(z + 8) * step + i];
            const float c = slab[(size_t)(z + 16) * step + i], d = slab[(size_t)(z + 24) * step + i];
            s += a;
            s += b;
            s += c;
            s += d;
        }
        for (; z < z1; z += 8) s += slab[(size_t)z * step + i];
    }
    part[g][ix] = s;
    __syncthreads();
    if (g == 0 && i < count) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += part[q][ix];
        out[(size_t)blockIdx.y * out_step + i] = t;
    }
}

int slice_len(int K, int slices, int multiple) {
    const int per = (K + slices - 1) / slices;
    return (per + multiple - 1) / multiple * multiple;
}

// ----------------------------------------------------------- thin K ----
// out(m, n) = sum_{k < K} A(m, k) B(n, k) for K <= 20 (the input layer's
// forward product, the output layer's backward product) with the BiasElu /
// EluGrad epilogues of the BF16 path.  M % 4 == 0: thread (m4, point)
// computes rows 4 m4 .. 4 m4 + 3 of one column, so every store is a vector
// (8 bytes of codes or bf16, 16 bytes of float).  A sits in shared memory as
// [k][m] and the CTA's columns of B as [n][k] (one coalesced pass).
// EluGrad's partial sums, each CTA's in a fixed order over its columns:
// colsum[blockIdx.x M + m] = sum_n out(m, n) (a bias gradient) and, with
// e.hin (bf16 H at [n ld + m]), outer[(blockIdx.x K + k) M + m] =
// sum_n B(n, k) H(n, m) (the output layer's weight gradient).
constexpr int kThinKMax = 20, kTkThreads = 256, kTkPoints = 128;

__device__ __forceinline__ uint2 pack_bf16x4(float a, float b, float c, float d) {
    return make_uint2(pack_bf16x2(a, b), pack_bf16x2(c, d));
}
__host__ __device__ inline int thin_k_nk(int K) { return (K + 3) / 4 * 4; }
__host__ __device__ inline size_t thin_k_smem(int M, int K) {
    const int ppass = kTkThreads / (M / 4);
    return sizeof(float) * ((size_t)kTkPoints * thin_k_nk(K) + (size_t)ppass * M);
}

template <int EPI, int NK>
__global__ void __launch_bounds__(kTkThreads)
k_thin_k(int M, int N, int K, const MatView A, const MatView B, const GemmEpilogue e) {
    extern __shared__ float tk_smem[];
    float *Bs = tk_smem;                          // [kTkPoints][NK], zero past K
    float *part = Bs + kTkPoints * NK;            // [ppass][M]
    const int q = M / 4, ppass = kTkThreads / q;  // threads per column, columns per pass
    const int p_beg = blockIdx.x * kTkPoints, np = min(kTkPoints, N - p_beg);
    for (int t = threadIdx.x; t < np * NK; t += kTkThreads)
        Bs[t] = t % NK < K ? view_at(B, p_beg + t / NK, t % NK) : 0.f;
    const int pofs = threadIdx.x / q, m = 4 * (threadIdx.x % q);
    const bool active = pofs < ppass;
    // this thread's rows of A, kept in registers for all its columns
    float a[NK][4];
#pragma unroll
    for (int k = 0; k < NK; ++k)
#pragma unroll
        for (int u = 0; u < 4; ++u) a[k][u] = (active && k < K) ? view_at(A, m + u, k) : 0.f;
    float bias[4] = {0.f, 0.f, 0.f, 0.f};
    if (EPI == kEpiBiasElu && active)
#pragma unroll
        for (int u = 0; u < 4; ++u) bias[u] = e.bias[m + u];
    __syncthreads();
    float cs[4] = {0.f, 0.f, 0.f, 0.f};
    constexpr int NO = EPI == kEpiEluGrad ? NK : 1;    // outer-product rows (K <= NK)
    float ot[NO][4];
#pragma unroll
    for (int k = 0; k < NO; ++k)
#pragma unroll
        for (int u = 0; u < 4; ++u) ot[k][u] = 0.f;
    const bool outer = EPI == kEpiEluGrad && e.hin != nullptr;
    // EluGrad: the codes (and H) of a column are loaded kAhead columns ahead,
    // into a ring of registers
    constexpr int kAhead = EPI == kEpiEluGrad ? 4 : 1;
    uint2 cr[kAhead], hr[kAhead];
#pragma unroll
    for (int t = 0; t < kAhead; ++t) cr[t] = hr[t] = make_uint2(0u, 0u);
    auto fetch = [&](int pl, int slot) {
        if (pl >= np) return;
        const size_t i = (size_t)(p_beg + pl) * e.ld + m;
#pragma unroll
        for (int t = 0; t < kAhead; ++t)
            if (t == slot) {
                cr[t] = *reinterpret_cast<const uint2 *>(e.dact + i);
                if (outer) hr[t] = *reinterpret_cast<const uint2 *>(e.hin + i);
            }
    };
    if (EPI == kEpiEluGrad && active)
#pragma unroll
        for (int t = 0; t < kAhead; ++t) fetch(pofs + t * ppass, t);
    if (active)
#pragma unroll 4
        for (int pl = pofs, it = 0; pl < np; pl += ppass, ++it) {
            const int slot = it % kAhead;
            uint2 c = make_uint2(0u, 0u), hv = make_uint2(0u, 0u);
#pragma unroll
            for (int t = 0; t < kAhead; ++t)
                if (t == slot) { c = cr[t]; hv = hr[t]; }
            if (EPI == kEpiEluGrad) fetch(pl + kAhead * ppass, slot);
            float b[NK];
#pragma unroll
            for (int k4 = 0; k4 < NK; k4 += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(Bs + pl * NK + k4);
                b[k4] = v.x; b[k4 + 1] = v.y; b[k4 + 2] = v.z; b[k4 + 3] = v.w;
            }
            // packed f32x2 FMAs (each lane rounds as fmaf does)
            float2 acc01 = make_float2(0.f, 0.f), acc23 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const float2 bb = make_float2(b[k], b[k]);
                acc01 = __ffma2_rn(make_float2(a[k][0], a[k][1]), bb, acc01);
                acc23 = __ffma2_rn(make_float2(a[k][2], a[k][3]), bb, acc23);
            }
            const float acc[4] = {acc01.x, acc01.y, acc23.x, acc23.y};
            const size_t i = (size_t)(p_beg + pl) * e.ld + m;
            if (EPI == kEpiBiasElu) {
                uint32_t c0, c1, h0, h1;
                elu2_codes(make_float2(acc[0], acc[1]), make_float2(bias[0], bias[1]), c0, h0);
                elu2_codes(make_float2(acc[2], acc[3]), make_float2(bias[2], bias[3]), c1, h1);
                *reinterpret_cast<uint2 *>(e.dact + i) = make_uint2(c0, c1);
                *reinterpret_cast<uint2 *>(e.h16 + i) = make_uint2(h0, h1);
            } else {
                const float2 o01 = mul_codes2(make_float2(acc[0], acc[1]), c.x);
                const float2 o23 = mul_codes2(make_float2(acc[2], acc[3]), c.y);
                const float o[4] = {o01.x, o01.y, o23.x, o23.y};
                if (e.out) *reinterpret_cast<float4 *>(e.out + i) = make_float4(o[0], o[1], o[2], o[3]);
                float hi[4], lo[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    hi[u] = __bfloat162float(__float2bfloat16_rn(o[u]));
                    lo[u] = o[u] - hi[u];
                    cs[u] += o[u];
                }
                *reinterpret_cast<uint2 *>(e.dhi + i) = pack_bf16x4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint2 *>(e.dlo + i) = pack_bf16x4(lo[0], lo[1], lo[2], lo[3]);
                if (outer) {
                    const float h[4] = {__uint_as_float(hv.x << 16), __uint_as_float(hv.x & 0xFFFF0000u),
                                        __uint_as_float(hv.y << 16), __uint_as_float(hv.y & 0xFFFF0000u)};
                    const float2 h01 = make_float2(h[0], h[1]), h23 = make_float2(h[2], h[3]);
#pragma unroll
                    for (int k = 0; k < NO; ++k) {
                        const float2 bb = make_float2(b[k], b[k]);
                        const float2 o01 = __ffma2_rn(bb, h01, make_float2(ot[k][0], ot[k][1]));
                        const float2 o23 = __ffma2_rn(bb, h23, make_float2(ot[k][2], ot[k][3]));
                        ot[k][0] = o01.x; ot[k][1] = o01.y; ot[k][2] = o23.x; ot[k][3] = o23.y;
                    }
                }
            }
        }
    if (EPI != kEpiEluGrad) return;
    // the CTA's partial sums over its columns, in pofs order
    auto flush = [&](const float (&v)[4], float *dst) {
        __syncthreads();
        if (active)
#pragma unroll
            for (int u = 0; u < 4; ++u) part[pofs * M + m + u] = v[u];
        __syncthreads();
        for (int mm = threadIdx.x; mm < M; mm += kTkThreads) {
            float t = 0.f;
            for (int u = 0; u < ppass; ++u) t += part[u * M + mm];
            dst[mm] = t;
        }
    };
    if (e.colsum) flush(cs, e.colsum + (size_t)blockIdx.x * M);
    if (outer)
#pragma unroll
        for (int k = 0; k < NO; ++k)
            if (k < K) flush(ot[k], e.outer + ((size_t)blockIdx.x * K + k) * M);
}

// ------------------------------------------------ input-layer backward ----
// With delta_0(p, o) (o < W) the cotangent of the input layer's
// pre-activation and inp(p, j) (j < K0) its inputs:
//   dinp(p, j) = sum_o W0[o][j] delta_0(p, o)      (toward the latent codes)
//   dW0[o][j]  = sum_p delta_0(p, o) inp(p, j),  db0[o] = sum_p delta_0(p, o).
// One pass over delta_0 (the bf16 hi + lo pairs or an FP32 array): a CTA
// stages 64 points x W of it and their inputs in shared memory, then
//   dinp: thread (point pair t / 8, channel group t % 8 of 32) sums its
//         group's channels for two points (each weight load serves both),
//         then a fixed xor-shuffle sum over the 8 groups;
//   dW0 / db0: thread (point quarter t / 64, channels 4 (t % 64) .. + 3)
//         accumulates its 16 points of every tile, in order;
// and at the end the four quarters' sums are added in order and written once
// as the CTA's slab in the gradient layout [W0 (W x K0) | b0].
constexpr int kIbPoints = 64, kIbThreads = 256, kIbRow = 8 * 33 + 1, kIbMaxGrid = 320;
constexpr int kIbLoads = 4;   // 16-byte pieces of delta_0 per thread and load round
__host__ __device__ inline int ib_k0p(int K0) { return (K0 + 3) / 4 * 4; }
__host__ __device__ inline size_t ib_smem(int K0) {
    const int k0p = ib_k0p(K0);
    const size_t tiles = (size_t)kIbPoints * kIbRow + kIbPoints * k0p + 8 * (32 * k0p + 4);
    const size_t comb = 4 * (size_t)NSF_MAX_WIDTH * (k0p + 1);   // the final combine
    return sizeof(float) * (tiles > comb ? tiles : comb);
}

template <int K0P>
__global__ void __launch_bounds__(kIbThreads)
k_input_bwd(int n, int W, int K0, const __nv_bfloat16 *__restrict__ dhi,
            const __nv_bfloat16 *__restrict__ dlo, const float *__restrict__ d32, long long ld,
            const float *__restrict__ inp, const float *__restrict__ W0, float *dinp, float *slab) {
    extern __shared__ float ib[];
    constexpr int k0p = K0P;
    float *sd = ib, *sx = sd + kIbPoints * kIbRow, *sw = sx + kIbPoints * k0p;
    const int tid = threadIdx.x;
    // W0 [o][j] as [group o / 32][(o % 32) k0p + j] + 4 per group (the groups'
    // rows in different banks)
    for (int i = tid; i < W * k0p; i += kIbThreads) {
        const int o = i / k0p, j = i % k0p;
        sw[(o >> 5) * (32 * k0p + 4) + (o & 31) * k0p + j] = j < K0 ? W0[(size_t)o * K0 + j] : 0.f;
    }
    const int pq = tid >> 3, og = tid & 7;           // dinp: points 2 pq, 2 pq + 1; group og
    const int qt = tid >> 6, c4 = 4 * (tid & 63);    // dW0: points 16 qt .. + 15; channels c4 .. + 3
    float acc[4][K0P + 1];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j <= K0P; ++j) acc[u][j] = 0.f;
    const int ntiles = (n + kIbPoints - 1) / kIbPoints, w8 = W / 8;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int p0 = tile * kIbPoints;
        __syncthreads();                 // the previous tile is no longer read
        // the tile's 8-channel pieces (kIbPoints * w8 = 8 W of them, a multiple
        // of the block size) in rounds of four per thread: a round's loads
        // are all issued before any of them is converted and stored
        for (int q0 = 0; q0 < kIbPoints * w8; q0 += kIbLoads * kIbThreads) {
            uint4 ra[kIbLoads], rb[kIbLoads];
#pragma unroll
            for (int i = 0; i < kIbLoads; ++i) {
                const int q = q0 + i * kIbThreads + tid;
                const int pt = q / w8, c8 = (q % w8) * 8, p = p0 + pt;
                ra[i] = rb[i] = make_uint4(0u, 0u, 0u, 0u);
                if (q < kIbPoints * w8 && p < n) {
                    if (d32) {
                        ra[i] = *reinterpret_cast<const uint4 *>(d32 + (size_t)p * ld + c8);
                        rb[i] = *reinterpret_cast<const uint4 *>(d32 + (size_t)p * ld + c8 + 4);
                    } else {
                        ra[i] = __ldg(reinterpret_cast<const uint4 *>(dhi + (size_t)p * ld + c8));
                        rb[i] = __ldg(reinterpret_cast<const uint4 *>(dlo + (size_t)p * ld + c8));
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < kIbLoads; ++i) {
                const int q = q0 + i * kIbThreads + tid;
                if (q >= kIbPoints * w8) break;
                const int pt = q / w8, c8 = (q % w8) * 8;
                float v[8];
                if (d32) {
                    v[0] = __uint_as_float(ra[i].x); v[1] = __uint_as_float(ra[i].y);
                    v[2] = __uint_as_float(ra[i].z); v[3] = __uint_as_float(ra[i].w);
                    v[4] = __uint_as_float(rb[i].x); v[5] = __uint_as_float(rb[i].y);
                    v[6] = __uint_as_float(rb[i].z); v[7] = __uint_as_float(rb[i].w);
                } else {
                    // bf16 hi + lo pairs (zero pairs past n give zero)
                    const uint32_t hw[4] = {ra[i].x, ra[i].y, ra[i].z, ra[i].w},
                                   lw[4] = {rb[i].x, rb[i].y, rb[i].z, rb[i].w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        v[2 * t] = __uint_as_float(hw[t] << 16) + __uint_as_float(lw[t] << 16);
                        v[2 * t + 1] = __uint_as_float(hw[t] & 0xFFFF0000u) +
                                       __uint_as_float(lw[t] & 0xFFFF0000u);
                    }
                }
                float *dst = sd + pt * kIbRow + (c8 >> 5) * 33 + (c8 & 31);
#pragma unroll
                for (int t = 0; t < 8; ++t) dst[t] = v[t];
            }
        }
        for (int q = tid; q < kIbPoints * k0p; q += kIbThreads) {
            const int pt = q / k0p, j = q % k0p, p = p0 + pt;
            sx[q] = (p < n && j < K0) ? inp[(size_t)p * K0 + j] : 0.f;
        }
        __syncthreads();
        {
            // this group's channels (W % 32 == 0: a group is whole or absent),
            // then a fixed-order sum over the 8 groups that every lane takes part in
            float s0[K0P], s1[K0P];
#pragma unroll
            for (int j = 0; j < K0P; ++j) s0[j] = s1[j] = 0.f;
            if (og * 32 < W) {
                const float *dp0 = sd + (2 * pq) * kIbRow + og * 33, *dp1 = dp0 + kIbRow;
                const float *wp = sw + og * (32 * k0p + 4);
#pragma unroll 4
                for (int oi = 0; oi < 32; ++oi) {
                    const float d0 = dp0[oi], d1 = dp1[oi];
#pragma unroll
                    for (int j4 = 0; j4 < K0P; j4 += 4) {
                        const float4 w = *reinterpret_cast<const float4 *>(wp + oi * k0p + j4);
                        s0[j4] = fmaf(w.x, d0, s0[j4]);
                        s0[j4 + 1] = fmaf(w.y, d0, s0[j4 + 1]);
                        s0[j4 + 2] = fmaf(w.z, d0, s0[j4 + 2]);
                        s0[j4 + 3] = fmaf(w.w, d0, s0[j4 + 3]);
                        s1[j4] = fmaf(w.x, d1, s1[j4]);
                        s1[j4 + 1] = fmaf(w.y, d1, s1[j4 + 1]);
                        s1[j4 + 2] = fmaf(w.z, d1, s1[j4 + 2]);
                        s1[j4 + 3] = fmaf(w.w, d1, s1[j4 + 3]);
                    }
                }
            }
#pragma unroll
            for (int off = 1; off < 8; off <<= 1)
#pragma unroll
                for (int j = 0; j < K0P; ++j) {
                    s0[j] += __shfl_xor_sync(0xffffffffu, s0[j], off);
                    s1[j] += __shfl_xor_sync(0xffffffffu, s1[j], off);
                }
            const int p = p0 + 2 * pq;
#pragma unroll
            for (int j = 0; j < K0P; ++j)
                if (j < K0 && (j & 7) == og) {
                    if (p < n) dinp[(size_t)p * K0 + j] = s0[j];
                    if (p + 1 < n) dinp[(size_t)(p + 1) * K0 + j] = s1[j];
                }
        }
        if (c4 < W) {
            const float *dcol = sd + (c4 >> 5) * 33 + (c4 & 31);
#pragma unroll 4
            for (int pt = 16 * qt; pt < 16 * qt + 16; ++pt) {
                const float d[4] = {dcol[pt * kIbRow], dcol[pt * kIbRow + 1], dcol[pt * kIbRow + 2],
                                    dcol[pt * kIbRow + 3]};
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u][K0P] += d[u];
#pragma unroll
                for (int j4 = 0; j4 < K0P; j4 += 4) {
                    const float4 x = *reinterpret_cast<const float4 *>(sx + pt * k0p + j4);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        acc[u][j4] = fmaf(d[u], x.x, acc[u][j4]);
                        acc[u][j4 + 1] = fmaf(d[u], x.y, acc[u][j4 + 1]);
                        acc[u][j4 + 2] = fmaf(d[u], x.z, acc[u][j4 + 2]);
                        acc[u][j4 + 3] = fmaf(d[u], x.w, acc[u][j4 + 3]);
                    }
                }
            }
        }
    }
    // the four point quarters' sums, added in quarter order
    __syncthreads();
    float *comb = ib;                    // [quarter][channel][k0p + 1]
    if (c4 < W)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j <= K0P; ++j) comb[((size_t)qt * W + c4 + u) * (k0p + 1) + j] = acc[u][j];
    __syncthreads();
    float *mine = slab + (size_t)blockIdx.x * ((size_t)W * K0 + W);
    for (int e = tid; e < W * (K0 + 1); e += kIbThreads) {
        const int o = e / (K0 + 1), j = e % (K0 + 1), jj = j < K0 ? j : K0P;
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) t += comb[((size_t)q * W + o) * (k0p + 1) + jj];
        if (j < K0) mine[(size_t)o * K0 + j] = t;
        else mine[(size_t)W * K0 + o] = t;
    }
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

// The same for a bf16 B with contiguous k (the output layer's forward
// product on the BF16 path): one warp per column n, lane l multiplying k =
// 8 l .. 8 l + 7 (one 16-byte load of B's row; A's matching values held in
// registers for all the warp's columns), then a fixed xor-shuffle sum over the
// lanes.  A row of B is read as one 512-byte stretch by the warp.
template <int NM>
__global__ void __launch_bounds__(256)
k_thin_m_warp(int M, int N, int K, const MatView A, const __nv_bfloat16 *__restrict__ B,
              long long ldb, float *out, long long ld) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const bool act = 8 * lane < K;
    float a[NM][8];
#pragma unroll
    for (int m = 0; m < NM; ++m)
#pragma unroll
        for (int j = 0; j < 8; ++j) a[m][j] = (act && m < M) ? view_at(A, m, 8 * lane + j) : 0.f;
    constexpr int kU = 4;                       // columns whose loads are in flight together
    for (int n0 = warp; n0 < N; n0 += kU * nwarps) {
        uint4 q[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int n = n0 + u * nwarps;
            q[u] = (act && n < N) ? __ldg(reinterpret_cast<const uint4 *>(B + (size_t)n * ldb) + lane)
                                  : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int n = n0 + u * nwarps;
            const uint32_t w[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
            float acc[NM];
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                acc[m] = 0.f;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    acc[m] = fmaf(a[m][2 * t], __uint_as_float(w[t] << 16), acc[m]);
                    acc[m] = fmaf(a[m][2 * t + 1], __uint_as_float(w[t] & 0xFFFF0000u), acc[m]);
                }
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
                for (int m = 0; m < NM; ++m) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], off);
            if (n < N)
#pragma unroll
                for (int m = 0; m < NM; ++m)
                    if (m < M && lane == m) out[(size_t)n * ld + m] = acc[m];
        }
    }
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
// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point
// query (no link against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// The tensor map of a bf16 operand with `rows` rows and K columns, stride
// `stride` elements along its strided dimension, 128-byte swizzle: boxes of
// 64 k x 128 rows (K-major) or 64 rows x 64 k (MN-major); out-of-range
// elements read as zero.
bool operand_map(CUtensorMap *map, const void *ptr, bool mn, int rows, int K, long long stride,
                 int box_rows = 128) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
    if (!fn) return false;
    cuuint64_t dims[2], strides[1] = {(cuuint64_t)stride * 2};
    cuuint32_t box[2], es[2] = {1, 1};
    if (mn) {
        dims[0] = (cuuint64_t)rows; dims[1] = (cuuint64_t)K;
        box[0] = 64; box[1] = 64;
    } else {
        dims[0] = (cuuint64_t)K; dims[1] = (cuuint64_t)rows;
        box[0] = 64; box[1] = (cuuint32_t)box_rows;
    }
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides,
              box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <bool AMN, bool BMN, int SPLIT, int EPI>
cudaError_t launch_tc(const CUtensorMap &mA, const CUtensorMap &mB, const CUtensorMap &mLo,
                      const WsShape &g, const GemmEpilogue &e, int *status, cudaStream_t s) {
    static bool attr = false;
    set_max_dynamic_smem(k_gemm_tc<AMN, BMN, SPLIT, EPI>, attr);
    const int grid = g.units < sm_count() ? g.units : sm_count();
    k_gemm_tc<AMN, BMN, SPLIT, EPI><<<grid, kWsThreads, ws_smem_bytes(SPLIT != 0), s>>>(
        mA, mB, mLo, g, e, status);
    return cudaGetLastError();
}
}  // namespace

namespace {
// One CTA per SM at most, a multiple of the column-tile count.
int layer_grid(int units, int tiles_n) {
    int grid = units < sm_count() ? units : sm_count();
    grid -= grid % tiles_n;
    return grid < tiles_n ? tiles_n : grid;
}

template <bool SPLIT, int EPI>
cudaError_t launch_layer(const CUtensorMap &mX, const CUtensorMap &mXlo, const CUtensorMap &mW,
                         const LayerShape &g, const GemmEpilogue &e, int *status, cudaStream_t s) {
    static bool attr = false;
    set_max_dynamic_smem(k_layer_tc<SPLIT, EPI>, attr);
    k_layer_tc<SPLIT, EPI><<<layer_grid(g.units, g.tiles_n), kLThreads,
                             layer_smem_bytes(g.K, SPLIT, g.stages), s>>>(mX, mXlo, mW, g, e, status);
    return cudaGetLastError();
}
}  // namespace

int layer_tc_parts(int n, int W) {
    const int tiles_n = (W + kLN - 1) / kLN;
    return 4 * layer_grid(((n + kLP - 1) / kLP) * tiles_n, tiles_n) / tiles_n;
}

cudaError_t layer_tc(int n, int W, int K, const MatView &X, const MatView &Wt,
                     const GemmEpilogue &e, int *status, cudaStream_t s) {
    if (n <= 0 || W <= 0) return cudaSuccess;
    const bool split = X.lo != nullptr;
    if (W > NSF_MAX_WIDTH || W % 16 || K <= 0 || K > NSF_MAX_WIDTH || e.ld % 8 || !e.dact)
        return cudaErrorInvalidValue;
    if (!X.bf16 || !Wt.bf16 || X.s_k != 1 || Wt.s_k != 1 || X.s_row % 8 || Wt.s_row % 8)
        return cudaErrorInvalidValue;
    auto al16 = [](const void *p) { return p == nullptr || ((size_t)p & 15) == 0; };
    if (!al16(X.ptr) || !al16(X.lo) || !al16(Wt.ptr) || !al16(e.dact)) return cudaErrorInvalidValue;
    if (e.mode == kEpiBiasElu) {
        if (split || !e.h16 || !al16(e.h16)) return cudaErrorInvalidValue;
    } else if (e.mode == kEpiEluGrad) {
        if (!split || !e.dhi || !e.dlo || !al16(e.dhi) || !al16(e.dlo) || !al16(e.out))
            return cudaErrorInvalidValue;
    } else {
        return cudaErrorInvalidValue;
    }
    LayerShape g;
    g.n = n;
    g.W = W;
    g.K = K;
    g.ld = e.ld;
    g.tiles_n = (W + kLN - 1) / kLN;
    g.units = ((n + kLP - 1) / kLP) * g.tiles_n;
    const int fixed = layer_smem_bytes(K, split, 0);
    g.stages = (kMaxSmem - fixed) / layer_stage_bytes(split);
    if (g.stages > kLStagesMax) g.stages = kLStagesMax;
    if (g.stages < 2) return cudaErrorInvalidValue;
    CUtensorMap mX, mXlo, mW;
    if (!operand_map(&mX, X.ptr, false, n, K, X.s_row)) return cudaErrorInvalidValue;
    mXlo = mX;
    if (split && !operand_map(&mXlo, X.lo, false, n, K, X.s_row)) return cudaErrorInvalidValue;
    if (!operand_map(&mW, Wt.ptr, false, W, K, Wt.s_row)) return cudaErrorInvalidValue;
    if (e.mode == kEpiBiasElu) return launch_layer<false, kEpiBiasElu>(mX, mXlo, mW, g, e, status, s);
    return launch_layer<true, kEpiEluGrad>(mX, mXlo, mW, g, e, status, s);
}

// The weight-gradient shape of training: the cotangent's hi/lo pairs and the
// activations, both with contiguous rows, K-slices into slabs.
cudaError_t gemm_tc(int M, int N, int K, const MatView &A, const MatView &B, int split,
                    const GemmEpilogue &e, int kslices, int *status, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (kslices < 1 || (kslices > 1 && e.mode != kEpiSlab)) return cudaErrorInvalidValue;
    WsShape g;
    g.M = M;
    g.N = N;
    g.K = K;
    g.kper = slice_len(K, kslices, kTK);
    g.tiles_m = (M + kTM - 1) / kTM;
    g.tiles_n = (N + kTN - 1) / kTN;
    g.units = g.tiles_m * g.tiles_n * (e.mode == kEpiSlab ? kslices : 1);
    const bool a_mn = A.s_row == 1 && A.s_k != 1, b_mn = B.s_row == 1 && B.s_k != 1;
    // bf16 operands, 16-byte aligned, strides multiples of 16 bytes
    auto ok = [&](const MatView &V, bool mn, bool lo) {
        if (!V.bf16 || (lo && !V.lo)) return false;
        const long long stride = mn ? V.s_k : V.s_row;
        if ((mn ? V.s_row : V.s_k) != 1 || stride % 8 || stride <= 0) return false;
        return !((((size_t)V.ptr) & 15) || (lo && (((size_t)V.lo) & 15)));
    };
    if (!ok(A, a_mn, split == 1) || !ok(B, b_mn, split == 2)) return cudaErrorInvalidValue;
    CUtensorMap mA, mB, mLo;
    if (!operand_map(&mA, A.ptr, a_mn, M, K, a_mn ? A.s_k : A.s_row) ||
        !operand_map(&mB, B.ptr, b_mn, N, K, b_mn ? B.s_k : B.s_row))
        return cudaErrorInvalidValue;
    mLo = mA;
    if (split == 1 && !operand_map(&mLo, A.lo, a_mn, M, K, a_mn ? A.s_k : A.s_row))
        return cudaErrorInvalidValue;
    if (split == 2 && !operand_map(&mLo, B.lo, b_mn, N, K, b_mn ? B.s_k : B.s_row))
        return cudaErrorInvalidValue;
    if (a_mn && b_mn && split == 1 && e.mode == kEpiSlab)
        return launch_tc<true, true, 1, kEpiSlab>(mA, mB, mLo, g, e, status, s);
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
        return reduce_slabs(slab, slices, count, out, s);
    return cudaGetLastError();
}

cudaError_t thin_m(int M, int N, int K, const MatView &A, const MatView &B, float *out,
                   long long ld, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (M > kThinA || K > kThinMaxK) return cudaErrorInvalidValue;
    if (B.bf16 && B.s_k == 1 && K % 8 == 0 && B.s_row % 8 == 0 && (((size_t)B.ptr) & 15) == 0 &&
        M <= 16) {
        const int grid = 2 * sm_count();   // two CTAs of 8 warps a SM share the columns
        const __nv_bfloat16 *b = reinterpret_cast<const __nv_bfloat16 *>(B.ptr);
        if (M <= 4) k_thin_m_warp<4><<<grid, 256, 0, s>>>(M, N, K, A, b, B.s_row, out, ld);
        else if (M <= 8) k_thin_m_warp<8><<<grid, 256, 0, s>>>(M, N, K, A, b, B.s_row, out, ld);
        else if (M <= 12) k_thin_m_warp<12><<<grid, 256, 0, s>>>(M, N, K, A, b, B.s_row, out, ld);
        else k_thin_m_warp<16><<<grid, 256, 0, s>>>(M, N, K, A, b, B.s_row, out, ld);
        return cudaGetLastError();
    }
    const int g = (N + kThinThreads - 1) / kThinThreads;
    if (M <= 4) k_thin_m<4><<<g, kThinThreads, 0, s>>>(M, N, K, A, B, out, ld);
    else if (M <= 16) k_thin_m<16><<<g, kThinThreads, 0, s>>>(M, N, K, A, B, out, ld);
    else k_thin_m<32><<<g, kThinThreads, 0, s>>>(M, N, K, A, B, out, ld);
    return cudaGetLastError();
}

int thin_k_parts(int N) { return (N + kTkPoints - 1) / kTkPoints; }

int input_bwd_parts(int n) {
    const int tiles = (n + kIbPoints - 1) / kIbPoints;
    int grid = 2 * sm_count();
    if (grid > kIbMaxGrid) grid = kIbMaxGrid;
    return tiles < grid ? tiles : grid;
}

cudaError_t input_bwd(int n, int W, int K0, const __nv_bfloat16 *dhi, const __nv_bfloat16 *dlo,
                      const float *d32, long long ld, const float *inp, const float *W0,
                      float *dinp, float *slab, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (W % 32 || W > NSF_MAX_WIDTH || K0 < 1 || K0 > kThinKMax || ld % 8) return cudaErrorInvalidValue;
    if (!d32 && (!dhi || !dlo)) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_input_bwd<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ib_smem(4));
        cudaFuncSetAttribute(k_input_bwd<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ib_smem(8));
        cudaFuncSetAttribute(k_input_bwd<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ib_smem(12));
        cudaFuncSetAttribute(k_input_bwd<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ib_smem(16));
        cudaFuncSetAttribute(k_input_bwd<20>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ib_smem(20));
        attr = true;
    }
    const int grid = input_bwd_parts(n), k0p = ib_k0p(K0);
    const size_t smem = ib_smem(K0);
#define NSF_IB(P_) k_input_bwd<P_><<<grid, kIbThreads, smem, s>>>(n, W, K0, dhi, dlo, d32, ld, inp, W0, dinp, slab)
    if (k0p == 4) NSF_IB(4);
    else if (k0p == 8) NSF_IB(8);
    else if (k0p == 12) NSF_IB(12);
    else if (k0p == 16) NSF_IB(16);
    else NSF_IB(20);
#undef NSF_IB
    return cudaGetLastError();
}

cudaError_t thin_k(int M, int N, int K, const MatView &A, const MatView &B,
                   const GemmEpilogue &e, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (K < 1 || K > kThinKMax || M % 4 || M > NSF_MAX_WIDTH || e.ld % 4 || !e.dact)
        return cudaErrorInvalidValue;
    auto al = [](const void *p, int a) { return (((size_t)p) % a) == 0; };
    if (!al(e.dact, 8)) return cudaErrorInvalidValue;
    if (e.mode == kEpiBiasElu && (!e.h16 || !al(e.h16, 8))) return cudaErrorInvalidValue;
    if (e.mode == kEpiEluGrad &&
        (!e.dhi || !e.dlo || !al(e.dhi, 8) || !al(e.dlo, 8) || (e.out && !al(e.out, 16))))
        return cudaErrorInvalidValue;
    if (e.mode == kEpiEluGrad && e.hin && (K > kMaxOut || !e.outer || !al(e.hin, 8)))
        return cudaErrorInvalidValue;
    const size_t smem = thin_k_smem(M, K);
    const int grid = thin_k_parts(N), nk = thin_k_nk(K);
#define NSF_TK(EPI_, NK_) k_thin_k<EPI_, NK_><<<grid, kTkThreads, smem, s>>>(M, N, K, A, B, e)
    if (e.mode == kEpiBiasElu) {
        if (nk == 4) NSF_TK(kEpiBiasElu, 4);
        else if (nk == 8) NSF_TK(kEpiBiasElu, 8);
        else if (nk == 12) NSF_TK(kEpiBiasElu, 12);
        else if (nk == 16) NSF_TK(kEpiBiasElu, 16);
        else NSF_TK(kEpiBiasElu, 20);
    } else if (e.mode == kEpiEluGrad) {
        if (nk == 4) NSF_TK(kEpiEluGrad, 4);
        else if (nk == 8) NSF_TK(kEpiEluGrad, 8);
        else if (nk == 12) NSF_TK(kEpiEluGrad, 12);
        else if (nk == 16) NSF_TK(kEpiEluGrad, 16);
        else NSF_TK(kEpiEluGrad, 20);
    } else {
        return cudaErrorInvalidValue;
    }
#undef NSF_TK
    return cudaGetLastError();
}

// Element-wise accumulation of float or float4 values (same order per element).
template <class T> __device__ __forceinline__ T vzero();
template <> __device__ __forceinline__ float vzero<float>() { return 0.f; }
template <> __device__ __forceinline__ float4 vzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void vadd(float &a, float b) { a += b; }
__device__ __forceinline__ void vadd(float4 &a, const float4 &b) {
    a.x += b.x;
    a.y += b.y;
    a.z += b.z;
    a.w += b.w;
}

// Weight and bias gradients of a hidden layer from the K-slices of the
// weight-gradient product: slab[z][n][m] (z < slices, n < N, m < M) ->
// out_w[m N + n] and bslab[z][m] -> out_b[m], each a fixed-order sum over z.
// A CTA takes 32 V consecutive slab entries (a lane V of them, coalesced
// reads), 8 groups of slices each, then a shared sum in group order; the
// CTAs past the M N / (32 V) of the weights do the same for the bias slab.
// V = 4 needs M % 4 == 0 and 16-byte aligned slabs.
template <int V>
__global__ void k_reduce_dw(const float *__restrict__ slab, const float *__restrict__ bslab,
                            int slices, int M, int N, float *out_w, float *out_b) {
    using Vec = typename std::conditional<V == 4, float4, float>::type;
    __shared__ Vec part[8][33];
    const int ix = threadIdx.x & 31, g = threadIdx.x >> 5;
    const long long count = (long long)M * N, wblocks = (count + 32 * V - 1) / (32 * V);
    const bool bias = blockIdx.x >= wblocks;
    const long long i = ((bias ? blockIdx.x - wblocks : blockIdx.x) * 32 + ix) * V;
    const long long cnt = bias ? M : count;
    const float *src = bias ? bslab : slab;
    auto ld = [&](int z) { return *reinterpret_cast<const Vec *>(src + (size_t)z * cnt + i); };
    Vec s = vzero<Vec>();
    if (i < cnt) {
        int z = g;
        for (; z + 24 < slices; z += 32) {
            const Vec a = ld(z), b = ld(z + 8), c = ld(z + 16), d = ld(z + 24);
            vadd(s, a);
            vadd(s, b);
            vadd(s, c);
            vadd(s, d);
        }
        for (; z < slices; z += 8) vadd(s, ld(z));
    }
    part[g][ix] = s;
    __syncthreads();
    if (g == 0 && i < cnt) {
        Vec t = vzero<Vec>();
#pragma unroll
        for (int q = 0; q < 8; ++q) vadd(t, part[q][ix]);
        const float *tv = reinterpret_cast<const float *>(&t);
#pragma unroll
        for (int u = 0; u < V; ++u) {
            if (bias) out_b[i + u] = tv[u];
            else out_w[(size_t)((i + u) % M) * N + (i + u) / M] = tv[u];
        }
    }
}

cudaError_t reduce_dw(const float *slab, const float *bslab, int slices, int M, int N,
                      float *out_w, float *out_b, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    const bool vec = M % 4 == 0 && ((uintptr_t)slab % 16) == 0 &&
                     (out_b == nullptr || ((uintptr_t)bslab % 16) == 0);
    const int V = vec ? 4 : 1;
    const long long wblocks = ((long long)M * N + 32 * V - 1) / (32 * V);
    const int blocks = (int)wblocks + (out_b ? (M + 32 * V - 1) / (32 * V) : 0);
    if (vec) k_reduce_dw<4><<<blocks, 256, 0, s>>>(slab, bslab, slices, M, N, out_w, out_b);
    else k_reduce_dw<1><<<blocks, 256, 0, s>>>(slab, bslab, slices, M, N, out_w, out_b);
    return cudaGetLastError();
}

// Few outputs over many slabs (the bias column sums): first sums of groups of
// rows in place, one CTA per group, then the sum of the groups' results.
// The slab is overwritten.
cudaError_t reduce_slabs(float *slab, int slices, long long count, float *out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int cx = (int)((count + 31) / 32);
    int groups = 1;
    if (slices >= 64 && cx < sm_count()) {
        groups = (2 * sm_count() + cx - 1) / cx;
        if (groups > slices / 16) groups = slices / 16;
    }
    if (groups > 1) {
        const int per = (slices + groups - 1) / groups;
        groups = (slices + per - 1) / per;
        k_reduce_slabs<<<dim3(cx, groups), 256, 0, s>>>(slab, slices, per, count, count, slab,
                                                         (long long)per * count);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_reduce_slabs<<<dim3(cx, 1), 256, 0, s>>>(slab, groups, groups, (long long)per * count,
                                                    count, out, 0);
        return cudaGetLastError();
    }
    k_reduce_slabs<<<dim3(cx, 1), 256, 0, s>>>(slab, slices, slices, count, count, out, 0);
    return cudaGetLastError();
}

}  // namespace nsf
