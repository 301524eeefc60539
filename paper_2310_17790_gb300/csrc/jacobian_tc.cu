// Jacobian of the deformation field g (forward mode) and the Gauss-Newton
// network inversion on the tcgen05 tensor cores (paper §5.3, Eq. 9; App. E:
// ELU MLP on [X; z]), BF16 operands with FP32 accumulation.
//
// Transposed products: the MMA rows are a layer's output neurons and its
// columns are the tile's point slots.  Each point owns L consecutive columns
// (L the smallest power of two >= 1 + r): slot 0 carries the value, slot 1 + k
// the tangent along latent component k (slots beyond r stay zero).  The
// accumulator D = W_l [h | t_1 .. t_r] then sits in tensor memory with lane =
// neuron and column = point slot, so the thread that owns neuron j holds a
// point's pre-activation and all of its tangents in its own registers, and
// ELU'(a_value) scales the tangents with no exchange between threads.  The
// thread writes its neuron's row of the next layer's B operand (MN-major:
// point slots contiguous per neuron).
//
// CTA: eight warpgroups.  Warp (index % 4) = q reads TMEM lanes 32 q .. 32 q +
// 31, i.e. neurons 32 q + lane (and 128 + 32 q + lane from a second
// accumulator for widths above 128); warpgroup w owns columns [w CW,
// (w + 1) CW), CW = max(8, L), so a tile has N = 8 CW columns and P = N / L
// points.  The per-layer latency grows with the columns a thread handles, so
// tiles stay small (8 points for r >= 3) and a point set spreads over many
// SMs.  Layer 0 (K = 3 + r) runs on the CUDA cores: value slot W0[:, :3] X
// + (b0 + W0[:, 3:] z), tangent slot k the column W0[:, 3 + k].  The output
// layer is an MMA with M = 128 whose first out_dim rows are the output
// weights.
//
// Products with M = 128 read 128 weight rows per K atom; for layers with fewer
// rows (widths below 128, the output layer's 16 rows, the second half of width
// 192) the extra rows are whatever follows in shared memory: the next layer's
// weights or the activation operand, which is placed right after the weights
// and takes at least 16 KB.  Those rows only produce accumulator lanes that no
// thread reads.
//
// Gauss-Newton (gn_on): all iterations in one cooperative launch; after its
// tiles every CTA combines the float-float normal equations of all CTAs and
// solves them itself (gn_ff.cuh), keeping z in shared memory.
#include "gn_ff.cuh"
#include "tc_common.cuh"

namespace nsf {

using namespace tc;

namespace {

constexpr int kBatchWG = 4;             // warpgroups per CTA of the batched kernel

__host__ __device__ inline int jac_slots(int r) {
    int L = 2;
    while (L < 1 + r) L <<= 1;
    return L;
}
__host__ __device__ inline int jac_cw(int r) {
    const int L = jac_slots(r);
    return L > 8 ? L : 8;
}
__host__ __device__ inline int jac_cols(int r) { return kWG * jac_cw(r); }
__host__ __device__ inline int jac_points(int r) { return jac_cols(r) / jac_slots(r); }
__host__ __device__ inline int jac_halves(int W) { return (W + 127) / 128; }

// Shared-memory carve of one CTA (byte offsets from a 1024-aligned base).
struct JacLayout {
    int blob, b, w0v, w0t, b0, bias, xs, tg, o3, bars, tmem, total;
};

// Layout for CW columns per warpgroup (N = 8 CW slots, N / L points per tile).
__host__ __device__ inline JacLayout jac_layout(int r, int W, int D, int CW, int NWG = kWG) {
    JacLayout L;
    const int N = NWG * CW, P = N / jac_slots(r);
    int o = 0;
    L.blob = o; o = align_to(o + (D - 1) * W * W * 2 + kMaxOut * W * 2, 1024);
    // activations (MN-major); at least 16 KB, the reach of the padded rows
    // of an M = 128 product past the end of the weights
    L.b = o;    o = align_to(o + (W * N * 2 > 16384 ? W * N * 2 : 16384), 1024);
    L.w0v = o;  o = align_to(o + W * 16, 16);                  // float4 {w_x, w_y, w_z, c0}
    L.w0t = o;  o = align_to(o + r * W * 4, 16);               // W0[:, 3 + k] as [k][W]
    L.b0 = o;   o = align_to(o + W * 4, 16);                   // input-layer bias
    L.bias = o; o = align_to(o + D * W * 4, 16);               // hidden biases, output bias
    L.xs = o;   o = align_to(o + P * 16, 16);                  // tile positions
    L.tg = o;   o = align_to(o + P * 16, 16);                  // tile Gauss-Newton targets
    L.o3 = o;   o = align_to(o + (3 * N + N / 8) * 4, 16);     // outputs, a pad per 8 columns
    L.bars = o; o = align_to(o + 2 * 8, 16);
    L.tmem = o; o = align_to(o + 16, 16);
    L.total = o + 1024;
    return L;
}

// Byte offset of the 16-byte chunk of B holding neuron k, columns n .. n + 7
// (n % 8 == 0): MN-major, 64-column blocks 1024 bytes apart, 8-neuron blocks
// sbo = (N / 64) * 1024 bytes apart.
__device__ __forceinline__ int b_chunk(int k, int n, int sbo) {
    return (k >> 3) * sbo + (n >> 6) * 1024 + (k & 7) * 128 + ((((n >> 3) & 7) ^ (k & 7)) << 4);
}

template <int CW>
__device__ __forceinline__ void store_b_row(uint8_t *B, int k, int n0, int sbo, const float *v) {
#pragma unroll
    for (int g = 0; g < CW / 8; ++g)
        *reinterpret_cast<uint4 *>(B + b_chunk(k, n0 + 8 * g, sbo)) = pack_bf16x8(v + 8 * g);
}

// One CTA's share of a Jacobian evaluation or Gauss-Newton run: the CTA is
// `rank` of the `gsize` CTAs that work on this point set (tiles rank, rank +
// gsize, ...) and, for Gauss-Newton, combine their sums behind gn.bar.  The
// CTA has NWG warpgroups of CW columns each (a tile of NWG CW point slots).
// Input-layer epilogue of one chunk of kC columns holding kC / LT whole
// points of LT slots: the value slot of a point is ELU(a), a = W0 [x; z] + b0
// (the z part folded into w.w), tangent slot s (1 <= s <= r) is
// ELU'(a) W0[:, 3 + s - 1], the slots past r are zero.  w0t points at this
// neuron's entry of the first z column of W0 (columns W apart); x at the
// chunk's first point.
template <int kC, int LT>
__device__ __forceinline__ void input_tangents(float *v, float4 w, const float4 *x, const float *w0t,
                                               int W, int r) {
    float t[LT];
    t[0] = 0.f;
#pragma unroll
    for (int s = 1; s < LT; ++s) t[s] = s <= r ? w0t[(s - 1) * W] : 0.f;
#pragma unroll
    for (int p = 0; p < kC; p += LT) {
        const float4 xp = x[p / LT];
        float g;
        v[p] = elu_fast(fmaf(w.x, xp.x, fmaf(w.y, xp.y, fmaf(w.z, xp.z, w.w))), g);
#pragma unroll
        for (int s = 1; s < LT; ++s) v[p + s] = g * t[s];
    }
}

// Hidden-layer epilogue of one chunk: ELU on each point's value slot (sum +
// bias b) and the chain rule ELU'(a) (W dh/dz) on its tangent slots.  Slots
// past r hold exact zeros (zero columns in, zero products out) and stay zero.
template <int kC, int LT>
__device__ __forceinline__ void elu_tangents(float *v, float b) {
#pragma unroll
    for (int p = 0; p < kC; p += LT) {
        float g;
        v[p] = elu_fast(v[p] + b, g);
        v[p + 1] *= g;
#pragma unroll
        for (int s = 2; s < LT; s += 2) {
            const float2 t = __fmul2_rn(make_float2(v[p + s], v[p + s + 1]), make_float2(g, g));
            v[p + s] = t.x;
            v[p + s + 1] = t.y;
        }
    }
}

// The two epilogues for the run-time slot count L (a power of two, 2 <= L <=
// kC): one uniform branch per chunk, straight-line code inside.
template <int kC>
__device__ __forceinline__ void input_tangents_l(int L, float *v, float4 w, const float4 *x,
                                                 const float *w0t, int W, int r) {
    if (L == 2) input_tangents<kC, 2>(v, w, x, w0t, W, r);
    else if (L == 4) input_tangents<kC, 4>(v, w, x, w0t, W, r);
    else if (L == 8) input_tangents<kC, 8>(v, w, x, w0t, W, r);
    else if (L == 16) { if constexpr (kC >= 16) input_tangents<kC, 16>(v, w, x, w0t, W, r); }
    else { if constexpr (kC >= 32) input_tangents<kC, 32>(v, w, x, w0t, W, r); }
}

template <int kC>
__device__ __forceinline__ void elu_tangents_l(int L, float *v, float b) {
    if (L == 2) elu_tangents<kC, 2>(v, b);
    else if (L == 4) elu_tangents<kC, 4>(v, b);
    else if (L == 8) elu_tangents<kC, 8>(v, b);
    else if (L == 16) { if constexpr (kC >= 16) elu_tangents<kC, 16>(v, b); }
    else { if constexpr (kC >= 32) elu_tangents<kC, 32>(v, b); }
}

template <int CW, int NWG = kWG>
__device__ void jac_body(const FieldsDev &fd, const float *__restrict__ X, int n, int ld,
                         const double *zj, float *u, float *dudz, const GnArgs &gn, int gn_on,
                         int rank, int gsize, bool last_alloc, uint8_t *smem_dyn, int *status) {
    __shared__ int s_abort;
    uint8_t *base = aligned_smem(smem_dyn);

    const FieldDev &F = fd.f[NSF_FIELD_G];
    const int W = F.width, D = F.depth, r = fd.r;
    const int L = jac_slots(r);
    const int lgL = __ffs(L) - 1;
    constexpr int N = NWG * CW;              // columns (point slots) per tile
    const int P = N / L;                     // points per tile
    const int MH = jac_halves(W);            // 128-neuron accumulators
    const int tiles = (n + P - 1) / P;
    const int tid = threadIdx.x;
    const int wg = tid >> 7;
    const int wq = (tid >> 5) & 3;           // TMEM lane quarter of this warp
    const int lane = tid & 31;
    const int n0 = wg * CW;                  // first column of this warpgroup
    const int sbo_b = (N / 64) * 1024;
    const JacLayout Lo = jac_layout(r, W, D, CW, NWG);
    uint8_t *blob = base + Lo.blob;
    uint8_t *B = base + Lo.b;
    float4 *W0v = reinterpret_cast<float4 *>(base + Lo.w0v);
    float *W0t = reinterpret_cast<float *>(base + Lo.w0t);
    float *b0s = reinterpret_cast<float *>(base + Lo.b0);
    float *bias = reinterpret_cast<float *>(base + Lo.bias);
    float4 *xs = reinterpret_cast<float4 *>(base + Lo.xs);
    float4 *tg = reinterpret_cast<float4 *>(base + Lo.tg);
    float *O3 = reinterpret_cast<float *>(base + Lo.o3);
    uint64_t *bar_w = reinterpret_cast<uint64_t *>(base + Lo.bars);
    uint64_t *bar_mma = bar_w + 1;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(base + Lo.tmem);
    uint32_t ncols = 32;
    while ((int)ncols < MH * N) ncols <<= 1;
    const int n_iter = gn_on ? gn.iters : 1;

    if (tid == 0) {
        s_abort = 0;
        mbar_init(bar_w, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) tmem_alloc(tmem_holder, ncols, last_alloc);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (tid == 0) bulk_load(blob, F.tc_blob, (uint32_t)F.tc_blob_bytes, bar_w);
    const int in0 = 3 + r;
    for (int j = tid; j < W; j += NWG * kWgThreads) {
        const float *w = F.W0 + (size_t)j * in0;
        W0v[j] = make_float4(w[0], w[1], w[2], 0.f);
        b0s[j] = F.b[0][j];
        for (int k = 0; k < r; ++k) W0t[k * W + j] = w[3 + k];
    }
    for (int l = 1; l <= D; ++l) {
        const int o = l == D ? F.out_dim : W;
        for (int j = tid; j < o; j += NWG * kWgThreads) bias[(l - 1) * W + j] = F.b[l][j];
    }
    // positions (and Gauss-Newton targets) of a tile of this CTA
    auto load_tile = [&](int t0) {
        if (tid < P) {
            const int p = t0 + tid;
            const bool in = p < n;
            xs[tid] = in ? make_float4(X[p], X[ld + p], X[2 * ld + p], 0.f)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
            if (gn_on) {
                const int tl = gn.target_ld;
                tg[tid] = in ? make_float4(gn.target[p], gn.target[tl + p], gn.target[2 * tl + p], 0.f)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
    load_tile(rank * P);
    int loaded = rank;                       // the tile whose points xs, tg hold
    if (gn_on) gn_ff_begin(gn, r);
    bool weights_ready = false;
    const uint32_t blob_addr = smem_u32(blob);
    const uint32_t b_addr = smem_u32(B);
    const uint32_t idesc_h = idesc_bf16(kM, N, true);
    const uint32_t tq = tmem + ((uint32_t)(wq * 32) << 16);
    uint32_t phase = 0;

    for (int it = 0; it < n_iter; ++it) {
        __syncthreads();
        // z-part of the input layer folded into its bias: c0 = b0 + W0[:, 3:] z
        for (int j = tid; j < W; j += NWG * kWgThreads) {
            float a = b0s[j];
            for (int k = 0; k < r; ++k) {
                const float zk = gn_on ? g_gn.z[k].hi : (float)__ldcg(&zj[k]);
                a = fmaf(W0t[k * W + j], zk, a);
            }
            W0v[j].w = a;
        }
        __syncthreads();

        for (int tile = rank; tile < tiles; tile += gsize) {
            const int p0 = tile * P;
            if (tile != loaded) {
                // a CTA with several tiles reloads its first one in every
                // Gauss-Newton iteration after the first
                __syncthreads();
                load_tile(p0);
                __syncthreads();
                loaded = tile;
            }
            // ---- layer 0 on the CUDA cores: this thread's neurons, its columns
            for (int h = 0; h < MH; ++h) {
                const int j = h * 128 + wq * 32 + lane;
                if (j < W) {
                    const float4 w = W0v[j];
                    constexpr int kC0 = CW < 32 ? CW : 32;      // whole points per chunk
#pragma unroll
                    for (int c0 = 0; c0 < CW; c0 += kC0) {
                        float v[kC0];
                        input_tangents_l<kC0>(L, v, w, xs + ((n0 + c0) >> lgL), W0t + j, W, r);
                        store_b_row<kC0>(B, j, n0 + c0, sbo_b, v);
                    }
                }
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
                    const uint32_t aoff = (uint32_t)((l - 1) * W * W * 2);
                    const int arows = out_layer ? kMaxOut : W;
                    const int halves = out_layer ? 1 : MH;
                    for (int h = 0; h < halves; ++h) {
                        for (int ks = 0; ks < W / 16; ++ks) {
                            const uint32_t koff = (uint32_t)((ks & 3) * 32);
                            const uint32_t atom = (uint32_t)(ks >> 2);
                            const uint64_t ad = sw128_desc(blob_addr + aoff + atom * (arows * 128) +
                                                           (uint32_t)h * 16384u + koff);
                            const uint64_t bd = sw128_desc(b_addr + (uint32_t)(2 * ks * sbo_b),
                                                           1024u, (uint32_t)sbo_b);
                            mma_bf16(tmem + (uint32_t)(h * N), ad, bd, idesc_h, ks > 0 ? 1u : 0u);
                        }
                    }
                    mma_commit(bar_mma);
                    // the issuing thread alone waits; the rest sleep at the barrier
                    if (!mbar_wait(bar_mma, phase)) s_abort = 1;
                    tc_fence_before();
                }
                phase ^= 1u;
                __syncthreads();
                tc_fence_after();
                if (s_abort) goto mma_timeout;
                if (!out_layer) {
                    const float *bl = bias + (l - 1) * W;
                    // in chunks of at most 32 columns (whole points: L <= 32
                    // divides the chunk), which bounds the live registers
                    constexpr int kC = CW < 32 ? CW : 32;
                    for (int h = 0; h < MH; ++h) {
                        const int j = h * 128 + wq * 32 + lane;
                        if (j < W) {                 // uniform per warp: W % 64 == 0
                            const float b = bl[j];
#pragma unroll
                            for (int c0 = 0; c0 < CW; c0 += kC) {
                                float v[kC];
#pragma unroll
                                for (int g8 = 0; g8 < kC / 8; ++g8)
                                    tmem_ld8(tq + (uint32_t)(h * N + n0 + c0 + 8 * g8), v + 8 * g8);
                                tmem_wait_ld();
                                elu_tangents_l<kC>(L, v, b);
                                store_b_row<kC>(B, j, n0 + c0, sbo_b, v);
                            }
                        }
                    }
                    tc_fence_before();
                    fence_proxy_async();
                    __syncthreads();
                } else {
                    // output layer: rows 0-2 (the three outputs) sit in TMEM
                    // lanes 0-2, which only warp 0 of a warpgroup reads; it
                    // parks the raw sums of its columns in O3, then every
                    // thread finishes whole entries (one column, one output)
                    constexpr int kC = CW < 32 ? CW : 32;
                    if (wq == 0) {
#pragma unroll
                        for (int c0 = 0; c0 < CW; c0 += kC) {
                            float v[kC];
#pragma unroll
                            for (int g8 = 0; g8 < kC / 8; ++g8)
                                tmem_ld8(tq + (uint32_t)(n0 + c0 + 8 * g8), v + 8 * g8);
                            tmem_wait_ld();
                            if (lane < 3) {
                                // n0 + c0 is a multiple of 8: the pads of this
                                // chunk sit at fixed offsets from its start
                                float *o3 = O3 + (n0 + c0) * 3 + ((n0 + c0) >> 3) + lane;
#pragma unroll
                                for (int c = 0; c < kC; ++c) o3[c * 3 + (c >> 3)] = v[c];
                            }
                        }
                    }
                    tc_fence_before();
                    __syncthreads();
                    bool bad = false;
                    for (int e = tid; e < 3 * N; e += NWG * kWgThreads) {
                        const int col = e / 3, a = e - 3 * col;
                        const int s = col & (L - 1);
                        const int p = p0 + (col >> lgL);
                        const bool valid = p < n && s <= r;
                        float *o = O3 + col * 3 + (col >> 3) + a;
                        const float v = *o;
                        const float sc = F.scale[a];
                        float y = s == 0 ? fmaf(sc, v + bias[(D - 1) * W + a], F.shift[a]) : sc * v;
                        if (valid) bad |= !isfinite(y);
                        if (valid && s == 0) {
                            if (u) u[(size_t)a * ld + p] = y;
                            if (gn_on) {
                                const float4 t = tg[col >> lgL];
                                y -= a == 0 ? t.x : (a == 1 ? t.y : t.z);
                            }
                        }
                        if (valid && s > 0 && dudz) dudz[(size_t)(a * r + s - 1) * ld + p] = y;
                        *o = valid ? y : 0.f;
                    }
                    if (bad) set_status(status, NSF_ERR_NONFINITE);
                    __syncthreads();
                    if (gn_on) {
                        // this tile's share of the normal equations
                        gn_ff_tile_partials(O3, L, max(0, min(P, n - p0)), r);
                        __syncthreads();
                    }
                }
            }
        }

        if (gn_on) {
            // Gauss-Newton iteration `it`: all CTAs' partials summed behind a
            // grid barrier (cooperative launch), then every CTA solves
            __syncthreads();
            if (!gn_ff_finish_iteration(gn, r, it, rank, gsize, status)) goto teardown;
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
    if (tid == 0) {
        // a batched launch runs further problems whose layouts reuse this memory
        mbar_inval(bar_w);
        mbar_inval(bar_mma);
    }
    // ... and whose weight copy (async proxy) may land where this problem's
    // threads stored activations: order those stores first
    fence_proxy_async();
    __syncthreads();
}

template <int CW>
__global__ void __launch_bounds__(kThreads, 1)
k_jac_tc(const __grid_constant__ FieldsDev fd, const float *__restrict__ X, int n, int ld,
         const double *zj, float *u, float *dudz, const __grid_constant__ GnArgs gn, int gn_on,
         int *status) {
    pdl_wait();
    extern __shared__ uint8_t smem_dyn[];
    jac_body<CW>(fd, X, n, ld, zj, u, dudz, gn, gn_on, (int)blockIdx.x, (int)gridDim.x, true,
                 smem_dyn, status);
}

// One Gauss-Newton problem of a batch (inlined: out of line, the bodies spilled
// ~450 bytes per thread at 128 registers; inlined, 112).
template <int CW>
__device__ __forceinline__ void jac_batch_problem(const GnBatchProblem &pb, const GnBatchEntry &en,
                                               uint8_t *smem_dyn, int *status) {
    jac_body<CW, kBatchWG>(*pb.fd, pb.X, pb.n, pb.ld, nullptr, nullptr, nullptr, pb.gn, 1,
                           en.rank, en.size, false, smem_dyn, status);
}

// Batched Gauss-Newton: CTA c runs the problems of its entries
// cta_entry[c] .. cta_entry[c + 1] - 1 in order; an entry names a problem, the
// CTA's rank in that problem's CTA group and the group size.  A problem
// shared by a group of CTAs (group size > 1) is the first entry of each of
// them, so every member reaches the group's barriers inside that problem and
// no barrier waits on a CTA that is still busy with another problem.  The CTAs
// have four warpgroups of CW = 64 (or, when a scene's operands need it, 32)
// columns: tiles of 256 (128) point slots, whose products take as many
// tcgen05.mma instructions as the single-problem kernel's 64-slot tiles (a
// layer's instructions cost about the same per issue up to this size).  One
// CW for the whole launch keeps a single body per kernel.  (Eight warpgroups
// of half the columns measured slower: 5.85 against 4.71 ms on the 256-scene
// batch.)
template <int CW>
__global__ void __launch_bounds__(kBatchWG * kWgThreads, 1)
k_jac_batch(const GnBatchProblem *__restrict__ probs, const GnBatchEntry *__restrict__ entries,
            const int *__restrict__ cta_entry, int *status) {
    extern __shared__ uint8_t smem_dyn[];
    const int e0 = cta_entry[blockIdx.x], e1 = cta_entry[blockIdx.x + 1];
    for (int e = e0; e < e1; ++e) {
        const GnBatchEntry en = entries[e];
        jac_batch_problem<CW>(probs[en.problem], en, smem_dyn, status);
        __syncthreads();
    }
}

}  // namespace

// Shared memory of the Jacobian kernel with CW columns per warpgroup; 0 if
// it (or its tensor memory) does not fit.
size_t jac_tc_smem_bytes_cw(int r, int width, int depth, int CW, int NWG) {
    if (CW < jac_slots(r)) return 0;
    const JacLayout L = jac_layout(r, width, depth, CW, NWG);
    if (jac_halves(width) * NWG * CW > 512) return 0;           // tensor memory columns
    if ((size_t)L.total + sizeof(GnFF) + 64 > (size_t)kMaxSmem) return 0;
    return (size_t)L.total;
}

size_t jac_tc_smem_bytes(int r, int width, int depth) {
    const JacLayout L = jac_layout(r, width, depth, jac_cw(r));
    if (jac_halves(width) * jac_cols(r) > 512) return 0;        // tensor memory columns
    if ((size_t)L.total + sizeof(GnFF) + 64 > (size_t)kMaxSmem) return 0;
    return (size_t)L.total;
}

// Points per tile of the Jacobian kernel: every tile holds as many points as
// its columns allow; the latency of a layer does not depend on how many
// columns are live, so fuller tiles only mean fewer CTAs to combine in each
// Gauss-Newton iteration.
int jac_points_per_tile(const FieldsDev &fd, int n) {
    (void)n;
    return jac_points(fd.r);
}

int jac_grid_size_tc(const FieldsDev &fd, int n) {
    const int P = jac_points_per_tile(fd, n);
    const int tiles = (n + P - 1) / P;
    const int cap = sm_count() < kGnMaxCtas ? sm_count() : kGnMaxCtas;
    return tiles < cap ? tiles : cap;
}

cudaError_t launch_jacobian_tc(const FieldsDev &fd, const float *X, int n, int ld,
                               const double *z, float *u, float *dudz, const GnArgs *gn,
                               int *status, cudaStream_t s) {
    const FieldDev &F = fd.f[NSF_FIELD_G];
    const size_t sm = jac_tc_smem_bytes(fd.r, F.width, F.depth);
    if (sm == 0) return cudaErrorInvalidValue;
    GnArgs g{};
    if (gn) g = *gn;
    const int gn_on = gn ? 1 : 0;
    const int grid = jac_grid_size_tc(fd, n);
    // A Gauss-Newton run waits between iterations on a grid barrier, so all
    // CTAs must be co-resident: cooperative launch (one CTA per SM).
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    // cooperative for Gauss-Newton (grid barriers); programmatic stream
    // serialisation either way (the kernel calls pdl_wait first)
    cudaLaunchAttribute attr[2];
    int na = 0;
    if (gn_on) {
        attr[na].id = cudaLaunchAttributeCooperative;
        attr[na].val.cooperative = 1;
        ++na;
    }
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
    cfg.attrs = attr;
    cfg.numAttrs = na;
    if (jac_cw(fd.r) == 8) {
        static bool done = false;
        set_max_dynamic_smem(k_jac_tc<8>, done);
        return cudaLaunchKernelEx(&cfg, k_jac_tc<8>, fd, X, n, ld, z, u, dudz, g, gn_on, status);
    }
    if (jac_cw(fd.r) == 16) {
        static bool done = false;
        set_max_dynamic_smem(k_jac_tc<16>, done);
        return cudaLaunchKernelEx(&cfg, k_jac_tc<16>, fd, X, n, ld, z, u, dudz, g, gn_on, status);
    }
    static bool done = false;
    set_max_dynamic_smem(k_jac_tc<32>, done);
    return cudaLaunchKernelEx(&cfg, k_jac_tc<32>, fd, X, n, ld, z, u, dudz, g, gn_on, status);
}

int jac_points_per_cta_tile(int r) { return jac_points(r); }

// Columns per warpgroup of a batched problem (four warpgroups per CTA): 64 if
// the operands fit (a 256-slot tile), else 32; at least the problem's slot
// count; 0 if neither fits.
int jac_batch_cw(int r, int width, int depth) {
    for (int cw = 64; cw >= 32; cw >>= 1)
        if (cw >= jac_slots(r) && jac_tc_smem_bytes_cw(r, width, depth, cw, kBatchWG)) return cw;
    return 0;
}
int jac_batch_points(int r, int cw) { return kBatchWG * cw / jac_slots(r); }

int jac_batch_wg() { return kBatchWG; }

cudaError_t launch_jac_batch(const GnBatchProblem *probs, const GnBatchEntry *entries,
                             const int *cta_entry, int nctas, size_t smem, int cw, int *status,
                             cudaStream_t s) {
    if (nctas <= 0) return cudaSuccess;
    if (cw != 32 && cw != 64) return cudaErrorInvalidValue;
    static bool done32 = false, done64 = false;
    if (cw == 32) set_max_dynamic_smem(k_jac_batch<32>, done32);
    else set_max_dynamic_smem(k_jac_batch<64>, done64);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nctas);
    cfg.blockDim = dim3(kBatchWG * kWgThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cw == 32) return cudaLaunchKernelEx(&cfg, k_jac_batch<32>, probs, entries, cta_entry, status);
    return cudaLaunchKernelEx(&cfg, k_jac_batch<64>, probs, entries, cta_entry, status);
}

}  // namespace nsf
