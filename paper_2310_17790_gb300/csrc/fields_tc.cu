// BF16 field networks on the tcgen05 tensor cores (precision NSF_PREC_BF16):
// value evaluation of g, h and l (paper §5.1, inference on the integration
// particles; App. E, fields are ELU MLPs on [X; z]).  The Jacobian and the
// Gauss-Newton iterations run in jacobian_tc.cu.
//
// A CTA holds one field's weights resident in shared memory (one bulk copy on
// an mbarrier with a transaction count) and runs up to two tile groups of 256
// threads (two warpgroups) side by side.  Each group owns a 128-point tile at
// a time, with its FP32 accumulator and its bf16 activation operand (the A
// operand of tcgen05.mma) both in tensor memory; point i of the tile is tile
// row i and TMEM lane i, which only the warps with (warp index % 4) == i / 32
// can access, and warpgroup h of the group owns the column half
// [h W / 2, (h + 1) W / 2).
// Per tile:
//   layer 0 (K = 3 + r)  on the CUDA cores in FP32, written as bf16 into the
//                        group's activation operand (tcgen05.st);
//   hidden layers        tcgen05.mma M = 128, N = width, K = width (16 per
//                        instruction, A from tensor memory) issued by the
//                        group's first thread; the epilogue reads the
//                        accumulator with tcgen05.ld, adds the FP32 bias,
//                        applies ELU (packed f32x2 arithmetic, one
//                        special-function exp per element), rounds to bf16 and
//                        rewrites the activation operand;
//   output layer         the same MMA with N = 16 (out_dim padded with zero
//                        rows), bias added when the outputs are read.
// The groups synchronise on their own named barriers, so while one group runs
// an epilogue on the CUDA cores the tensor core works on the other group's
// layer.  Every wait on an mbarrier is bounded by time: on expiry the kernel
// records NSF_ERR_ITER_CAP, waits (bounded) for its outstanding operations,
// frees its tensor memory and returns.
//
// Weight operands (B here, A in the Jacobian kernel) are K-major with the
// 128-byte swizzle (tc_common.cuh).
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

constexpr int kMaxGroups = 2;
// Warpgroups per tile group: each owns W / kWgPerGroup columns of every layer.
#ifndef NSF_VALUE_WG_PER_GROUP
#define NSF_VALUE_WG_PER_GROUP 2
#endif
constexpr int kWgPerGroup = NSF_VALUE_WG_PER_GROUP;
constexpr int kGroupThreads = kWgPerGroup * kWgThreads;

// Tensor-memory columns of one group: the FP32 accumulator (W columns) and,
// after it at column W, the bf16 activation operand (W / 2 columns).
__host__ __device__ inline int tmem_region(int W) { return W <= 64 ? 128 : (W <= 128 ? 256 : 512); }

// Shared-memory carve of one CTA (byte offsets from a 1024-aligned base).
struct TcLayout {
    int blob, w0v, bias, bars, tmem, total;
};

__host__ __device__ inline TcLayout tc_layout(int W, int D) {
    TcLayout L;
    int o = 0;
    L.blob = o; o = align_to(o + (D - 1) * W * W * 2 + kMaxOut * W * 2, 1024);
    L.w0v = o;  o = align_to(o + W * 16, 16);                 // input layer, column pairs
    L.bias = o; o = align_to(o + D * W * 4, 16);              // hidden biases, then output bias
    L.bars = o; o = align_to(o + (2 + kMaxGroups) * 8, 16);   // weights, go, MMA per group
    L.tmem = o; o = align_to(o + 16, 16);
    L.total = o + 1024;   // room to align the dynamic base to 1024 bytes
    return L;
}

struct TcJobs {
    int njobs;
    FieldJob job[4];
};

// C FP32 values (C = 16 or 32) -> C / 2 packed bf16 pairs (round to nearest
// even), stored to C / 2 consecutive tensor-memory columns.
template <int C>
__device__ __forceinline__ void store_act(uint32_t taddr, const float *v) {
    uint32_t q[C / 2];
#pragma unroll
    for (int i = 0; i < C / 2; ++i) q[i] = pack_bf16x2(v[2 * i], v[2 * i + 1]);
    if constexpr (C == 32) tmem_st16(taddr, q);
    else tmem_st8(taddr, q);
}

// C accumulator columns of this warp's lanes (C = 16 or 32).
template <int C>
__device__ __forceinline__ void load_acc(uint32_t taddr, float *v) {
    tmem_ld16(taddr, v);
    if constexpr (C == 32) tmem_ld16(taddr + 16, v + 16);
}

// ELU(v + bias) in place over C values.
template <int C>
__device__ __forceinline__ void bias_elu(float *v, const float *bl) {
#pragma unroll
    for (int i = 0; i < C; i += 4) {
        const float4 b = *reinterpret_cast<const float4 *>(bl + i);
        const float2 h0 = elu2(make_float2(v[i], v[i + 1]), make_float2(b.x, b.y));
        const float2 h1 = elu2(make_float2(v[i + 2], v[i + 3]), make_float2(b.z, b.w));
        v[i] = h0.x;
        v[i + 1] = h0.y;
        v[i + 2] = h1.x;
        v[i + 3] = h1.y;
    }
}

// One work item of the value kernel: field F at latent code z on the
// 128-point tiles [tile0, tile1) of the point set X ([3][ld], n points),
// outputs to out ([out_dim][ld]).
struct ItemView {
    const FieldDev *F;
    int r;
    const float *X;
    int n, ld;
    const double *z;
    float *out;
    int tile0, tile1;
};

// Work items of the single-problem launch: CTA (x, y) runs job y on its
// contiguous share of the tiles.
struct SingleSrc {
    const FieldsDev *fd;
    const float *X;
    int n, ld;
    const TcJobs *jobs;
    __device__ ItemView item(int) const {
        const FieldJob &job = jobs->job[blockIdx.y];
        const int tiles = (n + kM - 1) / kM;
        const int per = (tiles + (int)gridDim.x - 1) / (int)gridDim.x;
        const int t0 = (int)blockIdx.x * per;
        return ItemView{&fd->f[job.field], fd->r, X, n, ld, job.z, job.out, t0,
                        t0 + per < tiles ? t0 + per : tiles};
    }
};

// Work items of a batched launch: CTA c runs items cta_item[c] .. cta_item[c +
// 1] - 1; a g item writes the step's current displacement buffer (zsel 0, z_n)
// or the other one (zsel 1, z_{n-1}).
struct BatchSrc {
    const BatchSceneDev *scenes;
    const FieldBatchItem *items;
    int e0, parity;
    __device__ ItemView item(int k) const {
        const FieldBatchItem it = items[e0 + k];
        const BatchSceneDev &sc = scenes[it.scene];
        float *out = it.field == NSF_FIELD_G ? sc.u[it.zsel ? parity ^ 1 : parity]
                     : it.field == NSF_FIELD_H ? sc.tau6 : sc.C9;
        return ItemView{&sc.fd->f[it.field], sc.fd->r, sc.X, sc.n_N, sc.n_N,
                        it.zsel ? sc.z_prev : sc.z, out, it.tile0, it.tile1};
    }
};

template <int W, class Src>
__device__ __forceinline__ void fields_body(const Src &src, int nitems, int ng, int maxD,
                                            uint8_t *smem_dyn, int *status) {
    __shared__ int s_ok[kMaxGroups];
    uint8_t *base = aligned_smem(smem_dyn);

    const int tid = threadIdx.x;
    const int grp = tid / kGroupThreads;     // tile group
    const int gt = tid % kGroupThreads;      // thread within the group
    const int row = gt & (kM - 1);           // tile row == TMEM lane
    const int wq = row >> 5;                 // lane quarter of this warp
    constexpr int cw = W / kWgPerGroup;      // columns per warpgroup (multiple of 16)
    constexpr int kC = cw < 32 ? cw : 32;    // columns per chunk of the epilogue
    const int cbeg = (gt >> 7) * cw;
    const int bar_id = 1 + grp;              // the group's named barrier
    const TcLayout L = tc_layout(W, maxD);
    uint8_t *blob = base + L.blob;
    // input layer by column pairs (j, j + 1): {w_x j, w_x j+1, w_y j, w_y j+1},
    // {w_z j, w_z j+1, c0 j, c0 j+1}, so a pair's values load as register pairs
    float4 *W0v = reinterpret_cast<float4 *>(base + L.w0v);
    float *bias = reinterpret_cast<float *>(base + L.bias);  // [D][W]
    uint64_t *bar_w = reinterpret_cast<uint64_t *>(base + L.bars);
    uint64_t *bar_go = bar_w + 1;            // group 0 has issued its first MMA
    uint64_t *bar_mma = bar_w + 2 + grp;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(base + L.tmem);
    const uint32_t ncols = (uint32_t)(ng * tmem_region(W));

    if (tid == 0) {
        mbar_init(bar_w, 1);
        mbar_init(bar_go, 1);
        for (int g = 0; g < ng; ++g) mbar_init(bar_w + 2 + g, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) tmem_alloc(tmem_holder, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    const uint32_t acc = tmem + (uint32_t)(grp * tmem_region(W));   // FP32 accumulator
    const uint32_t act = acc + (uint32_t)W;                          // bf16 activations
    const uint32_t b_addr = smem_u32(blob);
    const uint32_t idesc_h = idesc_bf16(kM, W);
    const uint32_t idesc_o = idesc_bf16(kM, kMaxOut);
    const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
    const uint32_t acc_l = acc + lane_off;                           // this warp's lanes
    const uint32_t act_l = act + lane_off + (uint32_t)(cbeg / 2);    // its activation columns
    uint32_t phase = 0, phase_w = 0;
    bool go_sent = false, go_waited = false;
    bool copy_pending = false;
    const FieldDev *curF = nullptr;

    for (int it = 0; it < nitems; ++it) {
        const ItemView I = src.item(it);
        if (I.tile0 >= I.tile1) continue;
        const FieldDev &F = *I.F;
        const int D = F.depth, r = I.r;
        __syncthreads();                      // the previous item is done with shared memory
        const bool reload = I.F != curF;
        // weights: one bulk copy, landing while the CTA prepares the input layer
        if (reload && tid == 0) bulk_load(blob, F.tc_blob, (uint32_t)F.tc_blob_bytes, bar_w);
        copy_pending = reload;
        const int in0 = 3 + r;
        for (int j = tid; j < W; j += blockDim.x) {
            // z-part of the input layer folded into its bias: c0 = b0 + W0[:, 3:] z
            const float *w = F.W0 + (size_t)j * in0;
            float c0 = F.b[0][j];
            for (int k = 0; k < r; ++k) c0 = fmaf(w[3 + k], (float)__ldcg(&I.z[k]), c0);
            float *pr = reinterpret_cast<float *>(W0v + 2 * (j >> 1)) + (j & 1);
            pr[0] = w[0];
            pr[2] = w[1];
            pr[4] = w[2];
            pr[6] = c0;
        }
        for (int l = 1; l <= D; ++l) {
            const int o = l == D ? F.out_dim : W;
            for (int j = tid; j < o; j += blockDim.x) bias[(l - 1) * W + j] = F.b[l][j];
        }
        __syncthreads();
        if (reload) {
            if (!__syncthreads_and(mbar_wait(bar_w, phase_w))) {
                if (tid == 0) set_status(status, NSF_ERR_ITER_CAP);
                goto teardown;
            }
            phase_w ^= 1u;
            copy_pending = false;
            curF = I.F;
        }

        for (int tile = I.tile0 + grp; tile < I.tile1; tile += ng) {
            if (grp == 1 && !go_waited) {
                // Group 1 starts once group 0 has handed its first layer to the
                // tensor core, so that from then on each group's epilogue runs
                // while the tensor core works on the other group's product
                // (started together, both would run their epilogues at the
                // same time and leave the tensor core idle meanwhile).
                if (gt == 0) s_ok[1] = mbar_wait(bar_go, 0) ? 1 : 0;
                named_sync(bar_id, kGroupThreads);
                go_waited = true;
                if (!s_ok[1]) {
                    if (gt == 0) set_status(status, NSF_ERR_ITER_CAP);
                    goto teardown;
                }
            }
            const int p = tile * kM + row;
            const bool valid = p < I.n;
            // ---- layer 0 on the CUDA cores, into the activation operand
            float x0 = 0.f, x1 = 0.f, x2 = 0.f;
            if (valid) {
                x0 = I.X[p];
                x1 = I.X[I.ld + p];
                x2 = I.X[2 * I.ld + p];
            }
            const float2 xx0 = make_float2(x0, x0), xx1 = make_float2(x1, x1),
                         xx2 = make_float2(x2, x2);
#pragma unroll
            for (int c0 = 0; c0 < cw; c0 += kC) {
                const int cc = cbeg + c0;
                float v[kC];
#pragma unroll
                for (int i = 0; i < kC; i += 2) {
                    const float4 wa = W0v[cc + i], wb = W0v[cc + i + 1];
                    const float2 pre = __ffma2_rn(
                        make_float2(wa.x, wa.y), xx0,
                        __ffma2_rn(make_float2(wa.z, wa.w), xx1,
                                   __ffma2_rn(make_float2(wb.x, wb.y), xx2,
                                              make_float2(wb.z, wb.w))));
                    const float2 h = elu2(pre, make_float2(0.f, 0.f));
                    v[i] = h.x;
                    v[i + 1] = h.y;
                }
                store_act<kC>(act_l + (uint32_t)(c0 / 2), v);
            }

            // ---- hidden layers, then the output layer (l == D)
            for (int l = 1; l <= D; ++l) {
                const bool out_layer = l == D;
                tmem_wait_st();               // this thread's activation stores landed
                tc_fence_before();            // and its accumulator reads are done
                named_sync(bar_id, kGroupThreads);
                if (gt == 0) {
                    tc_fence_after();
                    const uint32_t boff = (uint32_t)((l - 1) * W * W * 2);
                    const int nrows = out_layer ? kMaxOut : W;
                    const uint32_t idesc = out_layer ? idesc_o : idesc_h;
#pragma unroll
                    for (int ks = 0; ks < W / 16; ++ks) {
                        const uint32_t koff = (uint32_t)((ks & 3) * 32);
                        const uint32_t atom = (uint32_t)(ks >> 2);
                        mma_bf16_ts(acc, act + (uint32_t)(8 * ks),
                                    sw128_desc(b_addr + boff + atom * (nrows * 128) + koff),
                                    idesc, ks > 0 ? 1u : 0u);
                    }
                    mma_commit(bar_mma);
                    if (grp == 0 && !go_sent) {
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                         smem_u32(bar_go))
                                     : "memory");
                        go_sent = true;
                    }
                    // the issuing thread alone waits; the rest of the group
                    // sleeps at the barrier while the other group computes
                    s_ok[grp] = mbar_wait(bar_mma, phase) ? 1 : 0;
                    tc_fence_before();
                }
                phase ^= 1u;
                named_sync(bar_id, kGroupThreads);
                tc_fence_after();
                if (!s_ok[grp]) goto mma_timeout;
                if (!out_layer) {
                    // chunk k + 1's accumulator load is in flight while chunk
                    // k is computed and stored
                    const float *bl = bias + (l - 1) * W + cbeg;
                    float v[kC], w[kC];
                    load_acc<kC>(acc_l + (uint32_t)cbeg, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int c0 = 0; c0 < cw; c0 += 2 * kC) {
                        const bool more = c0 + kC < cw;
                        if (more) load_acc<kC>(acc_l + (uint32_t)(cbeg + c0 + kC), w);
                        bias_elu<kC>(v, bl + c0);
                        store_act<kC>(act_l + (uint32_t)(c0 / 2), v);
                        if (!more) break;
                        tmem_wait_ld();
                        if (c0 + 2 * kC < cw) load_acc<kC>(acc_l + (uint32_t)(cbeg + c0 + 2 * kC), v);
                        bias_elu<kC>(w, bl + c0 + kC);
                        store_act<kC>(act_l + (uint32_t)((c0 + kC) / 2), w);
                        if (c0 + 2 * kC < cw) tmem_wait_ld();
                    }
                } else if (gt < kM) {
                    // outputs: the first warpgroup reads the 16 output columns
                    float v[16];
                    tmem_ld16(acc_l, v);
                    tmem_wait_ld();
                    const float *bo = bias + (D - 1) * W;
                    bool bad = false;
                    if (valid) {
#pragma unroll
                        for (int o = 0; o < 9; ++o) {
                            if (o < F.out_dim) {
                                const float y = fmaf(F.scale[o], v[o] + bo[o], F.shift[o]);
                                bad |= !isfinite(y);
                                I.out[(size_t)o * I.ld + p] = y;
                            }
                        }
                    }
                    if (bad) set_status(status, NSF_ERR_NONFINITE);
                }
            }
        }
    }
    goto teardown;

mma_timeout:
    if (gt == 0) {
        set_status(status, NSF_ERR_ITER_CAP);
        // bounded: let the outstanding MMA finish before the memory is released
        mbar_wait(bar_mma, phase ^ 1u);
    }

teardown:
    // a CTA must not leave while a weight copy may still be landing
    if (copy_pending && tid == 0) mbar_wait(bar_w, phase_w);
    tmem_wait_st();
    tc_fence_before();
    __syncthreads();
    if (tid < 32) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

template <int W>
__global__ void __launch_bounds__(kMaxGroups * kGroupThreads, 1)
k_fields_tc(const __grid_constant__ FieldsDev fd, const float *__restrict__ X, int n, int ld,
            const __grid_constant__ TcJobs jobs, int ng, int maxD, int *status) {
    pdl_wait();
    extern __shared__ uint8_t smem_dyn[];
    const SingleSrc src{&fd, X, n, ld, &jobs};
    fields_body<W>(src, 1, ng, maxD, smem_dyn, status);
}

template <int W>
__global__ void __launch_bounds__(kMaxGroups * kGroupThreads, 1)
k_fields_batch(const BatchSceneDev *__restrict__ scenes, const FieldBatchItem *__restrict__ items,
               const int *__restrict__ cta_item, int parity, int ng, int maxD, int *status) {
    extern __shared__ uint8_t smem_dyn[];
    const int e0 = cta_item[blockIdx.x], e1 = cta_item[blockIdx.x + 1];
    const BatchSrc src{scenes, items, e0, parity};
    fields_body<W>(src, e1 - e0, ng, maxD, smem_dyn, status);
}

// Tile groups a CTA runs for this field size (two where both groups' tensor
// memory fits), 0 if the weights do not fit in shared memory.
int value_groups(int width, int depth) {
    if ((size_t)tc_layout(width, depth).total + 64 > (size_t)kMaxSmem) return 0;
    return 2 * tmem_region(width) <= 512 ? 2 : 1;
}

size_t value_smem_bytes(int width, int depth) {
    return value_groups(width, depth) ? (size_t)tc_layout(width, depth).total : 0;
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

namespace {

template <int W>
cudaError_t launch_fields_tc_w(const FieldsDev &fd, const float *X, int n, int ld,
                               const TcJobs &tj, int *status, cudaStream_t s) {
    int ng = kMaxGroups;
    size_t sm = 0;
    for (int i = 0; i < tj.njobs; ++i) {
        const int g = value_groups(W, fd.f[tj.job[i].field].depth);
        if (g == 0) return cudaErrorInvalidValue;
        ng = g < ng ? g : ng;
    }
    for (int i = 0; i < tj.njobs; ++i) {
        const size_t b = (size_t)tc_layout(W, fd.f[tj.job[i].field].depth).total;
        sm = b > sm ? b : sm;
    }
    static bool attr_done = false;
    set_max_dynamic_smem(k_fields_tc<W>, attr_done);
    const int tiles = (n + kM - 1) / kM;
    int per_job = sm_count() / tj.njobs;
    if (per_job < 1) per_job = 1;
    if (per_job > tiles) per_job = tiles;
    dim3 grid(per_job, tj.njobs);
    int maxD = 1;
    for (int i = 0; i < tj.njobs; ++i) {
        const int d = fd.f[tj.job[i].field].depth;
        maxD = d > maxD ? d : maxD;
    }
    // programmatic stream serialisation: the kernel waits for its predecessor
    // (pdl_wait) before any global access
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(ng * kGroupThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_fields_tc<W>, fd, X, n, ld, tj, ng, maxD, status);
}

}  // namespace

size_t fields_batch_smem(int W, int maxD) { return (size_t)tc_layout(W, maxD).total; }
int fields_batch_groups(int W) { return 2 * tmem_region(W) <= 512 ? 2 : 1; }

namespace {
template <int W>
cudaError_t launch_batch_w(const BatchSceneDev *scenes, const FieldBatchItem *items,
                           const int *cta_item, int nctas, int parity, int maxD, int *status,
                           cudaStream_t s) {
    static bool attr_done = false;
    set_max_dynamic_smem(k_fields_batch<W>, attr_done);
    const int ng = fields_batch_groups(W);
    k_fields_batch<W><<<nctas, ng * kGroupThreads, tc_layout(W, maxD).total, s>>>(
        scenes, items, cta_item, parity, ng, maxD, status);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_fields_batch(int W, const BatchSceneDev *scenes, const FieldBatchItem *items,
                                const int *cta_item, int nctas, int parity, int maxD,
                                int *status, cudaStream_t s) {
    if (nctas <= 0) return cudaSuccess;
    switch (W) {
        case 64: return launch_batch_w<64>(scenes, items, cta_item, nctas, parity, maxD, status, s);
        case 128: return launch_batch_w<128>(scenes, items, cta_item, nctas, parity, maxD, status, s);
        case 192: return launch_batch_w<192>(scenes, items, cta_item, nctas, parity, maxD, status, s);
        case 256: return launch_batch_w<256>(scenes, items, cta_item, nctas, parity, maxD, status, s);
        default: return cudaErrorInvalidValue;
    }
}

// One launch per distinct field width among the jobs (the kernel is
// specialised on the width so that its column loops unroll completely).
cudaError_t launch_fields_tc(const FieldsDev &fd, const float *X, int n, int ld, int njobs,
                             const FieldJob *jobs, int *status, cudaStream_t s) {
    static const int widths[] = {64, 128, 192, 256};
    for (int w : widths) {
        TcJobs tj;
        tj.njobs = 0;
        for (int i = 0; i < njobs; ++i)
            if (fd.f[jobs[i].field].width == w) tj.job[tj.njobs++] = jobs[i];
        if (tj.njobs == 0) continue;
        cudaError_t e = cudaSuccess;
        switch (w) {
            case 64: e = launch_fields_tc_w<64>(fd, X, n, ld, tj, status, s); break;
            case 128: e = launch_fields_tc_w<128>(fd, X, n, ld, tj, status, s); break;
            case 192: e = launch_fields_tc_w<192>(fd, X, n, ld, tj, status, s); break;
            default: e = launch_fields_tc_w<256>(fd, X, n, ld, tj, status, s); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace nsf
