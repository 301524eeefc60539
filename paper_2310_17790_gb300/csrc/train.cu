// Fitting a field network to full-order snapshots (paper App. D): loss,
// hand-written backward and Adam, plus the device-side re-pack of updated
// weights into an nsf_fields.
//
// Activations are column-major per point (column p = point p).  Forward, per
// linear layer l:  A_l = W_l H_{l-1} + b_l,  H_l = ELU(A_l), with H_{-1} =
// [X; z].  Loss: the mean squared normalised error
// L = sum ((y - y*) / scale)^2 / (n out_dim).  Backward on the forward's
// activations:
//   delta_out = dL/draw = 2 (y - y*) / (scale n out_dim)
//   dW_l = delta_l H_{l-1}^T,  db_l = delta_l x ones (row sums),
//   delta_{l-1} = (W_l^T delta_l) * ELU'(A_{l-1}),
//   dz_t += (W_0^T delta_0)[3:, p] over the points p of snapshot t.
// Every product is the library's own (gemm.cu), its elementwise step fused
// into the product's epilogue (bias + ELU, or * ELU').  BF16 fields: the
// width x width products on the tcgen05 tensor cores -- forward with bf16
// operands (the activations entering a product rounded to bf16), backward
// with the FP32 cotangent split into two bf16 parts against the exact bf16
// weights or activations (~16 significant bits) -- and the thin input and
// output layers in FP32 on the CUDA cores; FP32 fields: every product in FP32
// on the CUDA cores.  Weight gradients split the sum over points into K
// slices (one slab each), summed in a fixed order.
#include <vector>

#include "tc_common.cuh"

namespace nsf {

using tc::sw128_kmajor_offset;

namespace {

constexpr int kT = 256;

inline int blocks(long long n) { return (int)((n + kT - 1) / kT); }

// [X_p; z_code(p)] as column p of a (3 + r) x n matrix.
__global__ void k_inputs(const float *__restrict__ X, const int *__restrict__ code,
                         const float *__restrict__ z_table, int n, int r, float *inp,
                         int *status) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int c = code[p];
    float *col = inp + (size_t)p * (3 + r);
    col[0] = X[p];
    col[1] = X[n + p];
    col[2] = X[2 * n + p];
    if (c < 0) {
        set_status(status, NSF_ERR_INVALID_ARG);
        for (int k = 0; k < r; ++k) col[3 + k] = 0.f;
        return;
    }
    for (int k = 0; k < r; ++k) col[3 + k] = z_table[(size_t)c * r + k];
}

// Outputs, loss and dL/draw.  raw: od x n (column-major), target [od][n].
// Also this CTA's sums of dL/draw over its points (the output bias gradient's
// partials) into dbias_part[blockIdx.x][od].
__global__ void k_loss(const float *__restrict__ raw, const float *__restrict__ bout,
                       const float *__restrict__ X, const float *__restrict__ target, int n,
                       int od, FieldDev F, int residual, float *delta, float *loss_part,
                       float *dbias_part) {
    __shared__ float part[kT];
    __shared__ float dsum[kT / 32][9];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc = 0.f;
    float d[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) d[a] = 0.f;
    if (p < n) {
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            if (a >= od) break;
            float y = fmaf(F.scale[a], raw[(size_t)p * od + a] + bout[a], F.shift[a]);
            if (residual) y += X[(size_t)a * n + p];
            const float e = (y - target[(size_t)a * n + p]) / F.scale[a];
            acc = fmaf(e, e, acc);
            d[a] = 2.f * e / ((float)n * (float)od);
            delta[(size_t)p * od + a] = d[a];
        }
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        float v = d[a];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) dsum[warp][a] = v;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < od) {
        float v = 0.f;
        for (int w = 0; w < kT / 32; ++w) v += dsum[w][threadIdx.x];
        dbias_part[(size_t)blockIdx.x * od + threadIdx.x] = v;
    }
    for (int s = kT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = part[0] / ((float)n * (float)od);
}

__global__ void k_fill(float *a, float v, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) a[i] = v;
}

constexpr int kDzShared = 4096;   // floats of a CTA's code table

// dz_code(p) summed over the points p with that code, in a fixed order, for
// the codes [c0, c0 + nc) (nc r <= kDzShared): CTA b takes the points
// [b per, (b + 1) per) in rounds of 256; in a round the lanes of a warp with
// the same code add their values in lane order (shuffles) and the warps then
// add their sums to the CTA's table in warp order.  The CTA writes its table
// to part[b][nc r]; the tables are then added in CTA order (reduce_slabs).
__global__ void __launch_bounds__(kT)
k_scatter_dz(const float *__restrict__ dinp, const int *__restrict__ code, int n, int r, int c0,
             int nc, int per, float *part) {
    __shared__ float tab[kDzShared];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p_beg = blockIdx.x * per, p_end = min(n, p_beg + per);
    for (int i = threadIdx.x; i < nc * r; i += kT) tab[i] = 0.f;
    __syncthreads();
    for (int base = p_beg; base < p_end; base += kT) {
        const int p = base + threadIdx.x;
        int c = -1;
        if (p < p_end) {
            c = code[p] - c0;
            if (c < 0 || c >= nc) c = -1;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        const bool leader = c >= 0 && lane == __ffs(peers) - 1;
        float sum[NSF_MAX_R];
#pragma unroll
        for (int k = 0; k < NSF_MAX_R; ++k) {
            sum[k] = 0.f;
            if (k < r) {
                const float v = c >= 0 ? dinp[(size_t)p * (3 + r) + 3 + k] : 0.f;
                for (unsigned m = peers; m; m &= m - 1u)
                    sum[k] += __shfl_sync(peers, v, __ffs(m) - 1);
            }
        }
        for (int w = 0; w < kT / 32; ++w) {
            if (warp == w && leader)
#pragma unroll
                for (int k = 0; k < NSF_MAX_R; ++k)
                    if (k < r) tab[c * r + k] += sum[k];
            __syncthreads();
        }
    }
    float *dst = part + (size_t)blockIdx.x * nc * r;
    for (int i = threadIdx.x; i < nc * r; i += kT) dst[i] = tab[i];
}

// bf16 copies of a hidden layer's weights from its transposed FP32 copy
// Wt [in][out]: Wb [out][in] and WTb [in][out] (the values are bf16 already
// for a BF16 field).
// The bf16 copies of the hidden layers' weights, both orientations, for
// layers 1 .. D - 1 in one launch (blockIdx.y = l - 1).
struct WeightCopies {
    const float *Wt[kMaxDepth];
    __nv_bfloat16 *Wb[kMaxDepth], *WTb[kMaxDepth];
};
__global__ void k_weights_bf16(WeightCopies wc, int W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, l = blockIdx.y + 1;
    if (i >= W * W) return;
    const int c = i / W, o = i % W;
    const __nv_bfloat16 v = __float2bfloat16_rn(wc.Wt[l][i]);
    wc.WTb[l][i] = v;
    wc.Wb[l][(size_t)o * W + c] = v;
}

// Adam (Kingma and Ba 2014), bias-corrected, in place.
__global__ void k_adam(float *p, const float *__restrict__ g, float *m, float *v, long long count,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Re-pack of one field from the flat layout (W_l row-major then b_l per
// layer).  One thread per flat element writes its FP32 copy (matrices rounded
// to bf16 for a BF16 field; hidden layers transposed) and, for BF16, its place
// in the swizzled tensor-core operand.
__global__ void k_repack(const float *__restrict__ flat, long long total, int r, int D,
                         int bf16, const __grid_constant__ FieldDev F) {
    const int W = F.width, od = F.out_dim;
    float *W0 = const_cast<float *>(F.W0);
    float *Wout = const_cast<float *>(F.Wout);
    __nv_bfloat16 *blob = const_cast<__nv_bfloat16 *>(F.tc_blob);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    long long off = 0;
    for (int l = 0; l <= D; ++l) {
        const int in = l == 0 ? 3 + r : W, out = l == D ? od : W;
        const long long nw = (long long)in * out;
        if (i < off + nw) {
            const int k = (int)(i - off);
            const int o = k / in, c = k - o * in;
            float v = flat[i];
            if (bf16) v = __bfloat162float(__float2bfloat16_rn(v));
            if (l == 0) {
                W0[k] = v;
            } else if (l == D) {
                Wout[k] = v;
                if (bf16) {
                    const size_t base = (size_t)(D - 1) * W * W;
                    blob[base + sw128_kmajor_offset(o, c, 16) / 2] = __float2bfloat16_rn(v);
                }
            } else {
                const_cast<float *>(F.Wt[l])[(size_t)c * W + o] = v;
                if (bf16) {
                    const size_t base = (size_t)(l - 1) * W * W;
                    blob[base + sw128_kmajor_offset(o, c, W) / 2] = __float2bfloat16_rn(v);
                }
            }
            return;
        }
        off += nw;
        if (i < off + out) {
            const_cast<float *>(F.b[l])[i - off] = flat[i];
            return;
        }
        off += out;
    }
}

// Most K slices of a weight-gradient product (the slab holds this many).
constexpr int kMaxSlices = 48;
// K slices of a thin product (one 256-thread CTA per slice): 256 points a
// slice, at most kMaxThinSlices.
constexpr int kMaxThinSlices = 256;
int thin_slices(int n) {
    const int k = n / 256;
    return k < 1 ? 1 : (k > kMaxThinSlices ? kMaxThinSlices : k);
}
// K slices of a weight-gradient product over n points whose output has
// `tiles` tiles: about one work unit per SM for the persistent tensor-core
// kernel, two CTAs per SM for the CUDA-core one; at least 256 points a slice.
int weight_slices(int n, int tiles, bool tc_kernel) {
    int k = tc_kernel ? tc::sm_count() / tiles : (2 * tc::sm_count() + tiles - 1) / tiles;
    k = k > kMaxSlices ? kMaxSlices : k;
    const int by_n = (n + 255) / 256;
    k = k > by_n ? by_n : k;
    return k < 1 ? 1 : k;
}

MatView view(const void *p, long long s_row, long long s_k, int bf16) {
    MatView v;
    v.ptr = p;
    v.s_row = s_row;
    v.s_k = s_k;
    v.bf16 = bf16;
    v.lo = nullptr;
    return v;
}

GemmEpilogue epi(int mode, float *out = nullptr, long long ld = 0) {
    GemmEpilogue e{};
    e.mode = mode;
    e.out = out;
    e.ld = ld;
    return e;
}

}  // namespace

// ------------------------------------------------------------ layout ---
TrainLayout train_layout(int r, int W, int D, int od, int n) {
    TrainLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t a = o;
        o = (o + bytes + 255) & ~(size_t)255;
        return a;
    };
    const size_t nn = (size_t)n;
    L.inp = take((size_t)(3 + r) * nn * 4);
    L.dinp = take((size_t)(3 + r) * nn * 4);
    for (int l = 0; l < D; ++l) {
        L.A[l] = take((size_t)W * nn * 4);
        L.H[l] = take((size_t)W * nn * 4);
        L.H16[l] = take((size_t)W * nn * 2);
    }
    L.raw = take((size_t)od * nn * 4);
    L.dout = take((size_t)od * nn * 4);
    L.d1 = take((size_t)W * nn * 4);
    L.d2 = take((size_t)W * nn * 4);
    for (int i = 0; i < 2; ++i) {       // the cotangents as bf16 hi / lo pairs
        L.dh[i] = take((size_t)W * nn * 2);
        L.dl[i] = take((size_t)W * nn * 2);
    }
    for (int l = 1; l < D; ++l) {       // bf16 W_l [out][in] and W_l^T [in][out]
        L.Wb[l] = take((size_t)W * W * 2);
        L.WTb[l] = take((size_t)W * W * 2);
    }
    L.ones = take(16);
    // slabs of the split sums: tensor-core weight gradients (W x W per
    // slice), thin products (at most max(3 + r, od) x W per slice), the loss
    // kernel's per-CTA output-bias sums
    const size_t thin_a = (size_t)(3 + r > od ? 3 + r : od);
    size_t slab = (size_t)kMaxSlices * W * (W + 1);     // weight and bias gradient slabs
    slab = slab > (size_t)kMaxThinSlices * thin_a * W ? slab : (size_t)kMaxThinSlices * thin_a * W;
    const size_t loss_parts = (nn + kT - 1) / kT * (size_t)(od + 1);   // + the loss partials
    // per-CTA partial sums: bias columns and the output layer's outer products
    // (thin_k, one part per 128 points), the input layer's slabs (at most 320)
    const size_t col_parts = ((nn + 127) / 128) * (size_t)(od + 1) * W + 320 * (size_t)W * (4 + r);
    slab = slab > loss_parts ? slab : loss_parts;
    slab = slab > col_parts ? slab : col_parts;
    L.slab = take(slab * 4);
    L.slab_floats = slab;
    L.total = o;
    return L;
}

cudaError_t run_loss_grad(const FieldsDev &fd, int field, const float *X, const int *code,
                          const float *target, int n, const float *z_table, int n_codes,
                          float *loss, float *grad_w, float *grad_z, char *ws, int *status,
                          cudaStream_t s) {
    const FieldDev &F = fd.f[field];
    const int r = fd.r, W = F.width, D = F.depth, od = F.out_dim, K0 = 3 + r;
    const int b16 = fd.precision == NSF_PREC_BF16 ? 1 : 0;
    const bool residual = field == NSF_FIELD_G && fd.residual_g;
    const TrainLayout L = train_layout(r, W, D, od, n);
    auto P = [&](size_t off) { return reinterpret_cast<float *>(ws + off); };
    auto P16 = [&](size_t off) { return reinterpret_cast<__nv_bfloat16 *>(ws + off); };
    float *slab = P(L.slab);
    const MatView ones = view(P(L.ones), 0, 0, 0);
    const int ks_thin = thin_slices(n);
#define NSF_GT(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return e_; } while (0)
    // sum over all n points (K) of an M x N product into dst, by K slices
    // (on the tensor cores, with bias_dst: also bias_dst[m] = sum over the n
    // points of A(m, .), from a product of A with ones)
    auto summed = [&](int M, int N, const MatView &A, const MatView &B, bool tc, int split,
                      float *dst, float *bias_dst = nullptr) -> cudaError_t {
        const int tiles = tc ? ((M + 127) / 128) * ((N + 127) / 128)
                             : ((M + 63) / 64) * ((N + 63) / 64);
        const int k = weight_slices(n, tiles, tc);
        GemmEpilogue e = epi(kEpiSlab, slab);
        float *bslab = slab + (size_t)kMaxSlices * M * N;
        if (bias_dst) e.colsum = bslab;
        cudaError_t err = tc ? gemm_tc(M, N, n, A, B, split, e, k, status, s)
                             : gemm_simt(M, N, n, A, B, e, k, s);
        if (err != cudaSuccess) return err;
        return reduce_dw(slab, bslab, k, M, N, dst, bias_dst, s);   // [z][n][m] -> dst[m N + n]
    };
    auto bias_elu = [&](int l) {
        GemmEpilogue e = epi(kEpiBiasElu);
        e.ld = W;
        e.bias = F.b[l];
        if (b16) {       // ELU' codes and the bf16 activations the products read
            e.dact = reinterpret_cast<unsigned short *>(ws + L.A[l]);
            e.h16 = P16(L.H16[l]);
        } else {
            e.pre = P(L.A[l]);
            e.h32 = P(L.H[l]);
        }
        return e;
    };
    auto elu_grad = [&](float *out, int l, int pair, float *colsum = nullptr) {
        GemmEpilogue e = epi(kEpiEluGrad, out, W);
        e.colsum = colsum;
        if (b16) {
            e.dact = reinterpret_cast<unsigned short *>(ws + L.A[l]);
            e.dhi = P16(L.dh[pair]);
            e.dlo = P16(L.dl[pair]);
        } else {
            e.apre = P(L.A[l]);
        }
        return e;
    };
    // the last hidden activation as the thin products read it
    const MatView Hlast_rows = b16 ? view(P16(L.H16[D - 1]), W, 1, 1) : view(P(L.H[D - 1]), W, 1, 0);
    const MatView Hlast_cols = b16 ? view(P16(L.H16[D - 1]), 1, W, 1) : view(P(L.H[D - 1]), 1, W, 0);
    // ---- forward
    k_inputs<<<blocks(n), kT, 0, s>>>(X, code, z_table, n, r, P(L.inp), status);
    // the input layer (K0 = 3 + r inputs)
    if (b16)
        NSF_GT(thin_k(W, n, K0, view(F.W0, K0, 1, 0), view(P(L.inp), K0, 1, 0), bias_elu(0), s));
    else
        NSF_GT(gemm_simt(W, n, K0, view(F.W0, K0, 1, 0), view(P(L.inp), K0, 1, 0), bias_elu(0),
                         1, s));
    if (b16 && D > 1) {
        WeightCopies wc{};
        for (int l = 1; l < D; ++l) {
            wc.Wt[l] = F.Wt[l];
            wc.Wb[l] = P16(L.Wb[l]);
            wc.WTb[l] = P16(L.WTb[l]);
        }
        k_weights_bf16<<<dim3(blocks((long long)W * W), D - 1), kT, 0, s>>>(wc, W);
    }
    for (int l = 1; l < D; ++l) {
        // A_l(o, p) = sum_c W_l[o][c] H_{l-1}(c, p), W_l[o][c] = Wt[l][c W + o]
        if (b16)
            NSF_GT(layer_tc(n, W, W, view(P16(L.H16[l - 1]), W, 1, 1), view(P16(L.Wb[l]), W, 1, 1),
                            bias_elu(l), status, s));
        else
            NSF_GT(gemm_simt(W, n, W, view(F.Wt[l], 1, W, 0), view(P(L.H[l - 1]), W, 1, 0),
                             bias_elu(l), 1, s));
    }
    NSF_GT(thin_m(od, n, W, view(F.Wout, W, 1, 0), Hlast_rows, P(L.raw), od, s));
    // ---- loss, dL/draw and the output bias gradient
    // the per-CTA loss partials sit after the output-bias partials and are
    // added in CTA order before the slab is reused
    float *loss_part = slab + (size_t)blocks(n) * od;
    k_loss<<<blocks(n), kT, 0, s>>>(P(L.raw), F.b[D], X, target, n, od, F, residual ? 1 : 0,
                                    P(L.dout), loss_part, slab);
    NSF_GT(reduce_slabs(loss_part, blocks(n), 1, loss, s));
    k_fill<<<1, 32, 0, s>>>(P(L.ones), 1.f, 4);
    // ---- backward; gradient offsets in the flat layout
    std::vector<size_t> goff(D + 1);
    {
        size_t o = 0;
        for (int l = 0; l <= D; ++l) {
            goff[l] = o;
            const int in = l == 0 ? K0 : W, out = l == D ? od : W;
            o += (size_t)in * out + out;
        }
    }
    // output layer: dbout[a] = sum_p dout(a, p) from k_loss's per-CTA sums,
    // dWout[a][c] = sum_p dout(a, p) H_{D-1}(c, p)
    NSF_GT(reduce_slabs(slab, blocks(n), od, grad_w + goff[D] + (size_t)od * W, s));
    if (!b16)
        NSF_GT(thin_outer(od, W, n, view(P(L.dout), 1, od, 0), Hlast_cols, slab, ks_thin,
                          grad_w + goff[D], false, s));
    float *dcur = P(L.d1), *dnext = P(L.d2);
    // flat offset of layer l's bias gradient
    auto boff = [&](int l) { return goff[l] + (size_t)(l == 0 ? K0 : W) * W; };
    // delta_{D-1}(c, p) = sum_a Wout[a][c] dout(a, p) * ELU'(A_{D-1}(c, p)), db_{D-1}
    int pair = 0;                       // the hi / lo buffers of dcur
    if (b16) {
        // with the output layer's weight gradient dWout[a][c] = sum_p dout(a, p)
        // H_{D-1}(p, c) from the same pass; the bias gradient of layer D - 1
        // comes with its weight gradient (or, D = 1, with the input layer's)
        GemmEpilogue e = elu_grad(nullptr, D - 1, pair);
        e.hin = P16(L.H16[D - 1]);
        e.outer = slab;
        NSF_GT(thin_k(W, n, od, view(F.Wout, 1, W, 0), view(P(L.dout), od, 1, 0), e, s));
        NSF_GT(reduce_slabs(slab, thin_k_parts(n), (long long)od * W, grad_w + goff[D], s));
    } else {
        NSF_GT(gemm_simt(W, n, od, view(F.Wout, 1, W, 0), view(P(L.dout), od, 1, 0),
                         elu_grad(dcur, D - 1, pair), 1, s));
        NSF_GT(thin_outer(1, W, n, ones, view(dcur, 1, W, 0), slab, ks_thin,
                          grad_w + boff(D - 1), false, s));
    }
    for (int l = D - 1; l >= 1; --l) {
        // dW_l[o][c] = sum_p delta_l(o, p) H_{l-1}(c, p); BF16 fields: the cotangent
        // as its hi / lo pairs, both operands with contiguous rows
        if (b16) {
            MatView dpair = view(P16(L.dh[pair]), 1, W, 1);
            dpair.lo = P16(L.dl[pair]);
            NSF_GT(summed(W, W, dpair, view(P16(L.H16[l - 1]), 1, W, 1), true, 1,
                          grad_w + goff[l], grad_w + boff(l)));
        } else {
            NSF_GT(summed(W, W, view(dcur, 1, W, 0), view(P(L.H[l - 1]), 1, W, 0), false, 0,
                          grad_w + goff[l]));
        }
        // delta_{l-1}(c, p) = sum_o W_l[o][c] delta_l(o, p) * ELU'(A_{l-1}(c, p)) and
        // db_{l-1}[c] = sum_p delta_{l-1}(c, p): on the tensor cores the product's
        // epilogue sums its columns, otherwise a thin reduction
        if (b16) {
            MatView dpair = view(P16(L.dh[pair]), W, 1, 1);
            dpair.lo = P16(L.dl[pair]);
            // (the bias gradients come with the weight gradients, layer 0's from
            // the input layer's pass)
            NSF_GT(layer_tc(n, W, W, dpair, view(P16(L.WTb[l]), W, 1, 1),
                            elu_grad(nullptr, l - 1, pair ^ 1), status, s));
        } else {
            NSF_GT(gemm_simt(W, n, W, view(F.Wt[l], W, 1, 0), view(dcur, W, 1, 0),
                             elu_grad(dnext, l - 1, pair ^ 1), 1, s));
            NSF_GT(thin_outer(1, W, n, ones, view(dnext, 1, W, 0), slab, ks_thin,
                              grad_w + boff(l - 1), false, s));
        }
        float *t = dcur;
        dcur = dnext;
        dnext = t;
        pair ^= 1;
    }
    // input layer: dW_0[o][j] = sum_p delta_0(o, p) inp(j, p), db_0 and
    // dinp(j, p) = sum_o W0[o][j] delta_0(o, p)
    if (b16) {
        NSF_GT(input_bwd(n, W, K0, P16(L.dh[pair]), P16(L.dl[pair]), nullptr, W, P(L.inp), F.W0,
                         P(L.dinp), slab, s));
        NSF_GT(reduce_slabs(slab, input_bwd_parts(n), (long long)W * K0 + W, grad_w + goff[0], s));
    } else {
        NSF_GT(thin_outer(K0, W, n, view(P(L.inp), 1, K0, 0), view(dcur, 1, W, 0), slab, ks_thin,
                          grad_w + goff[0], true, s));
    }
    if (grad_z) {
        if (!b16)
            NSF_GT(thin_m(K0, n, W, view(F.W0, 1, K0, 0), view(dcur, W, 1, 0), P(L.dinp), K0, s));
        // the codes in windows that fit the kernel's shared table; the slab
        // (free again) holds the CTAs' tables of a window
        const int win = kDzShared / r;
        for (int c0 = 0; c0 < n_codes; c0 += win) {
            const int nc = n_codes - c0 < win ? n_codes - c0 : win;
            long long g = (long long)(L.slab_floats / ((size_t)nc * r));
            g = g < 304 ? g : 304;
            g = g < blocks(n) ? g : blocks(n);
            g = g < 1 ? 1 : g;
            const int per = (int)((n + g - 1) / g);
            const int grid = (n + per - 1) / per;
            k_scatter_dz<<<grid, kT, 0, s>>>(P(L.dinp), code, n, r, c0, nc, per, slab);
            NSF_GT(cudaGetLastError());
            NSF_GT(reduce_slabs(slab, grid, (long long)nc * r, grad_z + (size_t)c0 * r, s));
        }
    }
#undef NSF_GT
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, long long count, int step,
                        float lr, float b1, float b2, float eps, cudaStream_t s) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<blocks(count), kT, 0, s>>>(p, g, m, v, count, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_repack(const FieldsDev &fd, int field, const float *flat, cudaStream_t s) {
    const FieldDev &F = fd.f[field];
    const int r = fd.r, W = F.width, D = F.depth, od = F.out_dim;
    long long total = 0;
    for (int l = 0; l <= D; ++l) {
        const int in = l == 0 ? 3 + r : W, out = l == D ? od : W;
        total += (long long)in * out + out;
    }
    k_repack<<<blocks(total), kT, 0, s>>>(flat, total, r, D, fd.precision == NSF_PREC_BF16 ? 1 : 0,
                                          F);
    return cudaGetLastError();
}

}  // namespace nsf
