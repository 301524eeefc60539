// Fitting a field network to full-order snapshots (paper App. D): loss,
// hand-written backward and Adam, plus the device-side re-pack of updated
// weights into an nsf_fields.
//
// Activations are column-major per point (column p = point p).  Forward, per
// linear layer l:  A_l = W_l H_{l-1} + b_l,  H_l = ELU(A_l), with H_{-1} =
// [X; z] and the input layer in FP32; the other products in the fields'
// precision (BF16 fields: bf16 operands, FP32 accumulation on the tensor
// cores; the activations entering a product are rounded to bf16).  Loss: the
// mean squared normalised error L = sum ((y - y*) / scale)^2 / (n out_dim).
// Backward in FP32 (TF32 products for BF16 fields) on the forward's
// activations:
//   delta_out = dL/draw = 2 (y - y*) / (scale n out_dim)
//   dW_l = delta_l H_{l-1}^T,  db_l = delta_l x ones (row sums),
//   delta_{l-1} = (W_l^T delta_l) * ELU'(A_{l-1}),
//   dz_t += (W_0^T delta_0)[3:, p] over the points p of snapshot t.
// The dense products go to cuBLAS (plain GEMMs); the chain rule around them
// runs in the kernels below.
#include <mutex>
#include <vector>

#include <cublas_v2.h>

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

// H = ELU(A + b) over a rows x n block (CTA y = a group of points, thread x a
// row); H32 gets the value entering the next product (bf16-rounded when
// round_bf16), H16 (optional) its bf16 copy.
__global__ void k_bias_elu(float *A, const float *__restrict__ b, int rows, int n, float *H32,
                           __nv_bfloat16 *H16, int round_bf16) {
    const int o = threadIdx.x;
    if (o >= rows) return;
    const float bo = b[o];
    for (int p = blockIdx.x; p < n; p += gridDim.x) {
    const size_t i = (size_t)p * rows + o;
    const float a = A[i] + bo;
    A[i] = a;
    float h = a > 0.f ? a : expm1f(a);
    const __nv_bfloat16 hb = __float2bfloat16_rn(h);
    if (round_bf16) h = __bfloat162float(hb);
    H32[i] = h;
    if (H16) H16[i] = hb;
    }
}

// Outputs, loss and dL/draw.  raw: od x n (column-major), target [od][n].
__global__ void k_loss(const float *__restrict__ raw, const float *__restrict__ bout,
                       const float *__restrict__ X, const float *__restrict__ target, int n,
                       int od, FieldDev F, int residual, float *delta, float *loss) {
    __shared__ float part[kT];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    if (p < n) {
        for (int a = 0; a < od; ++a) {
            float y = fmaf(F.scale[a], raw[(size_t)p * od + a] + bout[a], F.shift[a]);
            if (residual) y += X[(size_t)a * n + p];
            const float e = (y - target[(size_t)a * n + p]) / F.scale[a];
            acc = fmaf(e, e, acc);
            delta[(size_t)p * od + a] = 2.f * e / ((float)n * (float)od);
        }
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, part[0] / ((float)n * (float)od));
}

// delta *= ELU'(A)
__global__ void k_elu_grad(float *delta, const float *__restrict__ A, long long count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float a = A[i];
    delta[i] *= a > 0.f ? 1.f : expf(a);
}

__global__ void k_fill(float *a, float v, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) a[i] = v;
}

// dz_code(p) += dinp[3:, p]: per CTA into a shared copy of the table (when it
// fits), then one global atomic per entry the CTA touched.
constexpr int kDzShared = 4096;
__global__ void k_scatter_dz(const float *__restrict__ dinp, const int *__restrict__ code, int n,
                             int r, int n_codes, float *gz) {
    __shared__ float tab[kDzShared];
    const bool local = n_codes * r <= kDzShared;
    if (local)
        for (int i = threadIdx.x; i < n_codes * r; i += blockDim.x) tab[i] = 0.f;
    __syncthreads();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int c = code[p];
        if (c < 0 || c >= n_codes) continue;
        for (int k = 0; k < r; ++k) {
            const float v = dinp[(size_t)p * (3 + r) + 3 + k];
            if (local) atomicAdd(&tab[c * r + k], v);
            else atomicAdd(&gz[(size_t)c * r + k], v);
        }
    }
    if (!local) return;
    __syncthreads();
    for (int i = threadIdx.x; i < n_codes * r; i += blockDim.x)
        if (tab[i] != 0.f) atomicAdd(&gz[i], tab[i]);
}

__global__ void k_to_bf16(const float *__restrict__ a, __nv_bfloat16 *b, long long count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) b[i] = __float2bfloat16_rn(a[i]);
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

std::mutex g_mu;
cublasHandle_t g_handle[64] = {};

cublasHandle_t handle_for_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_handle[dev]) {
        cublasHandle_t h;
        if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return nullptr;
        cublasSetPointerMode(h, CUBLAS_POINTER_MODE_HOST);
        cublasSetMathMode(h, CUBLAS_DEFAULT_MATH);
        g_handle[dev] = h;
    }
    return g_handle[dev];
}

// C (m x n, ld ldc) = op(A) op(B), all column-major FP32.
cublasStatus_t sgemm(cublasHandle_t h, bool ta, bool tb, int m, int n, int k, const float *A,
                     int lda, const float *B, int ldb, float *C, int ldc) {
    const float one = 1.f, zero = 0.f;
    return cublasSgemm(h, ta ? CUBLAS_OP_T : CUBLAS_OP_N, tb ? CUBLAS_OP_T : CUBLAS_OP_N, m, n, k,
                       &one, A, lda, B, ldb, &zero, C, ldc);
}

// The same with bf16 operands and FP32 accumulation and result.
cublasStatus_t gemm_bf16(cublasHandle_t h, bool ta, bool tb, int m, int n, int k,
                         const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                         float *C, int ldc) {
    const float one = 1.f, zero = 0.f;
    return cublasGemmEx(h, ta ? CUBLAS_OP_T : CUBLAS_OP_N, tb ? CUBLAS_OP_T : CUBLAS_OP_N, m, n,
                        k, &one, A, CUDA_R_16BF, lda, B, CUDA_R_16BF, ldb, &zero, C, CUDA_R_32F,
                        ldc, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
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
    L.w16 = take((size_t)W * W * 2);
    L.ones = take(nn * 4);
    L.total = o;
    return L;
}

cudaError_t run_loss_grad(const FieldsDev &fd, int field, const float *X, const int *code,
                          const float *target, int n, const float *z_table, int n_codes,
                          float *loss, float *grad_w, float *grad_z, char *ws, int *status,
                          cudaStream_t s) {
    const FieldDev &F = fd.f[field];
    const int r = fd.r, W = F.width, D = F.depth, od = F.out_dim, K0 = 3 + r;
    const bool bf16 = fd.precision == NSF_PREC_BF16;
    const bool residual = field == NSF_FIELD_G && fd.residual_g;
    const TrainLayout L = train_layout(r, W, D, od, n);
    cublasHandle_t h = handle_for_current_device();
    if (!h) return cudaErrorNotReady;
    if (cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) return cudaErrorNotReady;
    auto P = [&](size_t off) { return reinterpret_cast<float *>(ws + off); };
    auto P16 = [&](size_t off) { return reinterpret_cast<__nv_bfloat16 *>(ws + off); };
    const long long nW = (long long)W * n;
#define NSF_CB(x) do { if ((x) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown; } while (0)
    // ---- forward
    k_inputs<<<blocks(n), kT, 0, s>>>(X, code, z_table, n, r, P(L.inp), status);
    NSF_CB(sgemm(h, true, false, W, n, K0, F.W0, K0, P(L.inp), K0, P(L.A[0]), W));
    const int ecta = n < 4 * 152 * 8 ? n : 4 * 152 * 8;      // CTAs of the row-wise kernels
    k_bias_elu<<<ecta, W, 0, s>>>(P(L.A[0]), F.b[0], W, n, P(L.H[0]),
                                  bf16 ? P16(L.H16[0]) : nullptr, bf16 ? 1 : 0);
    for (int l = 1; l < D; ++l) {
        if (bf16) {
            k_to_bf16<<<blocks((long long)W * W), kT, 0, s>>>(F.Wt[l], P16(L.w16), (long long)W * W);
            NSF_CB(gemm_bf16(h, false, false, W, n, W, P16(L.w16), W, P16(L.H16[l - 1]), W,
                             P(L.A[l]), W));
        } else {
            NSF_CB(sgemm(h, false, false, W, n, W, F.Wt[l], W, P(L.H[l - 1]), W, P(L.A[l]), W));
        }
        k_bias_elu<<<ecta, W, 0, s>>>(P(L.A[l]), F.b[l], W, n, P(L.H[l]),
                                      bf16 ? P16(L.H16[l]) : nullptr, bf16 ? 1 : 0);
    }
    if (bf16) {
        k_to_bf16<<<blocks((long long)od * W), kT, 0, s>>>(F.Wout, P16(L.w16), (long long)od * W);
        NSF_CB(gemm_bf16(h, true, false, od, n, W, P16(L.w16), W, P16(L.H16[D - 1]), W, P(L.raw),
                         od));
    } else {
        NSF_CB(sgemm(h, true, false, od, n, W, F.Wout, W, P(L.H[D - 1]), W, P(L.raw), od));
    }
    // ---- loss and dL/draw
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    k_loss<<<blocks(n), kT, 0, s>>>(P(L.raw), F.b[D], X, target, n, od, F, residual ? 1 : 0,
                                    P(L.dout), loss);
    // ---- backward; gradient offsets in the flat layout.  BF16 fields take
    // their backward products in TF32 on the tensor cores (10-bit mantissa
    // operands, FP32 accumulation: well inside the bf16 forward's rounding);
    // FP32 fields keep FP32 products.
    if (bf16) NSF_CB(cublasSetMathMode(h, CUBLAS_TF32_TENSOR_OP_MATH));
    struct MathReset {
        cublasHandle_t h;
        ~MathReset() { cublasSetMathMode(h, CUBLAS_DEFAULT_MATH); }
    } reset{h};
    std::vector<size_t> goff(D + 1);
    {
        size_t o = 0;
        for (int l = 0; l <= D; ++l) {
            goff[l] = o;
            const int in = l == 0 ? K0 : W, out = l == D ? od : W;
            o += (size_t)in * out + out;
        }
    }
    // output layer: dWout (row-major od x W) = H_{D-1} dout^T as a W x od column-major
    NSF_CB(sgemm(h, false, true, W, od, n, P(L.H[D - 1]), W, P(L.dout), od, grad_w + goff[D], W));
    // bias gradients: row sums of delta = delta x ones
    k_fill<<<blocks(n), kT, 0, s>>>(P(L.ones), 1.f, n);
    const float one = 1.f, zero = 0.f;
    NSF_CB(cublasSgemv(h, CUBLAS_OP_N, od, n, &one, P(L.dout), od, P(L.ones), 1, &zero,
                       grad_w + goff[D] + (size_t)od * W, 1));
    float *dcur = P(L.d1), *dnext = P(L.d2);
    NSF_CB(sgemm(h, false, false, W, n, od, F.Wout, W, P(L.dout), od, dcur, W));
    for (int l = D - 1; l >= 1; --l) {
        k_elu_grad<<<blocks(nW), kT, 0, s>>>(dcur, P(L.A[l]), nW);
        NSF_CB(sgemm(h, false, true, W, W, n, P(L.H[l - 1]), W, dcur, W, grad_w + goff[l], W));
        NSF_CB(cublasSgemv(h, CUBLAS_OP_N, W, n, &one, dcur, W, P(L.ones), 1, &zero,
                           grad_w + goff[l] + (size_t)W * W, 1));
        NSF_CB(sgemm(h, true, false, W, n, W, F.Wt[l], W, dcur, W, dnext, W));
        float *t = dcur;
        dcur = dnext;
        dnext = t;
    }
    k_elu_grad<<<blocks(nW), kT, 0, s>>>(dcur, P(L.A[0]), nW);
    NSF_CB(sgemm(h, false, true, K0, W, n, P(L.inp), K0, dcur, W, grad_w + goff[0], K0));
    NSF_CB(cublasSgemv(h, CUBLAS_OP_N, W, n, &one, dcur, W, P(L.ones), 1, &zero,
                       grad_w + goff[0] + (size_t)K0 * W, 1));
    if (grad_z) {
        e = cudaMemsetAsync(grad_z, 0, (size_t)n_codes * r * sizeof(float), s);
        if (e != cudaSuccess) return e;
        NSF_CB(sgemm(h, false, false, K0, n, W, F.W0, K0, dcur, W, P(L.dinp), K0));
        k_scatter_dz<<<blocks(n) < 304 ? blocks(n) : 304, kT, 0, s>>>(P(L.dinp), code, n, r,
                                                                   n_codes, grad_z);
    }
#undef NSF_CB
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
