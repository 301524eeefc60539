// FP32 field networks on the CUDA cores (precision NSF_PREC_FP32).
//
// Paper §4.2-§4.4 and App. E: each field is an MLP on [X; z] with ELU hidden
// layers.  §5.1 evaluates g, h, l at the integration particles; §5.3 needs g
// and dg/dz at the sample particles.
//
// A CTA evaluates one field on a tile of ROWS "rows".  In value mode a row is a
// point.  In Jacobian mode every point owns 1 + r consecutive rows: its value
// row and one forward-mode tangent row per latent component (d/dz_k).  All rows
// go through the same per-layer GEMM (tangent rows without the bias), and the
// activation maps a tangent row t to ELU'(a_value) * t using its point's value
// pre-activation, so values and the full Jacobian come out of one pass.
// The input layer (K = 3 + r) is applied per element: value rows take
// W0[:, 0:3] X + W0[:, 3:] z + b0 and tangent row k takes column 3 + k of W0.
#include "device_common.cuh"
#include "gn_solve.cuh"

namespace nsf {

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 32;      // K rows of the transposed weights staged per pass

template <int ROWS>
struct SimtSmem {
    static size_t bytes(int W) {
        return sizeof(float) * ((size_t)2 * ROWS * W + (size_t)kChunk * W +
                                (size_t)ROWS * 9 + W);
    }
};

// Forward pass of one field over a tile.  Leaves the raw output-layer values
// (before de-normalisation; tangent rows without bias) in OUT[ROWS][9].
template <int ROWS>
__device__ void mlp_tile(const FieldDev &F, int r, const float *__restrict__ X,
                         int ld, int n, const double *__restrict__ z, int p0,
                         int S, int npts, float *H, float *P, float *Ws,
                         float *OUT, float *c0) {
    const int tid = threadIdx.x;
    const int W = F.width;
    const int in0 = 3 + r;
    const int used = npts * S;

    // c0[j] = b0[j] + sum_k W0[j][3 + k] z_k  (constant over the tile)
    for (int j = tid; j < W; j += kThreads) {
        const float *w = F.W0 + (size_t)j * in0;
        float a = F.b[0][j];
        for (int k = 0; k < r; ++k) a = fmaf(w[3 + k], (float)z[k], a);
        c0[j] = a;
    }
    __syncthreads();

    // Input layer -> pre-activations P.
    for (int idx = tid; idx < ROWS * W; idx += kThreads) {
        int row = idx / W, j = idx - row * W;
        float a = 0.f;
        if (row < used) {
            int lp = row / S, slot = row - lp * S;
            const float *w = F.W0 + (size_t)j * in0;
            if (slot == 0) {
                int p = p0 + lp;
                float x0 = 0.f, x1 = 0.f, x2 = 0.f;
                if (p < n) {
                    x0 = X[p];
                    x1 = X[ld + p];
                    x2 = X[2 * ld + p];
                }
                a = fmaf(w[0], x0, fmaf(w[1], x1, fmaf(w[2], x2, c0[j])));
            } else {
                a = w[3 + slot - 1];
            }
        }
        P[idx] = a;
    }
    __syncthreads();

    const int rg = tid >> 5;            // row group (ROWS / 8 rows each)
    const int cg = tid & 31;            // column group: cols cg + 32 c
    constexpr int RPT = ROWS / 8;
    const int ncol = (W + 31) >> 5;

    for (int layer = 1; layer <= F.depth; ++layer) {
        // Activation of the previous layer: P -> H.
        for (int idx = tid; idx < ROWS * W; idx += kThreads) {
            int row = idx / W, j = idx - row * W;
            int lp = row / S, slot = row - lp * S;
            float pre = P[idx];
            float h;
            if (slot == 0) h = elu(pre);
            else h = elu_grad(P[(lp * S) * W + j]) * pre;
            H[idx] = h;
        }
        __syncthreads();
        if (layer == F.depth) break;

        // Hidden GEMM: P = H * Wt[layer] (+ b for value rows).
        const float *Wt = F.Wt[layer];
        float acc[RPT][8];
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[i][c] = 0.f;
        for (int k0 = 0; k0 < W; k0 += kChunk) {
            const int kc = min(kChunk, W - k0);
            for (int idx = tid; idx < kc * W; idx += kThreads)
                Ws[idx] = __ldg(&Wt[(size_t)k0 * W + idx]);
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < kc; ++kk) {
                float a[RPT];
#pragma unroll
                for (int i = 0; i < RPT; ++i) a[i] = H[(rg * RPT + i) * W + k0 + kk];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    if (c < ncol && cg + 32 * c < W) {
                        float b = Ws[kk * W + cg + 32 * c];
#pragma unroll
                        for (int i = 0; i < RPT; ++i) acc[i][c] = fmaf(a[i], b, acc[i][c]);
                    }
                }
            }
            __syncthreads();
        }
        const float *bl = F.b[layer];
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            int row = rg * RPT + i;
            int slot = row % S;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (c < ncol && cg + 32 * c < W) {
                    int col = cg + 32 * c;
                    P[row * W + col] = acc[i][c] + (slot == 0 ? bl[col] : 0.f);
                }
            }
        }
        __syncthreads();
    }

    // Output layer: OUT[row][o] = sum_k H[row][k] Wout[o][k] (+ b for value rows).
    const int od = F.out_dim;
    const float *bo = F.b[F.depth];
    for (int idx = tid; idx < ROWS * od; idx += kThreads) {
        int row = idx / od, o = idx - row * od;
        const float *w = F.Wout + (size_t)o * W;
        const float *h = H + (size_t)row * W;
        float a = 0.f;
        for (int k = 0; k < W; ++k) a = fmaf(h[k], __ldg(&w[k]), a);
        OUT[row * 9 + o] = a + ((row % S) == 0 ? bo[o] : 0.f);
    }
    __syncthreads();
}

struct FieldJobs {
    int njobs;
    FieldJob job[4];
};

template <int ROWS>
__global__ void __launch_bounds__(kThreads)
k_fields(const __grid_constant__ FieldsDev fd, const float *__restrict__ X,
         int n, int ld, const __grid_constant__ FieldJobs jobs, int *status) {
    extern __shared__ float smem[];
    const FieldJob &job = jobs.job[blockIdx.y];
    const FieldDev &F = fd.f[job.field];
    const int W = F.width;
    float *H = smem, *P = H + ROWS * W, *Ws = P + ROWS * W, *OUT = Ws + kChunk * W,
          *c0 = OUT + ROWS * 9;
    const int p0 = blockIdx.x * ROWS;
    const int npts = min(ROWS, n - p0);
    mlp_tile<ROWS>(F, fd.r, X, ld, n, job.z, p0, 1, npts, H, P, Ws, OUT, c0);
    const int od = F.out_dim;
    bool bad = false;
    for (int idx = threadIdx.x; idx < npts * od; idx += kThreads) {
        int row = idx / od, o = idx - row * od;
        float y = fmaf(F.scale[o], OUT[row * 9 + o], F.shift[o]);
        bad |= !isfinite(y);
        job.out[(size_t)o * ld + p0 + row] = y;
    }
    if (bad) set_status(status, NSF_ERR_NONFINITE);
}

constexpr int kJacRows = 64;

__global__ void __launch_bounds__(kThreads)
k_jacobian(const __grid_constant__ FieldsDev fd, const float *__restrict__ X,
           int n, int ld, const double *__restrict__ z, float *u, float *dudz,
           const __grid_constant__ GnArgs gn, int gn_on, int it, int *status) {
    extern __shared__ float smem[];
    __shared__ GnShared gsh;
    __shared__ float RES[kJacRows][3];
    __shared__ float JS[kJacRows][3][kMaxR];
    __shared__ double PART[kGnStrideMax];
    const FieldDev &F = fd.f[NSF_FIELD_G];
    const int r = fd.r, S = 1 + r, ppc = kJacRows / S;
    const int W = F.width;
    float *H = smem, *P = H + kJacRows * W, *Ws = P + kJacRows * W,
          *OUT = Ws + kChunk * W, *c0 = OUT + kJacRows * 9;
    const int p0 = blockIdx.x * ppc;
    const int npts = max(0, min(ppc, n - p0));
    mlp_tile<kJacRows>(F, r, X, ld, n, z, p0, S, npts, H, P, Ws, OUT, c0);

    bool bad = false;
    for (int idx = threadIdx.x; idx < ppc * 3; idx += kThreads) {
        int lp = idx / 3, a = idx - lp * 3;
        int p = p0 + lp;
        float ua = 0.f, res = 0.f;
        bool valid = lp < npts;
        if (valid) {
            ua = fmaf(F.scale[a], OUT[(lp * S) * 9 + a], F.shift[a]);
            bad |= !isfinite(ua);
            if (u) u[(size_t)a * ld + p] = ua;
            if (gn_on) res = ua - gn.target[(size_t)a * gn.target_ld + p];
        }
        RES[lp][a] = valid ? res : 0.f;
        for (int k = 0; k < r; ++k) {
            float j = valid ? F.scale[a] * OUT[(lp * S + 1 + k) * 9 + a] : 0.f;
            bad |= !isfinite(j);
            JS[lp][a][k] = j;
            if (valid && dudz) dudz[(size_t)(a * r + k) * ld + p] = j;
        }
    }
    if (bad) set_status(status, NSF_ERR_NONFINITE);
    if (!gn_on) return;
    __syncthreads();

    // Per-CTA float64 partial normal equations.
    const int T = r * (r + 1) / 2;
    const int stride = T + r + 1;
    for (int e = threadIdx.x; e < stride; e += kThreads) {
        double s = 0.0;
        if (e < T) {
            int i = 0, off = 0;
            while (e >= off + (r - i)) { off += r - i; ++i; }
            int j = i + (e - off);
            for (int lp = 0; lp < npts; ++lp)
                for (int a = 0; a < 3; ++a)
                    s = fma((double)JS[lp][a][i], (double)JS[lp][a][j], s);
        } else if (e < T + r) {
            int k = e - T;
            for (int lp = 0; lp < npts; ++lp)
                for (int a = 0; a < 3; ++a)
                    s = fma((double)JS[lp][a][k], (double)RES[lp][a], s);
        } else {
            for (int lp = 0; lp < npts; ++lp)
                for (int a = 0; a < 3; ++a)
                    s = fma((double)RES[lp][a], (double)RES[lp][a], s);
        }
        PART[e] = s;
    }
    __syncthreads();
    gn_arrive_and_solve(gn, r, it, status, gsh, PART);
}

}  // namespace

int gn_partial_stride(int r) { return r * (r + 1) / 2 + r + 1; }

int jac_grid_size_simt(const FieldsDev &fd, int n) {
    int ppc = kJacRows / (1 + fd.r);
    return (n + ppc - 1) / ppc;
}

cudaError_t launch_fields_simt(const FieldsDev &fd, const float *X, int n,
                               int ld, int njobs, const FieldJob *jobs,
                               int *status, cudaStream_t s) {
    constexpr int ROWS = 32;
    FieldJobs fj;
    fj.njobs = njobs;
    int W = 0;
    for (int i = 0; i < njobs; ++i) {
        fj.job[i] = jobs[i];
        W = max(W, fd.f[jobs[i].field].width);
    }
    size_t sm = SimtSmem<ROWS>::bytes(W);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_fields<ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SimtSmem<ROWS>::bytes(kMaxWidth));
        attr = true;
    }
    dim3 grid((n + ROWS - 1) / ROWS, njobs);
    k_fields<ROWS><<<grid, kThreads, sm, s>>>(fd, X, n, ld, fj, status);
    return cudaGetLastError();
}

cudaError_t launch_jacobian_simt(const FieldsDev &fd, const float *X, int n,
                                 int ld, const double *z, float *u, float *dudz,
                                 const GnArgs *gn, int it, int *status,
                                 cudaStream_t s) {
    const int W = fd.f[NSF_FIELD_G].width;
    size_t sm = SimtSmem<kJacRows>::bytes(W);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_jacobian, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SimtSmem<kJacRows>::bytes(kMaxWidth));
        attr = true;
    }
    int grid = jac_grid_size_simt(fd, n);
    GnArgs g{};
    if (gn) g = *gn;
    k_jacobian<<<grid, kThreads, sm, s>>>(fd, X, n, ld, gn ? gn_z_in(*gn, it) : z, u, dudz, g,
                                          gn ? 1 : 0, it, status);
    return cudaGetLastError();
}

}  // namespace nsf
