// Internal declarations of libnsf shared by the host API and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "nsf.h"

namespace nsf {

constexpr int kMaxR = NSF_MAX_R;
// float64 partial sums of one Gauss-Newton iteration (J^T J upper triangle,
// J^T res, |res|^2) for the largest latent dimension
constexpr int kGnStrideMax = kMaxR * (kMaxR + 1) / 2 + kMaxR + 1;
constexpr int kMaxWidth = NSF_MAX_WIDTH;
constexpr int kMaxDepth = NSF_MAX_DEPTH;
constexpr int kOutDim[3] = {3, 6, 9};

// ---------------------------------------------------------------- fields ---
// One field network in device memory.  FP32 layout (CUDA-core path):
//   W0  [width][3 + r] row-major (input layer, as given),
//   Wt[l] for hidden layers l = 1 .. depth-1: transposed, [in = width][out = width],
//   Wout [out_dim][width] row-major, b[l] biases of layer l (l = 0 .. depth).
// BF16 layout (tensor-core path): one contiguous blob per field holding the
// hidden matrices l = 1 .. depth-1 ([out][in]) and the output matrix
// (zero-padded to 16 rows) as bf16, K-major with the 128-byte swizzle of
// tcgen05.mma operands (tc_common.cuh); it is copied verbatim into shared
// memory.  W0 and the biases stay FP32 (W0 holding bf16-rounded values).
struct FieldDev {
    int width, depth, out_dim;
    const float *W0;
    const float *Wt[kMaxDepth];
    const float *Wout;
    const float *b[kMaxDepth + 1];
    const __nv_bfloat16 *tc_blob;          // BF16 packed weights (or null)
    int tc_blob_bytes;
    float scale[9], shift[9];
};

struct FieldsDev {
    int r;
    int residual_g;
    int precision;
    FieldDev f[3];
};

// ------------------------------------------------------------- workspace ---
// Counters of one MPM step.  Two sets alternate with the step's epoch parity:
// a step uses set (epoch & 1) and clears the other one, which no launch of
// this step reads (the previous step's launches are complete).
struct StepCtl {
    int n_p;            // active particle blocks (binned particles)
    int n_g;            // active grid blocks
    int n_over;         // particles past their block's bucket capacity
    unsigned bound;     // float bits of the largest P2G contribution bound
};

struct Ctl {
    int epoch;          // incremented once per MPM step (grid-block stamps)
    int pad0[3];
    StepCtl st[2];
    int pad1[20];
    // arrival word of the fused MPM kernel's grid barrier, alone in its
    // 128-byte line
    unsigned bar;
    unsigned pad2[31];
};

// Sparse-in-use, dense-in-address background grid.  Nodes are stored
// block-linear: 4x4x4-node blocks, block (bx, by, bz) at
// ((bx * nb1 + by) * nb2 + bz), node (lx, ly, lz) inside at (lx * 4 + ly) * 4 + lz.
// A particle belongs to the block of its stencil base node ("particle
// block"); its stencil reaches the 6^3 nodes from that block's first node on,
// i.e. that grid block and the next one along each axis.
// Largest bucket capacity per particle block.  The P2G tile of a block sums
// at most this many contributions per node, which bounds its 32-bit partial
// sums (mpm.cu).
constexpr int kMaxBucketCap = 1024;

struct GridWs {
    int n0, n1, n2;
    int nb0, nb1, nb2, nblocks;
    unsigned long long *acc;   // [nodes][4] fixed-point (m, p) sums; zero between steps
    float4 *vel;        // (v, m) after the grid update; valid on the step's active blocks
    int *gstamp;        // epoch stamp of each grid block
    int *bcount;        // particles binned to each particle block; zero between steps
    int *bucket;        // [nblocks][cap] particle indices of each particle block
    int cap;            // bucket capacity per particle block
    float4 *rec;        // [n][4] P2G record of each particle (x, m v, Q)
    int *plist;         // active particle blocks of the step
    int *glist;         // active grid blocks of the step
    int *over;          // particles whose block's bucket was full
    Ctl *ctl;
    int max_pblocks, max_gblocks;
};

struct GridParams {
    float dx, inv_dx;
    float gx, gy, gz;
    int wall_cells;
    int blade_enable;
    float blade_x, blade_z0, blade_vz;
};

// ------------------------------------------------------------- launchers ---
// All return cudaGetLastError() of their launches.

// Field evaluation on n points for up to 4 (field, z) jobs (value only).
struct FieldJob {
    int field;
    const double *z;
    float *out;          // [out_dim][ld]; for a residual g this is the displacement u
};

// Value + forward-mode Jacobian of g on n points.
//  - eval mode (gn == null): writes u [3][n] (if u) and dudz [3][r][n] (if dudz).
//  - Gauss-Newton mode (gn != null): per-CTA float64 partial normal
//    equations, and the last CTA to finish solves and updates z.
struct GnArgs {
    const float *target;      // [3][target_ld] target displacement d (x^{n+1} - X for residual g)
    int target_ld;
    int iters;                // Gauss-Newton iterations of the run
    const double *z_start;    // z at the start of the run (iteration 0 input)
    double *z_buf;            // z between iterations (one launch per iteration)
    double *z_out;            // z after the last iteration (may alias z_start)
    double *z_prev_out;       // if non-null: receives z_start after the last iteration
    double *z_taps;           // [iters][r] optional copy of z after every iteration
    double *gsum;             // [2][kGnStrideMax] float64 sums, zero before and after
    int *counter;             // arrival ticket (one launch per iteration), zero before and after
    unsigned *bar;            // grid-barrier arrival word (all iterations in one launch)
    float2 *slots;            // [2][gn_partial_stride(r)][grid] per-CTA float-float sums
    double damping;
};
int gn_partial_stride(int r);
// CTAs that combine one Gauss-Newton run on the tensor-core path are at most
// one per SM; a lane adds the slots of CTAs lane, lane + 32, ...
constexpr int kGnMaxSlotsPerLane = 5;
constexpr int kGnMaxCtas = 32 * kGnMaxSlotsPerLane;

// CUDA-core FP32 path (fields_simt.cu).
int jac_grid_size_simt(const FieldsDev &fd, int n);
cudaError_t launch_fields_simt(const FieldsDev &fd, const float *X, int n, int ld,
                               int njobs, const FieldJob *jobs, int *status,
                               cudaStream_t s);
// Eval mode (gn == null) or one Gauss-Newton iteration `it` (z read from
// gn_z_in(gn, it)); the host launches it once per iteration.
cudaError_t launch_jacobian_simt(const FieldsDev &fd, const float *X, int n, int ld,
                                 const double *z, float *u, float *dudz,
                                 const GnArgs *gn, int it, int *status, cudaStream_t s);

// Tensor-core BF16 path: value evaluation (fields_tc.cu), Jacobian and
// Gauss-Newton (jacobian_tc.cu).
int jac_grid_size_tc(const FieldsDev &fd, int n);
cudaError_t launch_fields_tc(const FieldsDev &fd, const float *X, int n, int ld,
                             int njobs, const FieldJob *jobs, int *status,
                             cudaStream_t s);
// Eval mode (gn == null) or all gn->iters Gauss-Newton iterations in one
// cooperative launch (a grid barrier between iterations).
cudaError_t launch_jacobian_tc(const FieldsDev &fd, const float *X, int n, int ld,
                               const double *z, float *u, float *dudz,
                               const GnArgs *gn, int *status, cudaStream_t s);

// ------------------------------------------------- integration particles ---
// Construction of N from S (subset.cu, paper §5.4).
struct SubsetArgs {
    const float *X;            // [3][n] reference positions of all particles
    const float *u;            // [3][n] g(X, z) (displacement for a residual g)
    int residual;              // 1: x = X + u
    int n;                     // |P|
    const int *sample;         // [n_S] indices of S in P
    int n_S;
    int dims[3];
    float inv_dx;
    unsigned *bitmap;          // ceil(nodes / 32) words, zero on entry
    unsigned char *in_S;       // [n], zero on entry
    int *block_count, *block_off;   // [ceil(n / 256)]
    int *index_out;            // [n] capacity
};
cudaError_t launch_subset(const SubsetArgs &a, int *count_out, float *X_out, int ld_out,
                          int *status, cudaStream_t s);

// ------------------------------------------------------------------ GEMM ---
// Dense products of training (gemm.cu): D(m, n) = sum_k A(m, k) B(n, k) for
// m < M, n < N, k < K, the operands read through strided views.
struct MatView {
    const void *ptr;       // element (row, k) at ptr[row * s_row + k * s_k]
    long long s_row, s_k;
    int bf16;              // element type: 1 bf16, 0 float
    const void *lo;        // bf16 views of a split operand: the lo parts (same strides)
};
enum { kEpiStore = 0, kEpiBiasElu = 1, kEpiEluGrad = 2, kEpiSlab = 3 };
struct GemmEpilogue {
    int mode;
    float *out;            // Store, EluGrad: out[n * ld + m]; Slab: out[z M N + n M + m]
    long long ld;
    const float *bias;     // BiasElu: pre = D + bias[m] -> pre[n ld + m]
    float *pre;
    float *h32;            // BiasElu: ELU(pre) (may be null)
    __nv_bfloat16 *h16;    // BiasElu: its bf16 copy (may be null)
    const float *apre;     // EluGrad: out = D * ELU'(apre[n ld + m])
    float *colsum;         // (may be null) partial sums for a bias gradient: see the
                           // products that take it
    __nv_bfloat16 *dhi, *dlo;   // EluGrad (may be null): out as hi = bf16(v), lo = bf16(v - hi)
    const __nv_bfloat16 *hin;   // thin_k EluGrad (may be null): H for the outer-product sums
    float *outer;          //   written per CTA (see thin_k)
    unsigned short *dact;  // BF16 path (replaces pre / apre): ELU'(pre) as the 16-bit code
                           // rint(ELU' 2^15) at [n ld + m]; BiasElu then writes only dact
                           // and h16 (ELU on the special-function unit)
};
// FP32 product on the CUDA cores; K split over `kslices` slices (only with
// the Slab epilogue, which writes one M x N slab per slice).
cudaError_t gemm_simt(int M, int N, int K, const MatView &A, const MatView &B,
                      const GemmEpilogue &e, int kslices, cudaStream_t s);
// BF16 product on the tcgen05 tensor cores with FP32 accumulation in tensor
// memory, operands brought in by TMA (the Slab epilogue; with e.colsum also
// the sums of A over each K-slice, colsum[z * M + m]).  Both operands bf16, each either with
// contiguous k (s_k = 1) or with contiguous rows (s_row = 1), 16-byte
// aligned, strides multiples of 8 elements; split = 1 (2) adds the product of
// operand A's (B's) lo parts (view.lo), so that an operand kept as hi + lo
// pairs counts with ~16 significant bits.
cudaError_t gemm_tc(int M, int N, int K, const MatView &A, const MatView &B, int split,
                    const GemmEpilogue &e, int kslices, int *status, cudaStream_t s);
// Thin shapes.  thin_outer: out(a, c) = sum_k U(a, k) V(c, k) for A <= 32,
// k split into `slices` slabs summed in a fixed order, out row-major [A][C]
// (or [C][A] when transposed).  thin_m: D(m, n) = sum_k A(m, k) B(n, k) for
// M <= 32, K <= 256, out[n * ld + m].
cudaError_t thin_outer(int A, int C, int K, const MatView &U, const MatView &V, float *slab,
                       int slices, float *out, bool transposed, cudaStream_t s);
cudaError_t thin_m(int M, int N, int K, const MatView &A, const MatView &B, float *out,
                   long long ld, cudaStream_t s);
// The hidden layers' products on the tensor cores, the points as the M
// dimension: Y(p, c) = sum_k X(p, k) Wt(c, k) for p < n, c < W (<= 256, a
// multiple of 16), k < K (<= 256); X bf16 [p][k] (with lo parts: the split
// cotangent of the backward product), Wt bf16 [c][k].  Epilogue BiasElu (X
// without lo; dact and h16) or EluGrad (X with lo; dact, dhi, dlo, optional
// out and colsum), all at [p ld + c].  EluGrad's colsum gets layer_tc_parts(n, W)
// partial sums per channel: colsum[part * W + c].
cudaError_t layer_tc(int n, int W, int K, const MatView &X, const MatView &Wt,
                     const GemmEpilogue &e, int *status, cudaStream_t s);
int layer_tc_parts(int n, int W);
// Thin K (<= 20): the input layer's forward product and the output layer's
// backward product on the BF16 path (epilogue BiasElu or EluGrad with dact;
// M % 4 == 0, ld % 4 == 0).  EluGrad's colsum gets thin_k_parts(N) partial
// sums per row: colsum[part * M + m].
// With e.hin (EluGrad, K <= 16) also outer[(part K + k) M + m] = sum over the
// part's columns of B(n, k) hin[n ld + m].
cudaError_t thin_k(int M, int N, int K, const MatView &A, const MatView &B,
                   const GemmEpilogue &e, cudaStream_t s);
int thin_k_parts(int N);
// The input layer's backward pass on the BF16 path, one read of delta_0 (bf16
// hi + lo pairs, or d32 in FP32) at [p ld + o]: dinp[p K0 + j] = sum_o
// W0[o K0 + j] delta_0(p, o), and input_bwd_parts(n) slabs of W K0 + W
// partial sums in the gradient layout of layer 0 (dW0[o K0 + j] = sum_p
// delta_0(p, o) inp[p K0 + j], then db0[o] = sum_p delta_0(p, o)).
cudaError_t input_bwd(int n, int W, int K0, const __nv_bfloat16 *dhi, const __nv_bfloat16 *dlo,
                      const float *d32, long long ld, const float *inp, const float *W0,
                      float *dinp, float *slab, cudaStream_t s);
int input_bwd_parts(int n);
// out[i] = sum over z < slices of slab[z * count + i] (fixed order); the slab
// may be overwritten.
cudaError_t reduce_slabs(float *slab, int slices, long long count, float *out, cudaStream_t s);
// A hidden layer's weight and bias gradients from the slabs of gemm_tc
// (slab[z][n][m] -> out_w[m N + n], bslab[z][m] -> out_b[m], out_b may be null).
cudaError_t reduce_dw(const float *slab, const float *bslab, int slices, int M, int N,
                      float *out_w, float *out_b, cudaStream_t s);


// --------------------------------------------------------------- training ---
// Workspace of one loss/gradient evaluation (train.cu).
struct TrainLayout {
    size_t inp, dinp, A[kMaxDepth], H[kMaxDepth], H16[kMaxDepth], raw, dout, d1, d2, ones, slab,
        dh[2], dl[2], Wb[kMaxDepth], WTb[kMaxDepth], total;
    size_t slab_floats;   // size of the slab region in floats
};
TrainLayout train_layout(int r, int W, int D, int od, int n);
cudaError_t run_loss_grad(const FieldsDev &fd, int field, const float *X, const int *code,
                          const float *target, int n, const float *z_table, int n_codes,
                          float *loss, float *grad_w, float *grad_z, char *ws, int *status,
                          cudaStream_t s);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, long long count, int step,
                        float lr, float b1, float b2, float eps, cudaStream_t s);
// Rewrites field `field`'s device weights (FP32 copies and, for BF16, the
// swizzled tensor-core operand) from a flat array in the host layout.
cudaError_t launch_repack(const FieldsDev &fd, int field, const float *flat, cudaStream_t s);

// ------------------------------------------------------------- batches ---
// One scene of a batched latent step, in device memory: its fields, reference
// positions and the per-scene part of the batch workspace.
struct BatchSceneDev {
    const FieldsDev *fd;       // device copy of the scene's fields
    const float *X;            // [3][n_N]
    int n_N, n_S;
    float mass, vol0, dt, inv_dt;
    int residual_g;
    float *u[2];               // g(X, z) displacement buffers (current / previous)
    float *tau6, *C9;          // [6][n_N], [9][n_N]
    float *dnext;              // [3][n_S] Gauss-Newton target
    double *z, *z_prev;        // caller's latent codes
    GridWs g;
    GridParams gp;
};
// A field evaluation of a batched step: field `field` of scene `scene` at z_n
// (zsel 0) or z_{n-1} (zsel 1) on 128-point tiles [tile0, tile1).
struct FieldBatchItem {
    int scene, field, zsel, tile0, tile1;
};
// Value kernel over a batch: CTA c runs items cta_item[c] .. cta_item[c+1]-1,
// all of width W (64, 128, 192 or 256).
cudaError_t launch_fields_batch(int W, const BatchSceneDev *scenes, const FieldBatchItem *items,
                                const int *cta_item, int nctas, int parity, int maxD,
                                int *status, cudaStream_t s);
size_t fields_batch_smem(int W, int maxD);
int fields_batch_groups(int W);

// MPM part of a batched latent step (mpm.cu): one cooperative launch.
constexpr int kMaxBatchScenes = 1024;
struct MpmBatchArgs {
    const BatchSceneDev *scenes;
    int nscenes;
    const int *n_off;          // [nscenes + 1] prefix sums of n_N
    const int *s_off;          // [nscenes + 1] prefix sums of n_S
    int parity;                // scenes' u[parity] holds g(X, z_n)
    double t0;                 // time of the call's first step
    int step;                  // step index within the call (t = t0 + step dt per scene)
    unsigned *bar;             // grid-barrier word, zero before the first launch
};
// p2g_group: threads per 4^3-block P2G tile, 64 or 128.
cudaError_t launch_mpm_batch(const MpmBatchArgs &b, int p2g_group, int *status, cudaStream_t s);

// Batched Gauss-Newton (jacobian_tc.cu): one problem per scene, each run by a
// group of CTAs of one cooperative launch.
struct GnBatchProblem {
    const FieldsDev *fd;       // device copy of the scene's fields
    const float *X;            // [3][ld] reference positions (first n are the samples)
    int n, ld;
    int cw;                    // columns per warpgroup of its tiles (32 or 64, four warpgroups)
    GnArgs gn;                 // target, z, slots (sized for the group), barrier word
};
struct GnBatchEntry {
    int problem, rank, size;
};
int jac_points_per_cta_tile(int r);
int jac_batch_cw(int r, int width, int depth);
int jac_batch_wg();
int jac_batch_points(int r, int cw);
size_t jac_tc_smem_bytes_cw(int r, int width, int depth, int CW, int NWG);
cudaError_t launch_jac_batch(const GnBatchProblem *probs, const GnBatchEntry *entries,
                             const int *cta_entry, int nctas, size_t smem, int cw, int *status,
                             cudaStream_t s);

// MPM step: one cooperative launch each (P2G, block activation, grid update
// and, for the latent step, G2P, with grid-wide barriers between the phases).  After a barrier timeout
// (NSF_ERR_ITER_CAP in *status) the workspace's control block is undefined.
struct P2gLatentArgs {
    const float *X;       // [3][n] or null (non-residual g: u is the position)
    const float *u;       // [3][n] displacement at z_n
    const float *u_prev;  // [3][n] displacement at z_{n-1}
    const float *tau6;    // [6][n]
    const float *C9;      // [9][n]
    int n;
    float mass, vol0;
    float inv_dt;
    float dt;
};
struct P2gFullArgs {
    const float *x, *v, *C, *F;   // SoA
    const float *tau6;            // [6][n] precomputed stress, or null (neo-Hookean inline)
    int n;
    float mass, vol0, dt;
    float mu, lam;
};
struct G2pFullArgs {
    float *x, *v, *C, *F;
    float *tau6;                  // [6][n] written for the next step (SVD models) or null
    int n;
    float dt;
    int model;
    float mu, lam, yield_stress, friction_deg;
};
cudaError_t launch_mpm_latent(const GridWs &g, const GridParams &gp, const P2gLatentArgs &a,
                              int n_S, double t, float *d_next, float *tap_mp, float *tap_v,
                              int *status, cudaStream_t s);
cudaError_t launch_mpm_full(const GridWs &g, const GridParams &gp, const P2gFullArgs &pa,
                            const G2pFullArgs &ga, double t, float *tap_mp, float *tap_v,
                            int *status, cudaStream_t s);
cudaError_t launch_stress(const float *F, float *tau6, int n, int model,
                          float mu, float lam, cudaStream_t s);

}  // namespace nsf
