/*
 * nsf.h -- C ABI of libnsf, a GB300 (sm_103a) implementation of one latent
 * time step of "Neural Stress Fields for Reduced-order Elastoplasticity and
 * Fracture" (Zong et al., SIGGRAPH Asia 2023), plus the full-order MLS-MPM step
 * it reduces.
 *
 * Conventions shared by every call
 * --------------------------------
 * - All particle arrays are float32, component-major ("SoA"): an array of k
 *   components for n particles is laid out [k][n], component c of particle p at
 *   index c * n + p.  3x3 matrices are stored row-major as 9 components
 *   (C_ab at component 3a + b).  Symmetric stresses use 6 components in the
 *   order (xx, yy, zz, yz, xz, xy).
 * - Latent codes z are float64 device arrays of r values.
 * - The background grid has n[0] x n[1] x n[2] nodes (each a multiple of 4),
 *   node (i, j, k) at position (i, j, k) * dx.  A particle's quadratic B-spline
 *   stencil is the 3x3x3 nodes base + {0,1,2} with base = floor(x / dx - 0.5);
 *   a particle whose stencil leaves the grid is reported as NSF_ERR_OUT_OF_GRID
 *   and skipped (never clamped).
 * - Every pointer argument named d_* is device memory owned by the caller.
 *   Nothing is retained after a call returns except inside an nsf_fields.
 * - Calls only enqueue work on the caller's CUDA stream (cudaStream_t passed as
 *   void*; NULL is the legacy default stream) and never synchronise or allocate,
 *   except nsf_create_fields / nsf_destroy_fields.
 * - Errors.  The return value reports argument errors (NSF_ERR_INVALID_ARG,
 *   NSF_ERR_WORKSPACE, NSF_ERR_UNSUPPORTED) and launch failures (NSF_ERR_CUDA).
 *   Conditions found on the device (out-of-grid particle, non-finite value,
 *   non-positive Cholesky pivot) are written asynchronously to the caller's
 *   int *d_status: the first error wins, later ones are dropped, and the
 *   computation carries on (a singular Gauss-Newton system leaves z unchanged
 *   for that iteration).  d_status must be 0 before the call for it to be read
 *   meaningfully.
 * - Workspaces.  Each stepping call takes a caller-allocated device workspace
 *   of at least the size reported by the matching *_workspace_size query.  It
 *   must be zero-filled (cudaMemsetAsync) before its first use; the library
 *   leaves it in that reusable state after every call that reported no device
 *   error.  After a device error, zero it again before reuse.  One workspace
 *   may serve any number of calls on the same scene, one call at a time.
 */
#ifndef NSF_H
#define NSF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum nsf_status {
    NSF_OK = 0,
    NSF_ERR_INVALID_ARG = -1,   /* bad pointer, size or descriptor field      */
    NSF_ERR_CUDA = -2,          /* a CUDA runtime call or launch failed       */
    NSF_ERR_OUT_OF_GRID = -3,   /* device: a particle stencil left the grid   */
    NSF_ERR_NONFINITE = -4,     /* device: NaN or Inf in a field output       */
    NSF_ERR_SINGULAR = -5,      /* device: Gauss-Newton matrix not SPD        */
    NSF_ERR_ITER_CAP = -6,      /* device: a bounded wait gave up             */
    NSF_ERR_UNSUPPORTED = -7,   /* valid request the library does not provide */
    NSF_ERR_NO_MEMORY = -8,     /* nsf_create_fields could not allocate       */
    NSF_ERR_WORKSPACE = -9      /* workspace pointer NULL or too small        */
} nsf_status;

/* Field indices: g (deformation, 3 outputs), h (Kirchhoff stress, 6), l (affine, 9). */
enum { NSF_FIELD_G = 0, NSF_FIELD_H = 1, NSF_FIELD_L = 2 };
/* Arithmetic of the field networks. */
enum { NSF_PREC_FP32 = 0, NSF_PREC_BF16 = 1 };

#define NSF_MAX_R 16
#define NSF_MAX_WIDTH 256
#define NSF_MAX_DEPTH 8

/*
 * Neural fields g(X, z), h(X, z), l(X, z)  (paper §4.2-§4.4, App. E).
 *
 * Each field is an MLP on the input [X; z] (3 + r values) with depth[f] hidden
 * layers of width[f] units, each followed by ELU(a) = a (a > 0), exp(a) - 1
 * (a <= 0), and a linear output layer of 3 (g), 6 (h) or 9 (l) units.  The raw
 * output y is de-normalised as  shift[f][o] + scale[f][o] * y[o]  (the paper
 * trains on data normalised to zero mean / unit variance, App. D); with
 * residual_g != 0 the deformation field returns X + that (x = X + MLP).
 *
 * Host weights of field f: one float32 array holding, for every linear layer
 * l = 0 .. depth[f] in order, W_l row-major [out_l][in_l] then b_l [out_l].
 *
 * precision NSF_PREC_FP32: FP32 weights and arithmetic on the CUDA cores.
 * precision NSF_PREC_BF16: weight matrices rounded to bfloat16 (nearest-even),
 *   hidden- and output-layer GEMMs on the tcgen05 tensor cores with FP32
 *   accumulation in tensor memory, activations entering them rounded to bf16;
 *   the K = 3 + r input layer, ELU and the output de-normalisation stay FP32,
 *   and biases keep ~16 significant bits (a bf16 head and tail).
 * Limits: 1 <= r <= NSF_MAX_R; width[f] a multiple of 16 in [16, NSF_MAX_WIDTH];
 * 1 <= depth[f] <= NSF_MAX_DEPTH.  BF16 widths are 64, 128, 192 or 256; the
 * tensor-core inference kernels keep a field's weights in shared memory, so a
 * BF16 fields object whose weights do not fit there (e.g. 256 wide and 5
 * deep) serves the training calls only: the inference calls (evaluation,
 * stepping, projection, integration sets, batches) return NSF_ERR_UNSUPPORTED.
 */
typedef struct nsf_fields_desc {
    int r;
    int width[3];
    int depth[3];
    int precision;
    int residual_g;
    float out_scale[3][9];
    float out_shift[3][9];
} nsf_fields_desc;

typedef struct nsf_fields nsf_fields;   /* opaque; owns device copies of the weights */

/* Validates desc, converts/packs the host weights and uploads them to the
 * current CUDA device (synchronously).  The only allocating call besides
 * nsf_destroy_fields.  *out is set only on NSF_OK. */
nsf_status nsf_create_fields(const nsf_fields_desc *desc,
                             const float *const host_weights[3],
                             nsf_fields **out);
void nsf_destroy_fields(nsf_fields *fields);
nsf_status nsf_fields_get_desc(const nsf_fields *fields, nsf_fields_desc *out);

/*
 * Evaluate the fields at n reference points (paper §5.1, network inference).
 * d_X: [3][n].  d_z: [r] (float64).  Each output may be NULL (not computed):
 *   d_x    [3][n]   g(X, z)
 *   d_tau6 [6][n]   h(X, z)
 *   d_C9   [9][n]   l(X, z)
 *   d_dxdz [3][r][n] dg_a/dz_k at component a * r + k (forward-mode chain rule)
 * Non-finite outputs set NSF_ERR_NONFINITE in *d_status (d_status may be NULL).
 */
nsf_status nsf_eval_fields(const nsf_fields *fields, const float *d_X, int n,
                           const double *d_z, float *d_x, float *d_tau6,
                           float *d_C9, float *d_dxdz, int *d_status,
                           void *stream);

/*
 * Background grid and boundary conditions (paper §3.3, grid update: "collision
 * and Dirichlet boundary conditions are handled at this stage").
 * Per step, for a node with m_i > 0:  v_i = p_i / m_i + dt * gravity, then
 *  - walls: if wall_cells > 0, a node with index < wall_cells along an axis has
 *    a negative velocity component along that axis set to 0, and a node with
 *    index > n - 1 - wall_cells a positive one;
 *  - blade (if blade_enable): nodes with |x_i - blade_x| < dx and
 *    z_i > blade_z0 + blade_vz * t move with the blade, v_i = (0, 0, blade_vz),
 *    where t is the time at the start of the step.
 * Nodes with m_i = 0 keep v_i = 0.
 */
typedef struct nsf_grid_desc {
    int n[3];
    float dx;
    float gravity[3];
    int wall_cells;
    int blade_enable;
    float blade_x, blade_z0, blade_vz;
} nsf_grid_desc;

/*
 * A reduced-order scene (paper §5): n_N integration particles, the first n_S of
 * which are the sample particles (S is a prefix of N).  d_X: [3][n_N]
 * reference positions X_p.  Uniform particle mass and initial volume V_p^0.
 */
typedef struct nsf_latent_scene {
    int n_N;
    int n_S;
    const float *d_X;
    float mass;
    float vol0;
    nsf_grid_desc grid;
} nsf_latent_scene;

/* Gauss-Newton options (paper §5.3): a fixed number of iterations (1..32, no
 * early exit) of (J^T J + damping I) dz = -J^T res, z += dz, in float64. */
typedef struct nsf_gn_opts {
    int iters;
    double damping;
} nsf_gn_opts;

/*
 * Optional device buffers receiving intermediate results of the LAST step of a
 * nsf_latent_step call (for testing and inspection).  Any member may be NULL.
 * The dense grid taps hold (m, p_x, p_y, p_z) after P2G and (v_x, v_y, v_z, m)
 * after the grid update per node, node (i, j, k) at ((i * n1 + j) * n2 + k) * 4;
 * only nodes of grid blocks the step touched are written, so zero them first.
 */
/* Stages of a latent step, for the optional stage events of nsf_latent_taps. */
enum {
    NSF_STAGE_INFERENCE = 0,   /* field networks on N (§5.1)                          */
    NSF_STAGE_MPM = 1,         /* binning, P2G with the stress force (§3.3, Eq. 5),
                                  grid update and G2P on S: one launch                */
    NSF_STAGE_GN = 2,          /* Gauss-Newton inversion (§5.3)                       */
    NSF_LATENT_STAGES = 3
};

typedef struct nsf_latent_taps {
    float *u_n;       /* [3][n_N]  raw deformation-field value at z_n: x^n - X for a
                                   residual g (the library works on displacements), x^n otherwise */
    float *u_prev;    /* [3][n_N]  the same at z_{n-1}               */
    float *tau6;      /* [6][n_N]  h(X, z_n)                         */
    float *C9;        /* [9][n_N]  l(X, z_n)                         */
    float *grid_mp;   /* [n0*n1*n2][4]                               */
    float *grid_v;    /* [n0*n1*n2][4]                               */
    float *u_next_S;  /* [3][n_S]  x^{n+1} - X on the sample particles (x^{n+1} for a
                                   non-residual g): the Gauss-Newton target   */
    double *z_iter;   /* [iters][r] z after each Gauss-Newton iteration */
    /* cudaEvent_t handles (or NULL) recorded on the call's stream right before
     * and right after each stage's launches of the last step (timing only). */
    void *ev_begin[NSF_LATENT_STAGES];
    void *ev_end[NSF_LATENT_STAGES];
} nsf_latent_taps;

/* Flags of nsf_latent_step. */
enum {
    /* The workspace still holds g(X, z_prev) from the previous nsf_latent_step
     * call on the same fields, scene and workspace, and d_z_prev is that call's
     * returned z_prev: the first step skips re-evaluating g(X, z_prev). */
    NSF_LATENT_REUSE_PREV = 1
};

nsf_status nsf_latent_workspace_size(const nsf_fields *fields,
                                     const nsf_latent_scene *scene,
                                     size_t *bytes);

/*
 * nsteps latent steps z_n -> z_{n+1} (paper §5, Fig. "latent space dynamics"):
 *  1. inference (§5.1): x^n = g(X, z_n), v^n = (g(X, z_n) - g(X, z_{n-1})) / dt,
 *     tau^n = h(X, z_n), C^n = l(X, z_n) on all integration particles;
 *  2. one MLS-MPM step (§3.3, §5.2) on N: particles binned by 4^3 grid block,
 *     P2G of mass, APIC momentum and the stress force of the node force balance
 *     (Eq. 5, MLS gradient w_ip (4/dx^2)(x_i - x_p)) summed per block in shared
 *     memory, grid update with gravity and boundary conditions, G2P of
 *     x^{n+1} = x^n + dt sum_i w_ip v_i on S;
 *  3. network inversion (§5.3, Eq. 9): opts->iters Gauss-Newton iterations from
 *     z_n on the sample particles.
 * In/out: d_z holds z_n on entry and z_{n+nsteps} on return; d_z_prev holds
 * z_{n-1} on entry (pass a copy of z_0 on the first step: zero initial
 * velocity) and z_{n+nsteps-1} on return.  g(X, z_{n-1}) is evaluated once per
 * call unless flags has NSF_LATENT_REUSE_PREV; later steps of the same call
 * reuse the previous step's g(X, z_n).  Every call leaves g(X, z_prev) of its
 * returned z_prev in the workspace for a following NSF_LATENT_REUSE_PREV call.
 * t0 is the time at the start of the first step (moves the blade).
 * taps may be NULL.
 * Reproducible: the P2G node sums are exact sums of contributions rounded
 * once to fixed point (2^-40 of the step's largest contribution bound), and
 * the BF16 path combines its Gauss-Newton sums in a fixed order, so the same
 * inputs give the same z bit for bit (the FP32 path adds float64 partials
 * with atomics, whose order may vary).
 */
nsf_status nsf_latent_step(const nsf_fields *fields,
                           const nsf_latent_scene *scene, double dt, double t0,
                           int nsteps, unsigned int flags, double *d_z,
                           double *d_z_prev,
                           const nsf_gn_opts *opts, void *d_workspace,
                           size_t workspace_bytes, int *d_status,
                           const nsf_latent_taps *taps, void *stream);

/*
 * Network inversion alone (paper §5.3, Eq. 9): Gauss-Newton on
 * min_z sum_p || g(X_p, z) - x_p ||^2 over n_S points, starting from *d_z_inout.
 * d_X_S, d_x_target: [3][n_S].  Optional outputs (may be NULL):
 * d_z_iter [iters][r] z after each iteration; d_residual [3][n_S] the final
 * g(X_p, z) - x_p.
 */
nsf_status nsf_project_workspace_size(const nsf_fields *fields, int n_S,
                                      size_t *bytes);
nsf_status nsf_project(const nsf_fields *fields, const float *d_X_S,
                       const float *d_x_target, int n_S, double *d_z_inout,
                       const nsf_gn_opts *opts, double *d_z_iter,
                       float *d_residual, void *d_workspace,
                       size_t workspace_bytes, int *d_status, void *stream);

/*
 * No-allocation form of nsf_project.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory at the point where
 * they need the inversion -- an application whose memory manager owns every
 * device allocation, a real-time loop that must never enter the CUDA
 * allocator, a plugin with nowhere to keep a workspace alive between calls.
 *
 * Same arguments and results as nsf_project minus the workspace.  The scratch
 * is a fixed array of NSF_PROJECT_STATIC_BYTES bytes inside the library, which
 * every GPU that loads the library holds until the process exits.  n_S above
 * NSF_PROJECT_STATIC_MAX_S, or a (fields, n_S) pair whose scratch would exceed
 * the array, is rejected with NSF_ERR_WORKSPACE before any device work.  The
 * call allocates nothing: it clears the part of the array it uses on the
 * caller's stream and then runs nsf_project there.  Its first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current and keeps it for the life of the process; make that first call
 * before any stream capture, and do not call it after cudaDeviceReset (or
 * anything else that destroys and recreates the device's primary context):
 * the kept address would then be stale.  All calls share the one array, so
 * calls that can overlap on the GPU (unordered streams) race with each other:
 * order them.
 */
#define NSF_PROJECT_STATIC_MAX_S 2048
#define NSF_PROJECT_STATIC_BYTES (1 << 20)
nsf_status nsf_project_static(const nsf_fields *fields, const float *d_X_S,
                              const float *d_x_target, int n_S,
                              double *d_z_inout, const nsf_gn_opts *opts,
                              double *d_z_iter, float *d_residual,
                              int *d_status, void *stream);

/*
 * Fitting a field to full-order snapshots (paper App. D): loss, gradients and
 * Adam.  Training points p = 0 .. n-1 each belong to a snapshot code[p] whose
 * latent code is row code[p] of the float32 table d_z_table [n_codes][r]
 * (learned jointly with the weights).  With y_p the de-normalised output of
 * field `field` at [X_p; z_code(p)] (X_p + MLP for a residual g) and y*_p the
 * target (d_target [out_dim][n]), the loss is the mean squared normalised
 * error  L = sum_p sum_a ((y_pa - y*_pa) / out_scale_a)^2 / (n out_dim)
 * (the training data are normalised, App. D).
 *
 * nsf_field_loss_grad writes L to *d_loss, dL/dW to d_grad_w (float32, the
 * flat host layout of that field's weights: W_l row-major then b_l per layer;
 * nsf_field_weight_count values) and, if d_grad_z is not NULL, dL/dz to
 * d_grad_z [n_codes][r] (rows of codes absent from the batch are zero).  The
 * forward pass runs in the fields' precision (BF16: every product with bf16
 * operands and FP32 accumulation on the tensor cores, the input layer in
 * FP32); the backward pass is FP32 on the forward's activations, which the
 * workspace keeps (nsf_train_workspace_size bytes).  For BF16 fields the
 * backward products of the hidden layers multiply the bf16 weights and
 * activations by the cotangent split into two bf16 parts (hi + lo, ~16
 * significant bits) on the tensor cores, FP32 accumulation.  Every product is
 * one of the library's own kernels (no BLAS library).  Every sum over points
 * (the loss, the weight and bias gradients, dL/dz) is taken in a fixed order,
 * so the same inputs give the same results bit for bit.
 * A negative code[p] sets NSF_ERR_INVALID_ARG in *d_status.
 *
 * nsf_adam_step: one Adam step (Kingma and Ba 2014; App. D) on count float32
 * parameters in place, step >= 1 (bias correction).
 *
 * nsf_fields_set_weights: replaces field `field`'s weights from a device
 * float32 array in the flat host layout (rounding the matrices to bf16 for a
 * BF16 fields object), on `stream`.  Shapes stay those of the descriptor.
 */
nsf_status nsf_field_weight_count(const nsf_fields *fields, int field, size_t *count);
nsf_status nsf_train_workspace_size(const nsf_fields *fields, int field, int n, size_t *bytes);
nsf_status nsf_field_loss_grad(const nsf_fields *fields, int field, const float *d_X,
                               const int *d_code, const float *d_target, int n,
                               const float *d_z_table, int n_codes, float *d_loss,
                               float *d_grad_w, float *d_grad_z, void *d_workspace,
                               size_t workspace_bytes, int *d_status, void *stream);
nsf_status nsf_adam_step(float *d_param, const float *d_grad, float *d_m, float *d_v,
                         size_t count, int step, float lr, float beta1, float beta2, float eps,
                         void *stream);
nsf_status nsf_fields_set_weights(nsf_fields *fields, int field, const float *d_weights,
                                  void *stream);

/*
 * Sample and integration particles (paper §5.4).  With the particle positions
 * x_p = g(X_p, z) of all n_all particles P at the latent code z:
 *   I = grid nodes in the quadratic B-spline stencil (base + {0,1,2}^3, base =
 *       floor(x_p / dx - 0.5)) of some sample particle p in S,
 *   N = every particle whose stencil contains a node of I.
 * An MPM step on N then moves the sample particles exactly as a step on all of
 * P does (§5.2).
 * d_X [3][n_all]: reference positions of P.  d_sample [n_S]: indices of S in P
 * (distinct, in [0, n_all); out-of-range ones are reported as
 * NSF_ERR_INVALID_ARG in *d_status and skipped).  d_z [r].
 * Outputs (device): d_index_out [n_all capacity]: N as indices into P, S first
 * in the given order, then the other members in increasing index; *d_count_out
 * = |N|; d_X_out (optional, [3][x_out_ld] with x_out_ld >= n_all) the
 * reference positions of N in the same order -- a nsf_latent_scene with d_X =
 * d_X_out, n_N = |N| and n_S has S as its prefix, as nsf_latent_step expects.
 * A sample particle whose stencil leaves the grid sets NSF_ERR_OUT_OF_GRID.
 * Enqueues on `stream` (workspace of nsf_integration_set_workspace_size bytes,
 * any contents; the call clears what it needs).
 */
nsf_status nsf_integration_set_workspace_size(const nsf_grid_desc *grid, int n_all,
                                              size_t *bytes);
nsf_status nsf_integration_set(const nsf_fields *fields, const nsf_grid_desc *grid,
                               const float *d_X, int n_all, const int *d_sample, int n_S,
                               const double *d_z, int *d_index_out, int *d_count_out,
                               float *d_X_out, int x_out_ld, void *d_workspace,
                               size_t workspace_bytes, int *d_status, void *stream);

/*
 * Batched latent stepping: many independent reduced-order scenes advanced
 * together, each step as a few launches for the whole batch (field inference
 * per field width, one MPM launch, one Gauss-Newton launch) instead of three
 * launches per scene.  Each scene is stepped exactly as nsf_latent_step steps it
 * (paper §5.1-§5.3).  Scenes may differ in fields (r, width, depth), particle
 * counts, grids and dt; their fields must be NSF_PREC_BF16 (the tensor-core
 * path; others give NSF_ERR_UNSUPPORTED) and at most NSF_MAX_BATCH scenes.
 *
 * An item names a scene, its fields and its caller-owned latent codes:
 * d_z [r] holds z_n on entry and z_{n+nsteps} on return, d_z_prev [r] z_{n-1}
 * and z_{n+nsteps-1}, as in nsf_latent_step.
 */
#define NSF_MAX_BATCH 1024
typedef struct nsf_latent_batch_item {
    const nsf_fields *fields;
    nsf_latent_scene scene;
    double dt;
    double *d_z;
    double *d_z_prev;
} nsf_latent_batch_item;

typedef struct nsf_latent_batch nsf_latent_batch;   /* opaque plan */

/* Workspace bytes a batch of these items needs (the items' pointers are not
 * read; only sizes, fields and grids). */
nsf_status nsf_latent_batch_workspace_size(int n_items, const nsf_latent_batch_item *items,
                                           size_t *bytes);

/*
 * Plans a batch: validates the items, lays the per-scene buffers out in the
 * caller's workspace (zero-filled before the first step, kept by the library in
 * that reusable state), splits the field evaluations into work lists of
 * 128-point tiles balanced over the SMs, and assigns each scene's Gauss-Newton
 * run a group of CTAs sized by its cost (large scenes get several dedicated
 * CTAs that combine their sums behind a per-scene barrier, small ones share
 * CTAs in longest-first order).  Allocates and uploads the plan's device
 * tables (synchronously, on the current device): the only allocating batch
 * call.  The items' fields, positions, latent codes and the workspace must
 * outlive the plan.  *out is set only on NSF_OK.
 */
nsf_status nsf_latent_batch_create(int n_items, const nsf_latent_batch_item *items,
                                   const nsf_gn_opts *opts, void *d_workspace,
                                   size_t workspace_bytes, nsf_latent_batch **out);

/*
 * Tile choices of a batch plan, for a tuner that times candidates (the
 * library's Python layer has one: paper_2310_17790_gb300.autotune).  Every
 * choice changes only the schedule and the tile shapes, not the arithmetic of
 * a scene's step beyond the order of some float sums.  0 keeps the default.
 *   gn_columns  columns per warpgroup of the Gauss-Newton tiles, 32 or 64
 *               (tiles of 128 or 256 point slots); default: 64 where every
 *               scene's operands fit in shared memory, else 32.
 *   gn_split    the cost above which a scene's Gauss-Newton run is split over
 *               a group of CTAs, as a multiple (> 0) of the per-SM share of the
 *               batch's estimated cost; default: the multiple with the smallest
 *               estimated makespan.
 *   p2g_group   threads per 4^3-block P2G tile of the MPM step, 64 or 128.
 */
typedef struct nsf_batch_tuning {
    int gn_columns;
    double gn_split;
    int p2g_group;
} nsf_batch_tuning;

/* nsf_latent_batch_create with explicit tile choices (tuning may be NULL: the
 * defaults); NSF_ERR_INVALID_ARG for a value outside the lists above or a
 * column count some scene's operands do not fit. */
nsf_status nsf_latent_batch_create_tuned(int n_items, const nsf_latent_batch_item *items,
                                         const nsf_gn_opts *opts,
                                         const nsf_batch_tuning *tuning, void *d_workspace,
                                         size_t workspace_bytes, nsf_latent_batch **out);
void nsf_latent_batch_destroy(nsf_latent_batch *batch);

/* Optional stage events of nsf_latent_step_batched (cudaEvent_t handles or
 * NULL), recorded around each stage's launches of the last step. */
typedef struct nsf_batch_events {
    void *ev_begin[NSF_LATENT_STAGES];
    void *ev_end[NSF_LATENT_STAGES];
} nsf_batch_events;

/*
 * nsteps latent steps of every scene of the batch (the steps of
 * nsf_latent_step).  t0 is the time at the start of the first step.  flags:
 * NSF_LATENT_REUSE_PREV as in nsf_latent_step (the workspace holds every
 * scene's g(X, z_prev) from the previous call on this plan).  Device-detected
 * errors of any scene go to the one status word *d_status.  Enqueues on
 * `stream` only; capturable in a CUDA graph.  events may be NULL.
 */
nsf_status nsf_latent_step_batched(const nsf_latent_batch *batch, double t0, int nsteps,
                                   unsigned int flags, int *d_status,
                                   const nsf_batch_events *events, void *stream);

/* Constitutive models of the full-order step (paper App. F; neo-Hookean is the
 * textbook tau = mu (F F^T - I) + lambda ln(J) I).  The two plastic models use
 * the Hencky (StVK, App. F.2) stress of F^E and return-map F in float64. */
enum {
    NSF_NEO_HOOKEAN = 0,
    NSF_FIXED_COROTATED = 1,
    NSF_VON_MISES = 2,        /* App. F.4, constant yield stress            */
    NSF_DRUCKER_PRAGER = 3    /* App. F.3, friction angle in degrees        */
};

typedef struct nsf_material {
    int model;
    float E, nu;
    float yield_stress;
    float friction_deg;
} nsf_material;

/* Full-order particle state, device SoA: x, v [3][n]; C, F [9][n] (F is the
 * elastic part F^E for the plastic models). */
typedef struct nsf_particles {
    int n;
    float *d_x;
    float *d_v;
    float *d_C;
    float *d_F;
    float mass;
    float vol0;
} nsf_particles;

typedef struct nsf_full_taps {
    float *grid_mp;   /* as in nsf_latent_taps, last step */
    float *grid_v;
} nsf_full_taps;

nsf_status nsf_full_workspace_size(const nsf_grid_desc *grid, int n,
                                   size_t *bytes);

/*
 * nsteps full-order explicit MLS-MPM steps (paper §3.3): stress tau(F_p), P2G
 * (mass, APIC momentum, MLS stress force; particles binned by 4^3 block and
 * summed per block in shared memory, exact fixed-point sums as in
 * nsf_latent_step), grid update, G2P of v, x, C = (4/dx^2) sum_i w_ip v_i
 * (x_i - x_p)^T, F <- (I + dt C) F, then the material's return map.  Updates
 * particles in place.  taps may be NULL.
 */
nsf_status nsf_full_step(const nsf_grid_desc *grid, const nsf_material *mat,
                         const nsf_particles *particles, double dt, double t0,
                         int nsteps, void *d_workspace, size_t workspace_bytes,
                         int *d_status, const nsf_full_taps *taps,
                         void *stream);

/*
 * Kirchhoff stress tau(F) of material `mat` at n deformation gradients (App. F
 * for the SVD-based models, the textbook neo-Hookean form for NSF_NEO_HOOKEAN),
 * with no return map: the stress the full-order step applies to a particle
 * whose (elastic) deformation gradient is F.  d_F [9][n] row-major per
 * particle, d_tau6 [6][n] in the Voigt order of this header.  The stress
 * field h is fitted to these values of full-order snapshots (App. D).
 * neo-Hookean in FP32, the SVD-based models in float64 (as the full step).
 */
nsf_status nsf_material_stress(const nsf_material *mat, const float *d_F, int n, float *d_tau6,
                               void *stream);

/* Human-readable name of a status code (static string). */
const char *nsf_status_string(int status);
/* Library ABI version (major * 10000 + minor * 100 + patch). */
int nsf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NSF_H */
