// MLS-MPM transfers (paper §3.2, §3.3, Eq. 5; §5.2 on the integration
// particles), fused into one cooperative launch per step.
//
// Phases of a launch, separated by a grid-wide barrier (all CTAs are
// co-resident; every wait is bounded in time):
//
//   bin      each particle forms its P2G record (position, m v and the matrix
//            Q = m C - dt V0 (4/dx^2) tau that carries the APIC term and the
//            MLS stress force of Eq. 5) and is binned by its 4^3-cell
//            particle block (the block of its stencil base node): a warp
//            aggregates the lanes that share a block (match, popc) into one
//            counter atomic whose old value gives each lane its slot in the
//            block's bucket; the first arrival in a block lists it.
//   P2G      each listed particle block is taken by one group of threads:
//            its particles' 27 node contributions are summed in the block's
//            6^3-node tile in shared memory (one lane per particle; in the
//            batched step a block of few particles gives each lane one
//            (particle, node) pair), then every nonzero node of the tile is
//            added once to the grid (one integer atomic per value), and the 8
//            grid blocks the tile covers are activated.
//   grid     v = p / m + dt g, walls, blade, over the activated grid blocks;
//            the sums are cleared on the way.
//   G2P      latent: x^{n+1} on the sample particles, in the same launch;
//            full-order: a separate launch (its float64 return map needs
//            far more registers than the other phases).
//
// Sums are exact.  Every node contribution is rounded once to a fixed-point
// integer (mass on a scale from the particle mass, momentum on a scale from
// this step's largest contribution bound, reduced warp by warp in the bin
// phase) and added as an integer, so a node's total does not depend on the
// order of the additions: the step is bit-for-bit reproducible.  A
// contribution of the bounding size maps to < 2^40 (2^23 such contributions
// of headroom per node in the 64-bit grid sums); the resolution is 2^-40 of
// the largest contribution, finer than float32 rounding of a sum of similar
// terms.

#include "constitutive.cuh"
#include "device_common.cuh"

namespace nsf {

namespace {

constexpr int kThreads = 256;


__device__ __forceinline__ bool cta0_thread0() { return blockIdx.x == 0 && threadIdx.x == 0; }

// First work item of this thread when items are dealt out warp by warp
// across all CTAs (warp w of every CTA before warp w + 1 of any): a set much
// smaller than the launch then still spreads over every SM instead of
// filling the first CTAs.  Consecutive items stay in one warp.
__device__ __forceinline__ int spread_index() {
    return (((threadIdx.x >> 5) * gridDim.x + blockIdx.x) << 5) + (threadIdx.x & 31);
}

// ------------------------------------------------------ particle state ----
// What P2G needs of one particle: position, m v and Q = m C - dt V0 (4/dx^2) tau
// (the APIC affine term and the MLS stress force of Eq. 5 in one matrix).
struct P2gParticle {
    float x[3], mv[3], Q[9];
};

// tau in Voigt order (xx, yy, zz, yz, xz, xy) -> row-major 3x3
__device__ __forceinline__ void voigt_to_full(const float t[6], float T[9]) {
    T[0] = t[0]; T[1] = t[5]; T[2] = t[4];
    T[3] = t[5]; T[4] = t[1]; T[5] = t[3];
    T[6] = t[4]; T[7] = t[3]; T[8] = t[2];
}

__device__ __forceinline__ void particle_position(const P2gLatentArgs &a, int p, float x[3]) {
    const int n = a.n;
    x[0] = a.u[p]; x[1] = a.u[n + p]; x[2] = a.u[2 * n + p];
    if (a.X) { x[0] += a.X[p]; x[1] += a.X[n + p]; x[2] += a.X[2 * n + p]; }
}

__device__ __forceinline__ void particle_position(const P2gFullArgs &a, int p, float x[3]) {
    const int n = a.n;
    x[0] = a.x[p]; x[1] = a.x[n + p]; x[2] = a.x[2 * n + p];
}

// Latent particles: v^n = (g(X, z_n) - g(X, z_{n-1})) / dt (§5.1), on
// displacements; tau = h(X, z_n), C = l(X, z_n).
__device__ __forceinline__ void load_particle(const P2gLatentArgs &a, float stress_k, int p,
                                              P2gParticle &q) {
    const int n = a.n;
    particle_position(a, p, q.x);
#pragma unroll
    for (int d = 0; d < 3; ++d)
        q.mv[d] = a.mass * (a.u[(size_t)d * n + p] - a.u_prev[(size_t)d * n + p]) * a.inv_dt;
    float t[6], T[9];
#pragma unroll
    for (int c = 0; c < 6; ++c) t[c] = a.tau6[(size_t)c * n + p];
    voigt_to_full(t, T);
#pragma unroll
    for (int c = 0; c < 9; ++c) q.Q[c] = a.mass * a.C9[(size_t)c * n + p] + stress_k * T[c];
}

// Neo-Hookean Kirchhoff stress (textbook): tau = mu (F F^T - I) + lambda ln(J) I.
__device__ __forceinline__ void neo_hookean_tau(const float F[9], float mu, float lam,
                                                float T[9]) {
    float J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
              F[2] * (F[3] * F[7] - F[4] * F[6]);
    float lj = lam * logf(J);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float b = F[3 * i] * F[3 * j] + F[3 * i + 1] * F[3 * j + 1] + F[3 * i + 2] * F[3 * j + 2];
            T[3 * i + j] = mu * (b - (i == j ? 1.f : 0.f)) + (i == j ? lj : 0.f);
        }
}

// Full-order particles: stored v and C; tau from F (neo-Hookean, inline) or
// the float64 stress of F^E kept from the previous G2P (SVD-based models).
__device__ __forceinline__ void load_particle(const P2gFullArgs &a, float stress_k, int p,
                                              P2gParticle &q) {
    const int n = a.n;
    particle_position(a, p, q.x);
#pragma unroll
    for (int d = 0; d < 3; ++d) q.mv[d] = a.mass * a.v[(size_t)d * n + p];
    float T[9];
    if (a.tau6) {
        float t[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) t[c] = a.tau6[(size_t)c * n + p];
        voigt_to_full(t, T);
    } else {
        float F[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) F[c] = a.F[(size_t)c * n + p];
        neo_hookean_tau(F, a.mu, a.lam, T);
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) q.Q[c] = a.mass * a.C[(size_t)c * n + p] + stress_k * T[c];
}

// Particle block (4^3 cells, by stencil base node) of position x, or -1 when
// the 3^3 stencil leaves the grid (status set).  The base nodes are those of
// bspline_axis, which the scatter uses too.
__device__ __forceinline__ int block_key(const GridWs &g, const float x[3], float inv_dx,
                                         int *status) {
    const int b0 = bspline_axis(x[0], inv_dx).base;
    const int b1 = bspline_axis(x[1], inv_dx).base;
    const int b2 = bspline_axis(x[2], inv_dx).base;
    const bool fin = finite3(x[0], x[1], x[2]);
    const bool ok = fin && b0 >= 0 && b1 >= 0 && b2 >= 0 && b0 + 2 <= g.n0 - 1 &&
                    b1 + 2 <= g.n1 - 1 && b2 + 2 <= g.n2 - 1;
    if (!ok) {
        set_status(status, fin ? NSF_ERR_OUT_OF_GRID : NSF_ERR_NONFINITE);
        return -1;
    }
    return ((b0 >> 2) * g.nb1 + (b1 >> 2)) * g.nb2 + (b2 >> 2);
}

// Contribution of particle q to node (a, b, c) of its stencil:
// (w m, w (m v + Q (x_i - x_p))).
struct Stencil {
    Axis ax, ay, az;
};

// The same with the weight w of node (a, b, c) given.
__device__ __forceinline__ float4 node_contribution_w(const P2gParticle &q, const Stencil &s,
                                                      float mass, float dx, int a, int b, int c,
                                                      float w) {
    const float dxa = ((float)a - s.ax.fx) * dx;
    const float dyb = ((float)b - s.ay.fx) * dx;
    const float dzc = ((float)c - s.az.fx) * dx;
    const float px = q.mv[0] + q.Q[0] * dxa + q.Q[1] * dyb + q.Q[2] * dzc;
    const float py = q.mv[1] + q.Q[3] * dxa + q.Q[4] * dyb + q.Q[5] * dzc;
    const float pz = q.mv[2] + q.Q[6] * dxa + q.Q[7] * dyb + q.Q[8] * dzc;
    return make_float4(w * mass, w * px, w * py, w * pz);
}

__device__ __forceinline__ float4 node_contribution(const P2gParticle &q, const Stencil &s,
                                                    float mass, float dx, int a, int b, int c) {
    return node_contribution_w(q, s, mass, dx, a, b, c, s.ax.w[a] * s.ay.w[b] * s.az.w[c]);
}

// w[i] by selects (i need not be a compile-time constant).
__device__ __forceinline__ float pick3(const float (&w)[3], int i) {
    return i == 0 ? w[0] : (i == 1 ? w[1] : w[2]);
}

// ------------------------------------------------------- fixed point ----
// A contribution of the bounding magnitude maps to < 2^kFixBits (integer
// sums of up to 2^(63 - kFixBits) of them cannot overflow).
constexpr int kFixBits = 40;
// In a particle block's tile each fixed-point value q is kept as two 32-bit
// sums, of lo = q mod 2^kLoBits (unsigned) and hi = floor(q / 2^kLoBits)
// (signed), so that it can use the native 32-bit shared-memory reductions:
// with at most kMaxTileAdds additions per node (the bucket capacity) neither
// sum can overflow, and the exact total is hi 2^kLoBits + lo.
constexpr int kLoBits = 22;
constexpr int kMaxTileAdds = kMaxBucketCap;
static_assert((long long)kMaxTileAdds * ((1ll << kLoBits) - 1) < (1ll << 32), "lo sums fit");
static_assert((long long)kMaxTileAdds << (kFixBits - kLoBits) < (1ll << 31), "hi sums fit");

// 2^(kFixBits - e) for the exponent e with bound < 2^e (a power of two, so
// scaling by it and by its reciprocal is exact); kept inside the normal range.
__device__ __forceinline__ float fix_scale(float bound) {
    int e = 0;
    if (bound > 0.f) frexpf(bound, &e);
    int k = kFixBits - e;
    k = k > 126 ? 126 : (k < -126 ? -126 : k);
    return ldexpf(1.f, k);
}

__device__ __forceinline__ unsigned long long to_fix(float v, float scale) {
    return (unsigned long long)__float2ll_rn(v * scale);
}

__device__ __forceinline__ float from_fix(unsigned long long q, float inv_scale) {
    return __ll2float_rn((long long)q) * inv_scale;
}

// Adds the fixed-point value of v (q = rint(v scale), as to_fix) to the (lo,
// hi) pair of 32-bit sums at the shared-window addresses lo_addr, hi_addr.
// The split is formed in float32 arithmetic, all exact: t = rint(v scale) is
// an integer below 2^kFixBits in magnitude, hi = floor(t / 2^kLoBits) and
// lo = t - hi 2^kLoBits, an integer in [0, 2^kLoBits) (one fused multiply-add
// with an exactly representable result).
__device__ __forceinline__ void red_shared_split(uint32_t lo_addr, uint32_t hi_addr, float v,
                                                 float scale) {
    const float t = rintf(v * scale);
    const float hf = floorf(t * (1.f / (float)(1u << kLoBits)));
    const float lf = fmaf(-hf, (float)(1u << kLoBits), t);
    const unsigned lo = (unsigned)__float2int_rn(lf);
    const int hi = __float2int_rn(hf);
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(lo_addr), "r"(lo) : "memory");
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(hi_addr), "r"(hi) : "memory");
}

// The fixed-point total of a (lo, hi) pair of sums.
__device__ __forceinline__ unsigned long long split_total(unsigned lo, int hi) {
    return (unsigned long long)(((long long)hi << kLoBits) + (long long)lo);
}

// Largest |component| of any node contribution of q: w <= 1 and
// |x_i - x_p| <= 1.5 dx per axis, so |w (m v + Q (x_i - x_p))| is at most
// max |m v| + 1.5 dx max_row sum |Q_row|.
__device__ __forceinline__ float contribution_bound(const P2gParticle &q, float dx) {
    const float mv = fmaxf(fabsf(q.mv[0]), fmaxf(fabsf(q.mv[1]), fabsf(q.mv[2])));
    float rmax = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
        rmax = fmaxf(rmax, fabsf(q.Q[3 * i]) + fabsf(q.Q[3 * i + 1]) + fabsf(q.Q[3 * i + 2]));
    return mv + 1.5f * dx * rmax;
}

// ----------------------------------------------------------- records ----
// P2G record of a particle, four float4: (x, mv0), (mv1, mv2, Q0, Q1),
// (Q2 .. Q5), (Q6, Q7, Q8, 0).
__device__ __forceinline__ void store_record(float4 *rec, int p, const P2gParticle &q) {
    float4 *r = rec + 4 * (size_t)p;
    r[0] = make_float4(q.x[0], q.x[1], q.x[2], q.mv[0]);
    r[1] = make_float4(q.mv[1], q.mv[2], q.Q[0], q.Q[1]);
    r[2] = make_float4(q.Q[2], q.Q[3], q.Q[4], q.Q[5]);
    r[3] = make_float4(q.Q[6], q.Q[7], q.Q[8], 0.f);
}

// ----------------------------------------------------------- binning ----
// Grid block (kx, ky, kz) + corner d (d = 0 .. 7 over {0,1}^3), one of the 8
// that the stencils of particle block (kx, ky, kz) reach: stamped with the
// step's epoch; the first stamp of the step lists it.
__device__ __forceinline__ void activate_grid_block(const GridWs &g, int kx, int ky, int kz,
                                                    int d, int epoch) {
    const int cx = kx + (d >> 2), cy = ky + ((d >> 1) & 1), cz = kz + (d & 1);
    if (cx >= g.nb0 || cy >= g.nb1 || cz >= g.nb2) return;
    const int gb = (cx * g.nb1 + cy) * g.nb2 + cz;
    if (atomicExch(&g.gstamp[gb], epoch) != epoch)
        g.glist[atomicAdd(&g.ctl->st[epoch & 1].n_g, 1)] = gb;
}

// Bin particle p (p < 0: no particle) of scene `tag` (0 for a single scene).
// Every lane of the warp calls (the matches below are warp-wide).  The lanes
// that share a particle block form a group: one counter atomic for the group
// (its old value plus the lane's rank in the group is the lane's bucket
// slot), and the group that finds the block empty lists it.  The step's
// contribution bound is reduced over the warp first.
template <class Args>
__device__ __forceinline__ void bin_particle(const GridWs &g, const GridParams &gp,
                                             const Args &a, float stress_k, int tag, int p,
                                             int epoch, int *status) {
    const int lane = threadIdx.x & 31;
    int key = -1;
    float bnd = 0.f;
    if (p >= 0) {
        P2gParticle q;
        load_particle(a, stress_k, p, q);
        key = block_key(g, q.x, gp.inv_dx, status);
        if (key >= 0) {
            bnd = contribution_bound(q, gp.dx);
            if (!isfinite(bnd)) {
                set_status(status, NSF_ERR_NONFINITE);
                key = -1;
            } else {
                store_record(g.rec, p, q);
            }
        }
    }
    StepCtl &st = g.ctl->st[epoch & 1];
    // the step's contribution bound: one max over the warp's lanes of each
    // scene, one atomic per scene and warp
    const unsigned same_scene = __match_any_sync(0xffffffffu, tag);
    const unsigned bmax = __reduce_max_sync(same_scene, key >= 0 ? __float_as_uint(bnd) : 0u);
    if (lane == __ffs(same_scene) - 1 && bmax) atomicMax(&st.bound, bmax);
    const unsigned long long gkey =
        key < 0 ? ~0ull : (((unsigned long long)(unsigned)tag << 32) | (unsigned)key);
    const unsigned peers = __match_any_sync(0xffffffffu, gkey);
    if (key < 0) return;
    const int leader = __ffs(peers) - 1;
    int old = 0;
    if (lane == leader) {
        old = atomicAdd(&g.bcount[key], __popc(peers));
        if (old == 0) g.plist[atomicAdd(&st.n_p, 1)] = key;
    }
    old = __shfl_sync(peers, old, leader);
    const int rank = old + __popc(peers & ((1u << lane) - 1u));
    if (rank < g.cap) g.bucket[(size_t)key * g.cap + rank] = p;
    else g.over[atomicAdd(&st.n_over, 1)] = p;
}

// --------------------------------------------------------------- P2G ----
// Scales of one step's fixed-point sums.
struct FixScales {
    float m, p, inv_m, inv_p;
};

__device__ __forceinline__ FixScales fix_scales(float mass, unsigned bound_bits) {
    FixScales s;
    s.m = fix_scale(mass);
    s.p = fix_scale(__uint_as_float(bound_bits));
    s.inv_m = 1.f / s.m;      // exact: powers of two
    s.inv_p = 1.f / s.p;
    return s;
}

__device__ __forceinline__ void unpack_record(const float4 *rec, int p, P2gParticle &q) {
    const float4 *r = rec + 4 * (size_t)p;
    const float4 r0 = __ldcg(r), r1 = __ldcg(r + 1), r2 = __ldcg(r + 2), r3 = __ldcg(r + 3);
    q.x[0] = r0.x; q.x[1] = r0.y; q.x[2] = r0.z;
    q.mv[0] = r0.w; q.mv[1] = r1.x; q.mv[2] = r1.y;
    q.Q[0] = r1.z; q.Q[1] = r1.w;
    q.Q[2] = r2.x; q.Q[3] = r2.y; q.Q[4] = r2.z; q.Q[5] = r2.w;
    q.Q[6] = r3.x; q.Q[7] = r3.y; q.Q[8] = r3.z;
}

// Tile of a particle block: its 6^3 nodes from the block's first node on,
// (m, p) as four fixed-point values per node, each a (lo, hi) pair of 32-bit
// sums.  Word w (0 .. 7: lo m, hi m, lo px, hi px, ...) of node l sits at
// w * kTileNodes + l: the lanes of one reduction touch the same word of
// different nodes, which then fall in different banks (node-major words
// would put all of them in 4 of the 32 banks).
constexpr int kTileNodes = 216;
constexpr int kTileWords = 8 * kTileNodes;

// Adds the 27 node contributions of particle p (block origin o, in nodes) to
// the tile at shared-window address `tile`.
__device__ __forceinline__ void tile_add_particle(const GridWs &g, const GridParams &gp,
                                                  float mass, const FixScales &fs, int p,
                                                  int ox, int oy, int oz, uint32_t tile,
                                                  int *status) {
    P2gParticle q;
    unpack_record(g.rec, p, q);
    const Stencil s{bspline_axis(q.x[0], gp.inv_dx), bspline_axis(q.x[1], gp.inv_dx),
                    bspline_axis(q.x[2], gp.inv_dx)};
    const int lx = s.ax.base - ox, ly = s.ay.base - oy, lz = s.az.base - oz;   // 0 .. 3
    if ((unsigned)lx > 3u || (unsigned)ly > 3u || (unsigned)lz > 3u) {
        // binned to another block than its stencil base: never expected (both
        // come from bspline_axis); recorded and skipped rather than written
        // outside the tile
        set_status(status, NSF_ERR_OUT_OF_GRID);
        return;
    }
#pragma unroll
    for (int ia = 0; ia < 3; ++ia)
#pragma unroll
        for (int ib = 0; ib < 3; ++ib)
#pragma unroll
            for (int ic = 0; ic < 3; ++ic) {
                const float4 c = node_contribution(q, s, mass, gp.dx, ia, ib, ic);
                const int l = ((lx + ia) * 6 + (ly + ib)) * 6 + (lz + ic);
                constexpr uint32_t W = 4u * kTileNodes;          // bytes per word array
                const uint32_t n = tile + 4u * (uint32_t)l;
                red_shared_split(n, n + W, c.x, fs.m);
                red_shared_split(n + 2u * W, n + 3u * W, c.y, fs.p);
                red_shared_split(n + 4u * W, n + 5u * W, c.z, fs.p);
                red_shared_split(n + 6u * W, n + 7u * W, c.w, fs.p);
            }
}

// Node nidx = 9 a + 3 b + c of particle p's stencil added to the tile: the
// work of tile_add_particle spread over 27 lanes, for blocks with few
// particles (the same contributions, so the same integer sums).
__device__ __forceinline__ void tile_add_node(const GridWs &g, const GridParams &gp, float mass,
                                              const FixScales &fs, int p, int nidx, int ox,
                                              int oy, int oz, uint32_t tile, int *status) {
    P2gParticle q;
    unpack_record(g.rec, p, q);
    const Stencil s{bspline_axis(q.x[0], gp.inv_dx), bspline_axis(q.x[1], gp.inv_dx),
                    bspline_axis(q.x[2], gp.inv_dx)};
    const int lx = s.ax.base - ox, ly = s.ay.base - oy, lz = s.az.base - oz;   // 0 .. 3
    if ((unsigned)lx > 3u || (unsigned)ly > 3u || (unsigned)lz > 3u) {
        set_status(status, NSF_ERR_OUT_OF_GRID);
        return;
    }
    const int ia = nidx / 9, ib = (nidx / 3) % 3, ic = nidx % 3;
    const float4 c = node_contribution_w(q, s, mass, gp.dx, ia, ib, ic,
                                         pick3(s.ax.w, ia) * pick3(s.ay.w, ib) * pick3(s.az.w, ic));
    const int l = ((lx + ia) * 6 + (ly + ib)) * 6 + (lz + ic);
    constexpr uint32_t W = 4u * kTileNodes;          // bytes per word array
    const uint32_t n = tile + 4u * (uint32_t)l;
    red_shared_split(n, n + W, c.x, fs.m);
    red_shared_split(n + 2u * W, n + 3u * W, c.y, fs.p);
    red_shared_split(n + 4u * W, n + 5u * W, c.z, fs.p);
    red_shared_split(n + 6u * W, n + 7u * W, c.w, fs.p);
}

// Particle p's 27 contributions straight into the grid's fixed-point sums
// (particles past their block's bucket capacity).
__device__ __forceinline__ void grid_add_particle(const GridWs &g, const GridParams &gp,
                                                  float mass, const FixScales &fs, int p) {
    P2gParticle q;
    unpack_record(g.rec, p, q);
    const Stencil s{bspline_axis(q.x[0], gp.inv_dx), bspline_axis(q.x[1], gp.inv_dx),
                    bspline_axis(q.x[2], gp.inv_dx)};
#pragma unroll
    for (int ia = 0; ia < 3; ++ia)
#pragma unroll
        for (int ib = 0; ib < 3; ++ib)
#pragma unroll
            for (int ic = 0; ic < 3; ++ic) {
                const float4 c = node_contribution(q, s, mass, gp.dx, ia, ib, ic);
                unsigned long long *n =
                    g.acc + 4 * (size_t)node_addr(g, s.ax.base + ia, s.ay.base + ib, s.az.base + ic);
                atomicAdd(n, to_fix(c.x, fs.m));
                atomicAdd(n + 1, to_fix(c.y, fs.p));
                atomicAdd(n + 2, to_fix(c.z, fs.p));
                atomicAdd(n + 3, to_fix(c.w, fs.p));
            }
}

// Group of TT threads (TT = 32: a warp; otherwise a named barrier) that runs
// the tile of one particle block at a time.
template <int TT>
__device__ __forceinline__ void group_sync(int bar_id) {
    if constexpr (TT == 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(TT) : "memory");
}

// P2G of particle block `key`: its particles' contributions summed in the
// tile (shared memory, exact integer sums), then every node of the tile with
// a nonzero sum added once to the grid (integer atomics, so the order in
// which tiles meet on their shared halo nodes does not matter).  kSparse
// (the batched step, whose scenes leave most blocks with a few particles):
// blocks of at most 4 TT / 27 particles take one lane per (particle, node)
// instead of one lane per particle (batched MPM 2.04 -> 1.74 ms; the
// single-scene latent step measured 1.4 us slower with it and keeps the
// per-particle lanes).
template <int TT, bool kSparse>
__device__ __forceinline__ void tile_block(const GridWs &g, const GridParams &gp, float mass,
                                           const FixScales &fs, int key, int epoch,
                                           unsigned long long *tile, int gt, int bar_id,
                                           int *status) {
    const int kz = key % g.nb2, t = key / g.nb2, ky = t % g.nb1, kx = t / g.nb1;
    const int ox = kx * 4, oy = ky * 4, oz = kz * 4;
    for (int i = gt; i < kTileWords / 2; i += TT) tile[i] = 0ull;
    group_sync<TT>(bar_id);
    const int np = min(__ldcg(&g.bcount[key]), g.cap);
    const int *bk = g.bucket + (size_t)key * g.cap;
    const uint32_t ts = (uint32_t)__cvta_generic_to_shared(tile);
    if (kSparse && np * 27 <= 4 * TT) {
        for (int w = gt; w < np * 27; w += TT) {
            const int k = w / 27;
            tile_add_node(g, gp, mass, fs, __ldcg(&bk[k]), w - 27 * k, ox, oy, oz, ts, status);
        }
    } else {
        for (int k = gt; k < np; k += TT)
            tile_add_particle(g, gp, mass, fs, __ldcg(&bk[k]), ox, oy, oz, ts, status);
    }
    group_sync<TT>(bar_id);
    if (gt < 8) activate_grid_block(g, kx, ky, kz, gt, epoch);
    const unsigned *tw = reinterpret_cast<const unsigned *>(tile);
    for (int l = gt; l < kTileNodes; l += TT) {
        unsigned h[8];
        unsigned any = 0u;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            h[w] = tw[w * kTileNodes + l];
            any |= h[w];
        }
        if (any == 0u) continue;
        const ulonglong2 v0 = make_ulonglong2(split_total(h[0], (int)h[1]),
                                              split_total(h[2], (int)h[3]));
        const ulonglong2 v1 = make_ulonglong2(split_total(h[4], (int)h[5]),
                                              split_total(h[6], (int)h[7]));
        // a nonzero sum lies in some particle's stencil, inside the grid
        const int i = ox + l / 36, j = oy + (l / 6) % 6, kk = oz + l % 6;
        if (i >= g.n0 || j >= g.n1 || kk >= g.n2) {
            set_status(status, NSF_ERR_OUT_OF_GRID);
            continue;
        }
        unsigned long long *n = g.acc + 4 * (size_t)node_addr(g, i, j, kk);
        if (v0.x) atomicAdd(n, v0.x);
        if (v0.y) atomicAdd(n + 1, v0.y);
        if (v1.x) atomicAdd(n + 2, v1.x);
        if (v1.y) atomicAdd(n + 3, v1.y);
    }
    group_sync<TT>(bar_id);
}

// Tiles of one CTA: kThreads / TT groups, each with its own tile.
template <int TT>
struct __align__(16) TileSmem {
    unsigned long long tile[kThreads / TT][kTileWords / 2];   // 8 word arrays per tile
};

// P2G phase of a single scene: every listed particle block's tile, then the
// overflow particles.
template <int TT, bool kSparse>
__device__ void phase_p2g(const GridWs &g, const GridParams &gp, float mass, int epoch,
                          TileSmem<TT> &sm, int *status) {
    const StepCtl &st = g.ctl->st[epoch & 1];
    constexpr int kGroups = kThreads / TT;
    const int grp = threadIdx.x / TT, gt = threadIdx.x % TT;
    const int n_p = __ldcg(&st.n_p), n_over = __ldcg(&st.n_over);
    const FixScales fs = fix_scales(mass, __ldcg(&st.bound));
    // group w of CTA c takes blocks w * gridDim.x + c, + all groups: a short
    // list still spreads over every SM
    for (int q = grp * gridDim.x + blockIdx.x; q < n_p; q += kGroups * gridDim.x)
        tile_block<TT, kSparse>(g, gp, mass, fs, __ldcg(&g.plist[q]), epoch, sm.tile[grp], gt, 1 + grp,
                       status);
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n_over; u += gridDim.x * blockDim.x)
        grid_add_particle(g, gp, mass, fs, __ldcg(&g.over[u]));
}

// --------------------------------------------------------------- grid ----
// Grid update of node l (0 .. 63) of grid block gb from its (m, p) = a:
// v = p / m + dt g, walls, blade, written with m to g.vel (§3.3).  Nodes
// with m = 0 get v = 0 and no boundary condition.
__device__ __forceinline__ void grid_node_update(const GridWs &g, const GridParams &gp, float dt,
                                                 double blade_z, int gb, int l, float4 a,
                                                 float *tap_mp, float *tap_v) {
    const int lx = l >> 4, ly = (l >> 2) & 3, lz = l & 3;
    const int bz = gb % g.nb2, tt = gb / g.nb2, by = tt % g.nb1, bx = tt / g.nb1;
    const int i = bx * 4 + lx, j = by * 4 + ly, k = bz * 4 + lz;
    float4 v = make_float4(0.f, 0.f, 0.f, a.x);
    if (a.x > 0.f) {
        const float im = 1.f / a.x;
        v.x = a.y * im + dt * gp.gx;
        v.y = a.z * im + dt * gp.gy;
        v.z = a.w * im + dt * gp.gz;
        const int wc = gp.wall_cells;
        if (wc > 0) {
            if ((i < wc && v.x < 0.f) || (i > g.n0 - 1 - wc && v.x > 0.f)) v.x = 0.f;
            if ((j < wc && v.y < 0.f) || (j > g.n1 - 1 - wc && v.y > 0.f)) v.y = 0.f;
            if ((k < wc && v.z < 0.f) || (k > g.n2 - 1 - wc && v.z > 0.f)) v.z = 0.f;
        }
        if (gp.blade_enable) {
            const float xi = (float)i * gp.dx;
            const double zi = (double)k * (double)gp.dx;
            if (fabsf(xi - gp.blade_x) < gp.dx && zi > blade_z) {
                v.x = 0.f;
                v.y = 0.f;
                v.z = gp.blade_vz;
            }
        }
    }
    g.vel[gb * 64 + l] = v;
    const size_t nat = (((size_t)i * g.n1 + j) * g.n2 + k) * 4;
    if (tap_mp) *reinterpret_cast<float4 *>(tap_mp + nat) = a;
    if (tap_v) *reinterpret_cast<float4 *>(tap_v + nat) = v;
}

// The fixed-point sums of node l of grid block gb as floats; the sums are
// cleared for the next step on the way.
__device__ __forceinline__ float4 take_node_sums(const GridWs &g, const FixScales &fs, int gb,
                                                 int l) {
    ulonglong2 *n = reinterpret_cast<ulonglong2 *>(g.acc + 4 * ((size_t)gb * 64 + l));
    const ulonglong2 v0 = __ldcg(n), v1 = __ldcg(n + 1);
    if ((v0.x | v0.y | v1.x | v1.y) != 0ull) {
        n[0] = make_ulonglong2(0ull, 0ull);
        n[1] = make_ulonglong2(0ull, 0ull);
    }
    return make_float4(from_fix(v0.x, fs.inv_m), from_fix(v0.y, fs.inv_p),
                       from_fix(v1.x, fs.inv_p), from_fix(v1.y, fs.inv_p));
}

// Grid blocks a thread updates per pass: their index and node loads are
// issued together, so a thread has kGridUnroll memory chains in flight
// instead of one.
constexpr int kGridUnroll = 4;

__device__ void phase_grid(const GridWs &g, const GridParams &gp, float mass, float dt, double t,
                           const StepCtl &st, float *tap_mp, float *tap_v) {
    const int ngb = __ldcg(&st.n_g);
    const FixScales fs = fix_scales(mass, __ldcg(&st.bound));
    const int per = blockDim.x >> 6;                 // grid blocks per CTA pass
    const int sub = threadIdx.x >> 6, l = threadIdx.x & 63;
    const int stride = gridDim.x * per;
    const double blade_z = (double)gp.blade_z0 + (double)gp.blade_vz * t;
    for (int i0 = sub * gridDim.x + blockIdx.x; i0 < ngb; i0 += kGridUnroll * stride) {
        int gb[kGridUnroll];
        float4 a[kGridUnroll];
#pragma unroll
        for (int u = 0; u < kGridUnroll; ++u) {
            const int idx = i0 + u * stride;
            gb[u] = idx < ngb ? __ldcg(&g.glist[idx]) : -1;
        }
#pragma unroll
        for (int u = 0; u < kGridUnroll; ++u)
            if (gb[u] >= 0) a[u] = take_node_sums(g, fs, gb[u], l);
#pragma unroll
        for (int u = 0; u < kGridUnroll; ++u)
            if (gb[u] >= 0) grid_node_update(g, gp, dt, blade_z, gb[u], l, a[u], tap_mp, tap_v);
    }
}

// Bin phase of a single scene.
template <class Args>
__device__ void phase_bin(const GridWs &g, const GridParams &gp, const Args &a, float stress_k,
                          int epoch, int *status) {
    const int n = a.n;
    const int stride = gridDim.x * blockDim.x;
    // the loop bound is uniform across each warp (the match in bin_particle)
    for (int base = spread_index() & ~31; base < n; base += stride) {
        const int p = base + (threadIdx.x & 31);
        bin_particle(g, gp, a, stress_k, 0, p < n ? p : -1, epoch, status);
    }
}

// Clears this step's bucket counters (its listed particle blocks) for the
// next step.
__device__ void clear_bins(const GridWs &g, const StepCtl &st) {
    const int n_p = __ldcg(&st.n_p);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_p; q += gridDim.x * blockDim.x)
        g.bcount[__ldcg(&g.plist[q])] = 0;
}

// Start of a step's MPM launch: the step's epoch and, by one thread, the
// other counter set cleared (no launch of this step uses it).
__device__ __forceinline__ int begin_step(const GridWs &g) {
    const int epoch = __ldcg(&g.ctl->epoch) + 1;
    if (cta0_thread0()) g.ctl->st[(epoch & 1) ^ 1] = StepCtl{0, 0, 0, 0u};
    return epoch;
}

// bin | barrier | P2G tiles | barrier | grid update.  Returns false if a
// barrier timed out.  After the first barrier (every CTA has read the old
// epoch) CTA 0 publishes the step's epoch, which later launches of the step
// read.
template <int TT, bool kSparse, class Args>
__device__ bool bin_p2g_grid(const GridWs &g, const GridParams &gp, const Args &a, double t,
                             int epoch, float *tap_mp, float *tap_v, int *status) {
    __shared__ TileSmem<TT> sm;
    const float stress_k = -a.dt * a.vol0 * 4.f * gp.inv_dx * gp.inv_dx;
    phase_bin(g, gp, a, stress_k, epoch, status);
    if (!grid_barrier(&g.ctl->bar, status)) return false;
    if (cta0_thread0()) g.ctl->epoch = epoch;
    const StepCtl &st = g.ctl->st[epoch & 1];
    phase_p2g<TT, kSparse>(g, gp, a.mass, epoch, sm, status);
    if (!grid_barrier(&g.ctl->bar, status)) return false;
    phase_grid(g, gp, a.mass, a.dt, t, st, tap_mp, tap_v);
    return true;
}

// ---------------------------------------------------------------- G2P ----
// Latent G2P on the sample particles (§5.2): only x^{n+1} is needed.  Writes
// the displacement target d = u_n + dt v_p (x^{n+1} - X for a residual g).
__device__ __forceinline__ void g2p_latent_particle(const GridWs &g, const GridParams &gp,
                                                    const float *X, const float *u, int ld,
                                                    int n_S, float dt, float *d_next, int p,
                                                    int *status) {
    {
        const float u0 = u[p], u1 = u[ld + p], u2 = u[2 * ld + p];
        float x0 = u0, x1 = u1, x2 = u2;
        if (X) { x0 += X[p]; x1 += X[ld + p]; x2 += X[2 * ld + p]; }
        const Axis ax = bspline_axis(x0, gp.inv_dx), ay = bspline_axis(x1, gp.inv_dx),
                   az = bspline_axis(x2, gp.inv_dx);
        const bool ok = ax.base >= 0 && ay.base >= 0 && az.base >= 0 && ax.base + 2 <= g.n0 - 1 &&
                        ay.base + 2 <= g.n1 - 1 && az.base + 2 <= g.n2 - 1;
        float vx = 0.f, vy = 0.f, vz = 0.f;
        if (ok) {
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float w = ax.w[a] * ay.w[b] * az.w[c];
                        const float4 v = __ldcg(&g.vel[node_addr(g, ax.base + a, ay.base + b, az.base + c)]);
                        vx = fmaf(w, v.x, vx);
                        vy = fmaf(w, v.y, vy);
                        vz = fmaf(w, v.z, vz);
                    }
        } else {
            set_status(status, NSF_ERR_OUT_OF_GRID);
        }
        d_next[p] = fmaf(dt, vx, u0);
        d_next[n_S + p] = fmaf(dt, vy, u1);
        d_next[2 * n_S + p] = fmaf(dt, vz, u2);
    }
}

__device__ void phase_g2p_latent(const GridWs &g, const GridParams &gp, const float *X,
                                 const float *u, int ld, int n_S, float dt, float *d_next,
                                 int *status) {
    for (int p = spread_index(); p < n_S; p += gridDim.x * blockDim.x)
        g2p_latent_particle(g, gp, X, u, ld, n_S, dt, d_next, p, status);
}

// Full-order G2P (§3.3): v, x, C = (4/dx^2) sum w v_i (x_i - x_p)^T and the
// deformation-gradient update F <- (I + dt C) F (MLS velocity gradient), then
// for the SVD-based models the float64 return map and the stress of F^E.
__device__ void phase_g2p_full(const GridWs &g, const GridParams &gp, const G2pFullArgs &a,
                               int *status) {
    const int n = a.n;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float x0 = a.x[p], x1 = a.x[n + p], x2 = a.x[2 * n + p];
        const Axis ax = bspline_axis(x0, gp.inv_dx), ay = bspline_axis(x1, gp.inv_dx),
                   az = bspline_axis(x2, gp.inv_dx);
        const bool ok = ax.base >= 0 && ay.base >= 0 && az.base >= 0 && ax.base + 2 <= g.n0 - 1 &&
                        ay.base + 2 <= g.n1 - 1 && az.base + 2 <= g.n2 - 1;
        if (!ok) {
            set_status(status, NSF_ERR_OUT_OF_GRID);
            continue;
        }
        float v[3] = {0.f, 0.f, 0.f};
        float B[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ia = 0; ia < 3; ++ia) {
            const float dxa = ((float)ia - ax.fx) * gp.dx;
#pragma unroll
            for (int ib = 0; ib < 3; ++ib) {
                const float dyb = ((float)ib - ay.fx) * gp.dx;
#pragma unroll
                for (int ic = 0; ic < 3; ++ic) {
                    const float dzc = ((float)ic - az.fx) * gp.dx;
                    const float w = ax.w[ia] * ay.w[ib] * az.w[ic];
                    const float4 vi = __ldcg(&g.vel[node_addr(g, ax.base + ia, ay.base + ib, az.base + ic)]);
                    const float wv[3] = {w * vi.x, w * vi.y, w * vi.z};
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        v[r] += wv[r];
                        B[3 * r + 0] = fmaf(wv[r], dxa, B[3 * r + 0]);
                        B[3 * r + 1] = fmaf(wv[r], dyb, B[3 * r + 1]);
                        B[3 * r + 2] = fmaf(wv[r], dzc, B[3 * r + 2]);
                    }
                }
            }
        }
        const float Dinv = 4.f * gp.inv_dx * gp.inv_dx;
        float C[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) C[c] = Dinv * B[c];
        float F[9], Fn[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) F[c] = a.F[(size_t)c * n + p];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                Fn[3 * i + j] = F[3 * i + j] + a.dt * (C[3 * i] * F[j] + C[3 * i + 1] * F[3 + j] +
                                                       C[3 * i + 2] * F[6 + j]);
        if (a.tau6) {
            double Fd[9], t6[6];
#pragma unroll
            for (int c = 0; c < 9; ++c) Fd[c] = (double)Fn[c];
            return_map_and_stress(a.model, Fd, a.mu, a.lam, a.yield_stress, a.friction_deg, true, t6);
            bool fin = true;
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                Fn[c] = (float)Fd[c];
                fin &= isfinite(Fn[c]);
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) a.tau6[(size_t)c * n + p] = (float)t6[c];
            if (!fin) set_status(status, NSF_ERR_NONFINITE);
        }
        a.x[p] = fmaf(a.dt, v[0], x0);
        a.x[n + p] = fmaf(a.dt, v[1], x1);
        a.x[2 * n + p] = fmaf(a.dt, v[2], x2);
#pragma unroll
        for (int r = 0; r < 3; ++r) a.v[(size_t)r * n + p] = v[r];
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            a.C[(size_t)c * n + p] = C[c];
            a.F[(size_t)c * n + p] = Fn[c];
        }
    }
}

// ------------------------------------------------------------- kernels ---
// Threads per tile group: 64 for the sparse latent sets (a few particles per
// block: four small tiles in flight per CTA), 128 for the dense full-order
// slab (up to 512 particles per block).  Each tile takes 6.9 KB of shared
// memory.
constexpr int kTileThreadsLatent = 64;
constexpr int kTileThreadsFull = 128;

__global__ void __launch_bounds__(kThreads)
k_mpm_latent(GridWs g, GridParams gp, P2gLatentArgs a, int n_S, double t, float *d_next,
             float *tap_mp, float *tap_v, int *status) {
    pdl_wait();
    const int epoch = begin_step(g);
    if (!bin_p2g_grid<kTileThreadsLatent, false>(g, gp, a, t, epoch, tap_mp, tap_v, status)) return;
    if (!grid_barrier(&g.ctl->bar, status)) return;
    phase_g2p_latent(g, gp, a.X, a.u, a.n, n_S, a.dt, d_next, status);
    clear_bins(g, g.ctl->st[epoch & 1]);
}

__global__ void __launch_bounds__(kThreads)
k_mpm_full(GridWs g, GridParams gp, P2gFullArgs a, double t, float *tap_mp, float *tap_v,
           int *status) {
    const int epoch = begin_step(g);
    bin_p2g_grid<kTileThreadsFull, false>(g, gp, a, t, epoch, tap_mp, tap_v, status);
}

// Full-order G2P, one thread per particle; it also clears the step's bucket
// counters (the MPM launch published the step's epoch).
__global__ void __launch_bounds__(kThreads)
k_g2p_full(GridWs g, GridParams gp, G2pFullArgs a, int *status) {
    phase_g2p_full(g, gp, a, status);
    clear_bins(g, g.ctl->st[__ldcg(&g.ctl->epoch) & 1]);
}

// Kirchhoff stress of F (no return map) for the SVD-based models, float64.
__global__ void __launch_bounds__(256)
k_stress(const float *__restrict__ F, float *tau6, int n, int model, float mu, float lam) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double Fd[9], t6[6];
#pragma unroll
    for (int c = 0; c < 9; ++c) Fd[c] = (double)F[(size_t)c * n + p];
    return_map_and_stress(model, Fd, mu, lam, 0.0, 0.0, false, t6);
#pragma unroll
    for (int c = 0; c < 6; ++c) tau6[(size_t)c * n + p] = (float)t6[c];
}

// ------------------------------------------------------------- batches ---
// Largest s with off[s] <= q (off ascending, off[0] = 0 <= q < off[ns]).
__device__ __forceinline__ int find_scene(const int *off, int ns, int q) {
    int lo = 0, hi = ns;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= q) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Exclusive prefix sums off[0 .. ns] of v(s), s < ns, over the CTA (ns <=
// kMaxBatchScenes); every thread calls.
template <class F>
__device__ void block_offsets(int ns, int *off, F v) {
    __shared__ int wsum[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (ns + kThreads - 1) / kThreads;
    const int s0 = threadIdx.x * per;
    int loc[kMaxBatchScenes / kThreads];
    int tot = 0;
#pragma unroll
    for (int k = 0; k < kMaxBatchScenes / kThreads; ++k) {
        const int sc = s0 + k;
        loc[k] = (k < per && sc < ns) ? v(sc) : 0;
        tot += loc[k];
    }
    int x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int run = x - tot, all = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
        if (w < warp) run += wsum[w];
        all += wsum[w];
    }
#pragma unroll
    for (int k = 0; k < kMaxBatchScenes / kThreads; ++k) {
        const int sc = s0 + k;
        if (k < per && sc < ns) off[sc] = run;
        run += loc[k];
    }
    if (threadIdx.x == 0) off[ns] = all;
    __syncthreads();
}

__device__ __forceinline__ P2gLatentArgs latent_args(const BatchSceneDev &sc, int parity) {
    P2gLatentArgs a;
    a.X = sc.residual_g ? sc.X : nullptr;
    a.u = sc.u[parity];
    a.u_prev = sc.u[parity ^ 1];
    a.tau6 = sc.tau6;
    a.C9 = sc.C9;
    a.n = sc.n_N;
    a.mass = sc.mass;
    a.vol0 = sc.vol0;
    a.inv_dt = sc.inv_dt;
    a.dt = sc.dt;
    return a;
}



// The MPM part of a batched latent step: every phase runs over all scenes at
// once (a flat index over the scenes' particles, listed particle blocks,
// active grid blocks and sample particles), with one grid barrier between
// phases for the whole batch.  Each scene keeps its own counters, epoch,
// buckets and fixed-point scales.
template <int TT>
__global__ void __launch_bounds__(kThreads, 4)
k_mpm_batch(MpmBatchArgs b, int *status) {
    __shared__ int off[kMaxBatchScenes + 1];
    __shared__ int s_epoch[kMaxBatchScenes];
    __shared__ TileSmem<TT> sm;
    constexpr int kGroups = kThreads / TT;
    const int ns = b.nscenes;
    const int stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    // every scene's step epoch, read before the first barrier; block 0 clears
    // each scene's other counter set
    for (int sc = threadIdx.x; sc < ns; sc += blockDim.x) {
        s_epoch[sc] = __ldcg(&b.scenes[sc].g.ctl->epoch) + 1;
        if (blockIdx.x == 0) b.scenes[sc].g.ctl->st[(s_epoch[sc] & 1) ^ 1] = StepCtl{0, 0, 0, 0u};
    }
    __syncthreads();
    // bin
    const int total_N = __ldg(&b.n_off[ns]);
    for (int base = spread_index() & ~31; base < total_N; base += stride) {
        const int q = base + lane;
        const int sidx = q < total_N ? find_scene(b.n_off, ns, q) : 0;
        const BatchSceneDev &sc = b.scenes[sidx];
        const float stress_k = -sc.dt * sc.vol0 * 4.f * sc.gp.inv_dx * sc.gp.inv_dx;
        bin_particle(sc.g, sc.gp, latent_args(sc, b.parity), stress_k, sidx,
                     q < total_N ? q - __ldg(&b.n_off[sidx]) : -1, s_epoch[sidx], status);
    }
    if (!grid_barrier(b.bar, status)) return;
    if (blockIdx.x == 0)                         // every CTA has read them
        for (int sc = threadIdx.x; sc < ns; sc += blockDim.x) b.scenes[sc].g.ctl->epoch = s_epoch[sc];
    // P2G: tiles of every scene's listed particle blocks, then overflow particles
    block_offsets(ns, off, [&](int sc) {
        return __ldcg(&b.scenes[sc].g.ctl->st[s_epoch[sc] & 1].n_p);
    });
    {
        const int grp = threadIdx.x / TT, gt = threadIdx.x % TT;
        const int nblk = off[ns];
        for (int q = grp * gridDim.x + blockIdx.x; q < nblk; q += kGroups * gridDim.x) {
            const int sidx = find_scene(off, ns, q);
            const BatchSceneDev &sc = b.scenes[sidx];
            const StepCtl &st = sc.g.ctl->st[s_epoch[sidx] & 1];
            const FixScales fs = fix_scales(sc.mass, __ldcg(&st.bound));
            tile_block<TT, true>(sc.g, sc.gp, sc.mass, fs, __ldcg(&sc.g.plist[q - off[sidx]]),
                           s_epoch[sidx], sm.tile[grp], gt, 1 + grp, status);
        }
    }
    block_offsets(ns, off, [&](int sc) {
        return __ldcg(&b.scenes[sc].g.ctl->st[s_epoch[sc] & 1].n_over);
    });
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < off[ns]; q += stride) {
        const int sidx = find_scene(off, ns, q);
        const BatchSceneDev &sc = b.scenes[sidx];
        const FixScales fs = fix_scales(sc.mass, __ldcg(&sc.g.ctl->st[s_epoch[sidx] & 1].bound));
        grid_add_particle(sc.g, sc.gp, sc.mass, fs, __ldcg(&sc.g.over[q - off[sidx]]));
    }
    if (!grid_barrier(b.bar, status)) return;
    // grid update
    block_offsets(ns, off, [&](int sc) {
        return __ldcg(&b.scenes[sc].g.ctl->st[s_epoch[sc] & 1].n_g);
    });
    {
        const int per = blockDim.x >> 6;
        const int sub = threadIdx.x >> 6, l = threadIdx.x & 63;
        const int nblk = off[ns], gstride = gridDim.x * per;
        for (int u0 = sub * gridDim.x + blockIdx.x; u0 < nblk; u0 += kGridUnroll * gstride) {
            int sidx[kGridUnroll], gb[kGridUnroll];
            float4 a[kGridUnroll];
#pragma unroll
            for (int k = 0; k < kGridUnroll; ++k) {
                const int u = u0 + k * gstride;
                sidx[k] = -1;
                if (u < nblk) {
                    sidx[k] = find_scene(off, ns, u);
                    gb[k] = __ldcg(&b.scenes[sidx[k]].g.glist[u - off[sidx[k]]]);
                }
            }
#pragma unroll
            for (int k = 0; k < kGridUnroll; ++k)
                if (sidx[k] >= 0) {
                    const BatchSceneDev &sc = b.scenes[sidx[k]];
                    const FixScales fs =
                        fix_scales(sc.mass, __ldcg(&sc.g.ctl->st[s_epoch[sidx[k]] & 1].bound));
                    a[k] = take_node_sums(sc.g, fs, gb[k], l);
                }
#pragma unroll
            for (int k = 0; k < kGridUnroll; ++k) {
                if (sidx[k] < 0) continue;
                const BatchSceneDev &sc = b.scenes[sidx[k]];
                const double t = b.t0 + (double)b.step * (double)sc.dt;
                const double blade_z = (double)sc.gp.blade_z0 + (double)sc.gp.blade_vz * t;
                grid_node_update(sc.g, sc.gp, sc.dt, blade_z, gb[k], l, a[k], nullptr, nullptr);
            }
        }
    }
    if (!grid_barrier(b.bar, status)) return;
    // G2P on the sample particles
    const int total_S = __ldg(&b.s_off[ns]);
    for (int q = spread_index(); q < total_S; q += stride) {
        const int sidx = find_scene(b.s_off, ns, q);
        const BatchSceneDev &sc = b.scenes[sidx];
        g2p_latent_particle(sc.g, sc.gp, sc.residual_g ? sc.X : nullptr, sc.u[b.parity], sc.n_N,
                            sc.n_S, sc.dt, sc.dnext, q - __ldg(&b.s_off[sidx]), status);
    }
    // clear every scene's bucket counters
    block_offsets(ns, off, [&](int sc) {
        return __ldcg(&b.scenes[sc].g.ctl->st[s_epoch[sc] & 1].n_p);
    });
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < off[ns]; q += stride) {
        const int sidx = find_scene(off, ns, q);
        const GridWs &g = b.scenes[sidx].g;
        g.bcount[__ldcg(&g.plist[q - off[sidx]])] = 0;
    }
}

// CTAs per SM of the latent MPM launch: its phases are separated by grid
// barriers over a few thousand particles, and one CTA per SM made the stage
// 7 % faster than four (cheaper barriers; the work does not fill more).
#ifndef NSF_LATENT_MPM_CTAS_PER_SM
#define NSF_LATENT_MPM_CTAS_PER_SM 1
#endif
template <class K>
int coop_grid(K kernel, int cap = 4) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kThreads, 0);
    if (per < 1) per = 1;
    if (per > cap) per = cap;
    return sms * per;
}

// A cooperative launch; pdl: also programmatic stream serialisation (the
// kernel calls pdl_wait() first).
template <class K, class... A>
cudaError_t launch_coop(K kernel, int grid, cudaStream_t s, bool pdl, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

// Kirchhoff stress of F for the neo-Hookean model, FP32 (as P2G computes it).
__global__ void __launch_bounds__(256)
k_stress_neo_hookean(const float *__restrict__ F, float *tau6, int n, float mu, float lam) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float Fp[9], T[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) Fp[c] = F[(size_t)c * n + p];
    neo_hookean_tau(Fp, mu, lam, T);
    const float t6[6] = {T[0], T[4], T[8], T[5], T[2], T[1]};   // xx yy zz yz xz xy
#pragma unroll
    for (int c = 0; c < 6; ++c) tau6[(size_t)c * n + p] = t6[c];
}

// ------------------------------------------------------------ launchers ---
cudaError_t launch_stress(const float *F, float *tau6, int n, int model, float mu, float lam,
                          cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (model == NSF_NEO_HOOKEAN)
        k_stress_neo_hookean<<<(n + 255) / 256, 256, 0, s>>>(F, tau6, n, mu, lam);
    else
        k_stress<<<(n + 255) / 256, 256, 0, s>>>(F, tau6, n, model, mu, lam);
    return cudaGetLastError();
}

cudaError_t launch_mpm_latent(const GridWs &g, const GridParams &gp, const P2gLatentArgs &a,
                              int n_S, double t, float *d_next, float *tap_mp, float *tap_v,
                              int *status, cudaStream_t s) {
    static const int grid = coop_grid(k_mpm_latent, NSF_LATENT_MPM_CTAS_PER_SM);
    return launch_coop(k_mpm_latent, grid, s, true, g, gp, a, n_S, t, d_next, tap_mp,
                       tap_v, status);
}

cudaError_t launch_mpm_batch(const MpmBatchArgs &b, int p2g_group, int *status, cudaStream_t s) {
    if (b.nscenes < 1 || b.nscenes > kMaxBatchScenes) return cudaErrorInvalidValue;
    if (p2g_group == 128) {
        static const int grid = coop_grid(k_mpm_batch<128>);
        return launch_coop(k_mpm_batch<128>, grid, s, false, b, status);
    }
    if (p2g_group != 64) return cudaErrorInvalidValue;
    static const int grid = coop_grid(k_mpm_batch<64>);
    return launch_coop(k_mpm_batch<64>, grid, s, false, b, status);
}

cudaError_t launch_mpm_full(const GridWs &g, const GridParams &gp, const P2gFullArgs &pa,
                            const G2pFullArgs &ga, double t, float *tap_mp, float *tap_v,
                            int *status, cudaStream_t s) {
    static const int grid = coop_grid(k_mpm_full);
    cudaError_t e = launch_coop(k_mpm_full, grid, s, false, g, gp, pa, t, tap_mp, tap_v,
                                status);
    if (e != cudaSuccess) return e;
    k_g2p_full<<<(ga.n + kThreads - 1) / kThreads, kThreads, 0, s>>>(g, gp, ga, status);
    return cudaGetLastError();
}

}  // namespace nsf
