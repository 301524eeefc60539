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
//            block's bucket.  The first arrival in a block lists it and
//            stamps the 8 grid blocks its stencils can reach.
//   P2G +    each active grid block is owned by one group of threads, which
//   grid     gathers the particles of the 8 particle blocks that reach it
//            from their buckets, accumulates their contributions to its 64
//            nodes in shared memory, then turns each node's (m, p) into
//            v = p / m + dt g with the walls and the blade, and writes v
//            once.  No grid value goes through a global atomic.
//   G2P      latent: x^{n+1} on the sample particles, in the same launch;
//            full-order: a separate launch (its float64 return map needs
//            far more registers than the other phases).
//
// Sums are exact.  Every node contribution is rounded once to a 64-bit fixed
// point number (mass on a scale from the particle mass, momentum on a scale
// from this step's largest contribution bound, reduced warp by warp in the
// bin phase) and added as an integer, so a node's total does not depend on
// the order of the additions: the step is bit-for-bit reproducible.  A
// contribution of the bounding size maps to < 2^44, leaving 2^19 such
// contributions of headroom per node; the resolution is 2^-44 of the largest
// contribution (a smaller one than float32 rounding of a sum of similar
// terms gives).

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
// the 3^3 stencil leaves the grid (status set).
__device__ __forceinline__ int block_key(const GridWs &g, const float x[3], float inv_dx,
                                         int *status) {
    const int b0 = __float2int_rd(x[0] * inv_dx - 0.5f);
    const int b1 = __float2int_rd(x[1] * inv_dx - 0.5f);
    const int b2 = __float2int_rd(x[2] * inv_dx - 0.5f);
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

__device__ __forceinline__ float4 node_contribution(const P2gParticle &q, const Stencil &s,
                                                    float mass, float dx, int a, int b, int c) {
    const float dxa = ((float)a - s.ax.fx) * dx;
    const float dyb = ((float)b - s.ay.fx) * dx;
    const float dzc = ((float)c - s.az.fx) * dx;
    const float w = s.ax.w[a] * s.ay.w[b] * s.az.w[c];
    const float px = q.mv[0] + q.Q[0] * dxa + q.Q[1] * dyb + q.Q[2] * dzc;
    const float py = q.mv[1] + q.Q[3] * dxa + q.Q[4] * dyb + q.Q[5] * dzc;
    const float pz = q.mv[2] + q.Q[6] * dxa + q.Q[7] * dyb + q.Q[8] * dzc;
    return make_float4(w * mass, w * px, w * py, w * pz);
}

// ------------------------------------------------------- fixed point ----
// A contribution of the bounding magnitude maps to < 2^kFixBits (integer
// sums of up to 2^(63 - kFixBits) of them cannot overflow).
constexpr int kFixBits = 44;

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
// Stamps the grid blocks (kx..kx+1, ky..ky+1, kz..kz+1) that the stencils of
// particle block `key` reach; the first stamp of this step lists the block.
__device__ __forceinline__ void activate_grid_blocks(const GridWs &g, int key, int epoch,
                                                     StepCtl &st) {
    const int kz = key % g.nb2, t = key / g.nb2, ky = t % g.nb1, kx = t / g.nb1;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int cx = kx + (d >> 2), cy = ky + ((d >> 1) & 1), cz = kz + (d & 1);
        if (cx >= g.nb0 || cy >= g.nb1 || cz >= g.nb2) continue;
        const int gb = (cx * g.nb1 + cy) * g.nb2 + cz;
        if (atomicExch(&g.gstamp[gb], epoch) != epoch) g.glist[atomicAdd(&st.n_g, 1)] = gb;
    }
}

// Bin particle p (p < 0: no particle) of scene `tag` (0 for a single scene).
// Every lane of the warp calls (the match below is warp-wide).  The lanes
// that share a particle block form a group: one counter atomic for the group
// (its old value plus the lane's rank in the group is the lane's bucket slot),
// one atomicMax of the group's largest contribution bound, and the group
// that finds the block empty lists it and activates its grid blocks.
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
    const unsigned long long gkey =
        key < 0 ? ~0ull : (((unsigned long long)(unsigned)tag << 32) | (unsigned)key);
    const unsigned peers = __match_any_sync(0xffffffffu, gkey);
    if (key < 0) return;
    const int leader = __ffs(peers) - 1;
    const unsigned bmax = __reduce_max_sync(peers, __float_as_uint(bnd));
    StepCtl &st = g.ctl->st[epoch & 1];
    int old = 0;
    if (lane == leader) {
        old = atomicAdd(&g.bcount[key], __popc(peers));
        atomicMax(&st.bound, bmax);
        if (old == 0) {
            g.plist[atomicAdd(&st.n_p, 1)] = key;
            activate_grid_blocks(g, key, epoch, st);
        }
    }
    old = __shfl_sync(peers, old, leader);
    const int rank = old + __popc(peers & ((1u << lane) - 1u));
    if (rank < g.cap) g.bucket[(size_t)key * g.cap + rank] = p;
    else g.over[atomicAdd(&st.n_over, 1)] = p;
}

// --------------------------------------------------- P2G + grid update ----
// Threads of one grid-block owner (a CTA runs kThreads / kOwnerThreads
// owners side by side, each on its own named barrier).
constexpr int kOwnerThreads = 64;      // one thread per node of the grid block
constexpr int kOwners = kThreads / kOwnerThreads;
static_assert(kOwnerThreads == 64 && kThreads % kOwnerThreads == 0, "owner layout");

struct OwnerSmem {
    unsigned long long acc[64 * 4];   // (m, p) of the block's 64 nodes, fixed point
    int nb[8];                        // the 8 particle blocks that reach it (-1: none)
    int off[9];                       // prefix of their particle counts
};

__device__ __forceinline__ void owner_sync(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kOwnerThreads) : "memory");
}

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

// Adds particle p's contributions to the nodes of grid block (ox, oy, oz) +
// [0, 4)^3 (its stencil nodes inside that block) to the owner's sums.
__device__ __forceinline__ void owner_add_particle(const GridWs &g, const GridParams &gp,
                                                   float mass, const FixScales &fs, int p,
                                                   int ox, int oy, int oz,
                                                   unsigned long long *acc) {
    const float4 *r = g.rec + 4 * (size_t)p;
    const float4 r0 = __ldcg(r);
    const Axis ax = bspline_axis(r0.x, gp.inv_dx), ay = bspline_axis(r0.y, gp.inv_dx),
               az = bspline_axis(r0.z, gp.inv_dx);
    const int a0 = max(0, ox - ax.base), a1 = min(2, ox + 3 - ax.base);
    const int b0 = max(0, oy - ay.base), b1 = min(2, oy + 3 - ay.base);
    const int c0 = max(0, oz - az.base), c1 = min(2, oz + 3 - az.base);
    if (a0 > a1 || b0 > b1 || c0 > c1) return;
    const float4 r1 = __ldcg(r + 1), r2 = __ldcg(r + 2), r3 = __ldcg(r + 3);
    P2gParticle q;
    q.x[0] = r0.x; q.x[1] = r0.y; q.x[2] = r0.z;
    q.mv[0] = r0.w; q.mv[1] = r1.x; q.mv[2] = r1.y;
    q.Q[0] = r1.z; q.Q[1] = r1.w;
    q.Q[2] = r2.x; q.Q[3] = r2.y; q.Q[4] = r2.z; q.Q[5] = r2.w;
    q.Q[6] = r3.x; q.Q[7] = r3.y; q.Q[8] = r3.z;
    const Stencil s{ax, ay, az};
    for (int ia = a0; ia <= a1; ++ia)
        for (int ib = b0; ib <= b1; ++ib)
            for (int ic = c0; ic <= c1; ++ic) {
                const float4 c = node_contribution(q, s, mass, gp.dx, ia, ib, ic);
                const int l = ((ax.base + ia - ox) * 4 + (ay.base + ib - oy)) * 4 +
                              (az.base + ic - oz);
                unsigned long long *n = acc + 4 * l;
                atomicAdd(n + 0, to_fix(c.x, fs.m));
                atomicAdd(n + 1, to_fix(c.y, fs.p));
                atomicAdd(n + 2, to_fix(c.z, fs.p));
                atomicAdd(n + 3, to_fix(c.w, fs.p));
            }
}

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

// One grid block gb owned by this thread group (gt: thread in the group):
// gather, accumulate, grid update.  Every thread of the group calls.
__device__ void owner_block(const GridWs &g, const GridParams &gp, float mass, float dt,
                            double blade_z, const FixScales &fs, int n_over, int gb,
                            OwnerSmem &sm, int gt, int bar_id, float *tap_mp, float *tap_v) {
    const int bz = gb % g.nb2, t = gb / g.nb2, by = t % g.nb1, bx = t / g.nb1;
    for (int i = gt; i < 64 * 4; i += kOwnerThreads) sm.acc[i] = 0ull;
    if (gt < 8) {
        const int kx = bx - (gt >> 2), ky = by - ((gt >> 1) & 1), kz = bz - (gt & 1);
        int key = -1, c = 0;
        if (kx >= 0 && ky >= 0 && kz >= 0) {
            key = (kx * g.nb1 + ky) * g.nb2 + kz;
            c = min(__ldcg(&g.bcount[key]), g.cap);
        }
        int v = c;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const int y = __shfl_up_sync(0xffu, v, o, 8);
            if (gt >= o) v += y;
        }
        sm.nb[gt] = key;
        sm.off[gt + 1] = v;
        if (gt == 0) sm.off[0] = 0;
    }
    owner_sync(bar_id);
    const int total = sm.off[8];
    const int ox = bx * 4, oy = by * 4, oz = bz * 4;
    for (int u = gt; u < total; u += kOwnerThreads) {
        int d = 0;
        while (u >= sm.off[d + 1]) ++d;
        const int p = __ldcg(&g.bucket[(size_t)sm.nb[d] * g.cap + (u - sm.off[d])]);
        owner_add_particle(g, gp, mass, fs, p, ox, oy, oz, sm.acc);
    }
    // particles that did not fit in their block's bucket (rare)
    for (int u = gt; u < n_over; u += kOwnerThreads)
        owner_add_particle(g, gp, mass, fs, __ldcg(&g.over[u]), ox, oy, oz, sm.acc);
    owner_sync(bar_id);
    {
        const int l = gt;                          // kOwnerThreads == 64 nodes
        const unsigned long long *n = sm.acc + 4 * l;
        const float4 a = make_float4(from_fix(n[0], fs.inv_m), from_fix(n[1], fs.inv_p),
                                     from_fix(n[2], fs.inv_p), from_fix(n[3], fs.inv_p));
        grid_node_update(g, gp, dt, blade_z, gb, l, a, tap_mp, tap_v);
    }
    owner_sync(bar_id);
}

// Owner loop of a single scene: grid blocks q = owner index, + all owners.
__device__ void phase_p2g_grid(const GridWs &g, const GridParams &gp, float mass, float dt,
                               double t, const StepCtl &st, float *tap_mp, float *tap_v) {
    __shared__ OwnerSmem sm[kOwners];
    const int grp = threadIdx.x / kOwnerThreads, gt = threadIdx.x % kOwnerThreads;
    const int n_g = __ldcg(&st.n_g), n_over = __ldcg(&st.n_over);
    const FixScales fs = fix_scales(mass, __ldcg(&st.bound));
    const double blade_z = (double)gp.blade_z0 + (double)gp.blade_vz * t;
    // owner w of CTA c is global owner w * gridDim.x + c: a short list still
    // spreads over every SM
    for (int q = grp * gridDim.x + blockIdx.x; q < n_g; q += kOwners * gridDim.x)
        owner_block(g, gp, mass, dt, blade_z, fs, n_over, __ldcg(&g.glist[q]), sm[grp], gt,
                    1 + grp, tap_mp, tap_v);
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

// bin | barrier | P2G + grid update.  Returns false if the barrier timed out.
// After the barrier (every CTA has read the old epoch) CTA 0 publishes the
// step's epoch, which later launches of the step read.
template <class Args>
__device__ bool bin_p2g_grid(const GridWs &g, const GridParams &gp, const Args &a, double t,
                             int epoch, float *tap_mp, float *tap_v, int *status) {
    const float stress_k = -a.dt * a.vol0 * 4.f * gp.inv_dx * gp.inv_dx;
    phase_bin(g, gp, a, stress_k, epoch, status);
    if (!grid_barrier(&g.ctl->bar, status)) return false;
    if (cta0_thread0()) g.ctl->epoch = epoch;
    phase_p2g_grid(g, gp, a.mass, a.dt, t, g.ctl->st[epoch & 1], tap_mp, tap_v);
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
__global__ void __launch_bounds__(kThreads)
k_mpm_latent(GridWs g, GridParams gp, P2gLatentArgs a, int n_S, double t, float *d_next,
             float *tap_mp, float *tap_v, int *status) {
    const int epoch = begin_step(g);
    if (!bin_p2g_grid(g, gp, a, t, epoch, tap_mp, tap_v, status)) return;
    if (!grid_barrier(&g.ctl->bar, status)) return;
    phase_g2p_latent(g, gp, a.X, a.u, a.n, n_S, a.dt, d_next, status);
    clear_bins(g, g.ctl->st[epoch & 1]);
}

__global__ void __launch_bounds__(kThreads)
k_mpm_full(GridWs g, GridParams gp, P2gFullArgs a, double t, float *tap_mp, float *tap_v,
           int *status) {
    const int epoch = begin_step(g);
    bin_p2g_grid(g, gp, a, t, epoch, tap_mp, tap_v, status);
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
// once (a flat index over the scenes' particles, active grid blocks and
// sample particles), with one grid barrier between phases for the whole
// batch.  Each scene keeps its own counters, epoch and buckets.
__global__ void __launch_bounds__(kThreads, 4)
k_mpm_batch(MpmBatchArgs b, int *status) {
    __shared__ int off[kMaxBatchScenes + 1];
    __shared__ int s_epoch[kMaxBatchScenes];
    __shared__ OwnerSmem sm[kOwners];
    const int ns = b.nscenes;
    const int stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    // every scene's step epoch, read before the first barrier; block 0 clears
    // each scene's other counter set
    for (int sc = threadIdx.x; sc < ns; sc += blockDim.x) {
        const Ctl *c = b.scenes[sc].g.ctl;
        s_epoch[sc] = __ldcg(&c->epoch) + 1;
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
    // P2G + grid update over every scene's active grid blocks
    block_offsets(ns, off, [&](int sc) {
        return __ldcg(&b.scenes[sc].g.ctl->st[s_epoch[sc] & 1].n_g);
    });
    {
        const int grp = threadIdx.x / kOwnerThreads, gt = threadIdx.x % kOwnerThreads;
        const int nblk = off[ns];
        for (int q = grp * gridDim.x + blockIdx.x; q < nblk; q += kOwners * gridDim.x) {
            const int sidx = find_scene(off, ns, q);
            const BatchSceneDev &sc = b.scenes[sidx];
            const StepCtl &st = sc.g.ctl->st[s_epoch[sidx] & 1];
            const FixScales fs = fix_scales(sc.mass, __ldcg(&st.bound));
            const double t = b.t0 + (double)b.step * (double)sc.dt;
            const double blade_z = (double)sc.gp.blade_z0 + (double)sc.gp.blade_vz * t;
            owner_block(sc.g, sc.gp, sc.mass, sc.dt, blade_z, fs, __ldcg(&st.n_over),
                        __ldcg(&sc.g.glist[q - off[sidx]]), sm[grp], gt, 1 + grp, nullptr,
                        nullptr);
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

template <class K, class... A>
cudaError_t launch_coop(K kernel, int grid, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

// ------------------------------------------------------------ launchers ---
cudaError_t launch_stress(const float *F, float *tau6, int n, int model, float mu, float lam,
                          cudaStream_t s) {
    k_stress<<<(n + 255) / 256, 256, 0, s>>>(F, tau6, n, model, mu, lam);
    return cudaGetLastError();
}

cudaError_t launch_mpm_latent(const GridWs &g, const GridParams &gp, const P2gLatentArgs &a,
                              int n_S, double t, float *d_next, float *tap_mp, float *tap_v,
                              int *status, cudaStream_t s) {
    static const int grid = coop_grid(k_mpm_latent, NSF_LATENT_MPM_CTAS_PER_SM);
    return launch_coop(k_mpm_latent, grid, s, g, gp, a, n_S, t, d_next, tap_mp,
                       tap_v, status);
}

cudaError_t launch_mpm_batch(const MpmBatchArgs &b, int *status, cudaStream_t s) {
    if (b.nscenes < 1 || b.nscenes > kMaxBatchScenes) return cudaErrorInvalidValue;
    static const int grid = coop_grid(k_mpm_batch);
    return launch_coop(k_mpm_batch, grid, s, b, status);
}

cudaError_t launch_mpm_full(const GridWs &g, const GridParams &gp, const P2gFullArgs &pa,
                            const G2pFullArgs &ga, double t, float *tap_mp, float *tap_v,
                            int *status, cudaStream_t s) {
    static const int grid = coop_grid(k_mpm_full);
    cudaError_t e = launch_coop(k_mpm_full, grid, s, g, gp, pa, t, tap_mp, tap_v,
                                status);
    if (e != cudaSuccess) return e;
    k_g2p_full<<<(ga.n + kThreads - 1) / kThreads, kThreads, 0, s>>>(g, gp, ga, status);
    return cudaGetLastError();
}

}  // namespace nsf
