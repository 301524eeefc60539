// MLS-MPM transfers (paper §3.2, §3.3, Eq. 5; §5.2 on the integration
// particles), fused into one cooperative launch per step.
//
// Phases of a launch, separated by a grid-wide barrier (all CTAs are
// co-resident; every wait is bounded in time):
//
//   P2G         each particle adds its 27 node contributions (mass, APIC
//               momentum, MLS stress force) straight into the grid with
//               vector atomics, and stamps its 4^3-cell particle block (the
//               block's first stamp of the step appends it to the active list)
//   activation  every active particle block stamps the 8 grid blocks its
//               stencils can reach and lists the newly stamped ones
//   grid        v = p / m + dt g, walls, blade, over the listed grid blocks;
//               the accumulators are re-zeroed on the way
//   G2P         latent: x^{n+1} on the sample particles, in the same launch;
//               full-order: a separate launch (its float64 return map needs
//               far more registers than the other phases)
//
// Direct vector atomics into L2 were measured faster than accumulating each
// particle block in a shared-memory tile first, for the sparse latent
// particle sets and for the dense full-order slab (8 particles per cell)
// alike: the tile's shared-memory float atomics conflict heavily, and the
// sorting the tile needs (count, scan, scatter) costs three more barriers.
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

// ---------------------------------------------------------------- P2G ----
// Particle p's 27 node contributions, added straight into the grid; returns
// its particle block, or -1 when its stencil leaves the grid (status set).
template <class Args>
__device__ __forceinline__ int p2g_particle(const GridWs &g, const GridParams &gp, const Args &a,
                                            float stress_k, int p, int *status) {
    P2gParticle q;
    load_particle(a, stress_k, p, q);
    const int key = block_key(g, q.x, gp.inv_dx, status);
    if (key >= 0) {
        Stencil s{bspline_axis(q.x[0], gp.inv_dx), bspline_axis(q.x[1], gp.inv_dx),
                  bspline_axis(q.x[2], gp.inv_dx)};
#pragma unroll
        for (int ia = 0; ia < 3; ++ia)
#pragma unroll
            for (int ib = 0; ib < 3; ++ib)
#pragma unroll
                for (int ic = 0; ic < 3; ++ic)
                    atomicAdd(&g.acc[node_addr(g, s.ax.base + ia, s.ay.base + ib, s.az.base + ic)],
                              node_contribution(q, s, a.mass, gp.dx, ia, ib, ic));
    }
    return key;
}

// One stamp per distinct (scene tag, block) in the warp; the first stamp of
// this step appends the block to the scene's active list.  Every lane of the
// warp calls; key < 0 means no particle.
__device__ __forceinline__ void stamp_block(const GridWs &g, int tag, int key, int epoch) {
    const unsigned peers = __match_any_sync(0xffffffffu, key < 0 ? -1 : (tag << 16) | key);
    if (key >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) {
        if (atomicExch(&g.pstamp[key], epoch) != epoch)
            g.plist[atomicAdd(&g.ctl->n_p_atomic, 1)] = key;
    }
}

template <class Args>
__device__ void phase_p2g(const GridWs &g, const GridParams &gp, const Args &a,
                                 float stress_k, int epoch, int *status) {
    const int n = a.n;
    const int stride = gridDim.x * blockDim.x;
    // the loop bound is uniform across each warp (match_any in stamp_block)
    for (int base = spread_index() & ~31; base < n; base += stride) {
        const int p = base + (threadIdx.x & 31);
        const int key = p < n ? p2g_particle(g, gp, a, stress_k, p, status) : -2;
        stamp_block(g, 0, key, epoch);
    }
}

// --------------------------------------------------------- activation ----
// Every active particle block stamps the grid blocks (bx..bx+1, by..by+1,
// bz..bz+1) that its particles' stencils can reach; the first stamp of this
// step lists the grid block.  One thread per (block, corner) pair.
__device__ void phase_activate(const GridWs &g, int np, int epoch) {
    for (int q = spread_index(); q < 8 * np; q += gridDim.x * blockDim.x) {
        const int key = __ldcg(&g.plist[q >> 3]), d = q & 7;
        const int bz = key % g.nb2, t = key / g.nb2, by = t % g.nb1, bx = t / g.nb1;
        const int cx = bx + (d >> 2), cy = by + ((d >> 1) & 1), cz = bz + (d & 1);
        if (cx >= g.nb0 || cy >= g.nb1 || cz >= g.nb2) continue;
        const int gb = (cx * g.nb1 + cy) * g.nb2 + cz;
        if (atomicExch(&g.gstamp[gb], epoch) != epoch) g.glist[atomicAdd(&g.ctl->n_g_atomic, 1)] = gb;
    }
}

// --------------------------------------------------------------- grid ----
// Node l (0 .. 63) of active grid block gb, whose accumulated (m, m v) is a:
// velocity update (gravity, walls, blade) into g.vel, and the accumulator
// cleared for the next step's P2G (skipped when it already holds zeros: in a
// sparse scene most nodes of an active block were not touched).
__device__ __forceinline__ void grid_node_update(const GridWs &g, const GridParams &gp, float dt,
                                                 double blade_z, int gb, int l, float4 a,
                                                 float *tap_mp, float *tap_v) {
    const int lx = l >> 4, ly = (l >> 2) & 3, lz = l & 3;
    const int bz = gb % g.nb2, tt = gb / g.nb2, by = tt % g.nb1, bx = tt / g.nb1;
    const int i = bx * 4 + lx, j = by * 4 + ly, k = bz * 4 + lz;
    const int addr = gb * 64 + l;
    if (a.x != 0.f || a.y != 0.f || a.z != 0.f || a.w != 0.f) g.acc[addr] = make_float4(0.f, 0.f, 0.f, 0.f);
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
    g.vel[addr] = v;
    const size_t nat = (((size_t)i * g.n1 + j) * g.n2 + k) * 4;
    if (tap_mp) *reinterpret_cast<float4 *>(tap_mp + nat) = a;
    if (tap_v) *reinterpret_cast<float4 *>(tap_v + nat) = v;
}

// Grid blocks a thread updates per pass: their index and node loads are
// issued together, so a thread has kGridUnroll memory chains in flight
// instead of one.
constexpr int kGridUnroll = 4;

__device__ void phase_grid(const GridWs &g, const GridParams &gp, float dt, double t,
                           float *tap_mp, float *tap_v) {
    const int ngb = __ldcg(&g.ctl->n_g_atomic);
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
            if (gb[u] >= 0) a[u] = __ldcg(&g.acc[gb[u] * 64 + l]);
#pragma unroll
        for (int u = 0; u < kGridUnroll; ++u)
            if (gb[u] >= 0) grid_node_update(g, gp, dt, blade_z, gb[u], l, a[u], tap_mp, tap_v);
    }
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

// ------------------------------------------------ P2G + grid update ----
// Returns false if a barrier timed out (the launch then ends early).
template <class Args>
__device__ bool p2g_and_grid(const GridWs &g, const GridParams &gp, const Args &a, double t,
                             int epoch, float *tap_mp, float *tap_v, int *status) {
    const float stress_k = -a.dt * a.vol0 * 4.f * gp.inv_dx * gp.inv_dx;
    phase_p2g(g, gp, a, stress_k, epoch, status);
    if (!grid_barrier(&g.ctl->bar, status)) return false;
    phase_activate(g, __ldcg(&g.ctl->n_p_atomic), epoch);
    if (!grid_barrier(&g.ctl->bar, status)) return false;
    if (cta0_thread0()) g.ctl->n_p_atomic = 0;          // every CTA has read it
    phase_grid(g, gp, a.dt, t, tap_mp, tap_v);
    return true;
}

__global__ void __launch_bounds__(kThreads)
k_mpm_latent(GridWs g, GridParams gp, P2gLatentArgs a, int n_S, double t, float *d_next,
             float *tap_mp, float *tap_v, int *status) {
    const int epoch = __ldcg(&g.ctl->epoch) + 1;
    if (!p2g_and_grid(g, gp, a, t, epoch, tap_mp, tap_v, status)) return;
    if (!grid_barrier(&g.ctl->bar, status)) return;
    phase_g2p_latent(g, gp, a.X, a.u, a.n, n_S, a.dt, d_next, status);
    if (cta0_thread0()) {
        g.ctl->n_g_atomic = 0;                            // read by the grid phase only
        g.ctl->epoch = epoch;
    }
}

__global__ void __launch_bounds__(kThreads)
k_mpm_full(GridWs g, GridParams gp, P2gFullArgs a, double t, float *tap_mp, float *tap_v,
           int *status) {
    const int epoch = __ldcg(&g.ctl->epoch) + 1;
    p2g_and_grid(g, gp, a, t, epoch, tap_mp, tap_v, status);
}

// Full-order G2P, one thread per particle; it also closes the step's
// bookkeeping (grid-block counter, epoch) that the MPM launch left open.
__global__ void __launch_bounds__(kThreads)
k_g2p_full(GridWs g, GridParams gp, G2pFullArgs a, int *status) {
    phase_g2p_full(g, gp, a, status);
    if (cta0_thread0()) {
        g.ctl->n_g_atomic = 0;
        g.ctl->epoch = g.ctl->epoch + 1;
    }
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
// once (a flat index over the scenes' particles, active particle blocks,
// active grid blocks and sample particles), with one grid barrier between
// phases for the whole batch.
__global__ void __launch_bounds__(kThreads, 4)
k_mpm_batch(MpmBatchArgs b, int *status) {
    __shared__ int off[kMaxBatchScenes + 1];
    const int ns = b.nscenes;
    const int stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    // P2G
    const int total_N = __ldg(&b.n_off[ns]);
    for (int base = spread_index() & ~31; base < total_N; base += stride) {
        const int q = base + lane;
        int key = -2, sidx = 0;
        if (q < total_N) sidx = find_scene(b.n_off, ns, q);
        const BatchSceneDev &sc = b.scenes[sidx];
        const int epoch = __ldcg(&sc.g.ctl->epoch) + 1;
        if (q < total_N) {
            const float stress_k = -sc.dt * sc.vol0 * 4.f * sc.gp.inv_dx * sc.gp.inv_dx;
            key = p2g_particle(sc.g, sc.gp, latent_args(sc, b.parity), stress_k,
                               q - __ldg(&b.n_off[sidx]), status);
        }
        stamp_block(sc.g, sidx, key, epoch);
    }
    if (!grid_barrier(b.bar, status)) return;
    // block activation
    block_offsets(ns, off, [&](int sc) { return 8 * __ldcg(&b.scenes[sc].g.ctl->n_p_atomic); });
    for (int q = spread_index(); q < off[ns]; q += stride) {
        const int sidx = find_scene(off, ns, q);
        const GridWs &g = b.scenes[sidx].g;
        const int epoch = __ldcg(&g.ctl->epoch) + 1;
        const int k = q - off[sidx];
        const int key = __ldcg(&g.plist[k >> 3]), d = k & 7;
        const int bz = key % g.nb2, t = key / g.nb2, by = t % g.nb1, bx = t / g.nb1;
        const int cx = bx + (d >> 2), cy = by + ((d >> 1) & 1), cz = bz + (d & 1);
        if (cx >= g.nb0 || cy >= g.nb1 || cz >= g.nb2) continue;
        const int gb = (cx * g.nb1 + cy) * g.nb2 + cz;
        if (atomicExch(&g.gstamp[gb], epoch) != epoch) g.glist[atomicAdd(&g.ctl->n_g_atomic, 1)] = gb;
    }
    if (!grid_barrier(b.bar, status)) return;
    if (blockIdx.x == 0)                         // every CTA has read them
        for (int sc = threadIdx.x; sc < ns; sc += blockDim.x) b.scenes[sc].g.ctl->n_p_atomic = 0;
    // grid update
    block_offsets(ns, off, [&](int sc) { return __ldcg(&b.scenes[sc].g.ctl->n_g_atomic); });
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
                if (sidx[k] >= 0) a[k] = __ldcg(&b.scenes[sidx[k]].g.acc[gb[k] * 64 + l]);
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
    if (blockIdx.x == 0)
        for (int sc = threadIdx.x; sc < ns; sc += blockDim.x) {
            Ctl *c = b.scenes[sc].g.ctl;
            c->n_g_atomic = 0;                   // read by the grid phase only
            c->epoch = c->epoch + 1;
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
