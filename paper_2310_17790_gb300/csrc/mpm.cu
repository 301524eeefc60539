// MLS-MPM transfer kernels (paper §3.2, §3.3, Eq. 5; §5.2 on the integration
// particles).
//
// Step structure on the device:
//   k_bin_count    particle -> 4^3 particle block of its stencil base node,
//                  warp-aggregated counting, first particle of a block claims
//                  a slot in the active-block list
//   k_bin_scan     one CTA: per-slot counts, exclusive scan, activation of
//                  the 8 grid blocks each particle block can touch
//   k_bin_scatter  particle -> its sorted position
//   k_p2g_*        one CTA per active particle block (persistent loop): mass,
//                  APIC momentum and MLS stress force accumulated in a 6^3-node
//                  shared-memory tile, then one vector atomic per touched node
//   k_grid_update  v = p / m + dt g, walls, blade; re-zeroes the accumulators
//   k_g2p_*        gather of the 27 node velocities per particle
#include "constitutive.cuh"
#include "device_common.cuh"

namespace nsf {

namespace {

constexpr int kBinThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kP2gThreads = 256;
constexpr int kTile = 6;                 // nodes per axis covered by one particle block
constexpr int kTileNodes = kTile * kTile * kTile;


// ------------------------------------------------------------------ bin ---
__global__ void __launch_bounds__(kBinThreads)
k_bin_count(GridWs g, const float *__restrict__ X, const float *__restrict__ u,
            int n, float inv_dx, int *status) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int key = -2;                                   // -2: no particle
    if (p < n) {
        float x0 = u[p], x1 = u[n + p], x2 = u[2 * n + p];
        if (X) { x0 += X[p]; x1 += X[n + p]; x2 += X[2 * n + p]; }
        int b0 = __float2int_rd(x0 * inv_dx - 0.5f);
        int b1 = __float2int_rd(x1 * inv_dx - 0.5f);
        int b2 = __float2int_rd(x2 * inv_dx - 0.5f);
        bool ok = finite3(x0, x1, x2) && b0 >= 0 && b1 >= 0 && b2 >= 0 &&
                  b0 + 2 <= g.n0 - 1 && b1 + 2 <= g.n1 - 1 && b2 + 2 <= g.n2 - 1;
        if (ok) key = ((b0 >> 2) * g.nb1 + (b1 >> 2)) * g.nb2 + (b2 >> 2);
        else {
            key = -1;
            set_status(status, finite3(x0, x1, x2) ? NSF_ERR_OUT_OF_GRID : NSF_ERR_NONFINITE);
        }
    }
    // Lanes with the same block share one atomic.
    unsigned peers = __match_any_sync(0xffffffffu, key);
    int leader = __ffs(peers) - 1;
    int before = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader && key >= 0) base = atomicAdd(&g.cnt[key], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (p < n) {
        g.key[p] = key;
        if (key >= 0) {
            int rk = base + before;
            g.rank[p] = rk;
            if (rk == 0) {
                int slot = atomicAdd(&g.ctl->n_p_atomic, 1);
                g.blk_slot[key] = slot;
                g.plist[slot] = key;
            }
        }
    }
}

__global__ void __launch_bounds__(kScanThreads) k_bin_scan(GridWs g) {
    __shared__ int s_np, s_ng, s_epoch;
    __shared__ int s_part[kScanThreads];
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_np = g.ctl->n_p_atomic;
        g.ctl->n_p_atomic = 0;
        s_epoch = g.ctl->epoch + 1;
        g.ctl->epoch = s_epoch;
        s_ng = 0;
    }
    __syncthreads();
    const int np = s_np;
    // counts per slot; the per-block counters return to zero for the next step
    for (int s = tid; s < np; s += kScanThreads) {
        int key = g.plist[s];
        g.pcount[s] = g.cnt[key];
        g.cnt[key] = 0;
    }
    __syncthreads();
    // exclusive scan: contiguous chunk per thread, then a scan of chunk sums
    const int chunk = (np + kScanThreads - 1) / kScanThreads;
    const int lo = min(np, tid * chunk), hi = min(np, lo + chunk);
    int sum = 0;
    for (int s = lo; s < hi; ++s) sum += g.pcount[s];
    s_part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        int v = tid >= off ? s_part[tid - off] : 0;
        __syncthreads();
        s_part[tid] += v;
        __syncthreads();
    }
    int run = s_part[tid] - sum;
    for (int s = lo; s < hi; ++s) {
        g.poff[s] = run;
        run += g.pcount[s];
    }
    // grid blocks reachable from each particle block: (bx..bx+1) x (by..by+1) x (bz..bz+1)
    const int epoch = s_epoch;
    for (int idx = tid; idx < np * 8; idx += kScanThreads) {
        int key = g.plist[idx >> 3];
        int d = idx & 7;
        int bz = key % g.nb2, t = key / g.nb2;
        int by = t % g.nb1, bx = t / g.nb1;
        int cx = bx + (d >> 2), cy = by + ((d >> 1) & 1), cz = bz + (d & 1);
        if (cx >= g.nb0 || cy >= g.nb1 || cz >= g.nb2) continue;
        int gb = (cx * g.nb1 + cy) * g.nb2 + cz;
        if (atomicExch(&g.gstamp[gb], epoch) != epoch) {
            int at = atomicAdd(&s_ng, 1);
            g.glist[at] = gb;
        }
    }
    __syncthreads();
    if (tid == 0) {
        g.ctl->n_pblocks = np;
        g.ctl->n_gblocks = s_ng;
    }
}

__global__ void __launch_bounds__(kBinThreads) k_bin_scatter(GridWs g, int n) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int key = g.key[p];
    if (key < 0) return;
    g.perm[g.poff[g.blk_slot[key]] + g.rank[p]] = p;
}

// ------------------------------------------------------------------ P2G ---
// Scatter of one particle into the block tile (origin = 4 * block coords):
//   m_i += w m,  p_i += w (m v + Q (x_i - x_p)),  Q = m C - dt V0 (4/dx^2) tau.
__device__ __forceinline__ void scatter_particle(float4 *tile, const float xp[3],
                                                 const float mv[3],
                                                 const float Q[9], float mass,
                                                 float dx, float inv_dx,
                                                 int ox, int oy, int oz) {
    Axis ax = bspline_axis(xp[0], inv_dx);
    Axis ay = bspline_axis(xp[1], inv_dx);
    Axis az = bspline_axis(xp[2], inv_dx);
    const int tx = ax.base - ox, ty = ay.base - oy, tz = az.base - oz;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float dxa = ((float)a - ax.fx) * dx;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float dyb = ((float)b - ay.fx) * dx;
            const float wab = ax.w[a] * ay.w[b];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float dzc = ((float)c - az.fx) * dx;
                const float w = wab * az.w[c];
                const float px = mv[0] + Q[0] * dxa + Q[1] * dyb + Q[2] * dzc;
                const float py = mv[1] + Q[3] * dxa + Q[4] * dyb + Q[5] * dzc;
                const float pz = mv[2] + Q[6] * dxa + Q[7] * dyb + Q[8] * dzc;
                float4 *t = &tile[((tx + a) * kTile + (ty + b)) * kTile + (tz + c)];
                atomicAdd(&t->x, w * mass);
                atomicAdd(&t->y, w * px);
                atomicAdd(&t->z, w * py);
                atomicAdd(&t->w, w * pz);
            }
        }
    }
}

__device__ __forceinline__ void flush_tile(const GridWs &g, float4 *tile, int ox,
                                           int oy, int oz) {
    for (int t = threadIdx.x; t < kTileNodes; t += blockDim.x) {
        float4 v = tile[t];
        if (v.x != 0.f) {
            int i = ox + t / (kTile * kTile), j = oy + (t / kTile) % kTile, k = oz + t % kTile;
            if (i < g.n0 && j < g.n1 && k < g.n2) atomicAdd(&g.acc[node_addr(g, i, j, k)], v);
        }
        tile[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void __launch_bounds__(kP2gThreads)
k_p2g_latent(GridWs g, GridParams gp, P2gLatentArgs a) {
    __shared__ float4 tile[kTileNodes];
    for (int t = threadIdx.x; t < kTileNodes; t += blockDim.x) tile[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int npb = g.ctl->n_pblocks;
    const int n = a.n;
    const float stress_k = -a.dt * a.vol0 * 4.f * gp.inv_dx * gp.inv_dx;
    for (int s = blockIdx.x; s < npb; s += gridDim.x) {
        const int key = g.plist[s];
        const int bz = key % g.nb2, t = key / g.nb2, by = t % g.nb1, bx = t / g.nb1;
        const int ox = bx * 4, oy = by * 4, oz = bz * 4;
        const int start = g.poff[s], cnt = g.pcount[s];
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const int p = g.perm[start + i];
            float u0 = a.u[p], u1 = a.u[n + p], u2 = a.u[2 * n + p];
            float xp[3] = {u0, u1, u2};
            if (a.X) { xp[0] += a.X[p]; xp[1] += a.X[n + p]; xp[2] += a.X[2 * n + p]; }
            // v^n = (g(X, z_n) - g(X, z_{n-1})) / dt  (§5.1), on displacements
            const float mv[3] = {a.mass * (u0 - a.u_prev[p]) * a.inv_dt,
                                 a.mass * (u1 - a.u_prev[n + p]) * a.inv_dt,
                                 a.mass * (u2 - a.u_prev[2 * n + p]) * a.inv_dt};
            float tau[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) tau[c] = a.tau6[(size_t)c * n + p];
            // tau in Voigt order (xx, yy, zz, yz, xz, xy)
            const float T[9] = {tau[0], tau[5], tau[4], tau[5], tau[1], tau[3], tau[4], tau[3], tau[2]};
            float Q[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) Q[c] = a.mass * a.C9[(size_t)c * n + p] + stress_k * T[c];
            scatter_particle(tile, xp, mv, Q, a.mass, gp.dx, gp.inv_dx, ox, oy, oz);
        }
        __syncthreads();
        flush_tile(g, tile, ox, oy, oz);
    }
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

__global__ void __launch_bounds__(kP2gThreads)
k_p2g_full(GridWs g, GridParams gp, P2gFullArgs a) {
    __shared__ float4 tile[kTileNodes];
    for (int t = threadIdx.x; t < kTileNodes; t += blockDim.x) tile[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int npb = g.ctl->n_pblocks;
    const int n = a.n;
    const float stress_k = -a.dt * a.vol0 * 4.f * gp.inv_dx * gp.inv_dx;
    for (int s = blockIdx.x; s < npb; s += gridDim.x) {
        const int key = g.plist[s];
        const int bz = key % g.nb2, t = key / g.nb2, by = t % g.nb1, bx = t / g.nb1;
        const int ox = bx * 4, oy = by * 4, oz = bz * 4;
        const int start = g.poff[s], cnt = g.pcount[s];
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const int p = g.perm[start + i];
            const float xp[3] = {a.x[p], a.x[n + p], a.x[2 * n + p]};
            const float mv[3] = {a.mass * a.v[p], a.mass * a.v[n + p], a.mass * a.v[2 * n + p]};
            float T[9];
            if (a.tau6) {
                float tau[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) tau[c] = a.tau6[(size_t)c * n + p];
                T[0] = tau[0]; T[1] = tau[5]; T[2] = tau[4];
                T[3] = tau[5]; T[4] = tau[1]; T[5] = tau[3];
                T[6] = tau[4]; T[7] = tau[3]; T[8] = tau[2];
            } else {
                float F[9];
#pragma unroll
                for (int c = 0; c < 9; ++c) F[c] = a.F[(size_t)c * n + p];
                neo_hookean_tau(F, a.mu, a.lam, T);
            }
            float Q[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) Q[c] = a.mass * a.C[(size_t)c * n + p] + stress_k * T[c];
            scatter_particle(tile, xp, mv, Q, a.mass, gp.dx, gp.inv_dx, ox, oy, oz);
        }
        __syncthreads();
        flush_tile(g, tile, ox, oy, oz);
    }
}

// --------------------------------------------------------- grid update ---
__global__ void __launch_bounds__(256)
k_grid_update(GridWs g, GridParams gp, float dt, double t, float *tap_mp,
              float *tap_v) {
    const int ngb = g.ctl->n_gblocks;
    const int sub = threadIdx.x >> 6, l = threadIdx.x & 63;
    const int lx = l >> 4, ly = (l >> 2) & 3, lz = l & 3;
    const double blade_z = (double)gp.blade_z0 + (double)gp.blade_vz * t;
    for (int idx = blockIdx.x * 4 + sub; idx < ngb; idx += gridDim.x * 4) {
        const int gb = g.glist[idx];
        const int bz = gb % g.nb2, tt = gb / g.nb2, by = tt % g.nb1, bx = tt / g.nb1;
        const int i = bx * 4 + lx, j = by * 4 + ly, k = bz * 4 + lz;
        const int addr = gb * 64 + l;
        float4 a = __ldcg(&g.acc[addr]);
        g.acc[addr] = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 v = make_float4(0.f, 0.f, 0.f, a.x);
        if (a.x > 0.f) {
            float im = 1.f / a.x;
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
                float xi = (float)i * gp.dx;
                double zi = (double)k * (double)gp.dx;
                if (fabsf(xi - gp.blade_x) < gp.dx && zi > blade_z) {
                    v.x = 0.f;
                    v.y = 0.f;
                    v.z = gp.blade_vz;
                }
            }
        }
        g.vel[addr] = v;
        if (i < g.n0 && j < g.n1 && k < g.n2) {
            size_t nat = (((size_t)i * g.n1 + j) * g.n2 + k) * 4;
            if (tap_mp) *reinterpret_cast<float4 *>(tap_mp + nat) = a;
            if (tap_v) *reinterpret_cast<float4 *>(tap_v + nat) = v;
        }
    }
}

// ------------------------------------------------------------------ G2P ---
// Latent G2P on the sample particles (§5.2): only x^{n+1} is needed.  Writes
// the displacement target d = u_n + dt v_p (x^{n+1} - X for a residual g).
__global__ void __launch_bounds__(256)
k_g2p_latent(GridWs g, GridParams gp, const float *__restrict__ X,
             const float *__restrict__ u, int ld, int n_S, float dt,
             float *d_next, int *status) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_S) return;
    float u0 = u[p], u1 = u[ld + p], u2 = u[2 * ld + p];
    float x0 = u0, x1 = u1, x2 = u2;
    if (X) { x0 += X[p]; x1 += X[ld + p]; x2 += X[2 * ld + p]; }
    Axis ax = bspline_axis(x0, gp.inv_dx), ay = bspline_axis(x1, gp.inv_dx),
         az = bspline_axis(x2, gp.inv_dx);
    bool ok = ax.base >= 0 && ay.base >= 0 && az.base >= 0 && ax.base + 2 <= g.n0 - 1 &&
              ay.base + 2 <= g.n1 - 1 && az.base + 2 <= g.n2 - 1;
    float vx = 0.f, vy = 0.f, vz = 0.f;
    if (ok) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float w = ax.w[a] * ay.w[b] * az.w[c];
                    float4 v = __ldcg(&g.vel[node_addr(g, ax.base + a, ay.base + b, az.base + c)]);
                    vx = fmaf(w, v.x, vx);
                    vy = fmaf(w, v.y, vy);
                    vz = fmaf(w, v.z, vz);
                }
    } else {
        set_status(status, NSF_ERR_OUT_OF_GRID);
    }
    float d0 = fmaf(dt, vx, u0), d1 = fmaf(dt, vy, u1), d2 = fmaf(dt, vz, u2);
    d_next[p] = d0;
    d_next[n_S + p] = d1;
    d_next[2 * n_S + p] = d2;
}

// Full-order G2P (§3.3): v, x, C = (4/dx^2) sum w v_i (x_i - x_p)^T and the
// deformation-gradient update F <- (I + dt C) F (MLS velocity gradient).
__global__ void __launch_bounds__(256)
k_g2p_full(GridWs g, GridParams gp, G2pFullArgs a, int *status) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = a.n;
    if (p >= n) return;
    const float x0 = a.x[p], x1 = a.x[n + p], x2 = a.x[2 * n + p];
    Axis ax = bspline_axis(x0, gp.inv_dx), ay = bspline_axis(x1, gp.inv_dx),
         az = bspline_axis(x2, gp.inv_dx);
    bool ok = ax.base >= 0 && ay.base >= 0 && az.base >= 0 && ax.base + 2 <= g.n0 - 1 &&
              ay.base + 2 <= g.n1 - 1 && az.base + 2 <= g.n2 - 1;
    if (!ok) {
        set_status(status, NSF_ERR_OUT_OF_GRID);
        return;
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
                float4 vi = __ldcg(&g.vel[node_addr(g, ax.base + ia, ay.base + ib, az.base + ic)]);
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
        // float64 SVD, return map and stress of F^E for the next step
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

}  // namespace

// ------------------------------------------------------------ launchers ---
cudaError_t launch_stress(const float *F, float *tau6, int n, int model, float mu, float lam,
                          cudaStream_t s) {
    k_stress<<<(n + 255) / 256, 256, 0, s>>>(F, tau6, n, model, mu, lam);
    return cudaGetLastError();
}

static int persistent_grid(int work, int per_sm) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    (void)work;
    return sms * per_sm;
}

cudaError_t launch_bin(const GridWs &g, const float *X, const float *u, int n,
                       float inv_dx, int *status, cudaStream_t s) {
    int blocks = (n + kBinThreads - 1) / kBinThreads;
    k_bin_count<<<blocks, kBinThreads, 0, s>>>(g, X, u, n, inv_dx, status);
    k_bin_scan<<<1, kScanThreads, 0, s>>>(g);
    k_bin_scatter<<<blocks, kBinThreads, 0, s>>>(g, n);
    return cudaGetLastError();
}

cudaError_t launch_p2g_latent(const GridWs &g, const GridParams &gp,
                              const P2gLatentArgs &a, cudaStream_t s) {
    k_p2g_latent<<<persistent_grid(g.max_pblocks, 4), kP2gThreads, 0, s>>>(g, gp, a);
    return cudaGetLastError();
}

cudaError_t launch_p2g_full(const GridWs &g, const GridParams &gp,
                            const P2gFullArgs &a, cudaStream_t s) {
    k_p2g_full<<<persistent_grid(g.max_pblocks, 4), kP2gThreads, 0, s>>>(g, gp, a);
    return cudaGetLastError();
}

cudaError_t launch_grid_update(const GridWs &g, const GridParams &gp, float dt,
                               double t, float *tap_mp, float *tap_v,
                               cudaStream_t s) {
    k_grid_update<<<persistent_grid(g.max_gblocks, 4), 256, 0, s>>>(g, gp, dt, t, tap_mp, tap_v);
    return cudaGetLastError();
}

cudaError_t launch_g2p_latent(const GridWs &g, const GridParams &gp,
                              const float *X, const float *u, int ld, int n_S,
                              float dt, float *d_next, int *status, cudaStream_t s) {
    k_g2p_latent<<<(n_S + 255) / 256, 256, 0, s>>>(g, gp, X, u, ld, n_S, dt, d_next, status);
    return cudaGetLastError();
}

cudaError_t launch_g2p_full(const GridWs &g, const GridParams &gp,
                            const G2pFullArgs &a, int *status, cudaStream_t s) {
    k_g2p_full<<<(a.n + 255) / 256, 256, 0, s>>>(g, gp, a, status);
    return cudaGetLastError();
}

}  // namespace nsf
