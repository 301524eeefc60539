// Gauss-Newton iterations of the network inversion (§5.3, Eq. 9) inside the
// cooperative tensor-core Jacobian kernel, in float-float arithmetic (ff.cuh).
//
// One iteration, after the CTA's tiles have produced residuals res_p and
// Jacobian columns J_p (in the O3 rows of the tile):
//   1. per CTA: partial sums over its points of the entries
//        [0, T)       J^T J, upper triangle (i <= j), T = r (r + 1) / 2
//        [T, T + r)   J^T res
//        [T + r]      |res|^2
//      each product exact (two_prod), sums in float-float
//   2. each CTA stores its partials in its own column of a per-iteration-parity
//      slot array [entry][CTA] (plain stores: no atomics, nothing to clear)
//   3. grid barrier
//   4. every CTA adds all CTAs' slots in the same fixed order (so all CTAs
//      hold bit-identical sums) and solves
//        (J^T J + damping I) dz = -J^T res
//      by Gauss-Jordan elimination without pivoting (the matrix is symmetric
//      positive definite for damping > 0; a non-positive or non-finite pivot
//      is reported as NSF_ERR_SINGULAR and leaves z unchanged)
//   5. z <- z + dz in every CTA; CTA 0 writes the taps and the final z.
// The slot parity alternates: a CTA that has finished iteration it + 1 writes
// the other parity while slower CTAs may still read iteration it's slots, and
// it can only come back to this parity after the barrier of iteration it + 1,
// which every reader passes after reading.
#pragma once

#include "device_common.cuh"
#include "ff.cuh"

namespace nsf {

struct GnFF {
    ff part[kGnStrideMax];          // this CTA's sums over its tiles
    ff sum[kGnStrideMax];           // sums over all CTAs
    ff M[kMaxR * (kMaxR + 1)];      // [A + damping I | -b], row-major, r + 1 columns
    ff z[kMaxR];                    // current iterate
    double z0[kMaxR];               // z at the start of the run
    ff damping;
    int singular;
};


// The CTA's Gauss-Newton state.  A namespace-scope shared variable, so that
// the out-of-line helpers below address it as shared memory (a reference
// passed to them would be a generic pointer).
static __shared__ GnFF g_gn;

__device__ __forceinline__ int gn_stride(int r) { return r * (r + 1) / 2 + r + 1; }

// (i, j) of entry e < T of the packed upper triangle.
__device__ __forceinline__ void gn_tri_pair(int e, int r, int &i, int &j) {
    int ii = 0, off = 0;
    while (e >= off + (r - ii)) {
        off += r - ii;
        ++ii;
    }
    i = ii;
    j = ii + (e - off);
}

// Start of a run: z from global memory, CTA sums cleared.
__device__ inline void gn_ff_begin(const GnArgs &g, int r) {
    GnFF &sh = g_gn;
    const int tid = threadIdx.x;
    if (tid < r) {
        const double z = __ldcg(&g.z_start[tid]);
        sh.z0[tid] = z;
        sh.z[tid] = ff_from_double(z);
    }
    if (tid == 0) sh.damping = ff_from_double(g.damping);
    for (int e = tid; e < gn_stride(r); e += blockDim.x) sh.part[e] = ff{0.f, 0.f};
}

// Step 1 for one tile whose point q has L slots, columns q L .. q L + L - 1
// (npts points live): output a of column c is O3[3 c + c / 8 + a], slot 0
// the residual and slot 1 + k the Jacobian column d/dz_k.  The pad after
// every 8 columns puts the same entry of consecutive points (3 L + L / 8
// floats apart) in distinct banks for the lanes of one group of G; a warp
// takes 32 / G entries at a time, so tiles of few points still use all
// lanes.  Every thread calls.
__device__ __noinline__ void gn_ff_tile_partials(const float *O3, int L, int npts, int r) {
    GnFF &sh = g_gn;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int T = r * (r + 1) / 2, S = gn_stride(r);
    int G = 1;
    while (G < npts && G < 32) G <<= 1;
    const int per = 32 / G, sub = lane / G, ql = lane - sub * G;
    for (int e0 = warp * per; e0 < S; e0 += nwarps * per) {
        const int e = e0 + sub;
        // rows of the two factors: slot 1 + i against slot 1 + j (J^T J),
        // slot 1 + k against the residual (J^T r), the residual against itself
        int si = 0, sj = 0;
        if (e < T) {
            int i, j;
            gn_tri_pair(e, r, i, j);
            si = 1 + i;
            sj = 1 + j;
        } else if (e < T + r) {
            si = 1 + e - T;
        }
        ff acc{0.f, 0.f};
        if (e < S) {
            for (int q = ql; q < npts; q += G) {
                const int ca = q * L + si, cb = q * L + sj;
                const float *ra = O3 + 3 * ca + (ca >> 3), *rb = O3 + 3 * cb + (cb >> 3);
                ff d = ff_prod(ra[0], rb[0]);
                d = ff_add(d, ff_prod(ra[1], rb[1]));
                d = ff_add(d, ff_prod(ra[2], rb[2]));
                acc = ff_add(acc, d);
            }
        }
        for (int m = G >> 1; m >= 1; m >>= 1) acc = ff_add(acc, ff_shfl_xor(acc, m));
        if (ql == 0 && e < S) sh.part[e] = ff_add(sh.part[e], acc);
    }
}

// Gauss-Jordan on the augmented r x (r + 1) system in sh.M by warp 0; leaves
// dz_i = M[i][r] / M[i][i] in sh.M[i][r] and sh.singular set on failure.
// Step k subtracts (M[i][k] / M[k][k]) times row k from every row i != k, in
// the columns j > k.  For r <= 7 lane = (row i = lane % 8, column slot lane / 8)
// and each lane updates columns k + 1 + slot and k + 5 + slot, independent of
// each other; larger r loop over the entries.  (Keeping each row in one lane's
// registers and broadcasting the pivot row by shuffles measured slower.)
__device__ __noinline__ void gn_ff_solve_warp(int r) {
    GnFF &sh = g_gn;
    const int lane = threadIdx.x & 31;
    const int C = r + 1;
    int singular = 0;
    if (r <= 7) {
        const int i = lane & 7, cs = lane >> 3;
        for (int k = 0; k < r; ++k) {
            const ff piv = sh.M[k * C + k];
            if (!(piv.hi > 0.f) || !ff_isfinite(piv)) {
                singular = 1;
                break;
            }
            const int j0 = k + 1 + cs, j1 = j0 + 4;
            const bool act = i < r && i != k;
            ff m{0.f, 0.f}, a0{0.f, 0.f}, a1{0.f, 0.f}, p0{0.f, 0.f}, p1{0.f, 0.f};
            if (act) {
                m = sh.M[i * C + k];
                if (j0 < C) { a0 = sh.M[i * C + j0]; p0 = sh.M[k * C + j0]; }
                if (j1 < C) { a1 = sh.M[i * C + j1]; p1 = sh.M[k * C + j1]; }
            }
            __syncwarp();
            if (act) {
                m = ff_mul(m, ff_rcp(piv));
                if (j0 < C) sh.M[i * C + j0] = ff_sub(a0, ff_mul(m, p0));
                if (j1 < C) sh.M[i * C + j1] = ff_sub(a1, ff_mul(m, p1));
            }
            __syncwarp();
        }
    } else {
        for (int k = 0; k < r; ++k) {
            const ff piv = sh.M[k * C + k];
            if (!(piv.hi > 0.f) || !ff_isfinite(piv)) {
                singular = 1;
                break;
            }
            const ff inv = ff_rcp(piv);
            const int ncol = C - 1 - k;
            for (int idx = lane; idx < (r - 1) * ncol; idx += 32) {
                int i = idx / ncol;
                const int j = k + 1 + (idx - i * ncol);
                i += i >= k ? 1 : 0;
                const ff m = ff_mul(sh.M[i * C + k], inv);
                sh.M[i * C + j] = ff_sub(sh.M[i * C + j], ff_mul(m, sh.M[k * C + j]));
            }
            __syncwarp();
        }
    }
    if (!singular && lane < r)
        sh.M[lane * C + r] = ff_mul(sh.M[lane * C + r], ff_rcp(sh.M[lane * C + lane]));
    if (lane == 0) sh.singular = singular;
    __syncwarp();
}

// Steps 2-5.  Every thread of every CTA calls; returns false if the barrier
// wait ran out.
// The CTA is `rank` of the `nblk` CTAs that share this run (the whole grid for
// one problem, a CTA group of a batched launch).
__device__ __noinline__ bool gn_ff_finish_iteration(const GnArgs &g, int r, int it, int rank,
                                                    int nblk, int *status) {
    GnFF &sh = g_gn;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int T = r * (r + 1) / 2, S = gn_stride(r), C = r + 1;
    float2 *slots = g.slots + (size_t)(it & 1) * nblk * S;
    __syncthreads();
    // entry-major: the CTAs' values of one entry are contiguous, so the
    // reads below are coalesced
    for (int e = tid; e < S; e += blockDim.x)
        __stcg(&slots[(size_t)e * nblk + rank], make_float2(sh.part[e].hi, sh.part[e].lo));
    if (!group_barrier(g.bar, rank, nblk, status)) return false;
    // all loads of a lane first (one memory round trip), then the sums
    for (int e = warp; e < S; e += nwarps) {
        float2 v[kGnMaxSlotsPerLane];
#pragma unroll
        for (int k = 0; k < kGnMaxSlotsPerLane; ++k) {
            const int b = lane + 32 * k;
            v[k] = b < nblk ? __ldcg(&slots[(size_t)e * nblk + b]) : make_float2(0.f, 0.f);
        }
        ff acc{v[0].x, v[0].y};
#pragma unroll
        for (int k = 1; k < kGnMaxSlotsPerLane; ++k) acc = ff_add(acc, ff{v[k].x, v[k].y});
        acc = ff_warp_sum(acc);
        if (lane == 0) sh.sum[e] = acc;
    }
    __syncthreads();
    const ff damp = sh.damping;
    for (int idx = tid; idx < r * C; idx += blockDim.x) {
        const int i = idx / C, j = idx - i * C;
        ff v;
        if (j == r) {
            v = ff_neg(sh.sum[T + i]);
        } else {
            v = sh.sum[i <= j ? tri_index(i, j, r) : tri_index(j, i, r)];
            if (i == j) v = ff_add(v, damp);
        }
        sh.M[idx] = v;
    }
    for (int e = tid; e < S; e += blockDim.x) sh.part[e] = ff{0.f, 0.f};
    __syncthreads();
    if (tid < 32) gn_ff_solve_warp(r);
    __syncthreads();
    const bool singular = sh.singular != 0;
    if (singular && tid == 0) set_status(status, NSF_ERR_SINGULAR);
    const bool fin = it == g.iters - 1;
    if (tid < r) {
        const ff z0 = sh.z[tid];
        ff zn = singular ? z0 : ff_add(z0, sh.M[tid * C + r]);
        if (!ff_isfinite(zn)) {
            set_status(status, NSF_ERR_NONFINITE);
            zn = z0;
        }
        sh.z[tid] = zn;
        if (rank == 0) {
            const double zd = ff_to_double(zn);
            if (g.z_taps) g.z_taps[(size_t)it * r + tid] = zd;
            if (fin) {
                if (g.z_prev_out) g.z_prev_out[tid] = sh.z0[tid];
                g.z_out[tid] = zd;
            }
        }
    }
    __syncthreads();
    return true;
}

}  // namespace nsf
