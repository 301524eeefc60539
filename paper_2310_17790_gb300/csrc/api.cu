// Host side of the libnsf C ABI (include/nsf.h): argument validation, weight
// packing, workspace layout and the launch sequence of each call.
#include <algorithm>
#include <cmath>
#include <queue>
#include <cstring>
#include <new>
#include <vector>

#include "device_common.cuh"
#include "tc_common.cuh"

using namespace nsf;

struct nsf_fields {
    nsf_fields_desc desc;
    FieldsDev dev;
    void *d_mem;
    size_t bytes;
    // the inference kernels can run these fields (a BF16 field whose weights do
    // not fit in shared memory is created for training only)
    int infer_ok;
};

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// Sequential sub-allocation of one caller workspace.
struct Carver {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return o;
    }
};

bool valid_grid(const nsf_grid_desc *g) {
    if (!g) return false;
    for (int d = 0; d < 3; ++d)
        if (g->n[d] < 8 || g->n[d] > 2048 || (g->n[d] & 3)) return false;
    if (!(g->dx > 0.f) || !std::isfinite(g->dx)) return false;
    if (g->wall_cells < 0) return false;
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(g->gravity[d])) return false;
    size_t nodes = (size_t)g->n[0] * g->n[1] * g->n[2];
    return nodes <= ((size_t)1 << 31) / 64;
}

GridParams make_params(const nsf_grid_desc *g) {
    GridParams p;
    p.dx = g->dx;
    p.inv_dx = 1.f / g->dx;
    p.gx = g->gravity[0];
    p.gy = g->gravity[1];
    p.gz = g->gravity[2];
    p.wall_cells = g->wall_cells;
    p.blade_enable = g->blade_enable;
    p.blade_x = g->blade_x;
    p.blade_z0 = g->blade_z0;
    p.blade_vz = g->blade_vz;
    return p;
}

// Grid part of a workspace.  The particle buckets hold up to `cap` particle
// indices per particle block (min(cap_max, n)); particles past that go to an
// overflow list and add their contributions with global atomics (correct,
// but slower), so cap_max is set well above the densest expected packing (8
// particles per cell fill a block with 512).
constexpr int kBucketCapScene = kMaxBucketCap;
constexpr int kBucketCapBatch = 256;
static_assert(kBucketCapBatch <= kMaxBucketCap, "bucket capacity");

struct GridLayout {
    size_t acc, vel, gstamp, bcount, bucket, rec, plist, glist, over, ctl;
    int nblocks, max_pblocks, max_gblocks, cap;
};

GridLayout carve_grid(Carver &c, const nsf_grid_desc *g, int n, int cap_max) {
    GridLayout L;
    size_t nodes = (size_t)g->n[0] * g->n[1] * g->n[2];
    L.nblocks = (int)(nodes / 64);
    L.max_pblocks = n < L.nblocks ? n : L.nblocks;
    long long mg = 8LL * L.max_pblocks;
    L.max_gblocks = mg < L.nblocks ? (int)mg : L.nblocks;
    L.cap = n < cap_max ? n : cap_max;
    L.ctl = c.take(sizeof(Ctl));
    L.acc = c.take(nodes * 4 * sizeof(unsigned long long));
    L.vel = c.take(nodes * sizeof(float4));
    L.gstamp = c.take((size_t)L.nblocks * 4);
    L.bcount = c.take((size_t)L.nblocks * 4);
    L.bucket = c.take((size_t)L.nblocks * L.cap * 4);
    L.rec = c.take((size_t)n * 4 * sizeof(float4));
    L.plist = c.take((size_t)L.max_pblocks * 4);
    L.glist = c.take((size_t)L.max_gblocks * 4);
    L.over = c.take((size_t)n * 4);
    return L;
}

GridWs grid_ws(char *base, const GridLayout &L, const nsf_grid_desc *g, int n) {
    (void)n;
    GridWs w;
    w.n0 = g->n[0];
    w.n1 = g->n[1];
    w.n2 = g->n[2];
    w.nb0 = w.n0 / 4;
    w.nb1 = w.n1 / 4;
    w.nb2 = w.n2 / 4;
    w.nblocks = L.nblocks;
    w.acc = reinterpret_cast<unsigned long long *>(base + L.acc);
    w.vel = reinterpret_cast<float4 *>(base + L.vel);
    w.gstamp = reinterpret_cast<int *>(base + L.gstamp);
    w.bcount = reinterpret_cast<int *>(base + L.bcount);
    w.bucket = reinterpret_cast<int *>(base + L.bucket);
    w.cap = L.cap;
    w.rec = reinterpret_cast<float4 *>(base + L.rec);
    w.plist = reinterpret_cast<int *>(base + L.plist);
    w.glist = reinterpret_cast<int *>(base + L.glist);
    w.over = reinterpret_cast<int *>(base + L.over);
    w.ctl = reinterpret_cast<Ctl *>(base + L.ctl);
    w.max_pblocks = L.max_pblocks;
    w.max_gblocks = L.max_gblocks;
    return w;
}

// Gauss-Newton scratch of a workspace: z between iterations and the float64
// sums (one launch per iteration, FP32 path), the per-CTA float-float slots
// (cooperative tensor-core path) and the control words (arrival ticket and
// grid-barrier word, each in its own 128-byte line).
struct GnLayout {
    size_t zgn, gsum, slots, ctl;
};

GnLayout carve_gn(Carver &c, const nsf_fields *f, int n_S) {
    GnLayout L;
    L.zgn = c.take(NSF_MAX_R * 8);
    L.gsum = c.take((size_t)kGnStrideMax * 8);
    size_t slots = 0;
    if (f->dev.precision == NSF_PREC_BF16)
        slots = 2 * (size_t)jac_grid_size_tc(f->dev, n_S) * gn_partial_stride(f->desc.r) * 8;
    L.slots = c.take(slots);
    L.ctl = c.take(256);
    return L;
}

GnArgs gn_args(char *base, const GnLayout &L) {
    GnArgs g{};
    g.z_buf = reinterpret_cast<double *>(base + L.zgn);
    g.gsum = reinterpret_cast<double *>(base + L.gsum);
    g.slots = reinterpret_cast<float2 *>(base + L.slots);
    g.counter = reinterpret_cast<int *>(base + L.ctl);
    g.bar = reinterpret_cast<unsigned *>(base + L.ctl + 128);
    return g;
}

struct LatentLayout {
    GridLayout grid;
    size_t u[2], tau, C, dnext;
    GnLayout gn;
    size_t total;
};

LatentLayout latent_layout(const nsf_fields *f, const nsf_latent_scene *sc,
                           int cap_max = kBucketCapScene) {
    Carver c;
    LatentLayout L;
    L.grid = carve_grid(c, &sc->grid, sc->n_N, cap_max);
    size_t n = (size_t)sc->n_N;
    L.u[0] = c.take(3 * n * 4);
    L.u[1] = c.take(3 * n * 4);
    L.tau = c.take(6 * n * 4);
    L.C = c.take(9 * n * 4);
    L.dnext = c.take(3 * (size_t)sc->n_S * 4);
    L.gn = carve_gn(c, f, sc->n_S);
    L.total = c.off;
    return L;
}

struct ProjectLayout {
    size_t target, u;
    GnLayout gn;
    size_t total;
};

ProjectLayout project_layout(const nsf_fields *f, int n_S) {
    Carver c;
    ProjectLayout L;
    L.target = c.take(3 * (size_t)n_S * 4);
    L.u = c.take(3 * (size_t)n_S * 4);
    L.gn = carve_gn(c, f, n_S);
    L.total = c.off;
    return L;
}

struct FullLayout {
    GridLayout grid;
    size_t tau, total;
};

FullLayout full_layout(const nsf_grid_desc *g, int n) {
    Carver c;
    FullLayout L;
    L.grid = carve_grid(c, g, n, kBucketCapScene);
    L.tau = c.take(6 * (size_t)n * 4);
    L.total = c.off;
    return L;
}

// ------------------------------------------------------- small kernels ---
// out[i] = a[i] + s * b[i]  over `count` floats.
__global__ void k_axpy(float *out, const float *a, const float *b, float s, int count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = a[i] + s * b[i];
}

cudaError_t axpy(float *out, const float *a, const float *b, float s, int count,
                 cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_axpy<<<(count + 255) / 256, 256, 0, st>>>(out, a, b, s, count);
    return cudaGetLastError();
}

cudaError_t run_fields(const FieldsDev &fd, const float *X, int n, int ld, int njobs,
                       const FieldJob *jobs, int *status, cudaStream_t s) {
    if (n <= 0 || njobs <= 0) return cudaSuccess;
    if (fd.precision == NSF_PREC_BF16) return launch_fields_tc(fd, X, n, ld, njobs, jobs, status, s);
    return launch_fields_simt(fd, X, n, ld, njobs, jobs, status, s);
}

// Evaluation (gn == null) or a whole Gauss-Newton run of gn->iters iterations:
// one cooperative launch on the tensor-core path, one launch per iteration on
// the CUDA-core path.
cudaError_t run_jacobian(const FieldsDev &fd, const float *X, int n, int ld, const double *z,
                         float *u, float *dudz, const GnArgs *gn, int *status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (fd.precision == NSF_PREC_BF16)
        return launch_jacobian_tc(fd, X, n, ld, z, u, dudz, gn, status, s);
    if (!gn) return launch_jacobian_simt(fd, X, n, ld, z, u, dudz, nullptr, 0, status, s);
    for (int it = 0; it < gn->iters; ++it) {
        cudaError_t e = launch_jacobian_simt(fd, X, n, ld, z, u, dudz, gn, it, status, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool valid_fields_desc(const nsf_fields_desc *d) {
    if (!d) return false;
    if (d->r < 1 || d->r > NSF_MAX_R) return false;
    if (d->precision != NSF_PREC_FP32 && d->precision != NSF_PREC_BF16) return false;
    for (int f = 0; f < 3; ++f) {
        int w = d->width[f];
        if (w < 16 || w > NSF_MAX_WIDTH || (w % 16)) return false;
        if (d->depth[f] < 1 || d->depth[f] > NSF_MAX_DEPTH) return false;
        for (int o = 0; o < kOutDim[f]; ++o)
            if (!std::isfinite(d->out_scale[f][o]) || !std::isfinite(d->out_shift[f][o])) return false;
    }
    return true;
}

bool valid_gn(const nsf_gn_opts *o) {
    return o && o->iters >= 1 && o->iters <= 32 && std::isfinite(o->damping) && o->damping >= 0.0;
}

#define NSF_CUDA_TRY(expr)                       \
    do {                                         \
        cudaError_t e_ = (expr);                 \
        if (e_ != cudaSuccess) return NSF_ERR_CUDA; \
    } while (0)

}  // namespace

// Defined in fields_tc.cu: the bf16 tensor-core operand order of one matrix
// [rows][k] (fp32 host values, rows padded with zeros to rows_pad), and the
// shared memory a field needs on the tensor-core path (0: does not fit).
namespace nsf {
size_t tc_layer_elems(int rows_pad, int k);
void tc_pack_layer(const float *W, int rows, int rows_pad, int k, __nv_bfloat16 *dst);
size_t tc_smem_bytes(int r, int width, int depth);
}

extern "C" {

int nsf_version(void) { return 100; }

const char *nsf_status_string(int s) {
    switch (s) {
        case NSF_OK: return "ok";
        case NSF_ERR_INVALID_ARG: return "invalid argument";
        case NSF_ERR_CUDA: return "CUDA error";
        case NSF_ERR_OUT_OF_GRID: return "particle stencil outside the grid";
        case NSF_ERR_NONFINITE: return "non-finite value";
        case NSF_ERR_SINGULAR: return "Gauss-Newton system not positive definite";
        case NSF_ERR_ITER_CAP: return "bounded wait gave up";
        case NSF_ERR_UNSUPPORTED: return "unsupported request";
        case NSF_ERR_NO_MEMORY: return "out of device memory";
        case NSF_ERR_WORKSPACE: return "workspace missing or too small";
        default: return "unknown status";
    }
}

nsf_status nsf_create_fields(const nsf_fields_desc *desc, const float *const host_weights[3],
                             nsf_fields **out) {
    if (!out || !valid_fields_desc(desc) || !host_weights) return NSF_ERR_INVALID_ARG;
    for (int f = 0; f < 3; ++f)
        if (!host_weights[f]) return NSF_ERR_INVALID_ARG;
    const bool bf16 = desc->precision == NSF_PREC_BF16;
    const int r = desc->r;

    // Host staging: float section then (bf16) packed section.
    std::vector<float> fbuf;
    std::vector<__nv_bfloat16> hbuf;
    struct Off {
        size_t W0, Wout, b[NSF_MAX_DEPTH + 1], Wt[NSF_MAX_DEPTH], blob, blob_elems;
    } off[3];
    auto push = [&](const float *src, size_t count) {
        size_t o = fbuf.size();
        fbuf.insert(fbuf.end(), src, src + count);
        while (fbuf.size() % 64) fbuf.push_back(0.f);   // keep 256-byte alignment
        return o;
    };
    auto round_bf16 = [](float v) { return __bfloat162float(__float2bfloat16_rn(v)); };
    int infer_ok = 1;
    if (bf16)
        for (int f = 0; f < 3; ++f)
            if (tc_smem_bytes(r, desc->width[f], desc->depth[f]) == 0) infer_ok = 0;
    for (int f = 0; f < 3; ++f) {
        const int W = desc->width[f], D = desc->depth[f], od = kOutDim[f];
        const float *src = host_weights[f];
        size_t pos = 0;
        off[f].blob = hbuf.size();
        for (int l = 0; l <= D; ++l) {
            int in = l == 0 ? 3 + r : W;
            int o = l == D ? od : W;
            std::vector<float> Wm(src + pos, src + pos + (size_t)in * o);
            pos += (size_t)in * o;
            for (float v : Wm)
                if (!std::isfinite(v)) return NSF_ERR_INVALID_ARG;
            if (bf16)
                for (float &v : Wm) v = round_bf16(v);
            if (l == 0) {
                off[f].W0 = push(Wm.data(), Wm.size());
            } else if (l == D) {
                off[f].Wout = push(Wm.data(), Wm.size());
                if (bf16) {
                    size_t o2 = hbuf.size();
                    hbuf.resize(o2 + tc_layer_elems(16, W));
                    tc_pack_layer(Wm.data(), od, 16, W, hbuf.data() + o2);
                }
            } else {
                std::vector<float> Wt((size_t)W * W);
                for (int j = 0; j < W; ++j)
                    for (int k = 0; k < W; ++k) Wt[(size_t)k * W + j] = Wm[(size_t)j * W + k];
                off[f].Wt[l] = push(Wt.data(), Wt.size());
                if (bf16) {
                    size_t o2 = hbuf.size();
                    hbuf.resize(o2 + tc_layer_elems(W, W));
                    tc_pack_layer(Wm.data(), W, W, W, hbuf.data() + o2);
                }
            }
            for (int q = 0; q < o; ++q)
                if (!std::isfinite(src[pos + q])) return NSF_ERR_INVALID_ARG;
            off[f].b[l] = push(src + pos, o);
            pos += o;
        }
        off[f].blob_elems = hbuf.size() - off[f].blob;
        while (hbuf.size() % 128) hbuf.push_back(__float2bfloat16_rn(0.f));
    }
    size_t fbytes = fbuf.size() * sizeof(float);
    size_t hbytes = hbuf.size() * sizeof(__nv_bfloat16);
    void *mem = nullptr;
    if (cudaMalloc(&mem, fbytes + hbytes) != cudaSuccess) {
        cudaGetLastError();
        return NSF_ERR_NO_MEMORY;
    }
    if (cudaMemcpy(mem, fbuf.data(), fbytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        (hbytes && cudaMemcpy((char *)mem + fbytes, hbuf.data(), hbytes, cudaMemcpyHostToDevice) !=
                       cudaSuccess)) {
        cudaFree(mem);
        return NSF_ERR_CUDA;
    }
    nsf_fields *F = new (std::nothrow) nsf_fields;
    if (!F) {
        cudaFree(mem);
        return NSF_ERR_NO_MEMORY;
    }
    std::memset(F, 0, sizeof(*F));
    F->desc = *desc;
    F->infer_ok = infer_ok;
    F->d_mem = mem;
    F->bytes = fbytes + hbytes;
    const float *fb = static_cast<const float *>(mem);
    const __nv_bfloat16 *hb = reinterpret_cast<const __nv_bfloat16 *>((char *)mem + fbytes);
    F->dev.r = r;
    F->dev.residual_g = desc->residual_g ? 1 : 0;
    F->dev.precision = desc->precision;
    for (int f = 0; f < 3; ++f) {
        FieldDev &d = F->dev.f[f];
        d.width = desc->width[f];
        d.depth = desc->depth[f];
        d.out_dim = kOutDim[f];
        d.W0 = fb + off[f].W0;
        d.Wout = fb + off[f].Wout;
        for (int l = 0; l <= d.depth; ++l) d.b[l] = fb + off[f].b[l];
        for (int l = 1; l < d.depth; ++l) d.Wt[l] = fb + off[f].Wt[l];
        d.tc_blob = bf16 ? hb + off[f].blob : nullptr;
        d.tc_blob_bytes = bf16 ? (int)(off[f].blob_elems * sizeof(__nv_bfloat16)) : 0;
        for (int o = 0; o < 9; ++o) {
            d.scale[o] = o < d.out_dim ? desc->out_scale[f][o] : 0.f;
            d.shift[o] = o < d.out_dim ? desc->out_shift[f][o] : 0.f;
        }
    }
    *out = F;
    return NSF_OK;
}

void nsf_destroy_fields(nsf_fields *f) {
    if (!f) return;
    cudaFree(f->d_mem);
    delete f;
}

nsf_status nsf_fields_get_desc(const nsf_fields *f, nsf_fields_desc *out) {
    if (!f || !out) return NSF_ERR_INVALID_ARG;
    *out = f->desc;
    return NSF_OK;
}

nsf_status nsf_eval_fields(const nsf_fields *f, const float *d_X, int n, const double *d_z,
                           float *d_x, float *d_tau6, float *d_C9, float *d_dxdz,
                           int *d_status, void *stream) {
    if (!f || n < 0 || (n > 0 && (!d_X || !d_z))) return NSF_ERR_INVALID_ARG;
    if (!f->infer_ok) return NSF_ERR_UNSUPPORTED;
    if (n == 0) return NSF_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FieldJob jobs[3];
    int nj = 0;
    if (d_x) jobs[nj++] = FieldJob{NSF_FIELD_G, d_z, d_x};
    if (d_tau6) jobs[nj++] = FieldJob{NSF_FIELD_H, d_z, d_tau6};
    if (d_C9) jobs[nj++] = FieldJob{NSF_FIELD_L, d_z, d_C9};
    NSF_CUDA_TRY(run_fields(f->dev, d_X, n, n, nj, jobs, d_status, s));
    if (d_x && f->dev.residual_g) NSF_CUDA_TRY(axpy(d_x, d_x, d_X, 1.f, 3 * n, s));
    if (d_dxdz) NSF_CUDA_TRY(run_jacobian(f->dev, d_X, n, n, d_z, nullptr, d_dxdz, nullptr, d_status, s));
    return NSF_OK;
}

nsf_status nsf_latent_workspace_size(const nsf_fields *f, const nsf_latent_scene *sc, size_t *bytes) {
    if (!f || !sc || !bytes || sc->n_N < 1 || sc->n_S < 1 || sc->n_S > sc->n_N ||
        !valid_grid(&sc->grid))
        return NSF_ERR_INVALID_ARG;
    *bytes = latent_layout(f, sc).total;
    return NSF_OK;
}

nsf_status nsf_latent_step(const nsf_fields *f, const nsf_latent_scene *sc, double dt, double t0,
                           int nsteps, unsigned int flags, double *d_z, double *d_z_prev,
                           const nsf_gn_opts *opts,
                           void *d_ws, size_t ws_bytes, int *d_status,
                           const nsf_latent_taps *taps, void *stream) {
    if (!f || !sc || !d_z || !d_z_prev || !valid_gn(opts) || nsteps < 0 || !sc->d_X ||
        sc->n_N < 1 || sc->n_S < 1 || sc->n_S > sc->n_N || !valid_grid(&sc->grid) ||
        !(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(t0) || !(sc->mass > 0.f) ||
        !(sc->vol0 > 0.f) || (flags & ~(unsigned)NSF_LATENT_REUSE_PREV))
        return NSF_ERR_INVALID_ARG;
    if (!f->infer_ok) return NSF_ERR_UNSUPPORTED;
    if (nsteps == 0) return NSF_OK;
    LatentLayout L = latent_layout(f, sc);
    if (!d_ws || ws_bytes < L.total) return NSF_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(d_ws);
    GridWs g = grid_ws(base, L.grid, &sc->grid, sc->n_N);
    GridParams gp = make_params(&sc->grid);
    const int nN = sc->n_N, nS = sc->n_S;
    float *ub[2] = {reinterpret_cast<float *>(base + L.u[0]), reinterpret_cast<float *>(base + L.u[1])};
    float *tau = reinterpret_cast<float *>(base + L.tau);
    float *C9 = reinterpret_cast<float *>(base + L.C);
    float *dnext = reinterpret_cast<float *>(base + L.dnext);
    const float *Xoff = f->dev.residual_g ? sc->d_X : nullptr;
    // ub[1] holds g(X, z_prev) between calls; step s writes g(X, z_n) to ub[s & 1 ^ 0]
    // and reads g(X, z_{n-1}) from the other buffer.
    const bool reuse = (flags & NSF_LATENT_REUSE_PREV) != 0;
    int cur = 0;
    // Stage events; under stream capture they become external event-record
    // nodes so that they still time each replay.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (taps) NSF_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
    const unsigned ev_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                   : cudaEventRecordDefault;
    auto ev = [&](bool on, void *const *arr, int stage) -> cudaError_t {
        if (!on || !arr[stage]) return cudaSuccess;
        return cudaEventRecordWithFlags(static_cast<cudaEvent_t>(arr[stage]), s, ev_flags);
    };
    for (int step = 0; step < nsteps; ++step) {
        const bool last = step == nsteps - 1;
        const bool tev = last && taps;
        float *u_n = ub[cur], *u_prev = ub[cur ^ 1];
        // 1. inference (§5.1)
        FieldJob jobs[4] = {{NSF_FIELD_G, d_z, u_n}, {NSF_FIELD_H, d_z, tau}, {NSF_FIELD_L, d_z, C9},
                            {NSF_FIELD_G, d_z_prev, u_prev}};
        const int njobs = (step == 0 && !reuse) ? 4 : 3;
        NSF_CUDA_TRY(ev(tev, tev ? taps->ev_begin : nullptr, NSF_STAGE_INFERENCE));
        NSF_CUDA_TRY(run_fields(f->dev, sc->d_X, nN, nN, njobs, jobs, d_status, s));
        NSF_CUDA_TRY(ev(tev, tev ? taps->ev_end : nullptr, NSF_STAGE_INFERENCE));
        // 2. MPM step on N (§5.2): binning, P2G, grid update and G2P on S
        P2gLatentArgs pa;
        pa.X = Xoff;
        pa.u = u_n;
        pa.u_prev = u_prev;
        pa.tau6 = tau;
        pa.C9 = C9;
        pa.n = nN;
        pa.mass = sc->mass;
        pa.vol0 = sc->vol0;
        pa.inv_dt = (float)(1.0 / dt);
        pa.dt = (float)dt;
        NSF_CUDA_TRY(ev(tev, tev ? taps->ev_begin : nullptr, NSF_STAGE_MPM));
        NSF_CUDA_TRY(launch_mpm_latent(g, gp, pa, nS, t0 + step * dt, dnext,
                                       last && taps ? taps->grid_mp : nullptr,
                                       last && taps ? taps->grid_v : nullptr, d_status, s));
        NSF_CUDA_TRY(ev(tev, tev ? taps->ev_end : nullptr, NSF_STAGE_MPM));
        if (last && taps) {
            if (taps->u_n) NSF_CUDA_TRY(cudaMemcpyAsync(taps->u_n, u_n, 12 * (size_t)nN, cudaMemcpyDeviceToDevice, s));
            if (taps->u_prev) NSF_CUDA_TRY(cudaMemcpyAsync(taps->u_prev, u_prev, 12 * (size_t)nN, cudaMemcpyDeviceToDevice, s));
            if (taps->u_next_S) NSF_CUDA_TRY(cudaMemcpyAsync(taps->u_next_S, dnext, 12 * (size_t)nS, cudaMemcpyDeviceToDevice, s));
            if (taps->tau6) NSF_CUDA_TRY(cudaMemcpyAsync(taps->tau6, tau, 24 * (size_t)nN, cudaMemcpyDeviceToDevice, s));
            if (taps->C9) NSF_CUDA_TRY(cudaMemcpyAsync(taps->C9, C9, 36 * (size_t)nN, cudaMemcpyDeviceToDevice, s));
        }
        // 3. network inversion (§5.3), Gauss-Newton from z_n
        NSF_CUDA_TRY(ev(tev, tev ? taps->ev_begin : nullptr, NSF_STAGE_GN));
        {
            GnArgs gn = gn_args(base, L.gn);
            gn.target = dnext;
            gn.target_ld = nS;
            gn.iters = opts->iters;
            gn.z_start = d_z;
            gn.z_out = d_z;
            gn.z_prev_out = d_z_prev;
            gn.z_taps = (last && taps) ? taps->z_iter : nullptr;
            gn.damping = opts->damping;
            NSF_CUDA_TRY(run_jacobian(f->dev, sc->d_X, nS, nN, d_z, nullptr, nullptr, &gn, d_status, s));
        }
        NSF_CUDA_TRY(ev(tev, tev ? taps->ev_end : nullptr, NSF_STAGE_GN));
        cur ^= 1;
    }
    // keep g(X, z_prev) of the returned z_prev in ub[1] for a NSF_LATENT_REUSE_PREV call
    if (((nsteps - 1) & 1) == 0)
        NSF_CUDA_TRY(cudaMemcpyAsync(ub[1], ub[0], 12 * (size_t)nN, cudaMemcpyDeviceToDevice, s));
    return NSF_OK;
}

nsf_status nsf_project_workspace_size(const nsf_fields *f, int n_S, size_t *bytes) {
    if (!f || !bytes || n_S < 1) return NSF_ERR_INVALID_ARG;
    *bytes = project_layout(f, n_S).total;
    return NSF_OK;
}

nsf_status nsf_project(const nsf_fields *f, const float *d_X_S, const float *d_x_target, int n_S,
                       double *d_z_inout, const nsf_gn_opts *opts, double *d_z_iter,
                       float *d_residual, void *d_ws, size_t ws_bytes, int *d_status,
                       void *stream) {
    if (!f || !d_X_S || !d_x_target || n_S < 1 || !d_z_inout || !valid_gn(opts))
        return NSF_ERR_INVALID_ARG;
    if (!f->infer_ok) return NSF_ERR_UNSUPPORTED;
    ProjectLayout L = project_layout(f, n_S);
    if (!d_ws || ws_bytes < L.total) return NSF_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(d_ws);
    float *target = reinterpret_cast<float *>(base + L.target);
    float *u = reinterpret_cast<float *>(base + L.u);
    // residual fields work on displacements: d = x_target - X
    if (f->dev.residual_g) NSF_CUDA_TRY(axpy(target, d_x_target, d_X_S, -1.f, 3 * n_S, s));
    else NSF_CUDA_TRY(cudaMemcpyAsync(target, d_x_target, 12 * (size_t)n_S, cudaMemcpyDeviceToDevice, s));
    {
        GnArgs gn = gn_args(base, L.gn);
        gn.target = target;
        gn.target_ld = n_S;
        gn.iters = opts->iters;
        gn.z_start = d_z_inout;
        gn.z_out = d_z_inout;
        gn.z_prev_out = nullptr;
        gn.z_taps = d_z_iter;
        gn.damping = opts->damping;
        NSF_CUDA_TRY(run_jacobian(f->dev, d_X_S, n_S, n_S, d_z_inout, nullptr, nullptr, &gn, d_status, s));
    }
    if (d_residual) {
        FieldJob job{NSF_FIELD_G, d_z_inout, u};
        NSF_CUDA_TRY(run_fields(f->dev, d_X_S, n_S, n_S, 1, &job, d_status, s));
        NSF_CUDA_TRY(axpy(d_residual, u, target, -1.f, 3 * n_S, s));
    }
    return NSF_OK;
}

}  // extern "C"

namespace {
struct SubsetLayout {
    size_t u, bitmap, in_S, bcount, boff, total;
    size_t bitmap_bytes;
};

SubsetLayout subset_layout(const nsf_grid_desc *g, int n) {
    Carver c;
    SubsetLayout L;
    const size_t nodes = (size_t)g->n[0] * g->n[1] * g->n[2];
    const size_t nb = ((size_t)n + 255) / 256;
    L.u = c.take(3 * (size_t)n * 4);
    L.bitmap_bytes = (nodes + 31) / 32 * 4;
    L.bitmap = c.take(L.bitmap_bytes);
    L.in_S = c.take((size_t)n);
    L.bcount = c.take(nb * 4);
    L.boff = c.take(nb * 4);
    L.total = c.off;
    return L;
}
}  // namespace

extern "C" {

nsf_status nsf_field_weight_count(const nsf_fields *f, int field, size_t *count) {
    if (!f || field < 0 || field > 2 || !count) return NSF_ERR_INVALID_ARG;
    const int r = f->desc.r, W = f->desc.width[field], D = f->desc.depth[field];
    size_t c = 0;
    for (int l = 0; l <= D; ++l) {
        const int in = l == 0 ? 3 + r : W, out = l == D ? kOutDim[field] : W;
        c += (size_t)in * out + out;
    }
    *count = c;
    return NSF_OK;
}

nsf_status nsf_train_workspace_size(const nsf_fields *f, int field, int n, size_t *bytes) {
    if (!f || field < 0 || field > 2 || n < 1 || !bytes) return NSF_ERR_INVALID_ARG;
    *bytes = train_layout(f->desc.r, f->desc.width[field], f->desc.depth[field], kOutDim[field],
                          n).total;
    return NSF_OK;
}

nsf_status nsf_field_loss_grad(const nsf_fields *f, int field, const float *d_X, const int *d_code,
                               const float *d_target, int n, const float *d_z_table, int n_codes,
                               float *d_loss, float *d_grad_w, float *d_grad_z, void *d_ws,
                               size_t ws_bytes, int *d_status, void *stream) {
    if (!f || field < 0 || field > 2 || !d_X || !d_code || !d_target || n < 1 || !d_z_table ||
        n_codes < 1 || !d_loss || !d_grad_w)
        return NSF_ERR_INVALID_ARG;
    const TrainLayout L = train_layout(f->desc.r, f->desc.width[field], f->desc.depth[field],
                                       kOutDim[field], n);
    if (!d_ws || ws_bytes < L.total) return NSF_ERR_WORKSPACE;
    cudaError_t e = run_loss_grad(f->dev, field, d_X, d_code, d_target, n, d_z_table, n_codes,
                                  d_loss, d_grad_w, d_grad_z, static_cast<char *>(d_ws), d_status,
                                  static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? NSF_OK : NSF_ERR_CUDA;
}

nsf_status nsf_adam_step(float *d_param, const float *d_grad, float *d_m, float *d_v, size_t count,
                         int step, float lr, float beta1, float beta2, float eps, void *stream) {
    if (!d_param || !d_grad || !d_m || !d_v || step < 1 || !(lr >= 0.f) || !(beta1 >= 0.f) ||
        !(beta1 < 1.f) || !(beta2 >= 0.f) || !(beta2 < 1.f) || !(eps >= 0.f))
        return NSF_ERR_INVALID_ARG;
    if (count == 0) return NSF_OK;
    NSF_CUDA_TRY(launch_adam(d_param, d_grad, d_m, d_v, (long long)count, step, lr, beta1, beta2,
                             eps, static_cast<cudaStream_t>(stream)));
    return NSF_OK;
}

nsf_status nsf_fields_set_weights(nsf_fields *f, int field, const float *d_weights, void *stream) {
    if (!f || field < 0 || field > 2 || !d_weights) return NSF_ERR_INVALID_ARG;
    NSF_CUDA_TRY(launch_repack(f->dev, field, d_weights, static_cast<cudaStream_t>(stream)));
    return NSF_OK;
}

nsf_status nsf_integration_set_workspace_size(const nsf_grid_desc *grid, int n_all,
                                              size_t *bytes) {
    if (!valid_grid(grid) || n_all < 1 || !bytes) return NSF_ERR_INVALID_ARG;
    *bytes = subset_layout(grid, n_all).total;
    return NSF_OK;
}

nsf_status nsf_integration_set(const nsf_fields *f, const nsf_grid_desc *grid, const float *d_X,
                               int n_all, const int *d_sample, int n_S, const double *d_z,
                               int *d_index_out, int *d_count_out, float *d_X_out, int x_out_ld,
                               void *d_ws, size_t ws_bytes, int *d_status, void *stream) {
    if (!f || !valid_grid(grid) || !d_X || n_all < 1 || n_S < 0 || n_S > n_all ||
        (n_S > 0 && !d_sample) || !d_z || !d_index_out || !d_count_out ||
        (d_X_out && x_out_ld < n_all))
        return NSF_ERR_INVALID_ARG;
    if (!f->infer_ok) return NSF_ERR_UNSUPPORTED;
    const SubsetLayout L = subset_layout(grid, n_all);
    if (!d_ws || ws_bytes < L.total) return NSF_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(d_ws);
    float *u = reinterpret_cast<float *>(base + L.u);
    NSF_CUDA_TRY(cudaMemsetAsync(base + L.bitmap, 0, L.bitmap_bytes, s));
    NSF_CUDA_TRY(cudaMemsetAsync(base + L.in_S, 0, (size_t)n_all, s));
    FieldJob job{NSF_FIELD_G, d_z, u};
    NSF_CUDA_TRY(run_fields(f->dev, d_X, n_all, n_all, 1, &job, d_status, s));
    SubsetArgs a;
    a.X = d_X;
    a.u = u;
    a.residual = f->dev.residual_g;
    a.n = n_all;
    a.sample = d_sample;
    a.n_S = n_S;
    for (int d = 0; d < 3; ++d) a.dims[d] = grid->n[d];
    a.inv_dx = 1.f / grid->dx;
    a.bitmap = reinterpret_cast<unsigned *>(base + L.bitmap);
    a.in_S = reinterpret_cast<unsigned char *>(base + L.in_S);
    a.block_count = reinterpret_cast<int *>(base + L.bcount);
    a.block_off = reinterpret_cast<int *>(base + L.boff);
    a.index_out = d_index_out;
    NSF_CUDA_TRY(launch_subset(a, d_count_out, d_X_out, x_out_ld, d_status, s));
    return NSF_OK;
}

nsf_status nsf_material_stress(const nsf_material *mat, const float *d_F, int n, float *d_tau6,
                               void *stream) {
    if (!mat || n < 0 || (n > 0 && (!d_F || !d_tau6)) || !(mat->E > 0.f) || !(mat->nu > -1.f) ||
        !(mat->nu < 0.5f) || mat->model < NSF_NEO_HOOKEAN || mat->model > NSF_DRUCKER_PRAGER)
        return NSF_ERR_INVALID_ARG;
    const float mu = mat->E / (2.f * (1.f + mat->nu));
    const float lam = mat->E * mat->nu / ((1.f + mat->nu) * (1.f - 2.f * mat->nu));
    NSF_CUDA_TRY(launch_stress(d_F, d_tau6, n, mat->model, mu, lam,
                               static_cast<cudaStream_t>(stream)));
    return NSF_OK;
}

nsf_status nsf_full_workspace_size(const nsf_grid_desc *g, int n, size_t *bytes) {
    if (!valid_grid(g) || n < 1 || !bytes) return NSF_ERR_INVALID_ARG;
    *bytes = full_layout(g, n).total;
    return NSF_OK;
}

nsf_status nsf_full_step(const nsf_grid_desc *grid, const nsf_material *mat,
                         const nsf_particles *P, double dt, double t0, int nsteps, void *d_ws,
                         size_t ws_bytes, int *d_status, const nsf_full_taps *taps,
                         void *stream) {
    if (!valid_grid(grid) || !mat || !P || P->n < 1 || !P->d_x || !P->d_v || !P->d_C || !P->d_F ||
        nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(t0) ||
        !(P->mass > 0.f) || !(P->vol0 > 0.f) || !(mat->E > 0.f) || !(mat->nu > -1.f) ||
        !(mat->nu < 0.5f))
        return NSF_ERR_INVALID_ARG;
    if (mat->model < NSF_NEO_HOOKEAN || mat->model > NSF_DRUCKER_PRAGER) return NSF_ERR_INVALID_ARG;
    if (mat->model == NSF_VON_MISES && !(mat->yield_stress > 0.f)) return NSF_ERR_INVALID_ARG;
    if (mat->model == NSF_DRUCKER_PRAGER &&
        !(mat->friction_deg > 0.f && mat->friction_deg < 90.f))
        return NSF_ERR_INVALID_ARG;
    if (nsteps == 0) return NSF_OK;
    FullLayout L = full_layout(grid, P->n);
    if (!d_ws || ws_bytes < L.total) return NSF_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(d_ws);
    GridWs g = grid_ws(base, L.grid, grid, P->n);
    GridParams gp = make_params(grid);
    const float mu = mat->E / (2.f * (1.f + mat->nu));
    const float lam = mat->E * mat->nu / ((1.f + mat->nu) * (1.f - 2.f * mat->nu));
    // SVD-based models keep the float64 stress of F^E in the workspace: computed
    // here for the first step, then by every G2P after its return map
    const bool svd_model = mat->model != NSF_NEO_HOOKEAN;
    float *tau6 = svd_model ? reinterpret_cast<float *>(base + L.tau) : nullptr;
    if (svd_model) NSF_CUDA_TRY(launch_stress(P->d_F, tau6, P->n, mat->model, mu, lam, s));
    for (int step = 0; step < nsteps; ++step) {
        const bool last = step == nsteps - 1;
        P2gFullArgs pa;
        pa.x = P->d_x;
        pa.v = P->d_v;
        pa.C = P->d_C;
        pa.F = P->d_F;
        pa.tau6 = tau6;
        pa.n = P->n;
        pa.mass = P->mass;
        pa.vol0 = P->vol0;
        pa.dt = (float)dt;
        pa.mu = mu;
        pa.lam = lam;
        G2pFullArgs ga;
        ga.x = P->d_x;
        ga.v = P->d_v;
        ga.C = P->d_C;
        ga.F = P->d_F;
        ga.tau6 = tau6;
        ga.n = P->n;
        ga.dt = (float)dt;
        ga.model = mat->model;
        ga.mu = mu;
        ga.lam = lam;
        ga.yield_stress = mat->yield_stress;
        ga.friction_deg = mat->friction_deg;
        NSF_CUDA_TRY(launch_mpm_full(g, gp, pa, ga, t0 + step * dt,
                                     last && taps ? taps->grid_mp : nullptr,
                                     last && taps ? taps->grid_v : nullptr, d_status, s));
    }
    return NSF_OK;
}

}  // extern "C"

// ================================================================ batches ===
// Batched latent stepping (nsf_latent_step_batched): host-side plan.
namespace nsf {
size_t jac_tc_smem_bytes(int r, int width, int depth);
}

namespace {

// u[1] <- u[0] for every scene (flat index over the scenes' 3 n_N values).
__global__ void k_batch_keep_prev(const BatchSceneDev *scenes, const int *n_off, int ns) {
    const int total = 3 * n_off[ns];
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        int lo = 0, hi = ns;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (3 * n_off[mid] <= q) lo = mid;
            else hi = mid;
        }
        const BatchSceneDev &sc = scenes[lo];
        const int i = q - 3 * n_off[lo];
        sc.u[1][i] = sc.u[0][i];
    }
}

bool valid_batch_item(const nsf_latent_batch_item &it) {
    const nsf_latent_scene *sc = &it.scene;
    return it.fields && it.d_z && it.d_z_prev && sc->d_X && sc->n_N >= 1 && sc->n_S >= 1 &&
           sc->n_S <= sc->n_N && valid_grid(&sc->grid) && it.dt > 0.0 && std::isfinite(it.dt) &&
           sc->mass > 0.f && sc->vol0 > 0.f;
}

// Per-scene layouts inside the batch workspace, after a 256-byte control block
// (the MPM launch's grid-barrier word).
struct BatchLayout {
    std::vector<size_t> base;
    std::vector<LatentLayout> scene;
    size_t total;
};

BatchLayout batch_layout(int n, const nsf_latent_batch_item *items) {
    BatchLayout B;
    size_t off = align_up(256);
    for (int i = 0; i < n; ++i) {
        LatentLayout L = latent_layout(items[i].fields, &items[i].scene, kBucketCapBatch);
        B.base.push_back(off);
        B.scene.push_back(L);
        off = align_up(off + L.total);
    }
    B.total = off;
    return B;
}

// Work lists of one field width: jobs cut into runs of tiles so that every
// CTA gets about the same cost (tiles x depth), in job order.
struct WidthPlan {
    int W = 0, maxD = 1, nctas = 0;
    std::vector<FieldBatchItem> items;
    std::vector<int> cta_item;     // nctas + 1 offsets
};

WidthPlan plan_width(int W, int n, const nsf_latent_batch_item *items, bool with_prev, int sms) {
    WidthPlan P;
    P.W = W;
    struct Job { int scene, field, zsel, tiles, depth; };
    std::vector<Job> jobs;
    double total = 0.0;
    for (int s = 0; s < n; ++s) {
        const nsf_fields_desc &d = items[s].fields->desc;
        const int tiles = (items[s].scene.n_N + 127) / 128;
        for (int f = 0; f < 3; ++f) {
            if (d.width[f] != W) continue;
            P.maxD = d.depth[f] > P.maxD ? d.depth[f] : P.maxD;
            jobs.push_back({s, f, 0, tiles, d.depth[f]});
            total += (double)tiles * d.depth[f];
            if (f == NSF_FIELD_G && with_prev) {
                jobs.push_back({s, f, 1, tiles, d.depth[f]});
                total += (double)tiles * d.depth[f];
            }
        }
    }
    long long all_tiles = 0;
    for (const Job &j : jobs) all_tiles += j.tiles;
    if (all_tiles == 0) return P;
    P.nctas = (int)(all_tiles < sms ? all_tiles : sms);
    const double target = total / P.nctas;
    std::vector<std::vector<FieldBatchItem>> per(P.nctas);
    double cum = 0.0;
    for (const Job &j : jobs) {
        int t = 0;
        while (t < j.tiles) {
            int cta = (int)((cum + 0.5 * j.depth) / target);
            if (cta >= P.nctas) cta = P.nctas - 1;
            // extend the run while the tiles fall to the same CTA
            int t1 = t + 1;
            double c = cum + j.depth;
            while (t1 < j.tiles) {
                int c2 = (int)((c + 0.5 * j.depth) / target);
                if (c2 >= P.nctas) c2 = P.nctas - 1;
                if (c2 != cta) break;
                ++t1;
                c += j.depth;
            }
            per[cta].push_back({j.scene, j.field, j.zsel, t, t1});
            cum = c;
            t = t1;
        }
    }
    P.cta_item.push_back(0);
    for (int c = 0; c < P.nctas; ++c) {
        for (const FieldBatchItem &it : per[c]) P.items.push_back(it);
        P.cta_item.push_back((int)P.items.size());
    }
    return P;
}

// Gauss-Newton CTA schedule.  A scene whose cost is above a threshold T is
// split over ceil(cost / T) CTAs (a group that combines its sums behind the
// scene's barrier) and is the FIRST entry of each of them, so that every
// member of a group reaches the group's barriers while inside that scene.
// The other scenes are then packed whole, longest first, each after the least
// loaded CTA's entries.  T is searched between half a CTA share and two
// shares for the smallest estimated makespan.
struct GnPlan {
    std::vector<int> cw;
    int batch_cw = 0;
    std::vector<GnBatchEntry> entries;
    std::vector<int> cta_entry;
    int nctas = 0;
    size_t smem = 0;
};

int jac_slots_host(int r) {
    int L = 2;
    while (L < 1 + r) L <<= 1;
    return L;
}

// Relative cost of one point through one layer of the batched Jacobian kernel
// with L slots a point and hidden width W.  A 256-slot tile costs about the
// same at every L, so per point the cost follows L; widths above 64 add
// ~14 % (a longer product), above 128 twice that again (a second 128-neuron
// product).  Fitted to GB300 timings of single-CTA scenes: 1 : 1.97 : 3.89
// for L = 8, 16, 32 at W = 64, and 1.10 : 2.30 : 4.41 at W = 128.
double jac_point_layer_cost(int L, int W) {
    return (double)L / 8.0 * (W > 64 ? 1.14 : 1.0) * (W > 128 ? 2.0 : 1.0);
}

// A scene split over g CTAs costs each of them a little more than cost / g
// (its group barriers and the combine of its sums).
constexpr double kGnSplitOverhead = 1.03;

GnPlan plan_gn(int n, const nsf_latent_batch_item *items, int sms, int want_cw, double split) {
    GnPlan G;
    std::vector<double> cost(n);
    std::vector<int> tiles(n);
    double total = 0.0;
    // one column width for the whole launch: the narrowest any scene needs,
    // or the requested one where every scene's operands fit
    G.batch_cw = 0;
    for (int s = 0; s < n; ++s) {
        const nsf_fields_desc &d = items[s].fields->desc;
        const int cw = jac_batch_cw(d.r, d.width[NSF_FIELD_G], d.depth[NSF_FIELD_G]);
        if (G.batch_cw == 0 || cw < G.batch_cw) G.batch_cw = cw;
        if (want_cw && (want_cw < jac_slots_host(d.r) ||
                        !jac_tc_smem_bytes_cw(d.r, d.width[NSF_FIELD_G], d.depth[NSF_FIELD_G],
                                              want_cw, jac_batch_wg())))
            G.batch_cw = -1;
    }
    if (want_cw) {
        if (G.batch_cw < 0) return G;        // not every scene fits: an empty plan
        G.batch_cw = want_cw;
    }
    for (int s = 0; s < n; ++s) {
        const nsf_fields_desc &d = items[s].fields->desc;
        const int W = d.width[NSF_FIELD_G], D = d.depth[NSF_FIELD_G];
        const int cw = G.batch_cw;
        G.cw.push_back(cw);
        const int P = jac_batch_points(d.r, cw);
        tiles[s] = (items[s].scene.n_S + P - 1) / P;
        // a group is no larger than the scene's Gauss-Newton slots hold
        const int slots = jac_grid_size_tc(items[s].fields->dev, items[s].scene.n_S);
        if (tiles[s] > slots) tiles[s] = slots;
        cost[s] = (double)items[s].scene.n_S * (D + 1) * jac_point_layer_cost(jac_slots_host(d.r), W);
        total += cost[s];
        const size_t sm = jac_tc_smem_bytes_cw(d.r, W, D, cw, jac_batch_wg());
        G.smem = sm > G.smem ? sm : G.smem;
    }
    const int cap = sms < kGnMaxCtas ? sms : kGnMaxCtas;
    const double share = total / cap;
    std::vector<int> order(n);
    for (int s = 0; s < n; ++s) order[s] = s;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });

    // the plan for threshold T and its estimated makespan
    auto plan_for = [&](double T, std::vector<std::vector<GnBatchEntry>> &per) -> double {
        per.assign(cap, {});
        std::vector<double> load(cap, 0.0);
        std::vector<int> group(n, 1);
        int used = 0;
        for (int s : order) {
            if (cost[s] <= T) continue;
            int g = (int)std::ceil(cost[s] / T);
            if (g > tiles[s]) g = tiles[s];
            if (g < 2 || used + g > cap) continue;
            group[s] = g;
            for (int k = 0; k < g; ++k) {
                per[used + k].push_back(GnBatchEntry{s, k, g});
                load[used + k] = cost[s] / g * kGnSplitOverhead;
            }
            used += g;
        }
        // least loaded CTA first (min-heap on load, then index)
        using Slot = std::pair<double, int>;
        std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
        for (int c = 0; c < cap; ++c) heap.push({load[c], c});
        for (int s : order) {
            if (group[s] > 1) continue;
            Slot top = heap.top();
            heap.pop();
            per[top.second].push_back(GnBatchEntry{s, 0, 1});
            top.first += cost[s];
            heap.push(top);
        }
        double span = 0.0;
        for (int c = 0; c < cap; ++c) span = std::max(span, load[c]);
        while (!heap.empty()) {
            span = std::max(span, heap.top().first);
            heap.pop();
        }
        // CTAs without entries are not launched
        per.erase(std::remove_if(per.begin(), per.end(),
                                 [](const std::vector<GnBatchEntry> &v) { return v.empty(); }),
                  per.end());
        return span;
    };

    std::vector<std::vector<GnBatchEntry>> per, trial;
    double best = plan_for(split > 0.0 ? share * split : share, per);
    for (int k = 0; k <= 150 && split <= 0.0; ++k) {
        const double span = plan_for(share * (0.5 + 0.01 * k), trial);
        if (span < best) {
            best = span;
            per.swap(trial);
        }
    }
    G.nctas = (int)per.size();
    G.cta_entry.push_back(0);
    for (auto &v : per) {
        for (auto &e : v) G.entries.push_back(e);
        G.cta_entry.push_back((int)G.entries.size());
    }
    return G;
}

// Device tables of a plan, laid out in one allocation.
struct TableCarver {
    size_t off = 0;
    template <class T>
    size_t take(size_t count) {
        size_t o = align_up(off);
        off = o + count * sizeof(T);
        return o;
    }
};

}  // namespace

struct nsf_latent_batch {
    int n;
    nsf_gn_opts opts;
    void *d_mem;
    BatchSceneDev *scenes;
    int *n_off, *s_off;
    unsigned *mpm_bar;
    struct Width {
        int W, maxD;
        int nctas[2];                 // [0]: g, h, l per scene; [1]: plus g at z_prev
        FieldBatchItem *items[2];
        int *cta_item[2];
    };
    std::vector<Width> widths;
    GnBatchProblem *probs;
    GnBatchEntry *entries;
    int *cta_entry;
    int gn_ctas;
    size_t gn_smem;
    int gn_cw;
    int p2g_group;
};

extern "C" {

nsf_status nsf_latent_batch_workspace_size(int n, const nsf_latent_batch_item *items,
                                           size_t *bytes) {
    if (n < 1 || n > NSF_MAX_BATCH || !items || !bytes) return NSF_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!items[i].fields || items[i].scene.n_N < 1 || items[i].scene.n_S < 1 ||
            items[i].scene.n_S > items[i].scene.n_N || !valid_grid(&items[i].scene.grid))
            return NSF_ERR_INVALID_ARG;
    *bytes = batch_layout(n, items).total;
    return NSF_OK;
}

nsf_status nsf_latent_batch_create(int n, const nsf_latent_batch_item *items,
                                   const nsf_gn_opts *opts, void *d_ws, size_t ws_bytes,
                                   nsf_latent_batch **out) {
    return nsf_latent_batch_create_tuned(n, items, opts, nullptr, d_ws, ws_bytes, out);
}

nsf_status nsf_latent_batch_create_tuned(int n, const nsf_latent_batch_item *items,
                                         const nsf_gn_opts *opts, const nsf_batch_tuning *tuning,
                                         void *d_ws, size_t ws_bytes, nsf_latent_batch **out) {
    if (!out || n < 1 || n > NSF_MAX_BATCH || n > kMaxBatchScenes || !items || !valid_gn(opts))
        return NSF_ERR_INVALID_ARG;
    nsf_batch_tuning tu{0, 0.0, 0};
    if (tuning) tu = *tuning;
    if ((tu.gn_columns != 0 && tu.gn_columns != 32 && tu.gn_columns != 64) ||
        !(tu.gn_split >= 0.0) || !std::isfinite(tu.gn_split) ||
        (tu.p2g_group != 0 && tu.p2g_group != 64 && tu.p2g_group != 128))
        return NSF_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!valid_batch_item(items[i])) return NSF_ERR_INVALID_ARG;
        const nsf_fields_desc &d = items[i].fields->desc;
        if (d.precision != NSF_PREC_BF16 || !items[i].fields->infer_ok) return NSF_ERR_UNSUPPORTED;
    }
    const BatchLayout BL = batch_layout(n, items);
    if (!d_ws || ws_bytes < BL.total) return NSF_ERR_WORKSPACE;
    char *ws = static_cast<char *>(d_ws);
    const int sms = tc::sm_count();

    // distinct fields objects
    std::vector<const nsf_fields *> fobj;
    std::vector<int> fidx(n);
    for (int i = 0; i < n; ++i) {
        int k = -1;
        for (size_t j = 0; j < fobj.size(); ++j)
            if (fobj[j] == items[i].fields) k = (int)j;
        if (k < 0) {
            k = (int)fobj.size();
            fobj.push_back(items[i].fields);
        }
        fidx[i] = k;
    }
    // work lists
    std::vector<WidthPlan> wp[2];
    static const int kWidths[4] = {64, 128, 192, 256};
    for (int w : kWidths)
        for (int set = 0; set < 2; ++set) {
            WidthPlan P = plan_width(w, n, items, set == 1, sms);
            if (P.nctas > 0) wp[set].push_back(P);
        }
    const GnPlan G = plan_gn(n, items, sms, tu.gn_columns, tu.gn_split);
    if (G.batch_cw <= 0) return NSF_ERR_INVALID_ARG;     // a requested width that does not fit

    // table layout
    TableCarver tc_;
    const size_t o_fd = tc_.take<FieldsDev>(fobj.size());
    const size_t o_sc = tc_.take<BatchSceneDev>(n);
    const size_t o_no = tc_.take<int>(n + 1), o_so = tc_.take<int>(n + 1);
    size_t o_items[2][4], o_cta[2][4];
    for (int set = 0; set < 2; ++set)
        for (size_t k = 0; k < wp[set].size(); ++k) {
            o_items[set][k] = tc_.take<FieldBatchItem>(wp[set][k].items.size());
            o_cta[set][k] = tc_.take<int>(wp[set][k].cta_item.size());
        }
    const size_t o_pr = tc_.take<GnBatchProblem>(n);
    const size_t o_en = tc_.take<GnBatchEntry>(G.entries.size());
    const size_t o_ce = tc_.take<int>(G.cta_entry.size());
    const size_t tbytes = align_up(tc_.off);
    std::vector<char> h(tbytes, 0);
    void *mem = nullptr;
    if (cudaMalloc(&mem, tbytes) != cudaSuccess) {
        cudaGetLastError();
        return NSF_ERR_NO_MEMORY;
    }
    char *dm = static_cast<char *>(mem);
    auto put = [&](size_t off, const void *src, size_t bytes) { std::memcpy(h.data() + off, src, bytes); };

    for (size_t j = 0; j < fobj.size(); ++j) put(o_fd + j * sizeof(FieldsDev), &fobj[j]->dev, sizeof(FieldsDev));
    std::vector<int> noff(n + 1, 0), soff(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        const nsf_latent_batch_item &it = items[i];
        const LatentLayout &L = BL.scene[i];
        char *base = ws + BL.base[i];
        BatchSceneDev sd;
        std::memset(&sd, 0, sizeof(sd));
        sd.fd = reinterpret_cast<const FieldsDev *>(dm + o_fd + fidx[i] * sizeof(FieldsDev));
        sd.X = it.scene.d_X;
        sd.n_N = it.scene.n_N;
        sd.n_S = it.scene.n_S;
        sd.mass = it.scene.mass;
        sd.vol0 = it.scene.vol0;
        sd.dt = (float)it.dt;
        sd.inv_dt = (float)(1.0 / it.dt);
        sd.residual_g = it.fields->dev.residual_g;
        sd.u[0] = reinterpret_cast<float *>(base + L.u[0]);
        sd.u[1] = reinterpret_cast<float *>(base + L.u[1]);
        sd.tau6 = reinterpret_cast<float *>(base + L.tau);
        sd.C9 = reinterpret_cast<float *>(base + L.C);
        sd.dnext = reinterpret_cast<float *>(base + L.dnext);
        sd.z = it.d_z;
        sd.z_prev = it.d_z_prev;
        sd.g = grid_ws(base, L.grid, &it.scene.grid, it.scene.n_N);
        sd.gp = make_params(&it.scene.grid);
        put(o_sc + i * sizeof(BatchSceneDev), &sd, sizeof(sd));
        noff[i + 1] = noff[i] + it.scene.n_N;
        soff[i + 1] = soff[i] + it.scene.n_S;

        GnBatchProblem pb;
        std::memset(&pb, 0, sizeof(pb));
        pb.fd = sd.fd;
        pb.X = it.scene.d_X;
        pb.n = it.scene.n_S;
        pb.ld = it.scene.n_N;
        pb.cw = G.cw[i];
        pb.gn = gn_args(base, L.gn);
        pb.gn.target = sd.dnext;
        pb.gn.target_ld = it.scene.n_S;
        pb.gn.iters = opts->iters;
        pb.gn.z_start = it.d_z;
        pb.gn.z_out = it.d_z;
        pb.gn.z_prev_out = it.d_z_prev;
        pb.gn.z_taps = nullptr;
        pb.gn.damping = opts->damping;
        put(o_pr + i * sizeof(GnBatchProblem), &pb, sizeof(pb));
    }
    if (noff[n] > (1 << 30) / 3) {
        cudaFree(mem);
        return NSF_ERR_INVALID_ARG;
    }
    put(o_no, noff.data(), (n + 1) * sizeof(int));
    put(o_so, soff.data(), (n + 1) * sizeof(int));
    for (int set = 0; set < 2; ++set)
        for (size_t k = 0; k < wp[set].size(); ++k) {
            put(o_items[set][k], wp[set][k].items.data(), wp[set][k].items.size() * sizeof(FieldBatchItem));
            put(o_cta[set][k], wp[set][k].cta_item.data(), wp[set][k].cta_item.size() * sizeof(int));
        }
    put(o_en, G.entries.data(), G.entries.size() * sizeof(GnBatchEntry));
    put(o_ce, G.cta_entry.data(), G.cta_entry.size() * sizeof(int));
    if (cudaMemcpy(mem, h.data(), tbytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(mem);
        return NSF_ERR_CUDA;
    }
    nsf_latent_batch *B = new (std::nothrow) nsf_latent_batch;
    if (!B) {
        cudaFree(mem);
        return NSF_ERR_NO_MEMORY;
    }
    B->n = n;
    B->opts = *opts;
    B->d_mem = mem;
    B->scenes = reinterpret_cast<BatchSceneDev *>(dm + o_sc);
    B->n_off = reinterpret_cast<int *>(dm + o_no);
    B->s_off = reinterpret_cast<int *>(dm + o_so);
    B->mpm_bar = reinterpret_cast<unsigned *>(ws);
    // width classes: the same widths appear in both sets
    for (size_t k = 0; k < wp[0].size(); ++k) {
        nsf_latent_batch::Width w;
        w.W = wp[0][k].W;
        w.maxD = wp[0][k].maxD;
        for (int set = 0; set < 2; ++set) {
            w.nctas[set] = wp[set][k].nctas;
            w.items[set] = reinterpret_cast<FieldBatchItem *>(dm + o_items[set][k]);
            w.cta_item[set] = reinterpret_cast<int *>(dm + o_cta[set][k]);
        }
        B->widths.push_back(w);
    }
    B->probs = reinterpret_cast<GnBatchProblem *>(dm + o_pr);
    B->entries = reinterpret_cast<GnBatchEntry *>(dm + o_en);
    B->cta_entry = reinterpret_cast<int *>(dm + o_ce);
    B->gn_ctas = G.nctas;
    B->gn_smem = G.smem;
    B->gn_cw = G.batch_cw;
    B->p2g_group = tu.p2g_group ? tu.p2g_group : 64;
    *out = B;
    return NSF_OK;
}

void nsf_latent_batch_destroy(nsf_latent_batch *b) {
    if (!b) return;
    cudaFree(b->d_mem);
    delete b;
}

nsf_status nsf_latent_step_batched(const nsf_latent_batch *b, double t0, int nsteps,
                                   unsigned int flags, int *d_status,
                                   const nsf_batch_events *events, void *stream) {
    if (!b || nsteps < 0 || !std::isfinite(t0) || (flags & ~(unsigned)NSF_LATENT_REUSE_PREV))
        return NSF_ERR_INVALID_ARG;
    if (nsteps == 0) return NSF_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool reuse = (flags & NSF_LATENT_REUSE_PREV) != 0;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (events) NSF_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
    const unsigned ev_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                   : cudaEventRecordDefault;
    auto ev = [&](bool on, void *const *arr, int stage) -> cudaError_t {
        if (!on || !arr[stage]) return cudaSuccess;
        return cudaEventRecordWithFlags(static_cast<cudaEvent_t>(arr[stage]), s, ev_flags);
    };
    for (int step = 0; step < nsteps; ++step) {
        const bool tev = step == nsteps - 1 && events;
        const int parity = step & 1;
        const int set = (step == 0 && !reuse) ? 1 : 0;
        NSF_CUDA_TRY(ev(tev, tev ? events->ev_begin : nullptr, NSF_STAGE_INFERENCE));
        for (const auto &w : b->widths)
            NSF_CUDA_TRY(launch_fields_batch(w.W, b->scenes, w.items[set], w.cta_item[set],
                                             w.nctas[set], parity, w.maxD, d_status, s));
        NSF_CUDA_TRY(ev(tev, tev ? events->ev_end : nullptr, NSF_STAGE_INFERENCE));
        MpmBatchArgs ma;
        ma.scenes = b->scenes;
        ma.nscenes = b->n;
        ma.n_off = b->n_off;
        ma.s_off = b->s_off;
        ma.parity = parity;
        ma.t0 = t0;
        ma.step = step;
        ma.bar = b->mpm_bar;
        NSF_CUDA_TRY(ev(tev, tev ? events->ev_begin : nullptr, NSF_STAGE_MPM));
        NSF_CUDA_TRY(launch_mpm_batch(ma, b->p2g_group, d_status, s));
        NSF_CUDA_TRY(ev(tev, tev ? events->ev_end : nullptr, NSF_STAGE_MPM));
        NSF_CUDA_TRY(ev(tev, tev ? events->ev_begin : nullptr, NSF_STAGE_GN));
        NSF_CUDA_TRY(launch_jac_batch(b->probs, b->entries, b->cta_entry, b->gn_ctas, b->gn_smem,
                                      b->gn_cw, d_status, s));
        NSF_CUDA_TRY(ev(tev, tev ? events->ev_end : nullptr, NSF_STAGE_GN));
    }
    // keep every scene's g(X, z_prev) of the returned z_prev in u[1]
    if (((nsteps - 1) & 1) == 0) {
        k_batch_keep_prev<<<2 * tc::sm_count(), 256, 0, s>>>(b->scenes, b->n_off, b->n);
        NSF_CUDA_TRY(cudaGetLastError());
    }
    return NSF_OK;
}

}  // extern "C"
