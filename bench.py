"""Benchmark: latent MPM steps/s on one GB300 (and the full-order step beside it).

One "step" is one pass of the whole latent hot path: field inference on the
integration particles, binning, P2G, grid update, G2P on the sample particles
and the Gauss-Newton inversion (5 iterations).  Workload: the 200,000-particle
slab scene with 10,000 integration and 700 sample particles, r = 6, fields of
5 hidden layers x 128 (BF16 on the tensor cores), 128^3 grid.  Each step is one
replay of a CUDA graph of one nsf_latent_step call; L2 is flushed (a 512 MB
write) between timed steps and the flush is outside the timed events.

The full-order MLS-MPM step on the same 200,000-particle slab (neo-Hookean,
sticky blade) is timed the same way and reported as "full_order".
"matched_error" fits the fields to a full-order run of that slab with the
library's training path and compares the latent step's speed and sample
particle error (dx units) with the full-order step's, for 1, 2, 3 and 5
Gauss-Newton iterations.  "config1" is the 1,024-particle FP32 latent scene.

--impl reference times the FP64 CPU oracle instead (the reference arm of this
benchmark): the same workload and metric on the host cores.

Multi-GPU (torchrun): replicas only, one independent scene per rank, no
collective on the data path; value = all ranks' steps / max-over-ranks time.
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "latent steps/s vs full-order MPM steps/s on 1 GB300; % tensor/HBM roofline"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def mlp_macs(r, width, depth, out_dim):
    return (3 + r) * width + (depth - 1) * width * width + width * out_dim


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value, world, device=None):
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ GPU ---
def run_gpu(args, rank, world, local):
    import torch
    import paper_2310_17790_gb300 as nsf
    from paper_2310_17790_gb300 import _native as N
    from scenes.synthetic import full_config2, latent_config3

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    sc = latent_config3(precision=args.precision, steps=args.steps)
    fs = sc.fields
    F = nsf.Fields.from_spec(fs)
    X = torch.from_numpy(np.ascontiguousarray(sc.X.T)).to(dev)
    gd = nsf.grid_desc(sc.grid.n, sc.grid.dx, sc.grid.gravity, sc.grid.wall_cells)
    stp = nsf.LatentStepper(F, X, sc.n_S, sc.mass, sc.vol0, gd)
    z = torch.tensor(sc.z0, dtype=torch.float64, device=dev)
    zp = z.clone()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # stage events (recorded by the library inside the captured step)
    nst = N.NSF_LATENT_STAGES
    taps = N.nsf_latent_taps()
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(nst)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(nst)]
    with torch.cuda.stream(stream):
        for e in ev_b + ev_e:
            e.record(stream)
    torch.cuda.synchronize()
    for i in range(nst):
        taps.ev_begin[i] = ev_b[i].cuda_event
        taps.ev_end[i] = ev_e[i].cuda_event

    # first step fills the g(X, z_prev) cache; later steps reuse it
    with torch.cuda.stream(stream):
        stp.step(z, zp, sc.dt, nsteps=1, iters=sc.gn_iters, damping=sc.damping, stream=stream)
    torch.cuda.synchronize()
    # the timed graph records no events; a second graph with the stage events
    # (the library's taps) gives the per-stage split
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        stp.step(z, zp, sc.dt, nsteps=1, iters=sc.gn_iters, damping=sc.damping,
                 stream=stream, reuse_prev=True)
    torch.cuda.synchronize()
    graph_taps = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_taps, stream=stream):
        stp.step(z, zp, sc.dt, nsteps=1, iters=sc.gn_iters, damping=sc.damping, taps=taps,
                 stream=stream, reuse_prev=True)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        graph.replay()
        graph_taps.replay()
    torch.cuda.synchronize()
    assert stp.read_status() == 0, nsf.status_string(stp.read_status())
    # clocks are sampled (200 ms period) from here through the stage and
    # throughput runs.  A 1 s pre-roll of the same step lets the sampler see the
    # GPU under this load before the short timed loop; the scene state (z,
    # z_prev, workspace) is put back to the post-warm-up snapshot every 100
    # replays and at the end, so the timed steps start where they would have.
    clocks = ClockSampler(local).__enter__()
    snap = (z.clone(), zp.clone(), stp.ws.clone())

    def restore():
        z.copy_(snap[0])
        zp.copy_(snap[1])
        stp.ws.copy_(snap[2])

    t_w = time.perf_counter()
    done = 0
    with torch.cuda.stream(stream):
        while time.perf_counter() - t_w < 1.0:
            graph.replay()
            done += 1
            if done % 100 == 0:
                restore()
                torch.cuda.synchronize()
        restore()
    torch.cuda.synchronize()
    assert stp.read_status() == 0, nsf.status_string(stp.read_status())

    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    stage_ms = np.zeros((K, nst))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(K):
            flush.fill_(float(k))
            starts[k].record(stream)
            graph.replay()
            ends[k].record(stream)
        torch.cuda.synchronize()
    # stage times are those of the last replay (events are reused each replay);
    # the total is summed per step
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    status = stp.read_status()
    total_ms = reduce_max(total_ms, world, dev if world > 1 else None)

    # per-stage durations averaged over a separate pass of graph replays
    stage_runs = min(K, 50)
    st_acc = np.zeros(nst)
    with torch.cuda.stream(stream):
        for k in range(stage_runs):
            flush.fill_(float(k))
            graph_taps.replay()
            torch.cuda.synchronize()
            st_acc += [ev_b[i].elapsed_time(ev_e[i]) for i in range(nst)]
    st_ms = st_acc / stage_runs

    steps_per_s = world * K / (total_ms / 1e3)
    ms_per_step = total_ms / K

    # roofline of the dominant stage
    peaks, peak_src = load_peaks()
    r = fs.r
    macs = [mlp_macs(r, fs.width[i], fs.depth[i], od) for i, od in enumerate((3, 6, 9))]
    n_N, n_S = sc.X.shape[0], sc.n_S
    # Gauss-Newton: per sample point and iteration one value pass plus the
    # cheaper of 3 reverse (VJP) and r forward (JVP) passes for dg/dz
    flops = {
        "inference": 2.0 * n_N * sum(macs),
        "gauss_newton": 2.0 * sc.gn_iters * n_S * (1 + min(3, r)) * macs[0],
    }
    names = N.NSF_STAGE_NAMES
    mpm_bytes, touched = latent_mpm_bytes([sc])
    peak_t = peaks["bf16_tflops"] if args.precision == "bf16" else None
    stage_roof = {}
    for i, nm in enumerate(names):
        if nm in flops:
            ach = flops[nm] / (st_ms[i] / 1e3) / 1e12
            stage_roof[nm] = {"kernel": KERNEL_OF_STAGE[nm], "bound": "tensor", "achieved": ach,
                              "peak": peak_t, "unit": "TFLOP/s",
                              "frac": (ach / peak_t) if peak_t else None, "work": flops[nm],
                              "peak_source": f"bf16 dense burst, {peak_src}"}
        else:
            ach = mpm_bytes / (st_ms[i] / 1e3) / 1e9
            stage_roof[nm] = {"kernel": KERNEL_OF_STAGE[nm], "bound": "hbm", "achieved": ach,
                              "peak": peaks["hbm_gbs"], "unit": "GB/s",
                              "frac": ach / peaks["hbm_gbs"], "work": mpm_bytes,
                              "touched_nodes": touched,
                              "peak_source": f"copy bandwidth, {peak_src}"}
    dom = int(np.argmax(st_ms))
    roof = dict(stage_roof[names[dom]])
    roof["traffic"] = load_traffic(KERNEL_OF_STAGE.get(names[dom]))
    roof["traffic_unit"] = "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
    if args.only == "latent":
        clocks.__exit__(None, None, None)
        return {"value": steps_per_s, "unit": "steps/s", "ms_per_step": ms_per_step,
                "stages_ms": {names[i]: float(st_ms[i]) for i in range(nst)},
                "roofline": roof, "status": status}, clocks
    throughput = run_throughput(args, nsf, fs, dev, peaks, peak_src) if args.precision == "bf16" else None

    # e2e: through the public API with host buffers, copies inside the timed region
    e2e = run_e2e(args, nsf, sc, F, gd, dev)

    batched = run_batched(args, nsf, dev, flush, peaks, peak_src) if args.precision == "bf16" else None
    training = run_training(args, nsf, dev, peaks, peak_src)
    clocks.__exit__(None, None, None)

    full = run_full(args, nsf, full_config2(steps=args.steps), dev, flush)
    full_plastic = run_full(args, nsf, full_config2(model="von_mises", steps=args.steps), dev,
                            flush)
    matched = run_matched(args, nsf, dev, flush, full["steps_per_s"]) if args.precision == "bf16" else None
    config1 = run_config1(args, nsf, dev, flush)

    # kernels per step: fields 1, MPM 1 (binning, P2G, grid update and G2P in
    # one cooperative launch), Gauss-Newton 1 (all iterations in one
    # cooperative launch on the BF16 path)
    launches_per_step = 3 if args.precision == "bf16" else 2 + sc.gn_iters
    out = {
        "metric": METRIC, "value": steps_per_s, "unit": "steps/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.precision, "data": "synthetic",
        "config": {"workload": sc.name, "n_integration": n_N, "n_sample": n_S, "r": r,
                   "width": fs.width[0], "depth": fs.depth[0], "grid": list(sc.grid.n),
                   "gn_iters": sc.gn_iters, "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"replicas{world}", "graph": "one CUDA graph per step"},
        "stages_ms": {names[i]: float(st_ms[i]) for i in range(nst)},
        "roofline": roof,
        "roofline_stages": stage_roof,
        "mlp_throughput": throughput,
        "e2e": e2e,
        "batched": batched,
        "training": training,
        "full_order": full,
        "full_order_plastic": full_plastic,
        "matched_error": matched,
        "config1": config1,
        "gpu_launches": launches_per_step * K,
        "status": status,
    }
    return out, clocks


def latent_mpm_bytes(scenes):
    """Algorithmic bytes of the MPM stage of a latent step over `scenes`: P2G
    reads X, u_n, u_{n-1}, tau, C (96 B per integration particle); every
    touched grid node is written by P2G (16 B), read and re-zeroed by the grid
    update (32 B) and its velocity written (16 B); G2P reads X, u_n and writes
    x^{n+1} (36 B per sample particle).  Touched nodes: the 3^3 stencils of the
    reference positions.  Returns (bytes, touched nodes)."""
    touched, n_N, n_S = 0, 0, 0
    off = np.array([(a, b, c) for a in range(3) for b in range(3) for c in range(3)])
    for sc in scenes:
        base = np.floor(sc.X.astype(np.float64) / sc.grid.dx - 0.5).astype(np.int64)
        ng = sc.grid.n[0]
        nodes = (base[:, None, :] + off[None]).reshape(-1, 3)
        touched += np.unique((nodes[:, 0] * ng + nodes[:, 1]) * ng + nodes[:, 2]).size
        n_N += sc.X.shape[0]
        n_S += sc.n_S
    return 96.0 * n_N + 64.0 * touched + 36.0 * n_S, int(touched)


# The library's kernel that implements each latent stage.
KERNEL_OF_STAGE = {"inference": "k_fields_tc", "gauss_newton": "k_jac_tc<8>",
                   "mpm": "k_mpm_latent"}


def load_traffic(kernel):
    """DRAM bytes per launch of `kernel` on this workload, from the ncu summary
    in profiles/ (None if absent)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.md")
    if kernel is None or not os.path.exists(path):
        return None
    for line in open(path):
        f = [x.strip() for x in line.strip().strip("|").split("|")]
        if len(f) >= 3 and f[0] == kernel:
            try:       # read + write bytes
                return float(f[1].replace(",", "")) + float(f[2].replace(",", ""))
            except ValueError:
                return None
    return None


def run_throughput(args, nsf, fs, dev, peaks, peak_src):
    """The inference kernel (g, h, l) on a throughput-sized point set (one
    launch, 2^20 points), timed with CUDA events: what the tensor-core MLP
    kernel sustains when the work is large enough to fill the GPU."""
    import torch
    n = 1 << 20
    rng = np.random.Generator(np.random.PCG64(77))
    X = torch.from_numpy(rng.uniform(0.3, 0.7, size=(3, n)).astype(np.float32)).to(dev)
    z = torch.tensor(rng.normal(0, 0.1, size=fs.r), dtype=torch.float64, device=dev)
    F = nsf.Fields.from_spec(fs)
    x = torch.empty(3, n, device=dev)
    tau = torch.empty(6, n, device=dev)
    Cm = torch.empty(9, n, device=dev)
    for _ in range(3):
        nsf.nsf_eval_fields(F, X, z, x=x, tau6=tau, C9=Cm)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    reps = 10
    a.record()
    for _ in range(reps):
        nsf.nsf_eval_fields(F, X, z, x=x, tau6=tau, C9=Cm)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    macs = [mlp_macs(fs.r, fs.width[i], fs.depth[i], od) for i, od in enumerate((3, 6, 9))]
    flops = 2.0 * n * sum(macs)
    achieved = flops / (ms / 1e3) / 1e12
    peak = peaks["bf16_tflops"]
    return {"kernel": "k_fields_tc", "points": n, "ms": ms, "achieved": achieved,
            "unit": "TFLOP/s", "peak": peak, "frac": achieved / peak,
            "peak_source": f"bf16 dense burst, {peak_src}",
            "note": "fields g, h, l on 2^20 points; the latent step's own launches are latency-bound"}


def run_e2e(args, nsf, sc, F, gd, dev):
    """Host-buffer end to end: per step, H2D of X and z (pinned), the step call
    through the public API, D2H of z."""
    import torch
    Kh = min(args.steps, 50)
    Xh = torch.from_numpy(np.ascontiguousarray(sc.X.T)).pin_memory()
    zh = torch.tensor(sc.z0, dtype=torch.float64).pin_memory()
    zph = zh.clone().pin_memory()
    out = torch.empty_like(zh).pin_memory()
    Xd = torch.empty_like(Xh, device=dev)
    zd = torch.empty_like(zh, device=dev)
    zpd = torch.empty_like(zh, device=dev)
    stp = nsf.LatentStepper(F, Xd, sc.n_S, sc.mass, sc.vol0, gd)
    for _ in range(3):
        Xd.copy_(Xh, non_blocking=True); zd.copy_(zh, non_blocking=True); zpd.copy_(zph, non_blocking=True)
        stp.step(zd, zpd, sc.dt, nsteps=1, iters=sc.gn_iters, damping=sc.damping)
        out.copy_(zd, non_blocking=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Kh):
        Xd.copy_(Xh, non_blocking=True)
        zd.copy_(zh, non_blocking=True)
        zpd.copy_(zph, non_blocking=True)
        stp.step(zd, zpd, sc.dt, nsteps=1, iters=sc.gn_iters, damping=sc.damping)
        out.copy_(zd, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    dt = time.perf_counter() - t0
    h2d = Xh.numel() * 4 + 2 * zh.numel() * 8
    return {"value": Kh / dt, "unit": "steps/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(out.numel() * 8), "steps": Kh,
            "note": "eager API call per step (no graph), host wall clock"}


def run_config1(args, nsf, dev, flush):
    """The 1,024-particle latent scene with FP32 fields (4 x 64 on the CUDA
    cores, r = 6, 32^3 grid, 5 Gauss-Newton iterations), one graph replay per
    step, L2 flushed between steps.  Latency-bound (~1 GFLOP and ~0.1 MB per
    step): reported as steps/s, not against a roofline."""
    import torch
    from scenes.synthetic import latent_config1
    sc = latent_config1(steps=args.steps)
    F = nsf.Fields.from_spec(sc.fields)
    X = torch.from_numpy(np.ascontiguousarray(sc.X.T)).to(dev)
    gd = nsf.grid_desc(sc.grid.n, sc.grid.dx, sc.grid.gravity, sc.grid.wall_cells)
    stp = nsf.LatentStepper(F, X, sc.n_S, sc.mass, sc.vol0, gd)
    z = torch.tensor(sc.z0, dtype=torch.float64, device=dev)
    zp = z.clone()
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        stp.step(z, zp, sc.dt, nsteps=1, iters=sc.gn_iters, damping=sc.damping, stream=stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        stp.step(z, zp, sc.dt, nsteps=1, iters=sc.gn_iters, damping=sc.damping, stream=stream,
                 reuse_prev=True)
    for _ in range(max(3, args.warmup)):
        graph.replay()
    torch.cuda.synchronize()
    K = min(args.steps, 200)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    with torch.cuda.stream(stream):
        for k in range(K):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            graph.replay()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / K
    return {"workload": sc.name, "steps_per_s": 1e3 / ms, "ms_per_step": ms, "steps": K,
            "status": stp.read_status(), "dtype": "fp32",
            "launches_per_step": 2 + sc.gn_iters,
            "note": "FP32 fields on CUDA cores; Gauss-Newton one launch per iteration"}


def run_full(args, nsf, fc, dev, flush):
    import torch
    Kf = min(args.steps, 200)
    x, v = (torch.from_numpy(np.ascontiguousarray(a.T)).to(dev) for a in (fc.x, fc.v))
    Cm, Fm = (torch.from_numpy(np.ascontiguousarray(a.T)).to(dev) for a in (fc.C, fc.F))
    gd = nsf.grid_desc(fc.grid.n, fc.grid.dx, fc.grid.gravity, fc.grid.wall_cells, fc.grid.blade)
    mat = nsf.material(**fc.material)
    st = nsf.FullStepper(gd, mat, x, v, Cm, Fm, fc.mass, fc.vol0)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        st.step(fc.dt, t0=0.0, nsteps=1, stream=stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        st.step(fc.dt, t0=0.0, nsteps=1, stream=stream)
    for _ in range(max(3, args.warmup)):
        graph.replay()
    torch.cuda.synchronize()
    s = [torch.cuda.Event(enable_timing=True) for _ in range(Kf)]
    e = [torch.cuda.Event(enable_timing=True) for _ in range(Kf)]
    with torch.cuda.stream(stream):
        for k in range(Kf):
            flush.fill_(float(k))
            s[k].record(stream)
            graph.replay()
            e[k].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in zip(s, e))
    return {"steps_per_s": Kf / (ms / 1e3), "ms_per_step": ms / Kf, "steps": Kf,
            "workload": fc.name, "status": st.read_status(),
            "note": "blade time frozen at t=0 inside the replayed graph"}


def run_batched(args, nsf, dev, flush, peaks, peak_src):
    """256 independent latent scenes stepped together (nsf_latent_step_batched),
    one CUDA-graph replay per batched step, L2 flushed between steps; stage
    times from the library's stage events and each stage against its
    roofline."""
    import torch
    from paper_2310_17790_gb300 import _native as N
    from scenes.synthetic import batch_config4

    scenes = batch_config4(n_scenes=args.batch_scenes, steps=args.steps)
    keep, entries = [], []
    for sc in scenes:
        F = nsf.Fields.from_spec(sc.fields)
        X = torch.from_numpy(np.ascontiguousarray(sc.X.T)).to(dev)
        z = torch.tensor(sc.z0, dtype=torch.float64, device=dev)
        zp = z.clone()
        gd = nsf.grid_desc(sc.grid.n, sc.grid.dx, sc.grid.gravity, sc.grid.wall_cells)
        keep.append((F, X, z, zp))
        entries.append((F, X, sc.n_S, sc.mass, sc.vol0, gd, sc.dt, z, zp))
    codes = [(e[7], e[8], e[7].clone(), e[8].clone()) for e in entries]
    nst = N.NSF_LATENT_STAGES
    K = max(1, min(args.steps, 100))

    def measure(tuning):
        """ms per batched step (mean of K graph replays, L2 flushed before each)
        and the stage times, for the plan with `tuning` (None: the defaults)."""
        b = nsf.LatentBatch(entries, iters=scenes[0].gn_iters, damping=scenes[0].damping,
                            tuning=tuning)
        for z, zp, z0, zp0 in codes:               # every plan starts from the same codes
            z.copy_(z0)
            zp.copy_(zp0)
        stream = torch.cuda.Stream(device=dev)
        ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(nst)]
        ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(nst)]
        with torch.cuda.stream(stream):
            for e in ev_b + ev_e:
                e.record(stream)
        torch.cuda.synchronize()
        evs = N.nsf_batch_events()
        for i in range(nst):
            evs.ev_begin[i] = ev_b[i].cuda_event
            evs.ev_end[i] = ev_e[i].cuda_event
        with torch.cuda.stream(stream):
            b.step(t0=0.0, nsteps=1, stream=stream)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            b.step(t0=0.0, nsteps=1, events=evs, stream=stream, reuse_prev=True)
        torch.cuda.synchronize()
        for _ in range(max(3, args.warmup)):
            graph.replay()
        torch.cuda.synchronize()
        assert b.read_status() == 0, nsf.status_string(b.read_status())
        s_ev = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        e_ev = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        st_acc = np.zeros(nst)
        with torch.cuda.stream(stream):
            for k in range(K):
                flush.fill_(float(k))
                s_ev[k].record(stream)
                graph.replay()
                e_ev[k].record(stream)
                if k < 20:
                    torch.cuda.synchronize()
                    st_acc += [ev_b[i].elapsed_time(ev_e[i]) for i in range(nst)]
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(c) for a, c in zip(s_ev, e_ev)) / K
        st_ms = st_acc / min(K, 20)
        status = b.read_status()
        b.close()
        return ms, st_ms, status

    from paper_2310_17790_gb300 import autotune
    cache = autotune.TuningCache(args.tuning_cache) if args.tuning_cache else None
    tuned = cache.get(entries) if cache else None
    tuner = None
    if args.tune:
        best, best_ms, results = autotune.tune_batch(entries, steps=3, iters=scenes[0].gn_iters,
                                                     damping=scenes[0].damping)
        for z, zp, z0, zp0 in codes:
            z.copy_(z0)
            zp.copy_(zp0)
        tuned = best
        if cache is not None and best is not None:
            cache.put(entries, best, best_ms)
        tuner = {"signature": autotune.batch_signature(entries),
                 "timed": [{"tuning": t, "ms_per_step": m} for t, m in results]}
    ms_default, st_default, status_default = measure(None)
    ms, st_ms, status = measure(tuned) if tuned else (ms_default, st_default, status_default)
    status = status or status_default

    n_N = np.array([sc.X.shape[0] for sc in scenes], np.float64)
    n_S = np.array([sc.n_S for sc in scenes], np.float64)
    fl_inf, fl_gn = 0.0, 0.0
    for sc, nn, ns in zip(scenes, n_N, n_S):
        fs = sc.fields
        macs = [mlp_macs(fs.r, fs.width[i], fs.depth[i], od) for i, od in enumerate((3, 6, 9))]
        fl_inf += 2.0 * nn * sum(macs)
        fl_gn += 2.0 * sc.gn_iters * ns * (1 + min(3, fs.r)) * macs[0]
    mpm_bytes, touched = latent_mpm_bytes(scenes)
    names = N.NSF_STAGE_NAMES
    stages = {names[i]: float(st_ms[i]) for i in range(nst)}
    pk = peaks["bf16_tflops"]

    def tf(flops, t_ms):
        return flops / (t_ms / 1e3) / 1e12
    roof = {
        "inference": {"kernel": "k_fields_batch", "bound": "tensor", "unit": "TFLOP/s",
                      "achieved": tf(fl_inf, st_ms[0]), "peak": pk,
                      "frac": tf(fl_inf, st_ms[0]) / pk, "work": fl_inf},
        "mpm": {"kernel": "k_mpm_batch", "bound": "hbm", "unit": "GB/s",
                "achieved": mpm_bytes / (st_ms[1] / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                "frac": mpm_bytes / (st_ms[1] / 1e3) / 1e9 / peaks["hbm_gbs"],
                "work": mpm_bytes, "touched_nodes": int(touched),
                "note": "96 B per integration particle + 64 B per touched node + 36 B per "
                        "sample particle; P2G sums each 4^3 block in a shared-memory tile "
                        "(exact integers), one integer atomic per touched node and value"},
        "gauss_newton": {"kernel": "k_jac_batch", "bound": "tensor", "unit": "TFLOP/s",
                         "achieved": tf(fl_gn, st_ms[2]), "peak": pk,
                         "frac": tf(fl_gn, st_ms[2]) / pk, "work": fl_gn},
    }
    return {"workload": f"batch-{len(scenes)}scenes-{int(n_N.sum())}N-{int(n_S.sum())}S-bf16",
            "scenes": len(scenes), "n_integration_total": int(n_N.sum()),
            "n_sample_total": int(n_S.sum()), "steps": K, "ms_per_step": ms,
            "batched_steps_per_s": 1e3 / ms, "scene_steps_per_s": len(scenes) * 1e3 / ms,
            "stages_ms": stages, "roofline": roof, "status": status,
            "launches_per_step": 2 + len({sc.fields.width[0] for sc in scenes}),
            "peak_source": f"measured ({peak_src})",
            "tuning": tuned, "default_plan_ms_per_step": ms_default,
            "default_plan_stages_ms": {names[i]: float(st_default[i]) for i in range(nst)},
            "tuner": tuner,
            "note": "one CUDA-graph replay of one batched step; L2 flushed between steps; "
                    "the plan with the tile choices of the tuning table (paper_2310_17790_gb300/"
                    "tuning_gb300.json) when it holds this batch's signature, else the "
                    "default plan"}


def run_training(args, nsf, dev, peaks, peak_src):
    """One training step of the deformation field on full-order snapshots
    (App. D): 64 snapshots of the 200,000-particle slab from the library's
    full-order step (5 steps apart), minibatches of 65,536 (particle,
    snapshot) pairs, field g of 5 hidden layers x 256 (BF16 forward, backward
    products with the cotangent split into bf16 hi + lo, FP32 master weights),
    per-snapshot latent codes r = 6 learned jointly, Adam lr 1e-4.  A step = loss and gradients + Adam on weights and
    codes + re-pack of the weights, all through the C ABI."""
    import torch
    from scenes.synthetic import full_config2, make_fields
    fc = full_config2(steps=1)
    x, v = (torch.from_numpy(np.ascontiguousarray(a.T)).to(dev) for a in (fc.x, fc.v))
    Cm, Fm = (torch.from_numpy(np.ascontiguousarray(a.T)).to(dev) for a in (fc.C, fc.F))
    X_ref = x.clone()
    gd = nsf.grid_desc(fc.grid.n, fc.grid.dx, fc.grid.gravity, fc.grid.wall_cells, fc.grid.blade)
    st = nsf.FullStepper(gd, nsf.material(**fc.material), x, v, Cm, Fm, fc.mass, fc.vol0)
    snaps = []
    for t in range(64):
        st.step(fc.dt, t0=t * 5 * fc.dt, nsteps=5)
        snaps.append(x.clone())
    torch.cuda.synchronize()
    snaps = torch.stack(snaps)                                   # [64, 3, n]
    n_all = X_ref.shape[1]
    B = 65536
    rng = np.random.Generator(np.random.PCG64(2315))
    spec = make_fields(rng, 6, 256, 5, "bf16", {"g": 1e-2, "h": 1e4, "l": 1.0})
    F = nsf.Fields.from_spec(spec)
    z0 = torch.from_numpy(rng.normal(0, 0.1, size=(64, 6)).astype(np.float32)).to(dev)
    w0 = torch.from_numpy(np.asarray(spec.weights["g"], np.float32)).to(dev)
    tr = nsf.FieldTrainer(F, "g", w0, z0, B, lr=1e-4)

    def batch(seed):
        r_ = np.random.Generator(np.random.PCG64(seed))
        p = torch.from_numpy(r_.integers(0, n_all, size=B)).to(dev)
        t = torch.from_numpy(r_.integers(0, 64, size=B)).to(dev)
        X = X_ref[:, p].contiguous()
        tgt = snaps[t, :, p].T.contiguous()
        return X, t.to(torch.int32).contiguous(), tgt
    batches = [batch(2400 + k) for k in range(4)]
    for k in range(3):
        tr.step(*batches[k % 4])
    torch.cuda.synchronize()
    K = max(1, min(args.steps, 50))
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    first = float(tr.step(*batches[0]).item())
    a.record()
    for k in range(K):
        tr.step(*batches[k % 4])
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / K
    last = float(tr.loss.item())
    mac = mlp_macs(6, 256, 5, 3)
    flops = 6.0 * B * mac        # forward 2 n MAC, backward 4 n MAC
    return {"workload": "train-g-w256d5-r6-bf16fwd-splitbf16bwd-batch65536-64snapshots-200k",
            "ms_per_step": ms, "steps": K, "points_per_s": B / (ms / 1e3),
            "tflops": flops / (ms / 1e3) / 1e12, "flops_per_step": flops,
            "loss_first": first, "loss_last": last,
            "note": "loss and gradients (the library's tcgen05 GEMMs: BF16 forward, backward "
                    "with hi/lo-split bf16 cotangents, FP32 accumulation; fused bias/ELU/ELU' "
                    "epilogues), Adam on weights and codes, weight re-pack"}


def run_matched(args, nsf, dev, flush, full_steps_per_s, steps=400, every=10,
                train_steps=4000, lr=1e-3, iters_list=(1, 2, 3, 5)):
    """The latent step against the full-order step on the same scene at
    matched particle-position error (§6; App. D training).

    1. Full-order run of the 200,000-particle slab (neo-Hookean, sticky blade),
       `steps` steps, a snapshot of x, C and tau(F) every `every` steps.
    2. Fields g, h, l (5 x 128, BF16, r = 6) fitted to the snapshots with the
       library's training path (Adam, hand-written backward): outputs
       normalised by the snapshots' per-component mean and std (App. D), one
       latent code per snapshot learned with g, h and l fitted on those codes.
    3. Latent runs from snapshot 0's code (zero initial velocity) on a seeded
       5 % integration set (10,000 particles) with 700 sample particles, for
       each Gauss-Newton iteration count (1 = the first-order Taylor
       projection of §5.3), and one graph-replayed step of each timed with L2
       flushed between steps.
    4. Error of the sample particles' fitted positions g(X_S, z_n) against the
       full-order positions, in dx units (max and rms over S), at the end and
       over the run; delta of Eq. 10 over S and all snapshots."""
    import torch
    from scenes.synthetic import full_config2, make_fields
    fc = full_config2(steps=1)
    soa = lambda a: torch.from_numpy(np.ascontiguousarray(a.T)).to(dev)
    x, v, Cm, Fm = soa(fc.x), soa(fc.v), soa(fc.C), soa(fc.F)
    X_ref = x.clone()
    gd = nsf.grid_desc(fc.grid.n, fc.grid.dx, fc.grid.gravity, fc.grid.wall_cells, fc.grid.blade)
    mat = nsf.material(**fc.material)
    st = nsf.FullStepper(gd, mat, x, v, Cm, Fm, fc.mass, fc.vol0)
    n = x.shape[1]
    snaps = {"g": [], "h": [], "l": []}

    def record():
        tau = torch.empty(6, n, device=dev)
        nsf.nsf_material_stress(mat, Fm, tau)
        snaps["g"].append(x.clone())
        snaps["h"].append(tau)
        snaps["l"].append(Cm.clone())
    record()
    for k in range(steps // every):
        st.step(fc.dt, t0=k * every * fc.dt, nsteps=every)
        record()
    torch.cuda.synchronize()
    assert st.read_status() == 0, nsf.status_string(st.read_status())
    S = {k: torch.stack(a) for k, a in snaps.items()}             # [T, comps, n]
    T = S["g"].shape[0]
    rng = np.random.Generator(np.random.PCG64(2318))
    spec = make_fields(rng, 6, 128, 5, "bf16", {"g": 1.0, "h": 1.0, "l": 1.0})
    for k in "ghl":
        A = S[k] - X_ref[None] if k == "g" else S[k]               # g is residual: x = X + y
        flat = A.permute(1, 0, 2).reshape(A.shape[1], -1)
        spec.out_shift[k] = flat.mean(1).cpu().numpy().astype(np.float32)
        spec.out_scale[k] = flat.std(1).clamp_min(1e-12).cpu().numpy().astype(np.float32)
    F = nsf.Fields.from_spec(spec)
    B = 65536
    gen = torch.Generator(device=dev)
    gen.manual_seed(2318)

    def batch(target):
        p = torch.randint(0, n, (B,), device=dev, generator=gen)
        t = torch.randint(0, T, (B,), device=dev, generator=gen)
        return X_ref[:, p].contiguous(), t.to(torch.int32).contiguous(), target[t, :, p].T.contiguous()
    codes0 = torch.from_numpy(rng.normal(0, 0.1, size=(T, 6)).astype(np.float32)).to(dev)
    trainers, losses = {}, {}
    t_train = time.perf_counter()
    for k in "ghl":
        w0 = torch.from_numpy(np.asarray(spec.weights[k], np.float32)).to(dev)
        tr = nsf.FieldTrainer(F, k, w0, codes0 if k == "g" else trainers["g"].z, B, lr=lr,
                              train_codes=(k == "g"))
        for it in range(train_steps):
            tr.lr = lr * (1.0 if it < train_steps // 2 else 0.3 if it < 3 * train_steps // 4 else 0.1)
            tr.step(*batch(S[k]))
        torch.cuda.synchronize()
        trainers[k], losses[k] = tr, float(tr.loss.item())
    t_train = time.perf_counter() - t_train
    codes = trainers["g"].z.double()
    r2 = np.random.Generator(np.random.PCG64(2319))
    sub = r2.choice(n, size=10000, replace=False)
    sub = torch.from_numpy(sub[r2.permutation(sub.size)]).to(dev)
    nS, dx = 700, fc.grid.dx
    X_N = X_ref[:, sub].contiguous()
    XS = X_N[:, :nS].contiguous()
    ref = S["g"][:, :, sub[:nS]]                                     # [T, 3, nS]

    def fitted(zz):
        out = torch.empty(3, nS, device=dev)
        nsf.nsf_eval_fields(F, XS, zz.contiguous(), x=out)
        return out
    fit_max = max(float((fitted(codes[t]) - ref[t]).abs().max()) / dx for t in range(T))
    disp_max = float((ref[-1] - XS).abs().max()) / dx
    runs = []
    for iters in iters_list:
        lat = nsf.LatentStepper(F, X_N, nS, fc.mass, fc.vol0, gd)
        z, zp = codes[0].clone().contiguous(), codes[0].clone().contiguous()
        err_max, err_rms, num, den = [], [], 0.0, 0.0
        for t in range(T):
            if t > 0:
                lat.step(z, zp, fc.dt, t0=(t - 1) * every * fc.dt, nsteps=every, iters=iters,
                         damping=1e-6)
            d = fitted(z) - ref[t]
            err_max.append(float(d.abs().max()) / dx)
            err_rms.append(float(d.pow(2).sum(0).mean().sqrt()) / dx)
            num += float(d.pow(2).sum())
            den += float(ref[t].pow(2).sum())
        torch.cuda.synchronize()
        status = lat.read_status()
        stream = torch.cuda.Stream(device=dev)
        zt, zpt = z.clone(), zp.clone()
        with torch.cuda.stream(stream):
            lat.step(zt, zpt, fc.dt, nsteps=1, iters=iters, damping=1e-6, stream=stream)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            lat.step(zt, zpt, fc.dt, nsteps=1, iters=iters, damping=1e-6, stream=stream,
                     reuse_prev=True)
        for _ in range(5):
            graph.replay()
        torch.cuda.synchronize()
        K = 100
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K)]
        with torch.cuda.stream(stream):
            for k in range(K):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                graph.replay()
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / K
        runs.append({"gn_iters": iters, "latent_steps_per_s": 1e3 / ms, "status": status,
                     "final_max_dx": err_max[-1], "final_rms_dx": err_rms[-1],
                     "run_max_dx": max(err_max), "delta_eq10": (num / den) ** 0.5})
    ok = [r for r in runs if r["status"] == 0]
    best = max(ok, key=lambda r: r["latent_steps_per_s"]) if ok else None
    return {"workload": f"full-order slab 200k neo-Hookean + blade, {steps} steps, snapshots every "
                        f"{every}; latent 10,000 N / 700 S, r = 6, fields 5 x 128 BF16 fitted to "
                        f"the snapshots ({train_steps} Adam steps per field, batch {B})",
            "full_order_steps_per_s": full_steps_per_s, "runs": runs,
            "fastest_latent": best,
            "speedup_fastest_vs_full": (best["latent_steps_per_s"] / full_steps_per_s) if best else None,
            "fit_max_dx": fit_max, "sample_displacement_max_dx": disp_max,
            "training_s": t_train, "final_losses": losses,
            "note": "errors of the sample particles' positions g(X_S, z_n) against the full-order "
                    "run, dx units; gn_iters 1 is the first-order Taylor projection (§5.3)"}


def run_part(args):
    """One part of the benchmark alone (for profiling captures)."""
    import torch
    import paper_2310_17790_gb300 as nsf
    from scenes.synthetic import latent_config3
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    peaks, peak_src = load_peaks()
    if args.only == "mlp":
        return run_throughput(args, nsf, latent_config3(precision="bf16", steps=1).fields, dev,
                              peaks, peak_src)
    if args.only == "training":
        return run_training(args, nsf, dev, peaks, peak_src)
    if args.only == "matched":
        from scenes.synthetic import full_config2
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        full = run_full(args, nsf, full_config2(steps=args.steps), dev, flush)
        return run_matched(args, nsf, dev, flush, full["steps_per_s"])
    if args.only == "full":
        from scenes.synthetic import full_config2
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        return run_full(args, nsf, full_config2(steps=args.steps), dev, flush)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    return run_batched(args, nsf, dev, flush, peaks, peak_src)


# ---------------------------------------------------------- CPU oracle ---
def run_oracle(args, budget_s):
    """The FP64 oracle's latent step on the same workload (bounded sample)."""
    from oracle import fields as ofields, latent as olatent, mpm as ompm
    from scenes.synthetic import latent_config3

    sc = latent_config3(precision=args.precision)
    fs = sc.fields
    fl = []
    for i, k in enumerate("ghl"):
        w = np.asarray(fs.weights[k], np.float64)
        if fs.precision == "bf16":     # the weight matrices the GPU path uses
            off = 0
            for a, b in ofields.layer_dims(fs.r, fs.width[i], fs.depth[i], ofields.OUT_DIM[k]):
                w[off:off + a * b] = ofields.round_to_bf16(w[off:off + a * b])
                off += a * b + b
        fl.append(ofields.Field(w, fs.r, fs.width[i], fs.depth[i], ofields.OUT_DIM[k],
                                fs.out_scale[k], fs.out_shift[k], residual=(k == "g"),
                                bf16_operands=(fs.precision == "bf16")))
    of = olatent.Fields(*fl)
    g = sc.grid
    og = ompm.Grid(g.n, g.dx, g.gravity, g.wall_cells, g.blade)
    X = sc.X.astype(np.float64)
    z, zp = sc.z0.copy(), sc.z0.copy()
    steps, t0 = 0, time.perf_counter()
    max_steps = max(1, args.steps)
    while steps < max_steps:
        zn, _ = olatent.latent_step(of, X, sc.n_S, sc.mass, sc.vol0, z, zp, sc.dt, og,
                                    t=steps * sc.dt, iters=sc.gn_iters, damping=sc.damping)
        z, zp = zn, z
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    return {"value": steps / el, "unit": "steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} consecutive latent steps of {sc.name} (FP64 NumPy oracle)",
            "seconds": el}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="nsf", choices=["nsf", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--only", default="all",
                    choices=["all", "latent", "batched", "mlp", "training", "full", "matched"],
                    help="latent / batched / mlp / training / full / matched: run that part "
                         "alone (profiling runs) and print its JSON")
    ap.add_argument("--batch-scenes", type=int, default=256)
    ap.add_argument("--tuning-cache", default=os.path.join(ROOT, "paper_2310_17790_gb300",
                                                           "tuning_gb300.json"),
                    help="JSON table of batch tile choices by batch signature ('' for none)")
    ap.add_argument("--tune", action="store_true",
                    help="time the tuner's candidates on the batch and record the winner")
    args = ap.parse_args()
    rank, world, local = dist_env()

    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        cb = run_oracle(args, budget_s=max(5.0, min(120.0, args.cpu_budget * 3)))
        out = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "steps/s",
               "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": 1e3 / cb["value"], "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": "latent-10000N-700S-r6-w128d5-grid128 (FP64 CPU oracle)"},
               "cpu_baseline": cb,
               "e2e": {"value": cb["value"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0},
               "wall_s": time.perf_counter() - t0}
        print(json.dumps(out))
        return

    if args.only == "latent":
        out, _ = run_gpu(args, rank, world, local)
        print(json.dumps(out))
        return
    if args.only != "all":
        print(json.dumps(run_part(args)))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out, clocks = run_gpu(args, rank, world, local)
    out["clocks"] = clocks.summary()
    if rank == 0:
        out["cpu_baseline"] = run_oracle(args, budget_s=args.cpu_budget)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
