"""Tile choices of a batched latent step, chosen by timing.

The batch plan has three tile choices (`nsf_batch_tuning`): the Gauss-Newton
tile width (128 or 256 point slots), the cost above which a scene's
Gauss-Newton run is split over a group of CTAs, and the P2G tile's thread
count.  `tune_batch` times every candidate on the caller's batch (one
CUDA-graph replay per timed step, on copies of the latent codes, so the
caller's state is untouched) and returns the fastest; `TuningCache` keeps the
winners in a JSON file keyed by a coarse signature of the batch (scene count,
the (r, width, depth) mix of its fields and its particle counts in powers of
two), so that batches of the same shape reuse them without timing again.
"""

import json
import math
import os

from . import LatentBatch, _torch
from . import _native as N


def default_candidates():
    """The tile choices that are timed: every combination of the Gauss-Newton
    width, a few split thresholds (0 = the library's own search) and the P2G
    group size."""
    out = []
    for cols in (64, 32):
        for split in (0.0, 0.75, 1.0, 1.5, 2.5):
            for p2g in (64, 128):
                out.append({"gn_columns": cols, "gn_split": split, "p2g_group": p2g})
    return out


def batch_signature(entries):
    """Coarse shape of a batch: scene count, the sorted (r, width, depth) mix
    of the g fields, and the total integration and sample particles rounded to
    powers of two."""
    mix = set()
    n_N = n_S = 0
    for F, X, n_S_i, *_ in entries:
        mix.add((int(F.r), int(F.width[0]), int(F.depth[0])))      # field g
        n_N += int(X.shape[1])
        n_S += int(n_S_i)
    p2 = lambda v: int(round(math.log2(max(v, 1))))
    return "n%d|%s|N2^%d|S2^%d" % (len(entries), ",".join("r%dw%dd%d" % m for m in sorted(mix)),
                                   p2(n_N), p2(n_S))


def time_batch(entries, tuning, steps=3, iters=5, damping=1e-6):
    """Milliseconds per batched step of `entries` with `tuning` (median of
    `steps` graph replays after one warm-up), on copies of the latent codes.
    None if the library rejects the tuning for this batch."""
    torch = _torch()
    copies = []
    for e in entries:
        F, X, n_S, mass, vol0, grid, dt, z, zp = e
        copies.append((F, X, n_S, mass, vol0, grid, dt, z.clone(), zp.clone()))
    try:
        b = LatentBatch(copies, iters=iters, damping=damping, tuning=tuning)
    except N.NsfError as e:
        if e.status == N.NSF_ERR_INVALID_ARG:      # a width some scene's operands do not fit
            return None
        raise
    try:
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            b.step(stream=stream)                  # fills the g(X, z_prev) cache
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            b.step(stream=stream, reuse_prev=True)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            a = torch.cuda.Event(enable_timing=True)
            c = torch.cuda.Event(enable_timing=True)
            a.record()
            graph.replay()
            c.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(c))
        if b.read_status() != 0:
            return None
        times.sort()
        return times[len(times) // 2]
    finally:
        b.close()


def tune_batch(entries, candidates=None, steps=3, iters=5, damping=1e-6):
    """Times every candidate tuning on this batch; returns (best tuning dict,
    its ms per step, [(tuning, ms or None), ...])."""
    results = []
    best, best_ms = None, None
    for cand in candidates or default_candidates():
        ms = time_batch(entries, cand, steps=steps, iters=iters, damping=damping)
        results.append((cand, ms))
        if ms is not None and (best_ms is None or ms < best_ms):
            best, best_ms = cand, ms
    return best, best_ms, results


class TuningCache:
    """Winning tunings by batch signature, in a JSON file."""

    def __init__(self, path):
        self.path = path
        self.table = {}
        if os.path.exists(path):
            with open(path) as f:
                self.table = json.load(f)

    def get(self, entries):
        rec = self.table.get(batch_signature(entries))
        return dict(rec["tuning"]) if rec else None

    def put(self, entries, tuning, ms):
        self.table[batch_signature(entries)] = {"tuning": dict(tuning), "ms_per_step": ms}
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.table, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def tuning_for(self, entries, **kw):
        """The cached tuning for this batch's signature, else tune and cache."""
        t = self.get(entries)
        if t is None:
            t, ms, _ = tune_batch(entries, **kw)
            if t is not None:
                self.put(entries, t, ms)
        return t
