"""Seeded synthetic scenes shaped like the paper's workloads.

No dataset or trained network of the paper is available, so every input is
drawn here from numpy's PCG64 with a fixed seed:

* Field weights: Xavier-uniform matrices (the initialisation named in the
  paper's training details), biases uniform in [-0.1, 0.1], stored float32 in the
  flat per-field layout (per linear layer: W row-major [out][in], then b).
* Latent scene, 1,024 particles: X uniform in [0.4, 0.6]^3, all of them sample
  particles, 32^3 grid, dx = 1/32, dt = 1e-4, gravity -9.8 z, rho = 1000,
  r = 6, z0 ~ N(0, 0.1^2), fields 4 hidden layers of width 64, FP32.
* Full-order slab, 200,000 particles: a 100 x 100 x 20 lattice of spacing dx/2
  jittered by U(-0.25, 0.25) spacing, centred at (0.5, 0.5, 0.2), 128^3 grid,
  dx = 1/128, dt = 5e-5, neo-Hookean E = 2e5, nu = 0.3, rho = 1000, a sticky
  blade (plane x = 0.5) starting 2 dx above the slab top and moving down at 1 m/s.
* Latent scene at full scale: the slab's particles are the reference domain;
  a seeded 5 % subset (10,000) are the integration particles, the first 700 of
  a seeded permutation of them the sample particles; r = 6, fields 5 hidden
  layers of width 128, BF16.
Particle volume is the slab (or cube) volume divided by the full particle
count, mass = rho * volume.
"""

from dataclasses import dataclass, field as dc_field
from typing import Dict, Optional, Tuple

import numpy as np

FIELD_NAMES = ("g", "h", "l")
FIELD_OUT = {"g": 3, "h": 6, "l": 9}


def _dims(r, width, depth, out_dim):
    dims = [(3 + r, width)] + [(width, width)] * (depth - 1) + [(width, out_dim)]
    return dims


def field_weights(rng, r, width, depth, out_dim, bias=0.1):
    """Flat float32 weights: Xavier-uniform W, uniform biases."""
    parts = []
    for fan_in, fan_out in _dims(r, width, depth, out_dim):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-a, a, size=(fan_out, fan_in)).ravel())
        parts.append(rng.uniform(-bias, bias, size=fan_out))
    return np.concatenate(parts).astype(np.float32)


@dataclass
class FieldSpec:
    r: int
    width: Tuple[int, int, int]
    depth: Tuple[int, int, int]
    precision: str                       # "fp32" | "bf16"
    weights: Dict[str, np.ndarray]
    out_scale: Dict[str, np.ndarray]
    out_shift: Dict[str, np.ndarray]
    residual_g: bool = True


@dataclass
class GridSpec:
    n: Tuple[int, int, int]
    dx: float
    gravity: Tuple[float, float, float] = (0.0, 0.0, -9.8)
    wall_cells: int = 3
    blade: Optional[dict] = None         # dict(x=..., z0=..., vz=...)


@dataclass
class LatentScene:
    X: np.ndarray                        # [n_N, 3] float32 reference positions
    n_S: int
    mass: float
    vol0: float
    grid: GridSpec
    dt: float
    z0: np.ndarray                       # [r] float64
    z_prev: np.ndarray                   # [r] float64
    fields: FieldSpec
    gn_iters: int = 5
    damping: float = 1e-6
    steps: int = 1
    name: str = ""


@dataclass
class FullScene:
    x: np.ndarray                        # [n, 3] float32
    v: np.ndarray                        # [n, 3]
    C: np.ndarray                        # [n, 9] row-major
    F: np.ndarray                        # [n, 9] row-major
    mass: float
    vol0: float
    grid: GridSpec
    dt: float
    material: dict = dc_field(default_factory=dict)
    steps: int = 1
    name: str = ""


def make_fields(rng, r, width, depth, precision, scales):
    width = (width,) * 3 if np.isscalar(width) else tuple(width)
    depth = (depth,) * 3 if np.isscalar(depth) else tuple(depth)
    w, sc, sh = {}, {}, {}
    for i, f in enumerate(FIELD_NAMES):
        w[f] = field_weights(rng, r, width[i], depth[i], FIELD_OUT[f])
        sc[f] = np.full(FIELD_OUT[f], scales[f], dtype=np.float32)
        sh[f] = np.zeros(FIELD_OUT[f], dtype=np.float32)
    return FieldSpec(r=r, width=width, depth=depth, precision=precision,
                     weights=w, out_scale=sc, out_shift=sh)


def latent_scene(seed, n_N, n_S, r, width, depth, precision, grid, dt,
                 X=None, lo=0.4, hi=0.6, E=1e5, rho=1000.0, vol_total=None,
                 n_total=None, z_std=0.1, steps=1, name=""):
    rng = np.random.Generator(np.random.PCG64(seed))
    if X is None:
        X = rng.uniform(lo, hi, size=(n_N, 3)).astype(np.float32)
        vol_total = (hi - lo) ** 3 if vol_total is None else vol_total
        n_total = n_N if n_total is None else n_total
    vol0 = vol_total / n_total
    scales = {"g": 1e-2, "h": 1e-2 * E, "l": 1.0}
    fs = make_fields(rng, r, width, depth, precision, scales)
    z0 = rng.normal(0.0, z_std, size=r)
    return LatentScene(X=np.ascontiguousarray(X, dtype=np.float32), n_S=n_S,
                       mass=rho * vol0, vol0=vol0, grid=grid, dt=dt, z0=z0,
                       z_prev=z0.copy(), fields=fs, steps=steps, name=name)


def latent_config1(seed=2311, steps=200):
    """1,024 sample = integration particles in [0.4, 0.6]^3, FP32 fields 4x64."""
    grid = GridSpec(n=(32, 32, 32), dx=1.0 / 32)
    return latent_scene(seed, 1024, 1024, 6, 64, 4, "fp32", grid, 1e-4,
                        steps=steps, name="latent-1024p-r6-w64d4-fp32-grid32")


def slab_lattice(rng, nx=100, ny=100, nz=20, dx=1.0 / 128,
                 centre=(0.5, 0.5, 0.2)):
    s = dx / 2
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                          indexing="ij")
    lat = np.stack([I, J, K], axis=-1).reshape(-1, 3).astype(np.float64)
    ext = np.array([nx, ny, nz], np.float64) * s
    pos = (lat + 0.5) * s + np.asarray(centre) - ext / 2
    pos += rng.uniform(-0.25, 0.25, size=pos.shape) * s
    vol0 = float(np.prod(ext)) / pos.shape[0]
    top = centre[2] + ext[2] / 2
    return pos.astype(np.float32), vol0, top


def full_scene(seed, lattice=(100, 100, 20), n_grid=128, dt=5e-5,
               model="neo_hookean", E=2e5, nu=0.3, rho=1000.0,
               yield_stress=1e4, friction_deg=30.0, blade=True, steps=1,
               name=""):
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = 1.0 / n_grid
    x, vol0, top = slab_lattice(rng, *lattice, dx=dx)
    n = x.shape[0]
    bl = dict(x=0.5, z0=top + 2 * dx, vz=-1.0) if blade else None
    grid = GridSpec(n=(n_grid,) * 3, dx=dx, blade=bl)
    eye = np.tile(np.eye(3, dtype=np.float32).ravel(), (n, 1))
    mat = dict(model=model, E=E, nu=nu, yield_stress=yield_stress,
               friction_deg=friction_deg)
    return FullScene(x=x, v=np.zeros((n, 3), np.float32),
                     C=np.zeros((n, 9), np.float32), F=eye, mass=rho * vol0,
                     vol0=vol0, grid=grid, dt=dt, material=mat, steps=steps,
                     name=name)


def full_config2(seed=2312, model="neo_hookean", steps=1000):
    return full_scene(seed, model=model, steps=steps,
                      name=f"full-200k-{model}-grid128")


def latent_config3(seed=2313, steps=1000, n_N=10000, n_S=700,
                   precision="bf16", width=128, depth=5):
    """Integration particles = seeded 5 % of the 200k slab; 700 sample particles."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = 1.0 / 128
    P, vol0, top = slab_lattice(rng, dx=dx)
    sub = rng.choice(P.shape[0], size=n_N, replace=False)
    perm = rng.permutation(n_N)
    X = P[sub][perm]
    grid = GridSpec(n=(128, 128, 128), dx=dx)
    sc = latent_scene(seed + 1000, n_N, n_S, 6, width, depth, precision, grid,
                      5e-5, X=X, E=2e5, vol_total=vol0 * P.shape[0],
                      n_total=P.shape[0], steps=steps,
                      name=f"latent-{n_N}N-{n_S}S-r6-w{width}d{depth}-{precision}-grid128")
    return sc


def tiny_latent(seed, n_N=200, n_S=60, r=6, width=32, depth=2,
                precision="fp32", n_grid=16, dt=1e-4, lo=0.35, hi=0.65):
    grid = GridSpec(n=(n_grid,) * 3, dx=1.0 / n_grid)
    return latent_scene(seed, n_N, n_S, r, width, depth, precision, grid, dt,
                        lo=lo, hi=hi, name="tiny")


def batch_config4(seed=2314, n_scenes=256, steps=500):
    """Independent latent scenes for batched stepping: |N| log-uniform in
    [1,000, 20,000]; r from {6, 12, 16}; grid 64^3 (dt 1e-4) or 128^3 (dt
    5e-5); BF16 fields of width 64 or 128 and depth 4 or 5 (the same for g, h,
    l of a scene); S = N when |N| <= 2,000, else the first 5 % of N.
    Positions uniform in [0.3, 0.7]^3, each scene with its own seeded fields
    and z0 ~ N(0, 0.1^2), z_prev = z0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_scenes):
        n_N = int(round(np.exp(rng.uniform(np.log(1000.0), np.log(20000.0)))))
        r = int(rng.choice([6, 12, 16]))
        ng = int(rng.choice([64, 128]))
        width = int(rng.choice([64, 128]))
        depth = int(rng.choice([4, 5]))
        n_S = n_N if n_N <= 2000 else max(1, n_N // 20)
        grid = GridSpec(n=(ng, ng, ng), dx=1.0 / ng)
        dt = 1e-4 if ng == 64 else 5e-5
        out.append(latent_scene(seed * 1000 + i, n_N, n_S, r, width, depth, "bf16", grid, dt,
                                lo=0.3, hi=0.7, steps=steps,
                                name=f"batch{i}-{n_N}N-{n_S}S-r{r}-w{width}d{depth}-grid{ng}"))
    return out
