"""GPU parity of the full-order MLS-MPM step (§3.3) against the FP64 oracle.

Teacher-forced per stage: P2G grid (m, p) within 1e-5 relative of the oracle's
P2G of the same particle state; grid velocities within 1e-5 of the oracle's
update of the GPU's (m, p); G2P x, v, C, F within 1e-5 (relative, norm-wise;
x in dx units) of the oracle's G2P of the GPU's grid velocities.  Also exact
conservation properties measured on the GPU output.
"""

import numpy as np
import pytest

from _support import grid_desc, oracle_grid, rel, soa
from oracle import constitutive as ocm, mpm as ompm
from scenes.synthetic import GridSpec, full_scene

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def nsf():
    import paper_2310_17790_gb300 as m
    return m


def _perturb(sc, seed, v=0.05, c=2.0, f=0.02):
    rng = np.random.Generator(np.random.PCG64(seed))
    n = sc.x.shape[0]
    sc.v = (v * rng.normal(size=(n, 3))).astype(np.float32)
    sc.C = (c * rng.normal(size=(n, 9))).astype(np.float32)
    sc.F = (np.eye(3).ravel() + f * rng.normal(size=(n, 9))).astype(np.float32)
    return sc


def _run(nsf, sc, nsteps=1, t0=0.0):
    import torch
    x, v, Cm, F = soa(sc.x), soa(sc.v), soa(sc.C), soa(sc.F)
    gd = grid_desc(nsf, sc.grid)
    mat = nsf.material(**sc.material)
    st = nsf.FullStepper(gd, mat, x, v, Cm, F, sc.mass, sc.vol0)
    nodes = int(np.prod(sc.grid.n))
    tp = nsf._native.nsf_full_taps()
    gmp = torch.zeros(nodes * 4, device="cuda")
    gv = torch.zeros(nodes * 4, device="cuda")
    tp.grid_mp, tp.grid_v = gmp.data_ptr(), gv.data_ptr()
    st.step(sc.dt, t0=t0, nsteps=nsteps, taps=tp)
    torch.cuda.synchronize()
    out = dict(x=x, v=v, C=Cm, F=F)
    out = {k: t.cpu().numpy().astype(np.float64).T for k, t in out.items()}
    out["grid_mp"] = gmp.cpu().numpy().astype(np.float64).reshape(*sc.grid.n, 4)
    out["grid_v"] = gv.cpu().numpy().astype(np.float64).reshape(*sc.grid.n, 4)
    out["status"] = st.read_status()
    return out


def _check(sc, out, t0=0.0):
    assert out["status"] == 0
    og = oracle_grid(sc.grid)
    m = sc.material
    mat = ocm.Material(m["model"], m["E"], m["nu"], m.get("yield_stress", 0.0),
                       m.get("friction_deg", 30.0))
    x0 = sc.x.astype(np.float64)
    v0 = sc.v.astype(np.float64)
    C0 = sc.C.astype(np.float64).reshape(-1, 3, 3)
    F0 = sc.F.astype(np.float64).reshape(-1, 3, 3)
    tau = mat.stress(F0)
    m, p, ok = ompm.p2g(x0, v0, C0, tau, sc.mass, sc.vol0, sc.dt, og)
    assert ok.all()
    gmp = out["grid_mp"]
    assert rel(gmp[..., 0], m) < TOL
    assert rel(gmp[..., 1:], p) < TOL
    vg = ompm.grid_update(gmp[..., 0], gmp[..., 1:], sc.dt, og, t0)
    gv = out["grid_v"]
    assert rel(gv[..., :3], vg) < TOL
    # G2P, the update of F and the return map of the oracle's full step (§3.3,
    # App. F), fed the GPU's grid velocities
    g2 = ompm.g2p_full(x0, F0, gv[..., :3], sc.dt, og, mat)
    assert g2["in_grid"]
    assert np.abs(out["x"] - g2["x"]).max() / sc.grid.dx < TOL
    assert rel(out["v"], g2["v"]) < TOL
    assert rel(out["C"], g2["C"].reshape(-1, 9)) < TOL
    assert rel(out["F"], g2["F"].reshape(-1, 9)) < TOL
    return g2["F_trial"], g2["F"]


def test_full_step_small_slab_with_blade(nsf):
    sc = _perturb(full_scene(71, lattice=(30, 30, 8), n_grid=64), 71)
    sc.grid.blade = dict(x=0.5, z0=0.205, vz=-1.0)
    out = _run(nsf, sc, t0=0.002)
    _check(sc, out, t0=0.002)


def test_full_step_end_to_end_matches_oracle_full_step(nsf):
    # one step from the same state, not teacher-forced: the GPU's x, v, C, F
    # against oracle.mpm.full_step (§3.3) in float64
    sc = _perturb(full_scene(77, lattice=(24, 24, 8), n_grid=64), 77)
    out = _run(nsf, sc)
    assert out["status"] == 0
    m = sc.material
    mat = ocm.Material(m["model"], m["E"], m["nu"])
    ref = ompm.full_step(sc.x, sc.v, sc.C.reshape(-1, 3, 3), sc.F.reshape(-1, 3, 3), sc.mass,
                         sc.vol0, sc.dt, oracle_grid(sc.grid), mat)
    assert ref["in_grid"]
    assert np.abs(out["x"] - ref["x"]).max() / sc.grid.dx < TOL
    assert rel(out["v"], ref["v"]) < TOL
    assert rel(out["C"], ref["C"].reshape(-1, 9)) < TOL
    assert rel(out["F"], ref["F"].reshape(-1, 9)) < TOL


def test_full_step_dense_block_overflows_its_bucket(nsf):
    # 3,000 particles whose stencil bases all lie in one 4^3-cell block, more
    # than the 1,024 its bucket holds: the particles past the bucket add their
    # contributions to the grid directly, and the grid must still be the
    # oracle's P2G of all of them (and the step reproducible bit for bit)
    from scenes.synthetic import FullScene
    rng = np.random.Generator(np.random.PCG64(78))
    n, dx = 3000, 1.0 / 32
    # x / dx in [16.5, 20.5): stencil bases 16 .. 19, the block starting at cell 16
    x = ((16.5 + rng.uniform(0.01, 3.99, size=(n, 3))) * dx).astype(np.float32)
    vol0 = (4 * dx) ** 3 / n
    sc = FullScene(x=x, v=np.zeros((n, 3), np.float32), C=np.zeros((n, 9), np.float32),
                   F=np.tile(np.eye(3, dtype=np.float32).ravel(), (n, 1)), mass=1000.0 * vol0,
                   vol0=vol0, grid=GridSpec(n=(32, 32, 32), dx=dx, gravity=(0.0, 0.0, -9.8),
                                            wall_cells=0),
                   dt=1e-5, material=dict(model="neo_hookean", E=1e4, nu=0.3,
                                          yield_stress=0.0, friction_deg=30.0))
    sc = _perturb(sc, 78, v=0.05, c=1.0, f=0.01)
    base = np.floor(sc.x.astype(np.float64) / dx - 0.5)
    assert base.min() >= 16 and base.max() <= 19
    out = _run(nsf, sc)
    _check(sc, out)
    again = _run(nsf, sc)
    for k in ("x", "v", "C", "F", "grid_mp", "grid_v"):
        np.testing.assert_array_equal(out[k], again[k])


def test_full_step_200k_slab(nsf):
    # the 200,000-particle slab on the 128^3 grid (one step, teacher-forced)
    sc = _perturb(full_scene(72), 72)
    out = _run(nsf, sc)
    _check(sc, out)


def test_full_step_conserves_momentum_on_gpu(nsf):
    sc = _perturb(full_scene(73, lattice=(20, 20, 20), n_grid=64), 73, v=0.2, c=1.0)
    sc.grid = GridSpec(n=(64, 64, 64), dx=1.0 / 64, gravity=(0.0, 0.0, 0.0), wall_cells=0)
    P0, L0 = ompm.momentum(sc.x, sc.v, sc.C.reshape(-1, 3, 3), sc.mass, sc.grid.dx)
    out = _run(nsf, sc)
    P1, L1 = ompm.momentum(out["x"], out["v"], out["C"].reshape(-1, 3, 3), sc.mass, sc.grid.dx)
    scaleP = np.abs(sc.mass * sc.v).sum()
    assert np.abs(P1 - P0).max() < 1e-5 * scaleP
    scaleL = np.abs(np.cross(sc.x, sc.mass * sc.v)).sum()
    assert np.abs(L1 - L0).max() < 1e-5 * scaleL


def test_full_step_multi_step_stays_in_grid(nsf):
    sc = full_scene(74, lattice=(24, 24, 6), n_grid=64)
    out = _run(nsf, sc, nsteps=20)
    assert out["status"] == 0
    assert np.isfinite(out["x"]).all() and np.isfinite(out["F"]).all()


@pytest.mark.parametrize("model,extra", [
    ("fixed_corotated", {}),
    ("von_mises", {"yield_stress": 2.5e3}),
    ("drucker_prager", {"friction_deg": 30.0}),
])
def test_full_step_svd_models(nsf, model, extra):
    # float64 SVD, return map and stress on the GPU (App. F) against the oracle
    sc = _perturb(full_scene(75, lattice=(24, 24, 8), n_grid=64, model=model, **extra), 75,
                  f=0.03)
    out = _run(nsf, sc)
    Fn, Fe = _check(sc, out)
    if model != "fixed_corotated":
        # some particles must have been projected for the test to mean anything
        moved = np.linalg.norm((Fe - Fn).reshape(-1, 9), axis=1) > 1e-6
        assert moved.mean() > 0.05, moved.mean()


def test_full_step_plastic_slab_multi_step(nsf):
    # the 200k slab with von Mises (yield stress 1e4) and the blade, 10 steps
    sc = full_scene(76, model="von_mises", yield_stress=1e4)
    out = _run(nsf, sc, nsteps=10)
    assert out["status"] == 0
    assert np.isfinite(out["x"]).all() and np.isfinite(out["F"]).all()


@pytest.mark.parametrize("model", ["neo_hookean", "fixed_corotated", "von_mises", "drucker_prager"])
def test_material_stress_matches_oracle(nsf, model):
    # tau(F) of every model (App. F; textbook neo-Hookean) against the oracle
    import torch
    rng = np.random.Generator(np.random.PCG64(79))
    n = 5000
    F = (np.eye(3) + 0.05 * rng.normal(size=(n, 3, 3))).astype(np.float32)
    mat = ocm.Material(model, 2e5, 0.3, 1e4, 30.0)
    ref = mat.stress(F.astype(np.float64))
    Fd = soa(F.reshape(n, 9))
    tau = torch.zeros(6, n, device="cuda")
    nsf.nsf_material_stress(nsf.material(model, 2e5, 0.3, 1e4, 30.0), Fd, tau)
    torch.cuda.synchronize()
    from oracle import fields as ofields
    got = ofields.voigt_to_sym(tau.cpu().numpy().T.astype(np.float64))
    assert rel(got, ref) < (1e-5 if model == "neo_hookean" else 1e-6)
