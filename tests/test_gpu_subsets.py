"""GPU parity of the integration-particle construction (paper §5.4).

The stencil bases are integers decided by float32 positions, so both sides
take them from the same positions: the library's own g(X, z) read through
nsf_eval_fields (the value of a point does not depend on the launch that
computes it).  The index list must then equal the oracle's exactly, S first.
The construction is also checked by what it is for (§5.2): an MPM step on the
constructed N moves the sample particles as a step on all of P does, up to the
order of the float32 P2G atomics.
"""

import numpy as np
import pytest

from _support import grid_desc, soa
from oracle import subsets
from scenes.synthetic import GridSpec, latent_config3, tiny_latent

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nsf():
    import paper_2310_17790_gb300 as m
    return m


def _positions(nsf, F, X, z):
    import torch
    x = torch.empty_like(X)
    nsf.nsf_eval_fields(F, X, z, x=x)
    torch.cuda.synchronize()
    return x.cpu().numpy().T.copy()            # float32 [n, 3]


def _run(nsf, sc, sample, precision=None):
    import torch
    F = nsf.Fields.from_spec(sc.fields)
    X = soa(sc.X)
    z = torch.tensor(sc.z0, dtype=torch.float64, device="cuda")
    smp = torch.tensor(sample, dtype=torch.int32, device="cuda")
    gd = grid_desc(nsf, sc.grid)
    idx, XN, status = nsf.integration_set(F, gd, X, smp, z)
    x32 = _positions(nsf, F, X, z)
    return idx.cpu().numpy(), XN.cpu().numpy().T, status, x32


@pytest.mark.parametrize("precision,n,n_S,r,width,depth,n_grid", [
    ("fp32", 2000, 40, 6, 32, 2, 16), ("bf16", 3000, 7, 12, 64, 3, 32),
    ("bf16", 1500, 300, 6, 128, 4, 16), ("fp32", 257, 1, 3, 32, 2, 16)])
def test_index_list_matches_oracle_exactly(nsf, precision, n, n_S, r, width, depth, n_grid):
    sc = tiny_latent(70 + n_S, n_N=n, n_S=n_S, r=r, width=width, depth=depth,
                     precision=precision, n_grid=n_grid)
    rng = np.random.Generator(np.random.PCG64(n_S))
    sample = rng.choice(n, size=n_S, replace=False)
    idx, XN, status, x32 = _run(nsf, sc, sample)
    assert status == 0
    ref = subsets.integration_particles(x32, sample, sc.grid.dx)
    np.testing.assert_array_equal(idx, ref)
    np.testing.assert_array_equal(XN, sc.X[ref])
    assert n_S <= idx.size <= n


def test_paper_scale_200k_slab_700_samples(nsf):
    # the config-3 reference domain: 200,000 particles, 700 random samples
    from scenes.synthetic import slab_lattice
    base = latent_config3(precision="bf16", n_N=10000, n_S=700)
    rng = np.random.Generator(np.random.PCG64(2400))
    P, _, _ = slab_lattice(rng, dx=base.grid.dx)
    sc = base
    sc.X = P
    sample = rng.choice(P.shape[0], size=700, replace=False)
    idx, XN, status, x32 = _run(nsf, sc, sample)
    assert status == 0
    ref = subsets.integration_particles(x32, sample, sc.grid.dx)
    np.testing.assert_array_equal(idx, ref)
    print(f"|N| = {idx.size} of {P.shape[0]} for |S| = 700")


def test_empty_and_full_sample_sets(nsf):
    sc = tiny_latent(77, n_N=500, n_S=10)
    idx, _, status, _ = _run(nsf, sc, np.zeros(0, np.int64))
    assert status == 0 and idx.size == 0
    allp = np.arange(500)[::-1].copy()
    idx, XN, status, _ = _run(nsf, sc, allp)
    assert status == 0
    np.testing.assert_array_equal(idx, allp)


def test_sample_outside_the_grid_is_reported(nsf):
    sc = tiny_latent(78, n_N=300, n_S=5)
    sc.X[0] = (0.02, 0.5, 0.5)                 # stencil below node 0
    idx, _, status, _ = _run(nsf, sc, np.array([0, 1, 2]))
    assert status == nsf._native.NSF_ERR_OUT_OF_GRID


def test_mpm_step_on_integration_particles_moves_samples_as_on_all(nsf):
    # §5.2: the sample particles' x^{n+1} from an MPM step on N equals the one
    # from a step on all of P (both scenes list S first)
    import torch
    sc = tiny_latent(79, n_N=4000, n_S=30, r=6, width=32, depth=2, n_grid=32,
                     lo=0.3, hi=0.7)
    rng = np.random.Generator(np.random.PCG64(79))
    sample = rng.choice(4000, size=30, replace=False)
    idx, XN, status, _ = _run(nsf, sc, sample)
    assert status == 0 and idx.size < 4000
    rest = np.setdiff1d(np.arange(4000), sample)
    XP = np.concatenate([sc.X[sample], sc.X[rest]])
    zp = sc.z0 - 0.05 * rng.normal(size=sc.z0.size)
    F = nsf.Fields.from_spec(sc.fields)
    out = []
    for Xs in (XP, XN):
        X = soa(Xs)
        st = nsf.LatentStepper(F, X, 30, sc.mass, sc.vol0, grid_desc(nsf, sc.grid))
        tgt = torch.zeros(3, 30, device="cuda")
        taps = nsf._native.nsf_latent_taps()
        taps.u_next_S = tgt.data_ptr()
        z = torch.tensor(sc.z0, device="cuda")
        zpv = torch.tensor(zp, device="cuda")
        st.step(z, zpv, sc.dt, nsteps=1, taps=taps)
        torch.cuda.synchronize()
        assert st.read_status() == 0
        out.append(tgt.cpu().numpy().astype(np.float64))
    err = np.abs(out[0] - out[1]).max() / sc.grid.dx
    print(f"|N| = {idx.size} of 4000; x^(n+1) on S differs by {err:.2e} dx")
    assert err < 1e-5
    # and without the construction (a random subset of the same size) it does not
    other = np.concatenate([sample, rng.choice(rest, size=idx.size - 30, replace=False)])
    X = soa(sc.X[other])
    st = nsf.LatentStepper(F, X, 30, sc.mass, sc.vol0, grid_desc(nsf, sc.grid))
    tgt = torch.zeros(3, 30, device="cuda")
    taps = nsf._native.nsf_latent_taps()
    taps.u_next_S = tgt.data_ptr()
    st.step(torch.tensor(sc.z0, device="cuda"), torch.tensor(zp, device="cuda"), sc.dt,
            nsteps=1, taps=taps)
    torch.cuda.synchronize()
    err_rand = np.abs(tgt.cpu().numpy() - out[0]).max() / sc.grid.dx
    print(f"random subset of the same size: {err_rand:.2e} dx")
    assert err_rand > 100 * max(err, 1e-9)
