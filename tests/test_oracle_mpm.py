"""Pins of the FP64 MPM oracle against what the method fixes (§3.2, §3.3, Eq. 5).

Each test checks the oracle against something other than itself: the textbook
quadratic B-spline kernel, brute force over all (node, particle) pairs, the
moment identities of the quadratic B-spline, exact conservation of mass and of
linear and angular momentum, and exact advection of rigid and affine motion.
"""

import numpy as np
import pytest

from oracle import constitutive, mpm


def _grid(n=12, dx=1.0 / 12, **kw):
    return mpm.Grid((n, n, n), dx, **kw)


def _particles(rng, npart, lo, hi):
    x = rng.uniform(lo, hi, size=(npart, 3))
    v = rng.normal(size=(npart, 3))
    C = rng.normal(size=(npart, 3, 3)) * 3.0
    A = rng.normal(size=(npart, 3, 3))
    tau = (A + np.transpose(A, (0, 2, 1))) * 50.0
    return x, v, C, tau


def test_weights_on_a_node_are_one_eighth_three_quarters_one_eighth():
    # A particle sitting on a node has 1D weights 1/8, 3/4, 1/8 (quadratic B-spline).
    dx = 0.1
    base, fx, w, _ = mpm.stencil(np.array([[0.3, 0.5, 0.7]]), dx)
    np.testing.assert_allclose(fx, 1.0, atol=1e-12)
    for d in range(3):
        np.testing.assert_allclose(w[0, d], [0.125, 0.75, 0.125], atol=1e-12)
    np.testing.assert_array_equal(base[0], [2, 4, 6])


def test_stencil_matches_textbook_kernel(rng):
    dx = 0.05
    x = rng.uniform(0.2, 0.8, size=(50, 3))
    base, fx, w, dw = mpm.stencil(x, dx)
    for a in range(3):
        xi = (base + a) * dx
        u = (x - xi) / dx
        np.testing.assert_allclose(w[:, :, a], mpm.kernel_1d(u), atol=1e-14)
        # derivative against a central difference of the kernel definition
        h = 1e-6
        fd = (mpm.kernel_1d(u + h) - mpm.kernel_1d(u - h)) / (2 * h) / dx
        np.testing.assert_allclose(dw[:, :, a], fd, atol=1e-6)


def test_bspline_moment_identities(rng):
    dx = 0.07
    x = rng.uniform(0.3, 0.7, size=(40, 3))
    base, fx, w, _ = mpm.stencil(x, dx)
    S0 = np.zeros(40)
    S1 = np.zeros((40, 3))
    S2 = np.zeros((40, 3, 3))
    for a in range(3):
        for b in range(3):
            for c in range(3):
                off = np.array([a, b, c])
                wip = w[:, 0, a] * w[:, 1, b] * w[:, 2, c]
                d = (off - fx) * dx
                S0 += wip
                S1 += wip[:, None] * d
                S2 += wip[:, None, None] * d[:, :, None] * d[:, None, :]
    np.testing.assert_allclose(S0, 1.0, atol=1e-14)
    np.testing.assert_allclose(S1, 0.0, atol=1e-15)
    np.testing.assert_allclose(S2, np.broadcast_to(np.eye(3) * dx * dx / 4, S2.shape),
                               atol=1e-15)


@pytest.mark.parametrize("grad", ["mls", "bspline"])
def test_p2g_brute_force(rng, grad):
    n, dx, dt = 7, 1.0 / 7, 1e-3
    g = mpm.Grid((n, n, n), dx)
    x, v, C, tau = _particles(rng, 11, 0.25, 0.75)
    mass = rng.uniform(0.5, 2.0, size=11)
    vol0 = rng.uniform(0.1, 0.3, size=11)
    m, p, ok = mpm.p2g(x, v, C, tau, mass, vol0, dt, g, grad=grad)
    assert ok.all()
    m_bf = np.zeros((n, n, n))
    p_bf = np.zeros((n, n, n, 3))
    hh = 1e-6
    for i in range(n):
        for j in range(n):
            for k in range(n):
                xi = np.array([i, j, k]) * dx
                for q in range(11):
                    u = (x[q] - xi) / dx
                    N = mpm.kernel_1d(u)
                    w = N.prod()
                    if w == 0.0:
                        continue
                    if grad == "mls":
                        gw = w * 4.0 / dx ** 2 * (xi - x[q])
                    else:
                        dN = (mpm.kernel_1d(u + hh) - mpm.kernel_1d(u - hh)) / (2 * hh) / dx
                        gw = np.array([dN[0] * N[1] * N[2], N[0] * dN[1] * N[2],
                                       N[0] * N[1] * dN[2]])
                    m_bf[i, j, k] += w * mass[q]
                    p_bf[i, j, k] += (w * mass[q] * (v[q] + C[q] @ (xi - x[q]))
                                      - dt * vol0[q] * tau[q] @ gw)
    np.testing.assert_allclose(m, m_bf, atol=1e-13)
    np.testing.assert_allclose(p, p_bf, atol=1e-6 if grad == "bspline" else 1e-12)


@pytest.mark.parametrize("grad", ["mls", "bspline"])
def test_p2g_conserves_mass_linear_and_angular_momentum(rng, grad):
    g = _grid()
    x, v, C, tau = _particles(rng, 300, 0.3, 0.7)
    mass, vol0, dt = 0.01, 1e-4, 1e-3
    m, p, ok = mpm.p2g(x, v, C, tau, mass, vol0, dt, g, grad=grad)
    assert ok.all()
    np.testing.assert_allclose(m.sum(), 300 * mass, rtol=1e-14)
    P0, L0 = mpm.momentum(x, v, C, mass, g.dx)
    Pg, Lg = mpm.grid_momentum(m, p, g.dx)
    np.testing.assert_allclose(Pg, P0, rtol=1e-12, atol=1e-12)
    # symmetric tau exerts no net torque; APIC angular momentum maps exactly
    np.testing.assert_allclose(Lg, L0, rtol=1e-11, atol=1e-12)


def test_p2g_flags_out_of_grid_particles():
    g = _grid()
    x = np.array([[0.5, 0.5, 0.5], [0.02, 0.5, 0.5], [0.5, 0.5, 0.98]])
    zeros = np.zeros((3, 3))
    m, p, ok = mpm.p2g(x, zeros, np.zeros((3, 3, 3)), np.zeros((3, 3, 3)),
                       1.0, 1.0, 1e-3, g)
    assert ok.tolist() == [True, False, False]
    np.testing.assert_allclose(m.sum(), 1.0)


def test_rigid_translation_is_advected_exactly(rng):
    g = _grid()
    x = rng.uniform(0.3, 0.7, size=(100, 3))
    vel = np.array([0.3, -0.2, 0.1])
    v = np.tile(vel, (100, 1))
    zero = np.zeros((100, 3, 3))
    dt = 1e-3
    m, p, _ = mpm.p2g(x, v, zero, zero, 0.02, 1e-4, dt, g)
    vg = mpm.grid_update(m, p, dt, g)
    xn, vp, Cp, Gp, ok = mpm.g2p(x, vg, dt, g, full=True)
    np.testing.assert_allclose(vp, v, atol=1e-13)
    np.testing.assert_allclose(xn, x + dt * vel, atol=1e-15)
    np.testing.assert_allclose(Cp, 0.0, atol=1e-10)


@pytest.mark.parametrize("grad", ["mls", "bspline"])
def test_g2p_reproduces_affine_velocity_fields(rng, grad):
    g = _grid()
    b = rng.normal(size=3)
    A = rng.normal(size=(3, 3))
    I, J, K = np.meshgrid(*(np.arange(12),) * 3, indexing="ij")
    xi = np.stack([I, J, K], -1) * g.dx
    vg = b + xi @ A.T
    x = rng.uniform(0.3, 0.7, size=(60, 3))
    xn, vp, Cp, Gp, ok = mpm.g2p(x, vg, 1e-3, g, full=True, grad=grad)
    np.testing.assert_allclose(vp, b + x @ A.T, atol=1e-12)
    np.testing.assert_allclose(Cp, np.broadcast_to(A, Cp.shape), atol=1e-10)
    np.testing.assert_allclose(Gp, np.broadcast_to(A, Gp.shape), atol=1e-10)


def test_free_fall_adds_dt_g():
    g = _grid(gravity=(0.0, 0.0, -9.8))
    x = np.array([[0.5, 0.45, 0.55], [0.52, 0.5, 0.5]])
    v = np.array([[0.1, 0.0, 0.0], [0.1, 0.0, 0.0]])
    zero = np.zeros((2, 3, 3))
    dt = 1e-3
    m, p, _ = mpm.p2g(x, v, zero, zero, 1.0, 1.0, dt, g)
    vg = mpm.grid_update(m, p, dt, g)
    xn, vp, Cp, Gp, ok = mpm.g2p(x, vg, dt, g, full=True)
    np.testing.assert_allclose(vp, v + dt * np.array([0, 0, -9.8]), atol=1e-13)


def test_grid_update_walls_and_blade():
    n, dx = 16, 1.0 / 16
    blade = dict(x=0.5, z0=0.6, vz=-1.0)
    g = mpm.Grid((n, n, n), dx, gravity=(0, 0, 0), wall_cells=3, blade=blade)
    m = np.ones((n, n, n))
    p = np.zeros((n, n, n, 3))
    p[..., 0] = -1.0           # every node moves towards -x
    p[..., 2] = 2.0            # and towards +z
    v = mpm.grid_update(m, p, 1e-3, g, t=0.1)
    # -x wall band: i < 3 stops the -x component, elsewhere it survives
    assert np.all(v[:3, 5:10, 5:8, 0] == 0.0)
    assert np.all(v[3:, 5:10, 5:8, 0] == -1.0)
    # +z wall band: k > n-1-3 stops the +z component
    assert np.all(v[5:7, 5:7, 13:, 2] == 0.0)
    assert np.all(v[5:7, 5:7, 5:13, 2] == 2.0)
    # blade at x = 0.5 (node 8, |x_i - 0.5| < dx -> only i = 8), above z = 0.5
    bz = 0.6 - 0.1
    sel = v[8, 5, :, :]
    for k in range(n):
        if k * dx > bz and k <= n - 1 - 3:
            np.testing.assert_array_equal(sel[k], [0.0, 0.0, -1.0])
    assert v[7, 5, 12, 2] == 2.0 and v[9, 5, 12, 0] == -1.0
    # massless nodes stay at rest and get no boundary condition
    m[4, 4, 4] = 0.0
    v = mpm.grid_update(m, p, 1e-3, g, t=0.1)
    np.testing.assert_array_equal(v[4, 4, 4], 0.0)


def test_full_step_conserves_linear_and_angular_momentum(rng):
    # One explicit step (P2G -> grid update -> G2P) with no gravity and no
    # boundary conditions conserves total linear and APIC angular momentum.
    g = _grid(n=16, dx=1.0 / 16)
    npart = 400
    x = rng.uniform(0.3, 0.7, size=(npart, 3))
    v = rng.normal(size=(npart, 3)) * 0.5
    C = rng.normal(size=(npart, 3, 3))
    F = np.eye(3) + 0.05 * rng.normal(size=(npart, 3, 3))
    mat = constitutive.Material("neo_hookean", 1e4, 0.3)
    tau = mat.stress(F)
    mass, vol0, dt = 1e-3, 1e-6, 1e-4
    m, p, _ = mpm.p2g(x, v, C, tau, mass, vol0, dt, g)
    vg = mpm.grid_update(m, p, dt, g)
    xn, vp, Cp, Gp, ok = mpm.g2p(x, vg, dt, g, full=True)
    P0, L0 = mpm.momentum(x, v, C, mass, g.dx)
    P1, L1 = mpm.momentum(xn, vp, Cp, mass, g.dx)
    np.testing.assert_allclose(P1, P0, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(L1, L0, rtol=1e-10, atol=1e-13)


def _no_stress():
    # E = 0: mu = lambda = 0, so tau(F) = 0 for any F (no grid force)
    return constitutive.Material("neo_hookean", 0.0, 0.3)


@pytest.mark.parametrize("grad", ["mls", "bspline"])
def test_full_step_affine_velocity_updates_F_in_closed_form(grad):
    # Particles moving with an affine velocity v = A x + b (C_p = A) and no
    # stress: P2G gives p_i = m_i (A x_i + b) exactly (first moment identity),
    # so v_i = A x_i + b, G2P returns v_p = A x_p + b and C_p = A (second
    # moment identity), the B-spline velocity gradient is A as well, and F
    # advects to the closed form (I + dt A) F for any F.
    rng = np.random.Generator(np.random.PCG64(601))
    g = _grid(n=16, dx=1.0 / 16)
    n = 120
    x = rng.uniform(0.3, 0.7, size=(n, 3))
    A = rng.normal(size=(3, 3))                       # not symmetric
    b = rng.normal(size=3)
    v = x @ A.T + b
    C = np.broadcast_to(A, (n, 3, 3)).copy()
    F = np.eye(3) + 0.2 * rng.normal(size=(n, 3, 3))
    dt = 1e-3
    out = mpm.full_step(x, v, C, F, 1e-3, 1e-6, dt, g, _no_stress(), grad=grad)
    assert out["in_grid"]
    np.testing.assert_allclose(out["v"], v, rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["x"], x + dt * v, rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["C"], C, rtol=0, atol=1e-10)
    expect_F = np.einsum("ij,njk->nik", np.eye(3) + dt * A, F)
    np.testing.assert_allclose(out["F"], expect_F, rtol=0, atol=1e-13)
    # a transposed update, F (I + dt A), would be off by dt |A F - F A| ~ 1e-3
    assert np.abs(np.einsum("nij,jk->nik", F, np.eye(3) + dt * A) - out["F"]).max() > 1e-5


def test_full_step_rigid_translation_leaves_F_unchanged():
    # F = I has zero neo-Hookean stress, a uniform velocity has zero gradient:
    # every particle translates by dt v and F stays the identity.
    rng = np.random.Generator(np.random.PCG64(602))
    g = _grid(n=16, dx=1.0 / 16)
    n = 90
    x = rng.uniform(0.3, 0.7, size=(n, 3))
    b = rng.normal(size=3)
    v = np.broadcast_to(b, (n, 3)).copy()
    F = np.broadcast_to(np.eye(3), (n, 3, 3)).copy()
    mat = constitutive.Material("neo_hookean", 1e5, 0.3)
    out = mpm.full_step(x, v, np.zeros((n, 3, 3)), F, 1e-3, 1e-6, 1e-4, g, mat)
    np.testing.assert_allclose(out["x"], x + 1e-4 * b, rtol=0, atol=1e-15)
    np.testing.assert_allclose(out["F"], F, rtol=0, atol=1e-13)
    np.testing.assert_allclose(out["C"], 0.0, atol=1e-11)


def test_full_step_von_mises_lands_on_the_yield_surface():
    # App. F.4 inside the step: a particle whose trial strain is past the yield
    # surface ends with ||dev eps(F^E)|| = tau_y / (2 mu) and the same volume;
    # one inside keeps F_trial, and F_trial = (I + dt C_p) F (MLS form).
    rng = np.random.Generator(np.random.PCG64(603))
    g = _grid(n=16, dx=1.0 / 16)
    n = 200
    x = rng.uniform(0.3, 0.7, size=(n, 3))
    v = 0.05 * rng.normal(size=(n, 3))
    C = rng.normal(size=(n, 3, 3))
    F = np.eye(3) + 0.03 * rng.normal(size=(n, 3, 3))
    mat = constitutive.Material("von_mises", 1e4, 0.3, yield_stress=300.0)
    dt = 1e-4
    out = mpm.full_step(x, v, C, F, 1e-3, 1e-6, dt, g, mat)
    np.testing.assert_allclose(out["F_trial"], np.einsum("nij,njk->nik",
                                                         np.eye(3) + dt * out["C"], F),
                               rtol=0, atol=1e-14)

    def dev_norm_and_trace(M):
        _, s, _ = constitutive.svd3(M)
        e = np.log(np.abs(s))
        return np.linalg.norm(e - e.mean(1, keepdims=True), axis=1), e.sum(1)

    d_tr, tr_tr = dev_norm_and_trace(out["F_trial"])
    d_new, tr_new = dev_norm_and_trace(out["F"])
    ry = mat.yield_stress / (2 * mat.mu)
    yielded = d_tr > ry
    assert 0.1 < yielded.mean() < 0.9
    np.testing.assert_allclose(d_new[yielded], ry, rtol=1e-9)
    np.testing.assert_allclose(tr_new, tr_tr, atol=1e-12)
    np.testing.assert_allclose(out["F"][~yielded], out["F_trial"][~yielded], atol=1e-14)
