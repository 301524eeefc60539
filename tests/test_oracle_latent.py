"""Pins of the FP64 latent-step oracle (§5): Gauss-Newton on zero-residual and
linear problems, the closed-form latent step of a translation field, the
exactness of the MPM sub-step (§5.2), well-posedness (§5.4) and the printed
reduction ratios (§6)."""

import os

import numpy as np
import pytest

from oracle import constitutive, fields, latent, metrics, mpm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_field(rng, r, width=16, depth=3, out=3, residual=True, s=0.6):
    flat = rng.normal(size=fields.n_params(r, width, depth, out)) * s
    return fields.Field(flat, r, width, depth, out, scale=np.full(out, 0.05),
                        residual=residual)


def _linear_in_z_field(rng, r, width=8):
    # one hidden layer with a large positive bias keeps every ELU in its linear
    # branch, so g(X, z) = X + A X + B z + c exactly
    W0 = rng.normal(size=(width, 3 + r)) * 0.3
    b0 = np.full(width, 40.0)
    W1 = rng.normal(size=(3, width)) * 0.3
    b1 = -W1 @ b0 + 0.01 * rng.normal(size=3)    # keeps the solution z small
    flat = np.concatenate([W0.ravel(), b0, W1.ravel(), b1])
    return fields.Field(flat, r, width, 1, 3, residual=True), (W0, b0, W1, b1)


def test_gauss_newton_recovers_zero_residual_solution(rng):
    r = 6
    g = _rand_field(rng, r)
    X = rng.uniform(0.3, 0.7, size=(50, 3))
    z_star = rng.normal(size=r) * 0.3
    target = g.value(X, z_star)
    z, hist, res = latent.gauss_newton(g, X, target, z_star + 0.02 * rng.normal(size=r),
                                       iters=6, damping=1e-12)
    np.testing.assert_allclose(z, z_star, atol=1e-10)
    # quadratic convergence: the error collapses within 2-3 iterations (§5.3)
    errs = [np.abs(zh - z_star).max() for zh in hist]
    assert errs[2] < 1e-8


def test_gauss_newton_fixed_point(rng):
    g = _rand_field(rng, 6)
    X = rng.uniform(0.3, 0.7, size=(30, 3))
    z0 = rng.normal(size=6) * 0.2
    z, _, res = latent.gauss_newton(g, X, g.value(X, z0), z0, iters=5, damping=1e-6)
    np.testing.assert_allclose(z, z0, atol=1e-13)
    np.testing.assert_allclose(res, 0.0, atol=1e-13)


def test_gauss_newton_linear_field_equals_least_squares(rng):
    # a field linear in z has a constant 3 x r Jacobian, so r = 3 keeps the
    # least-squares solution unique
    r = 3
    g, (W0, b0, W1, b1) = _linear_in_z_field(rng, r)
    X = rng.uniform(0.3, 0.7, size=(40, 3))
    target = rng.uniform(0.3, 0.7, size=(40, 3))
    # g = X + W1 (W0 [X; z] + b0) + b1  ->  (W1 W0z) z = target - X - W1 (W0x X + b0) - b1
    B = W1 @ W0[:, 3:]
    rhs = target - X - (X @ W0[:, :3].T + b0) @ W1.T - b1
    A = np.tile(B, (40, 1))
    z_ls = np.linalg.lstsq(A, rhs.ravel(), rcond=None)[0]
    z, _, _ = latent.gauss_newton(g, X, target, np.zeros(r), iters=5, damping=1e-6)
    np.testing.assert_allclose(z, z_ls, rtol=1e-9, atol=1e-11)


def _translation_fields(r=3, width=4):
    # g(X, z) = X + z via an ELU network kept in its linear branch by a +20 shift
    W0 = np.zeros((width, 3 + r))
    W0[:3, 3:] = np.eye(3)
    b0 = np.full(width, 20.0)
    W1 = np.eye(width)
    b1 = np.zeros(width)
    W2 = np.zeros((3, width))
    W2[:, :3] = np.eye(3)
    b2 = np.full(3, -20.0)
    flat_g = np.concatenate([W0.ravel(), b0, W1.ravel(), b1, W2.ravel(), b2])
    g = fields.Field(flat_g, r, width, 2, 3, residual=True)
    h = fields.Field(np.zeros(fields.n_params(r, width, 2, 6)), r, width, 2, 6)
    l = fields.Field(np.zeros(fields.n_params(r, width, 2, 9)), r, width, 2, 9)
    return latent.Fields(g, h, l)


def test_latent_step_closed_form_translation(rng):
    # h = 0, l = 0, g = X + z: P2G/G2P of a uniform velocity is exact, so the
    # latent step is symplectic Euler, z_{n+1} = 2 z_n - z_{n-1} + dt^2 g.
    f = _translation_fields()
    grid = mpm.Grid((16, 16, 16), 1.0 / 16, gravity=(0.0, -3.0, -9.8))
    X = rng.uniform(0.35, 0.65, size=(80, 3))
    dt = 1e-3
    z_prev = np.array([0.01, -0.02, 0.005])
    z_n = np.array([0.012, -0.019, 0.004])
    z_next, taps = latent.latent_step(f, X, 30, 0.01, 1e-5, z_n, z_prev, dt, grid)
    expect = 2 * z_n - z_prev + dt * dt * grid.gravity
    np.testing.assert_allclose(z_next, expect, atol=1e-12)
    np.testing.assert_allclose(taps["v_n"], np.broadcast_to((z_n - z_prev) / dt, (80, 3)),
                               atol=1e-9)


def test_latent_mpm_substep_equals_full_order_step(rng):
    # §5.2: a latent MPM sub-step on N = P, fed the full-order state (x, v,
    # tau(F) as the stress field's output, C as the affine field's output),
    # moves every particle to the x^{n+1} of mpm.full_step on the same state,
    # whose transfers are pinned against brute force and closed forms in
    # test_oracle_mpm.py.
    grid = mpm.Grid((16, 16, 16), 1.0 / 16, gravity=(0, 0, -9.8), wall_cells=3)
    n = 150
    x = rng.uniform(0.3, 0.7, size=(n, 3))
    v = rng.normal(size=(n, 3)) * 0.1
    C = rng.normal(size=(n, 3, 3))
    F = np.eye(3) + 0.03 * rng.normal(size=(n, 3, 3))
    mat = constitutive.Material("neo_hookean", 1e4, 0.3)
    dt, mass, vol0 = 1e-4, 1e-3, 1e-6
    full = mpm.full_step(x, v, C, F, mass, vol0, dt, grid, mat)
    sub = latent.mpm_substep(x, v, fields.sym_to_voigt(mat.stress(F)), C.reshape(n, 9), mass,
                             vol0, dt, grid, 0.0, n)
    assert full["in_grid"] and sub["in_grid"]
    np.testing.assert_array_equal(sub["x_next_S"], full["x"])
    np.testing.assert_array_equal(sub["v_grid"], full["v_grid"])
    # a prefix S of N gets the same positions (only S is read after G2P)
    sub_S = latent.mpm_substep(x, v, fields.sym_to_voigt(mat.stress(F)), C.reshape(n, 9), mass,
                               vol0, dt, grid, 0.0, 40)
    np.testing.assert_array_equal(sub_S["x_next_S"], full["x"][:40])


def test_too_few_sample_particles_is_singular_without_damping(rng):
    # §5.4: the least-squares problem needs |S| >= r / 3.
    g = _rand_field(rng, 6)
    X = rng.uniform(0.3, 0.7, size=(1, 3))
    with pytest.raises(latent.SingularSystem):
        latent.gauss_newton(g, X, X.copy(), np.zeros(6), iters=1, damping=0.0)
    z, _, _ = latent.gauss_newton(g, X, X.copy(), np.zeros(6), iters=1, damping=1e-6)
    assert np.all(np.isfinite(z))


def test_reduction_ratio_matches_printed_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "reduction_ratio.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for name, npart, r, gam, tol, *_ in rows:
        got = metrics.reduction_ratio(int(npart), int(r))
        assert abs(got - float(gam)) <= float(tol) * float(gam) + 1e-9, name


def test_relative_deformation_error():
    phi = np.ones((2, 4, 3))
    assert metrics.relative_deformation_error(phi, phi) == 0.0
    g = phi * 1.01
    assert metrics.relative_deformation_error(g, phi) == pytest.approx(0.01, rel=1e-12)
