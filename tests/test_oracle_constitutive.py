"""Pins of the FP64 constitutive oracle (App. F): closed forms at F = I and for
diagonal F, rotation covariance, SVD conventions, and the yield surfaces."""

import numpy as np
import pytest

from oracle import constitutive as cm


def _rot(rng, n):
    Q, _ = np.linalg.qr(rng.normal(size=(n, 3, 3)))
    Q[np.linalg.det(Q) < 0, :, 0] *= -1
    return Q


def test_lame_parameters_closed_form():
    mu, lam = cm.lame(1e5, 0.3)
    assert mu == pytest.approx(1e5 / 2.6, rel=1e-15)
    assert lam == pytest.approx(3e4 / (1.3 * 0.4), rel=1e-15)
    assert cm.bulk(1e5, 0.3) == pytest.approx(1e5 / 1.2, rel=1e-15)
    # kappa = lambda + 2 mu / 3
    assert cm.bulk(1e5, 0.3) == pytest.approx(lam + 2 * mu / 3, rel=1e-14)


@pytest.mark.parametrize("model", ["neo_hookean", "fixed_corotated", "hencky"])
def test_zero_stress_at_identity(model):
    f = {"neo_hookean": cm.neo_hookean, "fixed_corotated": cm.fixed_corotated,
         "hencky": cm.hencky}[model]
    np.testing.assert_allclose(f(np.eye(3)[None], 3.0, 5.0), 0.0, atol=1e-14)


def test_diagonal_closed_forms():
    mu, lam = 3.0, 5.0
    a, b, c = 1.3, 0.9, 1.1
    F = np.diag([a, b, c])[None]
    J = a * b * c
    nh = cm.neo_hookean(F, mu, lam)[0]
    np.testing.assert_allclose(nh, mu * (np.diag([a * a, b * b, c * c]) - np.eye(3))
                               + lam * np.log(J) * np.eye(3), rtol=1e-14)
    fc = cm.fixed_corotated(F, mu, lam)[0]
    np.testing.assert_allclose(fc, 2 * mu * np.diag([(a - 1) * a, (b - 1) * b, (c - 1) * c])
                               + lam * (J - 1) * J * np.eye(3), rtol=1e-13, atol=1e-13)
    he = cm.hencky(F, mu, lam)[0]
    eps = np.log([a, b, c])
    np.testing.assert_allclose(he, np.diag(2 * mu * eps + lam * eps.sum()), rtol=1e-13, atol=1e-13)
    # uniaxial neo-Hookean: tau = mu diag(a^2 - 1, 0, 0) + lambda ln a I
    nh1 = cm.neo_hookean(np.diag([a, 1, 1])[None], mu, lam)[0]
    np.testing.assert_allclose(nh1, mu * np.diag([a * a - 1, 0, 0]) + lam * np.log(a) * np.eye(3),
                               rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("model", ["neo_hookean", "fixed_corotated", "hencky"])
def test_isotropic_rotation_covariance(rng, model):
    f = {"neo_hookean": cm.neo_hookean, "fixed_corotated": cm.fixed_corotated,
         "hencky": cm.hencky}[model]
    F = np.eye(3) + 0.2 * rng.normal(size=(20, 3, 3))
    Q = _rot(rng, 20)
    t0 = f(F, 2.0, 3.0)
    t1 = f(Q @ F, 2.0, 3.0)
    np.testing.assert_allclose(t1, Q @ t0 @ np.transpose(Q, (0, 2, 1)), atol=1e-12)
    np.testing.assert_allclose(t0, np.transpose(t0, (0, 2, 1)), atol=1e-12)


def test_svd_conventions(rng):
    F = rng.normal(size=(200, 3, 3))
    F[:3] = np.diag([1.0, 1.0, -1.0])                  # pure reflection
    F[3] = np.diag([2.0, 2.0, 2.0])                    # repeated values
    U, s, V = cm.svd3(F)
    np.testing.assert_allclose(np.einsum("nij,nj,nkj->nik", U, s, V), F, atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(U), 1.0, atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(V), 1.0, atol=1e-13)
    np.testing.assert_allclose(U @ np.transpose(U, (0, 2, 1)), np.broadcast_to(np.eye(3), U.shape),
                               atol=1e-13)
    assert np.all(np.abs(s[:, 0]) >= np.abs(s[:, 1]) - 1e-12)
    assert np.all(s[:, 1] >= np.abs(s[:, 2]) - 1e-12)
    np.testing.assert_allclose(np.sign(s[:, 2]), np.sign(np.linalg.det(F)))


def _hencky_eps(Fe):
    _, s, _ = cm.svd3(Fe)
    return np.log(np.abs(s))


def test_von_mises_return_map(rng):
    mu, tau_y = 1e4 / 2.6, 450.0
    F = np.eye(3) + 0.05 * rng.normal(size=(300, 3, 3))
    Fe = cm.von_mises(F, mu, tau_y)
    e0, e1 = _hencky_eps(F), _hencky_eps(Fe)
    d0 = np.linalg.norm(e0 - e0.mean(1, keepdims=True), axis=1)
    d1 = np.linalg.norm(e1 - e1.mean(1, keepdims=True), axis=1)
    inside = d0 <= tau_y / (2 * mu)
    assert inside.any() and (~inside).any()
    np.testing.assert_allclose(Fe[inside], F[inside], atol=1e-12)
    np.testing.assert_allclose(d1[~inside], tau_y / (2 * mu), rtol=1e-9)
    # volume (trace of the Hencky strain) is preserved by the deviatoric flow
    np.testing.assert_allclose(e1.sum(1), e0.sum(1), atol=1e-12)


def test_drucker_prager_return_map(rng):
    mu, lam = cm.lame(1e4, 0.3)
    phi = 30.0
    F = np.eye(3) + 0.05 * rng.normal(size=(400, 3, 3))
    Fe = cm.drucker_prager(F, mu, lam, phi)
    U, s, V = cm.svd3(F)
    e0 = np.log(np.abs(s))
    tr = e0.sum(1)
    nrm = np.linalg.norm(e0 - tr[:, None] / 3, axis=1)
    sphi = np.sin(np.deg2rad(phi))
    alpha = np.sqrt(2 / 3) * 2 * sphi / (3 - sphi)
    dg = nrm + alpha * (3 * lam + 2 * mu) * tr / (2 * mu)
    expand = tr > 0
    inside = (~expand) & (dg <= 0)
    proj = (~expand) & (dg > 0)
    assert expand.any() and inside.any() and proj.any()
    # tension: the elastic part collapses to the rotation U V^T (sigma -> 1)
    np.testing.assert_allclose(Fe[expand], (U @ np.transpose(V, (0, 2, 1)))[expand], atol=1e-12)
    np.testing.assert_allclose(Fe[inside], F[inside], atol=1e-12)
    # projected points land on the cone ||dev eps|| + alpha (3 lam + 2 mu) tr eps / (2 mu) = 0
    e1 = _hencky_eps(Fe[proj])
    t1 = e1.sum(1)
    n1 = np.linalg.norm(e1 - t1[:, None] / 3, axis=1)
    np.testing.assert_allclose(n1 + alpha * (3 * lam + 2 * mu) * t1 / (2 * mu), 0.0, atol=1e-12)
    np.testing.assert_allclose(t1, tr[proj], atol=1e-12)
