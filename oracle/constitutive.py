"""Kirchhoff stresses and plastic return maps, in float64 (oracle).

Paper: App. F (Lame parameters from (E, nu); F.1 fixed corotated; F.2 StVK with
Hencky strain; F.3 Drucker-Prager; F.4 von Mises).  The neo-Hookean model used
by the elastic workloads is not in the paper; it is the textbook compressible
form tau = mu (F F^T - I) + lambda ln(J) I (Bonet & Wood; the MPM course of
Jiang et al. 2016 that §3 refers to).

Readings of printed formulas (each listed in the design notes):
* F.1 prints "lambda (J - 1) J" without the identity: read as lambda (J-1) J I.
* F.2 prints U (2 mu eps + lambda sum(eps) 1) V^T; a Kirchhoff stress is
  symmetric, so it is read as U diag(2 mu eps + lambda sum(eps)) U^T.
* F.3 "d lambda" uses d = 3 (the dimension); eps_hat = eps - sum(eps)/3.
* F.4 prints eps_hat / ||eps||: read as eps_hat / ||eps_hat||, yield test on the
  Hencky principal Kirchhoff stress, ||dev tau|| <= tau_y  <=>  dgamma <= 0.

SVD convention: F = U diag(sigma) V^T with sigma sorted descending and
det U = det V = +1; a reflection is absorbed into the smallest singular value,
which then carries the sign of det F.
"""

import numpy as np


def lame(E, nu):
    """(mu_hat, lambda) of App. F: mu = E / (2 (1 + nu)), lambda = E nu / ((1 + nu)(1 - 2 nu))."""
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def bulk(E, nu):
    return E / (3.0 * (1.0 - 2.0 * nu))


def svd3(F):
    """Rotation-preserving SVD of [n,3,3] matrices (convention above)."""
    F = np.asarray(F, np.float64).reshape(-1, 3, 3)
    U, s, Vt = np.linalg.svd(F)
    V = np.transpose(Vt, (0, 2, 1)).copy()
    U = U.copy()
    s = s.copy()
    dU = np.linalg.det(U) < 0
    U[dU, :, 2] *= -1.0
    s[dU, 2] *= -1.0
    dV = np.linalg.det(V) < 0
    V[dV, :, 2] *= -1.0
    s[dV, 2] *= -1.0
    return U, s, V


def neo_hookean(F, mu, lam):
    F = np.asarray(F, np.float64).reshape(-1, 3, 3)
    J = np.linalg.det(F)
    b = F @ np.transpose(F, (0, 2, 1))
    return mu * (b - np.eye(3)) + (lam * np.log(J))[:, None, None] * np.eye(3)


def fixed_corotated(F, mu, lam):
    """App. F.1: tau = 2 mu (F - R) F^T + lambda (J - 1) J I with R = U V^T."""
    F = np.asarray(F, np.float64).reshape(-1, 3, 3)
    U, s, V = svd3(F)
    R = U @ np.transpose(V, (0, 2, 1))
    J = np.prod(s, axis=1)
    return (2.0 * mu * (F - R) @ np.transpose(F, (0, 2, 1))
            + (lam * (J - 1.0) * J)[:, None, None] * np.eye(3))


def hencky(F, mu, lam):
    """App. F.2 (StVK with Hencky strain): tau = U diag(2 mu eps + lambda tr eps) U^T."""
    U, s, V = svd3(F)
    eps = np.log(np.maximum(np.abs(s), 1e-12))
    d = 2.0 * mu * eps + lam * eps.sum(axis=1, keepdims=True)
    return np.einsum("nij,nj,nkj->nik", U, d, U)


def von_mises(F, mu, tau_y):
    """App. F.4 return map (no hardening or softening): returns F^E."""
    U, s, V = svd3(F)
    eps = np.log(np.maximum(np.abs(s), 1e-12))
    tr = eps.sum(axis=1, keepdims=True)
    eh = eps - tr / 3.0
    nrm = np.linalg.norm(eh, axis=1)
    dgamma = nrm - tau_y / (2.0 * mu)
    yielded = dgamma > 0.0
    eps_new = eps.copy()
    safe = np.where(nrm > 0.0, nrm, 1.0)
    eps_new[yielded] = eps[yielded] - (dgamma / safe)[yielded, None] * eh[yielded]
    s_new = np.where(yielded[:, None], np.exp(eps_new), s)
    return np.einsum("nij,nj,nkj->nik", U, s_new, V)


def drucker_prager(F, mu, lam, friction_deg):
    """App. F.3 return map (Klar et al. 2016): returns F^E."""
    U, s, V = svd3(F)
    eps = np.log(np.maximum(np.abs(s), 1e-12))
    tr = eps.sum(axis=1)
    eh = eps - tr[:, None] / 3.0
    nrm = np.linalg.norm(eh, axis=1)
    sphi = np.sin(np.deg2rad(friction_deg))
    alpha = np.sqrt(2.0 / 3.0) * 2.0 * sphi / (3.0 - sphi)
    dgamma = nrm + alpha * (3.0 * lam + 2.0 * mu) * tr / (2.0 * mu)
    s_new = s.copy()
    expand = tr > 0.0
    s_new[expand] = 1.0
    proj = (~expand) & (dgamma > 0.0)
    safe = np.where(nrm > 0.0, nrm, 1.0)
    e2 = eps - (dgamma / safe)[:, None] * eh
    s_new[proj] = np.exp(e2[proj])
    return np.einsum("nij,nj,nkj->nik", U, s_new, V)


class Material:
    """Constitutive model of a full-order scene.

    model: "neo_hookean" | "fixed_corotated" | "von_mises" | "drucker_prager".
    The two plastic models use the Hencky (StVK) stress of their F^E.
    """

    def __init__(self, model, E, nu, yield_stress=0.0, friction_deg=30.0):
        self.model = model
        self.E, self.nu = float(E), float(nu)
        self.mu, self.lam = lame(self.E, self.nu)
        self.yield_stress = float(yield_stress)
        self.friction_deg = float(friction_deg)

    def stress(self, F):
        if self.model == "neo_hookean":
            return neo_hookean(F, self.mu, self.lam)
        if self.model == "fixed_corotated":
            return fixed_corotated(F, self.mu, self.lam)
        if self.model in ("von_mises", "drucker_prager"):
            return hencky(F, self.mu, self.lam)
        raise ValueError(self.model)

    def return_map(self, F):
        if self.model == "von_mises":
            return von_mises(F, self.mu, self.yield_stress)
        if self.model == "drucker_prager":
            return drucker_prager(F, self.mu, self.lam, self.friction_deg)
        return np.asarray(F, np.float64).reshape(-1, 3, 3).copy()
