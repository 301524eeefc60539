"""One reduced-order (latent) MPM step, in float64 (oracle).

Paper §5: (1) network inference (§5.1), (2) one MPM step on the integration
particles N (§5.2), (3) network inversion by Gauss-Newton (§5.3, Eq. 9).

Readings (listed in the design notes):
* The sample particles S are the first n_S integration particles.
* The first step has no z_{n-1}; callers pass z_prev = z_0 (zero velocity).
* Gauss-Newton runs a fixed number of iterations (default 5, no early exit),
  starting from z_n, with absolute damping:  (J^T J + lambda I) dz = -J^T res.
* Only x^{n+1} on S is used after the MPM step (§5.2 says S is exact; v, C and
  F of G2P are regenerated from the fields at the next step).
"""

import numpy as np

from .fields import voigt_to_sym
from .mpm import g2p, grid_update, p2g


class Fields:
    """The three fields g (residual deformation), h (stress), l (affine)."""

    def __init__(self, g, h, l):
        self.g, self.h, self.l = g, h, l


class SingularSystem(RuntimeError):
    pass


def inference(fields, X, z_n, z_prev, dt):
    """§5.1: x^n = g(X, z_n), v^n = (g(X, z_n) - g(X, z_{n-1})) / dt,
    tau^n = h(X, z_n) (Voigt -> symmetric), C^n = l(X, z_n) (row-major 3x3)."""
    x_n = fields.g.value(X, z_n)
    x_prev = fields.g.value(X, z_prev)
    v_n = (x_n - x_prev) / dt
    tau6 = fields.h.value(X, z_n)
    C9 = fields.l.value(X, z_n)
    return dict(x_n=x_n, x_prev=x_prev, v_n=v_n, tau6=tau6, C9=C9)


def mpm_substep(x_n, v_n, tau6, C9, mass, vol0, dt, grid, t, n_S):
    """§5.2: one MPM step of §3.3 on all integration particles; returns the
    grid (m, p after P2G, v after the update) and x^{n+1} on the first n_S."""
    tau = voigt_to_sym(tau6)
    C = np.asarray(C9, np.float64).reshape(-1, 3, 3)
    m_grid, p_grid, ok = p2g(x_n, v_n, C, tau, mass, vol0, dt, grid)
    v_grid = grid_update(m_grid, p_grid, dt, grid, t)
    x_next, ok_s = g2p(np.asarray(x_n)[:n_S], v_grid, dt, grid)
    return dict(m_grid=m_grid, p_grid=p_grid, v_grid=v_grid, x_next_S=x_next,
                in_grid=bool(ok.all() and ok_s.all()))


def gauss_newton(g, X_S, target, z0, iters=5, damping=1e-6):
    """§5.3, Eq. 9: z = argmin sum_{p in S} || g(X_p, z) - x_p^{n+1} ||^2.

    Each iteration linearises g around z with its Jacobian J = dg/dz, solves the
    damped normal equations (J^T J + damping I) dz = -J^T res by Cholesky and
    updates z += dz.  Returns (z, [z after each iteration], final residual).
    """
    z = np.asarray(z0, np.float64).copy()
    r = z.size
    target = np.asarray(target, np.float64).reshape(-1, 3)
    hist = []
    for _ in range(iters):
        val, J = g.value_and_jac_z(X_S, z)
        res = (val - target).reshape(-1)
        Jm = J.reshape(-1, r)
        A = Jm.T @ Jm + damping * np.eye(r)
        b = -Jm.T @ res
        try:
            L = np.linalg.cholesky(A)
        except np.linalg.LinAlgError as e:
            raise SingularSystem(str(e)) from e
        y = np.linalg.solve(L, b)
        dz = np.linalg.solve(L.T, y)
        z = z + dz
        hist.append(z.copy())
    val = g.value(X_S, z)
    resid = val - target
    return z, hist, resid


def latent_step(fields, X, n_S, mass, vol0, z_n, z_prev, dt, grid, t=0.0,
                iters=5, damping=1e-6):
    """One full latent step; returns (z_{n+1}, taps of every stage)."""
    X = np.asarray(X, np.float64).reshape(-1, 3)
    inf = inference(fields, X, z_n, z_prev, dt)
    sub = mpm_substep(inf["x_n"], inf["v_n"], inf["tau6"], inf["C9"], mass,
                      vol0, dt, grid, t, n_S)
    z, hist, resid = gauss_newton(fields.g, X[:n_S], sub["x_next_S"], z_n,
                                  iters, damping)
    taps = dict(inf)
    taps.update(sub)
    taps.update(z_hist=np.array(hist), residual=resid)
    return z, taps
