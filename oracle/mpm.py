"""Explicit MLS-MPM transfers with quadratic B-splines, in float64 (oracle).

Paper: §3.2 (MPM discretisation; w_ip = N(x_p - x_i); the grid force of the
node force balance, Eq. 5, is -sum_p tau_p grad(w_ip) V_p^0) and §3.3 (the
explicit MPM algorithm: P2G with the APIC momentum, grid update with gravity
and boundary conditions, G2P of v, x, C and the deformation-gradient update;
``full_step`` composes them with the stress and return map of App. F).

Conventions (shared with the library only through its documentation):

* Grid nodes are indexed (i, j, k) in [0, n_x) x [0, n_y) x [0, n_z); node i
  sits at x_i = i * dx.
* Quadratic B-spline (b = 2): base = floor(x_p / dx - 0.5), fx = x_p / dx - base
  in [0.5, 1.5); per axis the three weights of nodes base + {0, 1, 2} are
  0.5 (1.5 - fx)^2, 0.75 - (fx - 1)^2, 0.5 (fx - 0.5)^2.
* A particle whose stencil leaves the grid is "out of grid": it is skipped and
  reported, never clamped.
* grad="mls" (default) uses the MLS approximation grad(w_ip) = w_ip D^-1 (x_i - x_p)
  with D^-1 = 4 / dx^2 for the quadratic B-spline, which folds the stress force
  into the APIC affine term.  grad="bspline" uses the exact B-spline gradient.
* The APIC affine factor of G2P is 12 / (dx^2 (b + 1)) = 4 / dx^2 (§3.3).
* Grid update (§3.3): for m_i > 0, v_i = p_i / m_i + dt g; nodes with m_i = 0
  get v_i = 0 and no boundary condition.  Boundary conditions, in this order:
  walls (a node within ``wall_cells`` cells of a domain face has the velocity
  component pointing into that face set to zero) then a sticky blade (nodes with
  |x_i - blade_x| < dx and z_i > blade_z(t) move with the blade).
"""

import numpy as np


class Grid:
    """Background grid and boundary conditions of one scene."""

    def __init__(self, n, dx, gravity=(0.0, 0.0, 0.0), wall_cells=0,
                 blade=None):
        self.n = tuple(int(v) for v in n)
        self.dx = float(dx)
        self.gravity = np.asarray(gravity, dtype=np.float64)
        self.wall_cells = int(wall_cells)
        # blade: dict(x=plane x, z0=lower edge at t = 0, vz=velocity along z)
        self.blade = blade


def kernel_1d(u):
    """Textbook quadratic B-spline N(u) of u = (x_p - x_i) / dx (used by tests)."""
    a = np.abs(u)
    return np.where(a < 0.5, 0.75 - a * a,
                    np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))


def stencil(x, dx):
    """base [n,3] int, fx [n,3], w [n,3,3] and dw [n,3,3] (axis, node offset a).

    dw[p, d, a] is d w / d x_p along axis d for node offset a.
    """
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    s = x / dx
    base = np.floor(s - 0.5).astype(np.int64)
    fx = s - base
    w = np.stack([0.5 * (1.5 - fx) ** 2,
                  0.75 - (fx - 1.0) ** 2,
                  0.5 * (fx - 0.5) ** 2], axis=2)
    dw = np.stack([fx - 1.5, -2.0 * (fx - 1.0), fx - 0.5], axis=2) / dx
    return base, fx, w, dw


def in_grid(base, n):
    """True where the whole 3x3x3 stencil lies inside the grid."""
    n = np.asarray(n)
    return np.all((base >= 0) & (base + 2 <= n - 1), axis=1)


def _offsets():
    for a in range(3):
        for b in range(3):
            for c in range(3):
                yield a, b, c


def p2g(x, v, C, tau, mass, vol0, dt, grid, grad="mls"):
    """P2G of §3.3 with the stress force of Eq. 5 folded in.

    x, v: [n,3]; C: [n,3,3] affine matrices; tau: [n,3,3] Kirchhoff stresses;
    mass, vol0: scalars or [n].  Returns (m [nx,ny,nz], p [nx,ny,nz,3], ok [n])
    where p_i = m_i v_i^n + dt f_i is the momentum after the force of Eq. 5:
      m_i = sum_p w_ip m_p
      p_i = sum_p w_ip m_p (v_p + C_p (x_i - x_p)) - dt sum_p V_p^0 tau_p grad(w_ip).
    """
    x = np.asarray(x, np.float64).reshape(-1, 3)
    v = np.asarray(v, np.float64).reshape(-1, 3)
    C = np.asarray(C, np.float64).reshape(-1, 3, 3)
    tau = np.asarray(tau, np.float64).reshape(-1, 3, 3)
    npart = x.shape[0]
    mass = np.broadcast_to(np.asarray(mass, np.float64), (npart,))
    vol0 = np.broadcast_to(np.asarray(vol0, np.float64), (npart,))
    dx = grid.dx
    base, fx, w, dw = stencil(x, dx)
    ok = in_grid(base, grid.n)
    m_grid = np.zeros(grid.n)
    p_grid = np.zeros(grid.n + (3,))
    x, v, C, tau, mass, vol0 = x[ok], v[ok], C[ok], tau[ok], mass[ok], vol0[ok]
    base, fx, w, dw = base[ok], fx[ok], w[ok], dw[ok]
    Dinv = 4.0 / (dx * dx)
    for a, b, c in _offsets():
        off = np.array([a, b, c])
        idx = base + off
        wip = w[:, 0, a] * w[:, 1, b] * w[:, 2, c]
        dpos = (off[None, :] - fx) * dx                      # x_i - x_p
        if grad == "mls":
            gradw = (wip * Dinv)[:, None] * dpos
        elif grad == "bspline":
            gradw = np.stack([dw[:, 0, a] * w[:, 1, b] * w[:, 2, c],
                              w[:, 0, a] * dw[:, 1, b] * w[:, 2, c],
                              w[:, 0, a] * w[:, 1, b] * dw[:, 2, c]], axis=1)
        else:
            raise ValueError(grad)
        apic = v + np.einsum("nij,nj->ni", C, dpos)
        mom = (wip * mass)[:, None] * apic
        force = -vol0[:, None] * np.einsum("nij,nj->ni", tau, gradw)
        key = (idx[:, 0], idx[:, 1], idx[:, 2])
        np.add.at(m_grid, key, wip * mass)
        np.add.at(p_grid, key, mom + dt * force)
    return m_grid, p_grid, ok


def grid_update(m_grid, p_grid, dt, grid, t=0.0):
    """Grid update of §3.3: v_i = p_i / m_i + dt g, then the boundary conditions.

    t is the time at the start of the step (moves the blade).
    """
    m = np.asarray(m_grid, np.float64)
    p = np.asarray(p_grid, np.float64)
    v = np.zeros_like(p)
    has = m > 0.0
    v[has] = p[has] / m[has][:, None] + dt * grid.gravity
    nx, ny, nz = grid.n
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                          indexing="ij")
    idx = (I, J, K)
    wc = grid.wall_cells
    if wc > 0:
        for d in range(3):
            lo = (idx[d] < wc) & (v[..., d] < 0.0) & has
            hi = (idx[d] > grid.n[d] - 1 - wc) & (v[..., d] > 0.0) & has
            v[..., d][lo | hi] = 0.0
    if grid.blade is not None:
        bz = grid.blade["z0"] + grid.blade["vz"] * t
        xi = I * grid.dx
        zi = K * grid.dx
        sel = (np.abs(xi - grid.blade["x"]) < grid.dx) & (zi > bz) & has
        v[sel] = np.array([0.0, 0.0, grid.blade["vz"]])
    return v


def g2p(x, v_grid, dt, grid, full=False, grad="mls"):
    """G2P of §3.3.

    Returns x^{n+1} = x^n + dt v_p with v_p = sum_i w_ip v_i.  With full=True
    also returns v_p, C_p = 4/dx^2 sum_i w_ip v_i (x_i - x_p)^T and the velocity
    gradient sum_i v_i grad(w_ip)^T used by the F update (equal to C_p in the
    MLS form).
    """
    x = np.asarray(x, np.float64).reshape(-1, 3)
    dx = grid.dx
    base, fx, w, dw = stencil(x, dx)
    ok = in_grid(base, grid.n)
    vp = np.zeros_like(x)
    Cp = np.zeros((x.shape[0], 3, 3))
    Gp = np.zeros((x.shape[0], 3, 3))
    bsafe = np.where(ok[:, None], base, 0)
    for a, b, c in _offsets():
        off = np.array([a, b, c])
        idx = bsafe + off
        wip = w[:, 0, a] * w[:, 1, b] * w[:, 2, c]
        vi = v_grid[idx[:, 0], idx[:, 1], idx[:, 2]]
        dpos = (off[None, :] - fx) * dx
        vp += wip[:, None] * vi
        if full:
            Cp += (4.0 / (dx * dx)) * wip[:, None, None] * vi[:, :, None] * dpos[:, None, :]
            if grad == "bspline":
                gradw = np.stack([dw[:, 0, a] * w[:, 1, b] * w[:, 2, c],
                                  w[:, 0, a] * dw[:, 1, b] * w[:, 2, c],
                                  w[:, 0, a] * w[:, 1, b] * dw[:, 2, c]], axis=1)
                Gp += vi[:, :, None] * gradw[:, None, :]
    if full and grad == "mls":
        Gp = Cp.copy()
    vp[~ok] = 0.0
    xn = x + dt * vp
    if full:
        return xn, vp, Cp, Gp, ok
    return xn, ok


def g2p_full(x, F, v_grid, dt, grid, material, grad="mls"):
    """G2P of the full-order step (§3.3) and the update of F (steps 4-6 of
    ``full_step``): v_p, x_p^{n+1}, C_p, F_trial = (I + dt grad v_p) F_p and
    F^E = Z(F_trial), the material's return map (App. F).  Returns a dict with
    x, v, C, F (= F^E), F_trial and in_grid."""
    F = np.asarray(F, np.float64).reshape(-1, 3, 3)
    x_new, v_new, C_new, G, ok = g2p(x, v_grid, dt, grid, full=True, grad=grad)
    F_trial = np.einsum("nij,njk->nik", np.eye(3) + dt * G, F)
    F_new = material.return_map(F_trial)
    return dict(x=x_new, v=v_new, C=C_new, F=F_new, F_trial=F_trial, in_grid=bool(ok.all()))


def full_step(x, v, C, F, mass, vol0, dt, grid, material, t=0.0, grad="mls"):
    """One explicit full-order MPM step of §3.3, in the paper's order.

    x, v: [n,3]; C, F: [n,3,3] (F is the elastic part F^E for the plastic
    models); material: ``constitutive.Material``.
      1. Kirchhoff stress tau_p = tau(F_p) of the material (App. F);
      2. P2G of mass, APIC momentum and the stress force of Eq. 5;
      3. grid update with gravity and the boundary conditions at time t;
      4. G2P of v_p, x_p^{n+1} = x_p + dt v_p and C_p;
      5. deformation-gradient update F_trial = (I + dt grad v_p) F_p, with the
         MLS velocity gradient grad v_p = C_p (grad="mls") or the exact
         B-spline one sum_i v_i grad(w_ip)^T (grad="bspline");
      6. the material's return map F^E = Z(F_trial) (App. F.3, F.4; the
         identity for the elastic models).
    Returns a dict with the new x, v, C, F, the trial F, the grid (m, p after
    P2G, v after the update) and in_grid (every stencil inside the grid)."""
    x = np.asarray(x, np.float64).reshape(-1, 3)
    F = np.asarray(F, np.float64).reshape(-1, 3, 3)
    tau = material.stress(F)
    m_grid, p_grid, ok = p2g(x, v, C, tau, mass, vol0, dt, grid, grad)
    v_grid = grid_update(m_grid, p_grid, dt, grid, t)
    out = g2p_full(x, F, v_grid, dt, grid, material, grad)
    out.update(m_grid=m_grid, p_grid=p_grid, v_grid=v_grid,
               in_grid=bool(ok.all() and out["in_grid"]))
    return out


def momentum(x, v, C, mass, dx):
    """Total linear and APIC angular momentum of a particle set.

    For the quadratic B-spline the APIC angular momentum of particle p is
    x_p x m_p v_p + m_p (dx^2/4) eps_abc C_cb (from the second moment of the
    weights); P2G maps it exactly onto sum_i x_i x p_i when tau is symmetric.
    """
    x = np.asarray(x, np.float64).reshape(-1, 3)
    v = np.asarray(v, np.float64).reshape(-1, 3)
    C = np.asarray(C, np.float64).reshape(-1, 3, 3)
    mass = np.broadcast_to(np.asarray(mass, np.float64), (x.shape[0],))
    P = (mass[:, None] * v).sum(0)
    L = np.cross(x, mass[:, None] * v).sum(0)
    spin = np.stack([C[:, 2, 1] - C[:, 1, 2],
                     C[:, 0, 2] - C[:, 2, 0],
                     C[:, 1, 0] - C[:, 0, 1]], axis=1)
    L = L + (mass[:, None] * spin).sum(0) * (dx * dx / 4.0)
    return P, L


def grid_momentum(m_grid, p_grid, dx):
    """Total linear and angular momentum of grid momenta p_i at x_i = i dx."""
    nx, ny, nz = m_grid.shape
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                          indexing="ij")
    xi = np.stack([I, J, K], axis=-1) * dx
    P = p_grid.reshape(-1, 3).sum(0)
    L = np.cross(xi.reshape(-1, 3), p_grid.reshape(-1, 3)).sum(0)
    return P, L
