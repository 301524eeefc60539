"""Error and reduction measures of §6 (oracle)."""

import numpy as np


def relative_deformation_error(g_traj, phi_traj):
    """Eq. 10: delta = sqrt( sum_{n,p} ||g(X_p, z_n) - phi(X_p, t_n)||^2
                             / sum_{n,p} ||phi(X_p, t_n)||^2 ).

    g_traj, phi_traj: [steps, particles, 3] (any leading shape)."""
    g = np.asarray(g_traj, np.float64)
    phi = np.asarray(phi_traj, np.float64)
    return float(np.sqrt(((g - phi) ** 2).sum() / (phi ** 2).sum()))


def reduction_ratio(n_particles, r):
    """gamma = 3 |P| / r (§6): full-order dimension over latent dimension."""
    return 3.0 * n_particles / r
