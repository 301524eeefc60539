"""FP64 CPU oracle for the Neural Stress Fields latent MPM step (Zong et al. 2023).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may call it.  It shares no code, constants or helpers with the
CUDA library; both sides receive the same arrays from the seeded generators in
``scenes/`` and nothing else.

Everything here is plain NumPy in float64 and follows the paper's steps in the
paper's order and notation, so that it can be read against the paper by eye:

* ``fields``       neural deformation / stress / affine fields g, h, l
                   (§4.2-§4.4, App. E) with the analytic Jacobian dg/dz.
* ``mpm``          quadratic B-spline MLS-MPM: P2G, grid update, G2P
                   (§3.2, §3.3, Eq. 5).
* ``constitutive`` Kirchhoff stresses and return maps (App. F) plus the
                   textbook neo-Hookean model used by the elastic workloads.
* ``latent``       one reduced-order step: inference (§5.1), MPM on the
                   integration particles (§5.2), Gauss-Newton network inversion
                   (§5.3, Eq. 9).
* ``metrics``      the relative deformation error delta (Eq. 10) and the
                   dimension-reduction ratio gamma.
* ``subsets``      sample / integration particle construction (§5.4).
* ``training``     loss, reverse-mode weight / latent-code gradients and Adam
                   for fitting a field to snapshots (App. D).

Pinned by ``tests/test_oracle_*.py`` against closed forms, conservation laws,
brute force and finite differences.  Multi-step trajectories of random fields
have no external pin ("parity unpinned"); only their drift is reported.
"""

from . import constitutive, fields, latent, metrics, mpm, subsets, training  # noqa: F401
