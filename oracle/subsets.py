"""Sample and integration particles (paper §5.4), as plain set computations.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

With S a chosen set of sample particles and x_p the particle positions at the
current latent code:

  I = { grid nodes i : N_i(x_p) != 0 for some p in S }      (step a)
  N = { particles p in P : N_i(x_p) != 0 for some i in I }   (step b)

For the quadratic B-spline N_i(x_p) != 0 exactly on the 3 x 3 x 3 nodes
base_p + {0, 1, 2}^3 with base_p = floor(x_p / dx - 0.5) (the stencil of
mpm.stencil).  The stencil base is an integer decided by floating point: the
functions here take it in the precision of the positions they are given
(``float32`` positions -> float32 products x * (1 / dx) and differences, as
the library computes them; float64 otherwise).

Order of the result: S first, in the given order, then the other members of N
in increasing particle index.
"""

import numpy as np


def stencil_base(x, dx):
    """[n, 3] integer stencil base of positions x in their own precision."""
    x = np.asarray(x)
    if x.dtype == np.float32:
        s = x * np.float32(1.0 / dx)
        return np.floor(s - np.float32(0.5)).astype(np.int64)
    s = x.astype(np.float64) / dx
    return np.floor(s - 0.5).astype(np.int64)


def stencil_nodes(base):
    """[n, 27, 3] nodes of each stencil."""
    off = np.array([(a, b, c) for a in range(3) for b in range(3) for c in range(3)],
                   dtype=np.int64)
    return base[:, None, :] + off[None, :, :]


def relevant_nodes(x_S, dx):
    """Step a: the set I of nodes in the stencils of the sample particles."""
    nodes = stencil_nodes(stencil_base(x_S, dx)).reshape(-1, 3)
    return {tuple(v) for v in nodes.tolist()}


def integration_particles(x, sample, dx):
    """Step b: the members of N, S first (given order) then ascending index.

    x: [n_all, 3] positions of all particles; sample: indices of S in P.
    """
    sample = [int(s) for s in sample]
    I = relevant_nodes(np.asarray(x)[sample], dx)
    nodes = stencil_nodes(stencil_base(x, dx))
    in_S = set(sample)
    rest = [p for p in range(nodes.shape[0])
            if p not in in_S and any(tuple(v) in I for v in nodes[p].tolist())]
    return np.array(sample + rest, dtype=np.int64)
