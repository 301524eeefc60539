"""Pins of the sample / integration particle construction (paper §5.4)."""

import numpy as np

from oracle import subsets


def _overlap_bruteforce(x, sample, dx):
    """N by a second definition: p is in N iff its stencil and the stencil of
    some sample particle share a node, i.e. their bases differ by at most 2
    along every axis (two 3-node intervals overlap)."""
    b = subsets.stencil_base(x, dx)
    members = set(int(s) for s in sample)
    for p in range(b.shape[0]):
        for s in sample:
            if np.all(np.abs(b[p] - b[s]) <= 2):
                members.add(p)
                break
    return members


def test_matches_bruteforce_interval_overlap(rng):
    dx = 1.0 / 16
    for trial in range(5):
        x = rng.uniform(0.2, 0.8, size=(300, 3)).astype(np.float32)
        sample = rng.choice(300, size=7, replace=False)
        got = subsets.integration_particles(x, sample, dx)
        assert list(got[:7]) == list(sample)
        assert set(got.tolist()) == _overlap_bruteforce(x, sample, dx)
        rest = got[7:]
        assert np.all(np.diff(rest) > 0)
        assert not set(rest.tolist()) & set(sample.tolist())


def test_sample_set_is_contained_and_far_particles_are_not():
    dx = 0.1
    # sample at the centre of the domain; a particle 4 cells away along x has a
    # disjoint stencil, one 2 cells away shares nodes
    x = np.array([[0.55, 0.55, 0.55], [0.95, 0.55, 0.55], [0.75, 0.55, 0.55],
                  [0.55, 0.55, 0.15]], dtype=np.float64)
    got = subsets.integration_particles(x, [0], dx)
    assert list(got) == [0, 2]


def test_all_particles_in_one_cell_are_all_integration_particles(rng):
    dx = 1.0 / 32
    x = (0.5 + rng.uniform(0.0, dx, size=(50, 3))).astype(np.float32)
    got = subsets.integration_particles(x, [3], dx)
    assert sorted(got.tolist()) == list(range(50))
    assert got[0] == 3


def test_relevant_nodes_are_the_27_stencil_nodes():
    dx = 0.25
    I = subsets.relevant_nodes(np.array([[0.6, 0.6, 0.6]]), dx)
    # x / dx = 2.4 -> base = floor(1.9) = 1 -> nodes 1..3 per axis
    assert I == {(i, j, k) for i in (1, 2, 3) for j in (1, 2, 3) for k in (1, 2, 3)}
