"""nsf_project_static: the network inversion for callers that cannot allocate
device memory (their host application owns all device allocations, or they run
in a loop that must not enter the CUDA allocator).  It must give the same
result as nsf_project with a caller workspace, call after call, although its
scratch is one fixed array inside the library that every call reuses.

This file is collected last on purpose, so that a failure here leaves every
other test already run; it also passes when run alone in a fresh process.
"""

import numpy as np
import pytest

from _support import oracle_fields, soa
from scenes.synthetic import make_fields

pytestmark = pytest.mark.gpu

Z_TOL = 1e-4


@pytest.fixture(scope="module")
def nsf():
    import paper_2310_17790_gb300 as m
    return m


@pytest.mark.parametrize("precision,r,n_S,width,depth", [
    ("fp32", 6, 700, 64, 4), ("bf16", 6, 700, 128, 5), ("bf16", 16, 2048, 64, 3)])
def test_static_scratch_matches_workspace_call_twice_in_a_row(nsf, precision, r, n_S, width,
                                                              depth):
    import torch
    rng = np.random.Generator(np.random.PCG64(900 + r + n_S))
    spec = make_fields(rng, r, width, depth, precision, {"g": 0.2, "h": 1.0, "l": 1.0})
    F = nsf.Fields.from_spec(spec)
    X = rng.uniform(0.3, 0.7, size=(n_S, 3)).astype(np.float32)
    of = oracle_fields(spec)
    z_star = rng.normal(0, 0.3, size=r)
    Xd = soa(X)
    opts = nsf.gn_opts(5, 1e-6)
    z0 = z_star + 0.05 * rng.normal(size=r)
    z_ws = torch.tensor(z0, device="cuda")
    z_st = torch.tensor(z0, device="cuda")
    st_ws = torch.zeros(1, dtype=torch.int32, device="cuda")
    st_st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.zeros(nsf.nsf_project_workspace_size(F, n_S), dtype=torch.uint8, device="cuda")
    for call in range(2):
        # a new target each call: the second call starts from the first one's z
        target = soa(of.g.value(X, z_star + 0.01 * call * rng.normal(size=r)))
        nsf.nsf_project(F, Xd, target, z_ws, opts, ws, st_ws)
        nsf.nsf_project_static(F, Xd, target, z_st, opts, st_st)
        torch.cuda.synchronize()
        assert st_ws.item() == 0 and st_st.item() == 0
        a, b = z_st.cpu().numpy(), z_ws.cpu().numpy()
        assert np.abs(a - b).max() <= Z_TOL * max(1.0, np.abs(b).max()), (call, a, b)


def test_static_scratch_rejects_oversized_problems(nsf):
    import torch
    rng = np.random.Generator(np.random.PCG64(901))
    spec = make_fields(rng, 6, 32, 2, "fp32", {"g": 0.2, "h": 1.0, "l": 1.0})
    F = nsf.Fields.from_spec(spec)
    n = nsf._native.NSF_PROJECT_STATIC_MAX_S + 1
    X = torch.zeros(3, n, device="cuda")
    z = torch.zeros(6, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(nsf.NsfError) as e:
        nsf.nsf_project_static(F, X, X, z, nsf.gn_opts(), st)
    assert e.value.status == nsf._native.NSF_ERR_WORKSPACE
