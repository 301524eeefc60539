"""GPU parity of the field networks (§4.2-§4.4, §5.1) against the FP64 oracle.

FP32 path: outputs and dg/dz within 1e-5 relative (norm-wise over all points)
of the oracle evaluated on the same float32 weights.  Several widths, depths
and latent sizes, with point counts that leave a ragged last tile.
"""

import numpy as np
import pytest

from _support import oracle_fields, rel, soa
from scenes.synthetic import make_fields

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def nsf():
    import paper_2310_17790_gb300 as m
    return m


def _eval(nsf, spec, X, z):
    import torch
    F = nsf.Fields.from_spec(spec)
    Xd = soa(X)
    n = X.shape[0]
    zd = torch.tensor(z, dtype=torch.float64, device="cuda")
    x = torch.empty(3, n, device="cuda")
    tau = torch.empty(6, n, device="cuda")
    Cm = torch.empty(9, n, device="cuda")
    J = torch.empty(3 * spec.r, n, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    nsf.nsf_eval_fields(F, Xd, zd, x, tau, Cm, J, st)
    torch.cuda.synchronize()
    assert st.item() == 0
    return (x.cpu().numpy().T.astype(np.float64), tau.cpu().numpy().T.astype(np.float64),
            Cm.cpu().numpy().T.astype(np.float64),
            J.cpu().numpy().astype(np.float64).reshape(3, spec.r, n).transpose(2, 0, 1))


@pytest.mark.parametrize("r,width,depth,n", [
    (6, 64, 4, 1000), (3, 32, 2, 77), (16, 48, 3, 301), (6, 128, 5, 513),
    (1, 16, 1, 5), (6, (64, 96, 128), (3, 4, 5), 250), (12, 256, 2, 129)])
def test_fp32_fields_and_jacobian_match_oracle(nsf, r, width, depth, n):
    rng = np.random.Generator(np.random.PCG64(100 + r + n))
    spec = make_fields(rng, r, width, depth, "fp32", {"g": 1e-2, "h": 1e3, "l": 1.0})
    spec.out_shift["h"][:] = rng.normal(size=6).astype(np.float32)
    X = rng.uniform(0.3, 0.7, size=(n, 3)).astype(np.float32)
    z = rng.normal(0, 0.3, size=r)
    x, tau, Cm, J = _eval(nsf, spec, X, z)
    of = oracle_fields(spec)
    Xo = X.astype(np.float64)
    xo, Jo = of.g.value_and_jac_z(Xo, z)
    # x = X + u is returned in float32: besides the network error it carries the
    # rounding of X + u (half an ulp of |x| < 1, <= 6e-8 per coordinate)
    dx = x - xo
    assert np.linalg.norm(dx) <= FP32_TOL * np.linalg.norm(xo - Xo) + 6e-8 * np.sqrt(dx.size)
    assert rel(tau, of.h.value(Xo, z)) < FP32_TOL
    assert rel(Cm, of.l.value(Xo, z)) < FP32_TOL
    assert rel(J, Jo) < FP32_TOL


def test_eval_fields_empty_and_partial_outputs(nsf):
    import torch
    rng = np.random.Generator(np.random.PCG64(7))
    spec = make_fields(rng, 6, 32, 2, "fp32", {"g": 1e-2, "h": 1.0, "l": 1.0})
    F = nsf.Fields.from_spec(spec)
    X = soa(rng.uniform(0.3, 0.7, size=(40, 3)))
    z = torch.zeros(6, dtype=torch.float64, device="cuda")
    tau = torch.full((6, 40), float("nan"), device="cuda")
    nsf.nsf_eval_fields(F, X, z, tau6=tau)           # only h requested
    nsf.nsf_eval_fields(F, X[:, :0].contiguous(), z)  # n = 0 is a no-op
    torch.cuda.synchronize()
    assert torch.isfinite(tau).all()


def test_nonfinite_weights_rejected_on_create(nsf):
    rng = np.random.Generator(np.random.PCG64(8))
    spec = make_fields(rng, 6, 32, 2, "fp32", {"g": 1e-2, "h": 1.0, "l": 1.0})
    spec.weights["h"][5] = np.nan
    with pytest.raises(nsf.NsfError):
        nsf.Fields.from_spec(spec)


@pytest.mark.parametrize("r,width,depth,n", [
    (6, 128, 5, 1000), (6, 64, 4, 129), (16, 64, 2, 77), (3, 192, 2, 300), (1, 192, 2, 130),
    (6, (64, 128, 192), (4, 5, 2), 257)])
def test_bf16_fields_and_jacobian_match_oracle(nsf, r, width, depth, n):
    """BF16 tensor-core fields: within 2e-2 of the FP64 network on the original
    float32 weights, and within 2e-3 of the oracle's BF16 reading."""
    rng = np.random.Generator(np.random.PCG64(500 + r + n))
    spec = make_fields(rng, r, width, depth, "bf16", {"g": 1e-2, "h": 1e3, "l": 1.0})
    X = rng.uniform(0.3, 0.7, size=(n, 3)).astype(np.float32)
    z = rng.normal(0, 0.3, size=r)
    x, tau, Cm, J = _eval(nsf, spec, X, z)
    Xo = X.astype(np.float64)
    exact = oracle_fields(spec)                      # BF16 reading
    spec32 = make_fields(np.random.Generator(np.random.PCG64(0)), r, width, depth, "fp32",
                         {"g": 1.0, "h": 1.0, "l": 1.0})
    spec32.weights, spec32.out_scale, spec32.out_shift = spec.weights, spec.out_scale, spec.out_shift
    plain = oracle_fields(spec32)                    # FP64 network, float32 weights
    for of, tol in ((exact, 2e-3), (plain, 2e-2)):
        xo, Jo = of.g.value_and_jac_z(Xo, z)
        dx = x - xo
        assert np.linalg.norm(dx) <= tol * np.linalg.norm(xo - Xo) + 6e-8 * np.sqrt(dx.size)
        assert rel(tau, of.h.value(Xo, z)) < tol
        assert rel(Cm, of.l.value(Xo, z)) < tol
        assert rel(J, Jo) < tol
