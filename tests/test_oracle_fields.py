"""Pins of the FP64 field oracle (§4.2-§4.4, App. E): hand-computed networks,
central finite differences, forward vs reverse mode, bf16 rounding vs torch."""

import numpy as np
import pytest

from oracle import fields


def test_elu_values():
    a = np.array([-2.0, -1.0, 0.0, 0.5, 3.0])
    np.testing.assert_allclose(fields.elu(a), [np.exp(-2) - 1, np.exp(-1) - 1, 0, 0.5, 3.0],
                               rtol=1e-15)
    np.testing.assert_allclose(fields.elu_prime(a), [np.exp(-2), np.exp(-1), 1.0, 1.0, 1.0],
                               rtol=1e-15)


def test_weight_layout_against_hand_computed_network():
    # r = 1, width 2, depth 1, out 3: input [X; z] of size 4.
    W0 = np.array([[1.0, 0.0, 0.0, 2.0],
                   [0.0, -1.0, 0.0, 0.0]])
    b0 = np.array([0.5, -0.25])
    W1 = np.array([[1.0, 0.0], [0.0, 1.0], [2.0, -3.0]])
    b1 = np.array([0.1, 0.2, 0.3])
    flat = np.concatenate([W0.ravel(), b0, W1.ravel(), b1])
    f = fields.Field(flat, r=1, width=2, depth=1, out_dim=3,
                     scale=[1.0, 2.0, 1.0], shift=[0.0, 0.0, 1.0], residual=True)
    X = np.array([[0.2, 0.3, 0.4]])
    z = np.array([-0.4])
    a0 = 0.2 + 2 * (-0.4) + 0.5          # -0.1 -> ELU = e^-0.1 - 1
    a1 = -0.3 - 0.25                      # -0.55
    h = np.array([np.expm1(a0), np.expm1(a1)])
    raw = np.array([h[0] + 0.1, h[1] + 0.2, 2 * h[0] - 3 * h[1] + 0.3])
    expect = X[0] + np.array([0.0, 0.0, 1.0]) + np.array([1.0, 2.0, 1.0]) * raw
    np.testing.assert_allclose(f.value(X, z)[0], expect, rtol=1e-14)
    # dx/dz by hand: only W0[0,3] = 2 connects z to the hidden layer
    dh0 = np.exp(a0) * 2.0
    J = np.array([1.0 * dh0, 0.0, 2.0 * dh0]) * np.array([1.0, 2.0, 1.0])
    _, Jo = f.value_and_jac_z(X, z)
    np.testing.assert_allclose(Jo[0, :, 0], J, rtol=1e-14)


@pytest.mark.parametrize("depth,width,r,out", [(1, 4, 3, 3), (3, 8, 6, 6), (4, 6, 16, 9)])
def test_jacobian_matches_central_differences(rng, depth, width, r, out):
    n = fields.n_params(r, width, depth, out)
    flat = rng.normal(size=n) * 0.7
    f = fields.Field(flat, r, width, depth, out, scale=rng.uniform(0.5, 2, out),
                     shift=rng.normal(size=out), residual=(out == 3))
    X = rng.uniform(0, 1, size=(7, 3))
    z = rng.normal(size=r) * 0.5
    _, J = f.value_and_jac_z(X, z)
    for h in (1e-3, 1e-5):
        fd = np.empty_like(J)
        for k in range(r):
            e = np.zeros(r)
            e[k] = h
            fd[:, :, k] = (f.value(X, z + e) - f.value(X, z - e)) / (2 * h)
        tol = 5e-5 if h == 1e-3 else 1e-8
        np.testing.assert_allclose(J, fd, atol=tol, rtol=tol)


def test_forward_mode_equals_reverse_mode(rng):
    r, width, depth, out = 6, 16, 4, 9
    flat = rng.normal(size=fields.n_params(r, width, depth, out)) * 0.5
    f = fields.Field(flat, r, width, depth, out, scale=rng.uniform(0.5, 2, out))
    X = rng.uniform(0, 1, size=(5, 3))
    z = rng.normal(size=r)
    _, J = f.value_and_jac_z(X, z)
    for a in range(out):
        cot = np.zeros((5, out))
        cot[:, a] = 1.0
        np.testing.assert_allclose(f.vjp_z(X, z, cot), J[:, a, :], rtol=1e-12, atol=1e-14)


def test_round_to_bf16_matches_torch(rng):
    torch = pytest.importorskip("torch")
    a = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-6, 6, size=5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0]]).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(fields.round_to_bf16(a), ref)


def test_voigt_roundtrip(rng):
    t6 = rng.normal(size=(4, 6))
    T = fields.voigt_to_sym(t6)
    assert np.allclose(T, np.transpose(T, (0, 2, 1)))
    assert T[0, 1, 2] == t6[0, 3] and T[0, 0, 2] == t6[0, 4] and T[0, 0, 1] == t6[0, 5]
    np.testing.assert_array_equal(fields.sym_to_voigt(T), t6)


def test_bf16_operand_reading_against_hand_computed_network():
    # same network as the layout test, with every GEMM operand rounded to bf16:
    # the hidden activation is rounded before the output product, the output
    # itself is not; the tangent is rounded the same way
    W0 = np.array([[1.0, 0.0, 0.0, 2.0],
                   [0.0, -1.0, 0.0, 0.0]])
    b0 = np.array([0.5, -0.25])
    W1 = np.array([[1.0, 0.0], [0.0, 1.0], [2.0, -3.0]])
    b1 = np.array([0.1, 0.2, 0.3])
    flat = np.concatenate([W0.ravel(), b0, W1.ravel(), b1])
    f = fields.Field(flat, r=1, width=2, depth=1, out_dim=3, residual=False,
                     bf16_operands=True)
    X = np.array([[0.2, 0.3, 0.4]])
    z = np.array([-0.4])
    a0, a1 = 0.2 + 2 * (-0.4) + 0.5, -0.3 - 0.25
    h = fields.round_to_bf16(np.array([np.expm1(a0), np.expm1(a1)]))
    expect = np.array([h[0] + 0.1, h[1] + 0.2, 2 * h[0] - 3 * h[1] + 0.3])
    np.testing.assert_allclose(f.value(X, z)[0], expect, rtol=1e-15)
    assert not np.allclose(expect, fields.Field(flat, 1, 2, 1, 3).value(X, z)[0], rtol=1e-6)
    t0 = fields.round_to_bf16(np.exp(a0) * 2.0)
    _, J = f.value_and_jac_z(X, z)
    np.testing.assert_allclose(J[0, :, 0], [t0, 0.0, 2.0 * t0], rtol=1e-15)
