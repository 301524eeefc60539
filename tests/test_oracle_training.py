"""Pins of the training oracle (App. D): reverse-mode gradients against
central finite differences, Adam against its closed-form first step."""

import numpy as np

from oracle import fields as ofields
from oracle import training


def _field(rng, r=3, width=6, depth=3, out_dim=3, residual=True):
    dims = ofields.layer_dims(r, width, depth, out_dim)
    flat = np.concatenate([np.concatenate([rng.normal(0, 0.6, size=i * o), rng.normal(0, 0.2, size=o)])
                           for i, o in dims])
    scale = rng.uniform(0.5, 2.0, size=out_dim)
    shift = rng.normal(0, 0.1, size=out_dim)
    return flat, ofields.Field(flat, r, width, depth, out_dim, scale, shift, residual=residual)


def _loss(flat, r, width, depth, od, scale, shift, residual, X, zt, code, target):
    f = ofields.Field(flat, r, width, depth, od, scale, shift, residual=residual)
    return training.loss_and_grads(f, X, zt, code, target)[0]


def test_weight_and_code_gradients_match_central_differences(rng):
    for residual, od in ((True, 3), (False, 6)):
        flat, f = _field(rng, out_dim=od, residual=residual)
        n, r = 17, 3
        X = rng.uniform(0, 1, size=(n, 3))
        zt = rng.normal(0, 0.5, size=(4, r))
        code = rng.integers(0, 4, size=n)
        target = rng.normal(0, 1, size=(n, od))
        L, grads, gz = training.loss_and_grads(f, X, zt, code, target)
        gw = training.flatten_grads(grads)
        h = 1e-6
        args = (r, 6, 3, od, f.scale, f.shift, residual, X, zt, code, target)
        for k in rng.choice(flat.size, size=25, replace=False):
            fp, fm = flat.copy(), flat.copy()
            fp[k] += h
            fm[k] -= h
            fd = (_loss(fp, *args) - _loss(fm, *args)) / (2 * h)
            assert abs(fd - gw[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, gw[k])
        for c in range(4):
            for j in range(r):
                zp, zm = zt.copy(), zt.copy()
                zp[c, j] += h
                zm[c, j] -= h
                fd = (_loss(flat, r, 6, 3, od, f.scale, f.shift, residual, X, zp, code, target) -
                      _loss(flat, r, 6, 3, od, f.scale, f.shift, residual, X, zm, code, target)) / (2 * h)
                assert abs(fd - gz[c, j]) <= 1e-6 * max(1.0, abs(fd)), (c, j)


def test_gradient_vanishes_at_the_fit():
    # targets produced by the field itself: zero loss, zero gradient
    rng = np.random.Generator(np.random.PCG64(5))
    _, f = _field(rng)
    X = rng.uniform(0, 1, size=(9, 3))
    zt = rng.normal(size=(2, 3))
    code = rng.integers(0, 2, size=9)
    target = np.stack([f.value(X[p:p + 1], zt[code[p]])[0] for p in range(9)])
    L, grads, gz = training.loss_and_grads(f, X, zt, code, target)
    assert L < 1e-28
    assert np.abs(training.flatten_grads(grads)).max() < 1e-14
    assert np.abs(gz).max() < 1e-14


def test_adam_first_step_moves_by_lr_times_sign():
    g = np.array([3.0, -0.5, 1e-3, -7.0])
    p, m, v = training.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=1e-3, eps=0.0)
    np.testing.assert_allclose(p, -1e-3 * np.sign(g), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_closed_form():
    # with g fixed, m_t = g (1 - b1^t) and v_t = g^2 (1 - b2^t) (geometric
    # sums), so the bias-corrected moments are exactly g and g^2 and every
    # step moves by lr * sign(g): after T steps p = -T lr sign(g)
    g = np.array([2.0, -0.25, 5e-3])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    T, lr = 20, 1e-2
    for t in range(1, T + 1):
        p, m, v = training.adam_step(p, g, m, v, t, lr=lr, eps=0.0)
        np.testing.assert_allclose(m, g * (1 - 0.9 ** t), rtol=1e-12)
        np.testing.assert_allclose(v, g * g * (1 - 0.999 ** t), rtol=1e-12)
    np.testing.assert_allclose(p, -T * lr * np.sign(g), rtol=1e-10)


def test_adam_alternating_gradient_second_step_by_hand():
    # g then -g: m_2 = 0.9 * 0.1 g - 0.1 g = -0.01 g, v_2 = (0.999 * 0.001 + 0.001) g^2
    # = 0.001999 g^2; bias-corrected: m = -0.01 g / 0.19, v = g^2, so the second
    # step moves p by +lr * (1 / 19) sign(g) after the first step's -lr sign(g)
    g = np.array([4.0, -3.0])
    p, m, v = training.adam_step(np.zeros(2), g, np.zeros(2), np.zeros(2), 1, lr=1.0, eps=0.0)
    p, m, v = training.adam_step(p, -g, m, v, 2, lr=1.0, eps=0.0)
    np.testing.assert_allclose(m, -0.01 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001999 * g * g, rtol=1e-12)
    np.testing.assert_allclose(p, (-1.0 + 1.0 / 19.0) * np.sign(g), rtol=1e-12)
