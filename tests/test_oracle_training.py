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
