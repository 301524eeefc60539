"""Fitting a neural field to full-order snapshots (App. D), in float64 (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Each training point p is a particle of a snapshot t(p): input [X_p; z_t] (the
snapshot's latent code, learned jointly with the weights), target y*_p (the
snapshot's deformed position for g, stress for h, affine matrix for l).  The
training data are normalised (App. D): with the field's de-normalisation
y = shift + scale * raw, the loss is the mean squared normalised error

    L = 1 / (n * out_dim) * sum_p sum_a ((y_pa - y*_pa) / scale_a)^2,

and its gradient with respect to the weights of every linear layer and to the
latent codes follows the chain rule backwards through the layers (reverse
mode).  Adam (Kingma and Ba 2014, cited in App. D) updates the parameters.

``op_round`` is the reading of the BF16 forward pass (fields.round_to_bf16 on
every hidden activation entering a product); the backward pass is float64 on
the activations the forward pass produced.
"""

import numpy as np

from .fields import elu, elu_prime


def _identity(a):
    return a


def mlp_forward_store(layers, inp, op_round=_identity):
    """Forward pass keeping, per hidden layer, the pre-activation a_l and the
    activation h_l that enters the next product.  Returns (out, pre, hs) with
    hs[0] = inp."""
    h = np.asarray(inp, dtype=np.float64)
    pre, hs = [], [h]
    for W, b in layers[:-1]:
        a = h @ W.T + b
        pre.append(a)
        h = op_round(elu(a))
        hs.append(h)
    W, b = layers[-1]
    return h @ W.T + b, pre, hs


def mlp_param_grads(layers, inp, cot, op_round=_identity):
    """Gradient of sum_p cot_p . MLP(inp_p): per layer (dW, db) and the input
    gradient [n, in_dim]."""
    out, pre, hs = mlp_forward_store(layers, inp, op_round)
    delta = np.asarray(cot, dtype=np.float64)            # dL / d out
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        grads[li] = (delta.T @ hs[li], delta.sum(axis=0))
        g_in = delta @ W                                  # dL / d h_{li}
        if li > 0:
            delta = g_in * elu_prime(pre[li - 1])
    return out, grads, g_in


def loss_and_grads(field, X, z_table, code, target):
    """Loss L of one field on points X [n, 3] with codes z_table[code[p]] and
    targets [n, out_dim]; returns (L, weight grads, z_table grads)."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 3)
    z_table = np.asarray(z_table, dtype=np.float64)
    code = np.asarray(code)
    n, od = X.shape[0], field.out_dim
    inp = np.hstack([X, z_table[code]])
    raw, _, _ = mlp_forward_store(field.layers, inp, field.op_round)
    y = field.shift + field.scale * raw
    if field.residual:
        y = X + y
    e = (y - target) / field.scale
    L = float((e ** 2).sum() / (n * od))
    cot_raw = 2.0 * e / (n * od)                         # dL / d raw
    _, grads, g_in = mlp_param_grads(field.layers, inp, cot_raw, field.op_round)
    gz = np.zeros_like(z_table)
    np.add.at(gz, code, g_in[:, 3:])
    return L, grads, gz


def flatten_grads(grads):
    """Per-layer (dW, db) in the flat weight layout of fields.unpack."""
    return np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in grads])


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step t >= 1); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
