"""Neural fields g, h, l of the reduced-order model, in float64 (oracle).

Paper: §4.2 (neural deformation field g(X, z) ~ phi(X, t)), §4.3 (neural stress
field h(X, z) ~ Kirchhoff stress tau, 6 symmetric components), §4.4 (neural
affine field l(X, z) ~ APIC affine matrix C), App. E (network architecture: the
input is [X; z] of size 3 + r, hidden layers with ELU activations, a linear
output layer) and App. D (training data normalised to zero mean / unit variance,
so every field's raw output is de-normalised by an affine map).

Weight layout (one flat float array per field): for each linear layer
l = 0 .. depth, the matrix W_l stored row-major as [out_l][in_l], followed by the
bias b_l [out_l].  Layer sizes: (3 + r) -> width -> ... -> width -> out_dim,
i.e. ``depth`` hidden layers (each followed by ELU) and one output layer.

A field's value is   y = shift + scale * MLP([X; z])   and the deformation
field is residual when requested: x = X + y.

The Jacobian dg/dz is the analytic chain rule through the layers (forward mode).
An independent reverse-mode vector-Jacobian product is provided so that the two
can pin each other, alongside central finite differences.

BF16 reading.  A field evaluated "in BF16 with FP32 accumulation" multiplies
bfloat16 operands: its weight matrices are bfloat16 values and every
activation (or tangent) that enters a matrix product is rounded to bfloat16
first, while sums, biases and the activation function stay in higher
precision.  ``Field(..., bf16_operands=True)`` evaluates exactly that
definition (in float64 otherwise); the caller passes weights already rounded
with ``round_to_bf16``.
"""

import numpy as np

OUT_DIM = {"g": 3, "h": 6, "l": 9}


def layer_dims(r, width, depth, out_dim):
    """(in, out) of every linear layer: depth hidden layers then the output layer."""
    dims = [(3 + r, width)]
    dims += [(width, width)] * (depth - 1)
    dims.append((width, out_dim))
    return dims


def n_params(r, width, depth, out_dim):
    return sum(i * o + o for i, o in layer_dims(r, width, depth, out_dim))


def unpack(flat, r, width, depth, out_dim):
    """Split a flat weight array into [(W [out,in], b [out]), ...] in float64."""
    flat = np.asarray(flat, dtype=np.float64).ravel()
    layers, off = [], 0
    for i, o in layer_dims(r, width, depth, out_dim):
        W = flat[off:off + i * o].reshape(o, i)
        off += i * o
        b = flat[off:off + o]
        off += o
        layers.append((W.copy(), b.copy()))
    if off != flat.size:
        raise ValueError(f"weight array has {flat.size} values, layout needs {off}")
    return layers


def round_to_bf16(a):
    """Round to the nearest bfloat16 value (ties to even), returned as float64.

    The value is first rounded to float32 (the storage type of the weights given
    to the library), then its low 16 mantissa bits are rounded away.
    """
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    out = u.astype(np.uint32).view(np.float32).astype(np.float64)
    return out.reshape(np.shape(a))


def elu(a):
    """ELU (Clevert et al. 2015, cited in App. E): a if a > 0 else exp(a) - 1."""
    return np.where(a > 0.0, a, np.expm1(np.minimum(a, 0.0)))


def elu_prime(a):
    """d ELU / da: 1 if a > 0 else exp(a)."""
    return np.where(a > 0.0, 1.0, np.exp(np.minimum(a, 0.0)))


def _identity(a):
    return a


def mlp_value(layers, inp, op_round=_identity):
    """Plain forward pass.  inp: [n, in_dim] -> [n, out_dim].

    op_round is applied to every hidden activation before it enters the next
    matrix product (identity, or round_to_bf16 for the BF16 reading)."""
    h = np.asarray(inp, dtype=np.float64)
    for W, b in layers[:-1]:
        h = op_round(elu(h @ W.T + b))
    W, b = layers[-1]
    return h @ W.T + b


def mlp_jvp(layers, inp, tin, op_round=_identity):
    """Forward-mode derivative.

    inp: [n, in_dim];  tin: [in_dim, k] input tangents (shared by all points).
    Returns (out [n, out_dim], dout [n, out_dim, k]) with
    dout[p, :, j] = d MLP(inp_p) / d inp . tin[:, j].
    """
    h = np.asarray(inp, dtype=np.float64)
    n = h.shape[0]
    t = np.broadcast_to(np.asarray(tin, dtype=np.float64), (n,) + np.shape(tin))
    for W, b in layers[:-1]:
        a = h @ W.T + b
        da = np.einsum("oi,nik->nok", W, t)
        h = op_round(elu(a))
        t = op_round(elu_prime(a)[:, :, None] * da)
    W, b = layers[-1]
    return h @ W.T + b, np.einsum("oi,nik->nok", W, t)


def mlp_vjp(layers, inp, cot):
    """Reverse-mode vector-Jacobian product.

    inp: [n, in_dim]; cot: [n, out_dim].  Returns (out, g) with
    g[p, :] = cot[p, :] . d MLP(inp_p) / d inp   (shape [n, in_dim]).
    """
    h = np.asarray(inp, dtype=np.float64)
    pre = []
    hs = [h]
    for W, b in layers[:-1]:
        a = h @ W.T + b
        pre.append(a)
        h = elu(a)
        hs.append(h)
    W, b = layers[-1]
    out = h @ W.T + b
    g = np.asarray(cot, dtype=np.float64) @ W          # d/dh_last
    for li in range(len(layers) - 2, -1, -1):
        W, _ = layers[li]
        g = g * elu_prime(pre[li])                      # through ELU
        g = g @ W                                       # through W
    return out, g


class Field:
    """One neural field (g, h or l) with its output de-normalisation.

    flat:  the field's weights in the flat layout above (any float dtype; the
           values are used exactly as given, so a bf16 path passes weights that
           were already rounded with ``round_to_bf16``).
    scale, shift: per-output de-normalisation, y = shift + scale * raw.
    residual: if true, value = X + y (deformation field parameterised as
              x = X + MLP, as in the workloads).
    """

    def __init__(self, flat, r, width, depth, out_dim, scale=None, shift=None,
                 residual=False, bf16_operands=False):
        self.r, self.width, self.depth, self.out_dim = r, width, depth, out_dim
        self.layers = unpack(flat, r, width, depth, out_dim)
        self.scale = np.ones(out_dim) if scale is None else np.asarray(scale, np.float64)[:out_dim]
        self.shift = np.zeros(out_dim) if shift is None else np.asarray(shift, np.float64)[:out_dim]
        self.residual = bool(residual)
        self.op_round = round_to_bf16 if bf16_operands else _identity
        if self.residual and out_dim != 3:
            raise ValueError("only a 3-output field can be residual")

    def _inp(self, X, z):
        X = np.asarray(X, dtype=np.float64).reshape(-1, 3)
        z = np.asarray(z, dtype=np.float64).ravel()
        if z.size != self.r:
            raise ValueError("latent size mismatch")
        return X, np.hstack([X, np.broadcast_to(z, (X.shape[0], self.r))])

    def value(self, X, z):
        X, inp = self._inp(X, z)
        y = self.shift + self.scale * mlp_value(self.layers, inp, self.op_round)
        return X + y if self.residual else y

    def value_and_jac_z(self, X, z):
        """Value and J[p, a, k] = d value_a(X_p, z) / d z_k (forward mode)."""
        X, inp = self._inp(X, z)
        tin = np.zeros((3 + self.r, self.r))
        tin[3:, :] = np.eye(self.r)
        out, dout = mlp_jvp(self.layers, inp, tin, self.op_round)
        y = self.shift + self.scale * out
        J = self.scale[None, :, None] * dout
        return (X + y if self.residual else y), J

    def vjp_z(self, X, z, cot):
        """cot . d value / d z per point, by reverse mode: [n, r]."""
        X, inp = self._inp(X, z)
        _, g = mlp_vjp(self.layers, inp, np.asarray(cot, np.float64) * self.scale)
        return g[:, 3:]


def voigt_to_sym(t6):
    """6 stress components in the order (xx, yy, zz, yz, xz, xy) -> [n, 3, 3]."""
    t6 = np.asarray(t6, dtype=np.float64).reshape(-1, 6)
    T = np.empty((t6.shape[0], 3, 3))
    T[:, 0, 0], T[:, 1, 1], T[:, 2, 2] = t6[:, 0], t6[:, 1], t6[:, 2]
    T[:, 1, 2] = T[:, 2, 1] = t6[:, 3]
    T[:, 0, 2] = T[:, 2, 0] = t6[:, 4]
    T[:, 0, 1] = T[:, 1, 0] = t6[:, 5]
    return T


def sym_to_voigt(T):
    T = np.asarray(T, dtype=np.float64).reshape(-1, 3, 3)
    return np.stack([T[:, 0, 0], T[:, 1, 1], T[:, 2, 2],
                     T[:, 1, 2], T[:, 0, 2], T[:, 0, 1]], axis=1)
