"""Helpers shared by the tests: moving seeded scenes to both sides.

The oracle side receives float64 copies of the same float32 arrays the library
receives; nothing here computes any part of the method.
"""

import numpy as np

from oracle import fields as ofields
from oracle import latent as olatent
from oracle import mpm as ompm

FIELD_KEYS = ("g", "h", "l")


def bf16_weights(flat, r, width, depth, out_dim):
    """Round the weight matrices (not the biases) of a flat field to bf16,
    as the library's BF16 path stores them."""
    flat = np.asarray(flat, np.float64).copy()
    off = 0
    for i, o in ofields.layer_dims(r, width, depth, out_dim):
        flat[off:off + i * o] = ofields.round_to_bf16(flat[off:off + i * o])
        off += i * o + o
    return flat


def oracle_fields(spec, bf16_operands=None):
    """Oracle fields for a FieldSpec.  A bf16 spec uses bf16-rounded weight
    matrices and (by default) the BF16 reading of the products."""
    if bf16_operands is None:
        bf16_operands = spec.precision == "bf16"
    fs = []
    for i, k in enumerate(FIELD_KEYS):
        w = np.asarray(spec.weights[k], np.float64)
        if spec.precision == "bf16":
            w = bf16_weights(w, spec.r, spec.width[i], spec.depth[i], ofields.OUT_DIM[k])
        fs.append(ofields.Field(w, spec.r, spec.width[i], spec.depth[i], ofields.OUT_DIM[k],
                                spec.out_scale[k], spec.out_shift[k],
                                residual=(k == "g" and spec.residual_g),
                                bf16_operands=bf16_operands))
    return olatent.Fields(*fs)


def oracle_grid(g):
    return ompm.Grid(g.n, g.dx, g.gravity, g.wall_cells, g.blade)


def soa(a, device="cuda"):
    import torch
    a = np.asarray(a, dtype=np.float32)
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(device)


def aos(t):
    return t.detach().cpu().numpy().astype(np.float64).T.copy()


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.linalg.norm((a - b).ravel())
    nb = np.linalg.norm(b.ravel())
    return d / nb if nb > 0 else d


def dense_grid(t, n):
    """[n0*n1*n2*4] tap -> (m [n0,n1,n2], vec [n0,n1,n2,3])."""
    a = t.detach().cpu().numpy().astype(np.float64).reshape(n[0], n[1], n[2], 4)
    return a


def grid_desc(nsf, g):
    return nsf.grid_desc(g.n, g.dx, g.gravity, g.wall_cells, g.blade)
