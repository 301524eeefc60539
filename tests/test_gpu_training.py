"""GPU parity of field training (App. D): the library's loss and hand-written
gradients against the oracle's reverse mode (itself pinned by central
differences in test_oracle_training.py), the device-side weight re-pack
against fields built from the same host weights, Adam against its textbook
update, and a short training run against the oracle's trajectory.

Tolerances: FP32 fields 1e-5 on the loss and 1e-4 (norm-wise) on the
gradients (FP32 accumulation of sums over up to 1,000 points); BF16 fields
(bf16 operands in the forward products, the oracle's BF16 reading; backward
products with the cotangent split into bf16 hi + lo, ~16 significant bits;
ELU' kept as a 16-bit fixed-point code, absolute error <= 2^-16) 2e-3 on the
gradients: an activation whose FP32 and FP64 pre-activations round to
different bf16 values moves by one bf16 ulp.
"""

import numpy as np
import pytest

from _support import bf16_weights, rel, soa
from oracle import fields as ofields
from oracle import training as otraining
from scenes.synthetic import make_fields

pytestmark = pytest.mark.gpu

FIELD_KEYS = ("g", "h", "l")


@pytest.fixture(scope="module")
def nsf():
    import paper_2310_17790_gb300 as m
    return m


def _spec(seed, precision, r=6, width=64, depth=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    return make_fields(rng, r, width, depth, precision, {"g": 1e-2, "h": 3e3, "l": 1.0})


def _oracle_field(spec, k):
    i = FIELD_KEYS.index(k)
    w = np.asarray(spec.weights[k], np.float64)
    if spec.precision == "bf16":
        w = bf16_weights(w, spec.r, spec.width[i], spec.depth[i], ofields.OUT_DIM[k])
    return ofields.Field(w, spec.r, spec.width[i], spec.depth[i], ofields.OUT_DIM[k],
                         spec.out_scale[k], spec.out_shift[k], residual=(k == "g"),
                         bf16_operands=spec.precision == "bf16")


def _data(seed, n, r, n_codes, od, k):
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.uniform(0.3, 0.7, size=(n, 3)).astype(np.float32)
    z = rng.normal(0, 0.3, size=(n_codes, r)).astype(np.float32)
    code = rng.integers(0, n_codes, size=n).astype(np.int32)
    scale = {"g": 1e-2, "h": 3e3, "l": 1.0}[k]
    target = (rng.normal(0, 1, size=(n, od)) * scale).astype(np.float32)
    if k == "g":
        target += X
    return X, z, code, target


def _gpu_loss_grad(nsf, F, k, X, z, code, target):
    import torch
    field = nsf.FIELD_INDEX[k]
    n = X.shape[0]
    Xd, td = soa(X), soa(target)
    zd = torch.from_numpy(z).cuda()
    cd = torch.from_numpy(code).cuda()
    nw = nsf.nsf_field_weight_count(F, field)
    gw = torch.empty(nw, device="cuda")
    gz = torch.empty_like(zd)
    loss = torch.zeros(1, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.zeros(nsf.nsf_train_workspace_size(F, field, n), dtype=torch.uint8, device="cuda")
    nsf.nsf_field_loss_grad(F, field, Xd, cd, td, zd, loss, gw, gz, ws, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return float(loss.item()), gw.cpu().numpy().astype(np.float64), gz.cpu().numpy().astype(np.float64)


# BF16 shapes beyond the benchmark's: a width of 192 (a partial second
# 128-channel tile of the hidden-layer products), 256 at depth 1 (no hidden
# product), r = 16 (19 inputs, the widest thin-K and input-layer kernels),
# field l's 9 outputs, and point counts off every tile size
@pytest.mark.parametrize("precision,k,width,depth,r,n", [
    ("fp32", "g", 64, 3, 6, 1000), ("fp32", "h", 64, 4, 6, 1000), ("fp32", "l", 128, 2, 6, 1000),
    ("bf16", "g", 128, 5, 6, 1000), ("bf16", "h", 64, 3, 6, 1000),
    ("bf16", "l", 192, 3, 6, 1000), ("bf16", "g", 256, 1, 16, 777),
    ("bf16", "h", 64, 4, 16, 129), ("bf16", "g", 256, 3, 3, 2049),
    ("bf16", "g", 128, 3, 6, 1), ("bf16", "l", 256, 2, 6, 3)])
def test_loss_and_gradients_match_oracle(nsf, precision, k, width, depth, r, n):
    spec = _spec(7, precision, r=r, width=width, depth=depth)
    F = nsf.Fields.from_spec(spec)
    od = ofields.OUT_DIM[k]
    X, z, code, target = _data(8, n, spec.r, 5, od, k)
    L, gw, gz = _gpu_loss_grad(nsf, F, k, X, z, code, target)
    of = _oracle_field(spec, k)
    L_o, grads, gz_o = otraining.loss_and_grads(of, X, z.astype(np.float64), code,
                                                target.astype(np.float64))
    gw_o = otraining.flatten_grads(grads)
    tol = 1e-4 if precision == "fp32" else 2e-3
    print(f"{precision} {k}: loss {L:.6e} vs {L_o:.6e}; grad_w rel {rel(gw, gw_o):.2e}; "
          f"grad_z rel {rel(gz, gz_o):.2e}")
    assert abs(L - L_o) <= (1e-5 if precision == "fp32" else 1e-3) * L_o
    assert rel(gw, gw_o) < tol
    assert rel(gz, gz_o) < tol


def test_loss_grad_rejects_an_empty_batch(nsf):
    """n = 0 points through the C ABI itself: an argument error, nothing enqueued."""
    import torch
    spec = _spec(23, "bf16", width=128, depth=3)
    F = nsf.Fields.from_spec(spec)
    X, z, code, target = _data(24, 4, spec.r, 2, ofields.OUT_DIM["g"], "g")
    field = nsf.FIELD_INDEX["g"]
    nw = nsf.nsf_field_weight_count(F, field)
    Xd, td = soa(X), soa(target)
    cd, zd = torch.from_numpy(code).cuda(), torch.from_numpy(z).cuda()
    loss, gw = torch.zeros(1, device="cuda"), torch.empty(nw, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.zeros(nsf.nsf_train_workspace_size(F, field, 4), dtype=torch.uint8, device="cuda")
    rc = nsf._native.lib.nsf_field_loss_grad(F.handle, field, Xd.data_ptr(), cd.data_ptr(),
                                             td.data_ptr(), 0, zd.data_ptr(), zd.shape[0],
                                             loss.data_ptr(), gw.data_ptr(), None, ws.data_ptr(),
                                             ws.numel(), st.data_ptr(), None)
    assert rc == nsf._native.NSF_ERR_INVALID_ARG


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_loss_and_gradients_are_reproducible_bit_for_bit(nsf, precision):
    """Every sum behind the loss and the gradients (weight slabs, bias column
    sums, the input layer's per-CTA partials, the per-CTA loss partials, the
    latent codes' per-CTA tables) runs in a fixed order, so two calls on the
    same data agree in every bit."""
    spec = _spec(21, precision, width=256 if precision == "bf16" else 64, depth=3)
    F = nsf.Fields.from_spec(spec)
    X, z, code, target = _data(22, 4099, spec.r, 7, ofields.OUT_DIM["g"], "g")
    runs = [_gpu_loss_grad(nsf, F, "g", X, z, code, target) for _ in range(2)]
    assert runs[0][0] == runs[1][0]
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    np.testing.assert_array_equal(runs[0][2], runs[1][2])


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_set_weights_equals_fields_built_from_the_same_weights(nsf, precision):
    import torch
    spec = _spec(11, precision, width=128, depth=4)
    other = _spec(12, precision, width=128, depth=4)
    F = nsf.Fields.from_spec(spec)
    for k in FIELD_KEYS:
        nsf.nsf_fields_set_weights(F, nsf.FIELD_INDEX[k],
                                   torch.from_numpy(np.asarray(other.weights[k], np.float32)).cuda())
    G = nsf.Fields.from_spec(other)
    rng = np.random.Generator(np.random.PCG64(13))
    X = soa(rng.uniform(0.3, 0.7, size=(777, 3)))
    z = torch.tensor(rng.normal(0, 0.1, size=spec.r), device="cuda")
    outs = []
    for fld in (F, G):
        x = torch.empty(3, 777, device="cuda")
        tau = torch.empty(6, 777, device="cuda")
        C9 = torch.empty(9, 777, device="cuda")
        J = torch.empty(3 * spec.r, 777, device="cuda")
        nsf.nsf_eval_fields(fld, X, z, x=x, tau6=tau, C9=C9, dxdz=J)
        torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in (x, tau, C9, J)])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)


def test_adam_matches_textbook_update(nsf):
    import torch
    rng = np.random.Generator(np.random.PCG64(14))
    p = rng.normal(size=4097)
    m, v = np.zeros_like(p), np.zeros_like(p)
    pd = torch.tensor(p, dtype=torch.float32, device="cuda")
    md, vd = torch.zeros_like(pd), torch.zeros_like(pd)
    for t in range(1, 4):
        g = rng.normal(size=p.size)
        gd = torch.tensor(g, dtype=torch.float32, device="cuda")
        nsf.nsf_adam_step(pd, gd, md, vd, t, 1e-3)
        p, m, v = otraining.adam_step(p, g.astype(np.float32).astype(np.float64), m, v, t, 1e-3)
    torch.cuda.synchronize()
    assert np.abs(pd.cpu().numpy() - p).max() < 1e-6


def test_autograd_function_gives_the_library_gradients(nsf):
    import torch
    spec = _spec(15, "fp32")
    F = nsf.Fields.from_spec(spec)
    X, z, code, target = _data(16, 500, spec.r, 3, 3, "g")
    w = torch.tensor(np.asarray(spec.weights["g"], np.float32), device="cuda", requires_grad=True)
    zt = torch.tensor(z, device="cuda", requires_grad=True)
    loss = nsf.field_loss(w, zt, F, "g", soa(X), torch.from_numpy(code).cuda(), soa(target))
    (3.0 * loss).backward()
    of = _oracle_field(spec, "g")
    L_o, grads, gz_o = otraining.loss_and_grads(of, X, z.astype(np.float64), code,
                                                target.astype(np.float64))
    assert abs(float(loss.item()) - L_o) <= 1e-5 * L_o
    assert rel(w.grad.cpu().numpy(), 3.0 * otraining.flatten_grads(grads)) < 1e-4
    assert rel(zt.grad.cpu().numpy(), 3.0 * gz_o) < 1e-4


def test_training_run_tracks_oracle_and_reduces_the_loss(nsf):
    # fit g to targets made by a teacher field of the same shape
    import torch
    spec = _spec(17, "fp32", width=64, depth=3)
    teacher = _spec(18, "fp32", width=64, depth=3)
    n, r, nc = 2000, spec.r, 4
    rng = np.random.Generator(np.random.PCG64(19))
    X = rng.uniform(0.3, 0.7, size=(n, 3))
    z_true = rng.normal(0, 0.3, size=(nc, r))
    code = rng.integers(0, nc, size=n).astype(np.int32)
    tf = _oracle_field(teacher, "g")
    tgt = np.empty((n, 3))
    for c in range(nc):
        tgt[code == c] = tf.value(X[code == c], z_true[c])
    z0 = (z_true + rng.normal(0, 0.1, size=z_true.shape)).astype(np.float32)
    F = nsf.Fields.from_spec(spec)
    w0 = np.asarray(spec.weights["g"], np.float32)
    tr = nsf.FieldTrainer(F, "g", torch.from_numpy(w0).cuda(), torch.from_numpy(z0).cuda(), n,
                          lr=1e-3)
    Xd, cd, td = soa(X.astype(np.float32)), torch.from_numpy(code).cuda(), soa(tgt.astype(np.float32))
    # oracle trajectory of the same run
    of = _oracle_field(spec, "g")
    p = np.concatenate([w0.astype(np.float64), z0.astype(np.float64).ravel()])
    m, v = np.zeros_like(p), np.zeros_like(p)
    nw = w0.size
    losses, losses_o = [], []
    for t in range(1, 31):
        losses.append(float(tr.step(Xd, cd, td).item()))
        if t <= 3:
            of = ofields.Field(p[:nw], r, 64, 3, 3, spec.out_scale["g"], spec.out_shift["g"],
                               residual=True)
            L_o, grads, gz = otraining.loss_and_grads(of, X, p[nw:].reshape(nc, r), code, tgt)
            losses_o.append(L_o)
            g = np.concatenate([otraining.flatten_grads(grads), gz.ravel()])
            p, m, v = otraining.adam_step(p, g, m, v, t, 1e-3)
    torch.cuda.synchronize()
    print("losses", [f"{x:.4e}" for x in losses[:3]], "oracle", [f"{x:.4e}" for x in losses_o],
          "last", f"{losses[-1]:.4e}")
    for a, b in zip(losses[:3], losses_o):
        assert abs(a - b) <= 1e-3 * b
    assert losses[-1] < 0.5 * losses[0]
