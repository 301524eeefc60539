"""GB300 (sm_103a) latent MPM step of Neural Stress Fields (Zong et al. 2023).

Python binding of libnsf (include/nsf.h).  PyTorch only provides device memory
and streams; every computation runs in the library's CUDA kernels, and the
binding raises if the library is not built.  Particle arrays are float32
component-major tensors of shape [k, n] on the current CUDA device; latent
codes are float64 tensors of shape [r].

The functions named after the C entry points (``nsf_latent_step`` ...) take
torch tensors and forward them one to one; ``Fields``, ``LatentStepper`` and
``FullStepper`` add ownership of the weights, the workspace and the status
word.
"""

import ctypes as C

import numpy as np

from . import _native as N
from ._native import NsfError, check, status_string  # noqa: F401

PRECISION = {"fp32": N.NSF_PREC_FP32, "bf16": N.NSF_PREC_BF16}
MODELS = {"neo_hookean": N.NSF_NEO_HOOKEAN, "fixed_corotated": N.NSF_FIXED_COROTATED,
          "von_mises": N.NSF_VON_MISES, "drucker_prager": N.NSF_DRUCKER_PRAGER}
FIELD_NAMES = ("g", "h", "l")
OUT_DIM = (3, 6, 9)


def _torch():
    import torch
    return torch


def _ptr(t):
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _as3(v):
    return tuple(v) if np.ndim(v) else (int(v),) * 3


class Fields:
    """Owns an nsf_fields (device copies of the three field networks).

    weights: mapping 'g'/'h'/'l' (or a sequence of three) -> flat float32 array
    in the layout of nsf.h; width/depth: int or 3 ints; precision 'fp32'|'bf16'.
    """

    def __init__(self, r, width, depth, weights, precision="fp32", out_scale=None,
                 out_shift=None, residual_g=True):
        if isinstance(weights, dict):
            weights = [weights[k] for k in FIELD_NAMES]
        self.r = int(r)
        self.width = _as3(width)
        self.depth = _as3(depth)
        self.precision = precision
        d = N.nsf_fields_desc()
        d.r = self.r
        for f in range(3):
            d.width[f] = self.width[f]
            d.depth[f] = self.depth[f]
            sc = np.ones(OUT_DIM[f]) if out_scale is None else np.asarray(
                out_scale[FIELD_NAMES[f]] if isinstance(out_scale, dict) else out_scale[f])
            sh = np.zeros(OUT_DIM[f]) if out_shift is None else np.asarray(
                out_shift[FIELD_NAMES[f]] if isinstance(out_shift, dict) else out_shift[f])
            for o in range(OUT_DIM[f]):
                d.out_scale[f][o] = float(sc[o])
                d.out_shift[f][o] = float(sh[o])
        d.precision = PRECISION[precision]
        d.residual_g = 1 if residual_g else 0
        self._arrays = [np.ascontiguousarray(w, dtype=np.float32) for w in weights]
        ptrs = (C.c_void_p * 3)(*[a.ctypes.data for a in self._arrays])
        h = C.c_void_p()
        check(N.lib.nsf_create_fields(C.byref(d), C.byref(ptrs), C.byref(h)), "nsf_create_fields")
        self.handle = h
        self.desc = d
        self.residual_g = bool(residual_g)

    @classmethod
    def from_spec(cls, spec):
        """Build from any object with r, width, depth, precision, weights,
        out_scale, out_shift (and optionally residual_g) attributes."""
        return cls(spec.r, spec.width, spec.depth, spec.weights, spec.precision,
                   spec.out_scale, spec.out_shift, getattr(spec, "residual_g", True))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            N.lib.nsf_destroy_fields(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grid_desc(n, dx, gravity=(0.0, 0.0, -9.8), wall_cells=3, blade=None):
    g = N.nsf_grid_desc()
    for i, v in enumerate(_as3(n)):
        g.n[i] = int(v)
    g.dx = float(dx)
    for i in range(3):
        g.gravity[i] = float(gravity[i])
    g.wall_cells = int(wall_cells)
    if blade is not None:
        g.blade_enable = 1
        g.blade_x, g.blade_z0, g.blade_vz = float(blade["x"]), float(blade["z0"]), float(blade["vz"])
    return g


def latent_scene(X, n_S, mass, vol0, grid):
    sc = N.nsf_latent_scene()
    sc.n_N = int(X.shape[1])
    sc.n_S = int(n_S)
    sc.d_X = _ptr(X)
    sc.mass = float(mass)
    sc.vol0 = float(vol0)
    sc.grid = grid
    return sc


def gn_opts(iters=5, damping=1e-6):
    o = N.nsf_gn_opts()
    o.iters = int(iters)
    o.damping = float(damping)
    return o


# ------------------------------------------------ C-named thin wrappers ---
def nsf_eval_fields(fields, X, z, x=None, tau6=None, C9=None, dxdz=None, status=None,
                    stream=None):
    check(N.lib.nsf_eval_fields(fields.handle, _ptr(X), int(X.shape[1]), _ptr(z), _ptr(x),
                                _ptr(tau6), _ptr(C9), _ptr(dxdz), _ptr(status),
                                _stream(stream)), "nsf_eval_fields")


def nsf_latent_workspace_size(fields, scene):
    b = C.c_size_t()
    check(N.lib.nsf_latent_workspace_size(fields.handle, C.byref(scene), C.byref(b)),
          "nsf_latent_workspace_size")
    return b.value


def nsf_latent_step(fields, scene, dt, t0, nsteps, z, z_prev, opts, workspace, status,
                    taps=None, stream=None, flags=0):
    check(N.lib.nsf_latent_step(fields.handle, C.byref(scene), float(dt), float(t0),
                                int(nsteps), int(flags), _ptr(z), _ptr(z_prev), C.byref(opts),
                                _ptr(workspace), workspace.numel(), _ptr(status),
                                C.byref(taps) if taps is not None else None,
                                _stream(stream)), "nsf_latent_step")


def nsf_project_workspace_size(fields, n_S):
    b = C.c_size_t()
    check(N.lib.nsf_project_workspace_size(fields.handle, int(n_S), C.byref(b)),
          "nsf_project_workspace_size")
    return b.value


def nsf_project(fields, X_S, x_target, z, opts, workspace, status, z_iter=None,
                residual=None, stream=None):
    check(N.lib.nsf_project(fields.handle, _ptr(X_S), _ptr(x_target), int(X_S.shape[1]),
                            _ptr(z), C.byref(opts), _ptr(z_iter), _ptr(residual),
                            _ptr(workspace), workspace.numel(), _ptr(status),
                            _stream(stream)), "nsf_project")


def nsf_project_static(fields, X_S, x_target, z, opts, status, z_iter=None, residual=None,
                       stream=None):
    """nsf_project without a workspace: the scratch is a fixed array inside
    the library (for callers that cannot allocate device memory)."""
    check(N.lib.nsf_project_static(fields.handle, _ptr(X_S), _ptr(x_target),
                                   int(X_S.shape[1]), _ptr(z), C.byref(opts), _ptr(z_iter),
                                   _ptr(residual), _ptr(status), _stream(stream)),
          "nsf_project_static")


# ------------------------------------------------------------ training ---
FIELD_INDEX = {"g": N.NSF_FIELD_G, "h": N.NSF_FIELD_H, "l": N.NSF_FIELD_L}


def nsf_field_weight_count(fields, field):
    c = C.c_size_t()
    check(N.lib.nsf_field_weight_count(fields.handle, int(field), C.byref(c)),
          "nsf_field_weight_count")
    return c.value


def nsf_train_workspace_size(fields, field, n):
    b = C.c_size_t()
    check(N.lib.nsf_train_workspace_size(fields.handle, int(field), int(n), C.byref(b)),
          "nsf_train_workspace_size")
    return b.value


def nsf_field_loss_grad(fields, field, X, code, target, z_table, loss, grad_w, grad_z,
                        workspace, status, stream=None):
    check(N.lib.nsf_field_loss_grad(fields.handle, int(field), _ptr(X), _ptr(code), _ptr(target),
                                    int(X.shape[1]), _ptr(z_table), int(z_table.shape[0]),
                                    _ptr(loss), _ptr(grad_w), _ptr(grad_z), _ptr(workspace),
                                    workspace.numel(), _ptr(status), _stream(stream)),
          "nsf_field_loss_grad")


def nsf_adam_step(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    check(N.lib.nsf_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(),
                              int(step), float(lr), float(beta1), float(beta2), float(eps),
                              _stream(stream)), "nsf_adam_step")


def nsf_fields_set_weights(fields, field, weights, stream=None):
    check(N.lib.nsf_fields_set_weights(fields.handle, int(field), _ptr(weights), _stream(stream)),
          "nsf_fields_set_weights")


def _field_loss_function():
    """torch.autograd.Function whose backward is the library's hand-written
    one: forward(weights, z_table, fields, field, X, code, target) -> loss,
    with weights the field's flat float32 master weights (synced into the
    fields object first) and z_table [n_codes, r] float32."""
    torch = _torch()

    class FieldLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, weights, z_table, fields, field, X, code, target):
            dev = X.device
            nsf_fields_set_weights(fields, field, weights)
            ws = _zeros_u8(nsf_train_workspace_size(fields, field, X.shape[1]), dev)
            loss = torch.zeros(1, dtype=torch.float32, device=dev)
            gw = torch.empty_like(weights)
            gz = torch.empty_like(z_table)
            st = torch.zeros(1, dtype=torch.int32, device=dev)
            nsf_field_loss_grad(fields, field, X, code, target, z_table, loss, gw, gz, ws, st)
            ctx.save_for_backward(gw, gz)
            return loss[0]

        @staticmethod
        def backward(ctx, g):
            gw, gz = ctx.saved_tensors
            return g * gw, g * gz, None, None, None, None, None

    return FieldLoss


def field_loss(weights, z_table, fields, field, X, code, target):
    """Training loss of one field (App. D) with the library's gradients."""
    return _field_loss_function().apply(weights, z_table, fields, FIELD_INDEX.get(field, field),
                                        X, code, target)


class FieldTrainer:
    """Adam on one field's FP32 master weights and a table of per-snapshot
    latent codes, every step in the library: loss and gradients
    (nsf_field_loss_grad), Adam (nsf_adam_step), re-pack of the new weights
    into the fields object (nsf_fields_set_weights).  train_codes=False keeps
    the codes fixed (a field fitted on the codes another field learned)."""

    def __init__(self, fields, field, weights, z_table, batch, lr=1e-4, train_codes=True):
        torch = _torch()
        self.train_codes = train_codes
        self.fields, self.field = fields, FIELD_INDEX.get(field, field)
        self.w = weights.detach().clone().float().contiguous()
        self.z = z_table.detach().clone().float().contiguous()
        self.mw, self.vw = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mz, self.vz = torch.zeros_like(self.z), torch.zeros_like(self.z)
        self.gw, self.gz = torch.empty_like(self.w), torch.empty_like(self.z)
        dev = self.w.device
        self.ws = _zeros_u8(nsf_train_workspace_size(fields, self.field, batch), dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.lr, self.t = lr, 0
        nsf_fields_set_weights(fields, self.field, self.w)

    def step(self, X, code, target, stream=None):
        self.t += 1
        nsf_field_loss_grad(self.fields, self.field, X, code, target, self.z, self.loss, self.gw,
                            self.gz if self.train_codes else None, self.ws, self.status, stream)
        nsf_adam_step(self.w, self.gw, self.mw, self.vw, self.t, self.lr, stream=stream)
        if self.train_codes:
            nsf_adam_step(self.z, self.gz, self.mz, self.vz, self.t, self.lr, stream=stream)
        nsf_fields_set_weights(self.fields, self.field, self.w, stream)
        return self.loss


def nsf_integration_set_workspace_size(grid, n_all):
    b = C.c_size_t()
    check(N.lib.nsf_integration_set_workspace_size(C.byref(grid), int(n_all), C.byref(b)),
          "nsf_integration_set_workspace_size")
    return b.value


def nsf_integration_set(fields, grid, X, sample, z, index_out, count_out, workspace, status,
                        X_out=None, stream=None):
    check(N.lib.nsf_integration_set(fields.handle, C.byref(grid), _ptr(X), int(X.shape[1]),
                                    _ptr(sample), int(sample.numel()), _ptr(z), _ptr(index_out),
                                    _ptr(count_out), _ptr(X_out),
                                    int(X_out.shape[1]) if X_out is not None else 0,
                                    _ptr(workspace), workspace.numel(), _ptr(status),
                                    _stream(stream)), "nsf_integration_set")


def integration_set(fields, grid, X, sample, z, stream=None):
    """The integration particles of sample set `sample` (int32 indices into the
    particles X [3, n]) at latent code z: (indices [|N|] int32 with S first,
    X_N [3, |N|], status).  Synchronises to read |N|."""
    torch = _torch()
    n = int(X.shape[1])
    dev = X.device
    ws = _zeros_u8(nsf_integration_set_workspace_size(grid, n), dev)
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    Xo = torch.empty(3, n, dtype=torch.float32, device=dev)
    nsf_integration_set(fields, grid, X, sample, z, idx, cnt, ws, st, X_out=Xo, stream=stream)
    k = int(cnt.item())
    return idx[:k].clone(), Xo[:, :k].contiguous(), int(st.item())


def batch_items(entries):
    """entries: sequence of (Fields, X [3, n_N] tensor, n_S, mass, vol0, grid_desc, dt,
    z [r] float64 tensor, z_prev [r] float64 tensor) -> ctypes array of
    nsf_latent_batch_item."""
    arr = (N.nsf_latent_batch_item * len(entries))()
    for i, (F, X, n_S, mass, vol0, grid, dt, z, zp) in enumerate(entries):
        arr[i].fields = F.handle
        arr[i].scene = latent_scene(X, n_S, mass, vol0, grid)
        arr[i].dt = float(dt)
        arr[i].d_z = _ptr(z)
        arr[i].d_z_prev = _ptr(zp)
    return arr


def nsf_latent_batch_workspace_size(items):
    b = C.c_size_t()
    check(N.lib.nsf_latent_batch_workspace_size(len(items), items, C.byref(b)),
          "nsf_latent_batch_workspace_size")
    return b.value


def batch_tuning(gn_columns=0, gn_split=0.0, p2g_group=0):
    """nsf_batch_tuning (0 keeps a default)."""
    return N.nsf_batch_tuning(int(gn_columns), float(gn_split), int(p2g_group))


def nsf_latent_batch_create(items, opts, workspace, tuning=None):
    h = C.c_void_p()
    if tuning is None:
        check(N.lib.nsf_latent_batch_create(len(items), items, C.byref(opts), _ptr(workspace),
                                            workspace.numel(), C.byref(h)),
              "nsf_latent_batch_create")
    else:
        if isinstance(tuning, dict):
            tuning = batch_tuning(**tuning)
        check(N.lib.nsf_latent_batch_create_tuned(len(items), items, C.byref(opts),
                                                  C.byref(tuning), _ptr(workspace),
                                                  workspace.numel(), C.byref(h)),
              "nsf_latent_batch_create_tuned")
    return h


def nsf_latent_step_batched(batch, t0, nsteps, status, events=None, stream=None, flags=0):
    check(N.lib.nsf_latent_step_batched(batch, float(t0), int(nsteps), int(flags), _ptr(status),
                                        C.byref(events) if events is not None else None,
                                        _stream(stream)), "nsf_latent_step_batched")


def nsf_full_workspace_size(grid, n):
    b = C.c_size_t()
    check(N.lib.nsf_full_workspace_size(C.byref(grid), int(n), C.byref(b)),
          "nsf_full_workspace_size")
    return b.value


def material(model="neo_hookean", E=2e5, nu=0.3, yield_stress=0.0, friction_deg=30.0):
    m = N.nsf_material()
    m.model = MODELS[model]
    m.E, m.nu = float(E), float(nu)
    m.yield_stress, m.friction_deg = float(yield_stress), float(friction_deg)
    return m


def particles(x, v, Cm, F, mass, vol0):
    p = N.nsf_particles()
    p.n = int(x.shape[1])
    p.d_x, p.d_v, p.d_C, p.d_F = _ptr(x), _ptr(v), _ptr(Cm), _ptr(F)
    p.mass, p.vol0 = float(mass), float(vol0)
    return p


def nsf_material_stress(mat, F, tau6, stream=None):
    """Kirchhoff stress tau(F) of material `mat` (F [9, n], tau6 [6, n])."""
    check(N.lib.nsf_material_stress(C.byref(mat), _ptr(F), int(F.shape[1]), _ptr(tau6),
                                    _stream(stream)), "nsf_material_stress")


def nsf_full_step(grid, mat, parts, dt, t0, nsteps, workspace, status, taps=None,
                  stream=None):
    check(N.lib.nsf_full_step(C.byref(grid), C.byref(mat), C.byref(parts), float(dt),
                              float(t0), int(nsteps), _ptr(workspace), workspace.numel(),
                              _ptr(status), C.byref(taps) if taps is not None else None,
                              _stream(stream)), "nsf_full_step")


# ---------------------------------------------------------- ownership ---
def _zeros_u8(nbytes, device):
    torch = _torch()
    return torch.zeros(max(int(nbytes), 1), dtype=torch.uint8, device=device)


class LatentStepper:
    """Workspace + status word for repeated latent steps of one scene."""

    def __init__(self, fields, X, n_S, mass, vol0, grid):
        torch = _torch()
        self.fields = fields
        self.X = X
        self.scene = latent_scene(X, n_S, mass, vol0, grid)
        self.ws = _zeros_u8(nsf_latent_workspace_size(fields, self.scene), X.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=X.device)

    def step(self, z, z_prev, dt, t0=0.0, nsteps=1, iters=5, damping=1e-6, taps=None,
             stream=None, reuse_prev=False):
        nsf_latent_step(self.fields, self.scene, dt, t0, nsteps, z, z_prev,
                        gn_opts(iters, damping), self.ws, self.status, taps, stream,
                        N.NSF_LATENT_REUSE_PREV if reuse_prev else 0)

    def read_status(self):
        return int(self.status.item())


class LatentBatch:
    """Plan, workspace and status word of a batch of latent scenes stepped
    together (nsf_latent_step_batched).  entries as in batch_items; the
    tensors must stay alive with the batch."""

    def __init__(self, entries, iters=5, damping=1e-6, tuning=None):
        torch = _torch()
        self.entries = list(entries)
        self.items = batch_items(self.entries)
        dev = self.entries[0][1].device
        self.ws = _zeros_u8(nsf_latent_batch_workspace_size(self.items), dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.handle = nsf_latent_batch_create(self.items, gn_opts(iters, damping), self.ws,
                                              tuning)

    def step(self, t0=0.0, nsteps=1, events=None, stream=None, reuse_prev=False):
        nsf_latent_step_batched(self.handle, t0, nsteps, self.status, events, stream,
                                N.NSF_LATENT_REUSE_PREV if reuse_prev else 0)

    def read_status(self):
        return int(self.status.item())

    def close(self):
        if getattr(self, "handle", None):
            N.lib.nsf_latent_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FullStepper:
    def __init__(self, grid, mat, x, v, Cm, F, mass, vol0):
        torch = _torch()
        self.grid, self.mat = grid, mat
        self.tensors = (x, v, Cm, F)
        self.parts = particles(x, v, Cm, F, mass, vol0)
        self.ws = _zeros_u8(nsf_full_workspace_size(grid, x.shape[1]), x.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=x.device)

    def step(self, dt, t0=0.0, nsteps=1, taps=None, stream=None):
        nsf_full_step(self.grid, self.mat, self.parts, dt, t0, nsteps, self.ws, self.status,
                      taps, stream)

    def read_status(self):
        return int(self.status.item())


def project(fields, X_S, x_target, z, iters=5, damping=1e-6, z_iter=None, residual=None,
            stream=None):
    """Gauss-Newton network inversion (§5.3); updates z in place, returns status."""
    torch = _torch()
    ws = _zeros_u8(nsf_project_workspace_size(fields, X_S.shape[1]), X_S.device)
    status = torch.zeros(1, dtype=torch.int32, device=X_S.device)
    nsf_project(fields, X_S, x_target, z, gn_opts(iters, damping), ws, status, z_iter,
                residual, stream)
    return status
