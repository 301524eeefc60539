"""ctypes binding of libnsf's C ABI (include/nsf.h).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  The structures below mirror the header field for field.
Importing this module loads ``_build/libnsf.so`` and raises if it is missing:
there is no fallback implementation.
"""

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libnsf.so")

NSF_OK = 0
NSF_ERR_INVALID_ARG = -1
NSF_ERR_CUDA = -2
NSF_ERR_OUT_OF_GRID = -3
NSF_ERR_NONFINITE = -4
NSF_ERR_SINGULAR = -5
NSF_ERR_ITER_CAP = -6
NSF_ERR_UNSUPPORTED = -7
NSF_ERR_NO_MEMORY = -8
NSF_ERR_WORKSPACE = -9

NSF_FIELD_G, NSF_FIELD_H, NSF_FIELD_L = 0, 1, 2
NSF_PREC_FP32, NSF_PREC_BF16 = 0, 1
NSF_NEO_HOOKEAN, NSF_FIXED_COROTATED, NSF_VON_MISES, NSF_DRUCKER_PRAGER = 0, 1, 2, 3
NSF_MAX_R, NSF_MAX_WIDTH, NSF_MAX_DEPTH = 16, 256, 8
NSF_STAGE_NAMES = ("inference", "mpm", "gauss_newton")
NSF_LATENT_STAGES = 3
NSF_LATENT_REUSE_PREV = 1
NSF_PROJECT_STATIC_MAX_S = 2048
NSF_PROJECT_STATIC_BYTES = 1 << 20
NSF_MAX_BATCH = 1024


class nsf_fields_desc(C.Structure):
    _fields_ = [("r", C.c_int), ("width", C.c_int * 3), ("depth", C.c_int * 3),
                ("precision", C.c_int), ("residual_g", C.c_int),
                ("out_scale", (C.c_float * 9) * 3), ("out_shift", (C.c_float * 9) * 3)]


class nsf_grid_desc(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("dx", C.c_float), ("gravity", C.c_float * 3),
                ("wall_cells", C.c_int), ("blade_enable", C.c_int),
                ("blade_x", C.c_float), ("blade_z0", C.c_float), ("blade_vz", C.c_float)]


class nsf_latent_scene(C.Structure):
    _fields_ = [("n_N", C.c_int), ("n_S", C.c_int), ("d_X", C.c_void_p),
                ("mass", C.c_float), ("vol0", C.c_float), ("grid", nsf_grid_desc)]


class nsf_gn_opts(C.Structure):
    _fields_ = [("iters", C.c_int), ("damping", C.c_double)]


class nsf_latent_taps(C.Structure):
    _fields_ = [("u_n", C.c_void_p), ("u_prev", C.c_void_p), ("tau6", C.c_void_p),
                ("C9", C.c_void_p), ("grid_mp", C.c_void_p), ("grid_v", C.c_void_p),
                ("u_next_S", C.c_void_p), ("z_iter", C.c_void_p),
                ("ev_begin", C.c_void_p * NSF_LATENT_STAGES),
                ("ev_end", C.c_void_p * NSF_LATENT_STAGES)]


class nsf_latent_batch_item(C.Structure):
    _fields_ = [("fields", C.c_void_p), ("scene", nsf_latent_scene), ("dt", C.c_double),
                ("d_z", C.c_void_p), ("d_z_prev", C.c_void_p)]


class nsf_batch_tuning(C.Structure):
    _fields_ = [("gn_columns", C.c_int), ("gn_split", C.c_double), ("p2g_group", C.c_int)]


class nsf_batch_events(C.Structure):
    _fields_ = [("ev_begin", C.c_void_p * NSF_LATENT_STAGES),
                ("ev_end", C.c_void_p * NSF_LATENT_STAGES)]


class nsf_material(C.Structure):
    _fields_ = [("model", C.c_int), ("E", C.c_float), ("nu", C.c_float),
                ("yield_stress", C.c_float), ("friction_deg", C.c_float)]


class nsf_particles(C.Structure):
    _fields_ = [("n", C.c_int), ("d_x", C.c_void_p), ("d_v", C.c_void_p),
                ("d_C", C.c_void_p), ("d_F", C.c_void_p), ("mass", C.c_float),
                ("vol0", C.c_float)]


class nsf_full_taps(C.Structure):
    _fields_ = [("grid_mp", C.c_void_p), ("grid_v", C.c_void_p)]


_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_S = C.c_size_t
_ST = C.c_int

# (name, restype, argtypes) of every exported symbol of nsf.h
SIGNATURES = [
    ("nsf_create_fields", _ST, [C.POINTER(nsf_fields_desc), C.POINTER(C.c_void_p * 3), C.POINTER(_P)]),
    ("nsf_destroy_fields", None, [_P]),
    ("nsf_fields_get_desc", _ST, [_P, C.POINTER(nsf_fields_desc)]),
    ("nsf_eval_fields", _ST, [_P, _P, _I, _P, _P, _P, _P, _P, _P, _P]),
    ("nsf_latent_workspace_size", _ST, [_P, C.POINTER(nsf_latent_scene), C.POINTER(_S)]),
    ("nsf_latent_step", _ST, [_P, C.POINTER(nsf_latent_scene), _D, _D, _I, C.c_uint, _P, _P,
                              C.POINTER(nsf_gn_opts), _P, _S, _P, C.POINTER(nsf_latent_taps), _P]),
    ("nsf_project_workspace_size", _ST, [_P, _I, C.POINTER(_S)]),
    ("nsf_project", _ST, [_P, _P, _P, _I, _P, C.POINTER(nsf_gn_opts), _P, _P, _P, _S, _P, _P]),
    ("nsf_project_static", _ST, [_P, _P, _P, _I, _P, C.POINTER(nsf_gn_opts), _P, _P, _P, _P]),
    ("nsf_field_weight_count", _ST, [_P, _I, C.POINTER(_S)]),
    ("nsf_train_workspace_size", _ST, [_P, _I, _I, C.POINTER(_S)]),
    ("nsf_field_loss_grad", _ST, [_P, _I, _P, _P, _P, _I, _P, _I, _P, _P, _P, _P, _S, _P, _P]),
    ("nsf_adam_step", _ST, [_P, _P, _P, _P, _S, _I, C.c_float, C.c_float, C.c_float, C.c_float, _P]),
    ("nsf_fields_set_weights", _ST, [_P, _I, _P, _P]),
    ("nsf_integration_set_workspace_size", _ST, [C.POINTER(nsf_grid_desc), _I, C.POINTER(_S)]),
    ("nsf_integration_set", _ST, [_P, C.POINTER(nsf_grid_desc), _P, _I, _P, _I, _P, _P, _P, _P,
                                  _I, _P, _S, _P, _P]),
    ("nsf_latent_batch_workspace_size", _ST, [_I, C.POINTER(nsf_latent_batch_item), C.POINTER(_S)]),
    ("nsf_latent_batch_create", _ST, [_I, C.POINTER(nsf_latent_batch_item), C.POINTER(nsf_gn_opts),
                                      _P, _S, C.POINTER(_P)]),
    ("nsf_latent_batch_create_tuned", _ST, [_I, C.POINTER(nsf_latent_batch_item),
                                            C.POINTER(nsf_gn_opts), C.POINTER(nsf_batch_tuning),
                                            _P, _S, C.POINTER(_P)]),
    ("nsf_latent_batch_destroy", None, [_P]),
    ("nsf_latent_step_batched", _ST, [_P, _D, _I, C.c_uint, _P, C.POINTER(nsf_batch_events), _P]),
    ("nsf_full_workspace_size", _ST, [C.POINTER(nsf_grid_desc), _I, C.POINTER(_S)]),
    ("nsf_full_step", _ST, [C.POINTER(nsf_grid_desc), C.POINTER(nsf_material),
                            C.POINTER(nsf_particles), _D, _D, _I, _P, _S, _P,
                            C.POINTER(nsf_full_taps), _P]),
    ("nsf_material_stress", _ST, [C.POINTER(nsf_material), _P, _I, _P, _P]),
    ("nsf_status_string", C.c_char_p, [_I]),
    ("nsf_version", _I, []),
]


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"libnsf.so not found at {LIB_PATH}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class NsfError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = lib.nsf_status_string(status).decode()
        super().__init__(f"{where}: {msg} ({status})" if where else f"{msg} ({status})")


def check(status, where=""):
    if status != NSF_OK:
        raise NsfError(status, where)
    return status


def status_string(status):
    return lib.nsf_status_string(int(status)).decode()
