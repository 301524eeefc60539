"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
symbol include/nsf.h declares, its ctypes mirrors match the C layouts, and the
host-side argument validation answers without touching a GPU."""

import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nsf.h")


@pytest.fixture(scope="module")
def native():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2310_17790_gb300 import _native
    return _native


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"^[A-Za-z_][\w \*]*?\b(nsf_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for must in ("nsf_create_fields", "nsf_destroy_fields", "nsf_full_step",
                 "nsf_latent_step", "nsf_project", "nsf_eval_fields", "nsf_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(native):
    names = declared_functions()
    bound = {n for n, _, _ in native.SIGNATURES}
    assert names == bound, names ^ bound
    for n in names:
        assert hasattr(native.lib, n), n


def test_ctypes_structs_match_c_layout(native, tmp_path):
    structs = ["nsf_fields_desc", "nsf_grid_desc", "nsf_latent_scene", "nsf_gn_opts",
               "nsf_latent_taps", "nsf_material", "nsf_particles", "nsf_full_taps",
               "nsf_latent_batch_item", "nsf_batch_events", "nsf_batch_tuning"]
    prog = ['#include <stdio.h>', '#include <stddef.h>', '#include "nsf.h"', "int main(void){"]
    for s in structs:
        prog.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in getattr(native, s)._fields_:
            prog.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    prog.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(l.rsplit(" ", 1) for l in out.strip().splitlines())
    for s in structs:
        cls = getattr(native, s)
        assert int(got[s]) == C.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)


def test_status_strings_and_version(native):
    assert native.lib.nsf_status_string(0) == b"ok"
    assert b"grid" in native.lib.nsf_status_string(native.NSF_ERR_OUT_OF_GRID)
    assert native.lib.nsf_status_string(12345) == b"unknown status"
    assert native.lib.nsf_version() >= 100


def test_host_side_validation_without_gpu(native):
    lib = native.lib
    g = native.nsf_grid_desc()
    for i in range(3):
        g.n[i] = 32
    g.dx = 1.0 / 32
    size = C.c_size_t()
    assert lib.nsf_full_workspace_size(C.byref(g), 1000, C.byref(size)) == 0
    assert size.value >= 32 ** 3 * 32          # two float4 grids
    bad = native.nsf_grid_desc()
    bad.n[0], bad.n[1], bad.n[2] = 30, 32, 32  # not a multiple of 4
    bad.dx = 0.1
    assert lib.nsf_full_workspace_size(C.byref(bad), 1000, C.byref(size)) == native.NSF_ERR_INVALID_ARG
    assert lib.nsf_full_workspace_size(C.byref(g), 0, C.byref(size)) == native.NSF_ERR_INVALID_ARG
    # an invalid descriptor is rejected before any device allocation
    d = native.nsf_fields_desc()
    d.r = 0
    h = C.c_void_p()
    ptrs = (C.c_void_p * 3)()
    assert lib.nsf_create_fields(C.byref(d), C.byref(ptrs), C.byref(h)) == native.NSF_ERR_INVALID_ARG
    d.r = 17
    assert lib.nsf_create_fields(C.byref(d), C.byref(ptrs), C.byref(h)) == native.NSF_ERR_INVALID_ARG
    mat = native.nsf_material()
    parts = native.nsf_particles()
    assert lib.nsf_full_step(C.byref(g), C.byref(mat), C.byref(parts), 1e-4, 0.0, 1, None, 0,
                             None, None, None) == native.NSF_ERR_INVALID_ARG


def test_batch_validation_without_gpu(native):
    lib = native.lib
    size = C.c_size_t()
    items = (native.nsf_latent_batch_item * 2)()
    # no fields: rejected
    assert lib.nsf_latent_batch_workspace_size(2, items, C.byref(size)) == native.NSF_ERR_INVALID_ARG
    assert lib.nsf_latent_batch_workspace_size(0, items, C.byref(size)) == native.NSF_ERR_INVALID_ARG
    assert lib.nsf_latent_batch_workspace_size(native.NSF_MAX_BATCH + 1, items,
                                               C.byref(size)) == native.NSF_ERR_INVALID_ARG
    opts = native.nsf_gn_opts()
    opts.iters, opts.damping = 5, 1e-6
    h = C.c_void_p()
    assert lib.nsf_latent_batch_create(2, items, C.byref(opts), None, 0,
                                       C.byref(h)) == native.NSF_ERR_INVALID_ARG
    assert lib.nsf_latent_step_batched(None, 0.0, 1, 0, None, None, None) == native.NSF_ERR_INVALID_ARG


def test_integration_set_validation_without_gpu(native):
    lib = native.lib
    g = native.nsf_grid_desc()
    for i in range(3):
        g.n[i] = 32
    g.dx = 1.0 / 32
    size = C.c_size_t()
    assert lib.nsf_integration_set_workspace_size(C.byref(g), 1000, C.byref(size)) == 0
    assert size.value >= 32 ** 3 // 8 + 1000 * 12      # node bitmap + positions
    assert lib.nsf_integration_set_workspace_size(C.byref(g), 0, C.byref(size)) == native.NSF_ERR_INVALID_ARG
    assert lib.nsf_integration_set(None, C.byref(g), None, 10, None, 1, None, None, None, None, 0,
                                   None, 0, None, None) == native.NSF_ERR_INVALID_ARG
