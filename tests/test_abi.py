"""CPU checks of the C-ABI boundary: the library builds, loads and exports every
entry point include/ff.h declares; the Python view struct matches the C layout;
argument errors are rejected on the host (before any CUDA call) with the
documented status codes.  No kernel runs here."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1505_00344_gb300 as ff
from paper_1505_00344_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:ff_status|const char\*)\s+(ff_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ff.lib()


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    # and the binding wraps each of them under the same name
    for n in names:
        assert hasattr(ff, n), f"binding lacks {n}"


def test_view_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "ff.h"\nint main(void){\n'
                   'printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(ff_view),'
                   ' offsetof(ff_view, axes), offsetof(ff_view, lo), offsetof(ff_view, hi),'
                   ' offsetof(ff_view, mvp), offsetof(ff_view, width), offsetof(ff_view, height),'
                   ' offsetof(ff_view, group_mask), offsetof(ff_view, accumulate), sizeof(ff_status));'
                   'return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    c_vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    V = ff.ff_view
    py_vals = [ctypes.sizeof(V), V.axes.offset, V.lo.offset, V.hi.offset, V.mvp.offset, V.width.offset,
               V.height.offset, V.group_mask.offset, V.accumulate.offset, ctypes.sizeof(ctypes.c_int)]
    assert c_vals == py_vals


def test_sprite_struct_layout_matches_c(tmp_path):
    src = tmp_path / "sprite.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "ff.h"\nint main(void){\n'
                   'printf("%zu %zu %zu %zu %zu\\n", sizeof(ff_sprite), offsetof(ff_sprite, radius),'
                   ' offsetof(ff_sprite, gain), offsetof(ff_sprite, colour), offsetof(ff_sprite, technique));'
                   'return 0;}\n')
    exe = tmp_path / "sprite"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    c_vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    S = ff.ff_sprite
    assert c_vals == [ctypes.sizeof(S), S.radius.offset, S.gain.offset, S.colour.offset, S.technique.offset]


def _status(fn, *args):
    return fn(*args)


def test_host_side_argument_errors(lib):
    out = ctypes.c_void_p()
    p = (ctypes.c_double * 3)(10.0, 28.0, 8 / 3)
    # unknown system, wrong dim, wrong params count, bad method, flags, capacity: all host checks
    assert lib.ff_create_system(99, 3, p, 3, 0, 0, 16, None, ctypes.byref(out)) == ff.FF_ERR_INVALID_ARG
    assert "rhs_id" in ff.ff_last_error()
    assert lib.ff_create_system(ff.FF_RHS_LORENZ, 2, p, 3, 0, 0, 16, None, ctypes.byref(out)) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_create_system(ff.FF_RHS_LORENZ, 3, p, 2, 0, 0, 16, None, ctypes.byref(out)) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_create_system(ff.FF_RHS_LORENZ, 3, p, 3, 7, 0, 16, None, ctypes.byref(out)) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_create_system(ff.FF_RHS_LORENZ, 3, p, 3, 0, 2, 16, None, ctypes.byref(out)) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_create_system(ff.FF_RHS_LORENZ, 3, p, 3, 0, 0, 0, None, ctypes.byref(out)) == ff.FF_ERR_INVALID_ARG
    nan = (ctypes.c_double * 3)(10.0, float("nan"), 1.0)
    assert lib.ff_create_system(ff.FF_RHS_LORENZ, 3, nan, 3, 0, 0, 16, None, ctypes.byref(out)) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_create_system(ff.FF_RHS_LORENZ, 3, p, 3, 0, 0, 16, None, None) == ff.FF_ERR_INVALID_ARG
    assert out.value is None
    # NULL systems are rejected by every entry point
    assert lib.ff_step(None, 1, 0.1) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_seed_particles(None, 1, None, None, 1, 0, None) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_set_params(None, p, 3) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_project_splat(None, None, None, 1) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_get_state(None, None, 1) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_set_state(None, None, 1) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_stats(None, None, None, None) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_reset(None) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_set_launch(None, 1, 256, 0, 0) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_system_info(None, None, None, None, None) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_set_particle_param(None, 0, 0.0, 1.0) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_get_particle_param(None, None, 1, None) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_destroy_system(None) == ff.FF_OK
    assert lib.ff_backward(None, None, None, None) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_tape_begin(None, 100, 10) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_tape_end(None) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_set_reset(None, None, None, 0.0, 1) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_get_reset_state(None, None, None, 1) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_batch_create(None, 1, None, ctypes.byref(out)) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_batch_step(None, 1, None) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_batch_autotune(None, None, 8) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_batch_describe(None, None, 0) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_batch_destroy(None) == ff.FF_OK
    assert lib.ff_batch_tape_begin(None, 10, 10) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_batch_tape_end(None) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_batch_backward(None, None, None, None) == ff.FF_ERR_INVALID_ARG
    sp = ff.make_sprite(2.0)
    assert lib.ff_project_sprites(None, None, ctypes.byref(sp), None, 1) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_seed_particles_slice(None, 1, 0, 1, None, None, 1, 0, None) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_set_particle_param_slice(None, 0, 0.0, 1.0, 0, 1) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_last_launch(None, None, 0, None, None, None, None, None) == ff.FF_ERR_INVALID_ARG
    # the microbenchmark checks its arguments before touching a device
    rate = ctypes.c_double(0.0)
    assert lib.ff_pipe_rate(ff.FF_PIPE_FFMA, 0, None) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_pipe_rate(-1, 0, ctypes.byref(rate)) == ff.FF_ERR_INVALID_ARG
    assert lib.ff_pipe_rate(ff.FF_PIPE_LOGISTIC + 1, 0, ctypes.byref(rate)) == ff.FF_ERR_INVALID_ARG
    assert "unknown op" in ff.ff_last_error()


def test_binding_raises_with_message(lib):
    with pytest.raises(ff.FFError) as e:
        ff.ff_create_system(ff.FF_RHS_HH3, 15, [0.0] * 3, capacity=10)
    assert e.value.status == ff.FF_ERR_INVALID_ARG
    assert "rhs_id 4" in str(e.value)


def test_product_path_does_not_import_oracle():
    # the CUDA binding and its build must never reach the CPU oracle
    for f in os.listdir(os.path.join(ROOT, "paper_1505_00344_gb300")):
        if f.endswith(".py"):
            text = open(os.path.join(ROOT, "paper_1505_00344_gb300", f)).read()
            assert not re.search(r"^\s*(import|from)\s+oracle", text, flags=re.M), f
    for f in os.listdir(os.path.join(ROOT, "paper_1505_00344_gb300", "csrc")):
        text = open(os.path.join(ROOT, "paper_1505_00344_gb300", "csrc", f)).read()
        assert "ffo_" not in text and "oracle/" not in text, f
