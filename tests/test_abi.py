"""The C-ABI library loads without a GPU, exports every declared symbol, and
rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    return sorted(set(re.findall(r"VLBM_API[^;(]*?\b(vlbm_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def V():
    from paper_2411_15001_gb300 import build

    build.build()
    from paper_2411_15001_gb300 import vlbm

    return vlbm


def test_header_declares_the_api():
    names = _declared()
    for n in ("vlbm_init", "vlbm_step", "vlbm_moments", "vlbm_set_conserved", "vlbm_step_to",
              "vlbm_monitors", "vlbm_save", "vlbm_load", "vlbm_destroy", "vlbm_strerror",
              "vlbm_test_theta_faces", "vlbm_test_wait_probe"):
        assert n in names


def test_test_hooks_reject_bad_arguments(V):
    assert V.vlbm_test_theta_faces(-1, 1.0, 0.5, 0.0, None, None, None, None) == V.E_INVAL
    assert V.vlbm_test_theta_faces(0, 1.0, 0.5, 0.0, None, None, None, None) == V.OK
    assert V.vlbm_test_theta_faces(4, 1.0, 0.5, 0.0, None, None, None, None) == V.E_INVAL
    assert V.vlbm_test_theta_faces(4, 0.0, 0.5, 0.0, 8, 8, 8, None) == V.E_INVAL
    assert V.vlbm_test_theta_faces(4, 1.0, 0.4, 0.0, 8, 8, 8, None) == V.E_INVAL
    assert V.vlbm_test_wait_probe(None, 1000) == V.E_INVAL


def test_exports_every_declared_symbol(V):
    lib = ctypes.CDLL(V.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_codes(V):
    assert V.vlbm_strerror(V.OK) == "ok"
    for code in (V.E_INVAL, V.E_CUDA, V.E_POSITIVITY, V.E_NONFINITE, V.E_TIMEOUT,
                 V.E_UNSUPPORTED, V.E_NOMEM):
        assert V.vlbm_strerror(code) not in ("ok", "unknown error code")
    assert V.vlbm_strerror(12345) == "unknown error code"


def _grid(V, nx=16, ny=12, bc=(0, 0, 0, 0), dx=0.1):
    return V.vlbm_grid(nx, ny, dx, (ctypes.c_int32 * 4)(*bc))


def test_workspace_bytes(V):
    g = _grid(V)
    b32 = V.vlbm_workspace_bytes(g, V.FP32)
    b64 = V.vlbm_workspace_bytes(g, V.FP64)
    assert b32 >= 2 * 20 * (16 + 4) * (12 + 4) * 4 and b64 > b32
    assert V.vlbm_workspace_bytes(_grid(V, nx=3), V.FP32) == 0
    assert V.vlbm_workspace_bytes(_grid(V, bc=(0, 1, 0, 0)), V.FP32) == 0   # unpaired periodic side
    assert V.vlbm_workspace_bytes(_grid(V, dx=0.0), V.FP32) == 0
    assert V.vlbm_workspace_bytes(g, 7) == 0


@pytest.mark.parametrize("case", ["grid", "gamma", "limiter", "precision", "alpha", "workspace", "small",
                                  "dirichlet_without_field", "split_near_corner", "periodic_split",
                                  "types_differ_without_split", "field_state_outside_G", "field_planes"])
def test_init_rejects_bad_arguments(V, case):
    g = _grid(V)
    gamma, lim, prec = 1.4, V.LIM_PP, V.FP32
    opts = V.vlbm_opts(0.5, 1e-16, 0, 0)
    ws, nbytes = 256 * 1024, 10 ** 9
    if case == "grid":
        g = _grid(V, nx=2)
    elif case == "gamma":
        gamma = 1.0
    elif case == "limiter":
        lim = 9
    elif case == "precision":
        prec = 5
    elif case == "alpha":
        opts = V.vlbm_opts(0.3, 1e-16, 0, 0)
    elif case == "workspace":
        ws = 256 * 1024 + 8        # misaligned
    elif case == "small":
        nbytes = 100
    elif case == "dirichlet_without_field":
        g = _grid(V, bc=(3, 1, 1, 1))
    else:
        g = _grid(V, bc=(3, 1, 2, 1))
        good = ((1.0, 0.0, 0.0, 2.5), (0.5, 0.1, 0.0, 1.0), ((1.0, 0.0, 0.3, 0.0),))
        kw = dict(bc_hi=(3, 1, 3, 1), split=(0, 0, 5, 0), field=good)
        if case == "split_near_corner":
            kw["split"] = (0, 0, 1, 0)
        elif case == "periodic_split":
            g = _grid(V, bc=(0, 0, 2, 1))
            kw = dict(bc_hi=(0, 1, 2, 1), split=(0, 4, 0, 0))
        elif case == "types_differ_without_split":
            kw["split"] = (0, 0, 0, 0)
        elif case == "field_state_outside_G":
            kw["field"] = ((1.0, 3.0, 0.0, 2.5), good[1], good[2])   # E < |m|^2 / (2 rho)
        b = V.make_boundary((3, 1, 2, 1), **kw)
        if case == "field_planes":
            b.field.nplanes = 3
        opts = V._opts(0.5, 1e-16, 0, 0, b)
    rc, s = V.vlbm_init(g, gamma, 0.0, lim, prec, opts, ws, nbytes, None)
    assert rc in (V.E_INVAL, V.E_NOMEM) and not s.value
    assert V.vlbm_last_error_detail()


def test_init_without_device_memory_fails_cleanly(V):
    """A host address is never accepted as the workspace (E_INVAL with a device,
    E_CUDA without one)."""
    buf = ctypes.create_string_buffer(1 << 20)
    addr = (ctypes.addressof(buf) + 255) // 256 * 256
    g = _grid(V)
    rc, s = V.vlbm_init(g, 1.4, 0.0, V.LIM_PP, V.FP32, None, addr, 1 << 19, None)
    assert rc in (V.E_INVAL, V.E_CUDA) and not s.value


def test_calls_on_null_state(V):
    assert V.vlbm_step(None, 1) == V.E_INVAL
    assert V.vlbm_moments(None, None, None, None) == V.E_INVAL
    assert V.vlbm_checkpoint_bytes(None) == 0
    V.vlbm_destroy(None)


def test_struct_layouts_match_the_header(V, tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's sizes and offsets."""
    import subprocess
    src = tmp_path / "layout.c"
    src.write_text("""#include <stddef.h>
#include <stdio.h>
#include "vlbm.h"
int main(void) {
    printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(vlbm_opts), offsetof(vlbm_opts, boundary),
           sizeof(vlbm_boundary), offsetof(vlbm_boundary, field), sizeof(vlbm_field),
           offsetof(vlbm_field, nplanes), offsetof(vlbm_field, c1), sizeof(vlbm_grid));
    return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(V.vlbm_opts), V.vlbm_opts.boundary.offset, ctypes.sizeof(V.vlbm_boundary),
            V.vlbm_boundary.field.offset, ctypes.sizeof(V.vlbm_field), V.vlbm_field.nplanes.offset,
            V.vlbm_field.c1.offset, ctypes.sizeof(V.vlbm_grid)]
    assert got == want
