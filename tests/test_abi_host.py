"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function ``include/*.h`` declares, sizes workspaces and
rejects invalid arguments before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2112_08264_gb300 import _lib, build

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include")
HEADERS = sorted(os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h"))


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def declared_functions():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"\b(lb1?_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lb_create", "lb_init", "lb_step", "lb_moments", "lb_backward", "lb_stats",
                 "lb_get_state", "lb_set_state", "lb_destroy", "lb_workspace_bytes", "lb_status_str",
                 "lb1_create", "lb1_init", "lb1_step", "lb1_moments", "lb1_stats", "lb1_get_state"):
        assert must in names


def test_single_fluid_workspace_and_rejections(L):
    L.lb1_workspace_bytes.restype = ctypes.c_size_t
    n = 32 ** 3
    wb = L.lb1_workspace_bytes(32, 32, 32, 0)
    assert wb >= 2 * 19 * n * 4
    assert 0 < L.lb1_workspace_bytes(32, 32, 32, 1) < wb
    assert L.lb1_workspace_bytes(2, 32, 32, 0) == 0
    assert L.lb1_workspace_bytes(8, 8, 8, 7) == 0
    h = ctypes.c_void_p()
    # tau <= 1/2 and a missing workspace are rejected before any device call
    assert L.lb1_create(16, 16, 16, ctypes.c_float(0.5), None, 0, None, 0, None, ctypes.byref(h)) == 1
    assert L.lb1_create(16, 16, 16, ctypes.c_float(1.0), None, 0, None, 0, None, ctypes.byref(h)) == 1


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_library_is_sm103a_only():
    # the build emits exactly one -gencode for sm_103a
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_workspace_bytes(L):
    o = _lib.options()
    n = 32 ** 3
    wb = _lib.workspace_bytes(32, 32, 32, o)
    assert wb >= 2 * 38 * n * 4 + 2 * n * 4 + n * 4 + n
    o16 = _lib.options("fp16")
    assert _lib.workspace_bytes(32, 32, 32, o16) < wb
    oc = _lib.options(ckpt_every=10, ckpt_steps_max=50)
    assert _lib.workspace_bytes(32, 32, 32, oc) > wb + 6 * 38 * n * 4
    assert _lib.workspace_bytes(2, 32, 32, o) == 0          # dimension < 3
    assert _lib.workspace_bytes(2048, 1024, 1024, o) == 0   # N >= 2^31
    assert _lib.workspace_bytes(8, 8, 8, _lib.options(prec=7)) == 0
    assert _lib.workspace_bytes(8, 8, 8, _lib.options(ckpt_every=4, ckpt_steps_max=0)) == 0


def test_sphere_options_and_workspace(L):
    """Room for moving spheres: an owner word per site plus per-sphere state;
    spheres need the Shan-Chen model, the fused kernel and no recording."""
    n = 32 ** 3
    wb = _lib.workspace_bytes(32, 32, 32, _lib.options())
    wp = _lib.workspace_bytes(32, 32, 32, _lib.options(max_particles=100))
    assert wp >= wb + n * 4 + 100 * 15 * 8
    assert _lib.workspace_bytes(32, 32, 32, _lib.options(max_particles=-1)) == 0
    assert _lib.workspace_bytes(32, 32, 32, _lib.options(kernel="two_pass", max_particles=4)) == 0
    assert _lib.workspace_bytes(32, 32, 32, _lib.options(ckpt_every=4, ckpt_steps_max=8, max_particles=4)) == 0
    cg = dict(nu=(1 / 6, 1 / 6), sigma=0.01, beta=0.7)
    assert _lib.workspace_bytes(32, 32, 32, _lib.options(model="colour_gradient", cg=cg, max_particles=4)) == 0


@pytest.mark.parametrize("args", [
    dict(nx=2, ny=8, nz=8, tau=1.0, G=0.5),
    dict(nx=8, ny=8, nz=8, tau=0.5, G=0.5),
    dict(nx=8, ny=8, nz=8, tau=float("nan"), G=0.5),
    dict(nx=8, ny=8, nz=8, tau=1.0, G=float("inf")),
])
def test_create_rejects_bad_arguments(L, args):
    o = _lib.options()
    h = ctypes.c_void_p()
    st = L.lb_create(args["nx"], args["ny"], args["nz"], args["tau"], args["G"], None, ctypes.byref(o),
                     ctypes.c_void_p(1 << 20), 1 << 40, None, ctypes.byref(h))
    assert st == _lib.LB_EINVAL
    assert not h.value


def test_create_rejects_short_or_misaligned_workspace(L):
    o = _lib.options()
    need = _lib.workspace_bytes(8, 8, 8, o)
    h = ctypes.c_void_p()
    assert L.lb_create(8, 8, 8, 1.0, 0.5, None, ctypes.byref(o), ctypes.c_void_p(1 << 20), need - 1, None,
                       ctypes.byref(h)) == _lib.LB_ENOMEM
    assert L.lb_create(8, 8, 8, 1.0, 0.5, None, ctypes.byref(o), ctypes.c_void_p((1 << 20) + 4), need, None,
                       ctypes.byref(h)) == _lib.LB_EINVAL
    assert L.lb_create(8, 8, 8, 1.0, 0.5, None, ctypes.byref(o), None, need, None,
                       ctypes.byref(h)) == _lib.LB_EINVAL


def test_null_context_calls_are_rejected(L):
    assert L.lb_step(None, 1) == _lib.LB_EINVAL
    assert L.lb_init(None, None, None, None) == _lib.LB_EINVAL
    assert L.lb_moments(None, None, None, None) == _lib.LB_EINVAL
    assert L.lb_stats(None, None) == _lib.LB_EINVAL
    assert L.lb_backward(None, None, None, None, None, None) == _lib.LB_EINVAL
    assert L.lb_steps_done(None) == -1
    L.lb_destroy(None)


def test_status_strings(L):
    for s in range(7):
        assert L.lb_status_str(s)
    assert L.lb_status_str(99) == b"unknown status"
