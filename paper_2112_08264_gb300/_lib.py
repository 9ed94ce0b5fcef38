"""ctypes binding of the C ABI in ``include/lb.h`` (argument marshalling only).

The shared library must have been built (``build.build()``); there is no
fallback of any kind: loading fails with ``ImportError`` when it is missing.
"""
import ctypes
import os

from . import build as _build

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_ENONFINITE, LB_ESTATE, LB_ETIMEOUT = range(7)
PRECISIONS = {"fp32": 0, "fp16": 1, "bf16": 2}
KERNELS = {"fused": 0, "two_pass": 1, "fused_reg": 2}
MODELS = {"shan_chen": 0, "colour_gradient": 1}


class LbOptions(ctypes.Structure):
    _fields_ = [
        ("prec", ctypes.c_int),
        ("kernel", ctypes.c_int),
        ("rho0_A", ctypes.c_double),
        ("rho0_B", ctypes.c_double),
        ("body_force", ctypes.c_double * 3),
        ("ckpt_every", ctypes.c_int),
        ("ckpt_steps_max", ctypes.c_int),
        ("model", ctypes.c_int),
        ("cg_nu_A", ctypes.c_double),
        ("cg_nu_B", ctypes.c_double),
        ("cg_sigma", ctypes.c_double),
        ("cg_beta", ctypes.c_double),
        ("max_particles", ctypes.c_int),
        ("slab_halo", ctypes.c_int),
    ]


class LbError(RuntimeError):
    def __init__(self, status, what, detail=""):
        self.status = status
        msg = "%s failed: %s" % (what, lib().lb_status_str(status).decode())
        if detail:
            msg += " (%s)" % detail
        super().__init__(msg)


_lib = None

_VP = ctypes.c_void_p
_FP = ctypes.c_void_p   # device float* passed as an integer address


def lib():
    """Load the CUDA library (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(
            "liblbgb.so is not built (%s); run paper_2112_08264_gb300.build.build() "
            "(or __graft_entry__.build()) first" % path)
    L = ctypes.CDLL(path)
    L.lb_default_options.argtypes = [ctypes.POINTER(LbOptions)]
    L.lb_default_options.restype = None
    L.lb_workspace_bytes.argtypes = [ctypes.c_int] * 3 + [ctypes.POINTER(LbOptions)]
    L.lb_workspace_bytes.restype = ctypes.c_size_t
    L.lb_create.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_float, ctypes.c_float, _VP,
                                                   ctypes.POINTER(LbOptions), _VP, ctypes.c_size_t, _VP,
                                                   ctypes.POINTER(_VP)])
    L.lb_set_stream.argtypes = [_VP, _VP]
    L.lb_init.argtypes = [_VP, _FP, _FP, _FP]
    L.lb_step.argtypes = [_VP, ctypes.c_int]
    L.lb_moments.argtypes = [_VP, _FP, _FP, _FP]
    L.lb_stats.argtypes = [_VP, ctypes.POINTER(ctypes.c_double)]
    L.lb_get_state.argtypes = [_VP, _FP]
    L.lb_set_state.argtypes = [_VP, _FP]
    L.lb_steps_done.argtypes = [_VP]
    L.lb_steps_done.restype = ctypes.c_longlong
    L.lb_backward.argtypes = [_VP, _FP, _FP, _FP, _FP, ctypes.POINTER(ctypes.c_double)]
    L.lb_launch_info.argtypes = [_VP] + [ctypes.POINTER(ctypes.c_int)] * 4
    _DP = ctypes.POINTER(ctypes.c_double)
    L.lb_particles_set.argtypes = [_VP, ctypes.c_int, _DP, _DP, _DP, ctypes.c_double, ctypes.c_double]
    L.lb_particles_get.argtypes = [_VP, _DP, _DP, _DP, _DP, _DP]
    L.lb_particles_contact.argtypes = [_VP, ctypes.c_double, ctypes.c_double]
    L.lb_particles_lubrication.argtypes = [_VP, ctypes.c_double]
    L.lb_link_info.argtypes = [_VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                               ctypes.POINTER(ctypes.c_int)]
    L.lb_moments_noalloc.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_float, ctypes.POINTER(ctypes.c_double),
                                                             _FP, _VP, _FP, _FP, _FP, _VP])
    L.lb_moments_noalloc.restype = ctypes.c_int
    L.lb_step_fluid.argtypes = [_VP]
    L.lb_step_links.argtypes = [_VP]
    L.lb_planes.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_size_t)]
    L.lb_stats_planes.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.lb_destroy.argtypes = [_VP]
    L.lb_destroy.restype = None
    L.lb_status_str.argtypes = [ctypes.c_int]
    L.lb_status_str.restype = ctypes.c_char_p
    L.lb_last_error.argtypes = []
    L.lb_last_error.restype = ctypes.c_char_p
    for name in ("lb_create", "lb_set_stream", "lb_init", "lb_step", "lb_moments", "lb_stats",
                 "lb_get_state", "lb_set_state", "lb_backward", "lb_launch_info", "lb_link_info",
                 "lb_particles_set", "lb_particles_get", "lb_particles_contact",
                 "lb_particles_lubrication", "lb_step_fluid", "lb_step_links", "lb_planes",
                 "lb_stats_planes"):
        getattr(L, name).restype = ctypes.c_int
    # one-component BGK (include/lb1.h)
    L.lb1_workspace_bytes.argtypes = [ctypes.c_int] * 4
    L.lb1_workspace_bytes.restype = ctypes.c_size_t
    L.lb1_create.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_float, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                                   _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)])
    L.lb1_init.argtypes = [_VP, _FP, _FP]
    L.lb1_step.argtypes = [_VP, ctypes.c_int]
    L.lb1_moments.argtypes = [_VP, _FP, _FP]
    L.lb1_stats.argtypes = [_VP, ctypes.POINTER(ctypes.c_double)]
    L.lb1_get_state.argtypes = [_VP, _FP]
    L.lb1_launch_info.argtypes = [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.lb1_destroy.argtypes = [_VP]
    L.lb1_destroy.restype = None
    for name in ("lb1_create", "lb1_init", "lb1_step", "lb1_moments", "lb1_stats", "lb1_get_state",
                 "lb1_launch_info"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def check(status, what):
    if status != LB_OK:
        detail = lib().lb_last_error().decode() if status == LB_ECUDA else ""
        raise LbError(status, what, detail)


def options(prec="fp32", kernel="fused", rho0=(0.0, 0.0), body_force=(0.0, 0.0, 0.0),
            ckpt_every=0, ckpt_steps_max=0, model="shan_chen", cg=None, max_particles=0, slab_halo=0):
    """lb_options; ``cg`` = dict(nu=(nu_A, nu_B), sigma=, beta=) for the
    colour-gradient model."""
    o = LbOptions()
    lib().lb_default_options(ctypes.byref(o))
    o.model = MODELS[model] if isinstance(model, str) else int(model)
    if cg is not None:
        o.cg_nu_A, o.cg_nu_B = float(cg["nu"][0]), float(cg["nu"][1])
        o.cg_sigma = float(cg.get("sigma", 0.0))
        o.cg_beta = float(cg.get("beta", 0.0))
    o.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    o.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    o.rho0_A, o.rho0_B = float(rho0[0]), float(rho0[1])
    for a in range(3):
        o.body_force[a] = float(body_force[a])
    o.ckpt_every = int(ckpt_every)
    o.ckpt_steps_max = int(ckpt_steps_max)
    o.max_particles = int(max_particles)
    o.slab_halo = int(slab_halo)
    return o


def workspace_bytes(nx, ny, nz, opt=None):
    return int(lib().lb_workspace_bytes(nx, ny, nz, ctypes.byref(opt) if opt is not None else None))
