"""Python face of the one-component BGK step (``include/lb1.h``): the paper's
single-fluid case. PyTorch provides device memory and the stream; the step
runs in the library's kernels. Fields are float32 CUDA tensors of N elements
(density) or 3N (velocity, SoA); populations ``(19, nz, ny, nx)`` in the
public velocity order.
"""
import ctypes

import torch

from . import _lib
from .solver import _ptr


class SingleFluid:
    """D3Q19 BGK on an nx x ny x nz periodic grid (tau > 1/2, body force g
    as a velocity shift), storage ``prec`` in {"fp32", "fp16", "bf16"}."""

    def __init__(self, nx, ny, nz, tau, body_force=(0.0, 0.0, 0.0), prec="fp32", device=None, stream=None):
        L = _lib.lib()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.shape = (self.nz, self.ny, self.nx)
        self.N = self.nx * self.ny * self.nz
        p = _lib.PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        nbytes = int(L.lb1_workspace_bytes(self.nx, self.ny, self.nz, p))
        if nbytes == 0:
            raise ValueError("invalid grid or precision")
        self.device = torch.device(device if device is not None else "cuda")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        g = (ctypes.c_double * 3)(*[float(v) for v in body_force])
        h = ctypes.c_void_p()
        _lib.check(L.lb1_create(self.nx, self.ny, self.nz, float(tau), g, p, self.workspace.data_ptr(), nbytes,
                                self.stream.cuda_stream, ctypes.byref(h)), "lb1_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().lb1_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho, u=None):
        _lib.check(_lib.lib().lb1_init(self._h, _ptr(rho, self.N, "rho"), _ptr(u, 3 * self.N, "u", True)),
                   "lb1_init")

    def step(self, n=1):
        _lib.check(_lib.lib().lb1_step(self._h, int(n)), "lb1_step")

    def moments(self):
        rho = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        u = torch.empty((3,) + self.shape, dtype=torch.float32, device=self.device)
        _lib.check(_lib.lib().lb1_moments(self._h, rho.data_ptr(), u.data_ptr()), "lb1_moments")
        return rho, u

    def stats(self):
        out = (ctypes.c_double * 4)()
        _lib.check(_lib.lib().lb1_stats(self._h, out), "lb1_stats")
        return tuple(out)

    def get_state(self):
        f = torch.empty((19,) + self.shape, dtype=torch.float32, device=self.device)
        _lib.check(_lib.lib().lb1_get_state(self._h, f.data_ptr()), "lb1_get_state")
        return f

    def launch_info(self):
        b, t = ctypes.c_int(), ctypes.c_int()
        _lib.check(_lib.lib().lb1_launch_info(self._h, ctypes.byref(b), ctypes.byref(t)), "lb1_launch_info")
        return {"launches_per_step": 1, "grid_blocks": b.value, "block_threads": t.value}
