"""Python face of the C ABI: a solver object over a torch-allocated workspace.

PyTorch only provides device memory and the stream; every step of the method
runs in the library's CUDA kernels (``include/lb.h``). Field tensors are
float32, contiguous, on the solver's device, shaped ``(nz, ny, nx)`` (or any
shape with N elements); velocities ``(3, nz, ny, nx)``; populations
``(2, 19, nz, ny, nx)`` in the public velocity order of ``include/lb.h``.
"""
import ctypes

import numpy as np
import torch

from . import _lib


def _ptr(t, n, what, optional=False):
    if t is None:
        if optional:
            return None
        raise ValueError("%s is required" % what)
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % what)
    if t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != n:
        raise ValueError("%s must be a contiguous float32 tensor with %d elements" % (what, n))
    return t.data_ptr()


class _DeviceSpan:
    """Bytes of device memory owned by the library's workspace, exposed through
    the CUDA array interface so that torch can alias them without a copy."""

    def __init__(self, ptr, nbytes, device):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class Solver:
    """Two-component D3Q19 BGK Shan-Chen lattice-Boltzmann solver on one GPU.

    Parameters follow ``lb_create``: grid ``nx, ny, nz``, relaxation time
    ``tau`` (> 1/2), coupling ``G``, optional solid ``mask`` (numpy uint8,
    shape (nz, ny, nx), 1 = solid), storage ``prec`` in {"fp32", "fp16",
    "bf16"}, ``kernel`` in {"fused", "two_pass"}, deviation base ``rho0``
    (0 = mean of the initial densities), ``body_force`` g, and checkpoint
    recording for ``backward`` (``ckpt_every`` K, ``ckpt_steps_max``).
    ``model="colour_gradient"`` selects the paper's colour-gradient model
    with ``cg=dict(nu=(nu_A, nu_B), sigma=..., beta=...)`` (periodic grids;
    ``tau`` and ``G`` unused, ``tau`` must still exceed 1/2).
    """

    def __init__(self, nx, ny, nz, tau, G, mask=None, prec="fp32", kernel="fused", rho0=(0.0, 0.0),
                 body_force=(0.0, 0.0, 0.0), ckpt_every=0, ckpt_steps_max=0, device=None, stream=None,
                 model="shan_chen", cg=None, max_particles=0, slab_halo=0, workspace=None):
        L = _lib.lib()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.shape = (self.nz, self.ny, self.nx)
        self.N = self.nx * self.ny * self.nz
        self.tau, self.G = float(tau), float(G)
        self.prec, self.kernel = prec, kernel
        self.model = model
        self.opt = _lib.options(prec, kernel, rho0, body_force, ckpt_every, ckpt_steps_max, model, cg,
                                max_particles, slab_halo)
        self.n_particles = 0
        nbytes = _lib.workspace_bytes(self.nx, self.ny, self.nz, self.opt)
        if nbytes == 0:
            raise ValueError("invalid grid or options")
        self.device = torch.device(device if device is not None else "cuda")
        if workspace is None:
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        else:   # a caller's uint8 device tensor, 256-byte aligned, at least lb_workspace_bytes long
            if workspace.dtype != torch.uint8 or not workspace.is_cuda or workspace.numel() < nbytes:
                raise ValueError("workspace must be a uint8 CUDA tensor of at least %d bytes" % nbytes)
            self.workspace = workspace
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.mask = None
        mptr = None
        if mask is not None:
            self.mask = np.ascontiguousarray(mask, dtype=np.uint8)
            if self.mask.size != self.N:
                raise ValueError("mask must have nx*ny*nz elements")
            mptr = self.mask.ctypes.data_as(ctypes.c_void_p)
        h = ctypes.c_void_p()
        _lib.check(L.lb_create(self.nx, self.ny, self.nz, self.tau, self.G, mptr, ctypes.byref(self.opt),
                               self.workspace.data_ptr(), nbytes, self.stream.cuda_stream, ctypes.byref(h)),
                   "lb_create")
        self._h = h

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().lb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream):
        self.stream = stream
        _lib.check(_lib.lib().lb_set_stream(self._h, stream.cuda_stream), "lb_set_stream")

    # -- the method ----------------------------------------------------------
    def init(self, rhoA, rhoB, u=None):
        """Equilibrium initial state from device fields rho^A, rho^B (and u)."""
        _lib.check(_lib.lib().lb_init(self._h, _ptr(rhoA, self.N, "rhoA"), _ptr(rhoB, self.N, "rhoB"),
                                      _ptr(u, 3 * self.N, "u", optional=True)), "lb_init")

    def step(self, n=1):
        _lib.check(_lib.lib().lb_step(self._h, int(n)), "lb_step")

    def moments(self, velocity=True):
        """(rho_A, rho_B, u or None) as new device tensors."""
        rA = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        rB = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        u = torch.empty((3,) + self.shape, dtype=torch.float32, device=self.device) if velocity else None
        _lib.check(_lib.lib().lb_moments(self._h, rA.data_ptr(), rB.data_ptr(),
                                         u.data_ptr() if u is not None else None), "lb_moments")
        return rA, rB, u

    def stats(self):
        """FP64 [mass_A, mass_B, Px, Py, Pz] (synchronous)."""
        out = (ctypes.c_double * 5)()
        _lib.check(_lib.lib().lb_stats(self._h, out), "lb_stats")
        return np.array(out[:], dtype=np.float64)

    # -- one rank's slab of a decomposed lattice (slab_halo > 0) -------------
    def step_fluid(self):
        """The step kernel of one step, without the bounce-back pass (``lb_step_fluid``)."""
        _lib.check(_lib.lib().lb_step_fluid(self._h), "lb_step_fluid")

    def step_links(self):
        """The write-side bounce-back pass that completes the step (``lb_step_links``)."""
        _lib.check(_lib.lib().lb_step_links(self._h), "lb_step_links")

    def planes(self):
        """The current state as a (nz, bytes per plane) uint8 device tensor that
        aliases the library's storage (``lb_planes``; valid until the next
        step): plane z is row z, in the library's internal format, for
        copying border planes between ranks."""
        ptr, nbytes = ctypes.c_void_p(), ctypes.c_size_t()
        _lib.check(_lib.lib().lb_planes(self._h, 0, self.nz, ctypes.byref(ptr), ctypes.byref(nbytes)),
                   "lb_planes")
        span = _DeviceSpan(ptr.value, nbytes.value, self.device)
        return torch.as_tensor(span, device=self.device).view(self.nz, nbytes.value // self.nz)

    def stats_planes(self, z0, nplanes):
        """FP64 [mass_A, mass_B, Px, Py, Pz] over planes [z0, z0 + nplanes)."""
        out = (ctypes.c_double * 5)()
        _lib.check(_lib.lib().lb_stats_planes(self._h, int(z0), int(nplanes), out), "lb_stats_planes")
        return np.array(out[:], dtype=np.float64)

    def get_state(self, out=None):
        if out is None:
            out = torch.empty((2, 19) + self.shape, dtype=torch.float32, device=self.device)
        _lib.check(_lib.lib().lb_get_state(self._h, _ptr(out, 38 * self.N, "out")), "lb_get_state")
        return out

    def set_state(self, f):
        _lib.check(_lib.lib().lb_set_state(self._h, _ptr(f, 38 * self.N, "f")), "lb_set_state")

    @property
    def steps_done(self):
        return int(_lib.lib().lb_steps_done(self._h))

    def backward(self, dL_drhoA, dL_drhoB=None, want_rho=True):
        """Gradients of a loss of the final densities of a recorded run:
        (dL/drho_A0, dL/drho_B0, dL/dG)."""
        gA = torch.empty(self.shape, dtype=torch.float32, device=self.device) if want_rho else None
        gB = torch.empty(self.shape, dtype=torch.float32, device=self.device) if want_rho else None
        gG = ctypes.c_double(0.0)
        _lib.check(_lib.lib().lb_backward(
            self._h, _ptr(dL_drhoA, self.N, "dL_drhoA", optional=True),
            _ptr(dL_drhoB, self.N, "dL_drhoB", optional=True),
            gA.data_ptr() if gA is not None else None, gB.data_ptr() if gB is not None else None,
            ctypes.byref(gG)), "lb_backward")
        return gA, gB, gG.value

    def launch_info(self):
        v = [ctypes.c_int() for _ in range(4)]
        _lib.check(_lib.lib().lb_launch_info(self._h, *[ctypes.byref(x) for x in v]), "lb_launch_info")
        return {"launches_per_step": v[0].value, "grid_blocks": v[1].value,
                "block_threads": v[2].value, "z_split": v[3].value}

    def set_particles(self, r, v=None, w=None, radius=5.0, mass=1.0, contact=None, lubrication=None):
        """Place moving rigid spheres (``lb_particles_set``): centres ``r``,
        velocities ``v`` and angular velocities ``w`` as (n, 3) arrays, one
        radius and mass (mass <= 0: held fixed). Before ``init``.
        ``contact`` = (stiffness, range) sets the contact force
        (``lb_particles_contact``), ``lubrication`` = the gap below which the
        lubrication force acts (``lb_particles_lubrication``)."""
        r = np.ascontiguousarray(np.asarray(r, np.float64).reshape(-1, 3))
        n = len(r)
        arr = lambda a: None if a is None else np.ascontiguousarray(np.asarray(a, np.float64).reshape(n, 3))
        v, w = arr(v), arr(w)
        ptr = lambda a: None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _lib.check(_lib.lib().lb_particles_set(self._h, n, ptr(r), ptr(v), ptr(w), float(radius), float(mass)),
                   "lb_particles_set")
        self.n_particles = n
        if contact is not None:
            _lib.check(_lib.lib().lb_particles_contact(self._h, float(contact[0]), float(contact[1])),
                       "lb_particles_contact")
        if lubrication is not None:
            _lib.check(_lib.lib().lb_particles_lubrication(self._h, float(lubrication)), "lb_particles_lubrication")

    def particles(self):
        """The spheres after the last step: dict of (n, 3) arrays r, v, w and
        the last step's force F and torque T (``lb_particles_get``)."""
        n = self.n_particles
        out = {k: np.zeros((n, 3)) for k in ("r", "v", "w", "F", "T")}
        ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _lib.check(_lib.lib().lb_particles_get(self._h, *[ptr(out[k]) for k in ("r", "v", "w", "F", "T")]),
                   "lb_particles_get")
        return out

    def link_info(self):
        """Bounce-back links of the mask: ``listed`` in the per-velocity pass
        (-1: the pass scans every site), ``in_tile`` grouped by step-kernel
        tile, ``in_kernel`` whether the step kernel copies those itself."""
        a, b, k = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
        _lib.check(_lib.lib().lb_link_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(k)),
                   "lb_link_info")
        return {"listed": a.value, "in_tile": b.value, "in_kernel": bool(k.value)}


def create(nx, ny, nz, tau, G, mask=None, **kw):
    """``lb_create(nx, ny, nz, tau, G, mask)`` in Python form."""
    return Solver(nx, ny, nz, tau, G, mask=mask, **kw)


def run_host(rhoA, rhoB, steps, tau, G, mask=None, u=None, solver=None, **kw):
    """End-to-end run from host arrays: copy the initial fields to the device
    (from pinned memory), initialise, take ``steps`` steps, and copy rho_A,
    rho_B and u back. Returns numpy arrays (rho_A, rho_B, u) and the solver."""
    rhoA = np.ascontiguousarray(rhoA, dtype=np.float32)
    nz, ny, nx = rhoA.shape
    s = solver if solver is not None else Solver(nx, ny, nz, tau, G, mask=mask, **kw)
    dev = s.device
    hA = torch.from_numpy(rhoA).pin_memory()
    hB = torch.from_numpy(np.ascontiguousarray(rhoB, dtype=np.float32)).pin_memory()
    with torch.cuda.stream(s.stream):
        dA = hA.to(dev, non_blocking=True)
        dB = hB.to(dev, non_blocking=True)
        du = None
        if u is not None:
            du = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).pin_memory().to(dev, non_blocking=True)
    s.init(dA, dB, du)
    s.step(steps)
    rA, rB, uu = s.moments()
    with torch.cuda.stream(s.stream):
        out = [t.to("cpu", non_blocking=True) for t in (rA, rB, uu)]
    s.stream.synchronize()
    return tuple(t.numpy() for t in out), s
