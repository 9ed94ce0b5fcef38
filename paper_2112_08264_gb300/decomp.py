"""Z-slab domain decomposition of one lattice over ranks (Sec. 4: the domain
is cut into equal sub-domains, one per GPU, which exchange their border
planes every time step; Tables multiGPU and multiGPU2 measure it).

Rank r of W owns the planes [z0, z1) = [r nz / W, (r + 1) nz / W) and keeps
them as an extended slab with HALO = 2 ghost planes on each side, periodic
across the ranks. Two planes are what one step needs: the force at a plane
uses the densities of the planes next to it, and those densities sum
populations pulled from one plane further. So a rank that holds its
neighbours' two border planes steps its own planes exactly as the single
lattice would, node for node; its ghost planes come out wrong (they would
need planes further away) and the exchange overwrites them:

    step the extended slab  ->  exchange()  ->  the bounce-back pass (masked)

exchange() sends the first HALO interior planes to the lower neighbour and
the last HALO to the upper one, and receives theirs into the ghost planes.
It uses only point-to-point messages of torch.distributed, so one code path
serves any backend: gloo with CPU tensors, or a device backend with device
tensors. On a masked lattice the write-side bounce-back of the links whose
source is a ghost node must run after the exchange (the ghost's value is
only right then), which is why the library's step splits into the kernel
step and the link pass. Conserved totals add up over the interior planes of
all ranks (allreduce_sum, in FP64).

This module moves data and holds no arithmetic of the method.
"""
import torch
import torch.distributed as dist

HALO = 2
# message tags: what travels towards the lower / the upper neighbour
_TAG_DOWN, _TAG_UP = 11, 12


def slab_bounds(nz, world, rank):
    """Planes [z0, z1) owned by `rank` of `world` (equal up to one plane)."""
    if not (0 <= rank < world) or world < 1:
        raise ValueError("rank %d of %d" % (rank, world))
    z0 = rank * nz // world
    z1 = (rank + 1) * nz // world
    if z1 - z0 < HALO:
        raise ValueError("a slab needs at least %d planes (nz = %d over %d ranks)" % (HALO, nz, world))
    return z0, z1


def extended_planes(nz, world, rank):
    """Global plane index of every plane of the extended slab, in order:
    HALO ghosts below, the owned planes, HALO ghosts above (periodic)."""
    z0, z1 = slab_bounds(nz, world, rank)
    return [(z % nz) for z in range(z0 - HALO, z1 + HALO)]


def extend(field, nz, world, rank, axis):
    """The extended slab of a global field (any array indexable with a list
    of plane indices along `axis`, e.g. numpy or torch)."""
    idx = extended_planes(nz, world, rank)
    if isinstance(field, torch.Tensor):
        return field.index_select(axis, torch.tensor(idx, device=field.device)).contiguous()
    import numpy as np
    return np.ascontiguousarray(np.take(field, idx, axis=axis))


def interior(ext, axis):
    """View of the owned planes of an extended slab."""
    n = ext.shape[axis] - 2 * HALO
    if isinstance(ext, torch.Tensor):
        return ext.narrow(axis, HALO, n)
    import numpy as np
    sl = [slice(None)] * ext.ndim
    sl[axis] = slice(HALO, HALO + n)
    return ext[tuple(sl)]


def border_views(ext, axis):
    """(lower ghosts, first interior planes, last interior planes, upper
    ghosts) of an extended slab tensor, HALO planes each."""
    n = ext.shape[axis] - 2 * HALO
    return (ext.narrow(axis, 0, HALO), ext.narrow(axis, HALO, HALO), ext.narrow(axis, n, HALO),
            ext.narrow(axis, n + HALO, HALO))


def exchange(ext, axis, rank, world, group=None):
    """Fill the ghost planes of the extended slab tensor `ext` (in place)
    with the border planes of the neighbouring ranks. With one rank the slab
    is the whole periodic lattice and its own borders wrap around."""
    lo_ghost, lo_in, hi_in, hi_ghost = border_views(ext, axis)
    if world == 1:
        send_lo, send_hi = lo_in.clone(), hi_in.clone()
        lo_ghost.copy_(send_hi)
        hi_ghost.copy_(send_lo)
        return
    down, up = (rank - 1) % world, (rank + 1) % world
    send_down = lo_in.contiguous()    # my first planes: the upper ghosts of the rank below
    send_up = hi_in.contiguous()      # my last planes: the lower ghosts of the rank above
    recv_from_down = torch.empty_like(send_up)
    recv_from_up = torch.empty_like(send_down)
    # The same order on every rank (towards up, from down, towards down, from
    # up) and distinct tags keep the messages matched when both neighbours are
    # one rank (two ranks) and on backends that match by order.
    ops = [dist.P2POp(dist.isend, send_up, up, group, _TAG_UP),
           dist.P2POp(dist.irecv, recv_from_down, down, group, _TAG_UP),
           dist.P2POp(dist.isend, send_down, down, group, _TAG_DOWN),
           dist.P2POp(dist.irecv, recv_from_up, up, group, _TAG_DOWN)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    lo_ghost.copy_(recv_from_down)
    hi_ghost.copy_(recv_from_up)


def allreduce_sum(values, group=None):
    """Sum of per-rank FP64 totals (e.g. mass and momentum over each rank's
    interior planes) over all ranks."""
    t = torch.as_tensor(values, dtype=torch.float64).clone()
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t
