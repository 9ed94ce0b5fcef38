"""lb_moments_noalloc: the allocation-free entry point.

It serves callers that may not allocate device memory (no cudaMalloc, no
allocator of any library), and so cannot hand lb_create a workspace: they
pass a population field and output buffers they already own, and the entry
point keeps its neighbour-density scratch in a static device array. These
checks call it through the C ABI and compare its output with lb_moments on
the same state and with the FP64 oracle's moments of the same population
field, within the parity tolerances of the other GPU tests (1e-5
max-relative on densities, 1e-5 of max|u| on the velocity of a flowing case),
on two calls in a row with different grids and states. This file sorts last
so that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2112_08264_gb300 import _lib, build, inputs


def _call(L, nx, ny, nz, G, g, f, mask_dev, rA, rB, u, stream):
    bf = (ctypes.c_double * 3)(*g)
    return L.lb_moments_noalloc(nx, ny, nz, ctypes.c_float(G), bf, f.data_ptr(),
                                None if mask_dev is None else mask_dev.data_ptr(),
                                rA.data_ptr(), rB.data_ptr(), u.data_ptr(), stream)


def test_rejects_grids_beyond_the_static_scratch():
    build.build()
    L = _lib.lib()
    st = L.lb_moments_noalloc(128, 128, 65, ctypes.c_float(0.65), None, ctypes.c_void_p(1 << 20), None,
                              None, None, None, None)
    assert st == _lib.LB_EINVAL
    assert b"exceeds the static scratch limit" in L.lb_last_error()
    assert L.lb_moments_noalloc(2, 8, 8, ctypes.c_float(0.65), None, ctypes.c_void_p(1 << 20), None,
                                None, None, None, None) == _lib.LB_EINVAL


@pytest.mark.gpu
def test_noalloc_moments_match_lb_moments_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_08264_gb300 import Solver
    build.build()
    L = _lib.lib()
    cases = [((40, 24, 18), 0.8, 0.65, (2e-6, 0.0, -1e-6), 0.1, 7),
             ((20, 17, 11), 1.0, 0.9, (0.0, 0.0, 0.0), 0.0, 12)]
    for (nx, ny, nz), tau, G, g, solid, steps in cases:
        mask = inputs.random_mask(nx, ny, nz, seed=nx, solid_fraction=solid) if solid else None
        rA, rB = inputs.spinodal(nx, ny, nz, seed=ny)
        u0 = np.zeros((3, nz, ny, nx))
        u0[0] = 5e-3 * np.sin(2 * np.pi * np.arange(ny) / ny)[None, :, None]
        dev = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
        s = Solver(nx, ny, nz, tau, G, mask=mask, body_force=g)
        s.init(dev(rA), dev(rB), dev(u0))
        s.step(steps)
        f = s.get_state()
        refA, refB, refu = s.moments()
        oA = torch.empty_like(refA)
        oB = torch.empty_like(refB)
        ou = torch.empty_like(refu)
        mask_dev = None if mask is None else torch.tensor(mask, dtype=torch.uint8, device="cuda")
        st = _call(L, nx, ny, nz, G, g, f, mask_dev, oA, oB, ou, s.stream.cuda_stream)
        assert st == _lib.LB_OK, L.lb_last_error()
        torch.cuda.synchronize()
        for got, ref in ((oA, refA), (oB, refB)):
            err = float((got - ref).abs().max()) / float(ref.abs().max())
            assert err <= 1e-5
        uerr = float((ou - refu).abs().max())
        uscale = float(refu.pow(2).sum(dim=0).sqrt().max())
        assert uerr <= 1e-5 * uscale
        # the FP64 oracle's moments of the same (FP32) population field
        import oracle
        wA, wB, wu = oracle.moments(f.cpu().numpy().astype(np.float64), G, g, mask)
        for got, want in ((oA, wA), (oB, wB)):
            assert np.abs(got.cpu().numpy() - want).max() <= 1e-5 * np.abs(want).max()
        wscale = np.sqrt((wu * wu).sum(axis=0)).max()
        assert np.abs(ou.cpu().numpy() - wu).max() <= 1e-5 * wscale
        if mask is not None:
            m = torch.tensor(mask == 1, device="cuda")
            assert float(oA[m].abs().max()) == 0.0 and float(ou[:, m].abs().max()) == 0.0
        s.close()
