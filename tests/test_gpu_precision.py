"""Precision form: populations stored as FP32, FP16 or BF16 deviations from
w_i rho0, compared with the FP64 oracle on the seeded 64^3 spinodal case
(tau = 1, G = 0.65, rho_A = 0.5 + 0.05 U(-1,1) seed 1234), 500 steps.

Densities: max-relative error <= 1e-5 (FP32) and <= 2e-3 (FP16/BF16).
Velocity (a vector field): error <= the tolerance times max|u|, or the
storage floor -- 8 half-ulps of the largest initial moving-population
deviation over the smallest density -- whichever is larger (the flow of this
miscible case decays to |u| ~ 1e-6, below what any rounded storage resolves).
The measured errors are printed (pytest -s) for the record.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2112_08264_gb300 import Solver, build, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

HALF_ULP = {"fp32": 2.0 ** -24, "fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
TOL = {"fp32": 1e-5, "fp16": 2e-3, "bf16": 2e-3}


@pytest.fixture(scope="module")
def reference():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    n, steps = 64, 500
    rA, rB = inputs.spinodal(n, n, n, seed=1234)
    a0 = rA.astype(np.float32).astype(np.float64)
    b0 = rB.astype(np.float32).astype(np.float64)
    f0 = oracle.init(a0, b0)
    f = oracle.run(f0, steps, 1.0, 0.65)
    oA, oB, ou = oracle.moments(f, 0.65)
    c, w, _ = oracle.lattice()
    base = np.stack([w[:, None, None, None] * a0.mean(), w[:, None, None, None] * b0.mean()])
    dmax = np.abs((f0 - base)[:, 1:]).max()
    return dict(n=n, steps=steps, rA=rA, rB=rB, oA=oA, oB=oB, ou=ou, dmax=dmax)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_precision_against_oracle_64cubed_500_steps(reference, prec):
    R = reference
    n = R["n"]
    s = Solver(n, n, n, 1.0, 0.65, prec=prec)
    dev = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    s.init(dev(R["rA"]), dev(R["rB"]))
    s.step(R["steps"])
    gA, gB, gu = (t.cpu().numpy().astype(np.float64) for t in s.moments())
    s.close()
    out = {}
    for name, a, b in (("rho_A", gA, R["oA"]), ("rho_B", gB, R["oB"])):
        scale = np.abs(b).max()
        out[name] = (np.abs(a - b).max() / scale, np.sqrt(((a - b) ** 2).mean()) / scale)
    uscale = np.sqrt((R["ou"] ** 2).sum(axis=0)).max()
    du = gu - R["ou"]
    out["u"] = (np.abs(du).max() / uscale, np.sqrt((du ** 2).mean()) / uscale)
    print("\nprecision %s 64^3 x %d: " % (prec, R["steps"])
          + ", ".join("%s max %.3e rms %.3e" % (k, v[0], v[1]) for k, v in out.items())
          + " (max|u| = %.3e)" % uscale)
    assert out["rho_A"][0] <= TOL[prec] and out["rho_B"][0] <= TOL[prec]
    floor = 8 * HALF_ULP[prec] * R["dmax"] / min(R["oA"].min() + R["oB"].min(), 1.0)
    assert np.abs(du).max() <= max(TOL[prec] * uscale, floor)


# A flow-dominated two-component case: the decaying shear wave
# u_x = 1e-3 sin(2 pi y / ny) through the seeded spinodal mixture (40 x 32 x 24,
# tau = 0.8, G = 0.65, seed 55), 100 steps. rho_A, rho_B and u (as a vector
# field) are held to the plain 2e-3 max-relative bar with no storage floor.
# BF16 keeps 8 significant bits: every stored deviation (about w_i * 0.05 from
# the density noise, against about w_i * 1.5e-3 from the flow) is rounded to
# 2^-9 of itself, and the velocity, a difference of such values, comes out
# at 6.6e-3 of max|u| in an FP64 emulation of the rounding and at 6.6e-3 on
# the GPU; FP16 (11 bits) gives 8.9e-4 (GPU). The BF16 velocity therefore
# misses the bar, which stays 2e-3: the case is an expected failure.
@pytest.mark.parametrize("prec", [
    "fp16",
    pytest.param("bf16", marks=pytest.mark.xfail(
        strict=True, reason="BF16 storage resolves this flow's velocity to about 6e-3 of max|u| (bar 2e-3)")),
])
def test_flow_dominated_reduced_precision_100_steps(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    nx, ny, nz, tau, G, steps = 40, 32, 24, 0.8, 0.65, 100
    rA, rB = inputs.spinodal(nx, ny, nz, seed=55)
    u = np.zeros((3, nz, ny, nx))
    u[0] = 1e-3 * np.sin(2 * np.pi * np.arange(ny) / ny)[None, :, None]
    dev = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    s = Solver(nx, ny, nz, tau, G, prec=prec)
    s.init(dev(rA), dev(rB), dev(u))
    s.step(steps)
    gA, gB, gu = (t.cpu().numpy().astype(np.float64) for t in s.moments())
    s.close()
    r32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    f = oracle.run(oracle.init(r32(rA), r32(rB), r32(u)), steps, tau, G)
    oA, oB, ou = oracle.moments(f, G)
    eA = np.abs(gA - oA).max() / np.abs(oA).max()
    eB = np.abs(gB - oB).max() / np.abs(oB).max()
    eu = np.abs(gu - ou).max() / np.sqrt((ou * ou).sum(axis=0)).max()
    print("\nflow-dominated %s: rho_A %.3e rho_B %.3e u %.3e" % (prec, eA, eB, eu))
    assert eA <= TOL[prec] and eB <= TOL[prec]
    assert eu <= TOL[prec]
