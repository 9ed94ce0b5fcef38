"""Benchmark: GLUPS of the two-component D3Q19 Shan-Chen step on GB300.

Default workload: spinodal mixture on a 256^3 periodic grid (tau = 1,
G = 0.65, rho_A = 0.5 + 0.05 U(-1,1) seed 1234, rho_B = 1 - rho_A, u = 0),
FP32 populations, fused kernel; FP16/BF16 deviation storage and the two-pass
kernel are timed beside it. GLUPS = nx*ny*nz / (1e9 * seconds per step)
(Eq. glups). The state (2 x 2.55 GB at 256^3 FP32) is far larger than the
129 MB L2, so no flush is needed between steps.

One JSON line on rank 0. ``--impl reference`` times the FP64 CPU oracle on
the host cores instead (bounded sample of the same workload). With N > 1
(torchrun) every rank runs an independent replica by default, and value = all
site updates / max-over-ranks time; ``--decompose`` instead cuts the one
lattice into z-slabs over the ranks, which exchange their border planes every
step (strong scaling).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS, 2-comp D3Q19 Shan-Chen 256^3, FP32 vs FP16-store; % of HBM roofline"
BYTES_PER_SITE = {"fp32": 304, "fp16": 152, "bf16": 152}   # 38 pops read + written once
DTYPE_TAG = {"fp32": "f32", "fp16": "f16-store/f32-compute", "bf16": "bf16-store/f32-compute"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_per_site(prec):
    """Per-site DRAM bytes of the fused kernel from the committed ncu summary
    (dram__bytes_read.sum + dram__bytes_write.sum per launch / sites)."""
    p = os.path.join(ROOT, "profiles", "fused_step_traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        parts = line.split()
        if len(parts) >= 2 and parts[0] == prec and not line.startswith("#"):
            return float(parts[1])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(local)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    on_gpu = torch.cuda.is_available() and dist.get_backend() == "nccl"
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if on_gpu else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def main_decomposed(args, W, world, rank, local):
    """One lattice cut into z-slabs over the ranks (strong scaling; the paper's
    multi-GPU scheme, Sec. 4): each rank a context over its planes plus two
    ghost planes per side, stepped with lb_step_fluid, the exchange of border
    planes (decomp.exchange, point-to-point messages of the process group) and
    lb_step_links. value = the whole lattice's site updates / the slowest
    rank's timed region. With one rank the slab is the whole periodic lattice
    and its borders wrap onto its own ghosts (the same code path)."""
    import torch
    from paper_2112_08264_gb300 import Solver, decomp
    nx, ny, nz = W["shape"]
    N = nx * ny * nz
    idx = decomp.extended_planes(nz, world, rank)
    z0, z1 = decomp.slab_bounds(nz, world, rank)
    rho0 = (float(np.float32(W["rA"]).astype(np.float64).mean()), float(np.float32(W["rB"]).astype(np.float64).mean()))
    s = Solver(nx, ny, len(idx), W["tau"], W["G"], prec=args.prec, rho0=rho0, slab_halo=decomp.HALO)
    s.init(torch.tensor(np.ascontiguousarray(W["rA"][idx]), dtype=torch.float32, device="cuda"),
           torch.tensor(np.ascontiguousarray(W["rB"][idx]), dtype=torch.float32, device="cuda"))

    def one_step():
        s.step_fluid()
        decomp.exchange(s.planes(), 0, rank, world)
        s.step_links()

    decomp.exchange(s.planes(), 0, rank, world)
    s.step_links()
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record()
        for _ in range(args.steps):
            one_step()
        e1.record()
        e1.synchronize()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    step_s = ms / 1e3 / args.steps
    totals = decomp.allreduce_sum(s.stats_planes(decomp.HALO, z1 - z0)).numpy()
    s.close()
    glups = N / step_s / 1e9
    peak, peak_kind = measured_peaks()
    bps = BYTES_PER_SITE[args.prec]
    line = {
        "metric": W.get("metric", METRIC), "value": glups, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": DTYPE_TAG[args.prec], "data": "synthetic",
        "config": {"workload": W["desc"], "grid": [nx, ny, nz], "prec": args.prec, "kernel": "fused",
                   "parallelism": "z-slabs x%d (two ghost planes per side, exchanged every step)" % world,
                   "slab_planes": [z1 - z0, len(idx)]},
        "roofline": {"bound": "hbm", "achieved": bps * N / step_s / 1e9 / world, "peak": peak, "unit": "GB/s",
                     "frac": bps * N / step_s / 1e9 / world / peak, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_site": bps,
                     "timed": "per GPU: its share of the lattice's algorithmic bytes over the whole step "
                              "(kernel, border exchange, bounce-back pass)", "traffic": None},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "conserved_totals": [float(x) for x in totals],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def replica_throughput(ms_local, steps, sites_per_replica, world):
    """Whole-job GLUPS of `world` independent replicas: all site updates over
    the slowest rank's timed region (max over ranks), and that time per step."""
    ms_max = max_over_ranks(ms_local, world)
    step_s = ms_max / 1e3 / steps
    return world * sites_per_replica / step_s / 1e9, step_s


def workload(name, grid=None):
    from paper_2112_08264_gb300 import inputs
    if name == "spinodal256":
        n = grid or 256
        rA, rB = inputs.spinodal(n, n, n, seed=1234)
        return dict(shape=(n, n, n), tau=1.0, G=0.65, rA=rA, rB=rB, mask=None, traffic="" if n == 256 else None,
                    desc="spinodal %d^3 periodic, tau=1, G=0.65, rho_A=0.5+0.05U(-1,1) seed 1234" % n)
    if name == "colloid256":
        # the grid override keeps the solid fraction: 4000 spheres per 256^3 (profiling cases)
        n = grid or 256
        count = max(1, int(round(4000 * (n / 256.0) ** 3)))
        rA, rB = inputs.spinodal(n, n, n, seed=1234)
        mask, _ = inputs.colloid_mask(n, n, n, n_spheres=count, radius=5.0, seed=4321)
        return dict(shape=(n, n, n), tau=1.0, G=0.65, rA=rA, rB=rB, mask=mask,
                    traffic="colloid_" if n == 256 else None,
                    desc="%d^3, %d static spheres R=5 (seed 4321), halfway bounce-back" % (n, count))
    if name == "orderparam256":
        n = grid or 256
        rA, rB = inputs.random_order_parameter(n, n, n, seed=1234)
        return dict(shape=(n, n, n), tau=1.0, G=0.65, rA=rA, rB=rB, mask=None, traffic="" if n == 256 else None,
                    desc="%d^3 periodic, random order parameter +-0.9 per site (seed 1234), tau=1, G=0.65" % n)
    if name == "cg256":
        n = grid or 256
        rA, rB = inputs.random_order_parameter(n, n, n, seed=1234, phi0=1.0)
        cg = dict(nu=(1.0 / 6.0, 1.0 / 6.0), sigma=0.01, beta=0.7)
        return dict(shape=(n, n, n), tau=1.0, G=0.0, rA=rA, rB=rB, mask=None, model="colour_gradient", cg=cg,
                    traffic="cg_" if n == 256 else None,
                    solver_kw=dict(model="colour_gradient", cg=cg),
                    metric="GLUPS, 2-comp D3Q19 colour-gradient %d^3 (the paper's two-fluid case); "
                           "%% of HBM roofline" % n,
                    desc="colour gradient %d^3 periodic, random order parameter +-1 per site (seed 1234), "
                         "nu_A = nu_B = 1/6, sigma = 0.01, beta = 0.7" % n)
    if name == "single256":
        n = grid or 256
        rng = np.random.default_rng(1234)
        rho = 1.0 + 0.05 * rng.uniform(-1, 1, (n, n, n))
        return dict(shape=(n, n, n), tau=1.0, G=0.0, rA=rho, rB=None, mask=None, model="single",
                    metric="GLUPS, 1-comp D3Q19 BGK %d^3 (the paper's single-fluid case); %% of HBM roofline" % n,
                    desc="single fluid %d^3 periodic, tau=1, rho=1+0.05U(-1,1) seed 1234, u=0" % n)
    if name == "particles256":
        return particle_workload(grid or 256, 0.10)
    if name == "spinodal512":
        n = 512
        rA, rB = inputs.spinodal(n, n, n, seed=1234)
        return dict(shape=(n, n, n), tau=1.0, G=0.65, rA=rA, rB=rB, mask=None,
                    desc="spinodal 512^3 periodic, tau=1, G=0.65")
    raise ValueError(name)


def particle_workload(n, phi, seed=2112):
    """The paper's particle setup (case 3): spheres of radius 5.5 at random,
    non-overlapping places filling the volume fraction phi, at rest, with the
    mass of silica in a fluid of density 1 (2.2 times the sphere's volume),
    in the headline spinodal fill."""
    from paper_2112_08264_gb300 import inputs
    R = 5.5
    vol = 4.0 / 3.0 * np.pi * R ** 3
    count = max(1, int(round(phi * n ** 3 / vol)))
    mask, centres = inputs.colloid_mask(n, n, n, n_spheres=count, radius=R, seed=seed)
    rA, rB = inputs.spinodal(n, n, n, seed=1234)
    return dict(shape=(n, n, n), tau=1.0, G=0.65, rA=rA, rB=rB, mask=None, model="particles",
                spheres=dict(r=centres, radius=R, mass=2.2 * vol, contact=(10.0, 1.0)), phi=phi,
                fluid=float((mask == 0).mean()),
                metric="GLUPS, 2-comp D3Q19 Shan-Chen %d^3 with %d moving spheres R = 5.5 (volume fraction %g, "
                       "the paper's particle case); %% of HBM roofline" % (n, count, phi),
                desc="spinodal %d^3 (seed 1234), tau=1, G=0.65; %d spheres R=5.5 at rest, random places "
                     "(seed %d, gaps >= 1), mass 2.2 x volume, contact k = 10 within 1 node" % (n, count, seed))


def time_particles(W, prec, steps, warmup):
    """Device-resident timing of the step with moving spheres (CUDA events on
    the solver's stream around exactly `steps` steps)."""
    import torch
    from paper_2112_08264_gb300 import Solver
    nx, ny, nz = W["shape"]
    sp = W["spheres"]
    s = Solver(nx, ny, nz, W["tau"], W["G"], prec=prec, max_particles=len(sp["r"]))
    s.set_particles(sp["r"], radius=sp["radius"], mass=sp["mass"], contact=sp["contact"])
    s.init(torch.tensor(W["rA"], dtype=torch.float32, device="cuda"),
           torch.tensor(W["rB"], dtype=torch.float32, device="cuda"))
    s.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s.stream):
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    info, st = s.launch_info(), s.stats()
    p = s.particles()          # raises if spheres met or ran faster than a node per step
    s.close()
    torch.cuda.synchronize()
    return ms, info, st, p


def e2e_particles(W, prec, steps):
    """Host fields and sphere places -> pinned H2D -> lb_particles_set ->
    lb_init -> steps -> moments and spheres -> D2H, timed on the host (the
    context and its workspace are made before the timed region)."""
    import torch
    from paper_2112_08264_gb300 import Solver
    nx, ny, nz = W["shape"]
    sp = W["spheres"]
    hA = torch.from_numpy(W["rA"].astype(np.float32)).pin_memory()
    hB = torch.from_numpy(W["rB"].astype(np.float32)).pin_memory()

    def run(k):
        s = Solver(nx, ny, nz, W["tau"], W["G"], prec=prec, max_particles=len(sp["r"]))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s.stream):
            dA = hA.to("cuda", non_blocking=True)
            dB = hB.to("cuda", non_blocking=True)
            s.set_particles(sp["r"], radius=sp["radius"], mass=sp["mass"], contact=sp["contact"])
            s.init(dA, dB)
            s.step(k)
            oA, oB, ou = s.moments()
            out = [x.cpu() for x in (oA, oB, ou)]
        p = s.particles()
        t1 = time.perf_counter()
        s.close()
        del out, p
        return t1 - t0

    run(3)   # warm
    dt = run(steps)
    n = nx * ny * nz
    return dt, 2 * n * 4 + 3 * 8 * len(sp["r"]), 5 * n * 4 + 15 * 8 * len(sp["r"])


def particle_oracle_sample(W, n_xy=64, nz_s=24):
    """The particle oracle on a periodic 64 x 64 x 24 sample of the workload:
    the same fill and sphere size at the same volume fraction."""
    from oracle import particles as op
    from paper_2112_08264_gb300 import inputs
    sp = W["spheres"]
    R = sp["radius"]
    count = max(1, int(round(W["phi"] * n_xy * n_xy * nz_s / (4.0 / 3.0 * np.pi * R ** 3))))
    _, centres = inputs.colloid_mask(n_xy, n_xy, nz_s, n_spheres=count, radius=R, seed=7)
    rA, rB = inputs.spinodal(n_xy, n_xy, nz_s, seed=1234)
    parts = op.Particles(centres, radius=R, mass=sp["mass"], contact=sp["contact"])
    owner = op.coverage((nz_s, n_xy, n_xy), parts.r, R)
    fluid = owner < 0
    rho0 = (rA[fluid].mean(), rB[fluid].mean())
    state = [op.init(rA, rB, None, None, owner), owner]

    def step():
        state[0], state[1] = op.step(state[0], state[1], None, parts, W["tau"], W["G"], rho0)
    return step, n_xy * n_xy * nz_s, "%d spheres in a %dx%dx%d periodic sample" % (count, n_xy, n_xy, nz_s)


def main_particles(args, W, world, rank, local):
    """The step with moving spheres: same JSON contract as the other lines."""
    nx, ny, nz = W["shape"]
    N = nx * ny * nz
    peak, peak_kind = measured_peaks()
    barrier(world)
    with ClockSampler(local) as clk:
        ms, info, st, p = time_particles(W, args.prec, args.steps, args.warmup)
    clocks = clk.summary()
    if not clocks_ok(clocks):
        with ClockSampler(local) as clk:
            ms, info, st, p = time_particles(W, args.prec, args.steps, args.warmup)
        clocks = clk.summary()
        clocks["remeasured"] = True
    barrier(world)
    glups, step_s = replica_throughput(ms, args.steps, N, world)
    fluid = W["fluid"]
    alg_bytes = fluid * BYTES_PER_SITE[args.prec] + 4
    achieved = alg_bytes * N / step_s / 1e9
    line = {
        "metric": W["metric"], "value": glups, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
        # the paper's particle runs (Table partic: V100 0.484 / 0.446 / 0.299 GLUPS at 0.1 / 1 / 10 %) use
        # its colour-gradient fluid with contact and lubrication forces: context, not this workload
        "vs_baseline": None, "dtype": DTYPE_TAG[args.prec], "data": "synthetic",
        "config": {"workload": W["desc"], "grid": [nx, ny, nz], "prec": args.prec, "kernel": "fused",
                   "spheres": len(W["spheres"]["r"]), "volume_fraction": W["phi"],
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "state %.2f GB per buffer > 129 MB L2; no flush needed"
                         % (38 * N * (BYTES_PER_SITE[args.prec] / 76) / 1e9),
                   "launch": info},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "algorithmic_bytes_per_site": alg_bytes,
                     "timed": "the whole step (%d launches: sphere links, step kernel, contact, leap-frog, two "
                              "re-meshing passes that also update the flags)" % info["launches_per_step"],
                     "traffic": (lambda t: t * N if t is not None and (nx, ny, nz) == (256, 256, 256) else None)(
                         traffic_per_site("particles_" + args.prec))},
        "gpu_launches": args.steps * info["launches_per_step"],
        "fluid_glups": glups * fluid,
        "clocks": clocks,
        "conserved_totals": [float(x) for x in st],
        "spheres_after": {"max_speed": float(np.abs(p["v"]).max()), "max_force": float(np.abs(p["F"]).max())},
        "paper_context": {"V100_GLUPS": {"0.1%": 0.484, "1%": 0.446, "10%": 0.299}},
    }
    if rank == 0 and not args.no_e2e:
        dt, h2d, d2h = e2e_particles(W, args.prec, args.steps)
        line["e2e"] = {"value": N * args.steps / dt / 1e9, "unit": "GLUPS", "h2d_bytes_per_step": h2d / args.steps,
                       "d2h_bytes_per_step": d2h / args.steps,
                       "what": "host fields + sphere places -> pinned H2D -> lb_particles_set -> lb_init -> %d "
                               "steps -> moments + spheres -> D2H" % args.steps}
    if rank == 0 and not args.no_variants:
        var = {}
        for prec in ("fp16",):
            if prec == args.prec:
                continue
            vms, vinfo, _, _ = time_particles(W, prec, args.steps, args.warmup)
            var["%s_phi%g" % (prec, W["phi"])] = {"GLUPS": N / (vms / 1e3 / args.steps) / 1e9,
                                                   "ms_per_step": vms / args.steps}
        for phi in (0.01, 0.001):
            Wv = particle_workload(nx, phi)
            vms, _, _, _ = time_particles(Wv, args.prec, args.steps, args.warmup)
            var["%s_phi%g" % (args.prec, phi)] = {"GLUPS": N / (vms / 1e3 / args.steps) / 1e9,
                                                  "ms_per_step": vms / args.steps, "spheres": len(Wv["spheres"]["r"])}
        line["variants"] = var
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        step, sites, what = particle_oracle_sample(W)
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < 10.0 or k < 2:
            step()
            k += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sites * k / dt / 1e9, "unit": "GLUPS", "cores": 1, "kind": "oracle",
                                "sample": "%d FP64 particle-oracle steps (numpy, one thread), %s (%.1f s)"
                                          % (k, what, dt)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def time_device(W, prec, kernel, steps, warmup, events_per_step=False):
    """Device-resident timing: inputs already in HBM; CUDA events on the
    solver's stream around exactly `steps` steps."""
    import torch
    from paper_2112_08264_gb300 import Solver
    nx, ny, nz = W["shape"]
    s = Solver(nx, ny, nz, W["tau"], W["G"], mask=W["mask"], prec=prec, kernel=kernel, **W.get("solver_kw", {}))
    dA = torch.tensor(W["rA"], dtype=torch.float32, device="cuda")
    dB = torch.tensor(W["rB"], dtype=torch.float32, device="cuda")
    s.init(dA, dB)
    del dA, dB
    s.step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s.stream):
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    info = s.launch_info()
    st = s.stats()
    s.close()
    torch.cuda.synchronize()
    return ms, info, st


def time_e2e(W, prec, kernel, steps):
    """End to end through the public API from HOST arrays: pinned H2D of the
    initial fields, init, `steps` steps, moments, D2H of rho_A, rho_B, u."""
    import torch
    from paper_2112_08264_gb300 import Solver, run_host
    nx, ny, nz = W["shape"]
    s = Solver(nx, ny, nz, W["tau"], W["G"], mask=W["mask"], prec=prec, kernel=kernel, **W.get("solver_kw", {}))
    rA = W["rA"].astype(np.float32)
    rB = W["rB"].astype(np.float32)
    run_host(rA, rB, 3, W["tau"], W["G"], solver=s)      # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    (oA, oB, ou), _ = run_host(rA, rB, steps, W["tau"], W["G"], solver=s)
    t1 = time.perf_counter()
    s.close()
    n = nx * ny * nz
    h2d = 2 * n * 4
    d2h = 5 * n * 4
    return t1 - t0, h2d, d2h, bool(np.isfinite(oA).all())


def other_workloads(peak, peak_kind, steps=200, warmup=10):
    """Short device-timed runs of the other workloads (CUDA events over
    `steps` steps each, after `warmup`): the colloid mask (FP32 and FP16, the
    whole step: step kernel + bounce-back pass), the paper's colour-gradient
    model and single-fluid step, and 2407 moving spheres (10 %), each with its
    algorithmic bytes per site and its fraction of the HBM peak."""
    out = {}
    Wc = workload("colloid256")
    N = 256 ** 3
    fluid = float((Wc["mask"] == 0).mean())
    for prec in ("fp32", "fp16"):
        ms, info, _ = time_device(Wc, prec, "fused", steps, warmup)
        step_s = ms / 1e3 / steps
        alg = fluid * BYTES_PER_SITE[prec] + 4
        out["colloid256_" + prec] = {"GLUPS": N / step_s / 1e9, "fluid_GLUPS": fluid * N / step_s / 1e9,
                                     "ms_per_step": step_s * 1e3, "solid_fraction": 1.0 - fluid,
                                     "algorithmic_bytes_per_site": alg,
                                     "hbm_frac_of_%s" % peak_kind: alg * N / step_s / 1e9 / peak,
                                     "launches_per_step": info["launches_per_step"]}
    del Wc
    Wg = workload("cg256")
    for prec in ("fp32", "fp16", "bf16"):
        ms, info, _ = time_device(Wg, prec, "fused", steps, warmup)
        step_s = ms / 1e3 / steps
        out["cg256_" + prec] = {"GLUPS": N / step_s / 1e9, "ms_per_step": step_s * 1e3,
                                "hbm_frac_of_%s" % peak_kind: BYTES_PER_SITE[prec] * N / step_s / 1e9 / peak,
                                "paper_V100_GLUPS_context": 0.601}
    del Wg
    Ws = workload("single256")
    ms, info, _ = time_single(Ws, "fp32", steps, warmup)
    step_s = ms / 1e3 / steps
    out["single256_fp32"] = {"GLUPS": N / step_s / 1e9, "ms_per_step": step_s * 1e3,
                             "hbm_frac_of_%s" % peak_kind: 152 * N / step_s / 1e9 / peak,
                             "paper_V100_fused_GLUPS_context": 2.011}
    del Ws
    Wp = particle_workload(256, 0.10)
    ms, info, _, _ = time_particles(Wp, "fp32", steps, warmup)
    step_s = ms / 1e3 / steps
    alg = Wp["fluid"] * 304 + 4
    out["particles256_fp32"] = {"GLUPS": N / step_s / 1e9, "ms_per_step": step_s * 1e3,
                                "spheres": len(Wp["spheres"]["r"]), "volume_fraction": Wp["phi"],
                                "algorithmic_bytes_per_site": alg,
                                "hbm_frac_of_%s" % peak_kind: alg * N / step_s / 1e9 / peak,
                                "launches_per_step": info["launches_per_step"],
                                "paper_V100_GLUPS_context": 0.299}
    out["what"] = "%d timed steps each after %d warm-up steps, CUDA events on the solver's stream" % (steps, warmup)
    return out


def precision_512(peak, peak_kind, steps=500, warmup=5):
    """Precision form: the 512^3 spinodal run of `steps` steps with FP32,
    FP16 and BF16 storage, each timed over all its steps (CUDA events), and
    the max and RMS errors of the 16-bit runs' rho_A, rho_B and u against the
    FP32 run (max|a - b| / max|b| and rms(a - b) / max|b| per field; u as a
    vector field). The comparison with the FP64 oracle on the identical 64^3
    seeded case is tests/test_gpu_precision.py."""
    import torch
    from paper_2112_08264_gb300 import Solver
    W = workload("spinodal512")
    n = 512
    N = n ** 3
    out, ref = {}, None
    dA = torch.tensor(W["rA"], dtype=torch.float32, device="cuda")
    dB = torch.tensor(W["rB"], dtype=torch.float32, device="cuda")
    for prec in ("fp32", "fp16", "bf16"):
        s = Solver(n, n, n, W["tau"], W["G"], prec=prec)
        s.init(dA, dB)
        s.step(warmup)
        s.init(dA, dB)   # the measured run starts from the seeded state
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s.stream):
            e0.record(s.stream)
            s.step(steps)
            e1.record(s.stream)
        e1.synchronize()
        step_s = e0.elapsed_time(e1) / 1e3 / steps
        rA, rB, u = s.moments()
        s.close()
        del s
        torch.cuda.synchronize()
        out[prec] = {"GLUPS": N / step_s / 1e9, "ms_per_step": step_s * 1e3, "steps": steps,
                     "hbm_frac_of_%s" % peak_kind: BYTES_PER_SITE[prec] * N / step_s / 1e9 / peak}
        if ref is None:
            ref = (rA, rB, u)
            continue
        err = {}
        for name, a, b in (("rho_A", rA, ref[0]), ("rho_B", rB, ref[1])):
            d = (a.double() - b.double())
            scale = float(b.abs().max())
            err[name] = {"max": float(d.abs().max()) / scale, "rms": float(d.pow(2).mean().sqrt()) / scale}
        du = (u.double() - ref[2].double())
        uscale = float(ref[2].double().pow(2).sum(dim=0).sqrt().max())
        # this miscible mixture relaxes to rest: after 500 steps |u| is at the rounding level of the
        # stored deviations, so the absolute error is given with the relative one
        err["u"] = {"max": float(du.abs().max()) / uscale, "rms": float(du.pow(2).mean().sqrt()) / uscale,
                    "max_abs_error": float(du.abs().max()), "max_abs_u_fp32": uscale}
        out[prec]["error_vs_fp32"] = err
        del rA, rB, u, du
    out["fp16_over_fp32"] = out["fp16"]["GLUPS"] / out["fp32"]["GLUPS"]
    out["bf16_over_fp32"] = out["bf16"]["GLUPS"] / out["fp32"]["GLUPS"]
    out["workload"] = W["desc"] + ", %d steps per precision" % steps
    return out


def time_adjoint(prec, kernel, n=128, steps=400, K=40, warmup=1):
    """Differentiation form: forward with checkpoints every K steps, then
    lb_backward; returns per-step ms of both, their ratio and the workspace
    the recording needs."""
    import torch
    from paper_2112_08264_gb300 import Solver, inputs
    rA, rB = inputs.spinodal(n, n, n, seed=1234)
    target = torch.tensor(inputs.smoothed_target(n, n, n, seed=99), dtype=torch.float32, device="cuda")
    s = Solver(n, n, n, 1.0, 0.65, prec=prec, kernel=kernel, ckpt_every=K, ckpt_steps_max=steps)
    dA = torch.tensor(rA, dtype=torch.float32, device="cuda")
    dB = torch.tensor(rB, dtype=torch.float32, device="cuda")
    fwd, bwd = [], []
    for rep in range(warmup + 1):
        s.init(dA, dB)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
        fA, _, _ = s.moments(velocity=False)
        s.backward((2.0 * (fA - target)).contiguous(), want_rho=True)
        e2.record(s.stream)
        e2.synchronize()
        fwd.append(e0.elapsed_time(e1))
        bwd.append(e1.elapsed_time(e2))
    ws = int(s.workspace.numel())
    s.close()
    f_ms, b_ms = fwd[-1] / steps, bwd[-1] / steps
    return {"grid": [n, n, n], "steps": steps, "ckpt_every": K, "checkpoints": steps // K + 1,
            "forward_ms_per_step": f_ms, "backward_ms_per_step": b_ms, "backward_over_forward": b_ms / f_ms,
            "workspace_bytes": ws}


def oracle_sample(shape, tau, G, budget_s, min_steps=1, max_steps=1000, per_step_budget=None):
    """Time the FP64 oracle on a periodic slab of the workload (full x-y
    plane, nz_s planes) sized so the run takes about budget_s seconds."""
    import oracle
    from paper_2112_08264_gb300 import inputs
    nx, ny, nz = shape
    cores = oracle.max_threads()
    oracle.set_threads(cores)
    # probe the speed on a thin slab
    rA, rB = inputs.spinodal(nx, ny, 2, seed=1234)
    f = oracle.init(rA, rB)
    t0 = time.perf_counter()
    oracle.step(f, tau, G)
    rate = nx * ny * 2 / max(time.perf_counter() - t0, 1e-6)   # sites/s
    if per_step_budget is not None:
        nzs = int(max(1, min(nz, per_step_budget * rate / (nx * ny))))
        steps = None
    else:
        nzs = int(max(2, min(nz, 16)))
        steps = int(max(min_steps, min(max_steps, budget_s * rate / (nx * ny * nzs))))
    rA, rB = inputs.spinodal(nx, ny, nzs, seed=1234)
    return rA, rB, nzs, steps, cores


def cg_oracle_sample(W, budget_s=None, per_step_budget=None):
    """Colour-gradient oracle (numpy, one thread) on a periodic slab of the
    workload's recipe, sized like oracle_sample."""
    from oracle import colour_gradient as cgo
    from oracle import lb_numpy as ln
    from paper_2112_08264_gb300 import inputs
    nx, ny, nz = W["shape"]
    c = W["cg"]
    rA, rB = inputs.random_order_parameter(nx, ny, 2, seed=1234, phi0=1.0)
    f = ln.init(rA, rB)
    t0 = time.perf_counter()
    cgo.step(f, c["nu"][0], c["nu"][1], c["sigma"], c["beta"])
    rate = nx * ny * 2 / max(time.perf_counter() - t0, 1e-6)
    if per_step_budget is not None:
        nzs, steps = int(max(1, min(nz, per_step_budget * rate / (nx * ny)))), None
    else:
        nzs = int(max(2, min(nz, 16)))
        steps = int(max(1, min(1000, budget_s * rate / (nx * ny * nzs))))
    rA, rB = inputs.random_order_parameter(nx, ny, nzs, seed=1234, phi0=1.0)
    step = lambda g: cgo.step(g, c["nu"][0], c["nu"][1], c["sigma"], c["beta"])
    return ln.init(rA, rB), step, nzs, steps


def run_cpu_baseline(W, budget_s=15.0):
    import oracle
    nx, ny, nz = W["shape"]
    if W.get("model") == "colour_gradient":
        f, step, nzs, steps = cg_oracle_sample(W, budget_s)
        t0 = time.perf_counter()
        for _ in range(steps):
            f = step(f)
        dt = time.perf_counter() - t0
        return {"value": nx * ny * nzs * steps / dt / 1e9, "unit": "GLUPS", "cores": 1, "kind": "oracle",
                "sample": "%d FP64 colour-gradient oracle steps (numpy, one thread) on a %dx%dx%d periodic slab "
                          "of the workload (%.1f s)" % (steps, nx, ny, nzs, dt)}
    rA, rB, nzs, steps, cores = oracle_sample(W["shape"], W["tau"], W["G"], budget_s)
    f = oracle.init(rA, rB)
    t0 = time.perf_counter()
    oracle.run(f, steps, W["tau"], W["G"])
    dt = time.perf_counter() - t0
    glups = nx * ny * nzs * steps / dt / 1e9
    return {"value": glups, "unit": "GLUPS", "cores": cores, "kind": "oracle",
            "sample": "%d FP64 oracle steps on a %dx%dx%d periodic slab of the workload (%.1f s)"
                      % (steps, nx, ny, nzs, dt)}


def clocks_ok(c):
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if any(r in bad for r in c.get("reasons", [])):
        return False
    if c.get("sm_mhz") and c.get("sm_max_mhz") and c["sm_mhz"] < 0.5 * c["sm_max_mhz"] \
            and "sw_power_cap" not in c.get("reasons", []):
        return False
    return True


def main_reference(args, world, rank):
    if rank != 0:
        return 0
    W = workload(args.config, args.grid)
    nx, ny, nz = W["shape"]
    import oracle
    # each step a bounded slab sample sized so warmup + steps take ~150 s
    per_step = 150.0 / max(1, args.steps + args.warmup)
    if W.get("model") == "colour_gradient":
        f, step, nzs, _ = cg_oracle_sample(W, per_step_budget=per_step)
        cores = 1
    elif W.get("model") == "single":
        f, step, nzs, _ = single_oracle_sample(W, per_step_budget=per_step)
        cores = 1
    elif W.get("model") == "particles":
        pstep, sites, what = particle_oracle_sample(W)
        f, nzs, cores = None, sites / (nx * ny), 1

        def step(_):
            pstep()
            return None
    else:
        rA, rB, nzs, _, cores = oracle_sample(W["shape"], W["tau"], W["G"], None, per_step_budget=per_step)
        f = oracle.init(rA, rB)
        step = lambda g: oracle.step(g, W["tau"], W["G"])
    for _ in range(args.warmup):
        f = step(f)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = step(f)
    dt = time.perf_counter() - t0
    glups = nx * ny * nzs * args.steps / dt / 1e9
    sample = "each step: one FP64 oracle step on a %dx%dx%d periodic slab of the workload" % (nx, ny, nzs)
    if W.get("model") == "particles":
        sample = "each step: one FP64 particle-oracle step (numpy, one thread), " + what
    line = {"impl": "reference", "metric": W.get("metric", METRIC), "value": glups, "unit": "GLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": W["desc"], "sample": sample},
            "cpu_baseline": {"value": glups, "unit": "GLUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": glups, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_single(W, prec, steps, warmup):
    """Device-resident timing of the one-component step (CUDA events on its stream)."""
    import torch
    from paper_2112_08264_gb300 import SingleFluid
    nx, ny, nz = W["shape"]
    s = SingleFluid(nx, ny, nz, W["tau"], prec=prec)
    s.init(torch.tensor(W["rA"], dtype=torch.float32, device="cuda"))
    s.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s.stream):
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    info, st = s.launch_info(), s.stats()
    s.close()
    torch.cuda.synchronize()
    return ms, info, st


def e2e_single(W, prec, steps):
    """Host rho -> pinned H2D -> lb1_init -> steps -> moments -> D2H, timed on the host."""
    import torch
    from paper_2112_08264_gb300 import SingleFluid
    nx, ny, nz = W["shape"]
    s = SingleFluid(nx, ny, nz, W["tau"], prec=prec)
    host = torch.from_numpy(W["rA"].astype(np.float32)).pin_memory()
    out_r = torch.empty(host.shape, dtype=torch.float32).pin_memory()
    out_u = torch.empty((3,) + tuple(host.shape), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d = host.to("cuda", non_blocking=True)
    s.init(d)
    s.step(steps)
    r, u = s.moments()
    out_r.copy_(r, non_blocking=True)
    out_u.copy_(u, non_blocking=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    return dt, host.numel() * 4, (out_r.numel() + out_u.numel()) * 4


def single_oracle_sample(W, budget_s=None, per_step_budget=None):
    from oracle import single_bgk as sb
    nx, ny, nz = W["shape"]
    rng = np.random.default_rng(1234)
    probe = sb.WEIGHTS[:, None, None, None] * (1.0 + 0.05 * rng.uniform(-1, 1, (2, ny, nx)))
    t0 = time.perf_counter()
    sb.step(probe, W["tau"])
    rate = nx * ny * 2 / max(time.perf_counter() - t0, 1e-6)
    if per_step_budget is not None:
        nzs, steps = int(max(1, min(nz, per_step_budget * rate / (nx * ny)))), None
    else:
        nzs = int(max(2, min(nz, 16)))
        steps = int(max(1, min(1000, budget_s * rate / (nx * ny * nzs))))
    f = sb.WEIGHTS[:, None, None, None] * W["rA"][:nzs]
    return f, (lambda g: sb.step(g, W["tau"])), nzs, steps


def main_single(args, W, world, rank, local):
    """The one-component step: same JSON contract as the two-component line."""
    nx, ny, nz = W["shape"]
    N = nx * ny * nz
    peak, peak_kind = measured_peaks()
    barrier(world)
    with ClockSampler(local) as clk:
        ms, info, st = time_single(W, args.prec, args.steps, args.warmup)
    clocks = clk.summary()
    if not clocks_ok(clocks):
        with ClockSampler(local) as clk:
            ms, info, st = time_single(W, args.prec, args.steps, args.warmup)
        clocks = clk.summary()
        clocks["remeasured"] = True
    barrier(world)
    glups, step_s = replica_throughput(ms, args.steps, N, world)
    bps = BYTES_PER_SITE[args.prec] // 2   # 19 populations read and written once
    achieved = bps * N / (ms / 1e3 / args.steps) / 1e9
    line = {
        "metric": W["metric"], "value": glups, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
        # the paper's single-V100 fused figure at 256^3 (Table 1); context, other hardware
        "vs_baseline": glups / 2.011 if (nx, ny, nz) == (256, 256, 256) else None,
        "dtype": DTYPE_TAG[args.prec], "data": "synthetic",
        "config": {"workload": W["desc"], "grid": [nx, ny, nz], "prec": args.prec, "kernel": "fused",
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "state %.2f GB per buffer > 129 MB L2; no flush needed" % (19 * N * (bps / 38) / 1e9),
                   "launch": info},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "algorithmic_bytes_per_site": bps,
                     "timed": "the step kernel (one launch per step)",
                     "traffic": (traffic_per_site("single_" + args.prec) or 0) * N or None},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "conserved_totals": [float(x) for x in st],
    }
    if rank == 0 and not args.no_e2e:
        dt, h2d, d2h = e2e_single(W, args.prec, args.steps)
        line["e2e"] = {"value": N * args.steps / dt / 1e9, "unit": "GLUPS", "h2d_bytes_per_step": h2d / args.steps,
                       "d2h_bytes_per_step": d2h / args.steps,
                       "what": "host rho -> pinned H2D -> lb1_init -> %d steps -> moments -> D2H" % args.steps}
    if rank == 0 and not args.no_variants:
        var = {}
        for prec in ("fp32", "fp16", "bf16"):
            if prec == args.prec:
                continue
            vms, _, _ = time_single(W, prec, args.steps, args.warmup)
            vstep = vms / 1e3 / args.steps
            var[prec] = {"GLUPS": N / vstep / 1e9, "ms_per_step": vstep * 1e3,
                         "hbm_frac_of_%s" % peak_kind: BYTES_PER_SITE[prec] // 2 * N / vstep / 1e9 / peak}
        line["variants"] = var
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        f, step, nzs, steps = single_oracle_sample(W, 15.0)
        t0 = time.perf_counter()
        for _ in range(steps):
            f = step(f)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": nx * ny * nzs * steps / dt / 1e9, "unit": "GLUPS", "cores": 1,
                                "kind": "oracle",
                                "sample": "%d FP64 one-component oracle steps (numpy, one thread) on a %dx%dx%d "
                                          "periodic slab of the workload (%.1f s)" % (steps, nx, ny, nzs, dt)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="spinodal256",
                    choices=["spinodal256", "colloid256", "orderparam256", "cg256", "single256", "particles256",
                             "spinodal512"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--kernel", default="fused", choices=["fused", "two_pass"])
    ap.add_argument("--grid", type=int, default=None, help="override the spinodal grid size (profiling)")
    ap.add_argument("--no-variants", action="store_true", help="skip the FP16/BF16/two-pass lines")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--decompose", action="store_true",
                    help="cut one lattice into z-slabs over the ranks (strong scaling) instead of running "
                         "independent replicas")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world, rank, local = dist_setup()
    if args.impl == "reference":
        return main_reference(args, world, rank)

    import torch
    from paper_2112_08264_gb300 import build
    if rank == 0 or world > 1:
        build.build()
    W = workload(args.config, args.grid)
    if args.decompose:
        if W.get("model") is not None or W["mask"] is not None:
            raise SystemExit("--decompose runs the periodic Shan-Chen workloads")
        return main_decomposed(args, W, world, rank, local)
    if W.get("model") == "single":
        return main_single(args, W, world, rank, local)
    if W.get("model") == "particles":
        return main_particles(args, W, world, rank, local)
    nx, ny, nz = W["shape"]
    N = nx * ny * nz
    peak, peak_kind = measured_peaks()

    barrier(world)
    with ClockSampler(local) as clk:
        ms, info, st = time_device(W, args.prec, args.kernel, args.steps, args.warmup)
    clocks = clk.summary()
    if not clocks_ok(clocks):
        with ClockSampler(local) as clk:
            ms, info, st = time_device(W, args.prec, args.kernel, args.steps, args.warmup)
        clocks = clk.summary()
        clocks["remeasured"] = True
    barrier(world)
    glups, step_s = replica_throughput(ms, args.steps, N, world)

    bps = BYTES_PER_SITE[args.prec]
    if W["mask"] is not None:
        fluid = float((W["mask"] == 0).mean())
        alg_bytes = fluid * bps + 4          # populations of fluid nodes + 4-byte flag word
    else:
        fluid = 1.0
        alg_bytes = bps
    kernel_s = (ms / 1e3) / (args.steps * info["launches_per_step"])
    achieved = alg_bytes * N / kernel_s / 1e9 if info["launches_per_step"] == 1 else \
        alg_bytes * N / (ms / 1e3 / args.steps) / 1e9
    # measured DRAM bytes per site of this workload's step (ncu, 256^3), when committed
    tkey = W.get("traffic")
    tps = traffic_per_site(tkey + args.prec) if (args.kernel == "fused" and tkey is not None) else None

    # the paper prints a 256^3 number only for its colour-gradient runs: 0.601
    # GLUPS, one V100, plain two-pass step (Table cg); context, other hardware
    vs_base = glups / 0.601 if (W.get("model") == "colour_gradient" and (nx, ny, nz) == (256, 256, 256)) else None
    line = {
        "metric": W.get("metric", METRIC), "value": glups, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": vs_base, "dtype": DTYPE_TAG[args.prec], "data": "synthetic",
        "config": {"workload": W["desc"], "grid": [nx, ny, nz], "prec": args.prec, "kernel": args.kernel,
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "state %.2f GB per buffer > 129 MB L2; no flush needed" % (38 * N * (bps / 76) / 1e9),
                   "launch": info},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_site": alg_bytes,
                     "timed": ("the step kernel (one launch per step)" if info["launches_per_step"] == 1 else
                               "the whole step (%d launches: step kernel(s) + write-side bounce-back)"
                               % info["launches_per_step"]),
                     "traffic": (tps * N if tps is not None else None)},
        "gpu_launches": args.steps * info["launches_per_step"],
        "fluid_glups": glups * fluid,   # fluid site updates only (all sites count in value)
        "clocks": clocks,
        "conserved_totals": [float(x) for x in st],
    }
    if rank == 0 and not args.no_e2e:
        dt, h2d, d2h, ok = time_e2e(W, args.prec, args.kernel, args.steps)
        line["e2e"] = {"value": N * args.steps / dt / 1e9, "unit": "GLUPS",
                       "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                       "what": "host arrays -> pinned H2D -> lb_init -> %d steps -> moments -> D2H" % args.steps}
    if rank == 0 and not args.no_variants:
        var = {}
        for prec, kern in (("fp16", "fused"), ("bf16", "fused"), ("fp32", "two_pass"), ("fp32", "fused_reg")):
            if (prec, kern) == (args.prec, args.kernel):
                continue
            if kern == "fused_reg" and W.get("model") == "colour_gradient":
                continue   # the register kernel implements Shan-Chen only
            vms, vinfo, _ = time_device(W, prec, kern, args.steps, args.warmup)
            vstep = vms / 1e3 / args.steps
            vb = BYTES_PER_SITE[prec] * (fluid if W["mask"] is not None else 1.0)
            var["%s_%s" % (prec, kern)] = {"GLUPS": N / vstep / 1e9, "ms_per_step": vstep * 1e3,
                                          "hbm_frac_of_%s" % peak_kind: vb * N / vstep / 1e9 / peak,
                                          "launches_per_step": vinfo["launches_per_step"]}
        line["variants"] = var
        if "fp16_fused" in var and args.prec == "fp32":
            line["fp16_over_fp32"] = var["fp16_fused"]["GLUPS"] / glups
        if args.config == "spinodal256" and args.grid is None:
            line["precision_512"] = precision_512(peak, peak_kind)
            line["adjoint_128"] = time_adjoint("fp32", "fused")
            line["other_workloads"] = other_workloads(peak, peak_kind)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = run_cpu_baseline(W)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
