#!/usr/bin/env python3
"""Throughput of the multicomponent lattice Boltzmann timestep on GB300.

One "step" is one timestep of the whole hot path (pull streaming, moments,
Flory-Huggins potentials with the gradient term, Eq. definef force,
equilibria, forcing, BGK collision) over the full lattice.  Default workload:
N = 5 components on a periodic 2048 x 2048 D2Q9 lattice, FP32 storage, random
symmetric chi in [0.8, 1.5] x critical, tau = 1, kappa = 0.01, mean composition
1/5 with +-0.01 uniform noise (synthetic, seeded).  Its distributions (2 x 755 MB
ping-pong) exceed the 129 MB L2, so no flush is needed between steps.

Metric: MLUPS x components = sites * N * steps / seconds / 1e6, whole job.
Roofline: a step moves at least 9 loads + 9 stores of f per (site, component)
(72 B in FP32; 44 B in the 16-bit shifted modes, whose sites also carry an FP32
reference density).  Variants: BF16/FP16-shifted storage, the staged schedule and
a batch of 512 independent simulations, each with its speedup over FP32.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mclb|reference]
Under torchrun each rank advances its own copy of the workload (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS×components and % of HBM roofline; FP32 vs BF16-shifted vs batched"
UNIT = "MLUPS×components"
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["march.cuh", "tma.cuh", "physics.cuh", "lattice.cuh"]
PROFILE = os.path.join(ROOT, "profiles", "k_march_fp32_n5_2048x2048.md")


def walled(prob):
    """The same problem between solid walls in y."""
    prob.walls = 1
    prob.name = prob.name + "_walls"
    return prob


def workloads():
    from paper_0704_3444_gb300 import inputs
    return {
        "n5_2048x2048": lambda: inputs.multi_uniform(),
        "n5_1024x1024": lambda: inputs.multi_uniform(1024, 1024, name="n5_1024x1024"),
        "ternary_256x256": lambda: inputs.ternary_gauss(),
        "binary_64x64": lambda: inputs.binary_noise(precision="fp32"),
        "slab_8192x2048": lambda: inputs.slab(),
        "slab_8192x2048_walls": lambda: walled(inputs.slab()),
        "ternary3d_256": lambda: inputs.ternary3d(256),
        "ternary3d_128": lambda: inputs.ternary3d(128, name="ternary3d_128"),
    }


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_0704_3444_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the fused kernel from the committed ncu summary, or None
    if the summary is missing or was taken from different kernel sources."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    m_hash = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_bytes.group(1))


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = float(json.load(open(path))["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 20 ms) of SM clock, utilisation and throttle reasons over a
    window of GPU work; the summary keeps the samples taken under load (utilisation
    >= 50 %)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
              "utilization.gpu")

    def __init__(self, index: int, interval_ms: int = 20):
        self.index = index
        self.interval_ms = interval_ms
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        total = len(rows)
        rows = [r for r in rows if (num(r[8]) or 0.0) >= 50.0] or rows
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[4 + k]
                          and "Not" not in r[4 + k]})
        pw = [num(r[2]) for r in rows if num(r[2]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "power_w_max": max(pw) if pw else None, "samples": len(rows),
                "samples_total": total}


def gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            return int(vis.split(",")[local_rank])
        except (ValueError, IndexError):
            return local_rank
    return local_rank


def time_steps(torch, sim, steps, warmup, stream):
    """Device time of `steps` timesteps after `warmup` untimed ones (CUDA events on the
    stream the library launches on)."""
    sim.step(warmup)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    sim.step(steps)
    stop.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(stop) / 1e3


def job_rate(torch, dist, work, elapsed, world, device):
    """Whole-job rate over all ranks: every rank has done `work` site-component updates in
    `elapsed` seconds of its own; the job took as long as the slowest rank (barrier, then
    the maximum over ranks).  Returns (MLUPS x N of the whole job, that maximum)."""
    if dist is not None:
        dist.barrier()
        t = torch.tensor([elapsed], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    return world * work / elapsed / 1e6, elapsed


def run_slabs(torch, mclb, prob, warmup, fp32_value, parts=2, steps=200):
    """The workload's lattice cut into ``parts`` y slabs held by separate handles on this
    GPU (paper_0704_3444_gb300.slabs.LocalSlabs), every slab padded by 3 * period rows
    on each side and refreshed from its neighbours' bands every ``period`` steps: the cost
    of the decomposition a multi-GPU split of one lattice uses, measured without the
    interconnect (extra rows, band copies, twice the launches)."""
    from paper_0704_3444_gb300 import slabs as slabs_mod

    out = {}
    kw = dict(ncomp=prob.ncomp, tau=prob.tau, chi=prob.chi, m=prob.m, theta=prob.theta,
              kappa=prob.kappa, force=prob.force, precision="fp32", kernel=mclb.KERNEL_FUSED)
    ts = torch.cuda.Stream()   # one stream for every slab handle, its copies and the events
    for edges in ("walls", "periodic"):
        for period in (1, 4):
            ls = slabs_mod.LocalSlabs(prob.nx, prob.ny, parts, period, stream=ts.cuda_stream,
                                      edges=edges, **kw)
            ls.init_fields(prob.rho, prob.u)
            t = time_steps(torch, ls, steps, warmup, ts)
            val = prob.sites * prob.ncomp * steps / t / 1e6
            band = ls.slabs[0].handle.rows_bytes(ls.slabs[0].G)
            key = f"slabs_{parts}_{prob.name}_fp32_period{period}" + (
                "" if edges == "walls" else "_periodic_edges")
            out[key] = {
                "value": val, "steps": steps, "status_ok": all(v == 0 for v in ls.status()),
                "edges": edges, "slab_rows": [s.h for s in ls.slabs],
                "outer_rows_per_side": ls.slabs[0].G, "band_bytes": band,
                "launches_per_slab_step": ls.slabs[0].handle.launches_per_step,
                "speedup_vs_fp32": val / fp32_value,
                "note": "MLUPS x N of the lattice's own sites; every slab also computes its "
                        "outer rows, and every period steps 2 bands per slab are packed and "
                        "unpacked (device copies on the same stream)"}
            ls.close()
    return out


def run_batched(torch, mclb, sptr, stream, warmup, fp32_value, steps=1000):
    """512 independent binary/ternary FP32 simulations of uneven size advanced together
    for the workload's 1000 steps (one batch handle, graph-replayed launches) against the
    same instances advanced one after another, each with its own handle on the plain FP32
    single-pass path.  Instances whose density turned non-finite are counted at the end
    (the recipe's chi range reaches past the method's stability limit for its strongest
    binaries); the rate is also given over the instances that stayed finite, and the
    two-phase fits of those are compared between the batch and the single handles."""
    import numpy as np
    from paper_0704_3444_gb300 import inputs
    probs = inputs.batch(512)
    work = sum(p.sites * p.ncomp for p in probs)
    warmup = max(warmup, 64)   # both graph parities captured before the timed steps
    b = mclb.Batch(probs, precision="fp32", stream=sptr)
    b.init_all()
    b.step(warmup)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    b.step(steps)
    stop.record(stream)
    torch.cuda.synchronize()
    tb = start.elapsed_time(stop) / 1e3
    per = b.status()[1]
    finite = [k for k, v in enumerate(per) if v == 0]
    launches = b.launches_per_step
    tuning = [{"narrow_strips": nar, "waves": w} for nar, w in b.tuning()]
    sims = [mclb.Simulation.from_problem(p, precision="fp32", kernel=mclb.KERNEL_FUSED, stream=sptr)
            for p in probs]
    for sm in sims:
        sm.step(warmup)
    torch.cuda.synchronize()
    start.record(stream)
    for sm in sims:
        sm.step(steps)
    stop.record(stream)
    torch.cuda.synchronize()
    ts = start.elapsed_time(stop) / 1e3
    finite_one = [k for k, sm in enumerate(sims) if sm.status() == 0]
    # two-phase bulk compositions of the instances that stayed finite and have separated
    # into two phases (fitted phases at least 0.3 apart in some component: below that the
    # two clusters only split the noise of a still mixed state), batch vs handles
    diffs = []
    for k in sorted(set(finite) & set(finite_one)):
        try:
            fb = b.fit_equilibrium(k, 2)
            fs = sims[k].fit_equilibrium(2)
        except mclb.MclbError:       # no bulk site (still mixing): nothing to compare
            continue
        if min(np.max(np.abs(fb[0] - fb[1])), np.max(np.abs(fs[0] - fs[1]))) < 0.3:
            continue
        diffs.append(float(np.max(np.abs(fb - fs))))
    b.close()
    for sm in sims:
        sm.close()
    work_finite = sum(probs[k].sites * probs[k].ncomp for k in finite)
    vb, vs = work * steps / tb / 1e6, work * steps / ts / 1e6
    return {"value": vb, "steps": steps, "instances": len(probs),
            "diverged": len(probs) - len(finite), "diverged_one_by_one": len(probs) - len(finite_one),
            "value_finite_instances": work_finite * steps / tb / 1e6,
            "diverged_note": "binary instances with chi >= ~1.39 x critical leave the method's "
                             "stability range at kappa = 0.01 (non-finite density) within the "
                             "1000 steps; the same work is timed either way",
            "fit_vs_one_by_one": {
                "instances": len(diffs),
                "within_1e-3": sum(d <= 1e-3 for d in diffs),
                "median_abs_diff": float(np.median(diffs)) if diffs else None,
                "max_abs_diff": max(diffs) if diffs else None,
                "note": "two-phase fits of the same instance from the batch and from its own "
                        "handle after 1000 steps; the two kernels differ in the last bit, and "
                        "instances still coarsening amplify that into a different arrangement "
                        "of domains, which the fit then measures"},
            "sites": sum(p.sites for p in probs), "launches_per_step": launches,
            "autotuned_partition": tuning,
            "one_by_one_fp32_value": vs, "speedup_vs_one_by_one": vb / vs,
            "speedup_vs_fp32": vb / fp32_value}


def run_lines(torch, mclb, sptr, stream, count=512, nx=1024, steps=4096, precision="fp64"):
    """The paper's own lattice as its sweeps use it: `count` independent D1Q3 lines of `nx`
    sites (binary, chi = 2.2, 1/tau = 0.9, kappa = 0, the Sec. 4 sinusoid of amplitude 0.1),
    advanced together -- each line lives in one CTA's shared memory for the whole
    4096-step launch, so the populations cross HBM once per launch, not once per step."""
    import numpy as np
    from paper_0704_3444_gb300 import inputs
    x = np.arange(nx)
    probs = []
    for k in range(count):
        phi = 0.5 + 0.1 * np.sin(2 * np.pi * (x + 7 * k) / nx)
        probs.append(inputs.Problem(
            name=f"line{k}", ncomp=2, nx=nx, ny=1, tau=1 / 0.9, chi=inputs.uniform_chi(2, 2.2),
            m=np.ones(2), theta=1 / 3, kappa=0.0, force=(0.0, 0.0),
            rho=np.stack([phi, 1 - phi])[:, None, :], u=np.zeros((2, 1, nx)), lattice="d1q3"))
    b = mclb.Batch(probs, precision=precision, stream=sptr)
    b.init_all()
    b.step(steps)                              # warm-up: one full resident launch
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    b.step(steps)
    stop.record(stream)
    torch.cuda.synchronize()
    t = start.elapsed_time(stop) / 1e3
    rc, per = b.status()
    out = {"value": count * nx * 2 * steps / t / 1e6, "steps": steps, "lines": count, "sites": nx,
           "precision": precision,
           "launches_per_step_chunk": b.launches_per_step, "status_ok": rc == 0,
           "note": f"MLUPS x N of {count} D1Q3 lines advanced {steps} steps by one resident "
                   "launch (one CTA per line, the line in shared memory): bound by the "
                   "per-site arithmetic (FP64 runs at a small fraction of the FP32 rate on "
                   "this GPU), not by HBM"}
    b.close()
    return out


def run_cpu_baseline(prob, budget_s=15.0):
    """The FP64 oracle as it stands, on this host's cores, on a bounded number of
    timesteps of the same workload."""
    import oracle
    from oracle import Oracle
    o = Oracle.from_problem(prob)
    t0 = time.perf_counter()
    o.run(1)
    t1 = time.perf_counter() - t0
    k = max(1, min(50, int(budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    o.run(k)
    dt = time.perf_counter() - t0
    v = prob.sites * prob.ncomp * k / dt / 1e6
    return {"value": v, "unit": UNIT, "cores": oracle.nthreads(), "kind": "oracle",
            "sample": f"{k} FP64 oracle timesteps of the full {prob.nx}x{prob.ny} N={prob.ncomp} "
                      f"lattice ({dt:.1f} s)"}


def run_reference(args, world, rank):
    """--impl reference: the FP64 oracle, as it stands, on host cores.  Each step is one
    timestep of a bounded sample of the workload (a periodic band of rows of the same
    lattice, same parameters), sized so that warm-up plus timed steps take a few minutes."""
    if rank != 0:
        return
    import oracle
    from oracle import Oracle
    from paper_0704_3444_gb300 import inputs
    prob = workloads()[args.workload]()
    # calibrate the per-site cost on a 64-row band
    rows = min(prob.ny, 64)
    band = lambda r: inputs.Problem(
        name=prob.name, ncomp=prob.ncomp, nx=prob.nx, ny=r, tau=prob.tau, chi=prob.chi, m=prob.m,
        theta=prob.theta, kappa=prob.kappa, force=prob.force, walls=prob.walls,
        rho=prob.rho[:, :r].copy(), u=prob.u[:, :r].copy())
    o = Oracle.from_problem(band(rows))
    t0 = time.perf_counter()
    o.run(1)
    per_site = (time.perf_counter() - t0) / (prob.nx * rows)
    budget = 150.0 / max(1, args.steps + args.warmup)
    rows = int(max(3, min(prob.ny, budget / max(per_site * prob.nx, 1e-9))))
    sample = band(rows)
    o = Oracle.from_problem(sample)
    o.run(args.warmup)
    t0 = time.perf_counter()
    o.run(args.steps)
    dt = time.perf_counter() - t0
    value = sample.sites * sample.ncomp * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "nx": prob.nx, "ny": prob.ny,
                                        "ncomp": prob.ncomp},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.nthreads(),
                         "kind": "oracle",
                         "sample": f"each step one FP64 oracle timestep of a {prob.nx}x{rows} "
                                   f"periodic band of the {prob.nx}x{prob.ny} N={prob.ncomp} "
                                   "workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="mclb", choices=["mclb", "reference"])
    ap.add_argument("--workload", default="n5_2048x2048")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16", "fp64"])
    ap.add_argument("--kernel", default="fused", choices=["fused", "staged"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-batch", action="store_true",
                    help="run only the 512-instance batch variant and print its record")
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--only-lines", action="store_true",
                    help="run only the D1Q3 lines variant (512 lines x 1024 sites, --precision "
                         "fp32 or fp64, --lines-steps steps per resident launch) and print it")
    ap.add_argument("--lines-steps", type=int, default=4096)
    ap.add_argument("--only-slabs", action="store_true",
                    help="run only the slab-decomposition variant of the workload (two slabs "
                         "on this GPU) and print its record")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import paper_0704_3444_gb300 as mclb

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    mclb.load()
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    if args.only_batch:
        print(json.dumps(run_batched(torch, mclb, sptr, stream, args.warmup, float("nan"),
                                     args.batch_steps)), flush=True)
        return
    if args.only_lines:
        print(json.dumps(run_lines(torch, mclb, sptr, stream, steps=args.lines_steps,
                                   precision=args.precision)), flush=True)
        return
    prob = workloads()[args.workload]()
    N, S = prob.ncomp, prob.sites
    if args.only_slabs:
        print(json.dumps(run_slabs(torch, mclb, prob, args.warmup, float("nan"))),
              flush=True)
        return

    kern = mclb.KERNEL_FUSED if args.kernel == "fused" else mclb.KERNEL_STAGED
    sim = mclb.Simulation.from_problem(prob, precision=args.precision, kernel=kern, stream=sptr)
    launches = sim.launches_per_step
    bytes_step = sim.bytes_per_step
    # the clock sampler covers the warm-up, the timed steps, the end-to-end job and the
    # variants: the timed region alone can be shorter than one sampling interval
    clk = ClockSampler(gpu_index(local_rank))
    clk.__enter__()
    sim.step(args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    sim.step(args.steps)
    stop.record(stream)
    torch.cuda.synchronize()
    elapsed = start.elapsed_time(stop) / 1e3
    value, elapsed = job_rate(torch, dist, S * N * args.steps, elapsed, world, "cuda")
    status = sim.status()
    if status != 0:
        raise SystemExit(f"device status {status} after the timed steps")
    per_launch = elapsed / args.steps
    peak, peak_src = hbm_peak()
    achieved = bytes_step / per_launch / 1e9
    traffic = profiled_traffic() if args.precision == "fp32" and args.workload == "n5_2048x2048" else None

    # end to end through the C ABI with host buffers, one job of the workload's horizon
    # (2000 steps for the N = 5 workload, or --steps if longer): the initial fields from
    # pinned memory to the device, every step's status word back (mclb_step returns the
    # previous step's), and the final rho and U fields to the host
    e2e = None
    if not args.no_e2e:
        job = max(args.steps, int(prob.steps or 0))
        rho_h = torch.from_numpy(prob.rho).pin_memory().numpy()
        u_h = torch.from_numpy(prob.u).pin_memory().numpy()
        out_rho = torch.empty(prob.rho.shape, dtype=torch.float64).pin_memory().numpy()
        out_u = torch.empty(prob.u.shape, dtype=torch.float64).pin_memory().numpy()
        sim2 = mclb.Simulation(N, prob.nx, prob.ny, prob.tau, prob.chi, prob.m, prob.theta,
                               prob.kappa, prob.force, args.precision, kern, sptr,
                               lattice=prob.lattice, nz=prob.nz, walls=prob.walls)
        sim2.init_fields(rho_h, u_h)
        sim2.step(args.warmup)
        sim2.status()
        t0 = time.perf_counter()
        sim2.init_fields(rho_h, u_h)
        for _ in range(job):
            sim2.step(1)
        rc = sim2.lib.mclb_moments(sim2.h, mclb._dp(out_rho), mclb._dp(out_u), None, None)
        rc2 = sim2.status()
        t_e2e = time.perf_counter() - t0
        sim2.close()
        if rc == 0 and rc2 == 0:
            h2d = prob.rho.nbytes + prob.u.nbytes
            d2h = out_rho.nbytes + out_u.nbytes
            e2e = {"value": S * N * job / t_e2e / 1e6 * world, "unit": UNIT,
                   "h2d_bytes_per_step": h2d / job, "d2h_bytes_per_step": 4 + d2h / job,
                   "job_steps": job,
                   "note": "one job: upload of the initial fields, one mclb_step(1) call per "
                           "step (each returns the previous step's 4-byte status word), "
                           "download of rho and U; bytes per step are the job's copies / steps"}

    variants = {}
    if not args.no_variants and rank == 0 and args.precision == "fp32":
        ks = 500
        for prec in ("bf16", "fp16"):
            v = mclb.Simulation.from_problem(prob, precision=prec, kernel=mclb.KERNEL_FUSED,
                                             stream=sptr)
            t = time_steps(torch, v, ks, args.warmup, stream)
            ok = v.status() == 0
            variants[f"{prec}_shifted"] = {
                "value": S * N * ks / t / 1e6, "steps": ks, "status_ok": ok,
                "speedup_vs_fp32": (S * N * ks / t / 1e6) / (value / world),
                "hbm_gbs_algorithmic": v.bytes_per_step / (t / ks) / 1e9}
            v.close()
            # the same with the per-component mass compensation after every 64 steps
            v = mclb.Simulation.from_problem(prob, precision=prec, kernel=mclb.KERNEL_FUSED,
                                             stream=sptr, mass_every=64)
            t = time_steps(torch, v, 512, 64, stream)
            variants[f"{prec}_shifted"]["mass_every_64"] = {
                "value": S * N * 512 / t / 1e6, "steps": 512, "status_ok": v.status() == 0,
                "speedup_vs_fp32": (S * N * 512 / t / 1e6) / (value / world)}
            v.close()
        v = mclb.Simulation.from_problem(prob, precision="fp32", kernel=mclb.KERNEL_STAGED,
                                         stream=sptr)
        t = time_steps(torch, v, 200, args.warmup, stream)
        variants["fp32_staged_3_launches"] = {
            "value": S * N * 200 / t / 1e6, "steps": 200,
            "speedup_vs_fp32": (S * N * 200 / t / 1e6) / (value / world)}
        v.close()
        # the 8192 x 2048 ternary slab (polymer / solvent against non-solvent) in FP32 and
        # in BF16-shifted storage
        slab = workloads()["slab_8192x2048"]()
        slab_fp32 = None
        for prec in ("fp32", "bf16"):
            v = mclb.Simulation.from_problem(slab, precision=prec, kernel=mclb.KERNEL_FUSED,
                                             stream=sptr)
            t = time_steps(torch, v, 200, args.warmup, stream)
            val = slab.sites * slab.ncomp * 200 / t / 1e6
            slab_fp32 = val if prec == "fp32" else slab_fp32
            variants[f"slab_8192x2048_{prec}"] = {
                "value": val, "steps": 200, "status_ok": v.status() == 0,
                "hbm_gbs_algorithmic": v.bytes_per_step / (t / 200) / 1e9,
                "hbm_frac_of_measured": v.bytes_per_step / (t / 200) / 1e9 / peak,
                "speedup_vs_fp32": val / slab_fp32}
            v.close()
        # the same slab between solid walls in y, FP32: the single pass with the rows next
        # to the walls redone by the wall-aware staged launches, and the staged schedule
        slab.walls = 1
        for kern_w, key in ((mclb.KERNEL_FUSED, "slab_8192x2048_fp32_walls"),
                            (mclb.KERNEL_STAGED, "slab_8192x2048_fp32_walls_staged")):
            v = mclb.Simulation.from_problem(slab, precision="fp32", kernel=kern_w, stream=sptr)
            t = time_steps(torch, v, 100, args.warmup, stream)
            val = slab.sites * slab.ncomp * 100 / t / 1e6
            variants[key] = {
                "value": val, "steps": 100, "status_ok": v.status() == 0,
                "launches_per_step": v.launches_per_step,
                "hbm_gbs_algorithmic": v.bytes_per_step / (t / 100) / 1e9,
                "hbm_frac_of_measured": v.bytes_per_step / (t / 100) / 1e9 / peak,
                "speedup_vs_fp32": val / slab_fp32}
            v.close()
        # the periodic slab under the Gibbs-Duhem force reading (kappa = 0), FP32: the
        # single pass with its total-density gradient, and the staged schedule
        slab.walls = 0
        slab.kappa = 0.0
        slab.force_form = 1
        for kern_g, key in ((mclb.KERNEL_FUSED, "slab_8192x2048_fp32_gibbs_duhem"),
                            (mclb.KERNEL_STAGED, "slab_8192x2048_fp32_gibbs_duhem_staged")):
            v = mclb.Simulation.from_problem(slab, precision="fp32", kernel=kern_g, stream=sptr)
            t = time_steps(torch, v, 100, args.warmup, stream)
            val = slab.sites * slab.ncomp * 100 / t / 1e6
            variants[key] = {
                "value": val, "steps": 100, "status_ok": v.status() == 0,
                "launches_per_step": v.launches_per_step,
                "hbm_frac_of_measured": v.bytes_per_step / (t / 100) / 1e9 / peak,
                "speedup_vs_fp32": val / slab_fp32}
            v.close()
        # the D3Q19 lattice: the paper's ternary chi set on 256^3 in FP32, the density pass
        # + z-plane march and the staged schedule
        cube = workloads()["ternary3d_256"]()
        for kern_c, key, what in (
                (mclb.KERNEL_FUSED, "d3q19_ternary3d_256_fp32",
                 "two launches (density pass, z-plane march with the potentials on chip)"),
                (mclb.KERNEL_STAGED, "d3q19_ternary3d_256_fp32_staged",
                 "three launches (density, potential, collision)")):
            v = mclb.Simulation.from_problem(cube, precision="fp32", kernel=kern_c, stream=sptr)
            t = time_steps(torch, v, 50, args.warmup, stream)
            val = cube.sites * cube.ncomp * 50 / t / 1e6
            variants[key] = {
                "value": val, "steps": 50, "status_ok": v.status() == 0,
                "launches_per_step": v.launches_per_step,
                "hbm_gbs_algorithmic": v.bytes_per_step / (t / 50) / 1e9,
                "hbm_frac_of_measured": v.bytes_per_step / (t / 50) / 1e9 / peak,
                "note": "152 B per site and component (19 loads + 19 stores of f in FP32) per "
                        "step; " + what}
            v.close()
        for prec in ("fp64", "fp32"):
            variants[f"d1q3_lines_512x1024_{prec}"] = run_lines(torch, mclb, sptr, stream,
                                                                precision=prec)
        variants.update(run_slabs(torch, mclb, prob, args.warmup, value / world))
        variants["batched_512"] = run_batched(torch, mclb, sptr, stream, args.warmup, value / world)
    clk.__exit__()
    clocks = clk.summary()
    clocks["window"] = ("nvidia-smi every 20 ms from the warm-up of the timed steps through "
                        "the end-to-end job and the variants; samples at >= 50 % utilisation")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        del sim
        torch.cuda.synchronize()
        cpu = run_cpu_baseline(prob)

    d3 = getattr(prob, "lattice", "d2q9") == "d3q19"
    walls = getattr(prob, "walls", 0)
    if args.kernel == "staged":
        schedule, timed = "staged, 3 launches", "the three staged kernels"
    elif d3:
        schedule, timed = ("density pass + z-plane march, 2 launches",
                           "k19_density + k19_march (the march about 3/4 of it)")
    elif walls:
        schedule, timed = ("fused single pass + the rows next to the walls by 3 staged launches",
                           "k_march, the ghost-column refresh and the wall-row launches (about "
                           "5 % of it)")
    else:
        schedule, timed = ("fused single pass",
                           "k_march plus the ghost-column refresh, about 3 % of it")
    per = bytes_step / (S * N)
    config = {"workload": args.workload, "nx": prob.nx, "ny": prob.ny, "ncomp": N,
              "precision": args.precision, "schedule": schedule,
              "l2": "distributions (2 x %.0f MB) exceed the 129 MB L2; no flush" %
                    (bytes_step / 2 / 1e6)}
    if d3:
        config["nz"] = prob.nz
    if walls:
        config["walls"] = walls
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "bf16-storage/f32", "fp16": "f16-storage/f32"}[args.precision],
        "data": "synthetic",
        "config": config,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "note": f"{per:.0f} B per site and component (every stored value read once "
                             f"and written once) x sites x N / CUDA-event time per step ({timed}); "
                             f"peak = {peak_src} copy bandwidth; traffic = ncu dram bytes per "
                             f"k_march launch from profiles/ (the FP32 N = 5 2048^2 workload only)"},
        "mlups": world * S * args.steps / elapsed / 1e6,
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "variants": variants,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
