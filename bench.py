#!/usr/bin/env python
"""Benchmark: fine-level DOF-sweeps/s of SI-MLSDC time steps on GB300.

Workload (default, the largest single-GPU configuration): an ensemble of 512
independent 2D convection-diffusion problems on the periodic unit square
(element grids 8^2..48^2, fine degree 3..8, coarse degree ceil(P/2),
Radau-Right 5/3 collocation nodes, SI(2), Cascade start, 3 V-cycles + final
fine post-sweep per step, dt from CFL 0.5 per instance; 21.7 M fine nodes),
all instances of one degree in one persistent launch per sweep, one step as
one CUDA graph.  One "step" = one time step of every instance through the C
ABI (sisdc_ens_step): every row of the hot path runs in it.

Other workloads (--workload): burgers2d, euler_vortex, euler256 (the vortex
on 256^2 elements), ns_shear, convdiff1d (sisdc_step), stability_map,
mlp_ns_level, paper_convdiff (the Sec. 8 convection-diffusion studies),
burgers_front and sod (the Sec. 8 shock-capturing studies with artificial
viscosity).

Output: one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores instead (bounded samples of the same workload).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fine-level DOF-sweeps/s"
UNIT = "DOF-sweeps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sisdc", choices=["sisdc", "reference"])
    ap.add_argument("--workload", default="ensemble512")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--cg-rtol", type=float, default=1e-12)
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small", action="store_true", help="8x8 elements (profiling case)")
    ap.add_argument("--ninst", type=int, default=0, help="ensemble: first N instances only (profiling case)")
    ap.add_argument("--no-autotune", action="store_true", help="default tile shapes (no sisdc_autotune)")
    ap.add_argument("--capped", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--per-instance", type=int, default=0,
                    help="ensemble: also time this many sampled instances stepped one by one (single-problem path)")
    ap.add_argument("--no-forms", action="store_true", help="skip the other precision forms")
    ap.add_argument("--learned", action="store_true",
                    help="train the element-patch network on logged solves and time the learned initial guess")
    ap.add_argument("--learn-solves", type=int, default=10000, help="--learned: logged solves to train on")
    ap.add_argument("--learn-chunk", type=int, default=400, help="--learned: solves logged per training epoch")
    ap.add_argument("--part", default="all", choices=["all", "table", "study"],
                    help="paper_convdiff: the error table, the CFL iteration study, or both")
    ap.add_argument("--cfls", type=float, nargs="*", default=[64, 32, 16, 8, 4, 2, 1],
                    help="paper_convdiff: CFL numbers of the iteration study")
    ap.add_argument("--nus", type=float, nargs="*", default=None,
                    help="paper_convdiff study: the viscosities to run (1e-3 and/or 0; default both)")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-nel", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--shard", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--nshards", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--seconds", type=float, default=10.0, help=argparse.SUPPRESS)
    return ap.parse_args()


def workload(args):
    from paper_2504_18526_gb300 import inputs
    nel = (8, 8) if args.small else None
    if getattr(args, "oracle_nel", 0):
        nel = (args.oracle_nel, args.oracle_nel)
    return inputs.scaled(args.workload, nel=nel)


# the largest fine level (DOFs) on which the CPU baseline times one full
# oracle step; bigger workloads are sampled on a coarser element grid of the
# same physics and levels (the oracle's cost per DOF does not depend on the
# number of elements)
ORACLE_MAX_DOFS = 1_100_000


def fine_dofs(w):
    lv = w["levels"][-1]
    nq = lv["P"] + 1
    n = lv["nel"][0] * (lv["nel"][1] if w["dim"] == 2 else 1) * nq ** w["dim"]
    return n * w["ncomp"]


def initial_data(w, X, Y):
    from paper_2504_18526_gb300 import inputs
    name = [k for k, v in inputs.WORKLOADS.items() if v["id"] == w["id"]][0]
    u0 = inputs.initial_state(name, X, Y)
    lv = w["levels"][-1]
    h = (w["hi"][0] - w["lo"][0]) / lv["nel"][0]
    if "cfl" in w:
        dt = inputs.cfl_dt(w["cfl"], h, lv["P"], inputs.max_wave_speed(w["pde"], u0, w.get("gamma", 1.4),
                                                                          w.get("adv", (1, 0))))
    else:
        dt = w["dt"]
    return u0, dt


# ---------------------------------------------------------------------------
# clocks sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# oracle sample (run in a single-threaded child process)
# ---------------------------------------------------------------------------
def oracle_sample(args):
    import numpy as np
    from tests.helpers import oracle_ml
    w = workload(args)
    om = oracle_ml(w, rtol=args.cg_rtol)
    sp = om.levels[-1].space
    X, Y = sp.coords()
    u0, dt = initial_data(w, X, Y)
    ncyc = w["ncycles"]
    reps = max(1, args.steps)
    t0 = time.perf_counter()
    u = u0
    for _ in range(reps):
        u = om.step(u, dt, ncyc, start=w["start"])
    el = time.perf_counter() - t0
    sweeps = ncyc + 1
    print(json.dumps({"seconds": el, "steps": reps, "dof_sweeps": fine_dofs(w) * sweeps * reps,
                      "finite": bool(np.all(np.isfinite(u)))}))


def ensemble_oracle_sample(args):
    """One oracle time step of ensemble instances, smallest first, this
    shard's share of them (instances shard, shard + nshards, ...), until
    `seconds` have passed (at least one instance)."""
    import numpy as np
    from paper_2504_18526_gb300 import inputs
    from oracle.dg import ConvDiff, DGSpace
    from oracle.mlsdc import MLSDC
    from oracle.sdc import Level
    w = inputs.WORKLOADS["ensemble512"]
    insts = inputs.ensemble_instances(w["ninst"])
    order = list(np.argsort([d["nel"][0] * d["nel"][1] * (d["P"] + 1) ** 2 for d in insts], kind="stable"))
    order = order[args.shard::max(1, args.nshards)]
    t0 = time.perf_counter()
    dofs = 0
    k = 0
    while k < len(order) and (k < 1 or time.perf_counter() - t0 < args.seconds):
        d = insts[order[k]]
        sp = lambda P: DGSpace(2, d["nel"], P, (0.0, 0.0), (1.0, 1.0), ConvDiff(d["adv"], d["nu"]),
                               cg_rtol=args.cg_rtol, cg_maxit=1000)
        fine = sp(d["P"])
        ml = MLSDC([Level(sp((d["P"] + 1) // 2), w["nodes"], w["Mc"]), Level(fine, w["nodes"], w["M"])], stages=2, Nc=2)
        X, Y = fine.coords()
        ml.step(inputs.ensemble_exact(d, X, Y, 0.0), d["dt"], w["ncycles"], start=w["start"])
        dofs += X.size * (w["ncycles"] + 1)
        k += 1
    print(json.dumps({"seconds": time.perf_counter() - t0, "steps": 1, "instances": k, "dof_sweeps": dofs,
                      "finite": True}))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def ensemble_oracle_run(args, nshards, seconds):
    """The oracle on `nshards` single-threaded processes at once, each on its
    share of the instances for about `seconds`; DOF-sweeps/s over the wall
    time of the slowest shard."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    procs = []
    for sh in range(nshards):
        cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", "--workload", "ensemble512",
               "--cg-rtol", str(args.cg_rtol), "--shard", str(sh), "--nshards", str(nshards),
               "--seconds", str(seconds)]
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env,
                                      cwd=ROOT))
    res = []
    for p in procs:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("oracle shard failed: " + err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    wall = max(r["seconds"] for r in res)
    dofs = sum(r["dof_sweeps"] for r in res)
    return {"value": dofs / wall, "seconds": wall, "instances": sum(r["instances"] for r in res),
            "dof_sweeps": dofs}


def cpu_baseline_ensemble(args):
    """The oracle as it stands on every host core (one process per core, each
    on its share of the instances), and on one core."""
    try:
        n = host_cores()
        allc = ensemble_oracle_run(args, n, 10.0)
        one = ensemble_oracle_run(args, 1, 10.0)
        return {"value": allc["value"], "unit": UNIT, "cores": n, "kind": "oracle",
                "sample": "one FP64 numpy oracle time step of %d ensemble instances (smallest first, "
                          "spread over %d single-threaded processes), %.1f s wall" %
                          (allc["instances"], n, allc["seconds"]),
                "cpu": cpu_model(),
                "single_thread": {"value": one["value"], "cores": 1,
                                  "sample": "%d instances, smallest first, %.1f s" % (one["instances"],
                                                                                       one["seconds"])}}
    except Exception as e:   # reported, not fatal
        return {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": "failed: %s" % e}


def mlp_oracle_sample(args):
    """FP64 numpy loss and gradients of the oracle MLP (325 -> 112 -> 112 -> 36)
    over 4096 patch rows, repeated for about 10 s."""
    import numpy as np
    from oracle import mlp as omlp
    rows, n_in, H, q = 4096, 9 * 36 + 1, 112, 36
    rng = np.random.default_rng(3)
    p = omlp.init_params(n_in, H, q, 1)
    X = rng.standard_normal((rows, n_in))
    T = rng.standard_normal((rows, q))
    t0 = time.perf_counter()
    reps = 0
    while reps == 0 or time.perf_counter() - t0 < 10.0:
        omlp.loss_and_grads(p, X, T)
        reps += 1
    print(json.dumps({"seconds": time.perf_counter() - t0, "rows": rows * reps, "passes": reps}))


def oracle_nel_for(args):
    """0 = the workload's own grid, else the elements per side of the sample."""
    if args.small or args.workload in ("ensemble512", "mlp_ns_level", "stability_map"):
        return 0
    w = workload(args)
    n = fine_dofs(w)
    nel = w["levels"][-1]["nel"][0]
    while n > ORACLE_MAX_DOFS and nel % 2 == 0:
        nel //= 2
        n //= 4
    return 0 if nel == w["levels"][-1]["nel"][0] else nel


def run_oracle_child(args, steps, nel=0):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", "--steps", str(steps),
           "--workload", args.workload, "--cg-rtol", str(args.cg_rtol)] + (["--small"] if args.small else [])
    if nel:
        cmd += ["--oracle-nel", str(nel)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# ---------------------------------------------------------------------------
def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "ensemble512":
        return reference_arm_ensemble(args)
    w = workload(args)
    onel = oracle_nel_for(args)
    for _ in range(args.warmup):
        run_oracle_child(args, 1, onel)
    tot_s, tot_d = 0.0, 0
    for _ in range(args.steps):
        r = run_oracle_child(args, 1, onel)
        tot_s += r["seconds"]
        tot_d += r["dof_sweeps"]
    v = tot_d / tot_s
    sample = "%d oracle time steps (1 per bench step) of the %s workload%s, FP64 numpy, 1 thread" % (
        args.steps, args.workload, " on %d^2 elements (same physics, degrees and nodes)" % onel if onel else "")
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": args.workload, "fine_dofs": fine_dofs(w), "levels": w["levels"],
                      "fine_sweeps_per_step": w["ncycles"] + 1},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                            "cpu": cpu_model()},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def reference_arm_ensemble(args):
    """The oracle as it stands on every host core: each bench step is one
    bounded sample (about 3 s of wall time) of ensemble instances, one oracle
    time step each, spread over one single-threaded process per core."""
    from paper_2504_18526_gb300 import inputs
    w = inputs.WORKLOADS["ensemble512"]
    n = host_cores()
    for _ in range(args.warmup):
        ensemble_oracle_run(args, n, 1.0)
    tot_s, tot_d, tot_i = 0.0, 0, 0
    for _ in range(args.steps):
        r = ensemble_oracle_run(args, n, 3.0)
        tot_s += r["seconds"]
        tot_d += r["dof_sweeps"]
        tot_i += r["instances"]
    v = tot_d / tot_s
    sample = ("%d samples (1 per bench step) of about 3 s: one FP64 numpy oracle time step of each of %d "
              "ensemble instances in all (smallest first), %d single-threaded processes" % (args.steps, tot_i, n))
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": "ensemble512", "instances": w["ninst"],
                      "fine_sweeps_per_step": w["ncycles"] + 1},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": n, "kind": "oracle", "sample": sample,
                            "cpu": cpu_model()},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Algorithmic work of one correction-sweep launch (per fine DOF), from the
# per-unit operation counts of the path: an SIPG operator application costs
# 8(P+1) + 20 flop (the element's two (P+1)-term stiffness sums and the face
# derivatives and jumps of its four faces), a CG iteration adds 10 flop of
# vector updates, a right-hand side 12 flop, and the S.F quadrature 2M flop
# per collocation node.  A convective-operator application costs per node
# (all components) 4(P+1) flop per component for the two derivative sums,
# the flux evaluation, and the Rusanov face flux on the 4(P+1) face nodes of
# each (P+1)^2-node element; for Navier-Stokes also the BR1 viscous term
# (lifted gradients of three primitive variables and the divergence of
# three viscous-flux components: 24(P+1) + 40).  Per node of an SI(2)
# correction sweep: one SIPG application per CG iteration, one for the
# stage-2 start residual and one for the cached L u; two convective
# applications.
FLUX_FLOPS = {"convdiff": (2, 8), "burgers": (4, 20), "euler": (24, 60), "ns": (24, 60)}   # node, face node


def conv_flops_per_dof(P, ncomp, pde):
    f, r = FLUX_FLOPS[pde]
    node = ncomp * 4 * (P + 1) + f + 4.0 * r / (P + 1)
    if pde == "ns":
        node += 24 * (P + 1) + 40
    return node / ncomp


def sweep_flops(P, ncomp, M, nsweeps, iters, nv, pde="convdiff"):
    mv = 8 * (P + 1) + 20
    cv = conv_flops_per_dof(P, ncomp, pde)
    per_node = 2 * mv + 2 * cv + 2 * 12 + 2 * M
    return float(nv) * (nsweeps * M * per_node + iters * (mv + 10))


FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # SMs x DFMA/clk/SM x 2 flop x max clock


# Algorithmic memory traffic of one correction-sweep launch if no array
# stayed on chip (the HBM view of the roofline): per collocation node and
# DOF, 11 state-sized FP64 arrays (old and previous-node iterate, f, c and
# L u caches, S.F, FAS g; new iterate, f, c, L u) plus 4 per implicit solve
# of the two SI(2) stages (right-hand side terms, r, z); per CG iteration
# 11 (r, z, p_old, p, Ap, x read or written).
def sweep_bytes(M, nsweeps, iters, nv):
    return 8.0 * nv * (nsweeps * M * (11 + 2 * 4) + iters * 11)

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one
# fine-level correction-sweep launch, from an ncu capture of that launch, per
# (workload, form), with the digest of the kernel sources it was measured on;
# reported as null for any other kernel version.
SWEEP_TRAFFIC_BYTES = {}
SWEEP_KERNEL_SOURCES = ("sweep.cuh", "sipg.cuh", "pde.cuh", "common.cuh", "ds.cuh", "inputs.py")


# ---------------------------------------------------------------------------
# replicas (one process per GPU, no data-path collective): timing bookkeeping
# ---------------------------------------------------------------------------
def max_over_ranks(ms, dist=None, device=None):
    """The largest per-rank time (ms) of the timed region; identity on one rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_step_per_rank, steps, world, ms):
    """Units processed by all ranks per second (weak scaling: fixed work per rank)."""
    return world * units_per_step_per_rank * steps / (ms * 1e-3)


def sweep_traffic(args):
    rec = SWEEP_TRAFFIC_BYTES.get((args.workload, args.precision))
    if args.small or not rec or rec[1] != kernel_digest(SWEEP_KERNEL_SOURCES):
        return None
    return rec[0]


def make_ctx(S, w, stream, prec, rtol, use_graph, mixed_levels=0):
    return S.Context(w, stream=stream.cuda_stream, precision=prec, cg_rtol=rtol, cg_maxit=1000,
                     use_graph=use_graph, mixed_levels=mixed_levels)


def tune(S, args, ctx, du, dt, nlevels):
    """Tile shapes from the library's autotuner (setup, outside every timed region)."""
    if args.no_autotune:
        return [list(S.sisdc_level_config(lv)) for lv in ctx.levels]
    return S.sisdc_autotune(ctx.ctx, du, dt, nlevels).tolist()


def run_steps(S, ctx, du, dt, ncyc, start, nsteps):
    for _ in range(nsteps):
        S.sisdc_step(ctx.ctx, du, 0.0, dt, ncyc, start, 1)


def main_arm(args):
    import numpy as np
    import torch
    from paper_2504_18526_gb300 import sisdc as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0 or world == 1:
        from paper_2504_18526_gb300.build import build
        build()
    if dist:
        dist.barrier()
    S.load()

    w = workload(args)
    prec = S.SISDC_MIXED if args.precision == "mixed" else S.SISDC_FP64
    other = S.SISDC_FP64 if prec == S.SISDC_MIXED else S.SISDC_MIXED
    stream = torch.cuda.Stream(device=dev)
    use_graph = 0 if args.no_graph else 1
    ctx = make_ctx(S, w, stream, prec, args.cg_rtol, use_graph)
    nc, n, M = ctx.info(-1)
    hx, hy = np.zeros(n), np.zeros(n)
    S.sisdc_level_coords(ctx.levels[-1], hx, hy)
    lv = w["levels"][-1]
    shp = (lv["nel"][1] if w["dim"] == 2 else 1, lv["nel"][0], lv["P"] + 1 if w["dim"] == 2 else 1, lv["P"] + 1)
    u0, dt = initial_data(w, hx.reshape(shp), hy.reshape(shp))
    start = S.START_IDS[w["start"]]
    ncyc = w["ncycles"]
    nv = nc * n
    dofs_per_step = nv * (ncyc + 1)
    du = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2
    torch.cuda.synchronize()
    nlev = len(w["levels"])
    tiles = tune(S, args, ctx, du, dt, nlev)

    run_steps(S, ctx, du, dt, ncyc, start, args.warmup)
    S.sisdc_sync(ctx.ctx)
    S.sisdc_reset_stats(ctx.ctx)

    # ---- timed region: K steps, L2 flushed between steps -------------------
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        evs[k][0].record(stream)
        S.sisdc_step(ctx.ctx, du, 0.0, dt, ncyc, start, 1)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    S.sisdc_sync(ctx.ctx)
    ms = sum(a.elapsed_time(b) for a, b in evs)
    stats = S.sisdc_get_stats(ctx.ctx)
    ms = max_over_ranks(ms, dist, dev)
    value = whole_job_value(dofs_per_step, args.steps, world, ms)

    # ---- e2e: host buffers through the C ABI, copies inside the timed region --
    h_in = torch.from_numpy(np.ascontiguousarray(u0)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_e2e = torch.empty_like(du)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ke = max(3, args.steps // 2)
    torch.cuda.synchronize()
    t_e2e = 0.0
    for k in range(ke):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        e0.record(stream)
        with torch.cuda.stream(stream):
            d_e2e.copy_(h_in, non_blocking=True)
        S.sisdc_step(ctx.ctx, d_e2e, 0.0, dt, ncyc, start, 1)
        with torch.cuda.stream(stream):
            h_out.copy_(d_e2e, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        t_e2e += e0.elapsed_time(e1)
    S.sisdc_sync(ctx.ctx)
    e2e_val = world * dofs_per_step * ke / (t_e2e * 1e-3)
    ctx.close()

    # ---- dominant kernel: live CUDA-event timing of the fine-level sweeps ----
    kctx = make_ctx(S, w, stream, prec, args.cg_rtol, 0)
    dk = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
    tune(S, args, kctx, dk, dt, nlev)
    run_steps(S, kctx, dk, dt, ncyc, start, 2)
    S.sisdc_sync(kctx.ctx)
    S.sisdc_reset_stats(kctx.ctx)
    S.sisdc_set_kernel_timing(kctx.ctx, True, len(w["levels"]) - 1)
    t0 = time.perf_counter()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        S.sisdc_step(kctx.ctx, dk, 0.0, dt, ncyc, start, 1)
    kt = S.sisdc_get_kernel_timing(kctx.ctx)
    eager_s = time.perf_counter() - t0
    kstats = S.sisdc_get_stats(kctx.ctx)
    S.sisdc_sync(kctx.ctx)
    kctx.close()
    launches_per_step = kstats["launches"] / args.steps
    nsw = kt["dof_sweeps"] / max(1, nv)
    flops = sweep_flops(lv["P"], nc, M, nsw / max(1, kt["launches"]), kt["iters"] / max(1, kt["launches"]), nv,
                        w["pde"])
    avg_ms = kt["ms"] / max(1, kt["launches"])
    achieved = flops / (avg_ms * 1e-3) / 1e12
    hbm_peak, hbm_kind = measured_peaks()
    nbytes = sweep_bytes(M, nsw / max(1, kt["launches"]), kt["iters"] / max(1, kt["launches"]), nv)
    hbm_gbs = nbytes / (avg_ms * 1e-3) / 1e9

    # ---- the other precision form and time-to-solution at equal L2 error ----
    forms, tts = {}, None
    if not args.no_forms:
        win = max(4, min(20, args.steps))
        ref_ctx = make_ctx(S, w, stream, S.SISDC_FP64, min(args.cg_rtol, 1e-13), 1)
        ur = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
        torch.cuda.synchronize()
        run_steps(S, ref_ctx, ur, dt / 4, 6, start, 4 * win)
        S.sisdc_sync(ref_ctx.ctx)
        ref_ctx.close()
        # mixed form on every level, and on the finest level only (the coarse
        # level's sweeps are barrier-latency bound, where FP64 solves are faster)
        for pf, name, mask in ((S.SISDC_FP64, "fp64_plain", 0), (S.SISDC_MIXED, "mixed_all_levels", 0),
                               (S.SISDC_MIXED, "mixed_fine_level", 1 << (nlev - 1))):
            fctx = make_ctx(S, w, stream, pf, args.cg_rtol, 1, mask)
            uf = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
            tune(S, args, fctx, uf, dt, nlev)
            run_steps(S, fctx, uf, dt, ncyc, start, 2)                 # capture + warm
            S.sisdc_sync(fctx.ctx)                                     # the reset must follow them
            uf.copy_(torch.from_numpy(np.ascontiguousarray(u0)))
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            run_steps(S, fctx, uf, dt, ncyc, start, win)
            a1.record(stream)
            S.sisdc_sync(fctx.ctx)
            tms = a0.elapsed_time(a1)
            err = float(torch.linalg.vector_norm(uf - ur) / torch.linalg.vector_norm(ur))
            forms[name] = {"ms_per_step": tms / win, "dof_sweeps_per_s": dofs_per_step * win / (tms * 1e-3),
                           "time_to_solution_ms": tms, "rel_l2_error_vs_reference": err, "mixed_levels": mask}
            fctx.close()
        best = min(("mixed_all_levels", "mixed_fine_level"), key=lambda k: forms[k]["time_to_solution_ms"])
        forms["mixed_tuned"] = dict(forms[best], variant=best)
        tts = {"window_steps": win, "reference": "FP64 GPU path at dt/4 with 6 V-cycles per step",
               "error_ratio_tuned_over_plain": forms["mixed_tuned"]["rel_l2_error_vs_reference"] /
               max(1e-300, forms["fp64_plain"]["rel_l2_error_vs_reference"]),
               "speedup_tuned_over_plain": forms["fp64_plain"]["time_to_solution_ms"] /
               forms["mixed_tuned"]["time_to_solution_ms"]}


    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        try:
            onel = oracle_nel_for(args)
            r = run_oracle_child(args, 1 if not args.small else 3, onel)
            grid = " on %d^2 elements (same physics, degrees and nodes)" % onel if onel else ""
            cpu = {"value": r["dof_sweeps"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "%d full time step(s) of the %s workload%s by the FP64 numpy oracle "
                             "(single-threaded BLAS), %.1f s" % (r["steps"], args.workload, grid, r["seconds"]),
                   "cpu": cpu_model()}
        except Exception as e:   # reported, not fatal
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: %s" % e}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == S.SISDC_FP64 else "f32+f64",
        "data": "synthetic",
        "config": {"workload": args.workload + (" (8x8 elements)" if args.small else ""),
                   "precision": args.precision,
                   "fine_dofs": nv, "levels": w["levels"], "nodes": w["nodes"], "dt": dt,
                   "ncycles": ncyc, "fine_sweeps_per_step": ncyc + 1, "start": w["start"],
                   "si_stages": 2, "cg_rtol": args.cg_rtol, "cuda_graph": bool(use_graph),
                   "tiles": {"per_level_coarse_to_fine": tiles, "autotuned": not args.no_autotune,
                             "fields": "elements per tile, blocks, threads per block"},
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "kernel": "k_sweep correction launches, fine level",
                     "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": sweep_traffic(args),
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read + write)",
                     "peak_kind": "FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (measured 1.20)",
                     "avg_launch_us": avg_ms * 1e3, "launches": kt["launches"],
                     "cg_iters_per_launch": kt["iters"] / max(1, kt["launches"]),
                     "algorithmic_flop_per_launch": flops,
                     "kernel_share_of_step": kt["ms"] / max(1e-9, eager_s * 1e3)},
        "hbm_view": {"algorithmic_bytes_per_launch": nbytes, "achieved": hbm_gbs, "peak": hbm_peak,
                     "unit": "GB/s", "frac": hbm_gbs / hbm_peak, "peak_kind": hbm_kind + " copy bandwidth",
                     "note": "bytes a launch would move if no array stayed on chip; the level is L2-resident "
                             "(roofline.traffic) and the kernel is FP64-ALU bound, so this is not its limit"},
        "forms": forms, "time_to_solution": tts,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": nv * 8, "d2h_bytes_per_step": nv * 8},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "cg": {"solves_per_step": stats["cg_solves"] / args.steps,
               "iters_per_solve": stats["cg_iters"] / max(1, stats["cg_solves"]),
               "max_iters": stats["cg_max_iters"], "ir_steps": stats["ir_steps"]},
    }
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# ensemble workload: 512 independent convection-diffusion problems
# ---------------------------------------------------------------------------
def kernel_digest(files):
    """Short digest of the kernel sources and the workload definitions (ties
    a stored ncu traffic figure to the kernel version and the workload it was
    measured on).  An entry "ensemble_instances" stands for the ensemble's
    instance draw (sizes, degrees, coefficients, time steps), not for a file."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        if f == "ensemble_instances":
            # ten significant digits: the time steps depend on an eigenvalue
            # that LAPACK returns with last-bit differences across hosts
            from paper_2504_18526_gb300 import inputs
            g = lambda x: "%.10g" % x
            h.update(json.dumps([[d["P"], list(d["nel"]), g(d["nu"]), g(d["dt"]), [g(v) for v in d["adv"]], d["seed"]]
                                 for d in inputs.ensemble_instances()]).encode())
            continue
        path = os.path.join(ROOT, "paper_2504_18526_gb300", f if f.endswith(".py") else os.path.join("csrc", f))
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


ENS_KERNEL_SOURCES = ("ens.cuh", "sipg.cuh", "pde.cuh", "common.cuh", "ds.cuh", "ensemble_instances")

# DRAM traffic of the dominant ensemble launch (a fine-level correction sweep
# of the P = 8 group, FP64 form, the register-capped kernel with tiles of 6
# elements on two blocks per SM, the autotuner's pick):
# dram__bytes_read.sum + dram__bytes_write.sum
# of one ncu capture of that launch on the first 96 instances of the draw,
# per fine node of the group (the traffic grows with the group's nodes: the
# group's arrays exceed L2 in both cases), and the digest of the kernel
# sources it was measured on; traffic is reported as null for any other
# kernel version or form.
ENS_TRAFFIC = {"digest": "1890551bc379efe9", "bytes_per_node": 7258.4, "P": 8, "form": "fp64"}


def ens_cfg_apply(S, ens, cfg):
    """Set the tile shapes of sisdc_ens_config rows (fine, then coarse, per group)."""
    for g in range(len(cfg) // 2):
        for fine, row in ((1, cfg[2 * g]), (0, cfg[2 * g + 1])):
            S.sisdc_ens_set_tiles(ens, g, fine, int(row[2]), int(row[3]))


def ensemble_arm(args):
    import numpy as np
    import torch
    from paper_2504_18526_gb300 import inputs, sisdc as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0 or world == 1:
        from paper_2504_18526_gb300.build import build
        build()
    if dist:
        dist.barrier()
    S.load()

    w = inputs.WORKLOADS["ensemble512"]
    insts = inputs.ensemble_instances(w["ninst"])
    if args.ninst > 0:
        insts = insts[:args.ninst]
    stream = torch.cuda.Stream(device=dev)
    ncyc = w["ncycles"]
    nodes = [d["nel"][0] * d["nel"][1] * (d["P"] + 1) ** 2 for d in insts]
    dofs_per_step = sum(nodes) * (ncyc + 1)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    names = {"fp64": (S.SISDC_FP64, 0), "mixed": (S.SISDC_MIXED, 0), "mixed_fine_level": (S.SISDC_MIXED, 2)}

    def make(name, graph):
        prec, mask = names[name]
        return S.Ensemble(insts, stream=stream.cuda_stream, precision=prec, cg_rtol=args.cg_rtol, cg_maxit=1000,
                          M=w["M"], Mc=w["Mc"], nodes=w["nodes"], ncycles=ncyc, start=w["start"],
                          use_graph=graph, mixed_levels=mask)

    main_name = "fp64" if args.precision == "fp64" else "mixed"
    E = make(main_name, 0 if args.no_graph else 1)
    # initial data and exact solutions at the library's node coordinates
    hx, hy = np.zeros(E.total), np.zeros(E.total)
    S.sisdc_ens_coords(E.ens, hx, hy)

    def exact_field(t_of):
        u = np.zeros(E.total)
        for k, d in enumerate(insts):
            a, b = E.offsets[k], E.offsets[k] + nodes[k]
            u[a:b] = inputs.ensemble_exact(d, hx[a:b], hy[a:b], t_of(d)).ravel()
        return u

    u0_host = exact_field(lambda d: 0.0)
    u0 = torch.from_numpy(u0_host).to(dev)
    if args.no_autotune and args.capped:
        # profiling case: every level with its largest tile and two blocks per SM
        # (the register-capped kernel of the FP64 form)
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        for g in range(S.sisdc_ens_num_groups(E.ens)):
            for fine in (0, 1):
                P = int(S.sisdc_ens_config(E.ens)[2 * g + (0 if fine else 1)][1])   # rows: fine, coarse
                S.sisdc_ens_set_tiles(E.ens, g, fine, max(1, 512 // ((P + 1) ** 2)), 2 * nsm)
    cfg = S.sisdc_ens_config(E.ens) if args.no_autotune else S.sisdc_ens_autotune(E.ens, u0, 1)
    u = u0.clone()
    S.sisdc_ens_step(E.ens, u, args.warmup)
    S.sisdc_ens_sync(E.ens)
    S.sisdc_ens_reset_stats(E.ens)

    # ---- timed region: K steps, L2 flushed between steps -------------------
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        evs[k][0].record(stream)
        S.sisdc_ens_step(E.ens, u, 1)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    S.sisdc_ens_sync(E.ens)
    ms = sum(a.elapsed_time(b) for a, b in evs)
    st = S.sisdc_ens_get_stats(E.ens, len(insts))
    ms = max_over_ranks(ms, dist, dev)
    value = whole_job_value(dofs_per_step, args.steps, world, ms)
    nsteps_total = args.warmup + args.steps
    ex_host = exact_field(lambda d: nsteps_total * d["dt"])

    def errors(uu):
        ex = torch.from_numpy(ex_host).to(dev)
        rel = []
        for k in range(len(insts)):
            a, b = E.offsets[k], E.offsets[k] + nodes[k]
            rel.append(float(torch.linalg.vector_norm(uu[a:b] - ex[a:b]) / torch.linalg.vector_norm(ex[a:b])))
        return {"mean": float(np.mean(rel)), "max": float(np.max(rel))}

    err_main = errors(u)

    # ---- e2e: host buffers through the C ABI, copies inside the timed region --
    h_in = torch.from_numpy(u0_host).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_e2e = torch.empty_like(u0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ke = max(3, args.steps // 4)
    t_e2e = 0.0
    torch.cuda.synchronize()
    for k in range(ke):
        e0.record(stream)
        with torch.cuda.stream(stream):
            d_e2e.copy_(h_in, non_blocking=True)
        S.sisdc_ens_step(E.ens, d_e2e, 1)
        with torch.cuda.stream(stream):
            h_out.copy_(d_e2e, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        t_e2e += e0.elapsed_time(e1)
    S.sisdc_ens_sync(E.ens)
    t_e2e = max_over_ranks(t_e2e, dist, dev)
    e2e_val = world * dofs_per_step * ke / (t_e2e * 1e-3)
    E.close()

    # ---- dominant kernel: live CUDA-event timing of the fine correction launches --
    Ek = make(main_name, 0)
    ens_cfg_apply(S, Ek.ens, cfg)
    uk = u0.clone()
    S.sisdc_ens_step(Ek.ens, uk, 1)
    S.sisdc_ens_sync(Ek.ens)
    S.sisdc_ens_reset_stats(Ek.ens)
    S.sisdc_ens_set_kernel_timing(Ek.ens, True)
    kt_steps = 2
    t0 = time.perf_counter()
    for k in range(kt_steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        S.sisdc_ens_step(Ek.ens, uk, 1)
    g_ms, g_launch = S.sisdc_ens_get_kernel_timing(Ek.ens)
    eager_ms = (time.perf_counter() - t0) * 1e3
    kst = S.sisdc_ens_get_stats(Ek.ens, len(insts))
    S.sisdc_ens_sync(Ek.ens)
    Ek.close()
    degrees = sorted({d["P"] for d in insts})
    per_group = []
    for gi, P in enumerate(degrees):
        members = [k for k, d in enumerate(insts) if d["P"] == P]
        nl = max(1, int(g_launch[gi]))
        fl = sum(sweep_flops(P, 1, w["M"], 1, kst["inst_iters"][k] / nl, nodes[k]) for k in members)
        per_group.append({"P": P, "instances": len(members), "fine_nodes": sum(nodes[k] for k in members),
                          "launches": int(g_launch[gi]), "avg_launch_ms": float(g_ms[gi]) / nl,
                          "algorithmic_flop_per_launch": fl,
                          "tflops": fl / (float(g_ms[gi]) / nl * 1e-3) / 1e12 if g_ms[gi] > 0 else 0.0})
    dom = max(per_group, key=lambda r: r["avg_launch_ms"] * r["launches"])
    traffic = None
    if (ENS_TRAFFIC["digest"] == kernel_digest(ENS_KERNEL_SOURCES) and dom["P"] == ENS_TRAFFIC["P"]
            and main_name == ENS_TRAFFIC["form"] and ENS_TRAFFIC["bytes_per_node"]):
        traffic = ENS_TRAFFIC["bytes_per_node"] * dom["fine_nodes"]
    hbm_peak, hbm_kind = measured_peaks()
    dom_members = [k for k, d in enumerate(insts) if d["P"] == dom["P"]]
    nbytes = sum(sweep_bytes(w["M"], 1, kst["inst_iters"][k] / max(1, dom["launches"]), nodes[k])
                 for k in dom_members)

    # ---- the other precision forms: time-to-solution at equal error vs exact --
    forms = {main_name: {"ms_per_step": ms / args.steps, "dof_sweeps_per_s": value / world,
                         "rel_l2_error_vs_exact": err_main, "steps_for_error": nsteps_total,
                         "cg_iters_per_solve": st["cg_iters"] / max(1, st["cg_solves"]),
                         "ir_steps": st["ir_steps"], "tiles": cfg.tolist()}}
    if not args.no_forms:
        for name in [n for n in ("fp64", "mixed", "mixed_fine_level") if n != main_name]:
            Ef = make(name, 0 if args.no_graph else 1)
            cf = S.sisdc_ens_config(Ef.ens) if args.no_autotune else S.sisdc_ens_autotune(Ef.ens, u0, 1)
            uf = u0.clone()
            S.sisdc_ens_step(Ef.ens, uf, args.warmup)
            S.sisdc_ens_sync(Ef.ens)
            S.sisdc_ens_reset_stats(Ef.ens)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a0.record(stream)
            S.sisdc_ens_step(Ef.ens, uf, args.steps)
            a1.record(stream)
            S.sisdc_ens_sync(Ef.ens)
            tms = a0.elapsed_time(a1)
            sf = S.sisdc_ens_get_stats(Ef.ens, 0)
            forms[name] = {"ms_per_step": tms / args.steps, "dof_sweeps_per_s": dofs_per_step * args.steps / (tms * 1e-3),
                           "rel_l2_error_vs_exact": errors(uf), "steps_for_error": nsteps_total,
                           "cg_iters_per_solve": sf["cg_iters"] / max(1, sf["cg_solves"]),
                           "ir_steps": sf["ir_steps"], "tiles": cf.tolist()}
            Ef.close()
    tts = None
    mixed_names = [n for n in ("mixed", "mixed_fine_level") if n in forms]
    if "fp64" in forms and mixed_names:
        best = min(mixed_names, key=lambda n: forms[n]["ms_per_step"])
        tts = {"window_steps": nsteps_total, "reference": "exact solution of every instance", "tuned": best,
               "error_ratio_tuned_over_plain": forms[best]["rel_l2_error_vs_exact"]["mean"] /
               max(1e-300, forms["fp64"]["rel_l2_error_vs_exact"]["mean"]),
               "speedup_tuned_over_plain": forms["fp64"]["ms_per_step"] / forms[best]["ms_per_step"]}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline else cpu_baseline_ensemble(args)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if main_name == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": "ensemble512" + (" (first %d instances)" % len(insts) if args.ninst else ""),
                   "instances": len(insts), "fine_nodes": sum(nodes), "autotuned": not args.no_autotune,
                   "fine_sweeps_per_step": ncyc + 1, "levels": "fine P, coarse ceil(P/2); Radau-Right 5/3",
                   "start": w["start"], "si_stages": 2, "cg_rtol": args.cg_rtol,
                   "precision": main_name, "cuda_graph": not args.no_graph,
                   "l2": "state larger than L2 (%.0f MB per vector) and a 512 MB flush between timed steps"
                         % (sum(nodes) * 8 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "kernel": "k_ens_sweep fine-level correction launch of the P = %d group"
                                               % dom["P"],
                     "achieved": dom["tflops"], "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": dom["tflops"] / FP64_PEAK_TFLOPS, "traffic": traffic,
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read + write)",
                     "peak_kind": "FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (measured 1.20)",
                     "avg_launch_us": dom["avg_launch_ms"] * 1e3, "launches": dom["launches"],
                     "algorithmic_flop_per_launch": dom["algorithmic_flop_per_launch"],
                     "kernel_share_of_step": sum(r["avg_launch_ms"] * r["launches"] for r in per_group) /
                     max(1e-9, eager_ms),
                     "step_level_frac": sum(sweep_flops(d["P"], 1, w["M"], ncyc + 1,
                                                        st["inst_iters"][k] / args.steps, nodes[k])
                                            for k, d in enumerate(insts)) / (ms / args.steps * 1e-3) / 1e12
                     / FP64_PEAK_TFLOPS,
                     "groups": per_group},
        "hbm_view": {"algorithmic_bytes_per_launch": nbytes,
                     "achieved": nbytes / (dom["avg_launch_ms"] * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": nbytes / (dom["avg_launch_ms"] * 1e-3) / 1e9 / hbm_peak,
                     "peak_kind": hbm_kind + " copy bandwidth",
                     "note": "bytes the launch would move if no array stayed on chip; the kernel is FP64-ALU "
                             "bound, so this is not its limit"},
        "forms": forms, "time_to_solution": tts, "cpu_baseline": cpu, "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(sum(nodes)) * 8,
                "d2h_bytes_per_step": int(sum(nodes)) * 8},
        "gpu_launches": int(round(st["launches"])),
        "cg": {"solves_per_step": st["cg_solves"] / args.steps,
               "iters_per_solve": st["cg_iters"] / max(1, st["cg_solves"]), "max_iters": st["cg_max_iters"]},
    }
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# stability map of the Dahlquist problem (one GPU thread per point)
# ---------------------------------------------------------------------------
def stability_arm(args):
    import numpy as np
    import torch
    from paper_2504_18526_gb300 import sisdc as S
    from paper_2504_18526_gb300.build import build

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    build()
    S.load()
    nx = ny = 1024
    zr = torch.linspace(-40.0, 5.0, nx, dtype=torch.float64, device=dev)
    zi = torch.linspace(-40.0, 40.0, ny, dtype=torch.float64, device=dev)
    z = (zr[None, :] + 1j * zi[:, None]).reshape(-1)
    cfg = dict(Ms=[3, 5, 7], nodes="radau_right", stages=2, ncycles=3, start="fmg1")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        S.sisdc_stability(z, stream=stream.cuda_stream, **cfg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        R = S.sisdc_stability(z, stream=stream.cuda_stream, **cfg)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    stable = float((R.abs() <= 1.0 + 1e-12).double().mean())
    cpu = None
    if not args.no_cpu_baseline:
        from oracle.dahlquist import stability
        pts = z[:: max(1, z.numel() // 400)].cpu().numpy()
        t0 = time.perf_counter()
        for p in pts:
            stability(complex(p), cfg["Ms"], cfg["nodes"], cfg["stages"], cfg["ncycles"], cfg["start"])
        el = time.perf_counter() - t0
        cpu = {"value": len(pts) / el, "unit": "points/s", "cores": 1, "kind": "oracle",
               "sample": "%d points of the same map by the numpy oracle, %.1f s" % (len(pts), el)}
    print(json.dumps({"metric": "stability-map points/s", "value": z.numel() * args.steps / (ms * 1e-3),
                      "unit": "points/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": "stability_map", "grid": [nx, ny], "box": [[-40, 5], [-40, 40]],
                                 "method": cfg, "stable_fraction": stable},
                      "cpu_baseline": cpu}))


# ---------------------------------------------------------------------------
# the paper's 1D convection-diffusion studies through the library
# ---------------------------------------------------------------------------
def convdiff_run(S, dev, nels, P, Ms, nu, cfl, ncycles, start="cascade", T=5.0, rtol=1e-13):
    """One run of u_t + u_x = nu u_xx on the periodic unit interval to time T
    (the wave packet), levels with nels[l] elements of degree P and Ms[l]
    Radau-Right nodes, dt from the CFL number on the finest grid
    (dx = dx_e / (2 delta(P)), lambda = 1), ncycles V-cycles + post-sweep per step
    (one level: predictor + ncycles sweeps).  Returns (GLL L2 error at T,
    steps); the error is inf when the run blew up."""
    import math
    import numpy as np
    import torch
    from paper_2504_18526_gb300 import inputs
    w = dict(pde="convdiff", dim=1, ncomp=1, adv=(1.0, 0.0), nu=nu, lo=(0.0, 0.0), hi=(1.0, 0.0),
             nodes="radau_right", levels=[dict(nel=(ne, 1), P=P, M=M) for ne, M in zip(nels, Ms)])
    ctx = S.Context(w, cg_rtol=rtol, cg_maxit=20000, use_graph=1)
    nc, n, M = ctx.info(-1)
    X = np.zeros(n)
    S.sisdc_level_coords(ctx.levels[-1], X, None)
    dx = (1.0 / nels[-1]) / (2.0 * inputs.cfl_delta(P))
    nsteps = int(math.ceil(T / (cfl * dx) - 1e-9))
    dt = T / nsteps
    du = torch.from_numpy(inputs.wave_packet(X, 0.0, nu).ravel().copy()).to(dev)
    ex = torch.from_numpy(inputs.wave_packet(X, T, nu).ravel().copy()).to(dev)
    st = S.START_IDS[start]
    try:
        for k in range(nsteps):
            S.sisdc_step(ctx.ctx, du, k * dt, dt, ncycles, st, 1)
            if k % 256 == 255 and not bool(torch.isfinite(du).all()):
                raise FloatingPointError
        S.sisdc_sync(ctx.ctx)
        err = float(S.sisdc_norms(ctx.levels[-1], du, ex)[0][0])
        if not math.isfinite(err) or err > 1e3:
            err = float("inf")
    except (FloatingPointError, S.SisdcError):
        err = float("inf")
    ctx.close()
    return err, nsteps


CONVDIFF_TABLE_MESHES = ((5, 10, 20), (10, 20, 40), (20, 40, 80), (40, 80, 160))
CONVDIFF_TABLE_CFLS = (32, 64, 128, 256)


def converged_count(errs):
    """Iterations after which one more iteration changes the error by less
    than 10 % (the paper's convergence rule); errs[k] = error after k+1."""
    for k in range(len(errs) - 1):
        if abs(errs[k + 1] - errs[k]) <= 0.1 * abs(errs[k]):
            return k + 1
    return None


def paper_convdiff_arm(args):
    """The paper's Sec. 8 convection-diffusion studies on the GPU: the L2
    error table of the convergence analysis (MLSDC^10_{3,5,7}, P = 12,
    elements doubling per level) and the CFL study (nu = 1e-3: three levels
    16/32/64 elements of degree 15, M 3/5/7; nu = 0: two levels 32/64, M
    5/7; Cascade start, N_c = 2) against single-level SDC on the finest
    level: fine sweeps to convergence per CFL number."""
    import math
    import torch
    from paper_2504_18526_gb300 import sisdc as S
    from paper_2504_18526_gb300.build import build
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    build()
    S.load()
    t0 = time.perf_counter()
    table = {}
    for mesh in (CONVDIFF_TABLE_MESHES if args.part in ("all", "table") else ()):
        for cfl in CONVDIFF_TABLE_CFLS:
            e, n = convdiff_run(S, dev, mesh, 12, (3, 5, 7), 1e-3, cfl, 10)
            table["%d,%d,%d@%d" % (mesh + (cfl,))] = {"error": e, "steps": n}
    orders = {}
    for k in (range(1, len(CONVDIFF_TABLE_MESHES)) if table else ()):
        for cfl in CONVDIFF_TABLE_CFLS:
            a = table["%d,%d,%d@%d" % (CONVDIFF_TABLE_MESHES[k - 1] + (cfl,))]["error"]
            b = table["%d,%d,%d@%d" % (CONVDIFF_TABLE_MESHES[k] + (cfl,))]["error"]
            orders["space %s@%d" % (CONVDIFF_TABLE_MESHES[k], cfl)] = math.log2(a / b)
    study = {}
    for nu, nels, Ms in (((1e-3, (16, 32, 64), (3, 5, 7)), (0.0, (32, 64), (5, 7)))
                         if args.part in ("all", "study") else ()):
        if args.nus is not None and nu not in args.nus:
            continue
        for cfl in args.cfls:
            ml, sd = [], []
            for C in range(1, 13):
                ml.append(convdiff_run(S, dev, nels, 15, Ms, nu, cfl, C)[0])
                if converged_count(ml) or not math.isfinite(ml[-1]):
                    break
            for N in range(1, 21):
                sd.append(convdiff_run(S, dev, nels[-1:], 15, Ms[-1:], nu, cfl, N - 1)[0])
                if converged_count(sd) or not math.isfinite(sd[-1]):
                    break
            c_ml, c_sd = converged_count(ml), converged_count(sd)
            study["nu=%g@CFL%g" % (nu, cfl)] = {
                "mlsdc_errors_per_cycles": ml, "sdc_errors_per_sweeps": sd,
                "mlsdc_cycles": c_ml, "mlsdc_fine_sweeps": None if c_ml is None else c_ml + 1,
                "sdc_sweeps": c_sd}
            print("study nu=%g CFL %g: %s (%.0f s)" % (nu, cfl, json.dumps(study["nu=%g@CFL%g" % (nu, cfl)]),
                                                      time.perf_counter() - t0), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "paper 1D convection-diffusion studies", "workload": "paper_convdiff",
                      "error_table": table, "orders": orders, "cfl_study": study,
                      "seconds": time.perf_counter() - t0}))


BURGERS_FRONT_VARIANTS = (
    # (name, levels (nel_x, P, M) coarse to fine, start): the rows of the paper's
    # low-resolution iteration table (Sec. 8, Burgers moving front)
    ("SDC 40xP8 M7", ((40, 8, 7),), None),
    ("MLSDC {40,40,40} P8 FMG1", ((40, 8, 3), (40, 8, 5), (40, 8, 7)), "fmg1"),
    ("MLSDC {10,20,40} P8 FMG1", ((10, 8, 3), (20, 8, 5), (40, 8, 7)), "fmg1"),
    ("MLSDC {40,40,40} P{2,4,8} FMG1", ((40, 2, 3), (40, 4, 5), (40, 8, 7)), "fmg1"),
)


def shock_run(S, dev, w, levels, start, ncycles, dt, nsteps, rtol=1e-12, timed=False):
    """One run of a shock-capturing workload (artificial viscosity on every
    level) with the given levels (nel_x, P, M): nsteps steps of dt, ncycles
    V-cycles + post-sweep per step (one level: predictor + ncycles sweeps).
    Returns the final state (numpy, fine level), its coordinates and, when
    timed, the ms per step of a second, graph-replayed pass."""
    import numpy as np
    import torch
    from paper_2504_18526_gb300 import inputs
    wl = dict(w)
    wl["levels"] = [dict(nel=(ne, 1), P=P, M=M) for ne, P, M in levels]
    ctx = S.Context(wl, cg_rtol=rtol, cg_maxit=20000, use_graph=1)
    nc, n, M = ctx.info(-1)
    X = np.zeros(n)
    Y = np.zeros(n)
    S.sisdc_level_coords(ctx.levels[-1], X, Y)
    P = levels[-1][1]
    shape = (1, levels[-1][0], P + 1, P + 1)
    X = X.reshape(shape)
    u0 = inputs.initial_state(w["name"], X, Y.reshape(shape))
    du = torch.from_numpy(np.ascontiguousarray(u0).ravel().copy()).to(dev)
    st = S.START_IDS[start or "cascade"]
    for k in range(nsteps):
        S.sisdc_step(ctx.ctx, du, k * dt, dt, ncycles, st, 1)
    S.sisdc_sync(ctx.ctx)
    u = du.cpu().numpy().reshape((nc,) + shape)
    ms = None
    if timed:
        d2 = torch.from_numpy(np.ascontiguousarray(u0).ravel().copy()).to(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream(dev)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(nsteps):
            S.sisdc_step(ctx.ctx, d2, k * dt, dt, ncycles, st, 1)
        e1.record(stream)
        S.sisdc_sync(ctx.ctx)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / nsteps
    ctx.close()
    return u, X, ms


def shock_arm(args):
    """The paper's shock-capturing experiments with the Persson-Peraire
    artificial viscosity (Sec. 8): the Burgers moving front (under-resolved,
    nu = 1e-2, t in [0, 0.1]: fine iterations until convergence per CFL for
    single-level SDC and three MLSDC variants, the 10 % rule on the L2 error
    against the exact front away from the periodic seam) and Sod's shock tube
    (32 steps to t = 0.2, CFL ~ 7: density and velocity errors against the
    exact Riemann solution after C V-cycles of MLSDC and N sweeps of SDC,
    and the velocity overshoot)."""
    import math
    import numpy as np
    import torch
    from paper_2504_18526_gb300 import inputs, sisdc as S
    from paper_2504_18526_gb300.build import build
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    build()
    S.load()
    t0 = time.perf_counter()
    w = dict(inputs.WORKLOADS[args.workload])
    w["name"] = args.workload
    out = {"metric": "paper shock-capturing studies", "workload": args.workload}
    if args.workload == "burgers_front":
        lo, hi = w["window"]
        h = (w["hi"][0] - w["lo"][0]) / 40
        table = {}
        for name, levels, start in BURGERS_FRONT_VARIANTS:
            row = {}
            for cfl in args.cfls:
                dt0 = inputs.cfl_dt(cfl, h, 8, 2.0)                    # lam_max = 2 u_1 = 2
                nsteps = int(math.ceil(w["T"] / dt0 - 1e-9))
                dt = w["T"] / nsteps
                errs = []
                for k in range(1, 21):
                    nc = k - 1 if start is None else k
                    u, X, _ = shock_run(S, dev, w, levels, start, nc, dt, nsteps)
                    ex = inputs.burgers_front(X, w["T"], w["nu"])
                    win = (X >= lo) & (X <= hi)
                    e = float(np.sqrt(np.mean(((u[0] - ex[0]) ** 2)[np.broadcast_to(win, u[0].shape)])))
                    errs.append(e if math.isfinite(e) else float("inf"))
                    if converged_count(errs) or not math.isfinite(errs[-1]):
                        break
                c = converged_count(errs)
                fine = None if c is None else (c if start is None else c + 1)
                row["%g" % cfl] = {"fine_iterations": fine, "errors": errs, "steps": nsteps}
            table[name] = row
            print("front %s: %s (%.0f s)" % (name, {k: v["fine_iterations"] for k, v in row.items()},
                                              time.perf_counter() - t0), file=sys.stderr, flush=True)
        out["fine_iterations_until_convergence"] = table
    else:
        dt = w["T"] / w["nsteps"]
        levels = tuple((lv["nel"][0], lv["P"], lv["M"]) for lv in w["levels"])
        ps, us = inputs._sod_star()
        res = {}
        for name, lv, start, counts in (("MLSDC P{3,5} M{5,7} Cascade", levels, "cascade", range(1, 7)),
                                        ("SDC P5 M7", levels[-1:], None, range(1, 9))):
            rows = []
            for k in counts:
                nc = k - 1 if start is None else k
                u, X, ms = shock_run(S, dev, w, lv, start, nc, dt, w["nsteps"], timed=(k == 3))
                ex = inputs.sod_state(X, w["T"])
                half = np.broadcast_to(X <= 1.0, u[0].shape)
                v = u[1] / u[0]
                rows.append({"iterations": k, "fine_sweeps": k if start is None else k + 1,
                             "rho_l1": float(np.mean(np.abs(u[0] - ex[0])[half])),
                             "v_l1": float(np.mean(np.abs(v - ex[1] / ex[0])[half])),
                             "v_max_over_ustar": float(v[half].max() / us),
                             "ms_per_step": ms})
            res[name] = rows
            print("sod %s: %s (%.0f s)" % (name, [(r["iterations"], round(r["rho_l1"], 5)) for r in rows],
                                            time.perf_counter() - t0), file=sys.stderr, flush=True)
        out["sod"] = res
        out["dt"] = dt
        rho_e, v_e, p_e = inputs.sod_primitive(np.linspace(0.0, 1.0, 4001), w["T"])
        lam = float(np.max(np.abs(v_e) + np.sqrt(w["gamma"] * p_e / rho_e)))   # lam_max at t = 0.2
        h = (w["hi"][0] - w["lo"][0]) / levels[-1][0]
        out["cfl"] = dt * lam / (h / (2.0 * inputs.cfl_delta(levels[-1][1])))
    out["seconds"] = time.perf_counter() - t0
    print(json.dumps(out))


def learned_arm(args):
    """The learned initial guess inside the method on the Navier-Stokes shear
    layer (128^2 elements, P = 5/3): the network (325 -> 112 -> 112 -> 36,
    BF16) is trained on the GPU on about 10^4 implicit solves logged from the
    plain method's own fine-level sweeps (chunks of logged solves, one Adam
    epoch per chunk); then the same window of time steps runs with the plain
    persistent sweep kernel (CUDA graph), the plain composed sweep (eager)
    and the learned composed sweep, each against an FP64 reference at dt/4:
    time, CG iterations per solve and L2 error."""
    import numpy as np
    import torch
    from paper_2504_18526_gb300 import inputs, sisdc as S
    from paper_2504_18526_gb300.build import build
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    build()
    S.load()
    w = workload(args)
    stream = torch.cuda.Stream(device=dev)
    fine = len(w["levels"]) - 1

    def ctx_of(graph):
        return S.Context(w, stream=stream.cuda_stream, cg_rtol=args.cg_rtol, cg_maxit=2000, use_graph=graph)

    ctx = ctx_of(0)
    nc, n, M = ctx.info(-1)
    hx, hy = np.zeros(n), np.zeros(n)
    S.sisdc_level_coords(ctx.levels[-1], hx, hy)
    lv = w["levels"][-1]
    shp = (lv["nel"][1], lv["nel"][0], lv["P"] + 1, lv["P"] + 1)
    u0, dt = initial_data(w, hx.reshape(shp), hy.reshape(shp))
    ncyc, start = w["ncycles"], S.START_IDS[w["start"]]
    nv = nc * n
    # ---- training on logged solves of the plain method ----------------------
    chunk = max(16, min(args.learn_chunk, 600))
    lr_ = torch.zeros((chunk, nv), dtype=torch.float64, device=dev)
    ldx = torch.zeros_like(lr_)
    lc = torch.zeros(chunk, dtype=torch.float64, device=dev)
    m = S.sisdc_mlp_create(ctx.levels[fine], 112, seed=11, bf16=1)
    u = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
    trained, steps_run, t_log, t_train = 0, 0, 0.0, 0.0
    while trained < args.learn_solves:
        S.sisdc_set_solve_log(ctx.ctx, fine, lr_, ldx, lc, chunk)
        t0 = time.perf_counter()
        while S.sisdc_get_solve_log_count(ctx.ctx) < chunk:
            S.sisdc_step(ctx.ctx, u, steps_run * dt, dt, ncyc, start, 1)
            steps_run += 1
        t_log += time.perf_counter() - t0
        cs = lc.cpu().numpy()
        keep = np.nonzero((torch.abs(ldx).amax(dim=1).cpu().numpy() > 0) & (cs > 0))[0]
        t0 = time.perf_counter()
        if len(keep):
            S.sisdc_mlp_train(m, lr_[keep].contiguous(), ldx[keep].contiguous(), cs[keep], len(keep), 1, 1e-3)
        torch.cuda.synchronize()
        t_train += time.perf_counter() - t0
        trained += len(keep)
    S.sisdc_set_solve_log(ctx.ctx, fine)
    del lr_, ldx
    torch.cuda.empty_cache()
    # ---- the window: reference, plain kernel, plain composed, learned --------
    win = max(2, args.steps)
    ustart = u.clone()
    ref = ctx_of(1)
    ur = ustart.clone()
    for k in range(4 * win):
        S.sisdc_step(ref.ctx, ur, 0.0, dt / 4, 6, start, 1)
    S.sisdc_sync(ref.ctx)
    ref.close()
    forms = {}
    zero = S.sisdc_mlp_create(ctx.levels[fine], 112, seed=12, bf16=1)
    npar = S.sisdc_mlp_info(zero)[3]
    S.sisdc_mlp_params(zero, set_=np.zeros(npar, dtype=np.float32))   # correction z = r (no learning)
    for name, graph, model in (("fp64_plain_kernel", 1, None), ("fp64_composed_identity_guess", 0, zero),
                               ("fp64_composed_learned_guess", 0, m)):
        c2 = ctx_of(graph)
        if model is not None:
            S.sisdc_set_learned(c2.ctx, fine, model)
        uf = ustart.clone()
        for _ in range(args.warmup):
            S.sisdc_step(c2.ctx, uf, 0.0, dt, ncyc, start, 1)
        S.sisdc_sync(c2.ctx)
        uf.copy_(ustart)
        S.sisdc_reset_stats(c2.ctx)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a0.record(stream)
        for _ in range(win):
            S.sisdc_step(c2.ctx, uf, 0.0, dt, ncyc, start, 1)
        a1.record(stream)
        S.sisdc_sync(c2.ctx)
        tms = a0.elapsed_time(a1)
        st = S.sisdc_get_stats(c2.ctx)
        err = float(torch.linalg.vector_norm(uf - ur) / torch.linalg.vector_norm(ur))
        forms[name] = {"ms_per_step": tms / win, "cg_iters_per_solve": st["cg_iters"] / max(1, st["cg_solves"]),
                       "cg_solves": st["cg_solves"], "rel_l2_error_vs_reference": err}
        if model is not None:
            S.sisdc_set_learned(c2.ctx, fine, None)
        c2.close()
    S.sisdc_mlp_destroy(zero)
    S.sisdc_mlp_destroy(m)
    ctx.close()
    plain = forms["fp64_plain_kernel"]
    print(json.dumps({
        "metric": "learned initial guess: CG iterations and time at equal error", "workload": args.workload,
        "training": {"solves": trained, "steps_logged": steps_run, "chunk": chunk, "log_s": t_log,
                     "train_s": t_train, "network": "325-112-112-36 BF16 (tcgen05 inference)"},
        "window_steps": win, "forms": forms,
        "error_ratio_learned_over_plain": forms["fp64_composed_learned_guess"]["rel_l2_error_vs_reference"] /
        max(1e-300, plain["rel_l2_error_vs_reference"]),
        "iteration_ratio_learned_over_identity": forms["fp64_composed_learned_guess"]["cg_iters_per_solve"] /
        max(1e-300, forms["fp64_composed_identity_guess"]["cg_iters_per_solve"]),
        "time_ratio_learned_over_plain_kernel": forms["fp64_composed_learned_guess"]["ms_per_step"] /
        plain["ms_per_step"]}))


def mlp_flops(rows, n_in, H, q):
    """GEMM flops of one inference (forward) and one training step (forward,
    the five backward products) of the n_in -> H -> H -> q network."""
    fwd = 2.0 * rows * (n_in * H + H * H + H * q)
    bwd = 2.0 * rows * (n_in * H + 2 * H * H + 2 * H * q)
    return fwd, fwd + bwd


def mlp_arm(args):
    """The learned part on the Navier-Stokes level (128^2 elements, P = 5,
    four components: 65 536 patch rows, 325 -> 112 -> 112 -> 36): training
    steps (loss, gradients, Adam) on synthetic logged solves, and inference
    (gather, three layers, scatter), BF16 tensor-core mode against the FP32
    SIMT mode."""
    import numpy as np
    import torch
    from paper_2504_18526_gb300 import inputs, sisdc as S
    from paper_2504_18526_gb300.build import build

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    build()
    S.load()
    stream = torch.cuda.current_stream()
    w = inputs.WORKLOADS["ns_shear"]
    ctx = S.Context(w, stream=stream.cuda_stream)
    lv = ctx.levels[-1]
    nc, n, M = ctx.info(-1)
    nv = nc * n
    K = max(args.steps, 1)
    gen = torch.Generator(device=dev)
    gen.manual_seed(2504185260 + 7)
    r = torch.randn((K, nv), dtype=torch.float64, device=dev, generator=gen)
    dx = r + 0.1 * torch.randn((K, nv), dtype=torch.float64, device=dev, generator=gen)
    cs = np.full(K, 3e-3)
    hidden = 112
    res = {}
    clk = ClockSampler(dev.index or 0)
    for mode, name in ((1, "bf16_tensor_core"), (0, "fp32_simt")):
        m = S.sisdc_mlp_create(lv, hidden, seed=1, bf16=mode)
        n_in, H, q, npar = S.sisdc_mlp_info(m)
        rows = nv // q
        S.sisdc_mlp_train(m, r, dx, cs, min(K, max(args.warmup, 1)), 1, 1e-3)
        z = torch.zeros(nv, dtype=torch.float64, device=dev)
        for _ in range(max(args.warmup, 1)):
            S.sisdc_mlp_apply(m, r[0], 3e-3, z)
        torch.cuda.synchronize()
        if mode == 1:
            clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S.sisdc_mlp_train(m, r, dx, cs, K, 1, 1e-3)
        e1.record(stream)
        torch.cuda.synchronize()
        t_train = e0.elapsed_time(e1) / K
        e0.record(stream)
        for k in range(K):
            S.sisdc_mlp_apply(m, r[k], 3e-3, z)
        e1.record(stream)
        torch.cuda.synchronize()
        t_inf = e0.elapsed_time(e1) / K
        t_inf_tc = None
        if mode == 1:
            # the same inference through the fused tcgen05 kernel (gather, three
            # layers and output in one persistent launch) against the mma.sync path
            S.sisdc_mlp_set_tc(m, False)
            for _ in range(max(args.warmup, 1)):
                S.sisdc_mlp_apply(m, r[0], 3e-3, z)
            torch.cuda.synchronize()
            e0.record(stream)
            for k in range(K):
                S.sisdc_mlp_apply(m, r[k], 3e-3, z)
            e1.record(stream)
            torch.cuda.synchronize()
            t_inf_mma = e0.elapsed_time(e1) / K
            S.sisdc_mlp_set_tc(m, True)
            for _ in range(max(args.warmup, 1)):
                S.sisdc_mlp_apply(m, r[0], 3e-3, z)
            torch.cuda.synchronize()
            e0.record(stream)
            for k in range(K):
                S.sisdc_mlp_apply(m, r[k], 3e-3, z)
            e1.record(stream)
            S.sisdc_mlp_sync(m)
            t_inf_tc = e0.elapsed_time(e1) / K
            t_inf = t_inf_mma
        if mode == 1:
            clocks = clk.stop()
        f_inf, f_train = mlp_flops(rows, n_in, H, q)
        res[name] = {"train_ms_per_step": t_train, "train_rows_per_s": rows / (t_train * 1e-3),
                     "infer_ms": t_inf, "infer_rows_per_s": rows / (t_inf * 1e-3),
                     "train_gemm_tflops": f_train / (t_train * 1e-3) / 1e12,
                     "infer_gemm_tflops": f_inf / (t_inf * 1e-3) / 1e12}
        if t_inf_tc is not None:
            res[name].update({"infer_ms_tcgen05_fused": t_inf_tc, "infer_rows_per_s_tcgen05": rows / (t_inf_tc * 1e-3),
                              "infer_gemm_tflops_tcgen05": f_inf / (t_inf_tc * 1e-3) / 1e12,
                              "infer_ms_mma_sync": t_inf})
        S.sisdc_mlp_destroy(m)
    ctx.close()
    peak = 1940.5
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, pkind = float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        peak, pkind = 1900.0, "fallback"
    tc = res["bf16_tensor_core"]
    cpu = None
    if not args.no_cpu_baseline:
        o = run_oracle_child(args, 1)
        cpu = {"value": o["rows"] / o["seconds"], "unit": "rows/s", "cores": 1, "kind": "oracle",
               "sample": "%d FP64 numpy loss+gradient passes of the oracle MLP over 4096 rows (single-threaded "
                         "BLAS), %.1f s" % (o["passes"], o["seconds"])}
    print(json.dumps({
        "metric": "MLP training rows/s", "value": tc["train_rows_per_s"], "unit": "rows/s", "n_gpus": 1,
        "steps": K, "warmup": args.warmup, "ms_per_step": tc["train_ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic",
        "config": {"workload": "mlp_ns_level", "rows": rows, "layers": [n_in, H, H, q],
                   "step": "one training step (loss, gradients, Adam) on one logged solve of the level",
                   "l2": "weights L2-resident; each step reads a new 19 MB residual and correction pair"},
        "roofline": {"bound": "tensor", "kernel": "k_gemm_tc (all GEMMs of a training step, with the step's other kernels in the time)",
                     "achieved": tc["train_gemm_tflops"], "peak": peak, "unit": "TFLOP/s",
                     "frac": tc["train_gemm_tflops"] / peak, "traffic": None, "peak_kind": pkind + " bf16 dense"},
        "forms": res, "cpu_baseline": cpu, "clocks": clocks,
        "gpu_launches": None}))


if __name__ == "__main__":
    a = parse()
    if a.oracle_sample:
        if a.workload == "mlp_ns_level":
            mlp_oracle_sample(a)
        elif a.workload == "ensemble512":
            ensemble_oracle_sample(a)
        else:
            oracle_sample(a)
    elif a.impl == "reference":
        reference_arm(a)
    elif a.workload == "ensemble512":
        ensemble_arm(a)
    elif a.workload == "stability_map":
        stability_arm(a)
    elif a.workload == "paper_convdiff":
        paper_convdiff_arm(a)
    elif a.workload in ("burgers_front", "sod"):
        shock_arm(a)
    elif a.learned:
        learned_arm(a)
    elif a.workload == "mlp_ns_level":
        mlp_arm(a)
    else:
        main_arm(a)
