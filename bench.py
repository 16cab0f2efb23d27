"""Throughput of the fused coupled lattice Boltzmann step on one GB300 (or N replicas).

Workload: 512^3 lattice, D3Q19 flow + D3Q7 phi, c^A, c^B, FP32 population storage,
half-way bounce-back walls at the z ends, periodic in x and y, seeded droplets at
volume fraction 0.2 with radii in [6, 16] (seed 3). One "step" is one coupled time
step of the whole lattice: one launch of the fused collide-and-stream kernel, which
computes the capillary stencil's phi itself. The state (two copies of 21.5 GB) is far
larger than the 129 MB L2, so no flush is needed between timed steps.

Prints one JSON line. --impl reference times the FP64 CPU oracle instead (the
reference arm of this method), on a bounded slab of the same workload.
"""
import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled-step MLUPS at 512^3 + % HBM roofline; FP16-store and adjoint vs FP32"
N = 512
# bytes each node reads and writes per step: 40 populations; 16-bit storage keeps the
# four rest populations g_0, h^A_0, h^B_0, f_0 in FP32 (36 x 2 B + 4 x 4 B = 88 B each way)
ALG_BYTES_PER_NODE = {"f32": 320.0, "f16": 176.0, "bf16": 176.0, "f64": 640.0}
# DRAM bytes (read + write) per node of one fused_flow_kernel<float> launch, from an ncu capture
# of this kernel at 192^3; traffic scales with the
# node count. Set to None whenever the kernel changes until it is captured again.
NCU_DRAM_BYTES_PER_NODE_F32 = 164.05 + 153.90


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-planes", type=int, default=16)
    ap.add_argument("--cpu-sample-steps", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle leg (profiling runs)")
    ap.add_argument("--adjoint-only", action="store_true", help="time only the adjoint variant (profiling runs)")
    ap.add_argument("--drift", type=int, default=0, metavar="STEPS",
                    help="instead of the bench: the 384^3 drift study of sum phi and sum c (FP32 vs 16-bit)")
    ap.add_argument("--ripening-law", type=int, default=0, metavar="STEPS",
                    help="instead of the bench: <R>^3 against t on the 256^3 (3D) and 4096^2 (2D) ripening runs")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="population storage of the main line (profiling runs; the headline is f32)")
    ap.add_argument("--slabs", default="", metavar="N[,N...]",
                    help="instead of the bench: the 512^3 FP32 step split into N z slabs on this GPU "
                         "(halo exchange by device copies), against the undivided lattice")
    ap.add_argument("--adjoint-steps", type=int, default=200)
    ap.add_argument("--adjoint-k", type=int, default=100, help="checkpoint interval of the adjoint variant")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_workload(n, device, storage="f32"):
    from workloads import configs
    p, fields = configs.sedimentation(n=n, storage=storage)
    phi0, cA0, cB0 = fields(device=device)
    return p, fields, (phi0, cA0, cB0)


def host_info():
    """Core count and CPU model of the host the oracle is timed on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:                    # a description only: never let it stop the benchmark
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.machine()}


def cpu_baseline(init_fields, p, planes, steps):
    """The FP64 oracle, as it stands, on a z-slab of the same initial fields."""
    import torch
    from oracle.lbm import OracleLBM
    z0 = p.nz // 2 - planes // 2
    sl = [t[z0:z0 + planes].detach().cpu().double() for t in init_fields]
    q = p.with_(nz=planes)
    o = OracleLBM(q)
    o.init(*sl)
    o.step(1)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    mlups = q.nodes * steps / dt / 1e6
    return {"value": mlups, "unit": "MLUPS", "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"{q.nx}x{q.ny}x{planes} slab (z {z0}..{z0 + planes - 1}) of the {p.nx}x{p.ny}x{p.nz} "
                      f"initial fields, walls at the slab ends, {steps} steps after 1 untimed, {dt:.1f} s",
            "host": host_info()}


def time_device(sim, steps, warmup, dist):
    """Device-timed K steps with CUDA events on the simulation's stream, plus per-kernel
    event timing of the same region from the library."""
    import torch
    sim.step(warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    sim.profile_begin(steps)
    start.record(sim.stream)
    sim.step(steps)
    stop.record(sim.stream)
    torch.cuda.synchronize()
    ms = start.elapsed_time(stop)
    ms_phi, ms_step, nprof = sim.profile_end()
    if dist:
        ms = max_over_ranks(ms, dist, "cuda")
    return ms, ms_phi / max(nprof, 1), ms_step / max(nprof, 1)


def max_over_ranks(value, dist, device):
    """The largest of every rank's value (the job's time is its slowest replica's)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world_size, nodes_per_rank, steps, ms_max):
    """Whole-job throughput: every rank advances its own replica of nodes_per_rank nodes."""
    return world_size * nodes_per_rank * steps / (ms_max / 1e3) / 1e6


def time_adjoint(device, n=128, steps=200, K=100):
    """Cost of the hand-written adjoint on the 128^3 ripening workload (FP32, no flow):
    forward ms/step vs backward ms/step (recompute from checkpoints + adjoint sweep)."""
    import torch
    from workloads import configs
    from paper_2409_03401_gb300.adjoint import CoupledRun, forward_fields, misfit
    p, fields = configs.adjoint_problem(n=n)
    phi0, cA0, cB0 = fields(device=device)
    target = forward_fields(p, configs.THETA_TARGET, phi0, cA0, cB0, steps, device=device)

    def run():
        th = torch.tensor(configs.THETA_EVAL, dtype=torch.float64, requires_grad=True)
        p0 = phi0.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = CoupledRun.apply(p0, th, p, cA0, cB0, steps, K)
        L = misfit(out, target)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        L.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        return t1 - t0, t2 - t1, th

    run()                                            # warm-up (module loading, allocator)
    fwd, bwd, th = run()
    return {"workload": f"{n}^3 ripening, FP32, {steps} steps, checkpoint every {K}",
            "forward_ms_per_step": fwd / steps * 1e3,
            "backward_ms_per_step": bwd / steps * 1e3,
            "backward_over_forward": bwd / fwd,
            "timing": "wall clock around CoupledRun.apply + misfit (forward, with checkpoints) and "
                      "L.backward() (recompute from checkpoints + adjoint sweep), synchronised, after one warm-up run",
            "alg_bytes_per_node": {"forward": 168, "recompute": 168, "adjoint_step": 252},
            "grad_theta": [float(v) for v in th.grad]}


def run_e2e(p, init, steps, device):
    """Same metric through the public API with host buffers: pinned host inputs copied
    in, init, K steps, phi and mu copied out, FP64 sums read back, all in the timed region."""
    import torch
    from paper_2409_03401_gb300 import Simulation
    host = [t.cpu().pin_memory() for t in init]       # staged on the host before the timed region
    out_host = {k: torch.empty(p.shape, dtype=torch.float32).pin_memory() for k in ("phi", "muA", "muB")}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dev = [t.to(device, non_blocking=True) for t in host]
    sim = Simulation(p, *dev, device=device)
    sim.step(steps)
    f = sim.fields(names=("phi", "muA", "muB"))
    for k in out_host:
        out_host[k].copy_(f[k], non_blocking=True)
    sums = sim.sums()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h2d = sum(t.numel() * t.element_size() for t in host)
    d2h = sum(t.numel() * t.element_size() for t in out_host.values()) + 8 * len(sums)
    del sim, dev, f
    return {"value": p.nodes * steps / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "steps": steps, "seconds": dt}


def config_of(args, p, ws):
    """The workload both arms report (the reference arm times bounded samples of it)."""
    label = {"f32": "FP32", "f16": "FP16", "bf16": "BF16"}[args.storage]
    return {"workload": f"{args.n}^3 coupled step: D3Q19 flow + D3Q7 phi/cA/cB, {label} storage, "
                        "walls at z ends, droplets 0.2 vol. frac., r in [6,16], seed 3",
            "lattice": [p.nx, p.ny, p.nz], "storage": args.storage,
            "l2": "state 21.5 GB >> 129 MB L2, no flush", "parallelism": f"replicas x{ws}"}


def gb300(args):
    import torch
    ws, rank, local = dist_env()
    if args.adjoint_only:
        torch.cuda.set_device(local)
        print(json.dumps({"adjoint": time_adjoint(torch.device("cuda", local), steps=args.adjoint_steps,
                                                  K=args.adjoint_k)}))
        return
    dist = None
    if ws > 1:
        import torch.distributed as td
        td.init_process_group("nccl")
        dist = td
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_2409_03401_gb300 import Simulation

    p, fields_fn, init = make_workload(args.n, device, args.storage)
    sim = Simulation(p, *init, device=device)
    peak, peak_kind = peaks()
    with ClockSampler(local) as clk:
        ms, ms_phi, ms_step = time_device(sim, args.steps, args.warmup, dist)
    s = sim.sums()
    nodes = p.nodes
    value = job_mlups(ws, nodes, args.steps, ms)
    bytes_step = ALG_BYTES_PER_NODE[args.storage] * nodes
    achieved = bytes_step / (ms_step / 1e3) / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": config_of(args, p, ws),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (None if NCU_DRAM_BYTES_PER_NODE_F32 is None or args.storage != "f32"
                                 else NCU_DRAM_BYTES_PER_NODE_F32 * nodes),
                     "kernel": f"fused_flow_kernel<{'float' if args.storage == 'f32' else args.storage}, BGK> "
                               "(z-marching fused phi + collide + stream)",
                     "alg_bytes_per_launch": bytes_step, "ms_per_launch": ms_step,
                     "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                     "whole_step_frac": bytes_step / (ms / args.steps / 1e3) / 1e9 / peak,
                     "phi_pass_ms": ms_phi},
        "gpu_launches": sim.kernels_per_step * args.steps,
        "clocks": clk.summary(),
        "diagnostics": {"nonfinite": s["nonfinite"], "sum_cA": s["cA"], "umax": s["umax"]},
    }
    del sim
    torch.cuda.synchronize()

    if not args.no_variants:
        var = {}
        for storage in ("f16", "bf16"):
            q = p.with_(storage=storage)
            v = Simulation(q, *init, device=device)
            vms, _, vstep = time_device(v, max(20, args.steps // 2), args.warmup, dist)
            vs = max(20, args.steps // 2)
            vb = ALG_BYTES_PER_NODE[storage] * nodes
            var[storage] = {"value": ws * nodes * vs / (vms / 1e3) / 1e6, "unit": "MLUPS",
                            "ms_per_step": vms / vs, "speedup_vs_f32": (ms / args.steps) / (vms / vs),
                            "alg_bytes_per_node": ALG_BYTES_PER_NODE[storage],
                            "roofline_frac": vb / (vstep / 1e3) / 1e9 / peak}
            del v
            torch.cuda.synchronize()
        # the two-relaxation-time flow collision on the same workload, FP32 storage
        q = p.with_(collision="TRT")
        v = Simulation(q, *init, device=device)
        vs = max(20, args.steps // 2)
        vms, _, vstep = time_device(v, vs, args.warmup, dist)
        var["trt"] = {"value": ws * nodes * vs / (vms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": vms / vs,
                      "speedup_vs_f32": (ms / args.steps) / (vms / vs), "collision": "TRT, Lambda = 3/16",
                      "roofline_frac": ALG_BYTES_PER_NODE["f32"] * nodes / (vstep / 1e3) / 1e9 / peak}
        del v
        torch.cuda.synchronize()
        # the in-place layout (one AA-pattern copy: half the memory of the two-buffer fused
        # kernel), FP32: a phi pass, then the per-node AA step reading phi from it
        q = p.with_(inplace=True)
        v = Simulation(q, *init, device=device)
        vs = max(20, args.steps // 2)
        vms, vphi, vstep = time_device(v, vs, args.warmup, dist)
        var["inplace"] = {"value": ws * nodes * vs / (vms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": vms / vs,
                          "speedup_vs_f32": (ms / args.steps) / (vms / vs),
                          "kernels": "phi_kernel + step_kernel (AA pattern, in place)",
                          "phi_pass_ms": vphi, "step_kernel_ms": vstep, "state_gb": v.state.numel() / 1e9,
                          "roofline_frac": ALG_BYTES_PER_NODE["f32"] * nodes / (vms / vs / 1e3) / 1e9 / peak}
        del v
        torch.cuda.synchronize()
        # the same in-place layout with FP16 storage (10.7 GB of state at 512^3)
        q = p.with_(inplace=True, storage="f16")
        v = Simulation(q, *init, device=device)
        vs = max(20, args.steps // 2)
        vms, vphi, vstep = time_device(v, vs, args.warmup, dist)
        var["inplace_f16"] = {"value": ws * nodes * vs / (vms / 1e3) / 1e6, "unit": "MLUPS",
                              "ms_per_step": vms / vs, "speedup_vs_f32": (ms / args.steps) / (vms / vs),
                              "kernels": "phi_kernel + step_kernel (AA pattern, in place), FP16 storage",
                              "phi_pass_ms": vphi, "step_kernel_ms": vstep, "state_gb": v.state.numel() / 1e9,
                              "alg_bytes_per_node": ALG_BYTES_PER_NODE["f16"],
                              "roofline_frac": ALG_BYTES_PER_NODE["f16"] * nodes / (vms / vs / 1e3) / 1e9 / peak}
        del v
        torch.cuda.synchronize()
        # the multiple-relaxation-time flow collision (D3Q19 moment basis), FP32 storage
        q = p.with_(collision="MRT")
        v = Simulation(q, *init, device=device)
        vs = max(20, args.steps // 2)
        vms, _, vstep = time_device(v, vs, args.warmup, dist)
        var["mrt"] = {"value": ws * nodes * vs / (vms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": vms / vs,
                      "speedup_vs_f32": (ms / args.steps) / (vms / vs), "collision": "MRT, d'Humieres rates",
                      "roofline_frac": ALG_BYTES_PER_NODE["f32"] * nodes / (vstep / 1e3) / 1e9 / peak}
        del v
        torch.cuda.synchronize()
        # D3Q19 for phi, c^A, c^B (the paper's lattice for every equation): 76 populations,
        # phi pass + per-node pull step, FP32 storage
        q = p.with_(lattice="D3Q19")
        v = Simulation(q, *init, device=device)
        vs = max(10, args.steps // 10)
        vms, _, _ = time_device(v, vs, args.warmup, dist)
        b19 = 2 * 76 * 4.0
        var["d3q19_scalars"] = {"value": ws * nodes * vs / (vms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": vms / vs,
                                "alg_bytes_per_node": b19, "kernels": "phi_kernel + step_kernel (pull)",
                                "roofline_frac": b19 * nodes / (vms / vs / 1e3) / 1e9 / peak}
        del v
        torch.cuda.synchronize()
        # 3D ripening without flow (256^3, D3Q7, FP32, in place): 21 populations, 168 B/node
        from workloads import configs
        p3, f3 = configs.ripening()
        v = Simulation(p3, *f3(device=device), device=device)
        vs = max(20, args.steps // 2)
        vms, _, _ = time_device(v, vs, args.warmup, dist)
        s3 = v.sums()
        b3 = 2 * 21 * 4.0
        var["ripening_3d"] = {"value": ws * p3.nodes * vs / (vms / 1e3) / 1e6, "unit": "MLUPS",
                              "ms_per_step": vms / vs, "workload": "256^3 D3Q7, no flow, fraction 0.15, FP32, in place",
                              "alg_bytes_per_node": b3, "roofline_frac": b3 * p3.nodes / (vms / vs / 1e3) / 1e9 / peak,
                              "droplets_N": s3["euler"], "after_steps": args.warmup + vs}
        del v
        torch.cuda.synchronize()
        # 2D ripening without flow on D2Q9 (§4.2.2 table): 4096^2, 27 FP32 populations in place,
        # with the one-pass droplet count and mean radius of Eq. 67 after the timed steps
        from workloads import configs
        p2, f2 = configs.ripening_2d()
        v = Simulation(p2, *f2(device=device), device=device)
        vs = max(20, args.steps // 2)
        vms, _, _ = time_device(v, vs, args.warmup, dist)
        s2 = v.sums()
        b2 = 2 * 27 * 4.0
        n2 = p2.nodes
        var["ripening_2d"] = {"value": ws * n2 * vs / (vms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": vms / vs,
                              "workload": "4096^2 D2Q9, no flow, phase fraction 0.08, FP32, in place",
                              "alg_bytes_per_node": b2, "roofline_frac": b2 * n2 / (vms / vs / 1e3) / 1e9 / peak,
                              "droplets_N": s2["euler"], "mean_radius": s2["interface"] / (2 * math.pi * s2["euler"]),
                              "after_steps": args.warmup + vs}
        del v
        torch.cuda.synchronize()
        out["variants"] = var

    if not args.no_variants:
        out["variants"]["adjoint"] = time_adjoint(device, steps=args.adjoint_steps, K=args.adjoint_k)

    if not args.no_e2e:
        out["e2e"] = run_e2e(p, init, args.steps, device)

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(init, p, args.cpu_sample_planes, args.cpu_sample_steps)
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def reference(args):
    """The FP64 CPU oracle, as it stands, on the host cores: every step is one oracle step over
    a z-slab of the same 512^3 workload, the slab sized (2 to 16 planes) so that W + K steps
    take about a minute."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import torch
    from workloads import configs
    from oracle.lbm import OracleLBM
    p, fields_fn = configs.sedimentation(n=args.n)

    def slab(planes):
        z0 = p.nz // 2 - planes // 2
        q = p.with_(nz=planes)
        o = OracleLBM(q)
        o.init(*fields_fn(device="cpu", z_range=(z0, z0 + planes)))
        return q, o, z0
    q, o, _ = slab(2)                                  # calibration: rate of one step
    t0 = time.perf_counter()
    o.step(1)
    rate = q.nodes / (time.perf_counter() - t0)
    budget = 60.0
    planes = int(max(2, min(16, budget * rate / ((args.steps + args.warmup) * p.nx * p.ny))))
    q, o, z0 = slab(planes)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = q.nodes * args.steps / dt / 1e6
    sample = (f"{q.nx}x{q.ny}x{planes} slab (z {z0}..{z0 + planes - 1}) of the {args.n}^3 initial fields, "
              f"walls at the slab ends; {args.steps} timed steps after {args.warmup} untimed")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config_of(args, p, ws),
           "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": torch.get_num_threads(),
                            "kind": "oracle", "sample": sample, "host": host_info()},
           "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def drift_study(args):
    """Drift of the invariants sum c^A, sum c^B and of sum phi over a long run of the
    384^3 wall-bounded flow workload (droplets at 0.1, r in [8, 20]), FP32 against FP16 and
    BF16 storage; the FP64 sums come from the library's reduction."""
    import torch
    from workloads import configs
    from paper_2409_03401_gb300 import Simulation
    torch.cuda.set_device(0)
    p, fields = configs.drift()
    init = fields(device="cuda")
    every = max(1, args.drift // 10)
    runs = {}
    for storage in ("f32", "f16", "bf16"):
        sim = Simulation(p.with_(storage=storage), *init, device="cuda")
        series = []
        t0 = time.perf_counter()
        for t in range(0, args.drift + 1, every):
            if t:
                sim.step(every)
            s = sim.sums()
            series.append({"t": t, "phi": s["phi"], "cA": s["cA"], "cB": s["cB"], "p": s["p"], "umax": s["umax"],
                           "N": s["euler"]})
        torch.cuda.synchronize()
        runs[storage] = {"series": series, "seconds": time.perf_counter() - t0}
        del sim
        torch.cuda.empty_cache()
    ref = runs["f32"]["series"]
    out = {"study": "drift", "workload": "384^3, walls at z ends, D3Q19 flow + D3Q7, droplets 0.1, r in [8,20], seed 4",
           "steps": args.drift, "sample_every": every, "runs": {}}
    for storage, r in runs.items():
        s0, s1 = r["series"][0], r["series"][-1]
        out["runs"][storage] = {
            "rel_drift_cA": (s1["cA"] - s0["cA"]) / s0["cA"], "rel_drift_cB": (s1["cB"] - s0["cB"]) / s0["cB"],
            "max_rel_dev_phi_vs_f32": max(abs(a["phi"] - b["phi"]) / abs(b["phi"]) for a, b in zip(r["series"], ref)),
            "phi_change": (s1["phi"] - s0["phi"]) / s0["phi"], "umax_end": s1["umax"],
            "droplets_start": s0["N"], "droplets_end": s1["N"], "seconds": r["seconds"],
            "series": r["series"]}
    print(json.dumps(out))


def ripening_law(args):
    """<R>^3 against t. 3D (256^3, D3Q7, FP32): the Sauter radius R = 3 V / A from the
    volume V = sum phi and the interface area A = sum (4/W) phi (1 - phi), beside the droplet
    count N (Euler characteristic) and sqrt(A / (4 pi N)); 2D (4096^2, D2Q9):
    <R> = A / (2 pi N) of Eq. 67 with the droplet count N of the Euler characteristic. Least-
    squares line of <R>^3 over the second half of the run, with its R^2."""
    import torch
    from workloads import configs
    from paper_2409_03401_gb300 import Simulation
    torch.cuda.set_device(0)
    out = {"study": "ripening_law", "steps": args.ripening_law, "runs": {}}
    for name, build in (("3d_256", lambda: configs.ripening()), ("2d_4096", lambda: configs.ripening_2d())):
        p, fields = build()
        sim = Simulation(p, *fields(device="cuda"), device="cuda")
        every = max(1, args.ripening_law // 20)
        series = []
        for t in range(0, args.ripening_law + 1, every):
            if t:
                sim.step(every)
            s = sim.sums()
            if p.nz == 1:
                R = s["interface"] / (2 * math.pi * s["euler"]) if s["euler"] > 0 else float("nan")
                series.append({"t": t, "R": R, "N": s["euler"]})
            else:
                R_n = math.sqrt(s["interface"] / (4 * math.pi * s["euler"])) if s["euler"] > 0 else float("nan")
                series.append({"t": t, "R": 3.0 * s["phi"] / s["interface"], "N": s["euler"], "R_area_per_N": R_n})
        half = [e for e in series if e["t"] >= args.ripening_law / 2]
        ts = [e["t"] for e in half]
        ys = [e["R"] ** 3 for e in half]
        n = len(ts)
        mt, my = sum(ts) / n, sum(ys) / n
        sxx = sum((a - mt) ** 2 for a in ts)
        sxy = sum((a - mt) * (b - my) for a, b in zip(ts, ys))
        slope = sxy / sxx
        ss_res = sum((b - (my + slope * (a - mt))) ** 2 for a, b in zip(ts, ys))
        ss_tot = sum((b - my) ** 2 for b in ys)
        out["runs"][name] = {"R3_slope_per_step": slope, "R3_fit_r2": 1.0 - ss_res / ss_tot if ss_tot > 0 else None,
                             "series": series}
        del sim
        torch.cuda.empty_cache()
    print(json.dumps(out))


def slab_study(args):
    """Cost of the z-slab decomposition on one GPU: the same workload as the bench, advanced
    by a SlabGroup of N slabs (after every step each slab packs the populations leaving its
    faces, the neighbours unpack them, then phi of the edge planes goes the same way), timed
    with CUDA events around the steps and exchanges, against the undivided lattice."""
    import torch
    from paper_2409_03401_gb300 import Simulation
    from paper_2409_03401_gb300.slabs import SlabGroup
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    p, _, init = make_workload(args.n, device, "f32")
    steps = max(10, args.steps // 4)

    def timed(obj):
        obj.step(args.warmup)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        obj.step(steps)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    sim = Simulation(p, *init, device=device)
    ms0 = timed(sim)
    ref = sim.fields(("phi", "ux"))
    t_ref = sim.t
    del sim
    torch.cuda.synchronize()
    out = {"study": "slabs", "workload": f"{args.n}^3 FP32 flow (the bench workload), {steps} timed steps",
           "undivided_ms_per_step": ms0, "undivided_mlups": p.nodes / (ms0 / 1e3) / 1e6, "runs": {}}
    for n in [int(v) for v in args.slabs.split(",") if v]:
        grp = SlabGroup(p, n, *init)
        ms = timed(grp)
        same = grp.t == t_ref and all(torch.equal(grp.fields((k,))[k], ref[k]) for k in ref)
        out["runs"][str(n)] = {"ms_per_step": ms, "mlups": p.nodes / (ms / 1e3) / 1e6,
                               "overhead_vs_undivided": ms / ms0 - 1.0, "halo_bytes_per_face": grp.slabs[0].halo_bytes,
                               "fields_equal_to_undivided": bool(same)}
        del grp
        torch.cuda.synchronize()
    print(json.dumps(out))


def main():
    args = parse()
    if args.slabs:
        slab_study(args)
    elif args.drift:
        drift_study(args)
    elif args.ripening_law:
        ripening_law(args)
    elif args.impl == "reference":
        reference(args)
    else:
        gb300(args)


if __name__ == "__main__":
    main()
