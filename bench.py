"""Benchmark of the fused entropic lattice-BGK step on GB300.

Default workload (1 GPU): D3Q27, 512^3 periodic Taylor-Green vortex (u0 = 0.1, rho0 = 1,
Re = 1600 with nu = u0 (N / 2 pi) / Re), entropic equilibrium, populations stored as
binary16 f - w rho0 with FP32 collision, fused diagnostics every 10 steps.  One bench
step is one lattice time step of the whole grid.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W]
                  [--workload tgv3d|shear2d|tgv2d|batch|turb3d]
                  [--precision f16s|f32|f64] [--impl reference]
  python bench.py --accuracy [--workload tgv3d|shear2d|turb3d|batch] [--long-steps S]

--accuracy prints the long accuracy checks instead of a bench line: on the Taylor-Green
vortex the FP32 and binary16 velocity error against FP64 storage after four convective
times and the binary16-vs-FP32 energy and dissipation curves over 20000 steps; on the
shear layer the step at which each equilibrium first goes non-finite within 10000 steps.

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload
(rank 0 only).  Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (no data-path collective); the barrier and the max over ranks
bound the timed region.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GLUPS and % of HBM roofline; FP16-store vs FP32/FP64 at stated L2 velocity error"


def fp64_flops_per_cell(eq, bulk, D=2):
    """Algorithmic FP64 flops of one collision as the kernels write it (an FMA is two
    flops, a division or a square root one, a negation or a max none).
    D2Q9 entropic: the moment sums 15, rho^2 1, per axis 3j, T = sqrt(rho^2 + 3j^2) and
    q = rho + T (2 x 5), the one division of rho q_x q_y with its products (4), per axis u,
    S - 1, 3u, d(+1), d(-1) (2 x 9), drho 1, the rate terms 10 (1 - 2beta and, per weight
    class, 2beta w, 2beta w rho, 2beta w drho), t = 1 + d 3, per direction h and the
    relaxation 9 x 6.  Quadratic: moments 18 (the sums, 1/rho, two products), drho 1, rate
    terms 10, u^2 3, -3/2 u^2 1, the diagonal sums 2, 9 x 8.  Product form: moments 18,
    drho 1, rate terms 10, per-axis factors 2 x 7, t = 1 + d 3, 9 x 6.
    D3Q27 (the same conventions): moment sums 50; entropic: rho^2 1, per axis 3 x 5, the
    division with its products 7, per axis 3 x 9, drho 1, rate terms 13 (four weight
    classes), t = 1 + d 6, per (c_x, c_y) pair the partial products 9 x 3, per direction
    27 x 6.  Product form: moments 54, drho 1, rate terms 13, per-axis factors 3 x 7,
    t = 1 + d 6, 9 x 3, 27 x 6.  Quadratic: moments 54, drho 1, rate terms 13, u^2 5,
    -3/2 u^2 1, diagonal sums 2, 27 x 8 plus 18 c_z additions.  The bulk correction adds
    the rate formula (6 entropic, 5 otherwise)."""
    if D == 2:
        if eq == 0:
            return 15 + 1 + 10 + 4 + 18 + 1 + 10 + 3 + 54 + (6 if bulk else 0)
        base = 18 + 1 + 10
        if eq == 1:
            return base + 3 + 1 + 2 + 72 + (5 if bulk else 0)
        return base + 14 + 3 + 54 + (5 if bulk else 0)
    if eq == 0:
        return 50 + 1 + 15 + 7 + 27 + 1 + 13 + 6 + 27 + 162 + (6 if bulk else 0)
    if eq == 1:
        return 54 + 1 + 13 + 5 + 1 + 2 + 27 * 8 + 18 + (5 if bulk else 0)
    return 54 + 1 + 13 + 21 + 6 + 27 + 162 + (5 if bulk else 0)


def fp64_peak_gflops(sm_mhz):
    """FP64 peak of the GPU: 152 SMs x 2 FP64 FMA per cycle x 2 flops x the SM clock."""
    return 152 * 2 * 2 * (sm_mhz or 2070.0) / 1e3


PREC = {"f64": 0, "f32": 1, "f16s": 2}
ESIZE = {0: 8, 1: 4, 2: 2}
PREC_NAME = {0: "F64", 1: "F32", 2: "F16S"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--workload", default="tgv3d", choices=["tgv3d", "shear2d", "tgv2d", "batch", "turb3d"])
    p.add_argument("--precision", default=None, choices=list(PREC))
    p.add_argument("--bulk", type=int, default=0)
    p.add_argument("--eq", default="entropic", choices=["entropic", "poly2", "product"])
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--n", type=int, default=None, help="lattice side (default: the workload's)")
    p.add_argument("--diag-every", type=int, default=10)
    p.add_argument("--no-extras", action="store_true", help="skip the comparison runs")
    p.add_argument("--cpu-seconds", type=float, default=3.0,
                   help="length of each of the 3 timed oracle runs of the CPU baseline")
    p.add_argument("--batch-count", type=int, default=4096, help="instances of the batch workload")
    p.add_argument("--accuracy", action="store_true",
                   help="only run the long accuracy checks of the workload (Taylor-Green: FP32 and "
                        "binary16 against FP64; shear layer: divergence step) and print them")
    p.add_argument("--long-steps", type=int, default=None,
                   help="steps of the long accuracy runs (Taylor-Green 20000, shear layer 10000)")
    p.add_argument("--shape", default=None,
                   help="fixed launch shape (no tuning): kernel,threads,stages,rows,seg,cap; "
                        "for the batch workload threads,blocks")
    p.add_argument("--no-tune", action="store_true",
                   help="keep the default (or cached) launch shape instead of autotuning")
    return p.parse_args()


# ----------------------------------------------------------------------------- workloads

def workload(args):
    """Workload description: lattice, dims, tau, precision, field recipe."""
    eq = {"entropic": 0, "poly2": 1, "product": 2}[args.eq]
    if args.workload == "tgv3d":
        n = args.n or 512
        u0 = 0.1
        nu = u0 * (n / (2 * math.pi)) / 1600.0
        prec = PREC[args.precision or "f16s"]
        return dict(name=f"D3Q27 {n}^3 periodic Taylor-Green vortex (u0=0.1, rho0=1, Re=1600)",
                    D=3, dims=(n, n, n), tau=0.5 + 3 * nu, prec=prec, eq=eq, u0=u0)
    if args.workload == "turb3d":
        n = args.n or 512
        prec = PREC[args.precision or "f16s"]
        return dict(name=f"D3Q27 {2 * n}x{n}x{n} periodic decaying isotropic turbulence "
                         f"(E(k) ~ k^4 exp(-2 (k/8)^2), u_rms=0.05)",
                    D=3, dims=(2 * n, n, n), tau=0.5 + 1e-4, prec=prec, eq=eq, u0=0.05)
    if args.workload == "shear2d":
        n = args.n or 4096
        prec = PREC[args.precision or "f32"]
        return dict(name=f"D2Q9 {n}^2 periodic double shear layer (u0=0.1, kappa=80, delta=0.05)",
                    D=2, dims=(n, n, 1), tau=0.5 + 3e-5, prec=prec, eq=eq, u0=0.1)
    if args.workload == "tgv2d":
        n = args.n or 64
        prec = PREC[args.precision or "f64"]
        return dict(name=f"D2Q9 {n}^2 periodic Taylor-Green vortex (u0=0.05, tau=0.8)",
                    D=2, dims=(n, n, 1), tau=0.8, prec=prec, eq=eq, u0=0.05)
    return dict(name=f"{args.batch_count} independent D2Q9 periodic lattices, sides log-uniform in [16,256], "
                     "one shear or acoustic wave each (amplitude 1e-4), FP64",
                D=2, dims=None, tau=None, prec=0, eq=eq, u0=0.3)


def fields_device(w, torch, dev):
    """Initial fields as float32 device tensors (flat rho, u[D][ncell])."""
    D, (nx, ny, nz) = w["D"], w["dims"]
    if "turbulence" in w["name"]:
        from paper_2303_08163_gb300 import inputs
        return inputs.random_solenoidal_torch((nx, ny, nz), u_rms=0.05, device=dev)
    if w["name"].startswith("D3Q27"):
        n = nx
        t = torch.arange(n, device=dev, dtype=torch.float64) * (2 * math.pi / n)
        s, c, c2 = torch.sin(t), torch.cos(t), torch.cos(2 * t)
        u0 = w["u0"]
        ux = u0 * c[:, None, None] * c[None, :, None] * s[None, None, :]
        uy = -u0 * c[:, None, None] * s[None, :, None] * c[None, None, :]
        rho = 1.0 + u0 * u0 * 3.0 / 16.0 * (c2[None, :, None] + c2[None, None, :]) * (c2[:, None, None] + 2.0)
        u = torch.stack([ux.reshape(-1), uy.reshape(-1), torch.zeros_like(ux).reshape(-1)])
        return rho.reshape(-1).float().contiguous(), u.float().contiguous()
    from paper_2303_08163_gb300 import inputs
    if "shear" in w["name"]:
        rho, u = inputs.double_shear_layer(nx, dtype=np.float32)
    else:
        rho, u = inputs.taylor_green_2d(nx, u0=w["u0"])
    return (torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).to(dev))


# ------------------------------------------------------------------------------- helpers

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        load = [v for v, r in zip(sm, rows) if float(r[3]) > 200.0] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def source_hash():
    """Hash of the step-kernel sources, to match committed ncu traffic to the code."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2303_08163_gb300", "csrc")
    for name in ("k_tma.cuh", "lbm_device.cuh", "lbm_common.cuh", "ptx.cuh", "k_generic_step.cuh", "k_batch.cu"):
        h.update(open(os.path.join(d, name), "rb").read())
    return h.hexdigest()[:16]


LAUNCH_KEYS = ("threads", "blocks", "stages", "rows", "seg", "smem_bytes")


def traffic_records():
    try:
        return json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    except (OSError, ValueError):
        return []


def ncu_traffic(kernel, workload_name, units, launch=None, precision=None):
    """DRAM bytes per launch from the committed ncu records, scaled to `units` (cells, or
    cell updates for the batch) and the reason when there is none.  A record counts only
    for the kernel source it was taken on (the step-kernel source hash) and, for the
    single-lattice kernels, for the exact launch shape that ran (threads, blocks, stages,
    rows, segment, shared memory): another shape moves other bytes."""
    recs = [r for r in traffic_records() if r.get("kernel") == kernel and r.get("workload") == workload_name
            and (precision is None or r.get("precision") == precision)]
    if not recs:
        return None, "no ncu record for this kernel, workload and storage precision"
    recs = [r for r in recs if r.get("source_hash") == source_hash()]
    if not recs:
        return None, "the kernel source changed since the ncu records were taken"
    if launch is not None:
        recs = [r for r in recs if all(r.get("launch", {}).get(k) == launch.get(k) for k in LAUNCH_KEYS)]
        if not recs:
            shape = {k: launch.get(k) for k in LAUNCH_KEYS}
            return None, f"no ncu record for the launch shape that ran {shape}"
    return recs[0]["dram_bytes_per_cell"] * units, recs[0].get("captured_on")


def fp64_pipe(workload_name, bulk, launch, glups, sm_mhz):
    """FP64-pipe instruction roofline of an FP64-storage run from the committed ncu record of
    the same kernel source, workload, bulk setting and launch kind: executed FP64 thread
    instructions per cell update x GLUPS against the pipe's 2 instructions per SM per
    cycle (DADD, DMUL and DFMA alike).  None when no such record exists."""
    kname = "k_step_tma" if launch.get("kernel") == 2 else "k_step_generic"
    for r in traffic_records():
        if (r.get("kernel") == kname and r.get("workload") == workload_name and r.get("precision") == "F64"
                and r.get("bulk_corr") == bulk and r.get("source_hash") == source_hash()
                and r.get("launch", {}).get("threads") == launch.get("threads")
                and r.get("fp64_thread_inst_per_cell")):
            ipc = r["fp64_thread_inst_per_cell"]
            peak = 152 * 2 * (sm_mhz or 2070.0) / 1e3
            return {"fp64_thread_inst_per_cell_update": ipc, "achieved_ginst_s": ipc * glups,
                    "peak_ginst_s": peak, "frac": ipc * glups / peak, "source": r.get("captured_on")}
    return None


def aggregate(world, cells_per_rank, steps, rank_ms):
    """Whole-job GLUPS: every rank advances its own replica; the slowest rank's time
    bounds the job (weak scaling)."""
    return world * cells_per_rank * steps / (max(rank_ms) * 1e-3) / 1e9


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), ws


# ----------------------------------------------------------------------- CPU baseline leg

def cpu_info():
    """Model name and core counts of the host (reported beside the oracle timings)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    import platform
    return {"model": model or platform.machine(), "logical_cpus": os.cpu_count(), "usable_cpus": usable}


def cpu_sample(w):
    """The bounded sample of the workload the CPU oracle is timed on: (D, dims, eq, tau,
    rho, u, description).  Taylor-Green: the same vortex at 128^3; turbulence: the same
    spectrum on a 128 x 64 x 64 box; shear layer: the same layer at 1024^2; the small
    Taylor-Green configuration: itself; the batch: the 64^2 instance table's first
    instance kind at 256^2 (one shear wave on U0 = 0.1)."""
    from paper_2303_08163_gb300 import inputs
    D, eq = w["D"], w["eq"]
    if w["dims"] is None:
        dims = (256, 256, 1)
        table = {"nx": [256], "ny": [256], "nmode": [2], "U0": [0.1], "tau": [0.8], "kind": [0], "amp": 1e-4}
        rho, u = inputs.linear_mode_fields(table, 0)
        return D, dims, eq, 0.8, rho, u, "a D2Q9 256^2 lattice with one shear wave (amplitude 1e-4) on U0 = 0.1"
    if "turbulence" in w["name"]:
        dims = (128, 64, 64)
        rho, u = inputs.random_solenoidal(dims, u_rms=0.05)
        return D, dims, eq, w["tau"], rho, u, "the turbulence spectrum on a 128 x 64 x 64 box"
    if D == 3:
        n = 128
        rho, u = inputs.taylor_green_3d(n, u0=w["u0"])
        return D, (n, n, n), eq, w["tau"], rho, u, "the Taylor-Green vortex at 128^3 (same u0 and tau)"
    if "shear" in w["name"]:
        n = 1024
        rho, u = inputs.double_shear_layer(n)
        return D, (n, n, 1), eq, w["tau"], rho, u, "the double shear layer at 1024^2 (same tau)"
    n = w["dims"][0]
    rho, u = inputs.taylor_green_2d(n, u0=w["u0"])
    return D, (n, n, 1), eq, w["tau"], rho, u, f"the whole {n}^2 Taylor-Green workload"


def time_oracle(D, dims, eq, bulk, tau, f, threads, seconds, reps=3):
    """Median over `reps` runs of the oracle's GLUPS on state f with `threads` host
    threads, each run a whole number of steps of about `seconds`; returns (GLUPS, steps)."""
    from oracle import core
    used = core.set_threads(threads)
    try:
        t0 = time.perf_counter()
        core.step(D, dims, eq, bulk, tau, 1, f)
        one = time.perf_counter() - t0
        steps = max(1, int(round(seconds / max(one, 1e-6))))
        rates = []
        for _ in range(reps):
            t0 = time.perf_counter()
            core.step(D, dims, eq, bulk, tau, steps, f)
            rates.append(int(np.prod(dims)) * steps / (time.perf_counter() - t0) / 1e9)
    finally:
        core.set_threads(1)
    return statistics.median(rates), steps, used


def oracle_baseline(w, bulk, seconds=4.0):
    """The FP64 CPU oracle as it stands, timed on the host cores on a bounded sample of the
    workload: all cores (OpenMP over the rows of the lattice; the cells and their
    arithmetic are the same as with one thread, bit for bit) and a single thread, each the
    median of 3 runs of about `seconds`."""
    from oracle import core
    D, dims, eq, tau, rho, u, what = cpu_sample(w)
    f = core.init(D, dims, eq, rho, u)
    info = cpu_info()
    g_all, n_all, used = time_oracle(D, dims, eq, bulk, tau, f, info["usable_cpus"] or 1, seconds)
    g_one, n_one, _ = time_oracle(D, dims, eq, bulk, tau, f, 1, seconds)
    lat = f"D{D}Q{3 ** D} {'x'.join(str(d) for d in dims if d > 1)}"
    return {"value": g_all, "unit": "GLUPS", "cores": used, "kind": "oracle",
            "sample": (f"FP64 CPU oracle on {lat}: {what}; median of 3 runs of {n_all} steps on {used} "
                       f"threads (single thread: {n_one} steps)"),
            "single_thread": {"value": g_one, "unit": "GLUPS", "cores": 1},
            "cpu_model": info["model"], "host_logical_cpus": info["logical_cpus"],
            "host_usable_cpus": info["usable_cpus"]}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, as it stands, on the host cores; each step
    is one oracle step of the bounded sample the cpu_baseline leg times (all cores)."""
    rank, _, ws = dist_env()
    if rank != 0:
        return
    w = workload(args)
    from oracle import core
    D, dims, eq, tau, rho, u, what = cpu_sample(w)
    ncell = int(np.prod(dims))
    f = core.init(D, dims, eq, rho, u)
    info = cpu_info()
    used = core.set_threads(info["usable_cpus"] or 1)
    # W warm-up steps, then exactly K timed steps, each run as one oracle call (the
    # wrapper copies the state once per call, not once per step)
    if args.warmup > 0:
        f = core.step(D, dims, eq, args.bulk, tau, args.warmup, f)
    t0 = time.perf_counter()
    f = core.step(D, dims, eq, args.bulk, tau, args.steps, f)
    dt = time.perf_counter() - t0
    core.set_threads(1)
    glups = ncell * args.steps / dt / 1e9
    lat = f"D{D}Q{3 ** D} {'x'.join(str(d) for d in dims if d > 1)}"
    sample = f"each step: one FP64 CPU-oracle step of {lat} ({what}) on {used} threads"
    line = {"impl": "reference", "metric": METRIC, "value": glups, "unit": "GLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["name"], "sample": sample},
            "cpu_baseline": {"value": glups, "unit": "GLUPS", "cores": used, "kind": "oracle", "sample": sample,
                             "cpu_model": info["model"], "host_logical_cpus": info["logical_cpus"]},
            "e2e": {"value": glups, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------- native arm

def timed_steps(torch, lat, steps, diag_every, stream):
    """Run `steps` steps with an event pair around each; returns (total ms, per-step ms,
    indices of steps that carried fused diagnostics)."""
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    t_first = lat.step_count
    evs[0].record(stream)
    for s in range(steps):
        lat.step(1)
        evs[s + 1].record(stream)
    evs[-1].synchronize()
    per = [evs[s].elapsed_time(evs[s + 1]) for s in range(steps)]
    diag_steps = [s for s in range(steps) if diag_every > 0 and (t_first + s) % diag_every == 0]
    return evs[0].elapsed_time(evs[-1]), per, diag_steps


def precision_errors(torch, lbm, dev, n=128, every=5):
    """Errors of the F32 and F16S storage paths against the FP64 path (equal to the CPU
    oracle to 1e-12 in the parity tests) on two Taylor-Green cases:
    (1) D3Q27 n^3 at Re = 1600 over four convective times n / (2 pi u0): the relative L2
        velocity error at the end, and the relative error of the kinetic-energy decay rate
        (least-squares slope of -ln E(t) over the window, E from the fused diagnostics
        every `every` steps);
    (2) the small D2Q9 configuration (64^2, u0 = 0.05, tau = 0.8, 1000 steps), whose energy
        decays as exp(-2 nu (k_x^2 + k_y^2) t): the relative error of the fitted rate and the
        relative L2 velocity error after 1000 steps."""
    from paper_2303_08163_gb300 import fits, inputs
    u0 = 0.1
    nu = u0 * (n / (2 * math.pi)) / 1600.0
    tau = 0.5 + 3 * nu
    steps = int(round(4 * n / (2 * math.pi * u0)))
    w = dict(name="D3Q27", D=3, dims=(n, n, n), u0=u0)
    rho, u = fields_device(w, torch, dev)
    us, rate = {}, {}
    for prec in (0, 1, 2):
        lat = lbm.Lattice(lbm.D3Q27, (n, n, n), tau, 0, 0, prec)
        lat.init_fields(rho, u, dtype=np.float32)
        lat.set_option(lbm.OPT_DIAG_EVERY, every)
        lat.step(steps)
        r = torch.empty(n ** 3, device=dev, dtype=torch.float64)
        v = torch.empty(3, n ** 3, device=dev, dtype=torch.float64)
        lat.moments(dtype=np.float64, out=(r, v))
        hist = lat.diag_history()
        rate[prec] = fits.energy_decay_rate([h["step"] for h in hist], [h["kinetic"] for h in hist])
        us[prec] = v
        lat.close()
    out = {"case": f"D3Q27 {n}^3 Taylor-Green, Re=1600, {steps} steps (4 convective times)",
           "reference": "FP64 GPU path (equal to the CPU oracle to 1e-12 in the parity tests)"}
    for prec in (1, 2):
        out[PREC_NAME[prec]] = float(torch.linalg.norm(us[prec] - us[0]) / torch.linalg.norm(us[0]))
    out["decay_rate"] = {"definition": "least-squares slope of -ln E(t) over the window, E every "
                                       f"{every} steps; error = |rate / rate_F64 - 1|",
                         "F64_per_step": rate[0]}
    for prec in (1, 2):
        out["decay_rate"][PREC_NAME[prec]] = abs(rate[prec] / rate[0] - 1)
    del us
    torch.cuda.empty_cache()
    m, tau2, steps2 = 64, 0.8, 1000
    rho2, u2 = inputs.taylor_green_2d(m, u0=0.05)
    rate2, vel2 = {}, {}
    for prec in (0, 1, 2):
        lat = lbm.Lattice(lbm.D2Q9, (m, m, 1), tau2, 0, 0, prec)
        lat.set_option(lbm.OPT_DIAG_EVERY, 50)
        lat.init_fields(rho2, u2)
        lat.step(steps2 + 1)
        hist = lat.diag_history()
        rate2[prec] = fits.energy_decay_rate([h["step"] for h in hist], [h["kinetic"] for h in hist], skip=2)
        lat.close()
        lat = lbm.Lattice(lbm.D2Q9, (m, m, 1), tau2, 0, 0, prec)
        lat.init_fields(rho2, u2)
        lat.step(steps2)
        vel2[prec] = lat.moments()[1]
        lat.close()
    k = 2 * math.pi / m
    small = {"case": "D2Q9 64^2 Taylor-Green, u0=0.05, tau=0.8, 1000 steps",
             "definition": "least-squares slope of -ln E(t), E every 50 steps from step 100; "
                           "error = |rate / rate_F64 - 1|",
             "F64_rate_per_step": rate2[0], "theory_2nu_k2": 2 * (tau2 - 0.5) / 3 * 2 * k * k}
    for prec in (1, 2):
        small[PREC_NAME[prec]] = {"decay_rate_error": abs(rate2[prec] / rate2[0] - 1),
                                  "rel_l2_velocity": float(np.linalg.norm(vel2[prec] - vel2[0])
                                                           / np.linalg.norm(vel2[0]))}
    out["small_taylor_green_2d"] = small
    return out


def run_native(args):
    import torch
    from paper_2303_08163_gb300 import lbm

    rank, local, ws = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lbm.load()
    stream = torch.cuda.current_stream()
    w = workload(args)
    if w["dims"] is None:
        if args.accuracy:
            if rank == 0:
                steps = args.long_steps or 4000
                res = [batch_mode_sweep(lbm, eq, args.bulk, steps=steps) for eq in (0, 1)]
                print(json.dumps({"accuracy": res, "workload": w["name"]}), flush=True)
            return
        return run_batch(args, w, torch, lbm, dev, rank, ws)
    D, dims, prec = w["D"], w["dims"], w["prec"]
    Q = 3 ** D
    ncell = int(np.prod(dims))
    if args.accuracy:
        rho, u = fields_device(w, torch, dev)
        if rank == 0:
            if D == 3 and "Taylor" in w["name"]:
                args.long_steps = args.long_steps or 20000
                res = accuracy_gates(torch, lbm, dev, w, args, rho, u)
            elif "turbulence" in w["name"]:
                # the configured viscosity (tau - 1/2 = 1e-4) does not resolve this box and
                # is reported as is; nu = 0.01 resolves it (Kolmogorov scale about a cell)
                steps = args.long_steps or 5000
                res = {"configured": energy_decay_compare(torch, lbm, w, args, rho, u, steps=steps),
                       "nu_0.01": energy_decay_compare(torch, lbm, dict(w, tau=0.5 + 3 * 0.01), args, rho, u,
                                                       steps=steps)}
            else:
                res = shear_divergence(torch, lbm, w, args, rho, u, steps=args.long_steps or 10000)
            print(json.dumps({"accuracy": res, "workload": w["name"]}), flush=True)
        return
    lat = lbm.Lattice(lbm.D3Q27 if D == 3 else lbm.D2Q9, dims, w["tau"], w["eq"], args.bulk, prec)
    rho, u = fields_device(w, torch, dev)
    lat.init_fields(rho, u, dtype=np.float32)
    if args.shape:
        lat.set_launch_shape(*[int(v) for v in args.shape.split(",")])
    elif not args.no_tune:
        lat.set_option(lbm.OPT_TUNE, 1)
    lat.set_option(lbm.OPT_DIAG_EVERY, args.diag_every)
    lat.init_fields(rho, u, dtype=np.float32)
    for _ in range(args.warmup):
        lat.step(1)
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        total_ms, per, diag_steps = timed_steps(torch, lat, args.steps, args.diag_every, stream)
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = clk.summary()
    t_max = total_ms
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
        dist.barrier()
    hist = lat.diag_history()
    plain = [per[s] for s in range(len(per)) if s not in set(diag_steps)] or per
    launch_ms = statistics.mean(plain)
    algo_bytes = 2 * Q * ESIZE[prec] * ncell
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    achieved = algo_bytes / (launch_ms * 1e-3) / 1e9
    info = lat.launch_info()
    kname = "k_step_tma" if info["kernel"] == 2 else "k_step_generic"
    traffic, traffic_note = ncu_traffic(kname, w["name"], ncell, launch=info, precision=PREC_NAME[prec])
    glups = aggregate(ws, ncell, args.steps, [t_max])
    # end to end through the C ABI with pinned host buffers
    rho_h = rho.cpu().pin_memory()
    u_h = u.cpu().pin_memory()
    rout = torch.empty(ncell, dtype=torch.float32).pin_memory()
    uout = torch.empty(D, ncell, dtype=torch.float32).pin_memory()
    # untimed first host-buffer round trip (the library grows its staging buffers once)
    lat.init_fields(rho_h, u_h, dtype=np.float32)
    lat.moments(dtype=np.float32, out=(rout, uout))
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    hostt = [time.perf_counter()]
    ev[0].record(stream)
    lat.init_fields(rho_h, u_h, dtype=np.float32)
    ev[1].record(stream)
    hostt.append(time.perf_counter())
    lat.step(args.steps)
    ev[2].record(stream)
    hostt.append(time.perf_counter())
    lat.moments(dtype=np.float32, out=(rout, uout))
    ev[3].record(stream)
    ev[3].synchronize()
    hostt.append(time.perf_counter())
    e2e_ms = ev[0].elapsed_time(ev[3])
    in_ms, steps_ms, out_ms = (ev[q].elapsed_time(ev[q + 1]) for q in range(3))
    host_ms = [1e3 * (hostt[q + 1] - hostt[q]) for q in range(3)]
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    h2d_bytes = (rho_h.numel() + u_h.numel()) * 4
    d2h_bytes = (rout.numel() + uout.numel()) * 4
    e2e = {"value": ws * ncell * args.steps / (e2e_ms * 1e-3) / 1e9, "unit": "GLUPS",
           "h2d_bytes_per_step": h2d_bytes / args.steps,
           "d2h_bytes_per_step": d2h_bytes / args.steps,
           "path": "lbm_init_fields(host) + lbm_step(K) + lbm_moments(host), pinned buffers",
           # where the time goes: the field upload and the moment download run at the
           # host link's bandwidth (copy plus the init / moments kernel)
           "breakdown_ms": {"init_fields_from_host": in_ms, "steps": steps_ms, "moments_to_host": out_ms,
                            "host_clock": host_ms},
           "host_link_GB_s": {"h2d": h2d_bytes / (in_ms * 1e-3) / 1e9, "d2h": d2h_bytes / (out_ms * 1e-3) / 1e9}}
    launches = args.steps + len(diag_steps)
    extras = {}
    if not args.no_extras and rank == 0:
        lat.close()
        del lat
        torch.cuda.empty_cache()
        extras["precision_compare"] = compare_precisions(torch, lbm, dev, w, args, rho, u,
                                                         sm_mhz=clocks.get("sm_mhz"))
        if "turbulence" in w["name"]:
            extras["energy_decay"] = energy_decay_compare(torch, lbm, w, args, rho, u)
        elif "shear" in w["name"]:
            extras["divergence"] = shear_divergence(torch, lbm, w, args, rho, u)
        elif w["D"] == 3:
            errs = precision_errors(torch, lbm, dev)
            extras["l2_velocity_error"] = {k: v for k, v in errs.items() if k != "small_taylor_green_2d"}
            extras["decay_rate_error"] = {
                "taylor_green_3d": {"case": errs["case"], "F32": errs["decay_rate"]["F32"],
                                    "F16S": errs["decay_rate"]["F16S"],
                                    "F64_rate_per_step": errs["decay_rate"]["F64_per_step"],
                                    "definition": errs["decay_rate"]["definition"]},
                "taylor_green_2d": errs["small_taylor_green_2d"]}
    cpu = None
    if rank == 0:
        cpu = oracle_baseline(w, args.bulk, seconds=args.cpu_seconds)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": glups, "unit": "GLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32",
        "storage": PREC_NAME[prec], "data": "synthetic",
        "config": {"workload": w["name"], "lattice": f"D{D}Q{Q}", "dims": list(dims), "tau": w["tau"],
                   "equilibrium": args.eq, "bulk_corr": args.bulk, "precision": PREC_NAME[prec],
                   "diag_every": args.diag_every, "state_bytes": info["storage_bytes"],
                   "l2": "inputs larger than L2 (the population array is re-read every step)",
                   "parallelism": "replicas" if ws > 1 else "single GPU", "launch": info},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_note,
                     "peak_source": peak_src, "kernel": kname, "algorithmic_bytes_per_launch": algo_bytes,
                     "avg_launch_ms": launch_ms},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        "diag_last": {k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in hist[-1].items()} if hist else None,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)


def energy_decay_compare(torch, lbm, w, args, rho, u, steps=5000, every=100):
    """Kinetic-energy decay of the binary16 run against the FP32 run (fused diagnostics
    every `every` steps): the largest relative difference of E(t) over the steps both runs
    stayed finite, and the step at which each run first became non-finite (None if not)."""
    curves, diverged = {}, {}
    for prec in (2, 1):
        lat = lbm.Lattice(lbm.D3Q27, w["dims"], w["tau"], w["eq"], 0, prec)
        lat.init_fields(rho, u, dtype=np.float32)
        lat.set_option(lbm.OPT_DIAG_EVERY, every)
        diverged[prec] = None
        try:
            lat.step(steps + 1)
        except lbm.LBMError as e:
            if e.status != lbm.ENONFINITE:
                raise
        hist = lat.diag_history()
        bad = [h["step"] for h in hist if h["nonfinite"] > 0 or not np.isfinite(h["kinetic"])]
        diverged[prec] = bad[0] if bad else None
        curves[prec] = {h["step"]: h["kinetic"] for h in hist if h["nonfinite"] == 0 and np.isfinite(h["kinetic"])}
        lat.close()
        torch.cuda.empty_cache()
    common = sorted(set(curves[2]) & set(curves[1]))
    rel = [abs(curves[2][t] - curves[1][t]) / curves[1][t] for t in common]
    return {"steps": steps, "every": every, "compared_until": common[-1] if common else None,
            "max_rel_diff": max(rel) if rel else None,
            "E_last_over_E0": curves[1][common[-1]] / curves[1][common[0]] if common else None,
            "nonfinite_from_step": {"F16S": diverged[2], "F32": diverged[1]},
            "tau": w["tau"], "note": "constant-tau BGK without a nonlinear limiter"}


def energy_curve(torch, lbm, D, dims, tau, eq, bulk, prec, rho, u, steps, every):
    """Run one lattice for `steps` steps with fused diagnostics every `every` steps.
    Returns {step: kinetic energy} over the finite records, the first step with a
    non-finite cell (None if none) and the device seconds taken."""
    lat = lbm.Lattice(lbm.D3Q27 if D == 3 else lbm.D2Q9, dims, tau, eq, bulk, prec)
    lat.init_fields(rho, u, dtype=np.float32)
    lat.set_option(lbm.OPT_DIAG_EVERY, every)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    try:
        lat.step(steps + 1)
    except lbm.LBMError as e:
        if e.status != lbm.ENONFINITE:
            raise
    e1.record()
    e1.synchronize()
    hist = lat.diag_history()
    lat.close()
    torch.cuda.empty_cache()
    bad = [h["step"] for h in hist if h["nonfinite"] > 0 or not np.isfinite(h["kinetic"])]
    curve = {h["step"]: h["kinetic"] for h in hist if h["nonfinite"] == 0 and np.isfinite(h["kinetic"])}
    return curve, (bad[0] if bad else None), e0.elapsed_time(e1) * 1e-3


def shear_divergence(torch, lbm, w, args, rho, u, steps=10000, every=100):
    """Double shear layer at tau - 1/2 = 3e-5 (a nearly inviscid flow the paper's linear
    analysis does not cover): the step at which each equilibrium first produced a
    non-finite cell within `steps` steps (None: it stayed finite), reported, not asserted."""
    out = {"steps": steps, "every": every}
    for name, eq in (("entropic", 0), ("poly2", 1)):
        curve, bad, sec = energy_curve(torch, lbm, w["D"], w["dims"], w["tau"], eq, args.bulk, w["prec"],
                                       rho, u, steps, every)
        t = sorted(curve)
        out[name] = {"nonfinite_from_step": bad, "last_finite_record": t[-1] if t else None,
                     "E_last_over_E0": curve[t[-1]] / curve[t[0]] if t else None, "seconds": sec}
    return out


def accuracy_gates(torch, lbm, dev, w, args, rho, u):
    """Accuracy of the reduced-precision storage on the full-size Taylor-Green vortex at
    Re = 1600: (i) relative L2 velocity error of FP32 and binary16 storage against FP64
    storage after four convective times t_c = N / (2 pi u0), while the flow is still
    laminar and pointwise differences are meaningful; (ii) over `long_steps` steps, the
    kinetic-energy curve E(t) and the dissipation -dE/dt of binary16 against FP32, with
    the bulk correction off and on (after transition pointwise fields decorrelate, so the
    volume averages are compared)."""
    D, dims, ncell = w["D"], w["dims"], int(np.prod(w["dims"]))
    n = dims[0]
    steps_i = int(round(4 * n / (2 * math.pi * w["u0"])))
    from paper_2303_08163_gb300 import fits
    out = {"pointwise": {"steps": steps_i}, "curves": {}}
    vel, rate = {}, {}
    for prec in (0, 1, 2):
        lat = lbm.Lattice(lbm.D3Q27, dims, w["tau"], w["eq"], 0, prec)
        lat.init_fields(rho, u, dtype=np.float32)
        lat.set_option(lbm.OPT_DIAG_EVERY, 10)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        lat.step(steps_i)
        e1.record()
        hist = lat.diag_history()
        rate[prec] = fits.energy_decay_rate([h["step"] for h in hist], [h["kinetic"] for h in hist])
        r = torch.empty(ncell, device=dev, dtype=torch.float64)
        v = torch.empty(3, ncell, device=dev, dtype=torch.float64)
        lat.moments(dtype=np.float64, out=(r, v))
        torch.cuda.synchronize()
        out["pointwise"][PREC_NAME[prec] + "_seconds"] = e0.elapsed_time(e1) * 1e-3
        lat.close()
        del r
        vel[prec] = v
        torch.cuda.empty_cache()
    ref = torch.linalg.norm(vel[0])
    for prec in (1, 2):
        out["pointwise"][PREC_NAME[prec] + "_rel_l2_vs_F64"] = float(torch.linalg.norm(vel[prec] - vel[0]) / ref)
        # slope of -ln E over the same window (E every 10 steps), relative to FP64
        out["pointwise"][PREC_NAME[prec] + "_decay_rate_error_vs_F64"] = abs(rate[prec] / rate[0] - 1)
    out["pointwise"]["F64_decay_rate_per_step"] = rate[0]
    del vel
    torch.cuda.empty_cache()
    every = 100
    for bulk in (0, 1):
        curves, bad = {}, {}
        for prec in (1, 2):
            curves[prec], bad[prec], _ = energy_curve(torch, lbm, D, dims, w["tau"], w["eq"], bulk, prec,
                                                      rho, u, args.long_steps, every)
        common = sorted(set(curves[1]) & set(curves[2]))
        e32 = np.array([curves[1][t] for t in common])
        e16 = np.array([curves[2][t] for t in common])
        res = {"nonfinite_from_step": {"F32": bad[1], "F16S": bad[2]},
               "compared_until": common[-1] if common else None}
        if len(common) > 2:
            tt = np.array(common, dtype=float)
            d32, d16 = -np.gradient(e32, tt), -np.gradient(e16, tt)
            res.update({"E_max_rel_diff": float(np.max(np.abs(e16 - e32) / e32)),
                        "dissipation_max_diff_over_peak": float(np.max(np.abs(d16 - d32)) / np.max(np.abs(d32))),
                        "dissipation_peak_step": int(tt[np.argmax(d32)]),
                        "E_last_over_E0": float(e32[-1] / e32[0])})
        out["curves"]["bulk" if bulk else "no_bulk"] = res
    out["case"] = (f"{w['name']}, tau={w['tau']:.6f}; (i) {steps_i} steps, (ii) {args.long_steps} steps, "
                   f"diagnostics every {every}")
    return out


def compare_precisions(torch, lbm, dev, w, args, rho, u, sm_mhz=None):
    """Device-timed GLUPS of the same workload in the other storage precisions (FP64 with
    its roofline on the FP64 pipe, at the SM clock sampled during the timed region)."""
    out = {}
    D, dims = w["D"], w["dims"]
    ncell = int(np.prod(dims))
    Q = 3 ** D
    for prec in (2, 1, 0):
        for bulk in (0, 1):
            key = PREC_NAME[prec] + ("+bulk" if bulk else "")
            try:
                lat = lbm.Lattice(lbm.D3Q27 if D == 3 else lbm.D2Q9, dims, w["tau"], w["eq"], bulk, prec)
            except lbm.LBMError as e:
                out[key] = {"error": str(e)}
                continue
            lat.init_fields(rho, u, dtype=np.float32)
            lat.set_option(lbm.OPT_TUNE, 1)
            lat.init_fields(rho, u, dtype=np.float32)
            steps = 40 if prec != 0 else 10
            lat.step(4)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            lat.step(steps)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            gb = 2 * Q * ESIZE[prec] * ncell / (ms * 1e-3) / 1e9
            glups = ncell / (ms * 1e-3) / 1e9
            out[key] = {"GLUPS": glups, "ms_per_step": ms, "GB_s": gb,
                        "hbm_frac": gb / (measured_peaks().get("hbm_gbs") or 6800.0),
                        "launch": lat.launch_info()}
            if prec == 0:
                # FP64 collisions are bound by the FP64 pipe (1/64 of the FP32 rate)
                fpc = fp64_flops_per_cell(w["eq"], bulk, D)
                peak64 = fp64_peak_gflops(sm_mhz)
                out[key]["roofline"] = {"bound": "alu", "flops_per_cell_update": fpc,
                                        "achieved": fpc * glups, "peak": peak64,
                                        "unit": "GFLOP/s (FP64)", "frac": fpc * glups / peak64,
                                        "fp64_pipe": fp64_pipe(w["name"], bulk, out[key]["launch"], glups, sm_mhz)}
            lat.close()
            torch.cuda.empty_cache()
    return out


def batch_mode_sweep(lbm, eq, bulk, steps=4000, every=10, skip_steps=200):
    """The batched linear-mode sweep at full size (4096 instances, `steps` steps, probes
    every `every` steps), checked instance by instance against the scheme's linear theory:
    after `skip_steps` (the non-hydrodynamic transients), each probe series is fitted by a
    least-squares linear map (the shear wave on j_y, the two acoustic modes on rho and j_x)
    and every fitted per-sample multiplier is compared with the nearest lambda^K of the
    von Neumann matrix M = E (delta + J) at the instance's (tau, U0, k) from the library's
    eigen-solver.  The fit window holds the samples after `skip_steps` whose signal stays
    within 1e-9 .. 1e3 of the initial amplitude; instances with fewer than 8 samples in it
    (strongly damped waves) are counted, not fitted."""
    from paper_2303_08163_gb300 import fits, inputs
    table = inputs.linear_mode_batch(count=4096, seed=2303)
    count = len(table["nx"])
    dims = np.stack([table["nx"], table["ny"], np.ones(count, dtype=np.int32)], axis=1)
    fields = [inputs.linear_mode_fields(table, k) for k in range(count)]
    rho = np.concatenate([f[0] for f in fields])
    u = np.concatenate([f[1].reshape(-1) for f in fields])
    kvec = np.stack([table["nmode"], np.zeros(count, np.int32), np.zeros(count, np.int32)], axis=1)
    b = lbm.Batch(lbm.D2Q9, dims, table["tau"], eq, bulk)
    b.init_fields(rho, u)
    b.set_probe(kvec, every)
    t0 = time.time()
    b.step(steps)
    b.sync()
    run_s = time.time() - t0
    series = b.probe_series()
    status = b.status()
    b.close()
    k = 2 * math.pi * table["nmode"] / table["nx"]
    params = np.stack([table["tau"], np.ones(count), table["U0"], np.zeros(count), k, np.zeros(count)], axis=1)
    lam = lbm.vn_eigenvalues(eq, bulk, params)
    unstable = np.abs(lam[:, 0]) > 1 + 1e-12
    s0 = skip_steps // every
    errs, ks, short, nonfinite = [], [], 0, 0
    worst = None
    for i in range(count):
        chans = [2] if table["kind"][i] == 0 else [0, 1]
        ref = float(np.linalg.norm(series[i, 0, chans]))  # the initial amplitude
        x = series[i, s0:, :][:, chans]
        if not np.all(np.isfinite(x)):
            good = np.all(np.isfinite(x), axis=1)
            x = x[:np.argmin(good)] if not good.all() else x
            nonfinite += 1
        mag = np.linalg.norm(x, axis=1)
        if len(mag) == 0 or ref == 0:
            short += 1
            continue
        # fit while the signal stays within 1e-9 .. 1e3 of the initial amplitude (the
        # probe's round-off floor is about 1e-12 of it)
        inside = (mag > 1e-9 * ref) & (mag < 1e3 * ref)
        n = int(np.argmin(inside)) if not inside.all() else len(mag)
        if n < 8:
            short += 1
            continue
        mu = fits.mode_multipliers(x[:n], nmodes=len(chans))
        target = lam[i] ** every
        for m in mu:
            e = float(np.min(np.abs(target - m)))
            errs.append(e)
            ks.append(k[i])
            if worst is None or e > worst[0]:
                worst = (e, i)
    errs, ks = np.array(errs), np.array(ks)

    def stats(sel):
        e = errs[sel]
        return {"compared": int(len(e)), "median": float(np.median(e)) if len(e) else None,
                "p99": float(np.quantile(e, 0.99)) if len(e) else None, "max": float(e.max()) if len(e) else None}
    wi = worst[1] if worst else None
    return {"equilibrium": {0: "entropic", 1: "poly2", 2: "product"}[eq], "bulk_corr": bulk,
            "instances": count, "steps": steps, "every": every, "run_seconds": run_s,
            "linearly_unstable_by_von_neumann": int(unstable.sum()),
            "instances_with_nonfinite_probe": int(nonfinite), "batch_status_nonfinite": int((status > 0).sum()),
            "instances_fitted": int(count - short), "too_fast_to_fit": int(short),
            "multipliers_compared": int(len(errs)),
            "abs_error_median": float(np.median(errs)) if len(errs) else None,
            "abs_error_p99": float(np.quantile(errs, 0.99)) if len(errs) else None,
            "abs_error_max": float(errs.max()) if len(errs) else None,
            "abs_error_k_le_pi_4": stats(ks <= math.pi / 4 + 1e-12),
            "abs_error_k_gt_pi_4": stats(ks > math.pi / 4 + 1e-12),
            "worst_instance": None if wi is None else {
                "tau": float(table["tau"][wi]), "U0": float(table["U0"][wi]), "nx": int(table["nx"][wi]),
                "nmode": int(table["nmode"][wi]), "kind": int(table["kind"][wi])}}


def run_batch(args, w, torch, lbm, dev, rank, ws):
    from paper_2303_08163_gb300 import inputs
    table = inputs.linear_mode_batch(count=args.batch_count, seed=2303)
    count = len(table["nx"])
    dims = np.stack([table["nx"], table["ny"], np.ones(count, dtype=np.int32)], axis=1)
    fields = [inputs.linear_mode_fields(table, k) for k in range(count)]
    rho = np.concatenate([f[0] for f in fields])
    u = np.concatenate([f[1].reshape(-1) for f in fields])
    kvec = np.stack([table["nmode"], np.zeros(count, np.int32), np.zeros(count, np.int32)], axis=1)
    b = lbm.Batch(lbm.D2Q9, dims, table["tau"], w["eq"], args.bulk)
    b.init_fields(rho, u)
    b.set_probe(kvec, 10)
    total = int(b.cell_start[-1])
    if args.shape:
        b.set_launch_shape(*[int(v) for v in args.shape.split(",")])
    elif not args.no_tune:
        b.autotune(steps=10)
    b.step(args.warmup)
    b.sync()
    stream = torch.cuda.current_stream()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        b.step(args.steps)
        e1.record(stream)
        e1.synchronize()
    ms = e0.elapsed_time(e1)
    # end to end through the C ABI: pinned host fields in, all steps, moments out
    rho_h = torch.from_numpy(rho).pin_memory()
    u_h = torch.from_numpy(u).pin_memory()
    rout = torch.empty(total, dtype=torch.float64).pin_memory()
    uout = torch.empty(total * 2, dtype=torch.float64).pin_memory()
    b.init_fields(rho_h, u_h)
    b.moments(out=(rout, uout))  # untimed first round trip
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    b.init_fields(rho_h, u_h)
    b.step(args.steps)
    b.moments(out=(rout, uout))
    f1.record(stream)
    f1.synchronize()
    e2e_ms = f0.elapsed_time(f1)
    if ws > 1:
        t = torch.tensor([ms, e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, e2e_ms = float(t[0]), float(t[1])
        dist.barrier()
    glups = aggregate(ws, total, args.steps, [ms])
    e2e = {"value": aggregate(ws, total, args.steps, [e2e_ms]), "unit": "GLUPS",
           "h2d_bytes_per_step": (rho_h.numel() + u_h.numel()) * 8 / args.steps,
           "d2h_bytes_per_step": (rout.numel() + uout.numel()) * 8 / args.steps,
           "path": "lbm_batch_init_fields(host) + lbm_batch_step(K) + lbm_batch_moments(host), pinned buffers"}
    if rank != 0:
        return
    # FP64 collisions: the roofline is the FP64 pipe.  Peak = 152 SMs x 2 FP64 FMA per
    # cycle x 2 flops x the median SM clock under load
    fpc = fp64_flops_per_cell(w["eq"], args.bulk)
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    fp64_peak = fp64_peak_gflops(sm_mhz)
    achieved = fpc * glups / ws  # GFLOP/s of one GPU
    hbm = 2 * 9 * 8 * glups / ws  # GB/s of one GPU
    launch = b.launch_info()
    rec = [r for r in traffic_records() if r.get("kernel") == "k_step_batch" and r.get("source_hash") == source_hash()
           and r.get("workload") == w["name"]
           and all(r.get("launch", {}).get(k) == launch[k] for k in ("threads", "blocks"))]
    traffic = rec[0]["dram_bytes_per_cell"] * total * args.steps if rec else None
    pipe = None
    if rec and rec[0].get("fp64_thread_inst_per_cell") and rec[0].get("bulk_corr", 0) == args.bulk:
        # the FP64 pipe issues 2 thread instructions per SM per cycle (DADD, DMUL and DFMA
        # alike), so its roofline counts instructions, not flops
        ipc = rec[0]["fp64_thread_inst_per_cell"]
        pipe = {"fp64_thread_inst_per_cell_update": ipc, "achieved_ginst_s": ipc * glups / ws,
                "peak_ginst_s": 152 * 2 * sm_mhz / 1e3, "frac": ipc * glups / ws / (152 * 2 * sm_mhz / 1e3),
                "source": rec[0].get("captured_on")}
    cpu = oracle_baseline(w, args.bulk, seconds=args.cpu_seconds)
    line = {"metric": METRIC, "value": glups, "unit": "GLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "instances": count, "total_cells": total, "probe_every": 10,
                       "launch": launch, "l2": "inputs larger than L2 (the 4096-instance state is 2.2 GB)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "GFLOP/s (FP64)",
                         "frac": achieved / fp64_peak, "traffic": traffic,
                         "traffic_source": rec[0].get("captured_on") if rec else
                         "no ncu record for this kernel source and launch shape",
                         "kernel": "k_step_batch", "launches": 1,
                         "flops_per_cell_update": fpc, "fp64_pipe": pipe,
                         "hbm_GB_s": hbm, "hbm_frac": hbm / (measured_peaks().get("hbm_gbs") or 6800.0)},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 1, "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    run_native(args)


if __name__ == "__main__":
    main()
