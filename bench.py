#!/usr/bin/env python3
"""Throughput of the fused GMF-FLBM D3Q27 stream-and-collide step on GB300.

Workload (one "step" = one lattice time step of the whole hot path over the
box): periodic 512^3 box, FP32 deviation populations in place (AA pattern,
14.5 GB), GMF-FLBM, rho0 = 1, kT = 1e-5, tau = 0.6, fused FP64 reductions on
every step.  The box starts from a seeded sample of the lattice invariant
measure so the reported <u_a^2> is an equilibrium value.

Output: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (bounded sample of the same workload).

Extra lines (not the default): ``--precision fp16`` (FP16 storage),
``--state-form moments`` (the thread-safe moment-state form, ten numbers per
node), ``--workload ensemble`` (328 replica boxes in one persistent kernel
per step) and ``--workload learned`` (GMF-FLBM plus the tensor-core network
correction on 256^3, with its training and a statistics run).  The default
line also carries brief timings of these workloads under ``variants``
(single GPU only; ``--no-variants`` skips them).

Multi-GPU: the path runs independent replica boxes, one per rank ("replicas
only", weak scaling); torch.distributed is used for the barrier and the
max-over-ranks time only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(nx=512, ny=512, nz=512, tau=0.6, kT=1e-5, rho0=1.0, seed=20260101, scheme="gmf")
# algorithmic HBM bytes per lattice update: 27 reads + 27 writes of the
# storage type
BYTES_PER_NODE = {"fp32": 27 * 4 * 2, "fp16": 27 * 2 * 2, "fp64": 27 * 8 * 2}
CS2 = 1.0 / 3.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_step_rows_f32_gmf_traffic.txt")
KERNEL_SOURCES = ["step_kernel.cuh", "lattice.cuh", "internal.h", "step_f32.cu", "step_f32_paced.cu"]
TRAFFIC16_FILE = os.path.join(ROOT, "profiles", "k_step_rows_f16_gmf_traffic.txt")
KERNEL16_SOURCES = ["step_kernel.cuh", "lattice.cuh", "internal.h", "step_f16.cu", "step_f16_nx512.cu"]
ENS_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_step_ens_f32_gmf_traffic.txt")
ENS_KERNEL_SOURCES = ["ens_kernel.cuh", "step_kernel.cuh", "lattice.cuh", "internal.h", "stats.cuh",
                      "ens_f32.cu", "ens_f32p.cu"]
LEARNED_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_step_learned_f32_traffic.txt")
MS_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_ms_step_f32_gmf_traffic.txt")
MS_KERNEL_SOURCES = ["mstate.cu", "step_kernel.cuh", "lattice.cuh", "internal.h"]
MS_BYTES_PER_NODE = 10 * 4 * 2   # moment state: ten FP32 numbers read and written per node
LEARNED_KERNEL_SOURCES = ["step_learned.cu", "mlp_tc.cuh", "umma.cuh", "step_kernel.cuh", "lattice.cuh",
                          "internal.h"]


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=512, help="cube edge (512 = the benchmark workload)")
    ap.add_argument("--box", type=int, nargs=3, metavar=("NX", "NY", "NZ"), default=None,
                    help="non-cubic box (profiling runs); overrides --size")
    ap.add_argument("--precision", choices=["fp32", "fp16", "fp64"], default="fp32",
                    help="population storage (fp32 = the benchmark workload)")
    ap.add_argument("--state-form", choices=["populations", "moments"], default="populations",
                    help="box: what the box keeps between steps (moments: the thread-safe form, "
                         "ten FP32 numbers per node, FP32 GMF only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="box: skip the brief timings of the extra workloads (FP16 storage, moment "
                         "state, ensemble, learned step) that the default line reports under 'variants'")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", choices=["box", "ensemble", "learned"], default="box",
                    help="box: one 512^3 box (default); ensemble: 256 x 32^3 + 64 x 64^3 + "
                         "8 x 128^3 replicas in one persistent kernel per step")
    ap.add_argument("--no-plain", action="store_true",
                    help="ensemble: skip timing the same replicas one box at a time")
    ap.add_argument("--train-boxes", type=int, default=64,
                    help="learned: Reg-FLBM 64^3 boxes whose pairs train the network (64 = 2^24 pairs)")
    ap.add_argument("--train-epochs", type=int, default=6)
    ap.add_argument("--stat-steps", type=int, default=5000,
                    help="learned, ensemble: steps of the statistics run after the timed region (0: skip)")
    ap.add_argument("--ens-div", type=int, default=1,
                    help="ensemble: divide every replica count by this (profiling runs; 1 = the "
                         "benchmark workload)")
    ap.add_argument("--tuning", type=int, nargs=4, default=None,
                    metavar=("ITEM_NODES", "STAGES", "WARPS", "CTAS_PER_SM"),
                    help="ensemble: this launch shape instead of the autotuner's")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3 (untimed warm-up steps before the timed region)")
    return args


# ----------------------------------------------------------------------------
# distributed helpers (replicas only)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, local, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (the job's time is its
    slowest rank's)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes_per_rank: int, steps: int, max_ms: float, ws: int) -> float:
    """Whole-job lattice updates per second over all ranks, in MLUPS."""
    return ws * nodes_per_rank * steps / (max_ms / 1e3) / 1e6


# ----------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                   "-lms", "100"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "of measured"
    except Exception:
        return 6800.0, "of fallback"


def strip_comments(src: str) -> str:
    """C/C++ source without its comments, trailing blanks and empty lines
    (string and character literals are kept), so that the hash below
    follows the code and not its commentary."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = (ln.rstrip() for ln in "".join(out).split("\n"))
    return "\n".join(ln for ln in lines if ln)


def kernel_source_hash(sources=None) -> str:
    """sha256 (first 16 hex digits) of the kernel sources, comments left out."""
    h = hashlib.sha256()
    for f in (KERNEL_SOURCES if sources is None else sources):
        with open(os.path.join(ROOT, "paper_2601_03806_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(nodes: int, path=None, sources=None):
    """Per-launch DRAM bytes of the step kernel from the committed ncu summary,
    scaled to the box size; None if the kernel changed since the capture."""
    try:
        kv = {}
        for ln in open(TRAFFIC_FILE if path is None else path):
            if ":" in ln and not ln.startswith("#"):
                k, v = ln.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_hash") != kernel_source_hash(sources):
            return None
        per_node = float(kv["dram_bytes_per_node"])
        return per_node * nodes
    except Exception:
        return None


def bind_to_gpu_numa_node(torch, dev) -> str:
    """Run this process on the CPUs local to the GPU, so that pinned host
    buffers allocated afterwards sit next to it (host<->device copies cross
    no socket link).  Returns what was done, for the JSON line."""
    try:
        p = torch.cuda.get_device_properties(dev)
        bus = "%04x:%02x:%02x.0" % (getattr(p, "pci_domain_id", 0), p.pci_bus_id, p.pci_device_id)
        base = "/sys/bus/pci/devices/" + bus
        cpus = open(base + "/local_cpulist").read().strip()
        sel = set()
        for part in cpus.split(","):
            a, _, b = part.partition("-")
            sel.update(range(int(a), int(b or a) + 1))
        sel &= os.sched_getaffinity(0)
        if not sel:
            return "not bound (no local CPUs available)"
        os.sched_setaffinity(0, sel)
        return "bound to the %d CPUs local to GPU %s" % (len(sel), bus)
    except Exception as e:
        return "not bound (%s)" % type(e).__name__


def host_mem_available() -> int:
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                return int(ln.split()[1]) * 1024
    except Exception:
        pass
    return 0


def oracle_sample(tau, kT, rho0, seed, budget_s=2.0, n=64):
    """The FP64 oracle as it stands on this host's cores: a bounded sample
    (n^3 box from a thermal state, same tau/kT/rho0) stepped until ~budget_s
    of wall time.  Returns (MLUPS, threads, steps, u2 ratio)."""
    import numpy as np
    import oracle
    from synth import inputs
    oracle.build()
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    w = oracle.tables()["w"]
    box = oracle.Box(n, n, n, tau, kT, rho0=rho0, seed=seed)
    sd = np.sqrt(rho0 * kT * w / CS2)[:, None, None, None]
    box.set_f(w[:, None, None, None] * rho0 + sd * inputs.population_perturbation(n, n, n, seed))
    box.step(1)
    steps, t0 = 0, time.perf_counter()
    u2 = []
    while True:
        box.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el > budget_s and steps >= 3:
            break
    rho, j, _ = box.moments()
    u2 = ((j / rho) ** 2).mean(axis=(1, 2, 3)) / (kT / rho0)
    return n ** 3 * steps / el / 1e6, threads, steps, [float(x) for x in u2]


def oracle_single_thread(tau, kT, rho0, seed, budget_s=1.0, n=32):
    """The oracle on one host thread (MLUPS), a bounded sample."""
    import oracle
    oracle.build()
    prev = oracle.get_threads()
    oracle.set_threads(1)
    box = oracle.Box(n, n, n, tau, kT, rho0=rho0, seed=seed)
    steps, t0 = 0, time.perf_counter()
    while True:
        box.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el > budget_s and steps >= 2:
            break
    oracle.set_threads(prev)
    return n ** 3 * steps / el / 1e6


def run_reference(args, rank, ws):
    if rank != 0:
        return 0
    tau, kT, rho0, seed = WORKLOAD["tau"], WORKLOAD["kT"], WORKLOAD["rho0"], WORKLOAD["seed"]
    import numpy as np
    import oracle
    from synth import inputs
    oracle.build()
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    n = 64
    w = oracle.tables()["w"]
    box = oracle.Box(n, n, n, tau, kT, rho0=rho0, seed=seed)
    sd = np.sqrt(rho0 * kT * w / CS2)[:, None, None, None]
    box.set_f(w[:, None, None, None] * rho0 + sd * inputs.population_perturbation(n, n, n, seed))
    box.step(args.warmup)
    t0 = time.perf_counter()
    box.step(args.steps)
    el = time.perf_counter() - t0
    v = n ** 3 * args.steps / el / 1e6
    sample = "%d^3 box of the %d^3 workload's parameters, FP64 two-array oracle, %d threads" % (
        n, args.size, threads)
    line = {
        "impl": "reference", "metric": metric_name(), "value": v, "unit": "MLUPS",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.size, ws),
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def metric_name():
    return "MLUPS of the fused GMF-FLBM D3Q27 stream-and-collide step (HBM roofline fraction beside it)"


def workload_config(size, ws, precision="fp32", box=None, moments=False):
    es = BYTES_PER_NODE[precision] // 54
    nx, ny, nz = box if box else (size, size, size)
    shape = "%d^3" % size if nx == ny == nz else "%dx%dx%d" % (nx, ny, nz)
    if moments:
        return {"workload": "GMF-FLBM D3Q27 periodic %s in the moment-state (thread-safe) form: ten "
                            "FP32 numbers per node between steps, populations rebuilt from the "
                            "neighbours' numbers and regenerated noise; rho0=1, kT=1e-5, tau=0.6, "
                            "FP64 reductions every step" % shape,
                "nx": nx, "ny": ny, "nz": nz, "tau": WORKLOAD["tau"], "kT": WORKLOAD["kT"],
                "rho0": WORKLOAD["rho0"], "scheme": "gmf",
                "storage": "moment state, 2 x 10 FP32 arrays (ping-pong)",
                "stats_every": 1, "l2": "inputs larger than L2 (%.1f GB state vs 129 MB L2)"
                % (40 * nx * ny * nz / 1e9),
                "parallelism": "replicas x%d (one independent box per GPU)" % ws}
    return {"workload": "GMF-FLBM D3Q27 periodic %s, %s deviation populations AA in place, "
                        "rho0=1, kT=1e-5, tau=0.6, FP64 reductions every step"
                        % (shape, precision.upper()),
            "nx": nx, "ny": ny, "nz": nz, "tau": WORKLOAD["tau"], "kT": WORKLOAD["kT"],
            "rho0": WORKLOAD["rho0"], "scheme": "gmf",
            "storage": "%s deviations, AA in place" % precision,
            "stats_every": 1, "l2": "inputs larger than L2 (%.1f GB state vs 129 MB L2)"
            % (27 * es * nx * ny * nz / 1e9),
            "parallelism": "replicas x%d (one independent box per GPU)" % ws}


def run_ours(args, rank, local, ws):
    import numpy as np
    import torch
    from paper_2601_03806_gb300 import build as _b
    _b.build()
    from paper_2601_03806_gb300 import flbm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.size
    nx, ny, nz = args.box if args.box else (n, n, n)
    N = nx * ny * nz
    tau, kT, rho0 = WORKLOAD["tau"], WORKLOAD["kT"], WORKLOAD["rho0"]
    seed = WORKLOAD["seed"] + rank
    stream = torch.cuda.Stream(device=dev)
    prec = {"fp32": flbm.FLBM_FP32, "fp16": flbm.FLBM_FP16, "fp64": flbm.FLBM_FP64}[args.precision]
    es = BYTES_PER_NODE[args.precision] // 54
    moments = args.state_form == "moments"
    if moments and args.precision != "fp32":
        raise SystemExit("--state-form moments runs on FP32 storage")
    lat = flbm.Lattice(nx, ny, nz, tau, kT, rho0=rho0, seed=seed, precision=prec,
                       stats_every=1, torch_memory=True, stream=stream,
                       state_form=flbm.FLBM_STATE_MOMENTS if moments else flbm.FLBM_STATE_POPULATIONS)
    lat.init_thermal(seed)           # invariant-measure start (library kernel)
    lat.step(1)                      # first warm-up step: its reduction holds the start mass
    mass0 = lat.stats()["mass"]
    lat.step(args.warmup - 1)
    lat.stats_reset()
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    gpu_id = ("GPU-" + str(uuid)) if uuid is not None else os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]

    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(ws)
    with ClockSampler(gpu_id) as clk:
        lat.timing_enable(True)
        start.record(stream)
        lat.step(args.steps)
        end.record(stream)
        torch.cuda.synchronize()
    kernel_ms, launches = lat.timing_read()
    lat.timing_enable(False)
    barrier(ws)
    el_ms = start.elapsed_time(end)
    max_ms = max_over_ranks(el_ms, ws, dev)
    value = job_mlups(N, args.steps, max_ms, ws)
    st = lat.stats()

    k_ms = kernel_ms / max(launches, 1)
    peak, peak_src = measured_hbm_peak()
    node_bytes = MS_BYTES_PER_NODE if moments else BYTES_PER_NODE[args.precision]
    achieved = node_bytes * N / (k_ms / 1e3) / 1e9
    traffic = {"fp32": recorded_traffic(N),
               "fp16": recorded_traffic(N, TRAFFIC16_FILE, KERNEL16_SOURCES)}.get(args.precision)
    rows_path = nx % 32 == 0 and 2 * 27 * nx * es <= 200 * 1024 and os.environ.get("FLBM_ROWS", "1") != "0"
    # two nodes per thread for FP32 / FP16 rows of 256 and more (FLBM_ROW_PAIRS=0: one)
    pairs = (args.precision != "fp64" and nx >= 256 and 2 * 27 * nx * es <= 2 * 27 * 512 * 4
             and os.environ.get("FLBM_ROW_PAIRS", "1") != "0")
    st_name = {"fp32": "float", "fp16": "__half", "fp64": "double"}[args.precision]
    # FP16 rows of exactly 512 nodes run the kernel with the row length fixed at compile time
    fixed = pairs and args.precision == "fp16" and nx == 512
    # FP32 two-node rows staged twice (more than 256 nodes) run the PACED instance
    paced = pairs and args.precision == "fp32" and nx > 256
    kname = ("flbm::k_step_rows<%s,GMF,*,stats,NP=%d%s> (TMA row pipeline, %s)"
             % (st_name, 2 if pairs else 1, ",NXC=512" if fixed else (",PACED" if paced else ""),
                "two nodes per thread" if pairs else "one node per thread")
             if rows_path else "flbm::k_step<%s,GMF,*,stats> (direct)" % st_name)
    if rows_path and not pairs:
        traffic = None     # the records are of the two-node kernel
    if args.precision == "fp16" and not fixed:
        traffic = None     # the FP16 record is of the fixed-length (512) kernel
    if not rows_path:
        traffic = None
    if moments:
        kname = "flbm::k_ms_step<GMF,stats> (moment state, z-marching columns)"
        traffic = recorded_traffic(N, MS_TRAFFIC_FILE, MS_KERNEL_SOURCES)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "traffic": traffic, "kernel": kname,
                "kernel_ms": k_ms, "algorithmic_bytes_per_launch": node_bytes * N}

    u2_ratio = [x / (kT / rho0) for x in st["u2_avg"]]

    # e2e through the C ABI with pinned host buffers: upload the state, K steps
    # each followed by a stats read, then one moments snapshot to the host.
    e2e = None
    if not args.no_e2e:
        numa = bind_to_gpu_numa_node(torch, dev)
        state_bytes = 27 * es * N
        mom_bytes = 10 * 8 * N
        with_moments = host_mem_available() > 3 * (state_bytes + mom_bytes)
        tdt = {"fp32": torch.float32, "fp16": torch.float16, "fp64": torch.float64}[args.precision]
        hstate = torch.empty(27 * N, dtype=tdt, pin_memory=True)
        lat.get_state(hstate)
        if with_moments:
            hrho = torch.empty(N, dtype=torch.float64, pin_memory=True)
            hj = torch.empty(3 * N, dtype=torch.float64, pin_memory=True)
            hpi = torch.empty(6 * N, dtype=torch.float64, pin_memory=True)
        # the whole end-to-end pass three times (the host link is shared with
        # other work on the machine, so one upload can be several times
        # slower than the next); the line reports the median pass
        passes = []
        for _ in range(3):
            torch.cuda.synchronize()
            barrier(ws)
            t0 = time.perf_counter()
            lat.set_state(hstate)
            t1 = time.perf_counter()
            lat.set_step(args.warmup)
            for _ in range(args.steps):
                lat.step(1)
                lat.stats()
            t2 = time.perf_counter()
            if with_moments:
                rc = flbm.flbm_moments(lat.handle, hrho.data_ptr(), hj.data_ptr(), hpi.data_ptr())
                if rc != 0:
                    raise RuntimeError(flbm.flbm_last_error(lat.handle))
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            passes.append(((t3 - t0) * 1e3, {"upload_ms": (t1 - t0) * 1e3, "steps_ms": (t2 - t1) * 1e3,
                                              "snapshot_ms": (t3 - t2) * 1e3}))
        passes.sort(key=lambda p: p[0])
        e_ms, e2e_split = passes[1]
        e_max = max_over_ranks(e_ms, ws, dev)
        import ctypes
        stats_bytes = ctypes.sizeof(flbm.flbm_stats_t) + 16
        e2e = {"value": job_mlups(N, args.steps, e_max, ws), "unit": "MLUPS",
               "h2d_bytes_per_step": state_bytes // args.steps,
               "d2h_bytes_per_step": (mom_bytes if with_moments else 0) // args.steps + stats_bytes,
               "what": "flbm_set_state from pinned host + K x (flbm_step(1) + flbm_stats)"
                       + (" + flbm_moments snapshot to pinned host" if with_moments else ""),
               "split": e2e_split, "host_placement": numa,
               "passes_ms": [p[0] for p in passes], "reported": "median of 3 passes"}
        del hstate

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        v, threads, steps, u2o = oracle_sample(tau, kT, rho0, WORKLOAD["seed"])
        cpu = {"value": v, "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": "64^3 box with the workload's tau/kT/rho0 from a thermal state, %d steps, "
                         "FP64 two-array oracle on %d host threads" % (steps, threads),
               "single_thread_value": oracle_single_thread(tau, kT, rho0, WORKLOAD["seed"]),
               "u2_ratio": u2o}

    if rank == 0:
        line = {
            "metric": metric_name(), "value": value, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp16": "f16 storage / f32 arithmetic", "fp64": "f64"}[args.precision],
            "data": "synthetic", "config": workload_config(n, ws, args.precision, (nx, ny, nz), moments),
            "roofline": roofline,
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches) + int(args.steps),
            "clocks": clk.summary(),
            "equipartition": {"u2_avg_over_kT_rho0": u2_ratio,
                              "max_abs_error": max(abs(x - 1) for x in u2_ratio),
                              "er": st["er"], "samples": st["n_samples"]},
            # drift: the mass of the last reduced step against that of the
            # thermal start (args.warmup - 1 + args.steps steps apart); the
            # start's own offset from N rho0 is the sample's thermal spread
            "mass": {"rel_drift": st["mass"] / mass0 - 1.0,
                     "steps_apart": args.warmup - 1 + args.steps,
                     "start_offset": mass0 / (N * rho0) - 1.0,
                     "start_offset_sd": (3.0 * N * rho0 * kT) ** 0.5 / (N * rho0)},
        }
    lat.close()
    if rank == 0:
        default_box = (nx, ny, nz) == (512, 512, 512) and args.precision == "fp32" and not moments
        if ws == 1 and default_box and not args.no_variants:
            torch.cuda.empty_cache()
            line["variants"] = measure_variants(args, flbm, torch, stream, gpu_id)
        print(json.dumps(line), flush=True)
    return 0


def measure_variants(args, flbm, torch, stream, gpu_id):
    """Brief timings, in the process of the default line, of the extra
    workloads (their own lines give the full reports): FP16 storage and the
    moment-state form on the 512^3 box, the config-4 ensemble in the launch
    shape its autotuner picks (items 512, 2 stages, 4 compute warps, 2 CTAs
    per SM), and the learned step on 256^3 with an untrained network (the
    kernel's work does not depend on the weights) beside plain GMF on the
    same box.  Each: warm-up, then args.steps steps between CUDA events on
    the library's stream; MLUPS and the fraction of the measured HBM copy
    rate at its algorithmic bytes."""
    import numpy as np
    tau, kT, rho0, seed = WORKLOAD["tau"], WORKLOAD["kT"], WORKLOAD["rho0"], WORKLOAD["seed"]
    peak, _ = measured_hbm_peak()

    def timed(step, nodes, node_bytes):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        step(args.steps)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        return {"value": nodes / (ms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": ms,
                "roofline_frac": node_bytes * nodes / (ms / 1e3) / 1e9 / peak}

    def box(n, prec, node_bytes, what, state_form=flbm.FLBM_STATE_POPULATIONS, scheme=flbm.FLBM_GMF,
            t=tau, mlp=None):
        lat = flbm.Lattice(n, n, n, t, kT, rho0=rho0, seed=seed, scheme=scheme, precision=prec,
                           stats_every=1, torch_memory=True, stream=stream, state_form=state_form)
        try:
            if mlp is not None:
                lat.set_mlp(mlp)
            lat.init_thermal(seed)
            lat.step(args.warmup)
            r = timed(lat.step, n ** 3, node_bytes)
        finally:
            lat.close()
        r["what"] = what
        return r

    out = {}
    with ClockSampler(gpu_id) as clk:
        out["fp16_storage"] = box(512, flbm.FLBM_FP16, BYTES_PER_NODE["fp16"],
                                  "512^3 GMF, FP16 deviation storage, FP32 arithmetic (108 B/node)")
        torch.cuda.empty_cache()
        out["moment_state"] = box(512, flbm.FLBM_FP32, MS_BYTES_PER_NODE,
                                  "512^3 GMF, moment-state form (80 B/node)",
                                  state_form=flbm.FLBM_STATE_MOMENTS)
        torch.cuda.empty_cache()
        ens = flbm.Ensemble(ensemble_params(flbm, seed), stream=stream)
        try:
            ens.set_tuning(512, 2, 4, 2)
            for r, rep in enumerate(ens.replicas):
                rep.init_thermal(seed * 1000 + r)
            ens.step(args.warmup + (args.warmup % 2))
            out["ensemble"] = timed(ens.step, ens.nodes, BYTES_PER_NODE["fp32"])
            out["ensemble"]["what"] = ("256 x 32^3 + 64 x 64^3 + 8 x 128^3 GMF replicas, one persistent "
                                       "kernel + one statistics kernel per step, graph replay")
        finally:
            ens.close()
        torch.cuda.empty_cache()
        mlp = (0.05 * np.random.default_rng(1).standard_normal(flbm.MLP_NPARAM)).astype(np.float32)
        out["learned"] = box(256, flbm.FLBM_FP32, BYTES_PER_NODE["fp32"],
                             "256^3 learned collision (GMF + tcgen05 network correction), tau 0.8",
                             scheme=flbm.FLBM_LEARNED, t=0.8, mlp=mlp)
        out["plain_256"] = box(256, flbm.FLBM_FP32, BYTES_PER_NODE["fp32"],
                               "256^3 plain GMF, tau 0.8 (the learned step's reference)", t=0.8)
    out["clocks"] = clk.summary()
    return out


# ----------------------------------------------------------------------------
# batched ensemble


ENSEMBLE_SIZES = [32] * 256 + [64] * 64 + [128] * 8


def ensemble_sizes(div=1):
    return [32] * (256 // div) + [64] * (64 // div) + [128] * max(1, 8 // div)


def ensemble_params(flbm, seed, sizes=None):
    """The mixed ensemble: 256 x 32^3 + 64 x 64^3 + 8 x 128^3 periodic boxes,
    tau uniform in [0.51, 3.0] (seeded), kT = 1e-5, rho0 = 1, GMF-FLBM, FP32,
    one Philox key and one noise stream per replica."""
    import numpy as np
    sizes = ENSEMBLE_SIZES if sizes is None else sizes
    rng = np.random.default_rng(seed)
    taus = rng.uniform(0.51, 3.0, size=len(sizes))
    return [flbm.make_params(n, n, n, float(t), WORKLOAD["kT"], rho0=WORKLOAD["rho0"], seed=seed,
                             precision=flbm.FLBM_FP32, stats_every=1, noise_stream=r)
            for r, (n, t) in enumerate(zip(sizes, taus))]


def ensemble_config(ws, tuning=None, sizes=None):
    sizes = ENSEMBLE_SIZES if sizes is None else sizes
    nodes = sum(n ** 3 for n in sizes)
    mix = " + ".join("%d x %d^3" % (sizes.count(n), n) for n in sorted(set(sizes)))
    c = {"workload": "batched GMF-FLBM D3Q27 ensemble: %s periodic "
                     "replicas (%d nodes), tau ~ U[0.51, 3.0], kT=1e-5, rho0=1, FP32 deviations AA "
                     "in place, one noise stream per replica, FP64 per-replica reductions every "
                     "step, one persistent kernel + one statistics kernel per step, CUDA graph"
                     % (mix, nodes),
         "replicas": len(sizes), "nodes": nodes, "scheme": "gmf", "kT": WORKLOAD["kT"],
         "l2": "inputs larger than L2 (%.2f GB state vs 129 MB L2)" % (nodes * 108 / 1e9),
         "parallelism": "replicas x%d (one independent ensemble per GPU)" % ws}
    if tuning:
        c["tuning"] = tuning
    return c


def run_ensemble(args, rank, local, ws):
    import numpy as np
    import torch
    from paper_2601_03806_gb300 import build as _b
    _b.build()
    from paper_2601_03806_gb300 import flbm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    seed = WORKLOAD["seed"] + rank
    kT, rho0 = WORKLOAD["kT"], WORKLOAD["rho0"]
    stream = torch.cuda.Stream(device=dev)
    sizes = ensemble_sizes(args.ens_div)
    params = ensemble_params(flbm, seed, sizes)
    ens = flbm.Ensemble(params, stream=stream)
    N = ens.nodes
    if args.tuning:
        ens.set_tuning(*args.tuning)
        tuning = ens.tuning
    else:
        tuning = ens.autotune(steps_per_trial=3)
    for r, rep in enumerate(ens.replicas):
        rep.init_thermal(seed * 1000 + r)
    ens.step(args.warmup + (args.warmup % 2))
    for rep in ens.replicas:
        rep.stats_reset()
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    gpu_id = ("GPU-" + str(uuid)) if uuid is not None else os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(ws)
    with ClockSampler(gpu_id) as clk:
        start.record(stream)
        ens.step(args.steps)
        end.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    el_ms = start.elapsed_time(end)
    max_ms = max_over_ranks(el_ms, ws, dev)
    value = job_mlups(N, args.steps, max_ms, ws)
    step_ms = el_ms / args.steps
    peak, peak_src = measured_hbm_peak()
    achieved = BYTES_PER_NODE["fp32"] * N / (step_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "traffic": recorded_traffic(N, ENS_TRAFFIC_FILE, ENS_KERNEL_SOURCES),
                "kernel": "flbm::k_step_ens<float,float,GMF,*,stats,NP=%d> + flbm::k_ens_post (per-step "
                          "time of both, graph replay)" % (1 if os.environ.get("FLBM_ROW_PAIRS", "1") == "0" else 2),
                "kernel_ms": step_ms, "algorithmic_bytes_per_launch": BYTES_PER_NODE["fp32"] * N}

    # statistics run (config 4: 5000 steps): ensemble-averaged <u_a^2> of
    # every replica, and the S_jx(k) flatness of every replica (mean over
    # the run's snapshots), summarised per box size
    stat_steps = args.stat_steps if args.stat_steps > 0 else args.steps
    for rep in ens.replicas:
        rep.stats_reset()
    snaps, every = (10, max(1, stat_steps // 10)) if args.stat_steps > 0 else (1, args.steps)
    sacc = [None] * len(ens.replicas)
    for _ in range(snaps):
        ens.step(every)
        for r, rep in enumerate(ens.replicas):
            S, cnt = rep.structure_factor(flbm.FLBM_OBS_JX, sizes[r] // 2)
            m = cnt > 0
            v = float(np.sum(S[m] * cnt[m]) / np.sum(cnt[m]) / (rho0 * kT))
            sacc[r] = v if sacc[r] is None else sacc[r] + v
    u2 = np.array([rep.stats()["u2_avg"] for rep in ens.replicas]) / (kT / rho0)
    sk = np.array(sacc) / snaps
    per_size = {}
    for n in sorted(set(sizes)):
        idx = [r for r, m in enumerate(sizes) if m == n]
        per_size["%d^3" % n] = {"replicas": len(idx),
                                "u2_mean": float(u2[idx].mean()),
                                "u2_max_abs_error": float(np.abs(u2[idx] - 1).max()),
                                "S_jx_mean": float(sk[idx].mean()),
                                "S_jx_max_abs_error": float(np.abs(sk[idx] - 1).max())}
    equip = {"steps": snaps * every, "u2_avg_over_kT_rho0_mean": float(u2.mean()),
             "max_abs_error_over_replicas": float(np.abs(u2 - 1).max()),
             "S_jx_over_rho0_kT_mean": float(sk.mean()), "per_size": per_size}

    # the same replicas as independent boxes, one plain flbm_step call each
    plain = None
    if not args.no_plain:
        boxes = [flbm.Lattice(p.nx, p.ny, p.nz, p.tau, p.kT, seed=p.seed, precision=flbm.FLBM_FP32,
                              noise_stream=p.noise_stream, torch_memory=True, stream=stream)
                 for p in params]
        for b in boxes:
            b.init_thermal(seed)
            b.step(2)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for b in boxes:
            b.step(args.steps)
        t1.record(stream)
        torch.cuda.synchronize()
        p_ms = t0.elapsed_time(t1)
        plain = {"value": N * args.steps / (p_ms / 1e3) / 1e6, "unit": "MLUPS",
                 "what": "the same %d replicas as single-box contexts, flbm_step(K) on each in turn"
                         % len(params)}
        for b in boxes:
            b.close()

    e2e = None
    if not args.no_e2e:
        hstates = [torch.empty(27 * rep.n, dtype=torch.float32, pin_memory=True) for rep in ens.replicas]
        for rep, h in zip(ens.replicas, hstates):
            rep.get_state(h)
        # three passes (median reported) when K keeps the storage in the
        # natural form that a replica's state replacement needs
        passes = []
        for _ in range(3 if args.steps % 2 == 0 else 1):
            torch.cuda.synchronize()
            barrier(ws)
            t0 = time.perf_counter()
            for rep, h in zip(ens.replicas, hstates):
                rep.set_state(h)
            ens.step(args.steps)
            stats = [rep.stats() for rep in ens.replicas]
            torch.cuda.synchronize()
            passes.append((time.perf_counter() - t0) * 1e3)
        e_ms = sorted(passes)[len(passes) // 2]
        e_max = max_over_ranks(e_ms, ws, dev)
        import ctypes
        e2e = {"value": job_mlups(N, args.steps, e_max, ws), "unit": "MLUPS",
               "h2d_bytes_per_step": 4 * 27 * N // args.steps,
               "d2h_bytes_per_step": len(stats) * (ctypes.sizeof(flbm.flbm_stats_t) + 16),
               "what": "flbm_set_state of every replica from pinned host + flbm_ensemble_step(K) + "
                       "flbm_stats of every replica",
               "passes_ms": passes, "reported": "median of %d passes" % len(passes)}
        del hstates

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        v, threads, steps, _ = oracle_sample(1.0, kT, rho0, WORKLOAD["seed"], n=32)
        cpu = {"value": v, "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": "one 32^3 replica (tau = 1.0, kT = 1e-5) from a thermal state, %d steps, "
                         "FP64 two-array oracle on %d host threads" % (steps, threads)}
    if rank == 0:
        line = {
            "metric": "MLUPS of the batched GMF-FLBM ensemble step (persistent kernel, CUDA graph)",
            "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": ensemble_config(ws, tuning, sizes), "roofline": roofline, "cpu_baseline": cpu,
            "e2e": e2e, "plain_kernel": plain, "gpu_launches": 2 * int(args.steps),
            "clocks": clk.summary(), "equipartition": equip,
        }
        print(json.dumps(line), flush=True)
    ens.close()
    return 0


# ----------------------------------------------------------------------------
# learned collision


def run_learned(args, rank, local, ws):
    """Config 5: a network trained on Reg-FLBM pre/post-collision pairs
    (64^3 boxes, tau ~ U[0.51, 3.0], kT = 1e-5) corrects GMF-FLBM on a 256^3
    box (tau 0.8, kT 1e-5); timed like the box workload and compared with
    plain GMF-FLBM on the same GPU."""
    import numpy as np
    import torch
    from paper_2601_03806_gb300 import build as _b
    _b.build()
    from paper_2601_03806_gb300 import flbm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    seed = WORKLOAD["seed"] + rank
    kT, rho0, tau = WORKLOAD["kT"], WORKLOAD["rho0"], 0.8
    n = args.size if args.size != 512 else 256
    N = n ** 3
    rng = np.random.default_rng(seed)

    def pairs(taus, start):
        xs, ts = [], []
        for r, tb in enumerate(taus):
            box = flbm.Lattice(64, 64, 64, float(tb), kT, seed=seed, scheme=flbm.FLBM_REG,
                               noise_stream=start + r)
            box.init_thermal(seed * 7 + start + r)
            box.step(40)
            X = torch.empty((64 ** 3, 28), dtype=torch.float32, device=dev)
            T = torch.empty((64 ** 3, 27), dtype=torch.float32, device=dev)
            box.mlp_pairs(X, T)
            xs.append(X)
            ts.append(T)
            box.close()
        return torch.cat(xs), torch.cat(ts)

    t0 = time.perf_counter()
    X, T = pairs(rng.uniform(0.51, 3.0, size=args.train_boxes), 0)
    t1 = time.perf_counter()
    # initial parameters: He-style normal weights, zero biases (seeded)
    nin, nh, nout = 28, 64, 27
    theta0 = np.concatenate([rng.normal(0, np.sqrt(1.0 / nin), nh * nin), np.zeros(nh),
                             rng.normal(0, np.sqrt(1.0 / nh), nh * nh), np.zeros(nh),
                             rng.normal(0, np.sqrt(1.0 / nh), nout * nh), np.zeros(nout)]).astype(np.float32)
    theta, losses = flbm.mlp_train(theta0, X, T, epochs=args.train_epochs, batch=1024, lr=1e-2, seed=seed)
    t2 = time.perf_counter()
    del X, T
    Xh, Th = pairs([tau], 10 ** 6)
    yh = flbm.mlp_infer(theta, Xh.cpu().numpy())
    th = Th.cpu().numpy()
    rel = float(np.linalg.norm(yh - th) / np.linalg.norm(th))
    del Xh, Th
    training = {"pairs": args.train_boxes * 64 ** 3, "epochs": args.train_epochs, "batch": 1024,
                "first_epoch_loss": float(losses[0]), "last_epoch_loss": float(losses[-1]),
                "pairs_s": t1 - t0, "train_s": t2 - t1,
                "held_out_rel_error_of_correction": rel, "gmf_rel_error": 1.0}

    stream = torch.cuda.Stream(device=dev)
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    gpu_id = ("GPU-" + str(uuid)) if uuid is not None else os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]

    def timed(scheme):
        lat = flbm.Lattice(n, n, n, tau, kT, rho0=rho0, seed=seed, scheme=scheme, stats_every=1,
                           torch_memory=True, stream=stream)
        if scheme == flbm.FLBM_LEARNED:
            lat.set_mlp(theta)
        lat.init_thermal(seed)
        lat.step(args.warmup)
        lat.stats_reset()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier(ws)
        with ClockSampler(gpu_id) as clk:
            lat.timing_enable(True)
            start.record(stream)
            lat.step(args.steps)
            end.record(stream)
            torch.cuda.synchronize()
        kms, launches = lat.timing_read()
        lat.timing_enable(False)
        barrier(ws)
        el = start.elapsed_time(end)
        st = lat.stats()
        return lat, el, kms / max(launches, 1), launches, clk.summary(), st

    from paper_2601_03806_gb300 import analysis

    def statistics(lat):
        """Config-5 judgement: equipartition (time average over the run) and
        the S(k) spectra (mean over 10 snapshots) against their flat theory."""
        if args.stat_steps <= 0:
            return None
        lat.stats_reset()
        obs = analysis.PAPER_OBSERVABLES + (flbm.FLBM_OBS_JX,)
        names = {flbm.FLBM_OBS_RHO: "rho", flbm.FLBM_OBS_JSUM: "j_sum", flbm.FLBM_OBS_PI_DIAG: "pi_diag",
                 flbm.FLBM_OBS_PI_OFFDIAG: "pi_offdiag", flbm.FLBM_OBS_JX: "jx"}
        er = analysis.er_spectrum(lat, n // 2, snapshots=10, every=max(1, args.stat_steps // 10), observables=obs)
        stt = lat.stats()
        out = {"steps": 10 * max(1, args.stat_steps // 10),
               "u2_avg_over_kT_rho0": [x / (kT / rho0) for x in stt["u2_avg"]], "er": stt["er"]}
        for m in obs:
            ratio, cnt = er[m]
            k = cnt > 0
            lo, hi = analysis.window_extrema(ratio, cnt, 4, n // 2 - 1)
            out["S_" + names[m] + "_over_theory"] = {"mean": float(np.sum(ratio[k] * cnt[k]) / np.sum(cnt[k])),
                                                      "min_shell_4_up": lo, "max_shell_4_up": hi}
        return out

    lat, el_ms, k_ms, launches, clocks, st = timed(flbm.FLBM_LEARNED)
    max_ms = max_over_ranks(el_ms, ws, dev)
    value = job_mlups(N, args.steps, max_ms, ws)
    peak, peak_src = measured_hbm_peak()
    achieved = BYTES_PER_NODE["fp32"] * N / (k_ms / 1e3) / 1e9
    # the network's multiply-adds per node (28-64-64-27); the tensor pipe
    # executes the padded shapes with the bias columns, K 32 / 80 / 80 and
    # N 64 / 64 / 32
    flop_node = 2 * (28 * 64 + 64 * 64 + 64 * 27)
    flop_node_issued = 2 * (32 * 64 + 80 * 64 + 80 * 32)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            tpk, tsrc = float(json.load(fh)["bf16_tflops_sustained"]), "of measured (sustained)"
    except Exception:
        tpk, tsrc = 1700.0, "of fallback"
    tflops = flop_node * N / (k_ms / 1e3) / 1e12
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_src,
                "traffic": recorded_traffic(N, LEARNED_TRAFFIC_FILE, LEARNED_KERNEL_SOURCES),
                "kernel": "flbm::k_step_learned<uint32,*,stats> (GMF + tcgen05 MLP correction)",
                "kernel_ms": k_ms, "algorithmic_bytes_per_launch": BYTES_PER_NODE["fp32"] * N,
                "tensor": {"achieved_tflops": tflops, "peak_tflops": tpk, "frac": tflops / tpk,
                           "peak_source": tsrc, "flop_per_node": flop_node,
                           "issued_flop_per_node": flop_node_issued}}
    u2 = [x / (kT / rho0) for x in st["u2_avg"]]

    e2e = None
    if not args.no_e2e:
        hstate = torch.empty(27 * N, dtype=torch.float32, pin_memory=True)
        lat.get_state(hstate)
        passes = []
        for _ in range(3):   # median of three passes, as for the box workload
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lat.set_state(hstate)
            for _ in range(args.steps):
                lat.step(1)
                lat.stats()
            torch.cuda.synchronize()
            passes.append((time.perf_counter() - t0) * 1e3)
        e_ms = max_over_ranks(sorted(passes)[1], ws, dev)
        import ctypes
        e2e = {"value": job_mlups(N, args.steps, e_ms, ws), "unit": "MLUPS",
               "h2d_bytes_per_step": 4 * 27 * N // args.steps,
               "d2h_bytes_per_step": ctypes.sizeof(flbm.flbm_stats_t) + 16,
               "what": "flbm_set_state from pinned host + K x (flbm_step(1) + flbm_stats)",
               "passes_ms": passes, "reported": "median of 3 passes"}
        del hstate
    stats_learned = statistics(lat)
    lat.close()
    glat, gel, gk_ms, _, _, gst = timed(flbm.FLBM_GMF)
    stats_gmf = statistics(glat)
    glat.close()
    plain = {"value": job_mlups(N, args.steps, max_over_ranks(gel, ws, dev), ws), "unit": "MLUPS",
             "what": "plain GMF-FLBM (row pipeline) on the same box",
             "u2_avg_over_kT_rho0": [x / (kT / rho0) for x in gst["u2_avg"]]}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle
        from oracle import mlp as omlp
        oracle.build()
        threads = os.cpu_count() or 1
        oracle.set_threads(threads)
        m = 32
        w = oracle.tables()["w"]
        box = oracle.Box(m, m, m, tau, kT, rho0=rho0, seed=seed)
        steps, t0 = 0, time.perf_counter()
        while True:
            # the oracle's work per learned step: the network correction of
            # every node (numpy, FP64) and the GMF collision with streaming
            omlp.correction(theta, box.get_f().reshape(27, -1).T, rho0, kT, 1.0 / tau)
            box.step(1)
            steps += 1
            if time.perf_counter() - t0 > 2.0 and steps >= 3:
                break
        el = time.perf_counter() - t0
        cpu = {"value": m ** 3 * steps / el / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": "32^3 box, %d steps, each the oracle's network correction of every node "
                         "(numpy FP64) and its GMF collision + streaming (C, %d threads)" % (steps, threads)}
    if rank == 0:
        line = {
            "metric": "MLUPS of the learned-collision step (GMF-FLBM + tcgen05 network correction)",
            "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (network: bf16 operands, f32 accumulation)",
            "data": "synthetic",
            "config": {"workload": "learned collision: %d^3 box, tau 0.8, kT 1e-5, FP32 deviations AA in "
                                   "place, network 28-64-64-27 trained on %d Reg-FLBM pairs from 64^3 boxes "
                                   "with tau ~ U[0.51, 3.0]" % (n, args.train_boxes * 64 ** 3),
                       "nx": n, "ny": n, "nz": n, "tau": tau, "kT": kT, "rho0": rho0,
                       "l2": "inputs larger than L2 (%.2f GB state vs 129 MB L2)" % (108 * N / 1e9),
                       "parallelism": "replicas x%d" % ws},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "plain_kernel": plain,
            "gpu_launches": int(launches) + int(args.steps), "clocks": clocks,
            "training": training,
            "statistics": {"learned": stats_learned, "gmf": stats_gmf},
            "equipartition": {"u2_avg_over_kT_rho0": u2, "max_abs_error": max(abs(x - 1) for x in u2),
                              "samples": st["n_samples"]},
        }
        print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    rank, local, ws = dist_setup()
    try:
        if args.impl == "reference":
            return run_reference(args, rank, ws)
        if args.workload == "ensemble":
            return run_ensemble(args, rank, local, ws)
        if args.workload == "learned":
            return run_learned(args, rank, local, ws)
        return run_ours(args, rank, local, ws)
    finally:
        if ws > 1:
            import torch.distributed as dist
            if dist.is_initialized():
                dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
