"""Throughput benchmark of the fused growing-tissue LBM step on GB300.

Default workload: the 4096 x 2048 D2Q9 lattice with edge-restricted growth
(divisions within 8 rows of the front), tau = 0.8, sinusoidal initial front
(wavenumbers 1..64, amplitude 1), FP32 storage, fixed rear wall: about 4.2M
active nodes per step, so each FP32 population copy of the active window is
about 151 MB (a step reads one and writes the other), above the 129 MB L2 (no
L2 flush is needed between steps).

A step is one full time step of the method: the fused update kernel (App. A
steps 1-7) and the planner kernel, which computes the observables (front
heights, Eq. 6, the rear wall, the active mass) and selects the next step's
divisions.

Reports MLUPS = active-window node updates per second (whole job, all ranks),
the fused kernel's achieved HBM bandwidth against the measured copy peak,
an end-to-end figure through the C ABI with host buffers, the FP64 CPU oracle
timed on a bounded sample as the CPU baseline, and the SM clocks seen during
the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs one independent replica (its own seed); there is
no data-path collective.
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

from paper_2303_02210_gb300 import workloads as wl  # noqa: E402

METRIC = "MLUPS"
UNIT = "MLUPS"
WORKLOAD_NAME = "lattice_edge"


WIDTH = 4096  # lattice width of the headline workload (--width changes it, for profiling captures)
LATTICE = "d2q9"  # the headline lattice (--lattice d2q7, for profiling captures)


def workload_params(rank: int = 0) -> dict:
    return wl.lattice_edge(seed=1 + rank, sim_id=rank, width=WIDTH, lattice=LATTICE)


def workload_config(precision: str) -> dict:
    p = workload_params()
    nq = 7 if LATTICE == "d2q7" else 9  # population planes
    # one population copy of the ~1026-row active window, in MB
    mb = nq * p["width"] * 1026 * {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}[precision] / 1e6
    return {
        "workload": (f"{LATTICE.upper()} {p['width']}x{p['height']}, edge-restricted growth depth {p['edge_depth']}, "
                     f"tau {p['tau']}, g {p['growth_rate']}, sinusoidal front k {p['front_kmin']}-"
                     f"{p['front_kmax']} amplitude {p['front_amp']} at row {int(p['front_row'])}, "
                     f"sigma {p['sigma']}, fixed rear wall, {precision} storage"),
        "lattice": [p["width"], p["height"]],
        "growth_mode": p["growth_mode"],
        "precision": precision,
        "l2": (f"no flush: each step reads one {precision} population copy of the active window "
               f"(~{mb:.0f} MB) and writes the other; the 129 MB L2 holds less than that"
               if mb > 129 else
               f"no flush; NOTE each step reads only ~{mb:.0f} MB of {precision} populations, less than "
               f"the 129 MB L2" + (" (storage_16bit measures on a lattice twice as wide)"
                                   if precision in ("fp16", "bf16") else "")),
        "parallelism": "replicas",
    }


def reduce_over_ranks(ms: float, nodes: float, dist, device: str):
    """Whole-job timing of independent replicas: the slowest rank's time and
    the sum of the node updates over ranks (no data-path collective)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    n = torch.tensor([float(nodes)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("lbm_kernels.cuh", "lbm_common.cuh", "lbm_update_tma.cuh", "lbm_tma.cuh", "lbm_pair.cuh"):
        with open(os.path.join(ROOT, "paper_2303_02210_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(bytes_per_node_alg: int, nodes_per_launch: float):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    scaled to this launch's node count; None if absent or if the kernel source
    changed since the capture."""
    path = os.path.join(ROOT, "profiles", "k_update_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return float(d["dram_bytes_per_node"]) * nodes_per_launch


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region.

    Samples carry nvidia-smi's timestamp; `stop(since)` keeps those taken
    after the host time `since` (the start of the loaded window), so samples
    of an idle GPU before the run are not counted."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        """Starts sampling every 25 ms; returns once the first sample is in
        (or after 3 s)."""
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "25"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 3.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def stop(self, since: float = 0.0):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    if ts + 1.0 < since:
                        continue
                    sm.append(float(parts[2]))
                    smax.append(float(parts[3]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[6:10]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def measure_ensemble(n: int = 256, steps: int = 200, warm: int = 5) -> dict:
    """The batched form: n uneven realisations (widths 256..2048, height =
    width / 2, bulk or edge growth, FP32) advanced together by lbm_batch_step
    (graph replays of three batched launches per step: injection, the
    staged update over all members' tiles, and the planners: one block per
    member or the member's own cooperative grid), against the same
    simulations stepped one
    after another with lbm_step. Aggregate active-window node updates per
    second, device time by CUDA events around each region."""
    import torch
    from paper_2303_02210_gb300.lbm import Batch, Simulation
    params = wl.ensemble(n)
    sims = [Simulation(p, precision="fp32") for p in params]
    batch = Batch(sims)
    batch.step(warm)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def nodes():
        return sum(s.stats()["node_updates"] for s in sims)

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n0 = nodes()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return (nodes() - n0) / (e0.elapsed_time(e1) * 1e-3) / 1e6, e0.elapsed_time(e1)

    batched, ms_b = timed(lambda: batch.step(steps))

    def one_by_one():
        for s in sims:
            s.step(steps)

    single, ms_s = timed(one_by_one)
    batch.close()
    total = sum(p["width"] * p["height"] for p in params)
    del batch, sims
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return {"workload": (f"{n} realisations, widths uniform in {{256, 512, 1024, 2048}}, height = width/2, "
                         f"bulk or edge growth at random, FP32 ({total / 1e6:.0f}M lattice nodes)"),
            "steps": steps, "value": batched, "unit": UNIT, "ms_per_step": ms_b / steps,
            "one_at_a_time": single, "one_at_a_time_ms_per_step": ms_s / steps,
            "speedup": batched / single if single > 0 else None}


def measure_storage(params: dict, precision: str, steps: int = 1000, warm: int = 10,
                    update_kernel: str = "auto") -> dict:
    """One storage precision on `params`: whole-step rate by CUDA events
    over `steps` steps (no other events in that region), then the update
    kernel's average launch time over a separate pass of 200 steps with every
    update launch bracketed by events, against the measured copy peak."""
    import torch
    from paper_2303_02210_gb300.lbm import Simulation
    sim = Simulation(params, precision=precision, update_kernel=update_kernel)
    stream = sim.stream
    sim.step(warm)
    sim.sync()
    n0 = sim.stats()["node_updates"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    nodes = sim.stats()["node_updates"] - n0
    kern_steps = 200
    sim.lbm_timing_stride(1)
    sim.lbm_timing_enable(kern_steps)
    sim.step(kern_steps)
    k_launches, k_ms, k_nodes = sim.lbm_timing_read()
    bpn = sim.lbm_bytes_per_node()
    q7 = params.get("lattice", "d2q9") == "d2q7"
    kernel = {1: "k_update", 2: "k_update_tma"}[sim.stats()["update_kernel"]]
    if q7:
        kernel = kernel.replace("k_update", "k_update7")
    sim.close()
    del sim
    torch.cuda.empty_cache()
    peak, _ = measured_peak()
    launch_ms = k_ms / max(k_launches, 1)
    achieved = bpn * (k_nodes / max(k_launches, 1)) / (launch_ms * 1e-3) / 1e9 if k_ms > 0 else 0.0
    return {"precision": precision, "value": nodes / (ms * 1e-3) / 1e6, "unit": UNIT,
            "ms_per_step": ms / steps, "steps": steps, "bytes_per_node": bpn, "kernel": kernel,
            "avg_launch_ms": launch_ms, "achieved_gbs": achieved, "frac": achieved / peak}


def measure_storage_16bit() -> dict:
    """FP32 against 16-bit storage on the headline workload made twice as
    wide (8192 x 2048, front at row 1024: about 8.4M active nodes), so that
    one 16-bit population copy of the window (about 151 MB, read every step)
    is still larger than the 129 MB L2."""
    p = wl.lattice_edge(seed=1, width=8192)
    out = {"workload": (f"D2Q9 {p['width']}x{p['height']}, otherwise as the headline workload; per step "
                        f"one population copy of the window is read: ~{9 * p['width'] * 1026 * 2 / 1e6:.0f} MB "
                        f"16-bit, ~{9 * p['width'] * 1026 * 4 / 1e6:.0f} MB FP32, against the 129 MB L2")}
    for pr in ("fp32", "fp16", "bf16"):
        out[pr] = measure_storage(p, pr)
    return out


def measure_d2q7() -> dict:
    """The headline workload on the paper's triangular D2Q7 lattice (FP32:
    7 loads and 7 stores of 4 bytes per node update), with the TMA-staged
    update the automatic choice takes and, for comparison, the plain-load
    one. The sampled update launch includes k_inject, which adds the
    divisions to the stored slots just before it."""
    p = wl.lattice_edge(seed=1, lattice="d2q7")
    out = measure_storage(p, "fp32")
    plain = measure_storage(p, "fp32", update_kernel="plain")
    out["plain"] = {k: plain[k] for k in ("value", "ms_per_step", "kernel", "avg_launch_ms", "achieved_gbs", "frac")}
    out["workload"] = (f"D2Q7 {p['width']}x{p['height']}, otherwise as the headline workload "
                       f"(one window copy ~{7 * p['width'] * 1026 * 4 / 1e6:.0f} MB, just under the 129 MB L2)")
    return out


def dense_params() -> dict:
    """The headline workload with the tissue filling all but the top four of
    the 2048 rows (front at row 2044): about 8.4M active nodes, so a FP32
    step reads and writes about 604 MB of populations, twice the headline's."""
    return wl.lattice_edge(seed=1, front_row=2044.0)


def measure_dense(steps: int = 300) -> dict:
    """The dense variant (dense_params) by measure_storage. The front meets
    the top wall within the run (status bit 1); growth goes on below it."""
    p = dense_params()
    out = measure_storage(p, "fp32", steps=steps)
    out["workload"] = (f"D2Q9 {p['width']}x{p['height']}, front at row {int(p['front_row'])}, otherwise as the "
                       f"headline workload (one window copy ~{9 * p['width'] * p['height'] * 4 / 1e6:.0f} MB)")
    return out


def measure_serving(n: int = 500, rate: float = 200.0, steps=(1000, 20000), budget_gb: float = 100.0,
                    chunk: int = 100, slots: int = 256) -> dict:
    """The served form: a fixed trace of n requests (Poisson arrivals at
    `rate` per second, widths log-uniform 128..4096, height = width / 2, bulk,
    edge or density growth, g log-uniform 1e-5..1e-3, steps uniform in
    `steps`, FP32 or FP16 storage 50/50) through the continuous-batching
    loop with an HBM budget, the requests stepped through one slot batch per
    storage type; time to result per request (arrival to result on the host)
    and the aggregate node-update rate over the whole run (wall clock, from
    the first arrival to the last result)."""
    from paper_2303_02210_gb300 import serving
    trace = wl.serving_trace(n, rate=rate, steps=steps)
    reqs = [serving.Request(params=p, steps=k, arrival=t, precision=pr) for t, p, k, pr in trace]
    srv = serving.Server(hbm_budget=int(budget_gb * 2 ** 30), chunk=chunk, slots=slots)
    srv.run(reqs)
    out = serving.summary(reqs, srv)
    out["workload"] = (f"{n} requests, Poisson arrivals at {rate:g}/s, widths log-uniform 128-4096, "
                       f"height = width/2, bulk/edge/density growth, g log-uniform 1e-5..1e-3, "
                       f"{steps[0]}-{steps[1]} steps, FP32 or FP16 storage 50/50, {budget_gb:g} GB budget, "
                       f"slot batches of {slots} per storage type, ticks of at most {chunk} steps")
    return out


def oracle_rate(params: dict, steps: int):
    """The FP64 CPU oracle, as it stands, on `steps` steps of the workload.
    Returns (MLUPS counted over the same active window the GPU updates,
    seconds, window nodes per step)."""
    import numpy as np
    from oracle.oracle import OracleSim
    o = OracleSim(params)
    rho = o.pops().sum(0)
    rows = np.nonzero(rho.any(1))[0]
    y_hi = min(params["height"], int(rows.max()) + 2) if len(rows) else 1
    window = params["width"] * (y_hi - o.stats()["y_r"])
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    o.close()
    return window * steps / dt / 1e6, dt, window


def _oracle_child(steps: int, start_at: float):
    """One independent oracle process of the all-core baseline: creates the
    workload, waits for the common start time, steps, prints JSON."""
    from oracle.oracle import OracleSim
    params = workload_params()
    o = OracleSim(params)
    wait = start_at - time.time()
    if wait > 0:
        time.sleep(wait)
    t0 = time.time()
    o.step(steps)
    t1 = time.time()
    o.close()
    print(json.dumps({"start": t0, "end": t1}), flush=True)


def oracle_rate_cores(steps: int, want: int = 0):
    """The FP64 oracle, as it stands (single-threaded), run as independent
    processes on the host cores at once, each on `steps` steps of the same
    workload. Returns (aggregate MLUPS over the active window, processes,
    seconds of the common stepping region). The process count is nproc,
    capped so that their lattices take at most 60% of the available memory."""
    params = workload_params()
    nq = 7 if params.get("lattice") == "d2q7" else 9
    per = 3 * nq * params["width"] * params["height"] * 8 + (64 << 20)
    n = want or (os.cpu_count() or 1)
    try:
        with open("/proc/meminfo") as fh:
            avail = next(int(l.split()[1]) * 1024 for l in fh if l.startswith("MemAvailable"))
        n = max(1, min(n, int(0.6 * avail // per)))
    except Exception:
        pass
    start_at = time.time() + 12.0
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    procs = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-child", str(steps),
                               "--oracle-start", repr(start_at), "--width", str(WIDTH), "--lattice", LATTICE],
                              stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, env=env, cwd=ROOT)
             for _ in range(n)]
    spans = []
    for pr in procs:
        out, _ = pr.communicate()
        if pr.returncode == 0:
            spans.append(json.loads(out.decode().strip().splitlines()[-1]))
    if not spans:
        return None
    # the window the GPU updates (as oracle_rate counts it)
    from oracle.oracle import OracleSim
    import numpy as np
    o = OracleSim(params)
    rho = o.pops().sum(0)
    rows = np.nonzero(rho.any(1))[0]
    y_hi = min(params["height"], int(rows.max()) + 2) if len(rows) else 1
    window = params["width"] * (y_hi - o.stats()["y_r"])
    o.close()
    t0 = min(sp["start"] for sp in spans)
    t1 = max(sp["end"] for sp in spans)
    return len(spans) * window * steps / (t1 - t0) / 1e6, len(spans), t1 - t0


def run_reference(args):
    """Reference arm: the FP64 CPU oracle (no reference code exists for this
    paper) on the host cores, same workload, metric and unit: one process per
    host core (as many as memory allows), each an independent single-threaded
    oracle run of the bounded sample, stepping at the same time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    params = workload_params()
    warm = min(args.warmup, 1)
    steps = max(1, min(args.steps, 12))
    res = oracle_rate_cores(steps)
    if res is None:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle processes failed"}), flush=True)
        return
    rate, cores, dt = res
    sample = (f"{cores} independent single-threaded oracle processes at once, each {steps} steps of the full "
              f"{params['width']}x{params['height']} workload (created before the common start, so the "
              f"{warm} warm-up step is the creation); aggregate rate over the active-window nodes per step "
              f"the GPU updates")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": dt / steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        # our arm's workload description; the oracle computes in FP64 (dtype)
        "config": workload_config(args.precision),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16", "bf16"])
    ap.add_argument("--update-kernel", default="auto",
                    help="auto, plain, tma, tma1, tma_sel, shared, or the numeric lbm_params_t code")
    ap.add_argument("--cpu-steps", type=int, default=12)
    ap.add_argument("--width", type=int, default=4096,
                    help="lattice width (4096: the headline workload; others for profiling captures)")
    ap.add_argument("--lattice", default="d2q9", choices=["d2q9", "d2q7"],
                    help="lattice of the main run (d2q9: the headline workload; d2q7 for profiling captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-child", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-start", type=float, default=0.0, help=argparse.SUPPRESS)
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the batched-ensemble, serving and 16-bit storage measurements")
    args = ap.parse_args()
    if args.update_kernel.isdigit():
        args.update_kernel = int(args.update_kernel)
    global WIDTH, LATTICE
    WIDTH = args.width
    LATTICE = args.lattice
    if args.oracle_child:
        _oracle_child(args.oracle_child, args.oracle_start)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.warmup < 3:
        args.warmup = 3

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2303_02210_gb300.lbm import Simulation

    params = workload_params(rank)
    sim = Simulation(params, precision=args.precision, update_kernel=args.update_kernel)
    stream = sim.stream
    kernel_used = {1: "k_update (plain loads)", 2: "k_update_tma (bulk tensor copies)"}[sim.stats()["update_kernel"]]
    if LATTICE == "d2q7":
        kernel_used = kernel_used.replace("k_update", "k_update7")

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- device-resident throughput (inputs resident in HBM) ----
    # the timed region holds the K steps and nothing else: no per-launch
    # events (an event pair keeps the update from overlapping the planner
    # before it), only the outer pair
    # clocks: sampled from the warm-up to the end of a loaded window of at
    # least 0.3 s that contains the timed region (untimed steps follow it
    # when the timed region alone is shorter than the sampling interval)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t_load = time.time()
    sim.step(args.warmup)
    sim.sync()
    st0 = sim.stats()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    st1 = sim.stats()
    nodes = st1["node_updates"] - st0["node_updates"]
    launches = st1["launches"] - st0["launches"]
    status = st1["status"]
    # ---- the update kernel's launch duration: a separate pass right after,
    # every update launch bracketed by CUDA events on the simulation's stream
    kern_steps = max(64, min(args.steps, 500))
    sim.lbm_timing_stride(1)
    sim.lbm_timing_enable(kern_steps)
    sim.step(kern_steps)
    k_launches, k_ms, k_nodes = sim.lbm_timing_read()
    bpn = sim.lbm_bytes_per_node()
    while time.time() - t_load < 0.3:
        sim.step(200)
        sim.sync()
    clk = clocks.stop(since=t_load)
    if clk is not None:
        clk["window"] = (f"{clk['samples']} nvidia-smi samples (25 ms apart) from the warm-up through the timed "
                         f"region, the kernel-timing pass and untimed steps to 0.3 s of load")
    sim.close()
    del sim

    ms_max, nodes_all = reduce_over_ranks(ms, nodes, dist, "cuda")
    value = nodes_all / (ms_max * 1e-3) / 1e6

    # ---- end to end through the C ABI with host buffers ----
    # lbm_create from host parameters, then every step lbm_step(1) and the copy
    # of that step's front heights and exact Eq. 6 sums into pinned host
    # buffers (lbm_front_heights_async, no wait per step), one wait at the end,
    # Eq. 6 worked out on the host for every step, lbm_destroy
    from paper_2303_02210_gb300.lbm import lbm_eq6_n
    # (a fixed job of 1000 steps, whatever --steps is)
    e2e_steps = 1000
    W = params["width"]
    hbuf = torch.empty((e2e_steps, W), dtype=torch.int32, pin_memory=True)
    sbuf = torch.empty((e2e_steps, 2), dtype=torch.int64, pin_memory=True)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim2 = Simulation(params, precision=args.precision, update_kernel=args.update_kernel)
    for k in range(e2e_steps):
        sim2.step(1)
        sim2.lbm_front_heights_async(hbuf[k], sbuf[k])
    sim2.sync()
    eq6 = lbm_eq6_n(sbuf, W)[1]
    st2 = sim2.stats()
    sim2.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    assert len(eq6) == e2e_steps and int(hbuf[-1].max()) > 0
    e2e_max, e2e_nodes = reduce_over_ranks(e2e_s, st2["node_updates"], dist, "cuda")
    e2e_value = e2e_nodes / e2e_max / 1e6
    # bytes that cross the bus: the initial front profile (W int32) once at
    # creation; W int32 heights and the two int64 Eq. 6 sums every step
    h2d = W * 4 / e2e_steps
    d2h = W * 4 + 16

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peak, peak_kind = measured_peak()
    # nodes and time per launch over the kernel-timing pass
    nodes_per_launch = k_nodes / max(k_launches, 1)
    launch_ms = k_ms / max(k_launches, 1)
    achieved = bpn * nodes_per_launch / (launch_ms * 1e-3) / 1e9 if k_ms > 0 else 0.0
    # (the committed traffic figure is the D2Q9 update's)
    traffic = profiled_traffic(bpn, nodes_per_launch) if LATTICE == "d2q9" else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": "synthetic", "config": workload_config(args.precision),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": kernel_used + ": fused stream/collide/front/noise",
                     "algorithmic_bytes_per_launch": bpn * nodes_per_launch,
                     "avg_launch_ms": launch_ms, "timed_launches": int(k_launches),
                     "kernel_timing": (f"{int(k_launches)} consecutive update launches right after the timed "
                                       f"region, each bracketed by CUDA events on the simulation's stream"),
                     "peak_source": peak_kind},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "what": (f"lbm_create from host parameters, then {e2e_steps} x (lbm_step(1) + "
                         f"lbm_front_heights_async of that step's heights and Eq. 6 sums into pinned host "
                         f"buffers), one wait, Eq. 6 on the host for every step (lbm_eq6_n), lbm_destroy")},
        "gpu_launches": int(launches),
        "clocks": clk,
        "status": status,
    }
    if world == 1 and not args.no_ensemble:
        line["ensemble"] = measure_ensemble()
        line["serving"] = measure_serving()
        line["storage_16bit"] = measure_storage_16bit()
        line["d2q7"] = measure_d2q7()
        try:
            line["dense"] = measure_dense()
        except Exception as e:  # reported, not fatal: the headline line stands
            line["dense"] = {"error": f"{type(e).__name__}: {e}"}
    if world == 1 and not args.no_cpu_baseline:
        rate, dt, window = oracle_rate(workload_params(), args.cpu_steps)
        one = {"value": rate, "cores": 1,
               "sample": (f"{args.cpu_steps} steps of the FP64 CPU oracle on the full "
                          f"{params['width']}x{params['height']} workload ({dt:.1f} s, one thread); "
                          f"rate over the {window} active-window nodes per step")}
        allc = oracle_rate_cores(args.cpu_steps)
        if allc is not None:
            rate_n, cores, dt_n = allc
            line["cpu_baseline"] = {
                "value": rate_n, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": (f"{cores} independent single-threaded oracle processes stepping at once "
                           f"({os.cpu_count()} host cores), each {args.cpu_steps} steps of the full "
                           f"{params['width']}x{params['height']} workload ({dt_n:.1f} s); aggregate rate "
                           f"over the {window} active-window nodes per step"),
                "single_core": one,
            }
        else:
            line["cpu_baseline"] = dict(one, unit=UNIT, kind="oracle")
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
