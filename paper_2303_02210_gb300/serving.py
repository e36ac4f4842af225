"""Serving: a request loop with continuous batching over the C ABI.

Requests (a lattice to grow for a number of steps) arrive over time. The loop
admits queued requests while their device footprint (``lbm_footprint``) fits
in an HBM budget, keeps every admitted simulation resident with its own CUDA
stream, and advances all of them in ticks of ``chunk`` steps, each on its own
stream, so the kernels of different requests overlap on the GPU. Optionally
(``batch``), the resident requests with at least ``chunk`` steps to go and a
planner small enough for one block (``lbm_plan_capacity`` at most
``batch_max_divisions``) are stepped as batches instead (one per storage
type: three batched launches per step for all of them, see
``lbm_batch_create``; a batch is rebuilt when its membership changes). That
pays for many small requests; on a trace dominated by large lattices the
rebuilds cost more than the batched launches save. A request that has run its steps is
read back (front heights, Eq. 6 sums, counters, optionally the populations)
and released, which frees memory for the queue at the next tick. Every
simulation draws its own counter-based random streams, so a result does not
depend on what else was resident, nor on whether it was batched.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, List, Optional

import numpy as np

from .lbm import Simulation, lbm_footprint


@dataclasses.dataclass
class Request:
    params: dict
    steps: int
    arrival: float = 0.0          # seconds after the loop starts
    precision: str = "fp32"
    keep_populations: bool = False
    # filled in by the loop
    admitted: Optional[float] = None
    finished: Optional[float] = None
    result: Optional[dict] = None

    @property
    def latency(self) -> Optional[float]:
        """Time to result: from arrival to the result being on the host."""
        return None if self.finished is None else self.finished - self.arrival


class Server:
    """Continuous-batching loop over resident simulations.

    hbm_budget  bytes of device memory the resident simulations may use
                together (their arenas, as ``lbm_footprint`` reports);
    chunk       steps enqueued per resident simulation and tick;
    clock       a monotonic clock in seconds;
    simulation, footprint, new_stream, synchronize
                the simulation class, lbm_footprint, a CUDA stream factory and
                a device-wide wait (the defaults use this library and torch;
                tests of the loop's own logic pass stand-ins);
    batch       a factory of batches (list of simulations -> object with
                step(n) and close()), e.g. the library's Batch; None: no
                batching;
    capacity    divisions per step a request's planner holds (params,
                precision -> int; lbm_plan_capacity by default);
    batch_max_divisions  the largest capacity that is batched.
    """

    def __init__(self, hbm_budget: int, chunk: int = 100, clock: Callable[[], float] = time.perf_counter,
                 simulation=None, footprint=None, new_stream=None, synchronize=None, batch=None,
                 capacity=None, batch_max_divisions: int = 8192):
        if hbm_budget <= 0 or chunk <= 0:
            raise ValueError("hbm_budget and chunk must be positive")
        self.hbm_budget = int(hbm_budget)
        self.chunk = int(chunk)
        self.clock = clock
        self.node_updates = 0
        self.ticks = 0
        self.peak_resident = 0
        if simulation is None:
            # resident requests share the GPU: the update kernel's form for that
            # (15.1 against 12.5 G node updates/s aggregate on a hundred requests)
            def simulation(params, precision="fp32", stream=None):
                return Simulation(params, precision=precision, stream=stream, update_kernel="shared")
        self.simulation = simulation
        self.footprint = footprint or lbm_footprint
        self.new_stream = new_stream
        self.synchronize = synchronize
        self.batch = batch
        self.batches_built = 0
        if capacity is None and batch is not None:
            from .lbm import lbm_plan_capacity
            capacity = lbm_plan_capacity
        self.capacity = capacity
        self.batch_max_divisions = int(batch_max_divisions)

    def run(self, requests: List[Request]) -> List[Request]:
        """Serves `requests` (arrival times relative to the start of the run)
        and returns them with admission and finish times and results."""
        if self.new_stream is None or self.synchronize is None:
            import torch
            self.new_stream = self.new_stream or torch.cuda.Stream
            self.synchronize = self.synchronize or torch.cuda.synchronize
        for r in requests:
            r.footprint = self.footprint(r.params, r.precision)
            r.batchable = self.batch is not None and \
                self.capacity(r.params, r.precision) <= self.batch_max_divisions
            if r.footprint > self.hbm_budget:
                raise ValueError(f"a {r.params['width']} x {r.params['height']} request needs {r.footprint} bytes, "
                                 f"more than the budget of {self.hbm_budget}")
        pending = sorted(requests, key=lambda r: r.arrival)
        active = []  # [request, simulation, stream, steps done]
        batches = {}  # storage type -> (member ids, batch)
        used = 0
        t0 = self.clock()
        while pending or active:
            now = self.clock() - t0
            # admission in arrival order while the footprint fits (a request
            # that does not fit waits, and so does everything behind it)
            while pending and pending[0].arrival <= now and used + pending[0].footprint <= self.hbm_budget:
                r = pending.pop(0)
                stream = self.new_stream()
                sim = self.simulation(r.params, precision=r.precision, stream=stream)
                r.admitted = self.clock() - t0
                used += r.footprint
                active.append([r, sim, stream, 0])
            if not active:
                wait = pending[0].arrival - (self.clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.005))
                continue
            self.peak_resident = max(self.peak_resident, len(active))
            # one tick: `chunk` steps of the requests with that many to go,
            # as one batch per storage type; the rest finish on their own
            # streams (their kernels overlap with the batches')
            groups = {}
            for a in active:
                if a[0].batchable and a[0].steps - a[3] >= self.chunk:
                    groups.setdefault(a[0].precision, []).append(a)
                else:
                    n = min(self.chunk, a[0].steps - a[3])
                    a[1].step(n)
                    a[3] += n
            for prec, group in groups.items():
                key = tuple(id(a[1]) for a in group)
                if prec not in batches or batches[prec][0] != key:
                    if prec in batches:
                        batches.pop(prec)[1].close()
                    batches[prec] = (key, self.batch([a[1] for a in group]))
                    self.batches_built += 1
                batches[prec][1].step(self.chunk)
                for a in group:
                    a[3] += self.chunk
            self.synchronize()
            self.ticks += 1
            # a batch goes before any of its members is released
            done = {id(a[1]) for a in active if a[3] >= a[0].steps}
            for prec in [p for p, (key, _) in batches.items() if done.intersection(key)]:
                batches.pop(prec)[1].close()
            still = []
            for r, sim, stream, done in active:
                if done < r.steps:
                    still.append([r, sim, stream, done])
                    continue
                st = sim.stats()
                h, hbar, w = sim.front_heights()
                r.result = {"stats": st, "heights": h, "hbar": hbar, "w": w}
                if r.keep_populations:
                    r.result["populations"] = sim.pops()
                r.finished = self.clock() - t0
                self.node_updates += st["node_updates"]
                sim.close()
                used -= r.footprint
            active = still
        for _, b in batches.values():
            b.close()
        self.makespan = self.clock() - t0
        return requests


def summary(requests: List[Request], server: Server) -> dict:
    """Time-to-result percentiles and aggregate throughput of a served trace."""
    lat = np.array([r.latency for r in requests], dtype=np.float64)
    span = max(r.arrival for r in requests) - min(r.arrival for r in requests)
    return {
        "requests": len(requests),
        "p50_s": float(np.percentile(lat, 50)),
        "p99_s": float(np.percentile(lat, 99)),
        "aggregate_mlups": server.node_updates / server.makespan / 1e6,
        "makespan_s": server.makespan,
        "offered_req_per_s": (len(requests) - 1) / span if span > 0 else None,
        "sustained_req_per_s": len(requests) / server.makespan,
        "peak_resident": server.peak_resident,
        "ticks": server.ticks,
    }
