"""Serving: a request loop with continuous batching over the C ABI.

Requests (a lattice to grow for a number of steps) arrive over time. The loop
admits queued requests while their device footprint (``lbm_footprint``) fits
in an HBM budget and keeps every admitted simulation resident. Resident
requests are stepped through slot batches (``lbm_batch_create_empty``): one
per lattice and storage type, made once with a fixed number of slots. A
request joins its batch when it is admitted and leaves it when it has run its
steps (``lbm_batch_attach`` / ``lbm_batch_detach``). Neither rewrites more
than table entries in device memory, so the batch's captured graphs serve the
whole run. A tick advances every batch by ``chunk`` steps, or by fewer when a
member has fewer left, so that no member runs past its own step count. A step
of a batch is three launches for all of its members. A request that finds no
free slot (or none for its kind: a lattice periodic in y would take the
staged update from its whole batch) is stepped on its own stream, its kernels
overlapping with the batches'.

Each tick enqueues the steps first and then creates the simulations of
newly admitted requests while the GPU works. After the tick's
synchronisation, finished requests leave their batches and are read back
(front heights, Eq. 6 sums, counters, optionally the populations) and
released, and the new ones join. Every simulation draws its own
counter-based random streams, so a result does not depend on what else was
resident, nor on whether it was batched.
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


class _Resident:
    __slots__ = ("req", "sim", "done", "batch")

    def __init__(self, req, sim):
        self.req, self.sim, self.done, self.batch = req, sim, 0, None

    @property
    def left(self) -> int:
        return self.req.steps - self.done


class Server:
    """Continuous-batching loop over resident simulations.

    hbm_budget  bytes of device memory the resident simulations may use
                together (their arenas, as ``lbm_footprint`` reports);
    chunk       steps per tick (fewer when a batch member has fewer left);
    clock       a monotonic clock in seconds;
    simulation, footprint, new_stream, synchronize
                the simulation class, lbm_footprint, a CUDA stream factory and
                a device-wide wait (the defaults use this library and torch;
                tests of the loop's own logic pass stand-ins);
    batch       a factory of slot batches, (slots, precision, lattice) ->
                object with attach(sim), detach(sim), step(n), close()
                (attach raises when the batch is full); the library's
                ``Batch.empty`` by default; None: every request on its own;
    slots       slots per batch.
    """

    def __init__(self, hbm_budget: int, chunk: int = 100, clock: Callable[[], float] = time.perf_counter,
                 simulation=None, footprint=None, new_stream=None, synchronize=None, batch="default",
                 slots: int = 256):
        if hbm_budget <= 0 or chunk <= 0 or slots <= 0:
            raise ValueError("hbm_budget, chunk and slots must be positive")
        self.hbm_budget = int(hbm_budget)
        self.chunk = int(chunk)
        self.slots = int(slots)
        self.clock = clock
        self.node_updates = 0
        self.ticks = 0
        self.peak_resident = 0
        self.batched_requests = 0
        if batch == "default":
            from .lbm import Batch
            batch = Batch.empty
        self.batch = batch
        if simulation is None:
            # requests stepped on their own share the GPU with the batches:
            # the update kernel's form for that
            def simulation(params, precision="fp32", stream=None):
                kernel = "auto" if batch is not None else "shared"
                return Simulation(params, precision=precision, stream=stream, update_kernel=kernel)
        self.simulation = simulation
        self.footprint = footprint or lbm_footprint
        self.new_stream = new_stream
        self.synchronize = synchronize

    @staticmethod
    def batch_key(r: Request):
        """The slot batch a request can join (None: stepped on its own)."""
        if r.params.get("y_periodic"):
            return None
        return (r.params.get("lattice", "d2q9"), r.precision)

    def run(self, requests: List[Request]) -> List[Request]:
        """Serves `requests` (arrival times relative to the start of the run)
        and returns them with admission and finish times and results."""
        if self.new_stream is None or self.synchronize is None:
            import torch
            self.new_stream = self.new_stream or torch.cuda.Stream
            self.synchronize = self.synchronize or torch.cuda.synchronize
        for r in requests:
            r.footprint = self.footprint(r.params, r.precision)
            if r.footprint > self.hbm_budget:
                raise ValueError(f"a {r.params['width']} x {r.params['height']} request needs {r.footprint} bytes, "
                                 f"more than the budget of {self.hbm_budget}")
        pending = sorted(requests, key=lambda r: r.arrival)
        active: List[_Resident] = []
        joining: List[_Resident] = []  # created during the last tick, not yet in a batch
        batches = {}                   # batch key -> [batch, members]
        used = 0
        t0 = self.clock()

        def admit():
            nonlocal used
            # in arrival order while the footprint fits (a request that does
            # not fit waits, and so does everything behind it)
            now = self.clock() - t0
            while pending and pending[0].arrival <= now and used + pending[0].footprint <= self.hbm_budget:
                r = pending.pop(0)
                sim = self.simulation(r.params, precision=r.precision, stream=self.new_stream())
                r.admitted = self.clock() - t0
                used += r.footprint
                joining.append(_Resident(r, sim))

        def join():
            for a in joining:
                key = self.batch_key(a.req) if self.batch is not None else None
                if key is not None:
                    if key not in batches:
                        batches[key] = [self.batch(self.slots, key[1], key[0]), 0]
                    entry = batches[key]
                    if entry[1] < self.slots:
                        entry[0].attach(a.sim)
                        entry[1] += 1
                        a.batch = key
                        self.batched_requests += 1
                active.append(a)
            joining.clear()

        while pending or active or joining:
            join()
            if not active:
                admit()
                if not joining and pending:
                    wait = pending[0].arrival - (self.clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.005))
                continue
            self.peak_resident = max(self.peak_resident, len(active))
            # one tick: each batch by the steps its members all have left (at
            # most `chunk`), the rest on their own streams
            for key, entry in batches.items():
                left = [a.left for a in active if a.batch == key]
                if not left:
                    continue
                n = min(self.chunk, min(left))
                entry[0].step(n)
                for a in active:
                    if a.batch == key:
                        a.done += n
            for a in active:
                if a.batch is None:
                    n = min(self.chunk, a.left)
                    a.sim.step(n)
                    a.done += n
            admit()  # while the GPU works
            self.synchronize()
            self.ticks += 1
            still = []
            for a in active:
                if a.left > 0:
                    still.append(a)
                    continue
                if a.batch is not None:
                    entry = batches[a.batch]
                    entry[0].detach(a.sim)
                    entry[1] -= 1
                r, sim = a.req, a.sim
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
        for entry in batches.values():
            entry[0].close()
        self.batches_built = len(batches)
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
        "batched_requests": server.batched_requests,
        "ticks": server.ticks,
    }
