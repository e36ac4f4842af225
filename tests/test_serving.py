"""The serving loop (continuous batching): admission by footprint in arrival
order, slot batches that requests join and leave, ticks over the resident
simulations, release on completion — the loop's logic with stand-ins on the
CPU, and on the GPU that every served result equals the same request run
alone and the oracle's run of it."""
import numpy as np
import pytest

from paper_2303_02210_gb300 import serving
from paper_2303_02210_gb300 import workloads as wl


class FakeSim:
    """Stands in for Simulation: counts steps, reports them as node updates."""
    live = 0
    peak = 0

    def __init__(self, params, precision="fp32", stream=None):
        self.params, self.n = params, 0
        FakeSim.live += 1
        FakeSim.peak = max(FakeSim.peak, FakeSim.live)

    def step(self, n):
        self.n += n

    def stats(self):
        return {"node_updates": self.n * self.params["width"], "step": self.n}

    def front_heights(self):
        return np.zeros(self.params["width"], np.int32), 0.0, 0.0

    def close(self):
        FakeSim.live -= 1


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001  # every look at the clock advances it a millisecond
        return self.t


def test_loop_admits_by_footprint_in_arrival_order_and_finishes_all():
    FakeSim.live = FakeSim.peak = 0
    reqs = [serving.Request(params={"width": w, "height": w // 2}, steps=s, arrival=a)
            for a, w, s in [(0.0, 64, 250), (0.0, 64, 100), (0.002, 128, 300), (0.003, 64, 50), (0.05, 32, 120)]]
    srv = serving.Server(hbm_budget=200, chunk=100, clock=FakeClock(), simulation=FakeSim, batch=None,
                         footprint=lambda p, prec: p["width"], new_stream=lambda: None, synchronize=lambda: None)
    srv.run(reqs)
    assert FakeSim.live == 0 and FakeSim.peak <= 3  # never more than the budget holds (64+64+64 or 64+128)
    for r in reqs:
        assert r.result["stats"]["step"] == r.steps
        assert r.admitted >= r.arrival and r.finished > r.admitted
    # arrival order: the 128-wide request waited for room and nothing overtook it
    assert reqs[3].admitted >= reqs[2].admitted
    assert srv.node_updates == sum(r.steps * r.params["width"] for r in reqs)
    s = serving.summary(reqs, srv)
    assert s["p50_s"] <= s["p99_s"] and s["requests"] == 5


class FakeSlotBatch:
    """Stands in for Batch.empty: fixed slots, members join and leave; every
    member must be in the batch while it is stepped through it, and leave
    before it is released."""
    made = []

    def __init__(self, slots, precision, lattice):
        self.slots, self.precision, self.lattice = slots, precision, lattice
        self.members = []
        self.closed = False
        FakeSlotBatch.made.append(self)

    def attach(self, sim):
        assert not self.closed and sim not in self.members
        assert sim.precision == self.precision
        if len(self.members) >= self.slots:
            raise RuntimeError("full")
        self.members.append(sim)
        sim.in_batch = self

    def detach(self, sim):
        self.members.remove(sim)
        sim.in_batch = None

    def step(self, n):
        assert n >= 1
        for m in self.members:
            m.step(n)
            assert m.n <= m.steps_wanted, "a member ran past its step count"

    def close(self):
        assert not self.members
        self.closed = True


class FakeSimForBatch(FakeSim):
    wanted = {}

    def __init__(self, params, precision="fp32", stream=None):
        super().__init__(params, precision, stream)
        self.precision = precision
        self.in_batch = None
        self.steps_wanted = FakeSimForBatch.wanted[id(params)]

    def close(self):
        assert self.in_batch is None, "released while in its batch"
        super().close()


def test_loop_steps_requests_through_slot_batches():
    """Requests join the slot batch of their storage type at admission and
    leave it when done; a batch is made once per storage type and never
    rebuilt; a tick steps a batch by what its members all have left (at most
    a chunk), so every request runs exactly its steps; requests that find
    their batch full and requests periodic in y run on their own."""
    FakeSim.live = FakeSim.peak = 0
    FakeSlotBatch.made = []
    specs = [(0.0, 64, 250, "fp32", 0), (0.0, 64, 100, "fp16", 0), (0.0, 32, 430, "fp32", 0),
             (0.001, 32, 90, "fp32", 0), (0.002, 64, 300, "fp16", 0), (0.003, 32, 200, "fp32", 0),
             (0.003, 32, 170, "fp32", 1), (0.004, 16, 333, "fp32", 0)]
    reqs = []
    FakeSimForBatch.wanted = {}
    for a, w, k, pr, yp in specs:
        p = {"width": w, "height": w // 2, "y_periodic": yp}
        FakeSimForBatch.wanted[id(p)] = k
        reqs.append(serving.Request(params=p, steps=k, arrival=a, precision=pr))
    srv = serving.Server(hbm_budget=10_000, chunk=100, clock=FakeClock(), simulation=FakeSimForBatch,
                         footprint=lambda p, prec: p["width"], new_stream=lambda: None, synchronize=lambda: None,
                         batch=FakeSlotBatch, slots=3)
    srv.run(reqs)
    assert FakeSim.live == 0
    assert sorted((b.lattice, b.precision) for b in FakeSlotBatch.made) == [("d2q9", "fp16"), ("d2q9", "fp32")]
    assert all(b.closed and not b.members for b in FakeSlotBatch.made)
    for r in reqs:
        assert r.result["stats"]["step"] == r.steps
    assert srv.node_updates == sum(r.steps * r.params["width"] for r in reqs)
    # the y-periodic request never joins; with three slots per batch, at
    # least one of the five plain fp32 requests had to wait its turn alone
    assert 0 < srv.batched_requests < len(reqs)
    assert serving.Server.batch_key(reqs[6]) is None


@pytest.mark.gpu
def test_served_results_equal_requests_run_alone():
    """Requests of mixed sizes, growth modes and rates served together with
    a budget that forces queueing end exactly where each ends alone."""
    from paper_2303_02210_gb300.lbm import Simulation, lbm_footprint
    trace = wl.serving_trace(10, rate=500.0, steps=(100, 400), seed=7)
    trace = [(t, dict(p, width=min(p["width"], 512), height=min(p["width"], 512) // 2,
                      front_row=float(min(p["width"], 512) // 8)), n, pr) for t, p, n, pr in trace]
    assert {pr for *_, pr in trace} == {"fp16", "fp32"}
    reqs = [serving.Request(params=p, steps=n, arrival=t, precision=pr, keep_populations=True)
            for t, p, n, pr in trace]
    budget = 3 * max(lbm_footprint(r.params, "fp32") for r in reqs)
    srv = serving.Server(hbm_budget=budget, chunk=64, batch=None)
    srv.run(reqs)
    for r in reqs:
        alone = Simulation(r.params, precision=r.precision)
        alone.step(r.steps)
        assert np.array_equal(alone.pops(), r.result["populations"])
        assert alone.stats()["node_updates"] == r.result["stats"]["node_updates"]
        assert np.array_equal(alone.heights(), r.result["heights"])
        alone.close()
    s = serving.summary(reqs, srv)
    assert s["p50_s"] <= s["p99_s"] and s["aggregate_mlups"] > 0


@pytest.mark.gpu
@pytest.mark.parametrize("slots", [1, 256])
def test_served_results_equal_requests_run_alone_with_batching(slots):
    """The same through slot batches (members joining and leaving as
    requests come and go; with one slot per batch most requests run alone
    beside them): bit for bit what each request gives alone, and the
    batches' graphs captured once."""
    from paper_2303_02210_gb300.lbm import Batch, Simulation, lbm_footprint
    trace = wl.serving_trace(10, rate=500.0, steps=(100, 400), seed=8)
    trace = [(t, dict(p, width=min(p["width"], 512), height=min(p["width"], 512) // 2,
                      front_row=float(min(p["width"], 512) // 8)), n, pr) for t, p, n, pr in trace]
    reqs = [serving.Request(params=p, steps=n, arrival=t, precision=pr, keep_populations=True)
            for t, p, n, pr in trace]
    made = []

    def batch(n, precision, lattice):
        b = Batch.empty(n, precision, lattice)
        made.append(b)
        return b

    captures = {}
    orig_close = Batch.close

    def close(self):
        if getattr(self, "_h", None):
            captures[id(self)] = self.captures
        orig_close(self)

    Batch.close = close
    try:
        budget = 4 * max(lbm_footprint(r.params, "fp32") for r in reqs)
        srv = serving.Server(hbm_budget=budget, chunk=32, batch=batch, slots=slots)
        srv.run(reqs)
    finally:
        Batch.close = orig_close
    assert made and srv.batched_requests > 0
    if slots == 1:
        assert srv.batched_requests < len(reqs)
    assert all(captures[id(b)] == 1 for b in made), captures
    for r in reqs:
        alone = Simulation(r.params, precision=r.precision)
        alone.step(r.steps)
        assert np.array_equal(alone.pops(), r.result["populations"])
        assert np.array_equal(alone.heights(), r.result["heights"])
        alone.close()


@pytest.mark.gpu
@pytest.mark.parametrize("batching", [False, True])
def test_served_results_against_the_oracle(batching):
    """Small requests served together (queueing under a budget, optionally
    batched) against the FP64 oracle run of each request alone: FP64 requests
    bit for bit (populations, heights, counters), FP32 requests within 1e-5
    in density with no mask or height flips and the same divisions."""
    from oracle.oracle import OracleSim
    from paper_2303_02210_gb300.lbm import Batch, lbm_footprint
    trace = wl.serving_trace(8, rate=500.0, steps=(60, 240), seed=11)
    reqs = []
    for i, (t, p, n, _) in enumerate(trace):
        W = 32 * (2 + i % 5)  # 64 .. 192 columns
        p = dict(p, width=W, height=W // 2, front_row=float(W // 8))
        reqs.append(serving.Request(params=p, steps=n, arrival=t, precision="fp64" if i % 2 else "fp32",
                                    keep_populations=True))
    budget = 3 * max(lbm_footprint(r.params, "fp64") for r in reqs)
    srv = serving.Server(hbm_budget=budget, chunk=32, batch=Batch.empty if batching else None, slots=4)
    srv.run(reqs)
    for r in reqs:
        o = OracleSim(r.params)
        o.step(r.steps)
        st, so = r.result["stats"], o.stats()
        assert np.array_equal(r.result["heights"], o.heights())
        assert st["ns_total"] == so["ns_total"] and st["div_total"] == so["div_total"]
        if r.precision == "fp64":
            assert np.array_equal(r.result["populations"], o.pops())
            assert st["mass_fix"] == so["mass_fix"] and st["carry"] == so["carry"]
        else:
            rho_g = r.result["populations"].sum(0)
            rho_o = o.pops().sum(0)
            assert np.abs(rho_g - rho_o).max() / np.abs(rho_o).max() <= 1e-5
        o.close()
