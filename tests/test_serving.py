"""The serving loop (continuous batching): admission by footprint in arrival
order, ticks over the resident simulations, release on completion — the
loop's logic with stand-ins on the CPU, and on the GPU that every served
result equals the same request run alone."""
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
    srv = serving.Server(hbm_budget=200, chunk=100, clock=FakeClock(), simulation=FakeSim,
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


class FakeBatch:
    """Stands in for Batch: steps its members; members must outlive it."""
    open_members = set()
    built = 0

    def __init__(self, sims):
        self.sims = list(sims)
        assert not FakeBatch.open_members.intersection(id(m) for m in self.sims)
        FakeBatch.open_members.update(id(m) for m in self.sims)
        FakeBatch.built += 1

    def step(self, n):
        for m in self.sims:
            m.step(n)

    def close(self):
        FakeBatch.open_members.difference_update(id(m) for m in self.sims)


class FakeSimInBatch(FakeSim):
    def close(self):
        assert id(self) not in FakeBatch.open_members, "released while its batch was open"
        super().close()


def test_loop_batches_requests_with_a_chunk_to_go():
    """Requests with at least a chunk of steps left are stepped through one
    batch per storage type (rebuilt when the membership changes, closed
    before a member is released); the rest finish alone; every request still
    runs exactly its steps."""
    FakeSim.live = FakeSim.peak = 0
    FakeBatch.open_members, FakeBatch.built = set(), 0
    specs = [(0.0, 64, 250, "fp32"), (0.0, 64, 100, "fp16"), (0.0, 32, 430, "fp32"), (0.001, 32, 90, "fp32"),
             (0.002, 64, 300, "fp16"), (0.003, 32, 200, "fp32")]
    reqs = [serving.Request(params={"width": w, "height": w // 2}, steps=k, arrival=a, precision=pr)
            for a, w, k, pr in specs]
    srv = serving.Server(hbm_budget=10_000, chunk=100, clock=FakeClock(), simulation=FakeSimInBatch,
                         footprint=lambda p, prec: p["width"], new_stream=lambda: None, synchronize=lambda: None,
                         batch=FakeBatch, capacity=lambda p, prec: 100 * p["width"], batch_max_divisions=5000)
    srv.run(reqs)
    assert FakeSim.live == 0 and not FakeBatch.open_members
    assert FakeBatch.built >= 1 and srv.batches_built == FakeBatch.built
    # planner capacity 100 W against 5000: the 32-wide requests are batched
    assert [r.batchable for r in reqs] == [False, False, True, True, False, True]
    for r in reqs:
        assert r.result["stats"]["step"] == r.steps
    assert srv.node_updates == sum(r.steps * r.params["width"] for r in reqs)


def test_request_larger_than_the_budget_is_refused():
    r = serving.Request(params={"width": 512, "height": 256}, steps=10)
    srv = serving.Server(hbm_budget=100, simulation=FakeSim, footprint=lambda p, prec: p["width"],
                         new_stream=lambda: None, synchronize=lambda: None)
    with pytest.raises(ValueError):
        srv.run([r])


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
    srv = serving.Server(hbm_budget=budget, chunk=64)
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
def test_served_results_equal_requests_run_alone_with_batching():
    """The same with the small requests stepped through batches (rebuilt as
    requests come and go): bit for bit what each request gives alone."""
    from paper_2303_02210_gb300.lbm import Batch, Simulation, lbm_footprint
    trace = wl.serving_trace(10, rate=500.0, steps=(100, 400), seed=8)
    trace = [(t, dict(p, width=min(p["width"], 512), height=min(p["width"], 512) // 2,
                      front_row=float(min(p["width"], 512) // 8)), n, pr) for t, p, n, pr in trace]
    reqs = [serving.Request(params=p, steps=n, arrival=t, precision=pr, keep_populations=True)
            for t, p, n, pr in trace]
    budget = 4 * max(lbm_footprint(r.params, "fp32") for r in reqs)
    srv = serving.Server(hbm_budget=budget, chunk=32, batch=Batch)
    srv.run(reqs)
    assert srv.batches_built > 0 and any(r.batchable for r in reqs)
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
    srv = serving.Server(hbm_budget=budget, chunk=32, batch=Batch if batching else None)
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
