"""Failure detection on the GPU without a GPU fault: every wait in the kernels
is bounded, and a test makes each kind of wait run out.

``lbm_debug_waits`` shortens the wait budget of a simulation and withholds
what a wait is for: the TMA-staged update's bulk copies (each thread's first
wait for a staged tile then runs out), or one arrival at the planner's grid
barriers (each block's first barrier runs out). The step must come back in
well under a second with ``LBM_STATUS_TIMEOUT`` set and the CUDA context
intact; after the hook is reset, the status cleared and a state restored, the
same handle must step on normally (no timeout, a consistent state), and, on
the FP32 path, exactly as a fresh simulation does from the same state.
"""
import time

import numpy as np
import pytest

from paper_2303_02210_gb300 import workloads as wl
from paper_2303_02210_gb300.lbm import STATUS_TIMEOUT

pytestmark = pytest.mark.gpu

BUDGET = 200_000  # clock cycles, about 0.1 ms at 2 GHz


def _params(lattice="d2q9"):
    # a fixed rear wall, so that an abandoned step cannot move it
    return wl.lattice_small(seed=21, growth_rate=3e-3, front_row=30.0, wall_mode="fixed", lattice=lattice)


def _consistent(sim, params):
    rho, _, _ = sim.fields()
    f = sim.pops()
    assert np.isfinite(f).all() and (f >= 0).all()
    # the mask is decided on the pre-collision density, which the stored
    # populations keep up to rounding (and the negative fix's additions)
    rc = params["rho_c"]
    differ = sim.mask() != (rho >= rc)
    assert not differ[np.abs(rho - rc) > 1e-5].any()
    h = sim.heights()
    top = np.where(sim.mask(), np.arange(sim.H)[:, None], -1).max(axis=0) + 1
    assert np.array_equal(h, top)


def _abandon_and_recover(params, withhold, update_kernel="tma"):
    import torch
    from paper_2303_02210_gb300.lbm import Simulation
    sim = Simulation(params, precision="fp32", update_kernel=update_kernel)
    if withhold & 1:
        assert sim.stats()["update_kernel"] >= 2  # a TMA-staged update
    sim.step(4)
    f0 = sim.pops()
    m0 = sim.stats()["mass"]
    sim.lbm_debug_waits(BUDGET, withhold)
    t0 = time.perf_counter()
    sim.step(1)
    sim.sync()
    dt = time.perf_counter() - t0
    st = sim.stats()
    assert st["status"] & STATUS_TIMEOUT, st["status"]
    assert dt < 1.0, dt  # the waits gave up after the short budget
    # the context is intact: a fresh allocation and copy work
    assert int(torch.arange(10, device="cuda").sum().item()) == 45
    # recovery on the same handle
    sim.lbm_debug_waits(0, 0)
    sim.lbm_clear_status()
    sim.set_pops(f0)
    sim.step(6)
    st = sim.stats()
    assert st["status"] & STATUS_TIMEOUT == 0
    _consistent(sim, params)
    assert abs(st["mass"] - m0) < 0.05 * m0
    return sim, f0


@pytest.mark.parametrize("lattice,kernel", [("d2q9", "tma"), ("d2q9", "tma_st"), ("d2q7", "tma")])
def test_staged_copy_wait_runs_out_and_the_handle_recovers(lattice, kernel):
    sim, _ = _abandon_and_recover(_params(lattice), withhold=1, update_kernel=kernel)
    sim.close()


def test_planner_barrier_wait_runs_out_and_the_handle_recovers():
    sim, _ = _abandon_and_recover(_params(), withhold=2)
    sim.close()


def test_after_recovery_the_handle_steps_as_a_fresh_one():
    """Without growth (so that the carried fraction of n_s, which an abandoned
    planner step may leave different, plays no part): a handle whose planner
    step was abandoned, once recovered and set to the state a fresh handle
    reached at the same step, then steps bit for bit as that one."""
    from paper_2303_02210_gb300.lbm import Simulation
    p0 = dict(_params(), growth_rate=0.0, growth_mode="none")
    a = Simulation(p0, precision="fp32", update_kernel="tma")
    b = Simulation(p0, precision="fp32", update_kernel="tma")
    a.lbm_debug_waits(BUDGET, 2)
    a.step(1)
    assert a.stats()["status"] & STATUS_TIMEOUT
    a.lbm_debug_waits(0, 0)
    a.lbm_clear_status()
    b.step(1)
    assert a.stats()["step"] == b.stats()["step"] == 1
    a.set_pops(b.pops())
    a.step(10)
    b.step(10)
    assert a.stats()["status"] == 0 and b.stats()["status"] == 0
    assert np.array_equal(a.pops(), b.pops())
    assert np.array_equal(a.mask(), b.mask())
    a.close()
    b.close()


def test_debug_waits_rejects_bad_arguments():
    from paper_2303_02210_gb300.lbm import LbmError, Simulation
    sim = Simulation(_params(), precision="fp32")
    with pytest.raises(LbmError):
        sim.lbm_debug_waits(-1, 0)
    with pytest.raises(LbmError):
        sim.lbm_debug_waits(0, 4)
    sim.close()
