"""Batched stepping (``lbm_batch_*``): members of a batch advanced by graph
replays must end exactly where the same simulations end when stepped alone
with ``lbm_step`` (same kernels, same counter-based random streams), whatever
their size, growth mode, precision or update kernel, and also when batch
steps and single steps are interleaved."""
import numpy as np
import pytest

from paper_2303_02210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

STATS = ["step", "ns_last", "ns_total", "div_total", "starved_steps", "cand_last", "events_last", "mass_fix",
         "quiescent_fix", "S1", "S2", "y_r", "H_top", "hmin", "status", "carry", "node_updates", "y_hi"]

MEMBERS = [
    (wl.lattice_small(seed=31, growth_rate=3e-3), "fp32", "auto"),
    (wl.lattice_small(seed=32, width=300, height=70, front_row=30.0, growth_rate=3e-3, growth_mode="edge",
                      edge_depth=4, front_kind="sinusoidal", front_amp=2.0), "fp32", "auto"),
    (wl.lattice_small(seed=33, width=37, height=29, front_row=9.0, growth_rate=3e-3), "fp32", "plain"),
    (wl.lattice_small(seed=34, growth_mode="density", growth_rate=3e-3), "fp64", "auto"),
    (wl.lattice_small(seed=35, width=64, height=96, front_kind="sinusoidal", front_row=40.0, front_amp=3.0,
                      front_kmax=4, growth_rate=3e-3, wall_min_gap=2.0), "fp32", "auto"),
]


def make(m):
    from paper_2303_02210_gb300.lbm import Simulation
    p, prec, kern = m
    return Simulation(p, precision=prec, update_kernel=kern)


def same(a, b):
    sa, sb = a.stats(), b.stats()
    for k in STATS:
        assert sa[k] == sb[k], (k, sa[k], sb[k])
    assert np.array_equal(a.pops(), b.pops())
    assert np.array_equal(a.mask(), b.mask())
    assert np.array_equal(a.heights(), b.heights())
    for x, y in zip(a.last_events(), b.last_events()):
        assert np.array_equal(x, y)


def test_batch_matches_single_stepping():
    from paper_2303_02210_gb300.lbm import Batch
    members = [make(m) for m in MEMBERS]
    batch = Batch(members)
    batch.step(13)  # three replays of the four-step graph and one of the one-step graph
    for m, g in zip(MEMBERS, members):
        solo = make(m)
        solo.step(13)
        same(g, solo)
    batch.close()


def test_batch_and_single_steps_interleave():
    from paper_2303_02210_gb300.lbm import Batch
    members = [make(m) for m in MEMBERS[:3]]
    batch = Batch(members)
    batch.step(5)
    members[1].step(2)
    batch.step(3)
    solos = [make(m) for m in MEMBERS[:3]]
    for s, n in zip(solos, (8, 10, 8)):
        s.step(n)
    for g, s in zip(members, solos):
        same(g, s)
    batch.close()


FUSED_FP32 = [
    (wl.lattice_small(seed=41, growth_rate=3e-3), "fp32", "auto"),
    (wl.lattice_small(seed=42, width=300, height=70, front_row=30.0, growth_rate=3e-3, growth_mode="edge",
                      edge_depth=4, front_kind="sinusoidal", front_amp=2.0), "fp32", "auto"),
    (wl.lattice_small(seed=43, width=37, height=29, front_row=9.0, growth_rate=3e-3), "fp32", "plain"),
    (wl.lattice_small(seed=44, growth_mode="density", growth_rate=3e-3), "fp32", "auto"),
    (wl.lattice_small(seed=45, width=64, height=96, front_kind="sinusoidal", front_row=40.0, front_amp=3.0,
                      front_kmax=4, growth_rate=3e-3, wall_min_gap=2.0), "fp32", "auto"),
    (wl.base_params(width=48, height=32, front_kind="full", y_periodic=1, wall_mode="fixed",
                    growth_rate=2e-3, seed=46, sim_id=46), "fp32", "auto"),
    (wl.lattice_small(seed=47, growth_mode="none", width=1, height=24, front_row=8.0), "fp32", "auto"),
    (wl.lattice_small(seed=48, growth_mode="band", band_rows=10, growth_rate=3e-3, height=96,
                      front_row=40.0, wall_min_gap=12.0, sigma=0.05, negfix_mode="rescale"), "fp32", "auto"),
]


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_fused_batch_matches_single_stepping(precision):
    """Members sharing a storage type step with three batched launches per
    step (one planner block per member, a shared table of update blocks):
    every member ends bit for bit where lbm_step takes it, whichever update
    kernel it uses alone."""
    from paper_2303_02210_gb300.lbm import Batch
    ms = [(p, precision, k) for p, _, k in FUSED_FP32]
    members = [make(m) for m in ms]
    batch = Batch(members)
    assert batch.fused
    batch.step(13)
    for m, g in zip(ms, members):
        solo = make(m)
        solo.step(13)
        same(g, solo)
    batch.close()


def test_fused_batch_interleaves_with_single_steps():
    from paper_2303_02210_gb300.lbm import Batch
    members = [make(m) for m in FUSED_FP32[:4]]
    batch = Batch(members)
    assert batch.fused
    batch.step(6)
    members[0].step(3)
    members[3].step(1)
    batch.step(9)
    solos = [make(m) for m in FUSED_FP32[:4]]
    for s, n in zip(solos, (18, 15, 15, 16)):
        s.step(n)
    for g, s in zip(members, solos):
        same(g, s)
    batch.close()


def test_mixed_precision_batch_uses_branches():
    from paper_2303_02210_gb300.lbm import Batch
    members = [make(m) for m in MEMBERS[2:4]]  # fp32 and fp64
    batch = Batch(members)
    assert not batch.fused
    batch.close()
