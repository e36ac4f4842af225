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


# ---- against the FP64 oracle directly (not only against lbm_step) ----
ORACLE_MEMBERS = [
    wl.lattice_small(seed=51, width=64, height=48, front_row=12.0, growth_rate=3e-3),
    wl.lattice_small(seed=52, growth_mode="edge", edge_depth=4, front_kind="sinusoidal", front_amp=2.0,
                     front_kmax=6, growth_rate=3e-3),
    wl.lattice_small(seed=53, width=256, height=64, growth_rate=2e-3, wall_min_gap=8.0),
    wl.lattice_small(seed=54, width=96, height=40, growth_mode="density", growth_rate=3e-3),
    wl.lattice_small(seed=55, width=37, height=33, front_row=10.0, growth_mode="band", band_rows=5,
                     growth_rate=3e-3, wall_min_gap=4.0),
]


def _oracle_after(p, steps):
    from oracle.oracle import OracleSim
    o = OracleSim(p)
    o.step(steps)
    return o


def _bit_exact_with_oracle(g, o):
    assert np.array_equal(g.pops(), o.pops())
    assert np.array_equal(g.mask(), o.mask())
    assert np.array_equal(g.heights(), o.heights())
    sg, so = g.stats(), o.stats()
    for k in ("step", "ns_last", "ns_total", "div_total", "starved_steps", "cand_last", "events_last",
              "mass_fix", "quiescent_fix", "S1", "S2", "y_r", "H_top", "hmin", "carry", "w"):
        assert sg[k] == so[k], (k, sg[k], so[k])
    # (the negative fix's added mass is summed by atomic FP64 adds in any
    # order on the GPU: equal up to the last bits)
    assert abs(sg["clip_mass"] - so["clip_mass"]) <= 1e-12 * max(abs(so["clip_mass"]), 1e-300)
    for x, y in zip(g.last_events(), o.last_events()):
        assert np.array_equal(x, y)


def _fp32_close_to_oracle(g, o, tol=1e-5):
    rg, uxg, uyg = g.fields()
    ro, uxo, uyo = o.fields()
    assert np.abs(rg - ro).max() / np.abs(ro).max() <= tol
    occ = o.mask()
    du = np.hypot(uxg - uxo, uyg - uyo)[occ]
    uo = np.hypot(uxo, uyo)[occ]
    assert np.sqrt((du ** 2).sum()) / np.sqrt((uo ** 2).sum()) <= tol
    assert np.array_equal(g.mask(), o.mask())
    assert np.array_equal(g.heights(), o.heights())
    sg, so = g.stats(), o.stats()
    assert sg["ns_total"] == so["ns_total"] and sg["div_total"] == so["div_total"]


def test_fused_fp64_batch_bit_exact_with_the_oracle():
    """The batched launches in FP64 (their own kernels over the member
    tables) against the FP64 oracle, member by member, bit for bit: mixed
    widths 37..256, every growth mode, a moving rear wall."""
    from paper_2303_02210_gb300.lbm import Batch, Simulation
    members = [Simulation(p, precision="fp64") for p in ORACLE_MEMBERS]
    batch = Batch(members)
    assert batch.fused
    batch.step(200)
    for p, g in zip(ORACLE_MEMBERS, members):
        _bit_exact_with_oracle(g, _oracle_after(p, 200))
    assert any(m.stats()["y_r"] > 0 for m in members)  # the wall moved somewhere
    batch.close()


def test_fused_fp32_batch_within_tolerance_of_the_oracle():
    """The batched FP32 launches over 1000 steps at the workloads' growth rate
    g = 1e-4: every member within 1e-5 of the oracle in density and velocity,
    no mask or height flips, the same number of divisions. (At g = 3e-3 the
    carried fraction of n_s integrates the FP32 mass rounding and, after some
    hundreds of steps, floors to a different n_s: from then on the two runs
    are different realisations.)"""
    from paper_2303_02210_gb300.lbm import Batch, Simulation
    ps = [dict(p, growth_rate=1e-4) for p in ORACLE_MEMBERS]
    members = [Simulation(p, precision="fp32") for p in ps]
    batch = Batch(members)
    assert batch.fused
    batch.step(1000)
    for p, g in zip(ps, members):
        _fp32_close_to_oracle(g, _oracle_after(p, 1000))
    batch.close()


def test_branch_batch_fp64_members_bit_exact_with_the_oracle():
    """A batch of mixed storage types (one graph branch per member): its FP64
    members bit for bit with the oracle, its FP32 members within 1e-5."""
    from paper_2303_02210_gb300.lbm import Batch, Simulation
    precs = ["fp64", "fp32", "fp64", "fp32", "fp64"]
    members = [Simulation(p, precision=pr) for p, pr in zip(ORACLE_MEMBERS, precs)]
    batch = Batch(members)
    assert not batch.fused
    batch.step(150)
    for p, pr, g in zip(ORACLE_MEMBERS, precs, members):
        o = _oracle_after(p, 150)
        if pr == "fp64":
            _bit_exact_with_oracle(g, o)
        else:
            _fp32_close_to_oracle(g, o)
    batch.close()


# ---- the TMA-staged batched update (every member D2Q9, walls in y) ----
STAGED = [
    (wl.lattice_small(seed=61, growth_rate=3e-3), "auto"),
    (wl.lattice_small(seed=62, width=300, height=70, front_row=30.0, growth_rate=3e-3, growth_mode="edge",
                      edge_depth=4, front_kind="sinusoidal", front_amp=2.0), "auto"),
    (wl.lattice_small(seed=63, width=37, height=29, front_row=9.0, growth_rate=3e-3), "plain"),
    (wl.lattice_small(seed=64, growth_mode="density", growth_rate=3e-3, sigma=0.0), "auto"),
    (wl.lattice_small(seed=65, width=64, height=96, front_kind="sinusoidal", front_row=40.0, front_amp=3.0,
                      front_kmax=4, growth_rate=3e-3, wall_min_gap=2.0), "tma1"),
    (wl.lattice_small(seed=66, growth_mode="none", width=1, height=24, front_row=8.0), "auto"),
    (wl.lattice_small(seed=67, growth_mode="band", band_rows=10, growth_rate=3e-3, height=96,
                      front_row=40.0, wall_min_gap=12.0, sigma=0.05, negfix_mode="rescale"), "auto"),
    (wl.lattice_small(seed=68, width=512, height=40, front_row=20.0, growth_rate=2e-3, growth_mode="edge"), "tma_st"),
]


@pytest.mark.parametrize("precision,width4", [("fp32", False), ("fp32", True), ("fp16", False), ("bf16", False)])
def test_staged_batch_matches_single_stepping(precision, width4):
    """Members that all take the TMA-staged update step with one batched
    staged launch (tiles of all members dealt together, divisions injected
    beforehand, members with and without noise mixed): bit for bit what
    lbm_step gives each alone, whatever kernel that uses, also interleaved
    with single steps."""
    from paper_2303_02210_gb300.lbm import Batch
    staged = STAGED if not width4 else [  # bulk stores: members at least the tuned width (4096) wide
        (dict(p, width=4096 + 128 * i, sim_id=i), k) for i, (p, k) in enumerate(STAGED) if p["width"] % 4 == 0]
    ms = [(p, precision, k if precision == "fp32" or k != "tma_st" else "auto") for p, k in staged]
    members = [make(m) for m in ms]
    batch = Batch(members)
    assert batch.fused and batch.staged
    assert batch.bulk_stores == width4
    batch.step(13)
    members[1].step(2)
    batch.step(6)
    for i, (m, g) in enumerate(zip(ms, members)):
        solo = make(m)
        solo.step(21 if i == 1 else 19)
        same(g, solo)
    batch.close()


def test_staged_batch_within_tolerance_of_the_oracle_1000_steps():
    """The staged batched update against the FP64 oracle over 1000 steps at
    the workloads' growth rate: every member within 1e-5, no flips, the same
    divisions."""
    from paper_2303_02210_gb300.lbm import Batch, Simulation
    ps = [dict(p, growth_rate=1e-4) for p in ORACLE_MEMBERS]
    members = [Simulation(p, precision="fp32") for p in ps]
    batch = Batch(members)
    assert batch.staged
    batch.step(1000)
    for p, g in zip(ps, members):
        _fp32_close_to_oracle(g, _oracle_after(p, 1000))
    batch.close()


@pytest.mark.parametrize("precision,lattice", [("fp32", "d2q9"), ("fp16", "d2q9"), ("fp64", "d2q9"),
                                               ("fp32", "d2q7")])
def test_slot_batch_members_join_and_leave(precision, lattice):
    """A batch made with free slots (lbm_batch_create_empty): members join
    after stepping alone, leave, join again, share the batch with members
    that came later; the graphs are captured once (noisy and quiet members
    mixed, the room of the tables enough), a full batch refuses a member,
    and every member ends bit for bit where it ends stepped alone for the
    same number of steps."""
    from paper_2303_02210_gb300.lbm import Batch, LbmError
    if lattice == "d2q7":
        ps = [dict(wl.lattice_small(seed=80 + i, width=64 + 32 * i, growth_rate=3e-3), lattice="d2q7",
                   sigma=0.02 * (i % 2)) for i in range(4)]
    else:
        ps = [dict(p, sim_id=i) for i, (p, _) in enumerate(STAGED[:4])]
    ms = [(p, precision, "auto") for p in ps]
    sims = [make(m) for m in ms]
    steps = [0] * 4
    batch = Batch.empty(3, precision, lattice)
    assert batch.members == 0 and batch.captures == 1
    assert batch.fused and batch.staged == (lattice == "d2q9" and precision != "fp64")
    batch.step(3)  # nothing to step
    sims[0].step(2)
    steps[0] += 2
    assert batch.attach(sims[0]) == 0
    assert batch.attach(sims[1]) == 1
    batch.step(5)
    steps[0] += 5
    steps[1] += 5
    assert batch.attach(sims[2]) == 2
    with pytest.raises(LbmError):
        batch.attach(sims[3])  # full
    batch.step(6)
    for i in range(3):
        steps[i] += 6
    batch.detach(sims[1])
    sims[1].step(3)
    steps[1] += 3
    assert batch.attach(sims[3]) == 1  # the freed slot
    batch.step(9)
    for i in (0, 2, 3):
        steps[i] += 9
    batch.detach(sims[0])
    assert batch.attach(sims[1]) == 0
    batch.step(4)
    for i in (1, 2, 3):
        steps[i] += 4
    assert batch.members == 3 and batch.captures == 1
    for i, (m, g) in enumerate(zip(ms, sims)):
        solo = make(m)
        solo.step(steps[i])
        same(g, solo)
        solo.close()
    batch.close()


def test_slot_batch_recaptures_only_for_a_member_it_cannot_step():
    """A batch with bulk stores (made from two wide members: two slots) gives
    them up for a narrow member that takes a freed slot (one capture more),
    and the results stay exact."""
    from paper_2303_02210_gb300.lbm import Batch
    wide = [(dict(p, width=4096 + 128 * i, sim_id=i), "fp32", "auto")
            for i, (p, k) in enumerate(STAGED) if p["width"] % 4 == 0][:2]
    narrow = (dict(STAGED[0][0], sim_id=9), "fp32", "auto")
    sims = [make(m) for m in wide]
    batch = Batch(sims)
    assert batch.bulk_stores and batch.captures == 1
    batch.step(4)
    batch.detach(sims[1])
    s_n = make(narrow)
    assert batch.attach(s_n) == 1
    assert not batch.bulk_stores and batch.staged and batch.captures == 2
    batch.step(7)
    for m, g, k in zip(wide + [narrow], [sims[0], sims[1], s_n], [11, 4, 7]):
        solo = make(m)
        solo.step(k)
        same(g, solo)
        solo.close()
    batch.close()
