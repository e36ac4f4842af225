"""The triangular D2Q7 lattice (the paper's, Sec. II) on the GPU against the
FP64 oracle, through the C ABI: FP64 bit-exact (populations, mask, heights,
every counter, the division schedule), FP32 within 1e-5 with no flips, at
128 x 64 over 1000 steps and at the full 4096 x 2048 edge workload; the
TMA-staged FP32 update bit-exact with the plain-load one; and the batched
form bit-exact with single stepping."""
import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2303_02210_gb300 import workloads as wl
from tests.test_gpu_parity import EXACT_STATS, RTOL_FP32, assert_bit_exact, field_errors

pytestmark = pytest.mark.gpu


def q7(p):
    return dict(p, lattice="d2q7")


def gpu_sim(params, precision, kernel="auto"):
    from paper_2303_02210_gb300.lbm import Simulation
    return Simulation(params, precision=precision, update_kernel=kernel)


CASES = {
    "bulk_s1": q7(wl.lattice_small(seed=61)),
    "bulk_noise0": q7(wl.lattice_small(seed=62, sigma=0.0)),
    "bulk_fast_growth": q7(wl.lattice_small(seed=63, growth_rate=3e-3)),
    "density": q7(wl.lattice_small(seed=64, growth_mode="density", growth_rate=3e-3)),
    "edge": q7(wl.lattice_small(seed=65, growth_mode="edge", edge_depth=4, growth_rate=3e-3,
                                front_kind="sinusoidal", front_amp=3.0, front_kmax=8)),
    "band_wall": q7(wl.lattice_small(seed=66, growth_mode="band", band_rows=10, growth_rate=3e-3,
                                     height=96, front_row=40.0, wall_min_gap=12.0)),
    "rescale_strong_noise": q7(wl.lattice_small(seed=67, sigma=0.08, negfix_mode="rescale")),
    "literal_strong_noise": q7(wl.lattice_small(seed=68, sigma=0.08)),
    "ragged_37x29": q7(wl.lattice_small(seed=69, width=37, height=29, front_row=9.0, growth_rate=3e-3)),
    "width_1": q7(wl.lattice_small(seed=70, width=1, height=24, front_row=8.0, growth_rate=3e-3)),
    "periodic_full": q7(wl.base_params(width=48, height=32, front_kind="full", y_periodic=1,
                                       wall_mode="fixed", growth_rate=2e-3, seed=71)),
    "paper_params": q7(wl.paper_params(width=96, height=64, front_row=16.0, seed=72)),
    "fills_to_top": q7(wl.lattice_small(seed=73, height=24, growth_rate=5e-3, wall_mode="fixed")),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_bit_exact(name):
    p = CASES[name]
    o = OracleSim(p)
    g = gpu_sim(p, "fp64")
    assert o.Q == 7 and g.Q == 7
    for chunk in (1, 9, 90, 200):
        o.step(chunk)
        g.step(chunk)
        assert_bit_exact(g, o)


def test_fp32_within_tolerance_lattice_small():
    for seed in (61, 62):
        p = q7(wl.lattice_small(seed=seed))
        o = OracleSim(p)
        g = gpu_sim(p, "fp32")
        ns_diff = 0
        for _ in range(10):
            o.step(100)
            g.step(100)
            ns_diff += g.stats()["ns_total"] != o.stats()["ns_total"]
        flips = int((g.mask() != o.mask()).sum())
        hflips = int((g.heights() != o.heights()).sum())
        e_rho, e_u = field_errors(g, o)
        print(f"D2Q7 seed {seed}: rho {e_rho:.3e} u {e_u:.3e} flips {flips} {hflips} n_s {ns_diff}")
        assert flips == 0 and hflips == 0 and ns_diff == 0
        assert e_rho <= RTOL_FP32 and e_u <= RTOL_FP32


def test_full_size_edge_workload():
    p = q7(wl.lattice_edge(seed=1))
    o = OracleSim(p)
    o.step(3)
    g64 = gpu_sim(p, "fp64")
    g64.step(3)
    assert_bit_exact(g64, o)
    del g64
    g32 = gpu_sim(p, "fp32")
    g32.step(3)
    e_rho, e_u = field_errors(g32, o)
    assert int((g32.mask() != o.mask()).sum()) == 0
    assert e_rho <= RTOL_FP32 and e_u <= RTOL_FP32
    assert g32.stats()["ns_total"] == o.stats()["ns_total"]


def test_update_kinds_for_d2q7():
    """One TMA-staged D2Q7 form (two-row tiles, FP32, walls in y): "tma" and
    the automatic choice take it, "tma1" and "tma_sel" are refused, as are
    16-bit storage and "tma" on a lattice periodic in y."""
    from paper_2303_02210_gb300.lbm import lbm_validate
    p = q7(wl.lattice_small())
    for kind in ("tma1", "tma_sel"):
        with pytest.raises(Exception):
            gpu_sim(p, "fp32", kind)
    with pytest.raises(Exception):
        gpu_sim(p, "fp16")
    with pytest.raises(Exception):
        gpu_sim(CASES["periodic_full"], "fp32", "tma")
    assert lbm_validate(p, "fp32") == 0
    assert gpu_sim(p, "fp32").stats()["update_kernel"] == 2
    assert gpu_sim(p, "fp32", "tma").stats()["update_kernel"] == 2
    assert gpu_sim(p, "fp32", "plain").stats()["update_kernel"] == 1
    assert gpu_sim(CASES["periodic_full"], "fp32").stats()["update_kernel"] == 1
    assert gpu_sim(p, "fp64").stats()["update_kernel"] == 1


TMA_CASES = {k: v for k, v in CASES.items() if not v.get("y_periodic")}
TMA_CASES["ragged_300"] = q7(wl.lattice_small(seed=74, width=300, height=70, front_row=30.0,
                                              growth_rate=3e-3, sigma=0.05))
TMA_CASES["wide_edge"] = q7(wl.lattice_small(seed=75, width=384, height=96, front_row=40.0,
                                             growth_mode="edge", growth_rate=3e-3,
                                             front_kind="sinusoidal", front_amp=2.0))
TMA_CASES["odd_width_129"] = q7(wl.lattice_small(seed=76, width=129, height=41, front_row=15.0,
                                                 growth_rate=3e-3))


@pytest.mark.parametrize("name", sorted(TMA_CASES))
def test_tma_bit_exact_with_plain_kernel(name):
    """The TMA-staged D2Q7 update pulls from staged boxes (parity-dependent
    column offsets, ghost columns, zero-filled rows past the lattice) but runs
    update7_body's per-node arithmetic: every population, mask bit, height and
    counter must agree bit for bit with the plain-load kernel."""
    p = TMA_CASES[name]
    a = gpu_sim(p, "fp32", "plain")
    b = gpu_sim(p, "fp32", "tma")
    assert a.stats()["update_kernel"] == 1 and b.stats()["update_kernel"] >= 2
    for chunk in (1, 9, 90, 200):
        a.step(chunk)
        b.step(chunk)
        sa, sb = a.stats(), b.stats()
        for k in EXACT_STATS + ["node_updates", "y_hi"]:
            assert sa[k] == sb[k], (k, sa[k], sb[k])
        assert np.array_equal(a.pops(), b.pops())
        assert np.array_equal(a.mask(), b.mask())
        assert np.array_equal(a.heights(), b.heights())


def test_tma_full_size_repeatable_on_reused_memory():
    """Four fresh full-size TMA-staged D2Q7 runs, three steps each on reused
    device memory, agree bit for bit with the plain-load kernel (a stage
    refill overtaking a pending shared-memory read would show here)."""
    import torch
    p = q7(wl.lattice_edge(seed=1))
    a = gpu_sim(p, "fp32", "plain")
    a.step(3)
    ref = a.pops()
    del a
    for trial in range(4):
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        b = gpu_sim(p, "fp32", "tma")
        assert b.stats()["update_kernel"] >= 2
        b.step(3)
        fb = b.pops()
        del b
        assert np.array_equal(fb, ref), f"trial {trial}: {int((fb != ref).sum())} populations differ"


def test_batched_d2q7_matches_single_stepping():
    from paper_2303_02210_gb300.lbm import Batch
    ps = [CASES[k] for k in ("bulk_fast_growth", "edge", "ragged_37x29", "periodic_full", "band_wall")]
    members = [gpu_sim(p, "fp32") for p in ps]
    batch = Batch(members)
    assert batch.fused
    batch.step(13)
    for p, g in zip(ps, members):
        solo = gpu_sim(p, "fp32")
        solo.step(13)
        assert np.array_equal(g.pops(), solo.pops())
        assert np.array_equal(g.heights(), solo.heights())
        assert g.stats()["ns_total"] == solo.stats()["ns_total"]
    batch.close()
