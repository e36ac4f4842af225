"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

* FP64 debug path: bit-exact — populations, occupancy mask, front heights,
  Eq. 6 sums, proliferation schedule (n_s, carried fraction, candidates,
  events), active and quiescent mass, rear wall — on every growth mode, on
  ragged and degenerate lattices, with and without noise.
* FP32 fast path: within 1e-5 relative of the oracle on the density and
  velocity fields after the 1000-step run of the 128 x 64 workload; every
  occupancy-mask or front-height flip and every step whose n_s differs is
  counted and must be zero.
* Full size (4096 x 2048, edge growth, the benchmark's launch configuration):
  FP64 bit-exact and FP32 within tolerance after a few steps.
"""
import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2303_02210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

EXACT_STATS = ["step", "ns_last", "ns_total", "div_total", "starved_steps", "cand_last", "events_last",
               "mass_fix", "quiescent_fix", "S1", "S2", "y_r", "H_top", "hmin", "status", "carry",
               "hbar", "w"]
RTOL_FP32 = 1e-5


def gpu_sim(params, precision):
    from paper_2303_02210_gb300.lbm import Simulation
    return Simulation(params, precision=precision)


def assert_bit_exact(g, o, events=True):
    sg, so = g.stats(), o.stats()
    for k in EXACT_STATS:
        assert sg[k] == so[k], (k, sg[k], so[k])
    fg, fo = g.pops(), o.pops()
    if not np.array_equal(fg, fo):
        bad = np.argwhere(fg != fo)
        raise AssertionError(f"{len(bad)} populations differ, first {bad[:5].tolist()}")
    assert np.array_equal(g.mask(), o.mask())
    assert np.array_equal(g.heights(), o.heights())
    if events:
        for a, b in zip(g.last_events(), o.last_events()):
            assert np.array_equal(a, b)


FP64_CASES = {
    "bulk_s1": wl.lattice_small(seed=1),
    "bulk_s2_noise0": wl.lattice_small(seed=2, sigma=0.0),
    "bulk_fast_growth": wl.lattice_small(seed=3, growth_rate=3e-3),
    "density": wl.lattice_small(seed=4, growth_mode="density", growth_rate=3e-3),
    "edge": wl.lattice_small(seed=5, growth_mode="edge", edge_depth=4, growth_rate=3e-3,
                             front_kind="sinusoidal", front_amp=3.0, front_kmax=8),
    "band_wall": wl.lattice_small(seed=6, growth_mode="band", band_rows=10, growth_rate=3e-3,
                                  height=96, front_row=40.0, wall_min_gap=12.0),
    "none": wl.lattice_small(seed=7, growth_mode="none"),
    "rescale_strong_noise": wl.lattice_small(seed=8, sigma=0.08, negfix_mode="rescale"),
    "literal_strong_noise": wl.lattice_small(seed=9, sigma=0.08),
    "ragged_37x29": wl.lattice_small(seed=10, width=37, height=29, front_row=9.0, growth_rate=3e-3),
    "width_1": wl.lattice_small(seed=11, width=1, height=24, front_row=8.0, growth_rate=3e-3),
    "width_33": wl.lattice_small(seed=12, width=33, height=40, front_row=12.0, growth_rate=3e-3),
    "periodic_full": wl.base_params(width=48, height=32, front_kind="full", y_periodic=1,
                                    wall_mode="fixed", growth_rate=2e-3, seed=13),
    "paper_params": wl.paper_params(width=96, height=64, front_row=16.0, seed=14),
    "wall_advance_rough": wl.lattice_small(seed=15, width=64, height=96, front_kind="sinusoidal",
                                           front_row=40.0, front_amp=3.0, front_kmax=4,
                                           growth_rate=3e-3, wall_min_gap=2.0),
    "empty": wl.lattice_small(seed=16, front_row=0.0, front_amp=0.0),
    "fills_to_top": wl.lattice_small(seed=17, height=24, growth_rate=5e-3, wall_mode="fixed"),
    "starved_density": wl.base_params(width=32, height=32, front_kind="full", y_periodic=1,
                                      wall_mode="fixed", growth_mode="density", rho_init=2.0,
                                      growth_rate=2e-3, seed=18),
}


@pytest.mark.parametrize("name", sorted(FP64_CASES))
def test_fp64_bit_exact(name):
    p = FP64_CASES[name]
    o = OracleSim(p)
    g = gpu_sim(p, "fp64")
    assert_bit_exact(g, o, events=False)
    done = 0
    for chunk in (1, 9, 90, 300):
        o.step(chunk)
        g.step(chunk)
        done += chunk
        assert_bit_exact(g, o)
    st = g.stats()
    assert st["step"] == done
    if name == "fills_to_top":
        assert st["status"] & 1
    if name == "starved_density":
        assert st["starved_steps"] == done and st["div_total"] == 0
    if name in ("band_wall", "wall_advance_rough"):
        assert st["y_r"] > 0  # the rear wall moved and rows were frozen


def test_fp64_bit_exact_1000_steps_lattice_small():
    """The 128 x 64 workload over its full 1000 steps, three seeds."""
    for seed in (1, 2, 3):
        p = wl.lattice_small(seed=seed)
        o = OracleSim(p)
        g = gpu_sim(p, "fp64")
        o.step(1000)
        g.step(1000)
        assert_bit_exact(g, o)


MAX_CASES = {
    # the widest lattice the packed division key holds (x < 2^15), edge growth
    "max_width_32768": wl.lattice_small(seed=51, width=32768, height=40, front_row=12.0, growth_rate=3e-3,
                                        growth_mode="edge", edge_depth=4, front_kind="sinusoidal",
                                        front_amp=2.0, front_kmax=64, wall_mode="fixed"),
    # the front near the top of the tallest lattice (y < 2^15), advancing wall
    "max_height_32768": wl.lattice_small(seed=52, width=40, height=32768, front_row=32740.0,
                                         growth_rate=3e-3, wall_min_gap=8.0, wall_w_factor=2.0),
}


@pytest.mark.parametrize("name", sorted(MAX_CASES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_maximum_extents(name, precision):
    """The largest width and height the division key packs (32768), a few
    steps: FP64 bit-exact with the oracle; FP32 (the TMA-staged kernel)
    bit-exact with the plain-load FP32 kernel and within tolerance."""
    p = MAX_CASES[name]
    o = OracleSim(p)
    o.step(6)
    if precision == "fp64":
        g = gpu_sim(p, "fp64")
        g.step(6)
        assert_bit_exact(g, o)
        return
    from paper_2303_02210_gb300.lbm import Simulation
    a = Simulation(p, precision="fp32", update_kernel="plain")
    a.step(6)
    for kernel in ("auto", "tma_st"):
        b = Simulation(p, precision="fp32", update_kernel=kernel)
        b.step(6)
        assert b.stats()["update_kernel"] >= 2
        assert np.array_equal(a.pops(), b.pops()), kernel
        e_rho, e_u = field_errors(b, o)
        assert e_rho <= RTOL_FP32 and e_u <= RTOL_FP32
        assert np.array_equal(b.mask(), o.mask())
        assert b.stats()["ns_total"] == o.stats()["ns_total"]
        b.close()


def test_fp64_set_populations_matches_oracle():
    """A caller-supplied state (a shear wave on a periodic lattice) evolves
    identically through lbm_set_populations."""
    from tests.lattice_util import equilibrium
    W, H = 16, 64
    p = wl.base_params(width=W, height=H, front_kind="full", y_periodic=1, growth_mode="none",
                       wall_mode="fixed", tau=0.8)
    y = np.arange(H)[:, None] * np.ones((1, W))
    f0 = equilibrium(np.ones((H, W)), 0.01 * np.sin(2 * np.pi * y / H), np.zeros((H, W)))
    o = OracleSim(p)
    g = gpu_sim(p, "fp64")
    o.set_pops(f0)
    g.set_pops(f0)
    assert_bit_exact(g, o, events=False)
    o.step(200)
    g.step(200)
    assert_bit_exact(g, o, events=False)


def field_errors(g, o):
    rg, uxg, uyg = g.fields()
    ro, uxo, uyo = o.fields()
    e_rho = np.abs(rg - ro).max() / np.abs(ro).max()
    du = np.sqrt((uxg - uxo) ** 2 + (uyg - uyo) ** 2)
    uo = np.sqrt(uxo ** 2 + uyo ** 2)
    occ = o.mask()
    e_u = np.linalg.norm(du[occ]) / max(np.linalg.norm(uo[occ]), 1e-300)
    return e_rho, e_u


def test_fp32_within_tolerance_lattice_small():
    """FP32 storage and arithmetic against the FP64 oracle after the 1000 steps
    of the 128 x 64 workload: density max-abs error relative to max density,
    velocity 2-norm error relative to the 2-norm (occupied nodes), both
    <= 1e-5; no occupancy or height flips; identical division schedule."""
    for seed in (1, 2):
        p = wl.lattice_small(seed=seed)
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
        print(f"seed {seed}: rho {e_rho:.3e} u {e_u:.3e} mask flips {flips} height flips {hflips}"
              f" n_s mismatches {ns_diff}")
        assert flips == 0 and hflips == 0 and ns_diff == 0
        assert e_rho <= RTOL_FP32 and e_u <= RTOL_FP32


def test_full_size_edge_workload_fp64_exact_and_fp32_close():
    """4096 x 2048, edge growth within 8 rows of the front, sinusoidal front
    (k = 1..64, amplitude 1), fixed rear wall: the benchmark's workload in the
    benchmark's launch configuration. Three steps, compared over the whole
    lattice."""
    p = wl.lattice_edge(seed=1)
    o = OracleSim(p)
    o.step(3)
    g64 = gpu_sim(p, "fp64")
    g64.step(3)
    assert_bit_exact(g64, o)
    del g64
    g32 = gpu_sim(p, "fp32")
    g32.step(3)
    e_rho, e_u = field_errors(g32, o)
    flips = int((g32.mask() != o.mask()).sum())
    print(f"full size fp32: rho {e_rho:.3e} u {e_u:.3e} flips {flips}")
    assert flips == 0
    assert e_rho <= RTOL_FP32 and e_u <= RTOL_FP32
    assert g32.stats()["ns_total"] == o.stats()["ns_total"]


def test_set_populations_rejects_negative_values():
    p = wl.lattice_small(seed=1)
    g = gpu_sim(p, "fp32")
    f = g.pops()
    f[3, 5, 5] = -1e-3
    with pytest.raises(Exception):
        g.set_pops(f)


TMA_CASES = {k: v for k, v in FP64_CASES.items() if not v.get("y_periodic")}
TMA_CASES["edge_full_width"] = wl.lattice_small(seed=21, width=384, height=96, front_row=40.0,
                                                growth_mode="edge", growth_rate=3e-3,
                                                front_kind="sinusoidal", front_amp=2.0)
TMA_CASES["ragged_300"] = wl.lattice_small(seed=22, width=300, height=70, front_row=30.0,
                                           growth_rate=3e-3, sigma=0.05)


@pytest.mark.parametrize("kernel", ["tma", "tma1", "tma_st"])
@pytest.mark.parametrize("name", sorted(TMA_CASES))
def test_fp32_tma_kernel_bit_exact_with_plain_kernel(name, kernel):
    """The TMA-staged FP32 update moves data differently (bulk tensor tiles
    with halos, ghost columns, divisions added to staged slots, clipped
    stores) and computes the bulk's node pairs with packed FP32 instructions,
    but runs the same IEEE operations as the plain-load FP32 kernel: every
    population, mask bit, height and counter must agree bit for bit."""
    p = TMA_CASES[name]
    from paper_2303_02210_gb300.lbm import Simulation
    a = Simulation(p, precision="fp32", update_kernel="plain")
    b = Simulation(p, precision="fp32", update_kernel=kernel)
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


@pytest.mark.parametrize("kernel", ["tma", "tma_st"])
def test_fp32_tma_repeatable_on_reused_memory(kernel):
    """The TMA-staged update refills a shared-memory stage as soon as every
    warp holds its values; a refill that overtakes a pending shared-memory
    read would corrupt one warp's nodes now and then, depending on timing and
    on what the reused device memory held before. Eight fresh simulations of
    the full-size workload, three back-to-back steps each, must all agree bit
    for bit with the plain-load kernel."""
    import torch
    from paper_2303_02210_gb300.lbm import Simulation
    p = wl.lattice_edge(seed=1)
    a = Simulation(p, precision="fp32", update_kernel="plain")
    a.step(3)
    ref = a.pops()
    del a
    for trial in range(8):
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        b = Simulation(p, precision="fp32", update_kernel=kernel)
        b.step(3)
        fb = b.pops()
        del b
        assert np.array_equal(fb, ref), f"trial {trial}: {int((fb != ref).sum())} populations differ"


def test_runaway_mass_is_flagged_not_faulting():
    """With the paper's parameters the literal negative-population fix keeps
    adding mass once the front is pinned at the top wall, until the exact
    int64 fixed-point mass overflows. The planner must then skip growth and
    raise the capacity bit (a negative request once turned into a garbage
    division count and out-of-range reads)."""
    from paper_2303_02210_gb300.lbm import Simulation
    p = wl.paper_params(width=64, height=128, front_row=16.0, seed=1, sim_id=1)
    g = Simulation(p, precision="fp32")
    g.step(6000)
    st = g.stats()
    assert st["status"] & 1 and st["status"] & 4  # front at the top, growth skipped
    assert st["events_last"] >= 0
    f = g.pops()  # the context is still usable
    assert f.shape == (9, 128, 64)
    h, _, _ = g.front_heights()
    assert h.max() <= 128


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_async_heights_readback_equals_the_synchronous_one(pinned):
    """lbm_front_heights_async copies every step's heights and exact Eq. 6
    sums into host buffers without waiting (pinned buffers the device can
    address: stores by a small kernel; pageable ones: cudaMemcpyAsync);
    after one wait they hold what lbm_front_heights returns step by step."""
    import torch
    from paper_2303_02210_gb300.lbm import Simulation, lbm_eq6, lbm_eq6_n
    p = wl.lattice_small(seed=3, growth_rate=3e-3, front_kind="sinusoidal", front_amp=3.0, front_kmax=8,
                         width=300)
    a, b = gpu_sim(p, "fp32"), gpu_sim(p, "fp32")
    n = 20
    hb = torch.full((n, p["width"]), -7, dtype=torch.int32, pin_memory=pinned)
    sb = torch.full((n, 2), -7, dtype=torch.int64, pin_memory=pinned)
    sb_only = torch.full((n, 2), -7, dtype=torch.int64, pin_memory=pinned)
    want = []
    for k in range(n):
        a.step(1)
        a.lbm_front_heights_async(hb[k], sb[k])
        a.lbm_front_heights_async(None, sb_only[k])
        b.step(1)
        want.append(b.front_heights())
    a.sync()
    hbar_n, w_n = lbm_eq6_n(sb, p["width"])
    for k, (h, hbar, w) in enumerate(want):
        assert np.array_equal(hb[k].numpy(), h)
        assert lbm_eq6(int(sb[k, 0]), int(sb[k, 1]), p["width"]) == (hbar, w)
        assert (hbar_n[k], w_n[k]) == (hbar, w)
    assert np.array_equal(sb_only.numpy(), sb.numpy())
