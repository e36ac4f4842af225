"""The allocation-free front-height entry point, ``lbm_front_heights_noalloc``.

It serves callers that cannot allocate device memory (an application whose
device memory is held by another allocator, a loop that must not stall on the
allocator): its scratch is a fixed array inside the library (one partial sum
per 256-column block and a completion counter). Here it must reproduce

* what ``lbm_front_heights`` reports for a simulation after ``lbm_step``
  (heights exactly, mean height and width to the last bit), on two calls in a
  row that reuse the same scratch, on a ragged and a rough lattice;
* the heights and Eq. 6 values worked out on the host from synthetic rough
  masks (islands below the front, overhangs, empty columns) at widths that
  take one, two, 17, 33 and 128 blocks, so that the per-block partials, the
  completion counter and the last block's sum all run, twice in a row with
  different masks;
* the FP64 oracle's heights and Eq. 6 values for the same initial lattice at
  8200 and 32768 columns;

and it must refuse widths beyond its limit. This file is collected last on
purpose.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2303_02210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def pack_mask(mask):
    """Occupancy (H x W bools) -> H x ceil(W/32) uint32 words, bit x & 31 of word x >> 5."""
    H, W = mask.shape
    MW = (W + 31) // 32
    padded = np.zeros((H, MW * 32), dtype=np.uint64)
    padded[:, :W] = mask
    bits = padded.reshape(H, MW, 32) << np.arange(32, dtype=np.uint64)
    return bits.sum(axis=2).astype(np.uint32)


def host_heights(mask):
    """h(x) = 1 + highest set row of column x, 0 for an empty column (brute force)."""
    H, W = mask.shape
    rows = np.arange(H)[:, None]
    top = np.where(mask, rows, -1).max(axis=0)
    return (top + 1).astype(np.int32)


def host_eq6(h):
    """Eq. 6 from the exact integer sums, with the same IEEE operations as the
    kernel: hbar = S1 / W, w = sqrt(W S2 - S1^2) / W."""
    W = len(h)
    s1 = int(h.astype(np.int64).sum())
    s2 = int((h.astype(np.int64) ** 2).sum())
    return float(s1) / float(W), math.sqrt(float(W * s2 - s1 * s1)) / float(W)


def rough_mask(W, H, seed):
    """A rough front (a clipped random walk) with tissue islands below it, a
    few overhangs above it and some empty columns."""
    rng = np.random.default_rng(seed)
    walk = np.cumsum(rng.integers(-3, 4, size=W))
    h0 = np.clip(H // 2 + walk - int(walk.mean()), 0, H)
    mask = np.arange(H)[:, None] < h0[None, :]
    holes = rng.random((H, W)) < 0.05
    mask &= ~holes
    over = (rng.random((H, W)) < 0.002) & (np.arange(H)[:, None] >= h0[None, :])
    mask |= over
    mask[:, rng.integers(0, W, size=max(1, W // 97))] = False
    mask[H - 1, rng.integers(0, W)] = True  # one column reaches the top row
    return mask


def run_noalloc(mask, heights, stats):
    import torch
    from paper_2303_02210_gb300.lbm import lbm_front_heights_noalloc
    H, W = mask.shape
    words = torch.from_numpy(pack_mask(mask).view(np.int32)).to("cuda")
    heights.fill_(-1)
    stats.fill_(-1.0)
    lbm_front_heights_noalloc(words, W, H, heights, stats)
    torch.cuda.synchronize()
    hbar, w = stats.cpu().numpy()
    return heights.cpu().numpy(), float(hbar), float(w)


@pytest.mark.parametrize("params", [
    wl.lattice_small(seed=31, growth_rate=3e-3),
    wl.lattice_small(seed=32, width=37, height=50, front_kind="sinusoidal", front_row=20.0,
                     front_amp=8.0, front_kmax=5, growth_mode="edge", growth_rate=3e-3),
])
def test_noalloc_matches_front_heights_twice(params):
    import torch
    from paper_2303_02210_gb300.lbm import Simulation, lbm_front_heights_noalloc
    sim = Simulation(params, precision="fp32")
    W, H = sim.W, sim.H
    heights = torch.empty(W, dtype=torch.int32, device="cuda")
    stats = torch.empty(2, dtype=torch.float64, device="cuda")
    for _ in range(2):  # two calls in a row share the library's scratch
        sim.step(40)
        h_ref, hbar_ref, w_ref = sim.front_heights()
        mask = torch.from_numpy(pack_mask(sim.mask()).view(np.int32)).to("cuda")
        heights.fill_(-1)
        stats.fill_(-1.0)
        lbm_front_heights_noalloc(mask, W, H, heights, stats)
        torch.cuda.synchronize()
        assert np.array_equal(heights.cpu().numpy(), h_ref)
        hbar, w = stats.cpu().numpy()
        assert hbar == hbar_ref and w == w_ref
        assert w_ref > 0.0 or params["front_amp"] == 0.0
    sim.close()


@pytest.mark.parametrize("W,H", [(257, 40), (4100, 96), (8200, 64), (10000, 33), (32768, 70)])
def test_noalloc_cross_block_synthetic_masks(W, H):
    """Widths of 2, 17, 33, 40 and 128 blocks of 256 columns: every block
    writes its partial sums, the last one to finish adds them; two different
    masks in a row (the completion counter is zeroed by each call)."""
    import torch
    heights = torch.empty(W, dtype=torch.int32, device="cuda")
    stats = torch.empty(2, dtype=torch.float64, device="cuda")
    for seed in (W, W + 1):
        mask = rough_mask(W, H, seed)
        h_ref = host_heights(mask)
        assert h_ref.min() == 0 and h_ref.max() == H  # empty columns and a full one
        h, hbar, w = run_noalloc(mask, heights, stats)
        assert np.array_equal(h, h_ref)
        hbar_ref, w_ref = host_eq6(h_ref)
        assert hbar == hbar_ref and w == w_ref


@pytest.mark.parametrize("W", [8200, 32768])
def test_noalloc_matches_oracle_and_simulation_at_width(W):
    """The initial lattice of a rough sinusoidal front (amplitude 12 rows) on
    W columns: the oracle's heights and Eq. 6 values at step 0, then the
    simulation's own reduction after steps, two calls each."""
    import torch
    from oracle.oracle import OracleSim
    from paper_2303_02210_gb300.lbm import Simulation
    p = wl.lattice_small(seed=40 + W % 7, width=W, height=48, front_kind="sinusoidal", front_row=24.0,
                         front_amp=12.0, front_kmin=1, front_kmax=64, growth_mode="edge", growth_rate=3e-3)
    o = OracleSim(p)
    h_orc, st_orc = o.heights(), o.stats()
    o.close()
    sim = Simulation(p, precision="fp32")
    heights = torch.empty(W, dtype=torch.int32, device="cuda")
    stats = torch.empty(2, dtype=torch.float64, device="cuda")
    mask = sim.mask()
    for _ in range(2):
        h, hbar, w = run_noalloc(mask, heights, stats)
        assert np.array_equal(h, h_orc)
        assert hbar == st_orc["hbar"] and w == st_orc["w"]
    for _ in range(2):
        sim.step(15)
        h_ref, hbar_ref, w_ref = sim.front_heights()
        h, hbar, w = run_noalloc(sim.mask(), heights, stats)
        assert np.array_equal(h, h_ref)
        assert hbar == hbar_ref and w == w_ref
    sim.close()


def test_noalloc_rejects_width_beyond_its_scratch():
    import torch
    from paper_2303_02210_gb300 import lbm
    lib = lbm.load_library()
    W, H = 32769, 4
    mask = torch.zeros((H, (W + 31) // 32), dtype=torch.int32, device="cuda")
    heights = torch.empty(W, dtype=torch.int32, device="cuda")
    stats = torch.empty(2, dtype=torch.float64, device="cuda")
    rc = lib.lbm_front_heights_noalloc(ctypes.c_void_p(mask.data_ptr()), W, H,
                                       ctypes.c_void_p(heights.data_ptr()),
                                       ctypes.c_void_p(stats.data_ptr()), None)
    assert rc == -1
