"""The allocation-free front-height entry point, ``lbm_front_heights_noalloc``.

It serves callers that cannot allocate device memory (an application whose
device memory is held by another allocator, a loop that must not stall on the
allocator): its scratch is a fixed array
inside the library. Here it must reproduce what ``lbm_front_heights`` reports
for a simulation after ``lbm_step`` (heights exactly, mean height and width
to the last bit), on two calls in a row that reuse the same scratch, on a
ragged and a rough lattice, and it must refuse widths beyond its limit.
This file is collected last on purpose.
"""
import ctypes

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
