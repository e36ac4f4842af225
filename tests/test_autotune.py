"""The autotuner: its choice of the fastest form and planner grid per
storage type and width, the bulk-store threshold it derives, the header it
writes (checked on the CPU with a stand-in timer), the committed table's
entries, and on the GPU that the planner's grid, which the table sets, leaves
every result unchanged."""
import re

import numpy as np
import pytest

from paper_2303_02210_gb300 import autotune


def _fake_measure(params, precision, kernel, plan_blocks, steps):
    # a step time with a known optimum: the bulk-store form wins from 2048
    # columns on, the four-row form for 16 bits at 8192, 16 planner blocks
    w = params["width"]
    base = w * w * 1e-9
    form = {"tma": 1.0, "tma1": 1.05, "tma_st": 1.02}[kernel]
    if kernel == "tma_st" and w >= 2048:
        form = 0.95
    if kernel == "tma1" and precision != "fp32" and w >= 8192:
        form = 0.9
    return base * form + abs(plan_blocks - 16) * 1e-6


def test_sweep_chooses_the_fastest_form_and_grid_and_writes_the_table():
    rows = autotune.sweep(widths=(512, 2048, 8192), storages=("fp32", "fp16"), plan_blocks=(8, 16, 24),
                          measure=_fake_measure)
    assert len(rows) == 3 * 3 * 3 + 3 * 2 * 3
    best = autotune.choose(rows)
    assert best[("fp32", 512)]["kernel"] == "tma" and best[("fp32", 2048)]["kernel"] == "tma_st"
    assert best[("fp16", 8192)]["kernel"] == "tma1" and best[("fp16", 2048)]["kernel"] == "tma"
    assert all(r["plan_blocks"] == 16 for r in best.values())
    assert autotune.bulk_min_width(best) == 2048
    text = autotune.table_text(best, device="test", date="2000-01-01")
    entries = re.findall(r"\{(\d+), (\d+), (\d+), (\d+)\}", text)
    assert ("0", "2048", "2", "16") in entries and ("2", "8192", "1", "16") in entries
    assert "kTunedBatchBulkMinWidth = 2048;" in text


def test_bulk_threshold_needs_every_wider_width():
    best = {("fp32", 1024): {"variant": 2}, ("fp32", 2048): {"variant": 0}, ("fp32", 4096): {"variant": 2}}
    assert autotune.bulk_min_width(best) == 4096
    assert autotune.bulk_min_width({("fp32", 1024): {"variant": 0}}) == 1 << 30


def test_committed_table_is_well_formed():
    text = open(autotune.TABLE).read()
    entries = [tuple(int(v) for v in m) for m in re.findall(r"\{(\d+), (\d+), (\d+), (\d+)\}", text)]
    assert entries
    for prec, width, variant, pb in entries:
        assert prec in (0, 2, 3) and width >= 1 and 0 <= pb <= 1024
        assert variant in ((0, 1, 2) if prec == 0 else (0, 1))
    for prec in {e[0] for e in entries}:
        ws = [e[1] for e in entries if e[0] == prec]
        assert ws == sorted(set(ws))
    assert re.search(r"kTunedBatchBulkMinWidth = \d+;", text)


@pytest.mark.gpu
def test_planner_grid_leaves_results_unchanged():
    """The planner grid that the tuned table (or plan_blocks) sets changes
    no result: populations, mask, heights and every counter bit for bit with
    2, 7 and 38 blocks and the automatic choice; a grid larger than the
    resident count is refused."""
    from paper_2303_02210_gb300 import workloads as wl
    from paper_2303_02210_gb300.lbm import LbmError, Simulation
    p = wl.lattice_small(seed=21, width=300, height=96, front_row=30.0, growth_rate=3e-3, growth_mode="edge",
                         edge_depth=4, front_kind="sinusoidal", front_amp=2.0)
    ref = None
    for pb in (0, 2, 7, 38):
        s = Simulation(dict(p, plan_blocks=pb), precision="fp32")
        s.step(60)
        got = (s.pops(), s.mask(), s.heights(), {k: v for k, v in s.stats().items() if k != "launches"})
        s.close()
        if ref is None:
            ref = got
            continue
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
        assert got[3] == ref[3]
    with pytest.raises(LbmError):
        Simulation(dict(p, plan_blocks=1024), precision="fp32")
