"""bench.py's host-side description of the workload (no GPU): the headline
lattice, the L2 note (a population copy of the window larger than the 129 MB
L2, so no flush is needed, or a NOTE where it is not), and the lattice option
used for profiling captures."""
import bench


def _config(lattice: str, width: int, precision: str) -> dict:
    old = (bench.LATTICE, bench.WIDTH)
    bench.LATTICE, bench.WIDTH = lattice, width
    try:
        return bench.workload_config(precision), bench.workload_params()
    finally:
        bench.LATTICE, bench.WIDTH = old


def test_headline_workload_is_d2q9_4096_above_l2():
    cfg, p = _config("d2q9", 4096, "fp32")
    assert cfg["workload"].startswith("D2Q9 4096x2048")
    assert cfg["lattice"] == [4096, 2048] and p.get("lattice", "d2q9") == "d2q9"
    # 9 planes x 4096 columns x ~1026 rows x 4 B = ~151 MB > 129 MB
    assert cfg["l2"].startswith("no flush: each step reads") and "151 MB" in cfg["l2"]


def test_l2_note_follows_the_copy_size():
    cfg, _ = _config("d2q9", 4096, "fp16")
    assert "NOTE" in cfg["l2"] and "76 MB" in cfg["l2"]
    cfg, _ = _config("d2q9", 8192, "fp16")
    assert cfg["l2"].startswith("no flush: each step reads") and "151 MB" in cfg["l2"]
    cfg, p = _config("d2q7", 4096, "fp32")
    assert p["lattice"] == "d2q7" and cfg["workload"].startswith("D2Q7 4096x2048")
    assert "NOTE" in cfg["l2"] and "118 MB" in cfg["l2"]


def test_profiled_traffic_scales_with_nodes():
    """The committed DRAM-traffic figure of the D2Q9 update is used only for
    the kernel sources it was captured from, scaled to the launch's nodes."""
    import json
    import os
    with open(os.path.join(bench.ROOT, "profiles", "k_update_traffic.json")) as fh:
        d = json.load(fh)
    t = bench.profiled_traffic(72, 1000.0)
    if d["kernel_source_hash"] == bench.kernel_source_hash():
        assert abs(t - d["dram_bytes_per_node"] * 1000.0) < 1e-6 * t
        assert 0.5 * 72 < d["dram_bytes_per_node"] <= 1.5 * 72
    else:
        assert t is None


def test_dense_variant_doubles_the_window():
    """The dense C3 variant: the same lattice and growth as the headline with
    the front at row 2044, so the active window (all rows below the top mass
    row + 2) is about twice the headline's 1026 rows."""
    p = bench.dense_params()
    h = bench.workload_params()
    assert (p["width"], p["height"]) == (h["width"], h["height"]) == (4096, 2048)
    assert p["front_row"] == 2044.0 and h["front_row"] == 1024.0
    assert {k: v for k, v in p.items() if k != "front_row"} == {k: v for k, v in h.items() if k != "front_row"}
    assert p["wall_mode"] == "fixed"  # the whole tissue is updated every step


def test_workload_config_knows_every_storage_type():
    """The L2 note's byte count comes from a strict table: an unknown
    precision string is an error, not silently 2 bytes."""
    import pytest
    for pr, mb in (("fp64", 303), ("fp32", 151), ("fp16", 76), ("bf16", 76)):
        cfg, _ = _config("d2q9", 4096, pr)
        assert f"{mb} MB" in cfg["l2"]
    with pytest.raises(KeyError):
        _config("d2q9", 4096, "fp64 (oracle)")
