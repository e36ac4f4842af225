"""Autotuner: the update kernel's form and the planner's grid, per storage
type and lattice width, chosen by measurement.

For every storage type (FP32, FP16, BF16) and width of the sweep it builds
the benchmark's lattice shape at that width (edge-restricted growth, height
W / 2, sinusoidal front at H / 2, fixed rear wall: every tissue row is
updated), and times whole steps (update + planner, CUDA events around a run
of steps after a warm-up) for every staged form of the update (two-row
tiles, four-row tiles, and for FP32 the two-row tiles with bulk tensor
stores) against every planner grid of the sweep. The shortest step wins. It
writes

* ``csrc/lbm_tuned.h``, the table ``lbm_create`` reads (update form and
  planner grid for the entry of the largest tuned width not above W) and
  ``lbm_batch_create`` reads (the narrowest width from which FP32 members
  store in bulk: the narrowest swept width from which the bulk-store form
  wins at every wider swept width), and
* a JSON file with every measured step time (``--out``).

Rebuild the library afterwards (``build.build()``) for the table to take
effect. Run on the GPU the table is for:

    python -m paper_2303_02210_gb300.autotune --out results/autotune_sweep.json

The results of a simulation do not depend on these choices (the staged
forms are bit-exact with each other and the planner with any grid), only
its speed does.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
from typing import Dict, List, Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "csrc", "lbm_tuned.h")

WIDTHS = (256, 512, 1024, 2048, 4096, 8192)
STORAGES = ("fp32", "fp16", "bf16")
# update_kernel names of the staged forms and their table variant numbers
FORMS = {"fp32": (("tma", 0), ("tma1", 1), ("tma_st", 2)), "fp16": (("tma", 0), ("tma1", 1)),
         "bf16": (("tma", 0), ("tma1", 1))}
PLAN_BLOCKS = (4, 8, 16, 24, 38, 48, 64)
PRECISION_CODE = {"fp32": 0, "fp64": 1, "fp16": 2, "bf16": 3}


def shape(width: int, seed: int = 1) -> dict:
    """The benchmark's lattice (lattice_edge) scaled to `width`."""
    from . import workloads as wl
    h = width // 2
    return wl.lattice_edge(seed=seed, width=width, height=h, front_row=float(h // 2))


def step_ms(params: dict, precision: str, kernel: str, plan_blocks: int, steps: int, warm: int = 20) -> float:
    """Milliseconds per step by CUDA events around `steps` steps."""
    import torch
    from .lbm import Simulation
    sim = Simulation(dict(params, plan_blocks=plan_blocks), precision=precision, update_kernel=kernel)
    try:
        sim.step(warm)
        sim.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.step(steps)
        e1.record(sim.stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps
    finally:
        sim.close()


def sweep(widths: Sequence[int] = WIDTHS, storages: Sequence[str] = STORAGES,
          plan_blocks: Sequence[int] = PLAN_BLOCKS, measure=step_ms) -> List[dict]:
    """Every (storage, width, form, planner grid) step time; a form or grid
    the library refuses (more planner blocks than fit, say) is left out."""
    from .lbm import LbmError
    out = []
    for prec in storages:
        for w in widths:
            p = shape(w)
            nodes = w * (w // 2) // 2
            steps = int(min(3000, max(200, 4e8 / max(nodes, 1))))
            for kernel, variant in FORMS[prec]:
                for pb in plan_blocks:
                    try:
                        ms = measure(p, prec, kernel, pb, steps)
                    except LbmError:
                        continue
                    out.append({"precision": prec, "width": w, "kernel": kernel, "variant": variant,
                                "plan_blocks": pb, "steps": steps, "ms_per_step": ms})
    return out


def choose(rows: List[dict]) -> Dict[tuple, dict]:
    """The fastest row per (storage, width)."""
    best: Dict[tuple, dict] = {}
    for r in rows:
        k = (r["precision"], r["width"])
        if k not in best or r["ms_per_step"] < best[k]["ms_per_step"]:
            best[k] = r
    return best


def bulk_min_width(best: Dict[tuple, dict]) -> int:
    """The narrowest swept FP32 width from which the bulk-store form wins at
    every wider swept width (a large value if it never does)."""
    ws = sorted(w for (p, w) in best if p == "fp32")
    for i, w in enumerate(ws):
        if all(best[("fp32", v)]["variant"] == 2 for v in ws[i:]):
            return w
    return 1 << 30


def table_text(best: Dict[tuple, dict], device: str = "", date: Optional[str] = None) -> str:
    """The C header of the tuned table."""
    date = date or datetime.date.today().isoformat()
    lines = [
        "// Generated by paper_2303_02210_gb300/autotune.py; do not edit by hand.",
        "// The update form (KernelTable::tma_info variant: 0 two-row tiles, 1",
        "// four-row tiles, 2 two-row tiles with bulk tensor stores) and the planner's",
        "// cooperative grid (0: the width/capacity rule) with the shortest step, per",
        "// storage type (LBM_FP32 0, LBM_FP16 2, LBM_BF16 3) and lattice width.",
        f"// Measured on {device or 'the GPU the sweep ran on'}, {date}: whole steps of the",
        "// benchmark's lattice shape at each width, timed by CUDA events.",
        "#pragma once",
        "",
        "namespace lbm {",
        "struct TunedShape {",
        "    int precision, width, variant, plan_blocks;",
        "};",
        "constexpr TunedShape kTunedShapes[] = {",
    ]
    for (prec, w) in sorted(best, key=lambda k: (PRECISION_CODE[k[0]], k[1])):
        r = best[(prec, w)]
        lines.append(f"    {{{PRECISION_CODE[prec]}, {w}, {r['variant']}, {r['plan_blocks']}}}, "
                     f"// {r['kernel']}, {r['ms_per_step'] * 1e3:.1f} us per step")
    lines += [
        "};",
        "constexpr int kTunedShapeCount = (int)(sizeof(kTunedShapes) / sizeof(kTunedShapes[0]));",
        "// batched form: FP32 members at least this wide (all of them) store in bulk",
        f"constexpr int kTunedBatchBulkMinWidth = {bulk_min_width(best)};",
        "} // namespace lbm",
        "",
    ]
    return "\n".join(lines)


def main(argv: Optional[List[str]] = None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", default=None, help="write every measured step time here (JSON)")
    ap.add_argument("--table", default=TABLE, help="the header to write")
    ap.add_argument("--widths", type=int, nargs="+", default=list(WIDTHS))
    ap.add_argument("--storages", nargs="+", default=list(STORAGES))
    args = ap.parse_args(argv)
    import torch
    rows = sweep(args.widths, args.storages)
    best = choose(rows)
    device = torch.cuda.get_device_name(0)
    with open(args.table, "w") as fh:
        fh.write(table_text(best, device))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump({"device": device, "date": datetime.date.today().isoformat(), "rows": rows,
                       "best": [best[k] for k in sorted(best)]}, fh, indent=1)
    for k in sorted(best):
        r = best[k]
        print(f"{k[0]} {k[1]:5d}: {r['kernel']:6s} planner {r['plan_blocks']:3d} blocks {r['ms_per_step'] * 1e3:8.1f} us")


if __name__ == "__main__":
    main()
