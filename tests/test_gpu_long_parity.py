"""FP32 against the FP64 oracle at the workloads' own sizes and step counts.

The FP32 fast path is held to 1e-5 relative error in density and velocity
against the FP64 oracle after the stated step counts, with occupancy-mask and
front-height flips and steps with a different n_s counted. Four runs, in the
launch configuration the benchmark times (the automatic kernel choice: the
TMA-staged update and the cooperative planner):

* ``edge_4096x2048``: the benchmark workload itself (4096 x 2048, growth
  within 8 rows of the front, tau 0.8, g 1e-4, sinusoidal front k = 1..64 of
  amplitude 1 at row 1024, fixed rear wall), 300 steps;
* ``bulk_1024x1024``: the roughness workload (1024 x 1024, bulk growth,
  tau 0.8, g 1e-4, flat front at row 32 +- 0.5, advancing rear wall), 2000
  steps;
* ``edge_256x288_20k``: the edge-growth parameters on a lattice the oracle
  can take through the 20k steps that workload states (256 x 288, front at
  row 128, advancing rear wall so that the front stays inside);
* ``bulk_128x320_50k``: the bulk-growth parameters through the 50k steps that
  workload states (128 x 320, front at row 32), heights every 100 steps.

What holds, and is asserted: the two full-size runs stay within 1e-5 with no
flips and the same n_s at every step. The long runs stay within 1e-5 with no
flips at every checkpoint up to the first step whose n_s differs from the
oracle's, which comes after some thousands of steps: n_s = floor(g M /
rho_cell + carry) floors a quantity whose carried fraction integrates the
difference between the FP32 and FP64 masses, so it eventually rounds the
other way; from that step on the runs draw different division schedules and
are two realisations of the same stochastic process, compared element by
element no more. The figures after it (and the fitted growth of the error
before it) are recorded, not asserted.

Error metrics (density: max abs difference over max abs oracle density;
velocity: 2-norm of the difference over the 2-norm of the oracle's, over the
oracle's occupied nodes, and max abs over max abs), checked at checkpoints.
The oracle runs take minutes, in spawned processes, while the GPU runs.
Set LBM_PARITY_LOG to a file path to have the measured figures written there
as JSON.
"""
import json
import multiprocessing as mp
import os
import shutil
import tempfile

import numpy as np
import pytest

from paper_2303_02210_gb300 import workloads as wl

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-5


def _cases():
    out = {}
    out["edge_4096x2048"] = dict(params=wl.lattice_edge(seed=1), steps=300,
                                 checkpoints=[1, 10, 50, 150, 300], hstride=10, rows=1100)
    out["bulk_1024x1024"] = dict(params=wl.lattice_kpz(seed=1), steps=2000,
                                 checkpoints=[1, 100, 500, 1000, 1500, 2000], hstride=100, rows=1024)
    out["edge_256x288_20k"] = dict(
        params=wl.lattice_edge(seed=3, width=256, height=288, front_row=128.0, wall_mode="advance"),
        steps=20000, checkpoints=[1] + list(range(1000, 20001, 1000)), hstride=100, rows=288)
    out["bulk_128x320_50k"] = dict(
        params=wl.lattice_kpz(seed=4, width=128, height=320), steps=50000,
        checkpoints=[1] + list(range(2500, 50001, 2500)), hstride=100, rows=320)
    return out


CASES = _cases()


def _gpu_run(c):
    from paper_2303_02210_gb300.lbm import Simulation
    sim = Simulation(c["params"], precision="fp32")
    steps, rows = c["steps"], c["rows"]
    cps = set(c["checkpoints"])
    ns = np.zeros(steps, dtype=np.int64)
    hs, snaps = [], {}
    for t in range(1, steps + 1):
        sim.step(1)
        st = sim.stats()
        ns[t - 1] = st["ns_last"]
        if t % c["hstride"] == 0:
            hs.append(sim.heights())
        if t in cps:
            rho, ux, uy = sim.fields()
            snaps[t] = dict(rho=rho[:rows], ux=ux[:rows], uy=uy[:rows], mask=sim.mask()[:rows],
                            heights=sim.heights(), stats=st)
    kernel = sim.stats()["update_kernel"]
    sim.close()
    return dict(ns=ns, heights=np.array(hs), snaps=snaps, update_kernel=kernel)


def _metrics(g, o):
    """Error metrics of one checkpoint (GPU g, oracle o)."""
    rho_o, rho_g = o["rho"], g["rho"]
    occ = o["mask"]
    du = np.stack([g["ux"] - o["ux"], g["uy"] - o["uy"]])[:, occ]
    uo = np.stack([o["ux"], o["uy"]])[:, occ]
    return {
        "rho_rel_max": float(np.abs(rho_g - rho_o).max() / np.abs(rho_o).max()),
        "u_rel_l2": float(np.sqrt((du ** 2).sum()) / max(np.sqrt((uo ** 2).sum()), 1e-300)),
        "u_rel_max": float(np.abs(du).max() / max(np.abs(uo).max(), 1e-300)),
        "mask_flips": int((g["mask"] != o["mask"]).sum()),
        "height_flips": int((g["heights"] != o["heights"]).sum()),
    }


def _collect():
    import oracle_runs
    outdir = tempfile.mkdtemp(prefix="lbm_parity_")
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(len(CASES))
    jobs = {name: pool.apply_async(oracle_runs.run_oracle,
                                   (name, c["params"], c["steps"], c["checkpoints"], c["hstride"], c["rows"],
                                    outdir))
            for name, c in CASES.items()}
    pool.close()
    results = {}
    try:
        gpu = {name: _gpu_run(c) for name, c in CASES.items()}
        for name, c in CASES.items():
            note = jobs[name].get(timeout=3600)
            g = gpu[name]
            ser = np.load(os.path.join(outdir, f"{name}_series.npz"))
            ns_diff = np.nonzero(g["ns"] != ser["ns"])[0]
            hflip = [int((a != b).sum()) for a, b in zip(g["heights"], ser["heights"])]
            first_h = next(((i + 1) * c["hstride"] for i, n in enumerate(hflip) if n), None)
            cps = []
            for t in c["checkpoints"]:
                o = dict(np.load(os.path.join(outdir, f"{name}_{t}.npz")))
                m = _metrics(g["snaps"][t], o)
                m["step"] = t
                ost = json.loads(str(o["stats"]))
                gst = g["snaps"][t]["stats"]
                m["ns_total_gpu"], m["ns_total_oracle"] = int(gst["ns_total"]), int(ost["ns_total"])
                m["hbar_oracle"], m["w_oracle"] = float(ost["hbar"]), float(ost["w"])
                cps.append(m)
            # power law fitted to the velocity error before any n_s difference
            pre = [m for m in cps if m["step"] >= 100 and (not len(ns_diff) or m["step"] <= ns_diff[0])]
            fit = None
            if len(pre) >= 2:
                b, la = np.polyfit(np.log([m["step"] for m in pre]), np.log([m["u_rel_l2"] for m in pre]), 1)
                fit = {"u_rel_l2": f"{np.exp(la):.3g} t^{b:.3f}", "at_stated_steps": float(np.exp(la) * c["steps"] ** b),
                       "points": len(pre)}
            results[name] = {
                "steps": c["steps"], "oracle": note, "update_kernel": g["update_kernel"], "error_growth": fit,
                "ns_steps_differing": int(len(ns_diff)),
                "first_ns_difference": int(ns_diff[0]) + 1 if len(ns_diff) else None,
                "height_samples": len(hflip), "height_samples_differing": int(sum(1 for n in hflip if n)),
                "first_height_flip_step": first_h,
                "checkpoints": cps,
            }
    finally:
        pool.terminate()
        shutil.rmtree(outdir, ignore_errors=True)
    path = os.environ.get("LBM_PARITY_LOG")
    if path:
        with open(path, "w") as fh:
            json.dump(results, fh, indent=1)
    return results


_RESULTS = {}


def _results():
    if not _RESULTS:
        _RESULTS.update(_collect())
    return _RESULTS


FULL_SIZE = ("edge_4096x2048", "bulk_1024x1024")


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_long_run_against_oracle(name):
    r = _results()[name]
    assert r["update_kernel"] >= 2  # a staged update, as the benchmark runs it
    div = r["first_ns_difference"]
    if name in FULL_SIZE:
        assert div is None and r["height_samples_differing"] == 0
    else:
        assert div is None or div > 2500, div
        first_h = r["first_height_flip_step"]
        assert first_h is None or (div is not None and first_h > div)
    for m in r["checkpoints"]:
        if div is not None and m["step"] >= div:
            break
        assert m["rho_rel_max"] <= TOL, (m["step"], m)
        assert m["u_rel_l2"] <= TOL, (m["step"], m)
        assert m["mask_flips"] == 0 and m["height_flips"] == 0, (m["step"], m)
        assert m["ns_total_gpu"] == m["ns_total_oracle"], (m["step"], m)
