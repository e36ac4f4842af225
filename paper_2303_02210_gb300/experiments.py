"""Measurements on top of the simulation: the front's Fourier modes, their
growth rates and the dispersion fit of Eq. 8, the proliferation bias
around the most and least advanced parts of the front (Sec. IV, Fig. 3), and
the roughening of the front over an ensemble of realisations (Eq. 6 width
w(t) ~ t^beta, Sec. III).

The analysis functions take plain arrays (front heights h(x) over time,
division sites) and are independent of the GPU; `measure_*` run the
simulation through the C ABI (``lbm.Simulation``) to produce those arrays.

Geometry: the front is h(x), x = 0 .. W - 1 periodic, growing in +y (the
paper grows in x, with y along the front). A mode of wavenumber k has
q = 2 pi k / W.

Run ``python -m paper_2303_02210_gb300.experiments dispersion`` (or
``bias``, ``roughness``, ``kpz``) for a JSON summary.
"""
from __future__ import annotations

import json
import math
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np


# ---------------------------------------------------------------------------
# Analysis (host only)

def front_modes(h: np.ndarray) -> np.ndarray:
    """Complex Fourier amplitudes a_k, k = 0 .. W//2, of a front profile h(x)
    (the last axis), normalised so that h(x) = A cos(2 pi k x / W + phi)
    gives |a_k| = A (0 < k < W/2) and a_0 = mean h."""
    h = np.asarray(h, dtype=np.float64)
    W = h.shape[-1]
    a = np.fft.rfft(h, axis=-1) / W
    a[..., 1:] *= 2.0
    if W % 2 == 0:
        a[..., -1] /= 2.0
    return a


def growth_rates(times: Sequence[float], heights: np.ndarray, ks: Iterable[int],
                 t_min: Optional[float] = None, t_max: Optional[float] = None) -> Dict[int, float]:
    """Exponential growth rate omega_k of each mode k: the least-squares slope
    of log |a_k(t)| against t over the samples with t_min <= t <= t_max
    (heights: one row of h(x) per time). In the frame comoving with the mean
    height (mode 0 is left out), as in the linear stability analysis behind
    Eq. 8."""
    t = np.asarray(times, dtype=np.float64)
    a = np.abs(front_modes(heights))
    sel = np.ones_like(t, dtype=bool)
    if t_min is not None:
        sel &= t >= t_min
    if t_max is not None:
        sel &= t <= t_max
    out = {}
    for k in ks:
        y = a[sel, k]
        ok = y > 0
        if ok.sum() < 2:
            out[k] = float("nan")
            continue
        out[k] = float(np.polyfit(t[sel][ok], np.log(y[ok]), 1)[0])
    return out


def fit_dispersion(q: Sequence[float], omega: Sequence[float]) -> dict:
    """Least-squares fit of omega(q) = k - gamma q^2 (Eq. 8). Returns k,
    gamma, the unstable band q < q_c = sqrt(k / gamma) when k, gamma > 0, the
    paper's critical size L_c = sqrt(gamma / k), and the smallest unstable
    lattice width 2 pi / q_c."""
    q = np.asarray(q, dtype=np.float64)
    w = np.asarray(omega, dtype=np.float64)
    ok = np.isfinite(w)
    A = np.stack([np.ones(ok.sum()), -q[ok] ** 2], axis=1)
    (k, gamma), *_ = np.linalg.lstsq(A, w[ok], rcond=None)
    res = w[ok] - A @ np.array([k, gamma])
    out = {"k": float(k), "gamma": float(gamma), "rms_residual": float(np.sqrt(np.mean(res ** 2))),
           "points": int(ok.sum())}
    if k > 0 and gamma > 0:
        out["q_c"] = math.sqrt(k / gamma)
        out["L_c"] = math.sqrt(gamma / k)
        out["width_c"] = 2 * math.pi / out["q_c"]
    return out


def box_counts(h: np.ndarray, nodes: np.ndarray, counts: np.ndarray, W: int,
               half_width: int = 10, depth: int = 20) -> tuple:
    """Divisions in the two boxes of Fig. 3(c): columns within `half_width`
    of the most (least) advanced column, periodic in x, and the `depth` rows
    below that column's front height. `nodes` are y W + x, `counts` how often
    each was drawn. Returns (count near h_max, count near h_min)."""
    h = np.asarray(h)
    x_hi, x_lo = int(np.argmax(h)), int(np.argmin(h))
    y = np.asarray(nodes) // W
    x = np.asarray(nodes) % W
    c = np.asarray(counts)

    def in_box(xc):
        dx = (x - xc + W // 2) % W - W // 2
        hb = int(h[xc])
        return (np.abs(dx) <= half_width) & (y < hb) & (y >= hb - depth)

    return int(c[in_box(x_hi)].sum()), int(c[in_box(x_lo)].sum())


def ensemble_width(ws: np.ndarray) -> np.ndarray:
    """The ensemble's interface width at each sample time: the root mean
    square over realisations of their Eq. 6 widths, ws[time, realisation]."""
    ws = np.asarray(ws, dtype=np.float64)
    return np.sqrt(np.mean(ws * ws, axis=1))


def growth_exponent(times: Sequence[float], w: Sequence[float], lo: float, hi: float) -> Optional[float]:
    """beta of w ~ t^beta: the least-squares slope of log w against log t over
    the samples with lo <= t <= hi; None if fewer than three samples there
    or a width that is not positive."""
    t = np.asarray(times, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    m = (t >= lo) & (t <= hi)
    if m.sum() < 3 or np.any(w[m] <= 0) or np.any(t[m] <= 0):
        return None
    return float(np.polyfit(np.log(t[m]), np.log(w[m]), 1)[0])


# ---------------------------------------------------------------------------
# Measurements (GPU, through the C ABI)

def dispersion_params(width: int = 512, k: int = 4, amp: float = 4.0, seed: int = 1, **kw) -> dict:
    """One sinusoidal mode on a flat front: the lattice workloads' density
    scale (R22), density-dependent growth (Eq. 5), fixed rear wall, height
    width / 2 with the front at a quarter of it."""
    from . import workloads as wl
    H = width // 2
    p = wl.base_params(width=width, height=H, tau=0.8, growth_mode="density", growth_rate=1e-3,
                       front_kind="sinusoidal", front_row=float(H // 4), front_amp=amp,
                       front_kmin=k, front_kmax=k, wall_mode="fixed", seed=seed, sim_id=k)
    p.update(kw)
    return p


def measure_dispersion(width: int = 512, ks: Sequence[int] = (2, 4, 8, 16, 32), steps: int = 3000,
                       every: int = 50, amp: float = 4.0, precision: str = "fp32", **kw) -> dict:
    """omega(q) from single-mode runs (one simulation per k, the mode's
    amplitude sampled every `every` steps), then the Eq. 8 fit."""
    from .lbm import Simulation
    rows = []
    for k in ks:
        p = dispersion_params(width=width, k=k, amp=amp, **kw)
        sim = Simulation(p, precision=precision)
        times, hs = [], []
        for s in range(0, steps + 1, every):
            if s:
                sim.step(every)
            h, _, _ = sim.front_heights()
            times.append(s)
            hs.append(h.astype(np.float64))
        status = sim.stats()["status"]
        sim.close()
        hs = np.array(hs)
        om = growth_rates(times, hs, [k])[k]
        a = np.abs(front_modes(hs)[:, k])
        rows.append({"k": int(k), "q": 2 * math.pi * k / width, "omega": om,
                     "amp_start": float(a[0]), "amp_end": float(a[-1]), "status": int(status)})
    fit = fit_dispersion([r["q"] for r in rows], [r["omega"] for r in rows])
    return {"width": width, "steps": steps, "every": every, "modes": rows, "fit": fit}


def measure_bias(width: int = 1024, steps: int = 4000, warm: int = 1000, seed: int = 1,
                 precision: str = "fp32", **kw) -> dict:
    """Fig. 3(c): divisions per step near h_max and near h_min (boxes of 21
    columns by 20 rows below the front), density-dependent growth, after
    `warm` steps; and the share of the front's roughness in its longest
    mode at the end (the system-spanning instability of Fig. 3(b))."""
    from .lbm import Simulation
    from . import workloads as wl
    H = width // 2
    p = wl.base_params(width=width, height=H, tau=0.8, growth_mode="density", growth_rate=1e-3,
                       front_kind="flat", front_row=float(H // 4), front_amp=0.5, wall_mode="advance",
                       seed=seed, sim_id=seed)
    p.update(kw)
    sim = Simulation(p, precision=precision)
    sim.step(warm)
    n_hi = n_lo = 0
    for _ in range(steps):
        sim.step(1)
        h, _, _ = sim.front_heights()
        nodes, _, cnt = sim.last_events()
        a, b = box_counts(h, nodes, cnt, width)
        n_hi += a
        n_lo += b
    h, hbar, w = sim.front_heights()
    sim.close()
    a = np.abs(front_modes(h.astype(np.float64)))[1:]
    power = a ** 2
    return {"width": width, "steps": steps, "warm": warm, "divisions_near_hmax": n_hi,
            "divisions_near_hmin": n_lo, "ratio": (n_hi / n_lo) if n_lo else None,
            "hbar": float(hbar), "w": float(w),
            "longest_mode_share": float(power[0] / power.sum()) if power.sum() > 0 else None}


def roughness_params(width: int = 1024, height: int = 8192, seed: int = 1, **kw) -> dict:
    """One realisation of the roughening ensemble: the 1024-wide bulk-growth
    workload (flat front at row 32 with seeded noise, tau = 0.8, advancing
    rear wall) on a lattice tall enough that the front does not reach the top
    within the run, with faster growth (g = 1e-3) by default."""
    from . import workloads as wl
    p = wl.lattice_kpz(seed=seed, width=width, height=height, growth_rate=1e-3, sim_id=seed)
    p.update(kw)
    return p


def measure_roughness(width: int = 1024, seeds: int = 16, steps: int = 20000, every: int = 100,
                      height: int = 8192, windows: Sequence = ((300, 3000), (1000, 10000), (2000, 20000)),
                      precision: str = "fp32", simulation=None, batch=None, **kw) -> dict:
    """w(t) of `seeds` realisations stepped together as one batch, Eq. 6's w
    of each sampled every `every` steps; the ensemble width (ensemble_width)
    and beta over each window of `windows` (growth_exponent). `simulation`
    and `batch` default to lbm.Simulation and lbm.Batch."""
    if simulation is None or batch is None:
        from .lbm import Batch, Simulation
        simulation = simulation or Simulation
        batch = batch or Batch
    sims = [simulation(roughness_params(width=width, height=height, seed=1 + s, **kw), precision=precision)
            for s in range(seeds)]
    b = batch(sims)
    times, ws, hbar = [], [], []
    try:
        for k in range(steps // every):
            b.step(every)
            fh = [sm.front_heights() for sm in sims]
            times.append((k + 1) * every)
            ws.append([f[2] for f in fh])
            hbar.append(float(np.mean([f[1] for f in fh])))
        status = sorted({int(sm.stats()["status"]) for sm in sims})
    finally:
        b.close()
        for sm in sims:
            sm.close()
    w = ensemble_width(np.array(ws)) if ws else np.zeros(0)
    return {"width": width, "height": height, "seeds": seeds, "steps": steps, "every": every,
            "t": times, "w": [float(v) for v in w], "hbar": hbar, "status": status,
            "beta": {f"{lo}-{hi}": growth_exponent(times, w, lo, hi) for lo, hi in windows}}


def kpz_exponents(times: Sequence[float], ws_by_width: Dict[int, np.ndarray], beta_window: Sequence[float],
                  sat_from: float, resamples: int = 200, seed: int = 0,
                  t_end: Optional[Dict[int, float]] = None) -> dict:
    """The KPZ exponents of an ensemble with error bars over its seeds.

    ws_by_width[L][time, seed] are the Eq. 6 widths of the realisations of
    width L. beta (w ~ t^beta, Eq. 6 and Sec. III) is fitted to each L's
    ensemble width (ensemble_width) over beta_window = (lo, hi); hi = None
    ends each L's window at its crossover t_x, the first sample at which its
    ensemble width reaches 0.8 of its saturated width (fixed from the whole
    ensemble, before any resampling; no fit if t_x <= 2 lo); alpha
    (w_sat ~ L^alpha) to the saturated widths, each L's ensemble width
    averaged over the samples with t >= sat_from, against L on log-log axes.
    Error bars: the standard deviation over `resamples` bootstrap ensembles
    (the seeds of each width drawn with replacement). t_end[L], if given,
    drops L's samples after that time (e.g. once a front nears the top
    wall)."""
    t = np.asarray(times, dtype=np.float64)
    Ls = sorted(ws_by_width)
    rng = np.random.default_rng(seed)
    lo, hi = beta_window
    end = {L: (t_end or {}).get(L, np.inf) for L in Ls}
    sat = {L: (t >= sat_from) & (t <= end[L]) for L in Ls}
    his = {}
    for L in Ls:
        if hi is not None:
            his[L] = min(hi, end[L])
            continue
        w = ensemble_width(np.asarray(ws_by_width[L], dtype=np.float64))
        reach = np.nonzero(w >= 0.8 * np.mean(w[sat[L]]))[0] if sat[L].any() else []
        tx = float(t[reach[0]]) if len(reach) else float(t[-1])
        his[L] = min(tx, end[L]) if tx > 2 * lo else lo  # (lo: too short, growth_exponent gives None)

    def fits(sample):
        betas = {L: growth_exponent(t, ensemble_width(sample[L]), lo, his[L]) for L in Ls}
        wsat = np.array([float(np.mean(ensemble_width(sample[L])[sat[L]])) if sat[L].any() else np.nan
                         for L in Ls])
        ok = np.isfinite(wsat) & (wsat > 0)
        alpha = float(np.polyfit(np.log(np.array(Ls, dtype=np.float64)[ok]), np.log(wsat[ok]), 1)[0]) \
            if ok.sum() >= 2 else None
        return betas, wsat, alpha

    betas, wsat, alpha = fits({L: np.asarray(ws_by_width[L], dtype=np.float64) for L in Ls})
    boot_b = {L: [] for L in Ls}
    boot_a = []
    for _ in range(resamples):
        smp = {}
        for L in Ls:
            w = np.asarray(ws_by_width[L], dtype=np.float64)
            smp[L] = w[:, rng.integers(0, w.shape[1], w.shape[1])]
        b, _, a = fits(smp)
        for L in Ls:
            if b[L] is not None:
                boot_b[L].append(b[L])
        if a is not None:
            boot_a.append(a)
    return {
        "beta": {L: betas[L] for L in Ls},
        "beta_err": {L: float(np.std(boot_b[L])) if boot_b[L] else None for L in Ls},
        "beta_window": {L: [float(lo), float(his[L])] for L in Ls},
        "w_sat": {L: float(v) for L, v in zip(Ls, wsat)},
        "alpha": alpha,
        "alpha_err": float(np.std(boot_a)) if boot_a else None,
        "sat_from": float(sat_from),
    }


def kpz_params(width: int, seed: int, height: int, front_row: float = 60.0, **kw) -> dict:
    """One realisation in the paper's own regime (App. A parameter list): the
    triangular D2Q7 lattice, rho_init = 0.1 with the U[0.9, 1.1] jitter,
    sigma = 0.01, tau = 1, mu = 0.001, g = 1e-3, rho_cell = 0.01, bulk
    growth, the rear wall max(50, 10 w) behind the front, a flat front at
    `front_row` with seeded noise of amplitude 0.5."""
    from . import workloads as wl
    p = wl.paper_params(width=width, height=height, lattice="d2q7", growth_mode="bulk", wall_mode="advance",
                        wall_min_gap=50.0, wall_w_factor=10.0, front_kind="flat", front_row=front_row,
                        front_amp=0.5, seed=seed, sim_id=seed)
    p.update(kw)
    return p


def measure_kpz(widths: Sequence[int] = (64, 128, 256, 512), seeds: int = 32, steps: int = 40000,
                every: int = 200, height: int = 4096, beta_window: Optional[Sequence[float]] = None,
                sat_from: Optional[float] = None, precision: str = "fp32", simulation=None, batch=None,
                **kw) -> dict:
    """The roughening check of Sec. III in the paper's regime (kpz_params):
    `seeds` realisations of each width, all stepped together as one batch,
    Eq. 6's w and the mean height of each sampled every `every` steps (kept
    per realisation); kpz_exponents over them (beta over beta_window, default
    from 4 every to a tenth of the run; alpha from the last third of the run
    by default; each width's samples only up to the last one before any of
    its fronts came within 256 rows of the top wall), the mean front
    position, and per width the mass the literal negative-population fix
    (App. A step 7) added against the mass the divisions added."""
    if simulation is None or batch is None:
        from .lbm import Batch, Simulation
        simulation = simulation or Simulation
        batch = batch or Batch
    members = [(L, s) for L in widths for s in range(seeds)]
    sims = [simulation(kpz_params(L, 1 + 1000 * i + s, height, **kw), precision=precision)
            for i, L in enumerate(widths) for s in range(seeds)]
    b = batch(sims)
    times, ws, hbar = [], [], []
    try:
        for k in range(steps // every):
            b.step(every)
            fh = [sm.front_heights() for sm in sims]
            times.append((k + 1) * every)
            ws.append([f[2] for f in fh])
            hbar.append([f[1] for f in fh])
        stats = [sm.stats() for sm in sims]
    finally:
        b.close()
        for sm in sims:
            sm.close()
    ws = np.array(ws)
    hb = np.array(hbar)
    by = {L: ws[:, [j for j, (l, _) in enumerate(members) if l == L]] for L in widths}
    rho_cell = kpz_params(widths[0], 1, height, **kw)["rho_cell"]
    hby = {L: hb[:, [j for j, (l, _) in enumerate(members) if l == L]] for L in widths}
    t_end = {}
    for L in widths:
        near = np.nonzero(hby[L].max(axis=1) > height - 256)[0] if len(times) else []
        t_end[L] = float(times[near[0] - 1]) if len(near) and near[0] > 0 else (float(times[-1]) if len(near) == 0
                                                                                  else 0.0)
    out = {"widths": list(widths), "seeds": seeds, "steps": steps, "every": every, "height": height,
           "t": times, "w": {L: [float(v) for v in ensemble_width(by[L])] for L in widths},
           "hbar": {L: [float(v) for v in hby[L].mean(1)] for L in widths},
           "w_seeds": {L: by[L].tolist() for L in widths}, "hbar_seeds": {L: hby[L].tolist() for L in widths},
           "t_end": t_end, "status": sorted({int(st["status"]) for st in stats})}
    neg = {}
    for L in widths:
        sel = [st for st, (l, _) in zip(stats, members) if l == L]
        clip = float(np.mean([st["clip_mass"] for st in sel]))
        div = float(np.mean([st["div_total"] for st in sel])) * rho_cell
        neg[L] = {"negfix_mass_per_step": clip / steps, "division_mass_per_step": div / steps,
                  "negfix_share": clip / (clip + div) if clip + div > 0 else None}
    out["mass_sources"] = neg
    if times:
        lo, hi = beta_window if beta_window is not None else (4 * every, max(5 * every, steps / 10))
        out["fit"] = kpz_exponents(times, by, (lo, hi), sat_from if sat_from is not None else 2 * steps / 3,
                                   t_end=t_end)
    return out


def main(argv: Optional[List[str]] = None) -> None:
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("what", choices=["dispersion", "bias", "roughness", "kpz"])
    ap.add_argument("--width", type=int, default=None)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--seeds", type=int, default=None, help="realisations (roughness, kpz)")
    ap.add_argument("--widths", type=int, nargs="+", default=None, help="lattice widths (kpz)")
    ap.add_argument("--height", type=int, default=None)
    ap.add_argument("--every", type=int, default=None, help="steps between samples (roughness, kpz)")
    ap.add_argument("--negfix", choices=["literal", "rescale"], default=None,
                    help="reading of the negative-population fix (kpz)")
    ap.add_argument("--beta-from", type=float, default=None, help="start of the beta window (kpz)")
    ap.add_argument("--sat-from", type=float, default=None, help="start of the saturated samples (kpz)")
    ap.add_argument("--save", default=None, help="write the full output (per realisation) as JSON here (kpz)")
    args = ap.parse_args(argv)
    kw = {k: v for k, v in (("width", args.width), ("steps", args.steps)) if v is not None}
    if args.what == "dispersion":
        out = measure_dispersion(**kw)
    elif args.what == "bias":
        out = measure_bias(**kw)
    elif args.what == "kpz":
        kw.pop("width", None)
        for name, v in (("seeds", args.seeds), ("height", args.height), ("every", args.every),
                        ("sat_from", args.sat_from), ("negfix_mode", args.negfix)):
            if v is not None:
                kw[name] = v
        if args.widths:
            kw["widths"] = tuple(args.widths)
        if args.beta_from is not None:
            kw["beta_window"] = (args.beta_from, None)
        out = measure_kpz(**kw)
        if args.save:
            with open(args.save, "w") as fh:
                json.dump(out, fh)
        out = {k: v for k, v in out.items() if k not in ("w_seeds", "hbar_seeds")}
    else:
        if args.seeds is not None:
            kw["seeds"] = args.seeds
        out = measure_roughness(**kw)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
