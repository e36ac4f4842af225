"""Seeded synthetic workloads: parameter sets shaped like the paper's runs.

This module holds no arithmetic of the method. It only builds plain parameter
dictionaries; the CUDA binding and the CPU oracle each turn the same dictionary
into their own C struct and compute everything themselves (initial front,
densities, random numbers) from it.

Density scale. The paper works at rho_init = 0.1 with rho_c = 0.05,
rho_cell = 0.01, rho0 = 0.15, sigma = 0.01 (App. A, parameter list). The
lattice workloads here use rho_init = 1, so every density-valued parameter is
scaled by 10: rho_c = 0.5, rho_cell = 0.1, rho0 = 1.5. The dynamics are
invariant under that scaling. The noise amplitude is the exception: on D2Q9 the
diagonal rest populations are rho/36 (1/12 of rho on the paper's D2Q7), so the
scaled paper value sigma = 0.1 would drive about a third of all diagonal
populations negative every step, and the literal negative-population fix would
then add mass faster than proliferation does. The lattice workloads therefore
use sigma = 0.01 (noise on, rarely clipped); ``paper_params()`` keeps the
paper's own numbers for anyone who wants them.
"""
from __future__ import annotations


def base_params(**overrides) -> dict:
    """Defaults at the rho_init = 1 scale (see the module docstring)."""
    p = dict(
        width=128, height=64,
        tau=1.0, mu=0.001, rho_c=0.5, rho_cell=0.1, sigma=0.01, rho0=1.5,
        growth_rate=1e-4, growth_mode="bulk", edge_depth=8, band_rows=30,
        rho_init=1.0, rho_jitter=0.0,
        front_kind="flat", front_row=16.0, front_amp=0.5, front_kmin=1, front_kmax=64,
        wall_mode="advance", wall_min_gap=50.0, wall_w_factor=10.0,
        negfix_mode="literal", y_periodic=0,
        seed=1, sim_id=0, lattice="d2q9",
    )
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = v
    return p


def paper_params(**overrides) -> dict:
    """The paper's own parameter list (App. A): rho_init = 0.1 scale, jittered
    initial density U[0.9, 1.1] rho_init, g = 1e-3."""
    p = base_params(tau=1.0, mu=0.001, rho_c=0.05, rho_cell=0.01, sigma=0.01, rho0=0.15,
                    growth_rate=1e-3, rho_init=0.1, rho_jitter=0.1)
    p.update(overrides)
    return p


def lattice_small(seed: int = 1, **kw) -> dict:
    """128 x 64 D2Q9, tissue in the bottom 16 rows (front 16 +- 0.5 seeded
    noise), rho = 1, u = 0, tau = 1.0, bulk growth g = 1e-4 per step; the
    case the oracle finishes in seconds over 1000 steps."""
    p = base_params(width=128, height=64, tau=1.0, growth_rate=1e-4, growth_mode="bulk",
                    front_kind="flat", front_row=16.0, front_amp=0.5, seed=seed)
    p.update(kw)
    return p


def lattice_kpz(seed: int = 1, **kw) -> dict:
    """1024 x 1024, bulk-driven growth g = 1e-4, tau = 0.8, flat front at row 32
    with seeded noise, advancing rear wall (50k-step roughness runs)."""
    p = base_params(width=1024, height=1024, tau=0.8, growth_rate=1e-4, growth_mode="bulk",
                    front_kind="flat", front_row=32.0, front_amp=0.5, wall_mode="advance",
                    seed=seed)
    p.update(kw)
    return p


def lattice_edge(seed: int = 1, **kw) -> dict:
    """4096 x 2048, proliferation restricted to the 8 rows below the front,
    tau = 0.8, front at row 1024 perturbed by the sum of sinusoids with
    wavenumbers 1..64 and random phases, total amplitude 1.0. The rear wall is
    held fixed so that the whole tissue (about 4.2M nodes) is updated every
    step: one FP32 population copy of it is about 151 MB, and a step reads one
    copy and writes the other (about 303 MB), against the 129 MB L2."""
    p = base_params(width=4096, height=2048, tau=0.8, growth_rate=1e-4, growth_mode="edge",
                    edge_depth=8, front_kind="sinusoidal", front_row=1024.0, front_amp=1.0,
                    front_kmin=1, front_kmax=64, wall_mode="fixed", seed=seed)
    p.update(kw)
    return p


def ensemble(n: int = 256, seed: int = 1, **kw) -> list:
    """n independent realisations of uneven sizes, as roughness ensembles need:
    widths drawn uniformly from {256, 512, 1024, 2048} with height = width / 2,
    bulk or edge-restricted growth (depth 8) chosen at random per member,
    tau = 0.8, g = 1e-4, flat front at a quarter of the height with seeded
    noise, advancing rear wall for bulk growth, fixed for edge growth. Member
    i has seed seed + i and its own simulation id."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        W = int(rng.choice([256, 512, 1024, 2048]))
        edge = bool(rng.integers(0, 2))
        p = base_params(width=W, height=W // 2, tau=0.8, growth_rate=1e-4,
                        growth_mode="edge" if edge else "bulk", edge_depth=8,
                        front_kind="flat", front_row=float(W // 8), front_amp=0.5,
                        wall_mode="fixed" if edge else "advance", seed=seed + i, sim_id=i)
        p.update(kw)
        out.append(p)
    return out


def serving_trace(n: int = 200, rate: float = 200.0, steps=(1000, 20000), seed: int = 1,
                  fp16_share: float = 0.5, **kw) -> list:
    """A stream of requests: Poisson arrivals at `rate` per second, widths
    log-uniform in [128, 4096] (multiples of 32) with height = width / 2,
    bulk, edge or density-dependent growth at random, g log-uniform in
    [1e-5, 1e-3], step counts uniform in `steps`, a share `fp16_share` of
    them with FP16 population storage and the rest FP32. Returns (arrival
    seconds, parameters, steps, precision) tuples; request i has seed
    seed + i and its own id."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate)) if i else 0.0
        W = int(round(float(np.exp(rng.uniform(np.log(128), np.log(4096)))) / 32)) * 32
        mode = str(rng.choice(["bulk", "edge", "density"]))
        g = float(np.exp(rng.uniform(np.log(1e-5), np.log(1e-3))))
        nsteps = int(rng.integers(steps[0], steps[1] + 1))
        precision = "fp16" if float(rng.uniform()) < fp16_share else "fp32"
        p = base_params(width=W, height=W // 2, tau=0.8, growth_rate=g, growth_mode=mode, edge_depth=8,
                        front_kind="flat", front_row=float(W // 8), front_amp=0.5,
                        wall_mode="fixed" if mode == "edge" else "advance", seed=seed + i, sim_id=i)
        p.update(kw)
        out.append((t, p, nsteps, precision))
    return out


WORKLOADS = {
    "lattice_small": lattice_small,
    "lattice_kpz": lattice_kpz,
    "lattice_edge": lattice_edge,
}
