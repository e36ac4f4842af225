"""Pins for the FP64 CPU oracle against what the paper and the mathematics fix.

Each test names the property it checks and the passage it comes from. They are
chosen so that a plausible slip anywhere in the oracle (a dropped term, a wrong
sign or index, a transposed operand, a wrong coefficient of Eq. 3) fails one:

* streaming direction, periodic wrap and the half-way bounce-back walls:
  ballistic transport of a single population pulse (tau -> infinity);
* the two-step bounce-back of Sec. II: an isolated sub-threshold node returns
  exactly to its own state every two steps and its mass never spreads;
* Eq. 3 coefficients 3, 9/2, 3/2 and the mass conservation of Eqs. 2-4:
  exact mass conservation of a flowing, noisy lattice;
* the friction u* = (1 - mu) u (Sec. II): total momentum decays by exactly
  (1 - mu/tau) per step on a periodic lattice;
* the lattice viscosity of the BGK operator: shear-wave decay at
  nu = (tau - 1/2)/3 (textbook D2Q9 result, not in the paper);
* proliferation (Sec. II, Eq. 5): the growth ledger M(t) = M(0) + rho_cell *
  divisions, the carried site count, uniform site and pair selection, the
  density-dependent acceptance probability;
* Eq. 6 against numpy's standard deviation; the rear-wall rule of App. A;
* the sharp front of Sec. II ("one lattice site with rho < rho_c and beyond
  this the system is devoid of mass").
"""
import math

import numpy as np
import pytest

from oracle.oracle import OracleSim, philox4x32_10
from paper_2303_02210_gb300 import workloads as wl
from tests.lattice_util import E, OPP, WQ, equilibrium, total_mass, total_momentum


def periodic(**kw):
    p = wl.base_params(front_kind="full", y_periodic=1, growth_mode="none", sigma=0.0,
                       wall_mode="fixed")
    p.update(kw)
    return p


# ---------------------------------------------------------------- streaming

@pytest.mark.parametrize("i", range(1, 9))
def test_ballistic_streaming_periodic(i):
    """With tau -> infinity the collision is the identity, so one step moves a
    population pulse by exactly e_i (with periodic wrap at both edges)."""
    W, H = 7, 5
    p = periodic(width=W, height=H, tau=1e12, rho_c=0.0)
    s = OracleSim(p)
    for (x0, y0) in ((0, 0), (W - 1, H - 1), (3, 2)):
        f = np.zeros((9, H, W))
        f[:, :, :] = WQ[:, None, None]
        f[i, y0, x0] += 0.25
        s.set_pops(f)
        s.step(1)
        g = s.pops() - WQ[:, None, None]
        x1, y1 = (x0 + E[i, 0]) % W, (y0 + E[i, 1]) % H
        assert abs(g[i, y1, x1] - 0.25) < 1e-9
        g[i, y1, x1] = 0.0
        assert np.abs(g).max() < 1e-9


@pytest.mark.parametrize("i", [2, 4, 5, 6, 7, 8])
def test_halfway_bounce_back_walls(i):
    """A pulse leaving through the rear (y < 0) or top (y >= H) wall comes back
    into the node it left, in the opposite direction, one step later."""
    W, H = 6, 5
    p = wl.base_params(width=W, height=H, front_kind="full", growth_mode="none", sigma=0.0,
                       tau=1e12, rho_c=0.0, wall_mode="fixed")
    s = OracleSim(p)
    y0 = 0 if E[i, 1] < 0 else H - 1
    f = np.zeros((9, H, W))
    f[:, :, :] = WQ[:, None, None]
    f[i, y0, 2] += 0.25
    s.set_pops(f)
    s.step(1)
    g = s.pops() - WQ[:, None, None]
    assert abs(g[OPP[i], y0, 2] - 0.25) < 1e-9
    g[OPP[i], y0, 2] = 0.0
    assert np.abs(g).max() < 1e-9


def test_isolated_subthreshold_node_reverses_exactly():
    """Sec. II, two-step bounce-back: below rho_c populations are reversed
    instead of relaxed. A lone sub-threshold node sends its mass to its eight
    neighbours, which send it straight back: the state repeats every two steps
    exactly, and no mass ever leaves the 3x3 neighbourhood."""
    W, H = 9, 9
    p = wl.base_params(width=W, height=H, front_kind="full", rho_init=0.0,
                       growth_mode="none", sigma=0.05, wall_mode="fixed")
    s = OracleSim(p)
    f = np.zeros((9, H, W))
    f[:, 4, 4] = np.linspace(0.01, 0.05, 9)  # total 0.27 < rho_c = 0.5
    s.set_pops(f)
    for k in range(1, 41):
        s.step(1)
        g = s.pops()
        rho = g.sum(0)
        assert np.all(rho[:3, :] == 0) and np.all(rho[6:, :] == 0)
        assert np.all(rho[:, :3] == 0) and np.all(rho[:, 6:] == 0)
        assert not s.mask().any()
        if k % 2 == 0:
            assert np.array_equal(g, f)


# ---------------------------------------------------------------- conservation

def test_mass_conserved_without_growth_or_noise():
    """Eqs. 2-3: BGK towards a mass-conserving f^SS, reversal and bounce-back
    walls all conserve mass. A wrong Eq. 3 coefficient (3, 9/2, 3/2) breaks
    this at O(u^2) on a flowing lattice."""
    W, H = 24, 20
    p = periodic(width=W, height=H, tau=0.7, mu=0.01)
    s = OracleSim(p)
    y, x = np.mgrid[0:H, 0:W]
    ux = 0.08 * np.sin(2 * np.pi * y / H)
    uy = 0.06 * np.cos(2 * np.pi * x / W)
    s.set_pops(equilibrium(1.0 + 0.05 * np.cos(2 * np.pi * (x + y) / W), ux, uy))
    m0 = total_mass(s.pops())
    s.step(300)
    assert abs(total_mass(s.pops()) - m0) <= 1e-12 * m0


def test_mass_conserved_with_front_and_walls():
    p = wl.lattice_small(seed=4, growth_mode="none", sigma=0.0)
    s = OracleSim(p)
    m0 = total_mass(s.pops())
    s.step(400)
    assert abs(total_mass(s.pops()) - m0) <= 1e-12 * m0


def test_noise_is_mass_conserving_with_rescale():
    """Eq. 4: eta_i = eta~_i - mean(eta~) sums to zero; the rescaling form of
    the negative-population fix keeps the node's density. Strong noise makes
    many populations negative, so the fix is exercised."""
    p = wl.lattice_small(seed=5, growth_mode="none", sigma=0.08, negfix_mode="rescale")
    s = OracleSim(p)
    m0 = total_mass(s.pops())
    s.step(200)
    f = s.pops()
    assert abs(total_mass(f) - m0) <= 1e-11 * m0
    occ = s.mask()
    assert f[:, occ].min() >= 0.0


def test_noise_statistics_match_eq4():
    """Eq. 4: eta_i = eta~_i - mean_j(eta~_j) with eta~ iid uniform on
    [-sigma, sigma]. On a rest state the BGK step is the identity, so one step
    exposes eta directly: per node it sums to zero, var(eta_i) = (8/27) sigma^2,
    corr(eta_i, eta_j) = -1/8, |eta_i| <= (16/9) sigma, and all nine
    directions are alike."""
    sigma = 1e-3
    p = periodic(width=64, height=64, sigma=sigma)
    s = OracleSim(p)
    f0 = s.pops()
    s.step(1)
    eta = (s.pops() - f0).reshape(9, -1)
    assert np.abs(eta.sum(0)).max() < 1e-15
    var = eta.var(axis=1)
    assert np.all(np.abs(var / (8 / 27 * sigma ** 2) - 1) < 0.06)
    c = np.corrcoef(eta)
    off = c[~np.eye(9, dtype=bool)]
    assert np.all(np.abs(off + 1 / 8) < 0.05)
    assert np.abs(eta).max() <= 16 / 9 * sigma * (1 + 1e-12)
    assert np.abs(eta).max() > 1.3 * sigma  # well beyond a single 8/9 sigma term
    assert np.abs(eta.mean(axis=1)).max() < 3 * np.sqrt(8 / 27) * sigma / 64


def test_noise_uniforms_have_fourteen_bit_resolution():
    """Eq. 4 with the 14-bit reading of the uniforms: eta_i - eta_j =
    2 sigma (u_i - u_j) = 2 sigma (m_i - m_j) 2^-14 with m integer in
    [0, 2^14). On a rest state every difference, scaled by 2^14 / (2 sigma),
    is an integer of magnitude below 2^14, and the extremes come close to it.
    A field of the wrong width, a dropped 1/2 or a wrong scale breaks one of
    these."""
    sigma = 2.0 ** -6  # exact in binary, so the scaled differences are exact
    p = periodic(width=64, height=64, sigma=sigma)
    s = OracleSim(p)
    f0 = s.pops()
    s.step(1)
    eta = (s.pops() - f0).reshape(9, -1)
    d = (eta[1:] - eta[0]) * (2.0 ** 14) / (2.0 * sigma)
    assert np.abs(d - np.rint(d)).max() < 1e-6
    assert np.abs(d).max() < 2 ** 14
    assert np.abs(d).max() > 2 ** 14 * 0.99
    # the lowest bit of each field is random too: half the differences are odd
    odd = np.mod(np.rint(d), 2).astype(bool).mean()
    assert 0.47 < odd < 0.53


def test_literal_negative_fix_adds_twice_the_deficit():
    """App. A step 7 read literally: f_opp(i) += |f_i| and f_i = 0 adds 2|f_i|
    of mass (and keeps momentum). With growth off, the mass gained equals the
    clipped total."""
    p = wl.lattice_small(seed=6, growth_mode="none", sigma=0.08)
    s = OracleSim(p)
    m0 = total_mass(s.pops())
    s.step(100)
    st = s.stats()
    assert st["clip_mass"] > 1.0
    assert abs((total_mass(s.pops()) - m0) - st["clip_mass"]) <= 1e-9 * st["clip_mass"]
    assert s.pops()[:, s.mask()].min() >= 0.0


def test_rest_state_is_stationary():
    """u = 0 everywhere: f^SS = w_i rho, so a uniform rest state stays put."""
    p = periodic(width=10, height=8)
    s = OracleSim(p)
    f0 = s.pops()
    s.step(100)
    assert np.abs(s.pops() - f0).max() < 1e-14


# ---------------------------------------------------------------- friction / viscosity

def test_momentum_decays_by_friction_factor():
    """Sec. II: u* = (1 - mu) u. Since sum_i f^SS_i e_i = rho u*, one BGK step
    maps j -> j (1 - mu/tau); periodic streaming keeps the total. So the total
    momentum after t steps is J(0) (1 - mu/tau)^t exactly."""
    W, H, tau, mu = 16, 12, 0.8, 0.01
    p = periodic(width=W, height=H, tau=tau, mu=mu)
    s = OracleSim(p)
    rng = np.random.default_rng(0)
    s.set_pops(equilibrium(1 + 0.01 * rng.standard_normal((H, W)),
                           0.02 * rng.standard_normal((H, W)), 0.02 * rng.standard_normal((H, W))))
    j0 = total_momentum(s.pops())
    for t in (1, 10, 50):
        s.step(t - s.stats()["step"])
        expect = j0 * (1 - mu / tau) ** t
        assert np.allclose(total_momentum(s.pops()), expect, rtol=1e-10, atol=0)


def test_divisions_add_no_momentum():
    """Sec. II: a division loads two *opposite* populations with rho_cell/2
    each, adding mass but no momentum; so the friction law J(t) = J(0)
    (1 - mu/tau)^t still holds exactly while the lattice grows."""
    W, H, tau, mu = 16, 12, 0.8, 0.01
    p = periodic(width=W, height=H, tau=tau, mu=mu, growth_mode="bulk", growth_rate=5e-3)
    s = OracleSim(p)
    rng = np.random.default_rng(1)
    s.set_pops(equilibrium(1 + 0.01 * rng.standard_normal((H, W)),
                           0.02 * rng.standard_normal((H, W)), 0.02 * rng.standard_normal((H, W))))
    j0 = total_momentum(s.pops())
    s.step(40)
    assert s.stats()["div_total"] > 100
    assert np.allclose(total_momentum(s.pops()), j0 * (1 - mu / tau) ** 40, rtol=1e-10, atol=0)


@pytest.mark.parametrize("tau", [0.8, 1.0])
def test_shear_wave_decay_matches_bgk_viscosity(tau):
    """A shear wave u_x = U sin(2 pi y / H) decays as exp(-nu k^2 t) (1 - mu/tau)^t
    with nu = (tau - 1/2)/3 for D2Q9 BGK; 1% tolerance on the log-decay."""
    W, H, U, mu, T = 4, 128, 1e-3, 0.001, 1000
    p = periodic(width=W, height=H, tau=tau, mu=mu)
    s = OracleSim(p)
    y = np.arange(H)[:, None] * np.ones((1, W))
    s.set_pops(equilibrium(np.ones((H, W)), U * np.sin(2 * np.pi * y / H), np.zeros((H, W))))

    def amp():
        _, ux, _ = s.fields()
        return 2.0 / H * np.sum(ux.mean(1) * np.sin(2 * np.pi * np.arange(H) / H))

    a0 = amp()
    s.step(T)
    nu, k = (tau - 0.5) / 3.0, 2 * np.pi / H
    pred = -nu * k * k * T + T * math.log(1 - mu / tau)
    assert abs(math.log(amp() / a0) / pred - 1) < 0.01


# ---------------------------------------------------------------- proliferation

def test_growth_ledger_and_carried_site_count():
    """Sec. II: each division adds rho_cell (rho_cell/2 to each of two
    opposite populations); n_s = g M / rho_cell per step, carried so that the
    running total stays within one site of the integral; hence
    M(t) ~ M(0) (1 + g)^t."""
    g, rc = 1e-3, 0.1
    p = wl.lattice_small(seed=7, sigma=0.0, growth_rate=g, rho_cell=rc, wall_mode="fixed")
    s = OracleSim(p)
    m0 = total_mass(s.pops())
    ideal = 0.0
    for _ in range(300):
        ideal += g * s.stats()["mass"] / rc
        s.step(1)
        st = s.stats()
        assert abs(st["ns_total"] - ideal) < 1.0 + 1e-9
    assert st["div_total"] == st["ns_total"] and st["starved_steps"] == 0
    assert abs(total_mass(s.pops()) - m0 - rc * st["div_total"]) < 1e-9 * m0
    assert abs(st["mass"] / (m0 * (1 + g) ** 300) - 1) < 1e-4


def _collect_events(s, steps):
    nodes, pairs, counts, tops = [], [], [], []
    for _ in range(steps):
        h_prev = s.heights().copy()
        s.step(1)
        n, pr, c = s.last_events()
        nodes.append(np.repeat(n, c))
        pairs.append(np.repeat(pr, c))
        tops.append((h_prev, n))
    return np.concatenate(nodes), np.concatenate(pairs), tops


def test_bulk_sites_uniform_over_occupied_nodes():
    """Bulk-driven growth (Sec. III): sites are drawn uniformly, with
    replacement, over the occupied active portion; the opposite pair is
    uniform over the four D2Q9 pairs."""
    from scipy import stats as sst
    W, H = 32, 40
    p = wl.lattice_small(seed=8, width=W, height=H, front_row=20.0, front_amp=0.0,
                         sigma=0.0, growth_rate=5e-3, wall_mode="fixed")
    s = OracleSim(p)
    nodes, pairs, _ = _collect_events(s, 100)
    assert len(nodes) > 3000
    ys, xs = nodes // W, nodes % W
    assert ys.max() < 20  # only occupied rows receive divisions
    assert sst.chisquare(np.bincount(xs, minlength=W)).pvalue > 1e-3
    assert sst.chisquare(np.bincount(ys, minlength=20)).pvalue > 1e-3
    assert sst.chisquare(np.bincount(pairs, minlength=4)).pvalue > 1e-3


def test_density_dependent_acceptance_probability():
    """Eq. 5: a drawn site divides with probability 1 - rho/rho0 if rho > rho_c.
    On a uniform rho = 1 lattice with rho0 = 1.5 that is 1/3."""
    p = periodic(width=32, height=32, growth_mode="density", growth_rate=2e-3, rho0=1.5)
    s = OracleSim(p)
    acc = cand = 0
    for _ in range(20):
        s.step(1)
        st = s.stats()
        acc += st["events_last"]
        cand += st["cand_last"]
    assert acc > 300
    assert abs(acc / cand - 1 / 3) < 0.04


def test_density_dependent_growth_stops_above_rho0():
    """Eq. 5: no division where rho >= rho0; every step is starved."""
    p = periodic(width=16, height=16, growth_mode="density", growth_rate=2e-3, rho0=1.5,
                 rho_init=2.0)
    s = OracleSim(p)
    s.step(5)
    st = s.stats()
    assert st["div_total"] == 0 and st["starved_steps"] == 5 and st["ns_total"] > 0


def test_edge_restricted_sites_lie_within_depth_of_front():
    """Edge-restricted growth: every division lies in a node that is tissue
    this step (rho* >= rho_c, so it is occupied after the step) and at most
    `edge_depth` rows below the front of its column as it stood after the
    previous step; all of those depths are used."""
    W, depth = 48, 4
    p = wl.lattice_small(seed=9, width=W, height=48, front_row=24.0, front_amp=3.0,
                         growth_mode="edge", edge_depth=depth, sigma=0.01, growth_rate=5e-3,
                         wall_mode="fixed")
    s = OracleSim(p)
    seen = set()
    for _ in range(40):
        h_prev = s.heights().copy()
        s.step(1)
        n, _, _ = s.last_events()
        ys, xs = n // W, n % W
        d = h_prev[xs] - ys
        assert np.all(d <= depth)
        assert np.all(s.mask()[ys, xs])
        seen.update(d.tolist())
    assert set(range(1, depth + 1)) <= seen


def test_band_restricted_sites_lie_behind_rear_wall_band():
    """App. B: proliferation only in the first `band_rows` rows from the rear
    wall."""
    W = 32
    p = wl.lattice_small(seed=10, width=W, height=64, front_row=40.0, growth_mode="band",
                         band_rows=10, sigma=0.0, growth_rate=5e-3, wall_mode="advance",
                         wall_min_gap=12.0)
    s = OracleSim(p)
    for _ in range(30):
        yr = s.stats()["y_r"]
        s.step(1)
        n, _, _ = s.last_events()
        ys = n // W
        assert len(ys) > 0 and np.all(ys >= yr) and np.all(ys < yr + 10)


def test_candidate_draw_matches_its_definition():
    """The k-th candidate of step t is node y_lo*W + floor(v0 N_win / 2^32)
    with pair v1 >> 30, where (v0, v1, v2, v3) is Philox4x32-10 of counter
    (k, t, 1, sim) under the seed. Recomputed here from the Philox pin and
    compared with the oracle's accepted events (bulk mode, all draws land in
    occupied rows so every candidate is accepted)."""
    W = 16
    p = wl.lattice_small(seed=11, width=W, height=64, front_row=30.0, front_amp=0.0,
                         sigma=0.0, growth_rate=3e-3, wall_mode="fixed", sim_id=3)
    s = OracleSim(p)
    s.step(2)  # step index 2 is next
    st = s.stats()
    ns_expect = math.floor(3e-3 * st["mass"] / 0.1 + st["carry"])
    s.step(1)
    n, pr, c = s.last_events()
    assert s.stats()["ns_last"] == ns_expect
    assert s.stats()["cand_last"] == ns_expect
    nwin = 30 * W  # rows [0, H_top = 30)
    got = {}
    for k in range(ns_expect):
        v = philox4x32_10((k, 2, 1, 3), (11, 0))
        key = ((v[0] * nwin) >> 32, v[1] >> 30)
        got[key] = got.get(key, 0) + 1
    assert got == {(int(a), int(b)): int(cc) for a, b, cc in zip(n, pr, c)}


# ---------------------------------------------------------------- front and wall

def test_front_heights_and_width_match_eq6():
    """Eq. 6: w is the standard deviation of h over the columns (numpy std,
    ddof = 0); h(x) = 1 + highest occupied row."""
    p = wl.lattice_small(seed=12, width=96, height=64, front_kind="sinusoidal",
                         front_row=30.0, front_amp=6.0, front_kmax=8, sigma=0.01,
                         growth_rate=2e-3)
    s = OracleSim(p)
    for _ in range(4):
        s.step(50)
        m = s.mask()
        rows = np.arange(m.shape[0])[:, None]
        h = np.where(m.any(0), (np.where(m, rows, -1)).max(0) + 1, 0)
        assert np.array_equal(h, s.heights())
        st = s.stats()
        assert abs(st["hbar"] - h.mean()) < 1e-12
        assert abs(st["w"] - np.std(h)) < 1e-10
        assert st["H_top"] == h.max() and st["hmin"] == h.min()


def test_sinusoidal_initial_front():
    """Initial front at front_row + amplitude * (normalised sum of sinusoids):
    the tissue fills exactly ceil(h0(x)) rows per column; with k <= 2 the
    profile is smooth, so its discrete spectrum has no power above k = 2."""
    W = 128
    p = wl.lattice_small(seed=13, width=W, height=64, front_kind="sinusoidal",
                         front_row=32.0, front_amp=10.0, front_kmin=1, front_kmax=2)
    s = OracleSim(p)
    h = s.heights().astype(float)
    assert h.max() <= 42 + 1e-9 and h.min() >= 22
    assert h.max() - h.min() >= 15  # the normalised amplitude is reached
    spec = np.abs(np.fft.rfft(h - h.mean()))
    assert spec[3:].max() < 0.05 * spec[1:3].max()


def test_initial_density_jitter_is_uniform():
    """App. A: the initial density is uniform on [0.9, 1.1] rho_init below the
    front, zero above; u = 0 so f = w_i rho."""
    from scipy import stats as sst
    p = wl.paper_params(width=64, height=64, front_row=40.0, front_amp=0.0, seed=21)
    s = OracleSim(p)
    f = s.pops()
    rho = f.sum(0)
    tissue = rho[:40].ravel()
    assert np.all(rho[40:] == 0.0)
    assert tissue.min() >= 0.09 and tissue.max() <= 0.11
    assert sst.kstest((tissue - 0.09) / 0.02, "uniform").pvalue > 1e-3
    assert np.allclose(f[:, :40, :], WQ[:, None, None] * rho[None, :40, :], rtol=1e-15, atol=0)


def test_rear_wall_advances_and_freezes_rows():
    """App. A: the rear wall is kept at least max(gap, 10 w) behind hbar; the
    rows behind it are quiescent (unchanged), and active + quiescent mass is
    the whole lattice's mass."""
    W = 64
    p = wl.lattice_small(seed=14, width=W, height=96, front_kind="sinusoidal", front_row=40.0,
                         front_amp=3.0, front_kmax=4, sigma=0.01, growth_rate=3e-3,
                         wall_mode="advance", wall_min_gap=2.0, wall_w_factor=10.0)
    s = OracleSim(p)
    yr_prev, frozen, rough = 0, None, 0
    for _ in range(300):
        s.step(1)
        st = s.stats()
        f = s.pops()
        rough += 10.0 * st["w"] > 2.0
        expect = max(yr_prev, math.floor(st["hbar"] - max(2.0, 10.0 * st["w"])))
        assert st["y_r"] == min(expect, 95)
        if frozen is not None and yr_prev > 0:
            assert np.array_equal(f[:, :yr_prev, :], frozen[:, :yr_prev, :])
        fix = np.rint(f.sum(0) * 2.0 ** 24).astype(np.int64)
        assert st["mass_fix"] == fix[st["y_r"]:].sum()
        assert st["mass_fix"] + st["quiescent_fix"] == fix.sum()
        yr_prev, frozen = st["y_r"], f
    assert yr_prev > 0 and rough > 50


@pytest.mark.parametrize("mode,sigma", [("bulk", 0.0), ("bulk", 0.01), ("edge", 0.01),
                                        ("density", 0.01)])
def test_front_stays_sharp(mode, sigma):
    """Sec. II: the reversal leaves one sub-threshold layer at the edge and no
    mass beyond it. Exactly: no mass lies above row max(H_top(t), H_top(t-1)),
    H_top = 1 + highest occupied row (a node that has just dropped below rho_c
    still holds, for one step, the mass it emitted while occupied)."""
    p = wl.lattice_small(seed=15, height=96, growth_mode=mode, growth_rate=3e-3, sigma=sigma,
                         rho0=3.0, wall_mode="fixed")
    s = OracleSim(p)
    prev = s.stats()["H_top"]
    for _ in range(600):
        s.step(1)
        rho = s.pops().sum(0)
        st = s.stats()
        top_mass = np.nonzero(rho.any(1))[0].max()
        assert top_mass <= max(st["H_top"], prev)
        prev = st["H_top"]
    assert st["H_top"] > 30  # the front did advance
