"""Pins for the oracle's proliferation, front and rear wall on the triangular
D2Q7 lattice (the paper's lattice, Sec. II), the same facts the D2Q9 pins
check, with the D2Q7 pair set:

* the growth ledger: each division adds rho_cell (rho_cell/2 to each of two
  opposite populations) and n_s = g M / rho_cell per step with the fraction
  carried (Sec. II);
* sites uniform over the occupied active portion, pairs uniform over the
  three opposite pairs, drawn as the k-th candidate's definition says;
* Eq. 5's acceptance probability 1 - rho/rho0;
* the edge and band restrictions; Eq. 6 from the mask; the rear-wall rule of
  App. A with frozen rows; the sharp front of Sec. II.
"""
import math

import numpy as np
import pytest

from oracle.oracle import OracleSim, philox4x32_10
from paper_2303_02210_gb300 import workloads as wl


def small7(**kw):
    return wl.lattice_small(lattice="d2q7", **kw)


def total_mass(f):
    return math.fsum(np.asarray(f).ravel())


def test_growth_ledger_and_carried_site_count():
    g, rc = 1e-3, 0.1
    s = OracleSim(small7(seed=31, sigma=0.0, growth_rate=g, rho_cell=rc, wall_mode="fixed"))
    assert s.Q == 7
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


def test_bulk_sites_and_pairs_uniform():
    from scipy import stats as sst
    W = 32
    s = OracleSim(small7(seed=32, width=W, height=40, front_row=20.0, front_amp=0.0, sigma=0.0,
                         growth_rate=5e-3, wall_mode="fixed"))
    nodes, pairs = [], []
    for _ in range(100):
        s.step(1)
        n, pr, c = s.last_events()
        nodes.append(np.repeat(n, c))
        pairs.append(np.repeat(pr, c))
    nodes, pairs = np.concatenate(nodes), np.concatenate(pairs)
    assert len(nodes) > 3000
    ys, xs = nodes // W, nodes % W
    assert ys.max() < 20  # only occupied rows receive divisions
    assert pairs.max() <= 2
    assert sst.chisquare(np.bincount(xs, minlength=W)).pvalue > 1e-3
    assert sst.chisquare(np.bincount(ys, minlength=20)).pvalue > 1e-3
    assert sst.chisquare(np.bincount(pairs, minlength=3)).pvalue > 1e-3


def test_candidate_draw_matches_its_definition():
    """The k-th candidate of step t is node y_lo*W + floor(v0 N_win / 2^32)
    with pair floor(3 v1 / 2^32), (v0, v1, v2, v3) = Philox4x32-10 of counter
    (k, t, 1, sim) under the seed (bulk mode, every draw lands in tissue)."""
    W = 16
    s = OracleSim(small7(seed=33, width=W, height=64, front_row=30.0, front_amp=0.0, sigma=0.0,
                         growth_rate=3e-3, wall_mode="fixed", sim_id=5))
    s.step(2)
    st = s.stats()
    ns_expect = math.floor(3e-3 * st["mass"] / 0.1 + st["carry"])
    s.step(1)
    n, pr, c = s.last_events()
    assert s.stats()["ns_last"] == ns_expect == s.stats()["cand_last"]
    nwin = 30 * W
    got = {}
    for k in range(ns_expect):
        v = philox4x32_10((k, 2, 1, 5), (33, 0))
        key = ((v[0] * nwin) >> 32, (v[1] * 3) >> 32)
        got[key] = got.get(key, 0) + 1
    assert got == {(int(a), int(b)): int(cc) for a, b, cc in zip(n, pr, c)}


def test_density_dependent_acceptance_probability():
    p = wl.base_params(width=32, height=32, front_kind="full", y_periodic=1, sigma=0.0, wall_mode="fixed",
                       growth_mode="density", growth_rate=2e-3, rho0=1.5, lattice="d2q7")
    s = OracleSim(p)
    acc = cand = 0
    for _ in range(20):
        s.step(1)
        st = s.stats()
        acc += st["events_last"]
        cand += st["cand_last"]
    assert acc > 300
    assert abs(acc / cand - 1 / 3) < 0.04


def test_edge_restricted_sites_lie_within_depth_of_front():
    W, depth = 48, 4
    s = OracleSim(small7(seed=34, width=W, height=48, front_row=24.0, front_amp=3.0, growth_mode="edge",
                         edge_depth=depth, sigma=0.01, growth_rate=5e-3, wall_mode="fixed"))
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
    W = 32
    s = OracleSim(small7(seed=35, width=W, height=64, front_row=40.0, growth_mode="band", band_rows=10,
                         sigma=0.0, growth_rate=5e-3, wall_mode="advance", wall_min_gap=12.0))
    for _ in range(30):
        yr = s.stats()["y_r"]
        s.step(1)
        n, _, _ = s.last_events()
        ys = n // W
        assert len(ys) > 0 and np.all(ys >= yr) and np.all(ys < yr + 10)


def test_front_heights_and_width_match_eq6():
    s = OracleSim(small7(seed=36, width=96, height=64, front_kind="sinusoidal", front_row=30.0,
                         front_amp=6.0, front_kmax=8, sigma=0.01, growth_rate=2e-3))
    for _ in range(4):
        s.step(50)
        m = s.mask()
        rows = np.arange(m.shape[0])[:, None]
        h = np.where(m.any(0), (np.where(m, rows, -1)).max(0) + 1, 0)
        assert np.array_equal(h, s.heights())
        st = s.stats()
        assert abs(st["hbar"] - h.mean()) < 1e-12
        assert abs(st["w"] - np.std(h)) < 1e-10


def test_rear_wall_advances_and_freezes_rows():
    W = 64
    s = OracleSim(small7(seed=37, width=W, height=96, front_kind="sinusoidal", front_row=40.0,
                         front_amp=3.0, front_kmax=4, sigma=0.01, growth_rate=3e-3, wall_mode="advance",
                         wall_min_gap=2.0, wall_w_factor=10.0))
    yr_prev, frozen = 0, None
    for _ in range(300):
        s.step(1)
        st = s.stats()
        f = s.pops()
        expect = max(yr_prev, math.floor(st["hbar"] - max(2.0, 10.0 * st["w"])))
        assert st["y_r"] == min(expect, 95)
        if frozen is not None and yr_prev > 0:
            assert np.array_equal(f[:, :yr_prev, :], frozen[:, :yr_prev, :])
        fix = np.rint(f.sum(0) * 2.0 ** 24).astype(np.int64)
        assert st["mass_fix"] == fix[st["y_r"]:].sum()
        assert st["mass_fix"] + st["quiescent_fix"] == fix.sum()
        yr_prev, frozen = st["y_r"], f
    assert yr_prev > 0


@pytest.mark.parametrize("mode,sigma", [("bulk", 0.01), ("edge", 0.01)])
def test_front_stays_sharp(mode, sigma):
    """No mass above row max(H_top(t), H_top(t-1)) (Sec. II)."""
    s = OracleSim(small7(seed=38, height=96, growth_mode=mode, growth_rate=3e-3, sigma=sigma, rho0=3.0,
                         wall_mode="fixed"))
    prev = s.stats()["H_top"]
    for _ in range(400):
        s.step(1)
        rho = s.pops().sum(0)
        st = s.stats()
        assert np.nonzero(rho.any(1))[0].max() <= max(st["H_top"], prev)
        prev = st["H_top"]
    assert st["H_top"] > 25
