"""Pins for the oracle's triangular D2Q7 lattice (the paper's lattice, Sec. II)
against what the geometry and the mathematics fix.

* streaming: with tau -> infinity one step moves a population pulse by its
  lattice vector e_q = (cos, sin)((q - 1) pi / 3) in physical coordinates
  (node (x, y) sits at (x + (y & 1) / 2, y sqrt(3) / 2)), from even and odd
  rows, with periodic wrap; half-way bounce-back at both walls;
* Eq. 3 with 4, 8, 2 and weights 1/2, 1/12: exact mass conservation of a
  flowing lattice; the total momentum decays by exactly (1 - mu/tau) per step
  (sum_i f^SS_i e_i = rho u* needs c_s^2 = 1/4); shear waves along either
  axis decay at nu = (tau - 1/2)/4 (the textbook D2Q7 viscosity, not in the
  paper), which also pins the isotropy of the viscous term;
* Eq. 4 on seven uniforms: zero sum, var(eta_i) = (2/7) sigma^2 (4 sigma^2 x
  (1 - 1/7) / 12), corr(eta_i, eta_j) = -1/6, 18-bit resolution;
* divisions: three opposite pairs, uniform, no momentum added;
* the two-step reversal of an isolated sub-threshold node.
"""
import math

import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2303_02210_gb300 import workloads as wl

S3 = math.sqrt(3.0) / 2.0
E7 = np.array([[0.0, 0.0]] + [[math.cos(k * math.pi / 3), math.sin(k * math.pi / 3)] for k in range(6)])
W7 = np.array([0.5] + [1 / 12] * 6)
OPP7 = [0, 4, 5, 6, 1, 2, 3]


def periodic(**kw):
    p = wl.base_params(front_kind="full", y_periodic=1, growth_mode="none", sigma=0.0,
                       wall_mode="fixed", lattice="d2q7")
    p.update(kw)
    return p


def equilibrium7(rho, ux, uy):
    """Second-order D2Q7 equilibrium (c_s^2 = 1/4), to set up initial states."""
    eu = E7[:, 0, None, None] * ux + E7[:, 1, None, None] * uy
    uu = ux * ux + uy * uy
    return W7[:, None, None] * rho * (1 + 4 * eu + 8 * eu * eu - 2 * uu)


def position(x, y):
    return np.array([x + 0.5 * (y & 1), y * S3])


def total_mass(f):
    return math.fsum(np.asarray(f).ravel())


def total_momentum(f):
    f = np.asarray(f)
    return np.array([math.fsum((f * E7[:, 0, None, None]).ravel()),
                     math.fsum((f * E7[:, 1, None, None]).ravel())])


@pytest.mark.parametrize("q", range(1, 7))
def test_ballistic_streaming_moves_by_the_lattice_vector(q):
    W, H = 7, 6
    s = OracleSim(periodic(width=W, height=H, tau=1e12, rho_c=0.0))
    assert s.Q == 7
    for (x0, y0) in ((0, 0), (3, 1), (W - 1, H - 1), (2, 4), (5, 3)):
        f = np.zeros((7, H, W))
        f[:, :, :] = W7[:, None, None]
        f[q, y0, x0] += 0.25
        s.set_pops(f)
        s.step(1)
        g = s.pops() - W7[:, None, None]
        (y1, x1), = np.argwhere(np.abs(g[q]) > 0.1)
        assert abs(g[q, y1, x1] - 0.25) < 1e-9
        g[q, y1, x1] = 0.0
        assert np.abs(g).max() < 1e-9
        d = position(x1, y1) - position(x0, y0)
        d[0] = (d[0] + W / 2) % W - W / 2          # periodic in x
        d[1] = (d[1] + H * S3 / 2) % (H * S3) - H * S3 / 2  # and in y
        assert np.allclose(d, E7[q], atol=1e-12), (q, x0, y0, d)


@pytest.mark.parametrize("q", [2, 3, 5, 6])
def test_halfway_bounce_back_walls(q):
    """A pulse heading into the rear (q = 5, 6) or top (q = 2, 3) wall comes
    back in the opposite direction at the node it left."""
    W, H = 6, 8
    p = wl.base_params(width=W, height=H, front_kind="full", growth_mode="none", sigma=0.0,
                       wall_mode="fixed", tau=1e12, rho_c=0.0, lattice="d2q7")
    s = OracleSim(p)
    y0 = H - 1 if q in (2, 3) else 0
    for x0 in (0, 3):
        f = np.zeros((7, H, W))
        f[:, :, :] = W7[:, None, None]
        f[q, y0, x0] += 0.25
        s.set_pops(f)
        s.step(1)
        g = s.pops() - W7[:, None, None]
        assert abs(g[OPP7[q], y0, x0] - 0.25) < 1e-9
        g[OPP7[q], y0, x0] = 0.0
        assert np.abs(g).max() < 1e-9


def test_mass_conserved_on_a_flowing_lattice():
    W, H = 24, 20
    s = OracleSim(periodic(width=W, height=H, tau=0.7, mu=0.01))
    y, x = np.mgrid[0:H, 0:W]
    f0 = equilibrium7(1.0 + 0.05 * np.cos(2 * np.pi * (x + y) / W), 0.08 * np.sin(2 * np.pi * y / H),
                      0.06 * np.cos(2 * np.pi * x / W))
    s.set_pops(f0)
    m0 = total_mass(s.pops())
    s.step(300)
    assert abs(total_mass(s.pops()) - m0) <= 1e-12 * m0


def test_momentum_decays_by_friction_factor():
    W, H, tau, mu = 16, 12, 0.8, 0.01
    s = OracleSim(periodic(width=W, height=H, tau=tau, mu=mu))
    rng = np.random.default_rng(0)
    s.set_pops(equilibrium7(1 + 0.01 * rng.standard_normal((H, W)), 0.02 * rng.standard_normal((H, W)),
                            0.02 * rng.standard_normal((H, W))))
    j0 = total_momentum(s.pops())
    for t in (1, 10, 50):
        s.step(t - s.stats()["step"])
        assert np.allclose(total_momentum(s.pops()), j0 * (1 - mu / tau) ** t, rtol=1e-10, atol=0)


def test_rest_state_is_stationary():
    s = OracleSim(periodic(width=10, height=8))
    f0 = s.pops()
    s.step(100)
    assert np.abs(s.pops() - f0).max() < 1e-14


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("tau", [0.8, 1.0])
def test_shear_wave_decay_matches_d2q7_viscosity(tau, axis):
    """u_x = U sin(k y) (rows 128 x sqrt(3)/2 apart) or u_y = U sin(k x)
    decays as exp(-nu k^2 t) (1 - mu/tau)^t with nu = (tau - 1/2)/4; 1% on
    the log-decay."""
    U, mu, T = 1e-3, 0.001, 1000
    if axis == "x":
        W, H = 4, 128
        k = 2 * np.pi / (H * S3)
    else:
        W, H = 128, 4
        k = 2 * np.pi / W
    s = OracleSim(periodic(width=W, height=H, tau=tau, mu=mu))
    yy, xx = np.mgrid[0:H, 0:W]
    px, py = xx + 0.5 * (yy & 1), yy * S3
    if axis == "x":
        wave = np.sin(k * py)
        f0 = equilibrium7(np.ones((H, W)), U * wave, np.zeros((H, W)))
    else:
        wave = np.sin(k * px)
        f0 = equilibrium7(np.ones((H, W)), np.zeros((H, W)), U * wave)
    s.set_pops(f0)

    def amp():
        _, ux, uy = s.fields()
        u = ux if axis == "x" else uy
        return np.sum(u * wave) / np.sum(wave * wave)

    a0 = amp()
    s.step(T)
    nu = (tau - 0.5) / 4.0
    pred = -nu * k * k * T + T * math.log(1 - mu / tau)
    assert abs(math.log(amp() / a0) / pred - 1) < 0.01


def test_noise_statistics_for_seven_directions():
    sigma = 1e-3
    s = OracleSim(periodic(width=64, height=64, sigma=sigma))
    f0 = s.pops()
    s.step(1)
    eta = (s.pops() - f0).reshape(7, -1)
    assert np.abs(eta.sum(0)).max() < 1e-15
    var = eta.var(axis=1)
    assert np.all(np.abs(var / (2 / 7 * sigma ** 2) - 1) < 0.06)
    c = np.corrcoef(eta)
    off = c[~np.eye(7, dtype=bool)]
    assert np.all(np.abs(off + 1 / 6) < 0.05)
    assert np.abs(eta).max() <= 12 / 7 * sigma * (1 + 1e-12)


def test_noise_uniforms_have_eighteen_bit_resolution():
    sigma = 2.0 ** -6
    s = OracleSim(periodic(width=64, height=64, sigma=sigma))
    f0 = s.pops()
    s.step(1)
    eta = (s.pops() - f0).reshape(7, -1)
    d = (eta[1:] - eta[0]) * (2.0 ** 18) / (2.0 * sigma)
    assert np.abs(d - np.rint(d)).max() < 1e-4
    assert np.abs(d).max() < 2 ** 18
    assert np.abs(d).max() > 2 ** 18 * 0.99
    odd = np.mod(np.rint(d), 2).astype(bool).mean()
    assert 0.47 < odd < 0.53


def test_divisions_use_three_opposite_pairs_uniformly_and_add_no_momentum():
    W, H, tau, mu = 16, 12, 0.8, 0.01
    s = OracleSim(periodic(width=W, height=H, tau=tau, mu=mu, growth_mode="bulk", growth_rate=5e-3))
    rng = np.random.default_rng(1)
    s.set_pops(equilibrium7(1 + 0.01 * rng.standard_normal((H, W)), 0.02 * rng.standard_normal((H, W)),
                            0.02 * rng.standard_normal((H, W))))
    j0 = total_momentum(s.pops())
    counts = np.zeros(3)
    for _ in range(40):
        s.step(1)
        _, pair, cnt = s.last_events()
        assert pair.max(initial=0) <= 2
        np.add.at(counts, pair, cnt)
    assert s.stats()["div_total"] > 100
    assert np.allclose(total_momentum(s.pops()), j0 * (1 - mu / tau) ** 40, rtol=1e-10, atol=0)
    chi2 = ((counts - counts.mean()) ** 2 / counts.mean()).sum()
    assert chi2 < 13.8  # 2 degrees of freedom, p = 0.001


def test_isolated_subthreshold_node_reverses_exactly():
    """Sec. II two-step bounce-back: a node below rho_c with empty neighbours
    reverses its populations every step; its mass stays put and every other
    step the state returns exactly."""
    W, H = 9, 8
    p = wl.base_params(width=W, height=H, front_kind="full", growth_mode="none", sigma=0.0,
                       y_periodic=1, wall_mode="fixed", rho_c=0.5, lattice="d2q7")
    s = OracleSim(p)
    f = np.zeros((7, H, W))
    f[:, 3, 4] = [0.05, 0.03, 0.01, 0.04, 0.02, 0.06, 0.07]
    s.set_pops(f)
    for k in range(1, 7):
        s.step(1)
        g = s.pops()
        rho = g.sum(0)
        assert abs(total_mass(g) - f.sum()) < 1e-15
        assert not s.mask().any()
        if k % 2 == 0:
            assert np.array_equal(g, f)
