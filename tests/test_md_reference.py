"""Pins of the host MD reference (tests/md_reference.py) against facts that do not come
from it: the published Philox4x32-10 known answers, the normal distribution, the WCA
potential it differentiates, and the exact solutions the BAOAB splitting approaches."""
import numpy as np
import pytest

from tests import md_reference as R


def test_philox4x32_known_answers():
    """Known-answer vectors of Philox4x32-10 published with Random123 (Salmon et al.)."""
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in cases:
        got = R.philox4x32_10(np.array([ctr]), key)[0]
        assert tuple(int(x) for x in got) == want


def test_thermostat_normals_are_standard_normal():
    scipy_stats = pytest.importorskip("scipy.stats")
    xi = R.thermostat_normals(200000, step=3, seed=0x123456789ABC)
    assert abs(xi.mean()) < 0.01
    assert xi.var() == pytest.approx(1.0, abs=0.01)
    for d in range(3):
        assert scipy_stats.kstest(xi[:, d], "norm").pvalue > 1e-3
    c = np.corrcoef(xi.T)
    assert np.abs(c - np.eye(3)).max() < 0.01
    # another step and another key give other numbers
    assert not np.allclose(xi[:10], R.thermostat_normals(10, step=4, seed=0x123456789ABC))
    assert not np.allclose(xi[:10], R.thermostat_normals(10, step=3, seed=7))


def test_wca_wall_is_minus_the_derivative_of_the_shifted_lj_potential():
    sigma, eps = 0.25, 1.3
    U = lambda d: np.where(d < 2 ** (1 / 6) * sigma, 4 * eps * ((sigma / d) ** 12 - (sigma / d) ** 6) + eps, 0.0)
    d = np.linspace(0.13, 0.3, 40)
    h = 1e-7
    fd = -(U(d + h) - U(d - h)) / (2 * h)
    inside = d < 2 ** (1 / 6) * sigma - 2 * h
    np.testing.assert_allclose(R.wca_wall(d, sigma, eps)[inside], fd[inside], rtol=1e-6)
    assert R.wca_wall(np.array([sigma]), sigma, eps)[0] == pytest.approx(24 * eps / sigma)
    assert R.wca_wall(np.array([2 ** (1 / 6) * sigma * 1.0001]), sigma, eps)[0] == 0.0
    # the cap: no closer than sigma / 2
    assert R.wca_wall(np.array([0.01]), sigma, eps)[0] == R.wca_wall(np.array([0.5 * sigma]), sigma, eps)[0]
    # both walls push into the slab
    H = 3.0
    assert R.wall_force_z(np.array([0.2]), H, sigma, eps)[0] > 0
    assert R.wall_force_z(np.array([H - 0.2]), H, sigma, eps)[0] < 0


def test_baoab_without_friction_follows_the_harmonic_oscillator():
    """gamma = 0, kT = 0: BAOAB is velocity Verlet, second order in dt."""
    k, m, T = 2.0, 1.5, 3.0
    w = np.sqrt(k / m)
    errs = []
    for dt in (0.02, 0.01):
        x = np.array([[0.0, 0.0, 1.0]])
        v = np.zeros((1, 3))
        F = lambda y: -k * np.array([[0.0, 0.0, y[0, 2] - 0.0]])
        for _ in range(int(round(T / dt))):
            x1, _ = R.baoab_step(x, v, F(x), np.zeros((1, 3)), dt=dt, gamma=0.0, kT=0.0, mass=m, H=10.0, Lx=5.0,
                                 Ly=5.0)
            x, v = R.baoab_step(x, v, F(x), F(x1), dt=dt, gamma=0.0, kT=0.0, mass=m, H=10.0, Lx=5.0, Ly=5.0)
        errs.append(abs(x[0, 2] - np.cos(w * T)))
    assert errs[1] < 1e-3
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.15)


def test_baoab_ornstein_uhlenbeck_part_reaches_kT():
    """No force: the O step alone gives v ~ N(0, (1 - c1^2 n) kT/m) after n steps from rest."""
    N, dt, gamma, kT, m = 100000, 0.01, 2.0, 1.7, 1.3
    x = np.zeros((N, 3)) + 1.0
    v = np.zeros((N, 3))
    zero = np.zeros((N, 3))
    for step in range(3):
        xi = R.thermostat_normals(N, step, seed=11)
        x, v = R.baoab_step(x, v, zero, zero, dt=dt, gamma=gamma, kT=kT, mass=m, H=10.0, Lx=5.0, Ly=5.0, xi=xi)
    c1 = np.exp(-gamma * dt)
    assert v.var() == pytest.approx((1 - c1 ** 6) * kT / m, rel=0.01)
