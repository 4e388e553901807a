"""Pins of the oracle's background cosmology against closed forms."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle.cosmology import C_OVER_H0, Cosmology, time_grid


@pytest.fixture(scope="module")
def eds():
    return Cosmology(omega_m=1.0)


@pytest.fixture(scope="module")
def lcdm():
    return Cosmology(omega_m=0.3089)


def test_eds_growth_closed_forms(eds):
    a = np.array([0.05, 0.1, 0.33, 0.7, 1.0])
    assert np.allclose(eds.D1(a), a, rtol=1e-9)
    assert np.allclose(eds.D2(a), -3.0 / 7.0 * a ** 2, rtol=1e-9)
    assert np.allclose(eds.gp(a), a ** 1.5, rtol=1e-9)
    assert np.allclose(eds.gf(a), 1.5 * a, rtol=1e-9)


def test_lcdm_growth_heath_integral(lcdm):
    """D1 proportional to E(a) int_0^a da' / (a' E(a'))^3 (LCDM, no radiation)."""
    def heath(a):
        v, _ = quad(lambda x: 1.0 / (x * lcdm.E(x)) ** 3, 0.0, a, epsabs=0, epsrel=1e-12, limit=200)
        return lcdm.E(a) * v
    a = np.array([0.1, 0.3, 0.6, 0.9])
    ref = np.array([heath(x) for x in a]) / heath(1.0)
    assert np.allclose(lcdm.D1(a), ref, rtol=1e-8)


def test_growing_mode_identity_gf(lcdm):
    """For the growing mode, a^2 E d(a^3 E D1')/da = (3/2) Om D1."""
    a = np.linspace(0.1, 1.0, 7)
    assert np.allclose(lcdm.gf(a), 1.5 * lcdm.omega_m * lcdm.D1(a), rtol=1e-9)


def test_d2_early_limit(lcdm):
    a = np.array([0.02, 0.05])
    assert np.allclose(lcdm.D2(a) / lcdm.D1(a) ** 2, -3.0 / 7.0, rtol=1e-3)


def test_chi_eds_closed_form(eds):
    z = np.array([0.1, 0.5, 1.0, 2.0, 9.0])
    expect = 2 * C_OVER_H0 * (1 - 1 / np.sqrt(1 + z))
    assert np.allclose(eds.chi_z(z), expect, rtol=1e-10)


def test_chi_low_z_expansion(lcdm):
    """chi = (c/H0) [z - (1 + q0) z^2 / 2 + O(z^3)], q0 = 3 Om / 2 - 1."""
    z = 1e-3
    q0 = 1.5 * lcdm.omega_m - 1.0
    expect = C_OVER_H0 * (z - (1 + q0) * z * z / 2)
    assert abs(lcdm.chi_z(np.array([z]))[0] - expect) < C_OVER_H0 * 2 * z ** 3


def test_a_of_chi_roundtrip(lcdm):
    a = np.linspace(0.05, 1.0, 37)
    assert np.allclose(lcdm.a_of_chi(lcdm.chi(a)), a, rtol=1e-10, atol=1e-12)


def test_eh_limits(lcdm):
    assert abs(lcdm.eh_transfer(1e-6) - 1.0) < 1e-5
    t = lcdm.eh_transfer(np.logspace(-3, 1, 50))
    assert np.all(np.diff(t[t > 0]) < 1e-3)        # decreasing up to BAO wiggles
    assert np.all(t > 0) and np.all(t <= 1.0 + 1e-9)


def test_eh_sound_horizon_vs_fit(lcdm):
    """EH98's approximate sound horizon s ~ 44.5 ln(9.83/om)/sqrt(1+10 ob^{3/4}) Mpc
    (a separate fit of the same quantity) agrees with the full formula to 2%."""
    om = lcdm.omega_m * lcdm.h ** 2
    ob = lcdm.omega_b * lcdm.h ** 2
    fit = 44.5 * np.log(9.83 / om) / np.sqrt(1.0 + 10.0 * ob ** 0.75)
    assert abs(lcdm.eh_sound_horizon() / fit - 1.0) < 0.02


def test_eh_no_baryon_limit_shape():
    """Omega_b -> 0 removes the wiggles: T reduces to the pure-CDM T0(k,1,1)-type
    form, smooth (no oscillation in the log-derivative)."""
    c = Cosmology(omega_m=0.3, omega_b=1e-6)
    k = np.logspace(-2, 0, 400)
    t = c.eh_transfer(k)
    d = np.diff(np.log(t)) / np.diff(np.log(k))
    assert np.all(np.diff(d) < 1e-3)   # monotone steepening, no BAO wiggle


def test_sigma8_normalisation(lcdm):
    assert np.isclose(lcdm.sigma_R(8.0), lcdm.sigma8, rtol=1e-6)


def test_time_grid():
    a, ah = time_grid(0.1, 10)
    assert a[0] == 0.1 and a[-1] == 1.0 and len(a) == 11
    assert np.allclose(ah, 0.5 * (a[1:] + a[:-1]))
