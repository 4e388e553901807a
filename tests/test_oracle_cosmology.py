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


def eh98_no_wiggle(k_hmpc, omega_m, omega_b, h, t_cmb):
    """EH98's separately published zero-baryon ("no-wiggle") transfer fit: the
    baryons only through an effective shape parameter,
      s = 44.5 ln(9.83 / om) / sqrt(1 + 10 ob^(3/4)) Mpc,
      alpha_G = 1 - 0.328 ln(431 om) f_b + 0.38 ln(22.3 om) f_b^2,
      Gamma = Omega_m h [alpha_G + (1 - alpha_G) / (1 + (0.43 k s)^4)],
      q = k Theta^2 / Gamma  (k in h/Mpc),
      T = L / (L + C q^2),  L = ln(2 e + 1.8 q),  C = 14.2 + 731 / (1 + 62.5 q).
    Its constants differ from those of the full formula's T0 (e vs 2e, 386 and
    69.9 q^1.08 vs 731 and 62.5 q), so agreement is an independent check."""
    th = t_cmb / 2.7
    om, ob, fb = omega_m * h * h, omega_b * h * h, omega_b / omega_m
    s = 44.5 * np.log(9.83 / om) / np.sqrt(1.0 + 10.0 * ob ** 0.75)
    ag = 1.0 - 0.328 * np.log(431.0 * om) * fb + 0.38 * np.log(22.3 * om) * fb ** 2
    gam = omega_m * h * (ag + (1.0 - ag) / (1.0 + (0.43 * k_hmpc * h * s) ** 4))
    q = k_hmpc * th ** 2 / gam
    lg = np.log(2.0 * np.e + 1.8 * q)
    return lg / (lg + (14.2 + 731.0 / (1.0 + 62.5 * q)) * q * q)


@pytest.mark.parametrize("om,h", [(0.3089, 0.6774), (0.2, 0.5), (0.5, 0.7), (1.0, 0.7)])
def test_eh_zero_baryon_limit_vs_zero_baryon_fit(om, h):
    """Omega_b -> 0: the full EH formula reduces to its CDM piece T0(k, 1, 1),
    which must follow EH98's zero-baryon fit within 1.5% from k = 1e-3 to 20 h/Mpc
    (the two fits differ by at most 0.85%).  A 10% change of any constant of T0
    (e, 1.8, 14.2, 386, 69.9, 1.08), of q = k / (13.41 k_eq), of k_eq or of Theta
    breaks this."""
    k = np.logspace(-3, 1.3, 400)
    c = Cosmology(omega_m=om, omega_b=1e-7, h=h)
    r = c.eh_transfer(k) / eh98_no_wiggle(k, om, 1e-7, h, c.t_cmb)
    assert np.max(np.abs(r - 1.0)) < 0.015


def test_eh_baryon_suppression_vs_no_wiggle_fit(lcdm):
    """With baryons the full formula oscillates about the no-wiggle fit (BAO):
    averaged over +-0.5 in ln k the ratio stays within 2% of one (1.3% measured)
    and within 5% pointwise; pins the baryon suppression (alpha_c, z_d, R) on
    average, not the wiggle amplitude."""
    k = np.logspace(-3, 1.3, 400)
    r = lcdm.eh_transfer(k) / eh98_no_wiggle(k, lcdm.omega_m, lcdm.omega_b, lcdm.h, lcdm.t_cmb)
    lk = np.log(k)
    smooth = np.array([np.mean(r[np.abs(lk - x) < 0.5]) for x in lk])
    inner = (k > 3e-3) & (k < 5.0)
    assert np.max(np.abs(smooth[inner] - 1.0)) < 0.02
    assert np.max(np.abs(r - 1.0)) < 0.05


def test_tophat_series_and_values():
    """W(x) = 3 (sin x - x cos x) / x^3 = 1 - x^2/10 + x^4/280 - ...;
    W(pi) = 3/pi^2, W(2 pi) = -3/(4 pi^2), W(4.4934...) = 0 (tan x = x)."""
    x = np.array([1e-2, 3e-2, 0.1])
    assert np.allclose(Cosmology.tophat(x), 1 - x ** 2 / 10 + x ** 4 / 280, rtol=0, atol=2e-9)
    assert np.isclose(Cosmology.tophat(np.pi), 3 / np.pi ** 2, rtol=1e-13)
    assert np.isclose(Cosmology.tophat(2 * np.pi), -3 / (4 * np.pi ** 2), rtol=1e-13)
    assert abs(Cosmology.tophat(4.493409457909064)) < 1e-13


class _PowerLaw(Cosmology):
    """T(k) = 1: P(k) proportional to k^n_s (for the closed-form variance)."""

    def eh_transfer(self, k_hmpc):
        return np.ones_like(np.asarray(k_hmpc, dtype=np.float64))


def tophat_power_law_integral(n):
    """I(n) = int_0^inf x^(n+2) W(x)^2 dx for -3 < n < 1 in closed form: with
    (sin x - x cos x)^2 = 1/2 - cos(2x)/2 - x sin 2x + x^2/2 + x^2 cos(2x)/2 and the
    Mellin transforms int x^(s-1) cos 2x dx = Gamma(s) cos(pi s/2) / 2^s,
    int x^(s-1) sin 2x dx = Gamma(s) sin(pi s/2) / 2^s (power terms regularise
    to zero): I = 9 [-C(n-3)/2 - S(n-2) + C(n-1)/2]."""
    from scipy.special import gamma
    C = lambda s: gamma(s) * np.cos(np.pi * s / 2) / 2 ** s  # noqa: E731
    S = lambda s: gamma(s) * np.sin(np.pi * s / 2) / 2 ** s  # noqa: E731
    return 9.0 * (-0.5 * C(n - 3) - S(n - 2) + 0.5 * C(n - 1))


@pytest.mark.parametrize("n,R", [(-1.5, 8.0), (-0.5, 8.0), (-1.5, 2.0)])
def test_sigma_unnormalised_power_law_closed_form(n, R):
    """sigma^2(R) = 1/(2 pi^2) int k^(n+2) W(kR)^2 dk = I(n) / (2 pi^2 R^(n+3))
    for a pure power law: pins the window (a missing factor 3 fails), the
    measure k^3 P dlnk and the 2 pi^2, which the sigma_8 normalisation divides by."""
    c = _PowerLaw(omega_m=0.3, n_s=n)
    expect = tophat_power_law_integral(n) / (2 * np.pi ** 2 * R ** (n + 3))
    assert np.isclose(c._sigma2_unnorm(R), expect, rtol=1e-5)


def test_sigma_white_noise_parseval():
    """n = 0 (white noise): sigma^2 = P / V_R with V_R = 4 pi R^3 / 3, by Parseval
    (the real-space top-hat is 1/V_R inside the sphere), i.e. I(0) = 3 pi / 2."""
    c = _PowerLaw(omega_m=0.3, n_s=0.0)
    R = 8.0
    assert np.isclose(c._sigma2_unnorm(R), 3.0 / (4 * np.pi * R ** 3), rtol=3e-4)
    assert np.isclose(tophat_power_law_integral(1e-7), 1.5 * np.pi, rtol=1e-6)


def test_sigma8_normalisation(lcdm):
    """The normalised spectrum has sigma(8) = sigma_8 (its window and measure are
    pinned above) and sigma(R) / sigma(8) follows from the same P at any R."""
    assert np.isclose(lcdm.sigma_R(8.0), lcdm.sigma8, rtol=1e-6)
    pl = _PowerLaw(omega_m=0.3, n_s=-1.5, sigma8=0.8)
    assert np.isclose(pl.sigma_R(2.0), 0.8 * (2.0 / 8.0) ** (-0.75), rtol=1e-5)


def test_time_grid():
    a, ah = time_grid(0.1, 10)
    assert a[0] == 0.1 and a[-1] == 1.0 and len(a) == 11
    assert np.allclose(ah, 0.5 * (a[1:] + a[:-1]))
