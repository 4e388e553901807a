"""FP64 background cosmology for the oracle (TEST INFRASTRUCTURE ONLY).

Units: H0 = 1, distances in Mpc/h, c/H0 = 2997.92458 Mpc/h.  Flat LCDM without
radiation, E(a) = H/H0 = sqrt(Om a^-3 + 1 - Om) (Appendix A writes E for H^2/H0^2
and integrates E^-1/2; the two readings agree).

Time factors follow the FastPM scheme the paper builds on (Sec. 3: "kick and
drift ... enforcing correct linear displacement in each step"):
    momentum p = a^3 E dx/da,  dp/da = F / (a^2 E),  F = -(3/2) Om grad(phi),
    lap(phi) = delta;
    g_p(a) = a^3 E dD1/da,  g_f(a) = a^2 E dg_p/da.
A drift over [a_i, a_j] with momentum taken at a_r moves x by p dD1 / g_p(a_r);
a kick changes p by F(a_r) dg_p / g_f(a_r).  Both are exact for the linear
growing mode.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import quad, solve_ivp
from scipy.interpolate import CubicSpline

C_OVER_H0 = 2997.92458  # Mpc/h


class Cosmology:
    """Flat LCDM background, linear growth (D1, D2), comoving distance, EH P(k).

    Parameters are those of the paper's Table 1 (Omega_m, sigma_8) plus the
    Eisenstein-Hu inputs (h, n_s, Omega_b, T_cmb) that Appendix A relies on.
    """

    def __init__(self, omega_m=0.3089, sigma8=0.8159, h=0.6774, n_s=0.9667,
                 omega_b=0.0486, t_cmb=2.7255, a_min=0.02):
        self.omega_m = float(omega_m)
        self.sigma8 = float(sigma8)
        self.h = float(h)
        self.n_s = float(n_s)
        self.omega_b = float(omega_b)
        self.t_cmb = float(t_cmb)
        self.a_min = float(a_min)
        self._solve_growth()
        self._solve_distance()
        self._pk_norm = None

    # ------------------------------------------------------------------ E(a)
    def E(self, a):
        a = np.asarray(a, dtype=np.float64)
        return np.sqrt(self.omega_m * a ** -3 + (1.0 - self.omega_m))

    def dlnE_da(self, a):
        a = np.asarray(a, dtype=np.float64)
        return -1.5 * self.omega_m * a ** -4 / self.E(a) ** 2

    # ------------------------------------------------------------- growth ODE
    def _growth_rhs(self, a, y):
        """Linear growth in the scale factor a.

        D'' + (3/a + E'/E) D' - (3/2) Om / (a^5 E^2) D = 0 for the first order,
        with source -(3/2) Om / (a^5 E^2) D1^2 for the second order D2.
        """
        d1, d1p, d2, d2p = y
        coef = 3.0 / a + self.dlnE_da(a)
        src = 1.5 * self.omega_m / (a ** 5 * self.E(a) ** 2)
        return [d1p, -coef * d1p + src * d1,
                d2p, -coef * d2p + src * d2 - src * d1 * d1]

    def _solve_growth(self):
        a0 = 1e-5  # matter domination: growing modes D1 = a, D2 = -3/7 a^2
        y0 = [a0, 1.0, -3.0 / 7.0 * a0 * a0, -6.0 / 7.0 * a0]
        sol = solve_ivp(self._growth_rhs, (a0, 1.0), y0, method="DOP853",
                        rtol=1e-12, atol=1e-300, dense_output=True)
        assert sol.success
        self._gsol = sol.sol
        self._d1_today = float(sol.sol(1.0)[0])

    def _growth_state(self, a):
        a = np.asarray(a, dtype=np.float64)
        y = self._gsol(a.ravel())
        n = self._d1_today
        return (y[0].reshape(a.shape) / n, y[1].reshape(a.shape) / n,
                y[2].reshape(a.shape) / n ** 2, y[3].reshape(a.shape) / n ** 2)

    def D1(self, a):
        """First-order growth factor, growing mode, D1(a=1) = 1."""
        return self._growth_state(a)[0]

    def D2(self, a):
        """Second-order growth factor, D2 -> -(3/7) D1^2 at early times."""
        return self._growth_state(a)[2]

    def gp(self, a):
        """g_p(a) = a^3 E dD1/da."""
        a = np.asarray(a, dtype=np.float64)
        return a ** 3 * self.E(a) * self._growth_state(a)[1]

    def gp2(self, a):
        """Second-order counterpart a^3 E dD2/da (2LPT momentum)."""
        a = np.asarray(a, dtype=np.float64)
        return a ** 3 * self.E(a) * self._growth_state(a)[3]

    def gf(self, a):
        """g_f(a) = a^2 E dg_p/da, with d2D1/da2 taken from the growth ODE."""
        a = np.asarray(a, dtype=np.float64)
        d1, d1p, _, _ = self._growth_state(a)
        e = self.E(a)
        ep = self.dlnE_da(a) * e
        d1pp = -(3.0 / a + self.dlnE_da(a)) * d1p + 1.5 * self.omega_m / (a ** 5 * e ** 2) * d1
        dgp = 3 * a ** 2 * e * d1p + a ** 3 * ep * d1p + a ** 3 * e * d1pp
        return a ** 2 * e * dgp

    # ------------------------------------------------------ comoving distance
    def _solve_distance(self):
        """chi(a) = (c/H0) int_a^1 da' / (a'^2 E(a')) (Appendix A, in a)."""
        def rhs(a, y):
            return [-C_OVER_H0 / (a * a * self.E(a))]
        sol = solve_ivp(rhs, (1.0, self.a_min), [0.0], method="DOP853",
                        rtol=1e-12, atol=1e-12, dense_output=True)
        assert sol.success
        self._chisol = sol.sol
        ag = np.linspace(self.a_min, 1.0, 40001)
        cg = self._chisol(ag)[0]
        # a(chi): chi decreases with a; spline on increasing chi
        self._a_of_chi = CubicSpline(cg[::-1], ag[::-1])

    def chi(self, a):
        """Comoving distance to scale factor a, Mpc/h."""
        a = np.asarray(a, dtype=np.float64)
        return self._chisol(a.ravel())[0].reshape(a.shape)

    def chi_z(self, z):
        return self.chi(1.0 / (1.0 + np.asarray(z, dtype=np.float64)))

    def a_of_chi(self, chi):
        """Inverse of chi(a) (cubic spline on a 4e4-point grid)."""
        return self._a_of_chi(np.asarray(chi, dtype=np.float64))

    # ------------------------------------------------- Eisenstein-Hu transfer
    def eh_transfer(self, k_hmpc):
        """Eisenstein & Hu (1998) transfer function with baryon wiggles.

        Appendix A: the differentiable variant uses the EH transfer function
        including BAO.  k in h/Mpc; the fitting formulae are in Mpc^-1.
        """
        k = np.asarray(k_hmpc, dtype=np.float64) * self.h  # 1/Mpc
        om = self.omega_m * self.h ** 2
        ob = self.omega_b * self.h ** 2
        fb = self.omega_b / self.omega_m
        fc = 1.0 - fb
        th = self.t_cmb / 2.7
        z_eq = 2.50e4 * om * th ** -4
        k_eq = 7.46e-2 * om * th ** -2
        b1d = 0.313 * om ** -0.419 * (1.0 + 0.607 * om ** 0.674)
        b2d = 0.238 * om ** 0.223
        z_d = 1291.0 * om ** 0.251 / (1.0 + 0.659 * om ** 0.828) * (1.0 + b1d * ob ** b2d)
        R = lambda z: 31.5 * ob * th ** -4 * (z / 1.0e3) ** -1  # noqa: E731
        r_eq, r_d = R(z_eq), R(z_d)
        s = (2.0 / (3.0 * k_eq) * np.sqrt(6.0 / r_eq)
             * np.log((np.sqrt(1.0 + r_d) + np.sqrt(r_d + r_eq)) / (1.0 + np.sqrt(r_eq))))
        k_silk = 1.6 * ob ** 0.52 * om ** 0.73 * (1.0 + (10.4 * om) ** -0.95)
        q = k / (13.41 * k_eq)

        def t0(alpha, beta):
            lg = np.log(np.e + 1.8 * beta * q)
            c = 14.2 / alpha + 386.0 / (1.0 + 69.9 * q ** 1.08)
            return lg / (lg + c * q * q)

        a1 = (46.9 * om) ** 0.670 * (1.0 + (32.1 * om) ** -0.532)
        a2 = (12.0 * om) ** 0.424 * (1.0 + (45.0 * om) ** -0.582)
        alpha_c = a1 ** (-fb) * a2 ** (-fb ** 3)
        b1c = 0.944 / (1.0 + (458.0 * om) ** -0.708)
        b2c = (0.395 * om) ** -0.0266
        beta_c = 1.0 / (1.0 + b1c * (fc ** b2c - 1.0))
        ks = k * s
        f = 1.0 / (1.0 + (ks / 5.4) ** 4)
        t_c = f * t0(1.0, beta_c) + (1.0 - f) * t0(alpha_c, beta_c)

        y = (1.0 + z_eq) / (1.0 + z_d)
        sq = np.sqrt(1.0 + y)
        G = y * (-6.0 * sq + (2.0 + 3.0 * y) * np.log((sq + 1.0) / (sq - 1.0)))
        alpha_b = 2.07 * k_eq * s * (1.0 + r_d) ** -0.75 * G
        beta_node = 8.41 * om ** 0.435
        beta_b = 0.5 + fb + (3.0 - 2.0 * fb) * np.sqrt((17.2 * om) ** 2 + 1.0)
        with np.errstate(divide="ignore", invalid="ignore"):
            s_tilde = s / (1.0 + (beta_node / ks) ** 3) ** (1.0 / 3.0)
            x = k * s_tilde
            j0 = np.where(x > 0, np.sin(x) / np.where(x > 0, x, 1.0), 1.0)
            t_b = (t0(1.0, 1.0) / (1.0 + (ks / 5.2) ** 2)
                   + alpha_b / (1.0 + (beta_b / ks) ** 3) * np.exp(-(k / k_silk) ** 1.4)) * j0
        t_b = np.where(k > 0, t_b, 1.0)
        return fb * t_b + fc * t_c

    def eh_sound_horizon(self):
        """Sound horizon s (Mpc) of the full EH formula (used by a pin)."""
        om = self.omega_m * self.h ** 2
        ob = self.omega_b * self.h ** 2
        th = self.t_cmb / 2.7
        z_eq = 2.50e4 * om * th ** -4
        k_eq = 7.46e-2 * om * th ** -2
        b1d = 0.313 * om ** -0.419 * (1.0 + 0.607 * om ** 0.674)
        b2d = 0.238 * om ** 0.223
        z_d = 1291.0 * om ** 0.251 / (1.0 + 0.659 * om ** 0.828) * (1.0 + b1d * ob ** b2d)
        r_eq = 31.5 * ob * th ** -4 * (z_eq / 1e3) ** -1
        r_d = 31.5 * ob * th ** -4 * (z_d / 1e3) ** -1
        return (2.0 / (3.0 * k_eq) * np.sqrt(6.0 / r_eq)
                * np.log((np.sqrt(1.0 + r_d) + np.sqrt(r_d + r_eq)) / (1.0 + np.sqrt(r_eq))))

    # --------------------------------------------------------- linear power
    @staticmethod
    def tophat(x):
        x = np.asarray(x, dtype=np.float64)
        return 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3

    def _sigma2_unnorm(self, R=8.0):
        f = lambda lnk: (np.exp(lnk) ** (3.0 + self.n_s)  # noqa: E731
                         * self.eh_transfer(np.exp(lnk)) ** 2
                         * self.tophat(np.exp(lnk) * R) ** 2 / (2.0 * np.pi ** 2))
        val, _ = quad(f, np.log(1e-6), np.log(1e3), limit=2000, epsabs=0, epsrel=1e-11)
        return val

    def pk_lin(self, k):
        """Linear P(k) at z=0, (Mpc/h)^3, normalised to sigma_8 (top-hat R=8 Mpc/h)."""
        if self._pk_norm is None:
            self._pk_norm = self.sigma8 ** 2 / self._sigma2_unnorm(8.0)
        k = np.asarray(k, dtype=np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            p = self._pk_norm * k ** self.n_s * self.eh_transfer(k) ** 2
        return np.where(k > 0, p, 0.0)

    def sigma_R(self, R):
        """sigma(R) of the normalised linear P(k) (top-hat window)."""
        f = lambda lnk: (np.exp(lnk) ** 3 * self.pk_lin(np.exp(lnk))  # noqa: E731
                         * self.tophat(np.exp(lnk) * R) ** 2 / (2.0 * np.pi ** 2))
        val, _ = quad(f, np.log(1e-6), np.log(1e3), limit=2000, epsabs=0, epsrel=1e-11)
        return np.sqrt(val)


def time_grid(a_init: float, nsteps: int):
    """Steps linear in a from a_init to 1 (a_i, i = 0..nsteps) and midpoints."""
    a = a_init + (1.0 - a_init) * np.arange(nsteps + 1) / nsteps
    return a, 0.5 * (a[:-1] + a[1:])
