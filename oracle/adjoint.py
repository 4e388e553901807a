"""Reverse-mode derivative (VJP) of the forward model in FP64 (TEST INFRASTRUCTURE ONLY).

Sec. 3: the model is differentiable with respect to the initial Gaussian
modes; Appendix A: also with respect to Omega_m and sigma_8, where the
cosmology-dependent coefficients (LPT initial conditions, kick and drift
factors, lensing geometry) are differentiated by central finite differences
between two cached perturbed cosmologies, and sigma_8 enters linearly through
the initial field.

Every adjoint here is the transpose of the corresponding forward operation of
``oracle.mesh``, ``oracle.lpt``, ``oracle.nbody`` and ``oracle.lightcone``
written out by hand:
* CIC readout r(m, x) has d/dx = cic_readout_grad and d/dm = paint(x, .);
* the spectral operators with odd kernels (i k_j / k^2 ...) are antisymmetric,
  those with even kernels (k_i k_j / k^2) symmetric;
* the shell selection and the map's pixel assignment are piecewise constant
  (no derivative); inside a cell the CIC weights are linear.
Reading: the lensing shell boundaries stay at the central cosmology when the
Omega_m finite difference is taken (selection is not differentiated).
"""
from __future__ import annotations

import numpy as np

from .cosmology import C_OVER_H0, Cosmology
from . import dft
from .lightcone import LensGeometry, apply_rotation, apply_transform, candidate_replicas, replica_transform
from .lpt import linear_modes, lpt_displacements, lpt_state
from .mesh import (cic_paint, cic_readout, cic_readout_grad, force_mesh, gradient_multipliers,
                   particle_mass, pgd_filter, pgd_mesh, wavevectors)
from .nbody import Stepper


# ------------------------------------------------------------- mesh adjoints
def _odd_op(mesh_list, multipliers):
    """sum_c IDFT[m_c DFT(mesh_c)] for real meshes."""
    shape = mesh_list[0].shape
    acc = 0
    for m, mult in zip(mesh_list, multipliers):
        acc = acc + mult * dft.rfftn(m)
    return dft.irfftn(acc, s=shape, axes=(0, 1, 2))


def mesh_force_vjp(x, v, nc, nmesh, box, kernel_meshes, kernel_mults):
    """Transpose of x -> readout(K * paint(x, mass), x) for cotangent v (N, 3).

    kernel_meshes: the three output meshes K_c * rho at x (for the readout
    position gradient); kernel_mults: the three Fourier multipliers m_c of K_c
    (odd: the transpose of K_c is -K_c).
    """
    g = np.zeros_like(x)
    for c in range(3):
        g += v[:, c:c + 1] * cic_readout_grad(kernel_meshes[c], x, box)
    painted = [cic_paint(x, nmesh, box, v[:, c]) for c in range(3)]
    phi = -_odd_op(painted, kernel_mults)
    g += particle_mass(nc, nmesh) * cic_readout_grad(phi, x, box)
    return g


def force_vjp(x, v, nc, nmesh, box, omega_m):
    """Transpose of the PM force at positions x (paint, Poisson + gradient, readout)."""
    rho = cic_paint(x, nmesh, box, particle_mass(nc, nmesh))
    fm = force_mesh(rho - 1.0, box, omega_m)
    mults = [1.5 * omega_m * m for m in gradient_multipliers(nmesh, box)]
    return mesh_force_vjp(x, v, nc, nmesh, box, fm, mults)


def pgd_vjp(x, v, a, nc, nmesh, box, pgd_params):
    """Transpose of the PGD displacement S(x) at positions x."""
    alpha0, mu, k_l, k_s, n_s = pgd_params
    alpha = alpha0 * a ** mu
    rho = cic_paint(x, nmesh, box, particle_mass(nc, nmesh))
    sm = pgd_mesh(rho - 1.0, box, alpha, k_l, k_s, n_s)
    filt = pgd_filter(nmesh, box, k_l, k_s, n_s)
    mults = [alpha * filt * m for m in gradient_multipliers(nmesh, box)]
    return mesh_force_vjp(x, v, nc, nmesh, box, sm, mults)


# ---------------------------------------------------------- lensing adjoint
def project_vjp(geom: LensGeometry, i, x, p, S, lam):
    """Transpose of shell i's projection: (g_x, g_p, g_S) for map cotangent lam.

    Follows LensGeometry.project step by step: rotation/replication r = R x + n L,
    sub-evolution r_c = r + R p dt(|r|) (+ R S), flat-sky angles, CIC on the map
    and the Born weight w_s(chi_c) = K (chi_s - chi_c)/(chi_s chi_c a(chi_c)).
    """
    cosmo, st = geom.cosmo, geom.stepper
    gx, gp, gS = np.zeros_like(x), np.zeros_like(p), np.zeros_like(x)
    if not geom.active(i):
        return gx, gp, gS
    lo, hi = geom.shell(i)
    gp_half = cosmo.gp(st.ah[i])
    margin = 2.0 * geom.box / geom.nmesh
    if geom.sub_evolution:
        dd = float(cosmo.D1(st.a[i + 1]) - cosmo.D1(max(cosmo.a_min, cosmo.a_of_chi(hi))))
        margin += float(np.max(np.abs(p))) * abs(dd) / gp_half * np.sqrt(3)
    if S is not None:
        margin += float(np.max(np.abs(S))) * np.sqrt(3)
    half = 0.5 * geom.fov + geom.dtheta
    K = geom.prefac * geom.vp / geom.dtheta ** 2
    for n in candidate_replicas(lo, hi, geom.box, half, margin):
        tr = replica_transform(n, geom.seed, geom.rotate, geom.nmesh)
        r = apply_transform(x, tr, geom.box, geom.nmesh) + np.asarray(n, dtype=np.float64) * geom.box
        chi = np.linalg.norm(r, axis=1)
        sel = np.nonzero((chi > lo) & (chi <= hi) & (r[:, 2] > 0))[0]
        if sel.size == 0:
            continue
        rs, chis = r[sel], chi[sel]
        pr = apply_rotation(p[sel], tr)
        if geom.sub_evolution:
            ac = cosmo.a_of_chi(chis)
            dt = geom.subevolve_factor(i, ac)
            # d dt / d chi = dD1/da * da/dchi / g_p = [g_p(a)/(a^3 E)] (-a^2 E / c) / g_p(a_half)
            ddt = -cosmo.gp(ac) / (ac * C_OVER_H0) / gp_half
            rc = rs + pr * dt[:, None]
        else:
            dt = ddt = None
            rc = rs.copy()
        if S is not None:
            rc = rc + apply_rotation(S[sel], tr)
        ok = rc[:, 2] > 0
        chic = np.linalg.norm(rc, axis=1)
        ac2 = cosmo.a_of_chi(chic)
        inva = 1.0 / ac2
        dinva = cosmo.E(ac2) / C_OVER_H0            # d(1/a)/dchi
        tx, ty = rc[:, 0] / rc[:, 2], rc[:, 1] / rc[:, 2]
        u = (tx + 0.5 * geom.fov) / geom.dtheta - 0.5
        v = (ty + 0.5 * geom.fov) / geom.dtheta - 0.5
        iu, iv = np.floor(u).astype(np.int64), np.floor(v).astype(np.int64)
        fu, fv = u - iu, v - iv
        g_rc = np.zeros_like(rc)
        for s, cs in enumerate(geom.chi_s):
            if geom.nz[s] is None:
                inside = (chic < cs) & ok
                f = 1.0 / chic - 1.0 / cs                 # (chi_s - chi)/(chi_s chi)
                w = np.where(inside, K * f * inva, 0.0)
                dw = np.where(inside, K * (-inva / chic ** 2 + f * dinva), 0.0)
            else:
                # w = K q(chi) / (chi a): d/dchi = K [(q' chi - q) / chi^2 / a + q / chi d(1/a)/dchi]
                q, dq = geom.source_weight(s, chic)
                w = np.where(ok, K * q / chic * inva, 0.0)
                dw = np.where(ok, K * ((dq * chic - q) / chic ** 2 * inva + q / chic * dinva), 0.0)
            Lw = np.zeros(len(sel))
            Lu = np.zeros(len(sel))
            Lv = np.zeros(len(sel))
            for du in (0, 1):
                for dv in (0, 1):
                    jx, jy = iu + du, iv + dv
                    good = (jx >= 0) & (jx < geom.npix) & (jy >= 0) & (jy < geom.npix)
                    lamv = np.zeros(len(sel))
                    lamv[good] = lam[s][jy[good], jx[good]]
                    wu = fu if du else 1.0 - fu
                    wv = fv if dv else 1.0 - fv
                    Lw += lamv * wu * wv
                    Lu += lamv * (1.0 if du else -1.0) * wv
                    Lv += lamv * wu * (1.0 if dv else -1.0)
            # d/d rc of w * cw: radial part and angular part
            g_rc += (dw * Lw / chic)[:, None] * rc
            gu = w * Lu / geom.dtheta
            gv = w * Lv / geom.dtheta
            g_rc[:, 0] += gu / rc[:, 2]
            g_rc[:, 1] += gv / rc[:, 2]
            g_rc[:, 2] += -(gu * rc[:, 0] + gv * rc[:, 1]) / rc[:, 2] ** 2
        g_rc[~ok] = 0.0
        g_r = g_rc.copy()
        if geom.sub_evolution:
            g_r += (np.sum(g_rc * pr, axis=1) * ddt / chis)[:, None] * rs
        # back to the box frame: transpose of the rotation/flip
        inv = _inverse_rotation(tr)
        np.add.at(gx, sel, apply_rotation(g_r, inv))
        if geom.sub_evolution:
            np.add.at(gp, sel, apply_rotation(g_rc * dt[:, None], inv))
        if S is not None:
            np.add.at(gS, sel, apply_rotation(g_rc, inv))
    return gx, gp, gS


def _inverse_rotation(tr):
    """Transform whose apply_rotation is the transpose of tr's."""
    perm, flips, shift = tr
    iperm = [0, 0, 0]
    iflip = [0, 0, 0]
    for d in range(3):
        iperm[perm[d]] = d
        iflip[perm[d]] = flips[d]
    return tuple(iperm), tuple(iflip), shift


# --------------------------------------------------------------- IC adjoint
def lpt_vjp(lam_psi1, lam_psi2, delta_k, nc, box, cosmo, order):
    """Transpose of noise -> (Psi1, Psi2): returns d/d(noise) on the lattice."""
    shape = (nc, nc, nc)
    kx, ky, kz = wavevectors(nc, box)
    k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    amp = np.sqrt(cosmo.pk_lin(k) * nc ** 3 / box ** 3)
    amp[0, 0, 0] = 0.0
    mult = gradient_multipliers(nc, box)
    # Psi1_j = IDFT[m_j amp DFT(w)], odd -> transpose is minus itself
    acc = 0
    for j in range(3):
        acc = acc - mult[j] * amp * dft.rfftn(lam_psi1[:, j].reshape(shape))
    if order == 2 and lam_psi2 is not None:
        kk = (kx, ky, kz)
        kny = np.pi * nc / box
        odd = [np.where(np.abs(np.abs(q) - kny) < 1e-9 * kny, 0.0, q) for q in kk]
        k2 = kx ** 2 + ky ** 2 + kz ** 2
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = np.where(k2 > 0, 1.0 / k2, 0.0)
        d = {}
        mults = {}
        for a in range(3):
            for b in range(a, 3):
                mab = -(kk[a] * kk[a] if a == b else odd[a] * odd[b]) * inv
                mults[(a, b)] = mab
                d[(a, b)] = dft.irfftn(mab * delta_k, s=shape, axes=(0, 1, 2))
        # Psi2_j = IDFT[-m_j DFT(src)]  ->  lam_src = IDFT[+sum_j m_j DFT(lam_psi2_j)]
        ls = dft.irfftn(sum(mult[j] * dft.rfftn(lam_psi2[:, j].reshape(shape)) for j in range(3)),
                           s=shape, axes=(0, 1, 2))
        lam_d = {(0, 0): ls * (d[(1, 1)] + d[(2, 2)]), (1, 1): ls * (d[(0, 0)] + d[(2, 2)]),
                 (2, 2): ls * (d[(0, 0)] + d[(1, 1)]), (0, 1): -2 * ls * d[(0, 1)],
                 (0, 2): -2 * ls * d[(0, 2)], (1, 2): -2 * ls * d[(1, 2)]}
        for key, lv in lam_d.items():
            acc = acc + mults[key] * amp * dft.rfftn(lv)   # even kernels: symmetric
    return dft.irfftn(acc, s=shape, axes=(0, 1, 2))


# ------------------------------------------------------------ full pipeline
class Trajectory:
    """States of a forward run kept for the reverse sweep."""

    def __init__(self):
        self.x = []      # x(a_i), i = 0..n
        self.p = []      # p(a_{i-1/2}) for i = 0 (p0) .. n
        self.S = []      # PGD displacement at x(a_{i+1}) per shell (or None)


def forward_with_trajectory(sim, noise):
    """Run the oracle forward model, recording every state."""
    tr = Trajectory()
    psi1, psi2 = sim.ic(noise)
    tr.psi1, tr.psi2 = psi1, psi2
    tr.x.append(sim.state.x.copy())
    tr.p.append(sim.state.p.copy())
    for i in range(sim.nsteps):
        sim.step(i)
        tr.x.append(sim.state.x.copy())
        tr.p.append(sim.state.p.copy())
        S = sim.pgd_at(i) if sim.geom.active(i) else None
        tr.S.append(S)
        if sim.geom.active(i):
            inc, _ = sim.geom.project(i, sim.state.x, sim.state.p, S)
            sim.maps += inc
    return sim.kappa_maps(), tr


def _perturbed(sim, domega):
    c = sim.cosmo
    return Cosmology(c.omega_m + domega, c.sigma8, c.h, c.n_s, c.omega_b, c.t_cmb, a_min=c.a_min)


def vjp(sim, noise, lam, h_om=1e-4):
    """(dL/dnoise, dL/dOmega_m, dL/dsigma_8) for dL/dkappa = lam (n_zs, npix, npix).

    Runs the forward model on `sim` (an oracle.sim.Simulation) and then the
    reverse sweep.  Omega_m: central finite differences (step h_om) of every
    cosmology-dependent coefficient, contracted with the adjoint state.
    """
    kappa, tr = forward_with_trajectory(sim, noise)
    nc, M, L = sim.nc, sim.nmesh, sim.box
    st, geom, cosmo = sim.stepper, sim.geom, sim.cosmo
    om = cosmo.omega_m
    n = sim.nsteps
    # perturbed coefficient sets
    cp, cm = _perturbed(sim, h_om), _perturbed(sim, -h_om)
    stp, stm = Stepper(cp, st.a[0], n), Stepper(cm, st.a[0], n)
    dkick = (stp.kick * (om + h_om) - stm.kick * (om - h_om)) / (2 * h_om)   # d(Om * kick)/dOm
    ddrift = (stp.drift - stm.drift) / (2 * h_om)

    def geom_for(c, stp_):
        gg = LensGeometry(c, stp_, geom.zs, geom.npix, np.rad2deg(geom.fov), L, nc, M,
                          rotate=geom.rotate, seed=geom.seed, sub_evolution=geom.sub_evolution)
        gg.chi_a = geom.chi_a      # selection at the central cosmology
        for s, spec in enumerate(geom.nz):
            if spec is not None:   # the same n(z); its distances in the perturbed cosmology
                gg.set_source_nz(s, spec[0], spec[1])
        return gg

    gp_, gm_ = geom_for(cp, stp), geom_for(cm, stm)
    dL_dom = 0.0
    # mean term
    dmean = (gp_.mean_term() - gm_.mean_term()) / (2 * h_om)
    dL_dom += -float(np.sum(lam.sum(axis=(1, 2)) * dmean))

    lam_x = np.zeros_like(tr.x[0])
    lam_p = np.zeros_like(tr.p[0])
    for i in range(n - 1, -1, -1):
        x1, ph = tr.x[i + 1], tr.p[i + 1]
        if geom.active(i):
            S = tr.S[i]
            gx, gpp, gS = project_vjp(geom, i, x1, ph, S, lam)
            lam_x += gx
            lam_p += gpp
            if S is not None:
                lam_x += pgd_vjp(x1, gS, st.a[i + 1], nc, M, L, sim.pgd_params)
            mp = gp_.project(i, x1, ph, S)[0]
            mm = gm_.project(i, x1, ph, S)[0]
            dL_dom += float(np.sum(lam * (mp - mm))) / (2 * h_om)
        # drift x_{i+1} = x_i + drift_i p_{i+1/2}
        dL_dom += ddrift[i] * float(np.sum(lam_x * ph))
        lam_p += st.drift[i] * lam_x
        # kick p_{i+1/2} = p_{i-1/2} + kick_i F(x_i), F proportional to Om
        xi = tr.x[i]
        f_unit = sim_force_unit(xi, nc, M, L)          # F / Om
        dL_dom += dkick[i] * float(np.sum(lam_p * f_unit))
        lam_x += force_vjp(xi, st.kick[i] * lam_p, nc, M, L, om)
    # initial conditions: x0 = q + D1 Psi1 + D2 Psi2, p0 = gp Psi1 + gp2 Psi2
    a0 = st.a[0]
    psi1, psi2 = tr.psi1, tr.psi2
    lp1 = cosmo.D1(a0) * lam_x + cosmo.gp(a0) * lam_p
    lp2 = None
    if psi2 is not None:
        lp2 = cosmo.D2(a0) * lam_x + cosmo.gp2(a0) * lam_p
    dk = linear_modes(noise, cosmo, L)
    dL_dnoise = lpt_vjp(lp1, lp2, dk, nc, L, cosmo, sim.lpt_order)
    dL_ds8 = float(np.sum(lp1 * psi1)) / cosmo.sigma8
    if psi2 is not None:
        dL_ds8 += 2.0 * float(np.sum(lp2 * psi2)) / cosmo.sigma8
    # Omega_m through the initial state (P(k), growth factors), finite difference
    xs = []
    for c in (cp, cm):
        dkc = linear_modes(noise, c, L)
        p1, p2 = lpt_displacements(dkc, nc, L, sim.lpt_order)
        xs.append(lpt_state(p1, p2, c, a0, nc, L, M))
    dx0 = (xs[0][0] - xs[1][0] + L / 2) % L - L / 2
    dp0 = xs[0][1] - xs[1][1]
    dL_dom += (float(np.sum(lam_x * dx0)) + float(np.sum(lam_p * dp0))) / (2 * h_om)
    return kappa, dL_dnoise, dL_dom, dL_ds8


def sim_force_unit(x, nc, nmesh, box):
    """PM force at x per unit Omega_m."""
    rho = cic_paint(x, nmesh, box, particle_mass(nc, nmesh))
    fm = force_mesh(rho - 1.0, box, 1.0)
    return np.stack([cic_readout(m, x, box) for m in fm], axis=1)
