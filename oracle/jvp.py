"""Forward-mode derivative (JVP) of the forward model in FP64 (TEST INFRASTRUCTURE ONLY).

Sec. 3: the model is differentiable with respect to the initial Gaussian
modes, and the paper checks its Jacobian-vector product against finite
differences by changing the initial field in one pixel (Fig. 8).  This module
is the tangent-linear model: the derivative of every forward operation of
``oracle.lpt``, ``oracle.nbody`` and ``oracle.lightcone`` along a direction
d of the white noise, propagated alongside the forward run:

* the linear modes and Psi1 are linear in the noise; the 2LPT source
  sum_{i<j} (phi_ii phi_jj - phi_ij^2) has the tangent
  sum_{i<j} (dphi_ii phi_jj + phi_ii dphi_jj - 2 phi_ij dphi_ij);
* the PM force at x, F(x) = readout(K * paint(x), x), has the tangent
  readout_grad(K * paint(x), x) . dx + readout(K * paint_tangent(x, dx), x),
  where paint_tangent deposits dx . grad of the CIC weights; the PGD
  displacement likewise with the PGD kernel;
* the kick and drift are linear in (p, F) and (x, p);
* the projection: the shell selection and the pixel of each deposit are held
  fixed (piecewise constant), and the Born weight w(chi_c) and the CIC weights
  in angle are differentiated along the sub-evolved, PGD-displaced position.
"""
from __future__ import annotations

import itertools

import numpy as np

from .cosmology import C_OVER_H0
from . import dft
from .lightcone import LensGeometry, apply_rotation, apply_transform, candidate_replicas, replica_transform
from .lpt import _odd, linear_modes
from .mesh import (cic_paint, cic_readout, cic_readout_grad, force_mesh, gradient_multipliers,
                   particle_mass, pgd_mesh, wavevectors)


def cic_paint_tangent(pos, dpos, nmesh, box, weight):
    """d/de cic_paint(pos + e dpos, weight) at e = 0: sum_j weight dpos_j . grad w_c(pos_j).

    The CIC weights are piecewise linear; the derivative is taken in the cell
    that contains the particle (floor convention), as in cic_readout_grad.
    """
    pos = np.asarray(pos, dtype=np.float64)
    g = pos * (nmesh / box)
    i0 = np.floor(g).astype(np.int64)
    f = g - i0
    out = np.zeros(nmesh ** 3, dtype=np.float64)
    for dx, dy, dz in itertools.product((0, 1), repeat=3):
        w = [f[:, 0] if dx else 1.0 - f[:, 0],
             f[:, 1] if dy else 1.0 - f[:, 1],
             f[:, 2] if dz else 1.0 - f[:, 2]]
        dw = [1.0 if dx else -1.0, 1.0 if dy else -1.0, 1.0 if dz else -1.0]
        t = (dw[0] * w[1] * w[2] * dpos[:, 0] + w[0] * dw[1] * w[2] * dpos[:, 1]
             + w[0] * w[1] * dw[2] * dpos[:, 2]) * (nmesh / box) * weight
        flat = (((i0[:, 2] + dz) % nmesh) * nmesh + (i0[:, 1] + dy) % nmesh) * nmesh + (i0[:, 0] + dx) % nmesh
        out += np.bincount(flat, weights=t, minlength=nmesh ** 3)
    return out.reshape(nmesh, nmesh, nmesh)


def _mesh_field_tangent(x, dx, meshes, dmeshes, box):
    """Tangent of readout(meshes(x), x): readout_grad(m, x) . dx + readout(dm, x), (N, 3)."""
    return np.stack([np.sum(cic_readout_grad(m, x, box) * dx, axis=1) + cic_readout(dm, x, box)
                     for m, dm in zip(meshes, dmeshes)], axis=1)


def force_tangent(x, dx, nc, nmesh, box, omega_m):
    """Tangent of the PM force F(x) along dx (N, 3), Mpc/h units as oracle.mesh."""
    mass = particle_mass(nc, nmesh)
    fm = force_mesh(cic_paint(x, nmesh, box, mass) - 1.0, box, omega_m)
    dfm = force_mesh(cic_paint_tangent(x, dx, nmesh, box, mass), box, omega_m)
    return _mesh_field_tangent(x, dx, fm, dfm, box)


def pgd_tangent(x, dx, a, nc, nmesh, box, pgd_params):
    """Tangent of the PGD displacement S(x) along dx."""
    alpha0, mu, k_l, k_s, n_s = pgd_params
    alpha = alpha0 * a ** mu
    mass = particle_mass(nc, nmesh)
    sm = pgd_mesh(cic_paint(x, nmesh, box, mass) - 1.0, box, alpha, k_l, k_s, n_s)
    dsm = pgd_mesh(cic_paint_tangent(x, dx, nmesh, box, mass), box, alpha, k_l, k_s, n_s)
    return _mesh_field_tangent(x, dx, sm, dsm, box)


def lpt_tangent(delta_k, ddelta_k, nc, box, order):
    """(dPsi1, dPsi2) for a tangent ddelta_k of the linear modes."""
    shape = (nc, nc, nc)
    mult = gradient_multipliers(nc, box)
    dpsi1 = np.stack([dft.irfftn(m * ddelta_k, s=shape, axes=(0, 1, 2)).ravel() for m in mult], axis=1)
    if order == 1:
        return dpsi1, None
    kx, ky, kz = wavevectors(nc, box)
    kk = (kx, ky, kz)
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(k2 > 0, 1.0 / k2, 0.0)
    d, dd = {}, {}
    for i in range(3):
        for j in range(i, 3):
            mij = (-kk[i] * kk[i] if i == j else -_odd(kk[i], nc, box) * _odd(kk[j], nc, box)) * inv
            d[(i, j)] = dft.irfftn(mij * delta_k, s=shape, axes=(0, 1, 2))
            dd[(i, j)] = dft.irfftn(mij * ddelta_k, s=shape, axes=(0, 1, 2))
    dsrc = (dd[(0, 0)] * d[(1, 1)] + d[(0, 0)] * dd[(1, 1)] + dd[(0, 0)] * d[(2, 2)] + d[(0, 0)] * dd[(2, 2)]
            + dd[(1, 1)] * d[(2, 2)] + d[(1, 1)] * dd[(2, 2)]
            - 2 * d[(0, 1)] * dd[(0, 1)] - 2 * d[(0, 2)] * dd[(0, 2)] - 2 * d[(1, 2)] * dd[(1, 2)])
    sk = dft.rfftn(dsrc)
    dpsi2 = np.stack([dft.irfftn(-m * sk, s=shape, axes=(0, 1, 2)).ravel() for m in mult], axis=1)
    return dpsi1, dpsi2


def project_tangent(geom: LensGeometry, i, x, p, S, dx, dp, dS):
    """Tangent (n_zs, npix, npix) of shell i's map increments along (dx, dp, dS).

    Follows LensGeometry.project: the same replicas and selection (held fixed),
    r_c = r + R p dt(|r|) (+ R S), angles, CIC weights in angle and the Born
    weight w_s(chi_c) = K (chi_s - chi_c)/(chi_s chi_c a(chi_c)).
    """
    cosmo, st = geom.cosmo, geom.stepper
    out = np.zeros((len(geom.zs), geom.npix, geom.npix))
    if not geom.active(i):
        return out
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
        drs = apply_rotation(dx[sel], tr)
        rc, drc = rs.copy(), drs.copy()
        if geom.sub_evolution:
            pr, dpr = apply_rotation(p[sel], tr), apply_rotation(dp[sel], tr)
            ac = cosmo.a_of_chi(chis)
            dt = geom.subevolve_factor(i, ac)
            ddt = -cosmo.gp(ac) / (ac * C_OVER_H0) / gp_half          # d dt / d chi
            rc = rc + pr * dt[:, None]
            drc = drc + dpr * dt[:, None] + pr * (ddt * np.sum(rs * drs, axis=1) / chis)[:, None]
        if S is not None:
            rc = rc + apply_rotation(S[sel], tr)
            drc = drc + apply_rotation(dS[sel], tr)
        ok = rc[:, 2] > 0
        rc, drc = rc[ok], drc[ok]
        chic = np.linalg.norm(rc, axis=1)
        dchic = np.sum(rc * drc, axis=1) / chic
        ac2 = cosmo.a_of_chi(chic)
        inva = 1.0 / ac2
        dinva = cosmo.E(ac2) / C_OVER_H0                                # d(1/a)/dchi
        u = (rc[:, 0] / rc[:, 2] + 0.5 * geom.fov) / geom.dtheta - 0.5
        v = (rc[:, 1] / rc[:, 2] + 0.5 * geom.fov) / geom.dtheta - 0.5
        du_ = (drc[:, 0] / rc[:, 2] - rc[:, 0] * drc[:, 2] / rc[:, 2] ** 2) / geom.dtheta
        dv_ = (drc[:, 1] / rc[:, 2] - rc[:, 1] * drc[:, 2] / rc[:, 2] ** 2) / geom.dtheta
        iu, iv = np.floor(u).astype(np.int64), np.floor(v).astype(np.int64)
        fu, fv = u - iu, v - iv
        for s, cs in enumerate(geom.chi_s):
            if geom.nz[s] is None:
                inside = chic < cs
                f = 1.0 / chic - 1.0 / cs
                w = np.where(inside, K * f * inva, 0.0)
                dw = np.where(inside, K * (-inva / chic ** 2 + f * dinva), 0.0) * dchic
            else:
                q, dq = geom.source_weight(s, chic)
                w = K * q / chic * inva
                dw = K * ((dq * chic - q) / chic ** 2 * inva + q / chic * dinva) * dchic
            for du in (0, 1):
                for dv in (0, 1):
                    wu = fu if du else 1.0 - fu
                    wv = fv if dv else 1.0 - fv
                    dwu = du_ if du else -du_
                    dwv = dv_ if dv else -dv_
                    t = dw * wu * wv + w * (dwu * wv + wu * dwv)
                    jx, jy = iu + du, iv + dv
                    good = (jx >= 0) & (jx < geom.npix) & (jy >= 0) & (jy < geom.npix)
                    np.add.at(out[s], (jy[good], jx[good]), t[good])
    return out


def jvp(sim, noise, dnoise):
    """(kappa, dkappa): the forward maps and their derivative along dnoise.

    Runs the forward model on `sim` (an oracle.sim.Simulation) with the tangent
    state (dx, dp, dF) carried alongside: dx0 = D1 dPsi1 + D2 dPsi2,
    dp0 = g_p dPsi1 + g_p2 dPsi2; kick dp += kick_i dF(x_i); drift
    dx += drift_i dp; dF at the new positions; each shell's tangent deposit.
    """
    nc, M, L = sim.nc, sim.nmesh, sim.box
    st, geom, cosmo = sim.stepper, sim.geom, sim.cosmo
    om = cosmo.omega_m
    a0 = st.a[0]
    dk = linear_modes(noise, cosmo, L)
    ddk = linear_modes(dnoise, cosmo, L)          # linear in the noise
    dpsi1, dpsi2 = lpt_tangent(dk, ddk, nc, L, sim.lpt_order)
    sim.ic(noise)
    dx = cosmo.D1(a0) * dpsi1
    dp = cosmo.gp(a0) * dpsi1
    if dpsi2 is not None:
        dx = dx + cosmo.D2(a0) * dpsi2
        dp = dp + cosmo.gp2(a0) * dpsi2
    dF = force_tangent(sim.state.x, dx, nc, M, L, om)
    dmaps = np.zeros_like(sim.maps)
    for i in range(sim.nsteps):
        dp = dp + st.kick[i] * dF
        dx = dx + st.drift[i] * dp
        sim.step(i)
        dF = force_tangent(sim.state.x, dx, nc, M, L, om)
        if geom.active(i):
            S = sim.pgd_at(i)
            dS = None
            if S is not None:
                dS = pgd_tangent(sim.state.x, dx, st.a[i + 1], nc, M, L, sim.pgd_params)
            inc, _ = geom.project(i, sim.state.x, sim.state.p, S)
            sim.maps += inc
            dmaps += project_tangent(geom, i, sim.state.x, sim.state.p, S, dx, dp, dS)
    return sim.kappa_maps(), dmaps
