"""Born-approximation lightcone projection in FP64 (TEST INFRASTRUCTURE ONLY).

Eq. (conv):  kappa(theta) = (3 H0^2 Om / 2 c^2) int_0^chi_s dchi q(chi)/a(chi)
             delta(chi theta, chi),   q = chi (chi_s - chi) / chi_s
for a source plane at chi_s (n(chi') a Dirac delta in the lensing kernel).

Discretised with particles (Sec. 3): each step i projects the particles whose
comoving distance lies in the shell (chi(a_{i+1}), chi(a_i)], replicating the
box along and across the line of sight, each replica rotated; with the
sub-evolution scheme each selected particle is first moved to the time at which
it crosses the lightcone.  A particle of volume V_p = (L/Nc)^3 adds
    w = (3/2) Om (H0/c)^2 (chi_s - chi)/(chi_s chi a) V_p / Omega_pix
to the map (CIC in the flat-sky angle), and the mean-density term
    (3/2) Om (H0/c)^2 int_0^chi_s chi (chi_s - chi) / (chi_s a(chi)) dchi
is subtracted at the end (delta = density / mean - 1).

Readings (paper silent): observer at the origin looking along +z, flat-sky
gnomonic angles theta = (r_x/r_z, r_y/r_z), map pixel centres at
(j + 1/2) dtheta - FOV/2; replica n = (nx, ny, nz) covers [n L, (n+1) L) and
gets one of the 48 cube symmetries plus a periodic shift in whole force-mesh
cells drawn from one SplitMix64 output of seed ^ pack(n); selection uses the
distance of the particle at a_{i+1}; sub-evolution drifts it with p(a_{i+1/2})
to a(chi): x_c = x + p [D1(a(chi)) - D1(a_{i+1})] / g_p(a_{i+1/2}); PGD adds
its displacement to the projected position only; the weight uses chi_c = |r_c|
and a(chi_c).
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import quad

from .cosmology import C_OVER_H0

MASK64 = (1 << 64) - 1
PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def splitmix64(state: int) -> int:
    """One output of SplitMix64 (Steele, Lea & Flood 2014; Vigna's constants)
    for the given 64-bit state: advance by the golden gamma, then mix."""
    z = (state + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def pack_replica(nx: int, ny: int, nz: int) -> int:
    """20-bit two's-complement fields: nx << 40 | ny << 20 | nz."""
    return ((nx & 0xFFFFF) << 40) | ((ny & 0xFFFFF) << 20) | (nz & 0xFFFFF)


def replica_transform(n, seed: int, rotate: bool, nmesh: int):
    """(perm, flips, shift_cells) of replica n; identity when rotate is off."""
    if not rotate:
        return (0, 1, 2), (0, 0, 0), (0, 0, 0)
    h = splitmix64((seed ^ pack_replica(*n)) & MASK64)
    perm = PERMS[h % 6]
    flips = tuple((h >> (8 + d)) & 1 for d in range(3))
    shift = tuple(((h >> (16 + 16 * d)) & 0xFFFF) % nmesh for d in range(3))
    return perm, flips, shift


def apply_transform(x, tr, box, nmesh):
    """Rotate/flip/shift box positions x (N, 3) in [0, L) into [0, L)."""
    perm, flips, shift = tr
    y = np.empty_like(x)
    for d in range(3):
        v = x[:, perm[d]]
        if flips[d]:
            v = box - v
        y[:, d] = np.mod(v + shift[d] * (box / nmesh), box)
    return y


def apply_rotation(v, tr):
    """Rotate/flip a displacement or momentum vector (no shift)."""
    perm, flips, _ = tr
    out = np.empty_like(v)
    for d in range(3):
        out[:, d] = -v[:, perm[d]] if flips[d] else v[:, perm[d]]
    return out


def candidate_replicas(chi_lo, chi_hi, box, half_fov_rad, margin):
    """Every replica whose box may hold a particle of the shell inside the cone.

    Conservative: the bounding box of (shell within the field of view, widened
    by `margin`) intersected with the sphere-shell distance test.
    """
    t = np.tan(half_fov_rad)
    cos_corner = 1.0 / np.sqrt(1.0 + 2.0 * t * t)
    z0 = max(0.0, chi_lo * cos_corner - margin)
    z1 = chi_hi + margin
    w = chi_hi * t + margin
    out = []
    for nz in range(int(np.floor(z0 / box)), int(np.floor(z1 / box)) + 1):
        for ny in range(int(np.floor(-w / box)), int(np.floor(w / box)) + 1):
            for nx in range(int(np.floor(-w / box)), int(np.floor(w / box)) + 1):
                lo = np.array([nx, ny, nz], dtype=np.float64) * box
                hi = lo + box
                near = np.clip(0.0, lo, hi)
                dmin = np.linalg.norm(near)
                far = np.where(np.abs(lo) > np.abs(hi), lo, hi)
                dmax = np.linalg.norm(far)
                if dmin <= chi_hi + margin and dmax >= chi_lo - margin:
                    out.append((nx, ny, nz))
    return out


class LensGeometry:
    """Shells, source distances and map geometry for one simulation."""

    def __init__(self, cosmo, stepper, zs, npix, fov_deg, box, nc, nmesh,
                 rotate=True, seed=42, sub_evolution=True):
        self.cosmo = cosmo
        self.stepper = stepper
        self.zs = np.atleast_1d(np.asarray(zs, dtype=np.float64))
        self.chi_s = cosmo.chi_z(self.zs)
        self.npix = int(npix)
        self.fov_deg = float(fov_deg)
        self.fov = np.deg2rad(fov_deg)
        self.dtheta = self.fov / self.npix
        self.box, self.nc, self.nmesh = float(box), int(nc), int(nmesh)
        self.rotate, self.seed = bool(rotate), int(seed)
        self.sub_evolution = bool(sub_evolution)
        self.chi_a = cosmo.chi(stepper.a)  # chi at every step boundary
        self.prefac = 1.5 * cosmo.omega_m / C_OVER_H0 ** 2
        self.vp = (self.box / self.nc) ** 3
        self.nz = [None] * len(self.zs)      # per source: None (a plane at zs) or (z, n, tables)

    def set_source_nz(self, s, z, n):
        """Source s becomes the distribution n(z) (Eq. conv with a general n(chi')):
        n tabulated at ascending redshifts z, linear in between and zero outside,
        normalised to unit integral over z.  Its lensing efficiency is

            q(chi) = int dz' n(z') (1 - chi / chi(z'))_+ = A(chi) - chi B(chi),
            A(chi) = int_{z(chi)} n dz',  B(chi) = int_{z(chi)} n / chi(z') dz',

        and dq/dchi = -B(chi) (the boundary terms cancel).  A and B are cumulative
        trapezoid integrals from the top on a 200001-point redshift grid.
        """
        z = np.asarray(z, dtype=np.float64)
        n = np.asarray(n, dtype=np.float64)
        zz = np.linspace(z[0], z[-1], 200001)
        nn = np.interp(zz, z, n)
        nn = nn / float(np.sum(0.5 * (nn[1:] + nn[:-1]) * np.diff(zz)))
        chi = self.cosmo.chi_z(zz)

        def cum_top(f):      # int_{zz[k]}^{zz[-1]} f dz'
            seg = 0.5 * (f[1:] + f[:-1]) * np.diff(zz)
            return np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
        A = cum_top(nn)
        B = cum_top(np.where(chi > 0, nn / np.where(chi > 0, chi, 1.0), 0.0))
        self.nz[s] = (z, n, chi, A, B)
        self.chi_s[s] = chi[-1]          # farthest contributing distance

    def source_weight(self, s, chi):
        """(q_s(chi), dq_s/dchi): the lensing efficiency of source s at comoving chi."""
        chi = np.asarray(chi, dtype=np.float64)
        if self.nz[s] is None:
            cs = self.chi_s[s]
            inside = chi < cs
            return np.where(inside, (cs - chi) / cs, 0.0), np.where(inside, -1.0 / cs, 0.0)
        _, _, cg, A, B = self.nz[s]
        a = np.interp(chi, cg, A, left=A[0], right=0.0)
        b = np.interp(chi, cg, B, left=B[0], right=0.0)
        return np.maximum(a - chi * b, 0.0), -b

    def shell(self, i):
        return self.chi_a[i + 1], self.chi_a[i]

    def active(self, i):
        lo, _ = self.shell(i)
        return lo < self.chi_s.max()

    def mean_term(self):
        """(3/2) Om (H0/c)^2 int_0^chi_s chi (chi_s - chi) / (chi_s a(chi)) dchi, or with a
        source distribution (3/2) Om (H0/c)^2 int chi q(chi) / a(chi) dchi."""
        out = []
        for s, cs in enumerate(self.chi_s):
            if self.nz[s] is None:
                f = lambda c: c * (cs - c) / (cs * self.cosmo.a_of_chi(c))  # noqa: E731
            else:
                f = lambda c, s=s: c * float(self.source_weight(s, c)[0]) / self.cosmo.a_of_chi(c)  # noqa: E731
            v, _ = quad(f, 0.0, cs, limit=2000, epsabs=0, epsrel=1e-12)
            out.append(self.prefac * v)
        return np.array(out)

    def subevolve_factor(self, i, a_c):
        """[D1(a_c) - D1(a_{i+1})] / g_p(a_{i+1/2}): multiplies p(a_{i+1/2}) to move
        x(a_{i+1}) to its lightcone-crossing time a_c (sub-evolution, Sec. 3)."""
        st = self.stepper
        return (self.cosmo.D1(a_c) - self.cosmo.D1(st.a[i + 1])) / self.cosmo.gp(st.ah[i])

    def project(self, i, x, p, S=None, margin=None):
        """Map increments (n_zs, npix, npix) of shell i [iy, ix] from x(a_{i+1}), p(a_{i+1/2}).

        Returns the increments and the number of particle-replica hits.
        """
        cosmo, st = self.cosmo, self.stepper
        maps = np.zeros((len(self.zs), self.npix, self.npix))
        if not self.active(i):
            return maps, 0
        lo, hi = self.shell(i)
        a_next, a_half = st.a[i + 1], st.ah[i]
        gp_half = cosmo.gp(a_half)
        if margin is None:
            margin = 2.0 * self.box / self.nmesh
            if self.sub_evolution:
                dd = float(cosmo.D1(a_next) - cosmo.D1(max(cosmo.a_min, cosmo.a_of_chi(hi))))
                margin += float(np.max(np.abs(p))) * abs(dd) / gp_half * np.sqrt(3)
            if S is not None:
                margin += float(np.max(np.abs(S))) * np.sqrt(3)
        half = 0.5 * self.fov + self.dtheta
        hits = 0
        for n in candidate_replicas(lo, hi, self.box, half, margin):
            tr = replica_transform(n, self.seed, self.rotate, self.nmesh)
            r = apply_transform(x, tr, self.box, self.nmesh) + np.asarray(n, dtype=np.float64) * self.box
            chi = np.linalg.norm(r, axis=1)
            sel = (chi > lo) & (chi <= hi) & (r[:, 2] > 0)
            if not np.any(sel):
                continue
            rs = r[sel]
            if self.sub_evolution:
                dt = self.subevolve_factor(i, cosmo.a_of_chi(chi[sel]))
                rs = rs + apply_rotation(p[sel], tr) * dt[:, None]
            if S is not None:
                rs = rs + apply_rotation(S[sel], tr)
            hits += int(sel.sum())
            self._deposit(maps, rs)
        return maps, hits

    def _deposit(self, maps, rc):
        chic = np.linalg.norm(rc, axis=1)
        ok = rc[:, 2] > 0
        rc, chic = rc[ok], chic[ok]
        ac = self.cosmo.a_of_chi(chic)
        tx = rc[:, 0] / rc[:, 2]
        ty = rc[:, 1] / rc[:, 2]
        u = (tx + 0.5 * self.fov) / self.dtheta - 0.5
        v = (ty + 0.5 * self.fov) / self.dtheta - 0.5
        iu, iv = np.floor(u).astype(np.int64), np.floor(v).astype(np.int64)
        fu, fv = u - iu, v - iv
        omega_pix = self.dtheta ** 2
        for s, cs in enumerate(self.chi_s):
            if self.nz[s] is None:
                w = np.where(chic < cs,
                             self.prefac * (cs - chic) / (cs * chic * ac) * self.vp / omega_pix, 0.0)
            else:
                w = self.prefac * self.source_weight(s, chic)[0] / (chic * ac) * self.vp / omega_pix
            for du in (0, 1):
                for dv in (0, 1):
                    ww = w * (fu if du else 1.0 - fu) * (fv if dv else 1.0 - fv)
                    jx, jy = iu + du, iv + dv
                    ok2 = (jx >= 0) & (jx < self.npix) & (jy >= 0) & (jy < self.npix)
                    np.add.at(maps[s], (jy[ok2], jx[ok2]), ww[ok2])
