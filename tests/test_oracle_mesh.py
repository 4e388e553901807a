"""Pins of the oracle's mesh operations against closed forms and brute force."""
import itertools

import numpy as np
import pytest

from oracle import mesh


def test_rfftn_matches_bruteforce_dft_8cubed():
    """The FFT primitive and its sign/normalisation against an explicit DFT."""
    rng = np.random.default_rng(0)
    M = 8
    f = rng.standard_normal((M, M, M))
    n = np.arange(M)
    # explicit sum_x f(x) exp(-2 pi i k.x / M), axes [z, y, x]
    ez = np.exp(-2j * np.pi * np.outer(n, n) / M)
    brute = np.einsum("az,by,cx,zyx->abc", ez, ez, ez[: M // 2 + 1], f)
    assert np.allclose(np.fft.rfftn(f), brute, rtol=0, atol=1e-11)
    # Parseval
    full = np.fft.fftn(f)
    assert np.isclose(np.sum(np.abs(full) ** 2) / M ** 3, np.sum(f ** 2), rtol=1e-13)


@pytest.mark.parametrize("nvec", [(1, 0, 0), (0, 2, 0), (0, 0, 3), (1, 2, -1), (3, -1, 2)])
def test_force_plane_wave_closed_form(nvec):
    """delta = A cos(k.x)  =>  F = -(3/2) Om A k / k^2 sin(k.x), exact."""
    M, L, om, A = 16, 100.0, 0.31, 0.7
    k = 2 * np.pi * np.asarray(nvec, dtype=float) / L
    g = np.arange(M) * L / M
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    phase = k[0] * x + k[1] * y + k[2] * z
    delta = A * np.cos(phase)
    F = mesh.force_mesh(delta, L, om)
    k2 = np.sum(k * k)
    for j in range(3):
        expect = -1.5 * om * A * k[j] / k2 * np.sin(phase)
        assert np.allclose(F[j], expect, rtol=0, atol=1e-12)


def test_force_direct_sum_green_function_8cubed():
    """FFT Poisson + gradient equals an O(M^6) direct sum against the periodic
    discrete Green's function G_j(r) = M^-3 sum_k (3/2) Om i k_j / k^2 e^{i k.r}."""
    M, L, om = 8, 40.0, 0.3
    rng = np.random.default_rng(3)
    delta = rng.standard_normal((M, M, M))
    F = mesh.force_mesh(delta, L, om)
    n = np.fft.fftfreq(M, 1.0 / M)
    kf = 2 * np.pi / L
    kz, ky, kx = np.meshgrid(kf * n, kf * n, kf * n, indexing="ij")
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k2[0, 0, 0] = 1.0
    nyq = np.pi * M / L
    idx = np.arange(M)
    rz, ry, rx = np.meshgrid(idx, idx, idx, indexing="ij")
    for j, kj in enumerate((kx, ky, kz)):
        mult = 1.5 * om * 1j * np.where(np.isclose(np.abs(kj), nyq), 0.0, kj) / k2
        mult[0, 0, 0] = 0.0
        G = np.zeros((M, M, M))
        for a, b, c in itertools.product(range(M), repeat=3):   # modes (kz, ky, kx)
            ph = 2 * np.pi * (n[a] * rz + n[b] * ry + n[c] * rx) / M
            G += np.real(mult[a, b, c] * np.exp(1j * ph))
        G /= M ** 3
        direct = np.zeros((M, M, M))
        for s in itertools.product(range(M), repeat=3):   # source cell (z, y, x)
            direct += delta[s] * np.roll(G, shift=s, axis=(0, 1, 2))
        assert np.allclose(F[j], direct, rtol=0, atol=1e-12)


def test_cic_mass_conservation_and_node():
    rng = np.random.default_rng(1)
    M, L = 16, 50.0
    pos = rng.uniform(0, L, size=(1000, 3))
    w = rng.uniform(0.5, 2.0, size=1000)
    rho = mesh.cic_paint(pos, M, L, w)
    assert np.isclose(rho.sum(), w.sum(), rtol=1e-14)
    # a particle exactly on a node puts all its mass on that node
    p = np.array([[3, 5, 7]], dtype=float) * (L / M)
    rho = mesh.cic_paint(p, M, L, 1.0)
    assert rho[7, 5, 3] == 1.0 and rho.sum() == 1.0


def test_cic_explicit_weights():
    """A particle at mesh coordinates (1.25, 2.5, 3.75): eight explicit weights."""
    M, L = 8, 8.0
    rho = mesh.cic_paint(np.array([[1.25, 2.5, 3.75]]), M, L, 1.0)
    expect = {}
    for (ix, wx), (iy, wy), (iz, wz) in itertools.product(
            [(1, 0.75), (2, 0.25)], [(2, 0.5), (3, 0.5)], [(3, 0.25), (4, 0.75)]):
        expect[(iz, iy, ix)] = wx * wy * wz
    for key, val in expect.items():
        assert np.isclose(rho[key], val, rtol=0, atol=1e-15)
    assert np.isclose(rho.sum(), 1.0)
    # periodic wrap across the upper face
    rho = mesh.cic_paint(np.array([[7.5, 0.0, 0.0]]), M, L, 1.0)
    assert np.isclose(rho[0, 0, 7], 0.5) and np.isclose(rho[0, 0, 0], 0.5)


def test_cic_paint_readout_adjoint_dot_product():
    """<paint(w), m> = <w, readout(m)> (paint and readout are transposes)."""
    rng = np.random.default_rng(2)
    M, L = 12, 30.0
    pos = rng.uniform(0, L, size=(500, 3))
    w = rng.standard_normal(500)
    m = rng.standard_normal((M, M, M))
    lhs = np.sum(mesh.cic_paint(pos, M, L, w) * m)
    rhs = np.sum(w * mesh.cic_readout(m, pos, box=L))
    assert np.isclose(lhs, rhs, rtol=1e-13)


def test_cic_readout_exact_for_linear_field_and_gradient():
    """Trilinear interpolation reproduces a field linear inside one cell, and
    the CIC position gradient equals that field's slope."""
    M, L = 8, 8.0
    g = np.arange(M, dtype=float)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    field = 2.0 * x - 3.0 * y + 0.5 * z + 1.0
    pos = np.array([[2.3, 4.1, 1.7], [5.5, 5.5, 5.5], [0.01, 6.99, 3.2]])
    val = mesh.cic_readout(field, pos, L)
    assert np.allclose(val, 2.0 * pos[:, 0] - 3.0 * pos[:, 1] + 0.5 * pos[:, 2] + 1.0)
    grad = mesh.cic_readout_grad(field, pos, L)
    assert np.allclose(grad, np.array([2.0, -3.0, 0.5])[None, :])


def test_cic_readout_grad_finite_difference():
    rng = np.random.default_rng(5)
    M, L = 10, 20.0
    m = rng.standard_normal((M, M, M))
    pos = rng.uniform(0, L, size=(50, 3))
    g = mesh.cic_readout_grad(m, pos, L)
    eps = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = eps
        fd = (mesh.cic_readout(m, pos + e, L) - mesh.cic_readout(m, pos - e, L)) / (2 * eps)
        assert np.allclose(g[:, d], fd, atol=1e-6)


def test_pgd_plane_wave_closed_form():
    """delta = A cos(k.x) => S = -alpha O_L(k) O_S(k) A k/k^2 sin(k.x)."""
    M, L, A = 16, 64.0, 0.3
    alpha, kl, ks, n = 0.05, 0.2, 0.5, 4.0
    nvec = np.array([2.0, -1.0, 1.0])
    k = 2 * np.pi * nvec / L
    kk = np.sqrt(np.sum(k * k))
    g = np.arange(M) * L / M
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    ph = k[0] * x + k[1] * y + k[2] * z
    S = mesh.pgd_mesh(A * np.cos(ph), L, alpha, kl, ks, n)
    filt = np.exp(-(kl / kk) ** 2) * np.exp(-(kk / ks) ** n)
    for j in range(3):
        assert np.allclose(S[j], -alpha * filt * A * k[j] / kk ** 2 * np.sin(ph), atol=1e-13)
