"""Pins of the oracle's sampled statistics: the unitary transform of Sec. III (notation)
and the radially binned density / longitudinal / transverse momentum spectra."""
import numpy as np

import oracle
from oracle import theory as th

RNG = np.random.default_rng(3)


def test_unitary_transform_parseval_and_plane_wave():
    a = RNG.normal(size=(10, 12))
    ak = oracle.unitary_ft(a)
    np.testing.assert_allclose((np.abs(ak) ** 2).sum(), (a * a).sum(), rtol=1e-13)
    # a(k) = n^-1/2 sum_r exp(+i k.r) a(r): a plane wave exp(-i k0.r) lands on k0 alone
    nx, ny = 12, 10
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    mx, my = 3, 2
    w = np.exp(-1j * 2 * np.pi * (mx * X / nx + my * Y / ny))
    wk = oracle.unitary_ft(w)
    expect = np.zeros((ny, nx), complex)
    expect[my, mx] = np.sqrt(nx * ny)
    np.testing.assert_allclose(wk, expect, atol=1e-12)


def test_k_bins():
    nx, ny, nb = 16, 8, 10
    b, KX, KY, kmag = oracle.k_bins(nx, ny, nb)
    assert b[0, 0] == -1
    assert b[b >= 0].size == nx * ny - 1 and b.max() <= nb - 1
    order = np.argsort(kmag.ravel())
    bb = b.ravel()[order][1:]
    assert np.all(np.diff(bb) >= 0)                     # bins increase with |k|
    assert np.all(np.abs(KX) <= np.pi + 1e-15) and np.all(np.abs(KY) <= np.pi + 1e-15)


def _state_from_fields(rho0, drho, jx, jy):
    # populations carrying exactly (rho0 + drho, jx, jy) and no other moment
    m = np.zeros((9,) + drho.shape)
    m[0] = rho0 + drho
    m[1] = jx
    m[2] = jy
    return np.einsum("ia,ayx->iyx", th.TINV, m)


def test_spectra_of_known_fields():
    nx, ny, nb = 16, 16, 8
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    mx, my = 2, 3
    kx, ky = 2 * np.pi * mx / nx, 2 * np.pi * my / ny
    A = 1e-3
    c = np.cos(kx * X + ky * Y)
    kh = np.array([kx, ky]) / np.hypot(kx, ky)
    b, _, _, _ = oracle.k_bins(nx, ny, nb)
    target_bin = b[my, mx]
    n = nx * ny
    # density wave
    S, Jl, Jt, cnt = oracle.spectra_sample(_state_from_fields(1.0, A * c, 0 * c, 0 * c), 1.0, nb)
    expect = np.zeros(nb)
    expect[target_bin] = 2 * n * A * A / 4
    np.testing.assert_allclose(S, expect, atol=1e-18)
    np.testing.assert_allclose(Jl, 0, atol=1e-20)
    # longitudinal and transverse momentum waves
    S, Jl, Jt, _ = oracle.spectra_sample(_state_from_fields(1.0, 0 * c, A * kh[0] * c, A * kh[1] * c), 1.0, nb)
    np.testing.assert_allclose(Jl, expect, atol=1e-18)
    np.testing.assert_allclose(Jt, 0, atol=1e-18)
    S, Jl, Jt, _ = oracle.spectra_sample(_state_from_fields(1.0, 0 * c, -A * kh[1] * c, A * kh[0] * c), 1.0, nb)
    np.testing.assert_allclose(Jt, expect, atol=1e-18)
    np.testing.assert_allclose(Jl, 0, atol=1e-18)
    assert cnt.sum() == n - 1
