"""Pins of the oracle's two-phase model: the Landau double-well bulk free energy of Sec. II A
(Eq. f0-bulk) with p0 = rho df0/drho - f0 and c_s^2 = rho d2f0/drho2, a flat interface
relaxing to the tanh profile of width xi of Eq. (interf-width), and the uncorrelated noise
evaluated with the local density and sound speed (Sec. IV; Sec. V B)."""
import numpy as np
import pytest

import oracle
from oracle import theory as th

WELLS = [th.DoubleWell(0.04, 0.5, 1.0), th.DoubleWell(0.01, 0.1, 1.0)]


@pytest.mark.parametrize("eos", WELLS)
def test_double_well_thermodynamics(eos):
    rho = np.linspace(0.05, 1.3, 57)
    h = 1e-5
    # p0 = rho f0' - f0 with f0' the derivative of f0, and c_s^2 = dp0/drho = rho f0''
    np.testing.assert_allclose(eos.df0(rho), (eos.f0(rho + h) - eos.f0(rho - h)) / (2 * h), atol=1e-9)
    np.testing.assert_allclose(eos.d2f0(rho), (eos.df0(rho + h) - eos.df0(rho - h)) / (2 * h), atol=1e-9)
    np.testing.assert_allclose(eos.cs2(rho), (eos.p0(rho + h) - eos.p0(rho - h)) / (2 * h), atol=1e-9)
    # coexistence: equal bulk pressure and chemical potential df0/drho at rhoV and rhoL
    for r in (eos.rhoV, eos.rhoL):
        assert abs(eos.p0(r)) < 1e-15 and abs(eos.df0(r)) < 1e-15
    # single phase: beta = c_s^2 / (2 rho0 (rhoL - rhoV)^2) (Sec. II A) at both densities
    for r in (eos.rhoV, eos.rhoL):
        assert abs(eos.cs2(r) / (2 * r * (eos.rhoL - eos.rhoV) ** 2) - eos.beta) < 1e-15
    # the spinodal region between them has c_s^2 < 0
    assert eos.cs2(0.5 * (eos.rhoV + eos.rhoL)) < 0
    # Eq. (interf-width): the two forms of xi agree with rho0 and c_s of either phase
    k = 0.03
    for r in (eos.rhoV, eos.rhoL):
        assert abs(eos.width(k) - 4 * np.sqrt(r * k) / np.sqrt(eos.cs2(r))) < 1e-12
    assert eos.surface_tension(k) > 0


@pytest.mark.parametrize("eos", WELLS)
def test_uniform_states_are_fixed_points_of_the_double_well_collision(eos):
    # a uniform state at rest with the Table II equilibrium of its own density (bulk
    # pressure p0(rho) of the double well) is left unchanged by a step: the C core's
    # equation of state is the theory's, at the coexisting densities and between them
    for rho in (eos.rhoV, eos.rhoL, 0.5 * (eos.rhoV + eos.rhoL), 1.2):
        m = th.Model(rho0=rho, cs2=eos.cs2(rho), kappa=0.05, tau_s=0.8, tau_b=1.1, tau_ghost=0.9,
                     p0_rest=eos.p0(rho))
        f = np.broadcast_to(m.rest()[:, None, None], (9, 4, 6)).copy()
        g = oracle.step(f, m, eos=eos)
        np.testing.assert_allclose(g, f, atol=1e-15)
        # and with p0 = cs2 rho instead, the same state is not (p0(rho) != cs2(rho) rho)
        if abs(eos.p0(rho) - eos.cs2(rho) * rho) > 1e-6:
            assert np.abs(oracle.step(f, m) - f).max() > 1e-6


@pytest.mark.parametrize("eos,kappa", [(WELLS[0], 0.03), (WELLS[1], 0.02), (WELLS[0], 0.1)])
def test_flat_interface_relaxes_to_the_tanh_profile_of_width_xi(eos, kappa):
    # A liquid slab in vapour with sharp edges, noise off: the stationary profile is
    # rho(x) = (rhoL + rhoV)/2 + (rhoL - rhoV)/2 tanh(2 x / xi), xi of Eq. (interf-width), with
    # the bulk at the coexisting densities.  The lattice's second differences shorten xi by a
    # relative O(1/xi^2) (0.45/xi^2 here).
    from scipy.optimize import curve_fit
    nx, ny = 128, 2
    L = oracle.Lattice(nx, ny, rho0=0.5 * (eos.rhoV + eos.rhoL), seed=1, eos=eos)
    L.set_params(0.0, kappa, 1.0, 1.0, 1.0, oracle.NOISE_OFF)
    x = np.arange(nx)
    prof = np.where((x >= 32) & (x < 96), eos.rhoL, eos.rhoV)
    for i, r in enumerate(prof):
        m = th.Model(rho0=r, cs2=eos.cs2(r), p0_rest=eos.p0(r))
        L.f[:, :, i] = m.rest()[:, None]
    mass0 = L.f.sum()
    L.step(10000)
    rho = L.f.sum(axis=0)
    assert np.abs(rho[0] - rho[1]).max() < 1e-12              # flat: no y dependence
    assert abs(L.f.sum() - mass0) < 1e-9                       # mass conserved
    xi = eos.width(kappa)
    fun = lambda xx, x0, w, a, b: a + b * np.tanh(2 * (xx - x0) / w)
    p, _ = curve_fit(fun, x[16:64].astype(float), rho[0, 16:64], p0=[32, xi, 0.5 * (eos.rhoL + eos.rhoV),
                                                                    0.5 * (eos.rhoL - eos.rhoV)])
    print("xi: Eq. (interf-width) %.4f, stationary profile %.4f" % (xi, p[1]))
    assert abs(p[1] / xi - 1) < 0.7 / xi ** 2
    assert abs(rho[0, 64] - eos.rhoL) < 1e-3 and abs(rho[0, 0] - eos.rhoV) < 1e-3


@pytest.mark.parametrize("rho,c2", [(1.0, 1 / 3), (0.8, 0.02), (0.3, 0.12), (1.1, 0.0702)])
def test_local_noise_variances_are_xi0_at_the_local_state(rho, c2):
    # the entries the local noise uses are Xi(0) of Eq. (noise-matrix-k0) (the FDT route,
    # -G Omega^T - Omega G - Omega G Omega^T) for a homogeneous system at that density and
    # sound speed
    m = th.Model(rho0=1.0, cs2=1 / 3, kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    x44, x49, x99, x55, x66, x77 = oracle.xi_zero_local(m, np.array([rho]), c2)
    X = th.Model(rho0=rho, cs2=c2, kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9).Xi_zero()
    got = [x44[0], x49[0], x99[0], x55[0], x66[0], x77[0]]
    want = [X[3, 3], X[3, 8], X[8, 8], X[4, 4], X[5, 5], X[6, 6]]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-20)
    assert abs(X[7, 7] - X[6, 6]) < 1e-20


def test_local_noise_at_uniform_density_is_the_uniform_noise():
    # Sec. IV: the uncorrelated noise applies to inhomogeneous systems with local values; at
    # a uniform density it is the long-wavelength noise of Xi(0), draw for draw
    for cs2, rho0 in [(1 / 3, 1.0), (0.15 ** 2, 0.9)]:
        m = th.Model(rho0=rho0, cs2=cs2, kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
        nx, ny = 12, 7
        rho = np.full((ny, nx), rho0)
        a = oracle.local_noise_fields(m, rho, cs2, seed=9, step=4)
        b = oracle.noise_fields(m, oracle.NOISE_LW, nx, ny, 9, 4)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-13 * np.abs(b).max())   # rounding order only


def test_local_noise_covariance_follows_the_density_field():
    # a fixed inhomogeneous density (a double-well interface): the sample covariance of the
    # noise at each node over many steps is Xi(0) at that node's density and c_s^2
    eos = WELLS[0]
    m = th.Model(rho0=0.75, cs2=eos.cs2(0.75), kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    nx, ny = 16, 2
    x = np.arange(nx)
    rho = np.broadcast_to((0.75 + 0.25 * np.tanh((x - 8) / 2.0))[None, :], (ny, nx)).copy()
    c2 = eos.cs2(rho)
    steps = 3000
    acc = np.zeros((9, 9, ny, nx))
    for t in range(steps):
        xi = oracle.local_noise_fields(m, rho, c2, seed=2, step=t)
        acc += np.einsum("ayx,byx->abyx", xi, xi)
    C = acc / steps
    x44, x49, x99, x55, x66, x77 = oracle.xi_zero_local(m, rho, c2)
    # where the local (4,9) block is positive semidefinite the covariance is Xi(0) there
    psd = (x44 >= 0) & (x99 >= 0) & (x44 * x99 >= x49 * x49)
    assert psd.sum() >= 20
    for (a, b), X in [((3, 3), x44), ((8, 8), x99), ((3, 8), x49), ((4, 4), x55), ((5, 5), x66), ((6, 6), x77),
                      ((7, 7), x77)]:
        sd = np.sqrt((np.abs(C[a, a] * C[b, b]) + X ** 2) / steps)
        z = np.abs(C[a, b] - X)[psd] / sd[psd]
        assert z.max() < 5, ((a, b), z.max())
    # no noise on the conserved moments, none between different shear/ghost modes
    assert np.all(C[:3] == 0)
