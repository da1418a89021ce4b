"""Pins of the oracle's linear theory (oracle/theory.py) against what arXiv:1009.0254
prints or implies: Table I, Eq. (Tmat), Eqs. (g-mat-yeo), (noise-yeo), (noise-matrix),
(noise-matrix-k0), Appendix B, Appendix C and continuum hydrodynamics (Sec. II C)."""
import os

import numpy as np
import pytest

from oracle import theory as th

GOLD = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(20100902)


def _load(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def _models():
    yield th.Model(rho0=1.0, cs2=1 / 3, kappa=0.01, kT=1e-4, tau_s=1.0, tau_b=1.0, tau_ghost=1.0)
    yield th.Model(rho0=1.0, cs2=1 / 3, kappa=0.05, kT=1e-4, tau_s=0.8, tau_b=1.0, tau_ghost=1.0)
    yield th.Model(rho0=0.7, cs2=0.265 ** 2, kappa=0.08, kT=1e-7, tau_s=1.0, tau_b=1.0, tau_ghost=1.0)
    yield th.Model(rho0=1.3, cs2=0.15 ** 2, kappa=0.03, kT=2e-5, tau_s=0.6, tau_b=1.4, tau_ghost=0.9)


def _ks():
    ks = [(0.0, 0.0), (np.pi, np.pi), (np.pi, 0.0), (0.3, -1.1)]
    ks += [tuple(RNG.uniform(-np.pi, np.pi, 2)) for _ in range(4)]
    return ks


# --- Table I / Eq. (Tmat) --------------------------------------------------------

def test_basis_matches_printed_matrix():
    printed = np.array([[float(v) for v in r] for r in _load("tmat.txt")])
    assert printed.shape == (9, 9)
    np.testing.assert_array_equal(th.T, printed)


def test_lengths_match_table_I():
    rows = _load("table1_lengths.txt")
    gold = np.array([float(r[1]) / float(r[2]) for r in rows])
    np.testing.assert_allclose(th.N, gold, rtol=0, atol=1e-15)


def test_weighted_orthogonality_and_inverse():
    # Eq. (scalar-prod): w_i T_ai T_bi = N_a delta_ab ; f_i = w_i T_ai m_a / N_a inverts m = T f
    np.testing.assert_allclose(th.T @ np.diag(th.W) @ th.T.T, np.diag(th.N), atol=1e-14)
    np.testing.assert_allclose(th.TINV @ th.T, np.eye(9), atol=1e-14)
    np.testing.assert_allclose(th.W.sum(), 1.0, atol=1e-15)


def test_ideal_equilibrium_has_no_ghost_projection():
    # Sec. III A: with these weights the ideal-gas equilibrium has no ghost components
    for _ in range(5):
        rho = RNG.uniform(0.5, 2)
        u = RNG.uniform(-0.1, 0.1, 2)
        cu = th.C @ u
        feq = th.W * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * u @ u)
        m = th.T @ feq
        np.testing.assert_allclose(m[6:], 0.0, atol=1e-15)
        np.testing.assert_allclose(m[:3], [rho, rho * u[0], rho * u[1]], atol=1e-14)


# --- Appendix B ---------------------------------------------------------------------

def test_laplacian_symbol_matches_stencil_on_plane_waves():
    nx, ny = 12, 10
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    for mx, my in [(0, 1), (3, 2), (6, 5), (1, 0), (5, 3)]:
        kx, ky = 2 * np.pi * mx / nx, 2 * np.pi * my / ny
        a = np.cos(kx * X + ky * Y)
        lap = th.laplacian_stencil(a)
        np.testing.assert_allclose(lap, -th.k2_lattice(kx, ky) * a, atol=1e-13)


def test_laplacian_stencil_weights_and_continuum_limit():
    # the stencil is 2/3 on axis neighbours, 1/6 on diagonals and -10/3 at the centre
    a = np.zeros((7, 7))
    a[3, 3] = 1.0
    lap = th.laplacian_stencil(a)
    np.testing.assert_allclose(lap[3, 3], -10 / 3, atol=1e-15)
    np.testing.assert_allclose([lap[3, 4], lap[4, 3], lap[2, 3], lap[3, 2]], 2 / 3, atol=1e-15)
    np.testing.assert_allclose([lap[4, 4], lap[2, 2], lap[2, 4], lap[4, 2]], 1 / 6, atol=1e-15)
    for k in [1e-2, 3e-2]:
        for th_ in np.linspace(0, np.pi, 5):
            kx, ky = k * np.cos(th_), k * np.sin(th_)
            assert abs(th.k2_lattice(kx, ky) - k * k) < 0.2 * k ** 4
    assert abs(th.k2_lattice(np.pi, np.pi) - 16 / 3) < 1e-14


# --- Sec. III C: G, Omega, Xi ----------------------------------------------------------

@pytest.mark.parametrize("m", list(_models()))
def test_G_printed_equals_ansatz(m):
    # Eq. (g-mat-yeo) is T diag(fbar(k)) T^T S/rho0 by Eq. (f-correl-yeo)
    for kx, ky in _ks():
        G1 = m.G_closed(kx, ky)
        G2 = m.G_ansatz(kx, ky)
        np.testing.assert_allclose(G1, G2, atol=1e-13 * np.abs(G1).max())


@pytest.mark.parametrize("m", list(_models()))
def test_generic_ansatz_with_k_dependent_mass_gives_G(m):
    # Appendix A: Eq. (g-correl) with mu(k) = S(k)/rho0 and fbar(k) reduces to Eq. (g-mat-yeo)
    for kx, ky in _ks():
        S = m.S_k(kx, ky)
        mu = S / m.rho0
        mb = m.mbar(kx, ky)
        fb = m.fbar(kx, ky)
        G = np.outer(mb, mb) * (S / m.rho0 - mu) / m.rho0 + mu * (th.T * fb[None, :]) @ th.T.T
        np.testing.assert_allclose(G, m.G_closed(kx, ky), atol=1e-13 * np.abs(G).max())


def test_ideal_gas_mass_parameter():
    # Appendix A: ideal gas, fbar = w rho0, mu = kT/sigma_s^2 gives <j j> = rho0 kT
    rho0, kT = 1.2, 3e-4
    fb = th.W * rho0
    mu = kT / th.SIGMA_S2
    corr = mu * np.diag(fb)
    jj = th.C.T.astype(float) @ corr @ th.C.astype(float)
    np.testing.assert_allclose(jj, rho0 * kT * np.eye(2), rtol=1e-14)


@pytest.mark.parametrize("m", list(_models()))
def test_Xi_printed_equals_fdt(m):
    # Eq. (noise-yeo) equals Eq. (noise-matrix) evaluated with Eqs. (coll-op-yeo), (g-mat-yeo)
    for kx, ky in _ks():
        X1 = m.Xi_closed(kx, ky)
        X2 = m.Xi_fdt(kx, ky)
        np.testing.assert_allclose(X1, np.real(X2), atol=1e-13 * np.abs(X1).max())


@pytest.mark.parametrize("m", list(_models()))
def test_advection_leaves_G_invariant(m):
    # text above Eq. (noise-yeo): A G A^dagger = G for all k
    for kx, ky in _ks():
        A = m.A(kx, ky)
        G = m.G_closed(kx, ky)
        np.testing.assert_allclose(A @ G @ A.conj().T, G, atol=1e-13 * np.abs(G).max())
        # Eq. (lb-adv): A^-1(k) = A*(k)
        np.testing.assert_allclose(A @ A.conj(), np.eye(9), atol=1e-13)


@pytest.mark.parametrize("m", list(_models()))
def test_long_wavelength_noise(m):
    # Eq. (noise-matrix-k0) is the k -> 0 limit of Eq. (noise-yeo)
    np.testing.assert_allclose(m.Xi_zero(), m.Xi_closed(0.0, 0.0), atol=1e-15 + 1e-13 * m.kT)
    for k in [1e-3, 1e-4]:
        np.testing.assert_allclose(m.Xi_closed(k, 0.3 * k), m.Xi_zero(), atol=10 * k * k * m.kT * 100)
    # conserved rows vanish: no noise on rho, j (Table I, eigenvalue 0)
    X0 = m.Xi_zero()
    assert np.abs(X0[:3]).max() <= 1e-13 * np.abs(X0).max()


@pytest.mark.parametrize("m", list(_models()))
def test_stationarity_lyapunov_returns_G(m):
    # with Xi(k) of Eq. (noise-yeo), the stationary covariance of Eq. (lb-lang-ft) is G(k).
    # Skipped where M(k) has a unit-modulus eigenvalue: k = 0 and k = (pi, 0), (0, pi),
    # where the staggered momentum is an exact invariant of D2Q9 (see the next test).
    for kx, ky in _ks()[1:]:
        if np.abs(np.linalg.eigvals(m.M(kx, ky))).max() > 1 - 1e-9:
            continue
        G = th.lyapunov_G(m, kx, ky, m.Xi_closed(kx, ky))
        np.testing.assert_allclose(G, m.G_closed(kx, ky), atol=1e-10 * np.abs(G).max())


@pytest.mark.parametrize("m", list(_models()))
def test_staggered_momentum_is_invariant_and_unforced(m):
    # at k = (pi, 0) the propagator keeps j_x unchanged (left eigenvector e_2, eigenvalue
    # of modulus 1) and the noise has no component along it, so its variance never
    # relaxes to rho0 kT; the equipartition checks exclude these two wavevectors
    for (kx, ky), a in [((np.pi, 0.0), 1), ((0.0, np.pi), 2)]:
        M = m.M(kx, ky)
        e = np.zeros(9); e[a] = 1.0
        np.testing.assert_allclose(np.abs(e @ M), e, atol=1e-12)
        Am = m.A(-kx, -ky)
        Q = Am @ m.Xi_closed(kx, ky) @ Am.conj().T
        assert abs(e @ Q @ e) < 1e-25


def _continuum_stress_variances(m, kx, ky):
    """<xi_4^2>, <xi_5^2>, <xi_6^2> from the continuum FDT of Eq. (fluct-hydro-fdt-latt)
    with eta (text after Eq. bulkv-yeo) and zeta(k) of Eq. (bulkv-yeo), mapped to the LB
    noise through Eq. (lb-fluct-stress): xi_4 = 3 lambda_b tr R, xi_5 = lambda_s (Rxx - Ryy),
    xi_6 = lambda_s (Rxy + Ryx)/2."""
    eta = m.shear_viscosity()
    zeta = m.bulk_viscosity(kx, ky)
    d = 2
    dl = np.eye(2)
    RR = np.zeros((2, 2, 2, 2))
    for a in range(2):
        for b in range(2):
            for c in range(2):
                for e in range(2):
                    RR[a, b, c, e] = 2 * m.kT * (
                        eta * (dl[a, c] * dl[b, e] + dl[a, e] * dl[b, c] - 2 / d * dl[a, b] * dl[c, e])
                        + zeta * dl[a, b] * dl[c, e])
    lb, ls = m.lam[3], m.lam[4]
    v_tr = np.zeros((2, 2)); v_tr[0, 0] = v_tr[1, 1] = 3 * lb
    v_5 = np.zeros((2, 2)); v_5[0, 0] = ls; v_5[1, 1] = -ls
    v_6 = np.zeros((2, 2)); v_6[0, 1] = v_6[1, 0] = ls / 2
    var = lambda v: np.einsum("ab,abce,ce->", v, RR, v)
    return var(v_tr), var(v_5), var(v_6)


@pytest.mark.parametrize("m", list(_models()))
def test_stress_noise_equals_continuum_fdt(m):
    # Appendix C: the stress-noise variances follow from fluctuating hydrodynamics; they
    # match Xi_44, Xi_55, Xi_66 of Eq. (noise-yeo) (rho = rho0) at every k
    for kx, ky in _ks():
        v4, v5, v6 = _continuum_stress_variances(m, kx, ky)
        X = m.Xi_closed(kx, ky)
        np.testing.assert_allclose([X[3, 3], X[4, 4], X[5, 5]], [v4 * m.rho0 / m.rho0, v5, v6],
                                   rtol=1e-12)


def test_relation_between_stress_and_noise_is_consistent():
    # Eq. (lb-fluct-stress) inverted gives the three relations quoted in Appendix C
    lb, ls = -0.9, -1.3
    xi = RNG.normal(size=3)
    s = th.SIGMA_S2
    R = s * np.array([[xi[0] / (lb * np.sqrt(th.N[3])) + xi[1] / (ls * np.sqrt(th.N[4])), xi[2] / (ls * np.sqrt(th.N[5]))],
                      [xi[2] / (ls * np.sqrt(th.N[5])), xi[0] / (lb * np.sqrt(th.N[3])) - xi[1] / (ls * np.sqrt(th.N[4]))]])
    np.testing.assert_allclose(3 * lb * np.trace(R), xi[0], rtol=1e-14)
    np.testing.assert_allclose(ls * (R[0, 0] - R[1, 1]), xi[1], rtol=1e-14)
    np.testing.assert_allclose(ls * (R[0, 1] + R[1, 0]) / 2, xi[2], rtol=1e-14)


def test_ideal_gas_special_case_is_flat():
    # kappa = 0, cs2 = 1/3: S = 3 rho0 kT and G_aa = N_a rho0 kT / sigma_s^2 at every k
    m = th.Model(rho0=1.1, cs2=1 / 3, kappa=0.0, kT=2e-4, tau_s=0.9, tau_b=1.2, tau_ghost=0.8)
    for kx, ky in _ks():
        G = m.G_closed(kx, ky)
        Tt = m.rho0 * m.kT / th.SIGMA_S2
        np.testing.assert_allclose(np.diag(G)[3:], th.N[3:] * Tt, rtol=1e-13)
        np.testing.assert_allclose(G[0, 0], Tt, rtol=1e-13)
        np.testing.assert_allclose(m.Xi_closed(kx, ky), m.Xi_zero(), atol=1e-18)


# --- Sec. II C: hydrodynamic limit of the propagator ------------------------------------

@pytest.mark.parametrize("m", list(_models()))
def test_propagator_hydrodynamic_eigenvalues(m):
    # transverse momentum decays as exp(-nu k^2), nu = eta/rho0 (Eq. lin-ns3, text after
    # Eq. bulkv-yeo); sound propagates with c_s(k) (Eq. sound-speed-k)
    nu = m.shear_viscosity() / m.rho0
    for k in [0.01, 0.02]:
        for ang in [0.0, 0.4, np.pi / 4]:
            kx, ky = k * np.cos(ang), k * np.sin(ang)
            ev = np.linalg.eigvals(m.M(kx, ky))
            # the shear eigenvalue is the real one closest to 1
            real = ev[np.abs(ev.imag) < 1e-12]
            shear = real[np.argmin(np.abs(real - 1))]
            assert abs(shear - np.exp(-nu * k * k)) < 5 * k ** 4
            cplx = ev[ev.imag > 1e-9]
            snd = cplx[np.argmin(np.abs(np.abs(cplx) - 1))]
            phase = np.angle(snd)
            c = np.sqrt(m.cs2_k(kx, ky))
            assert abs(phase - c * k) < 5 * k ** 3


# --- Sec. III C: positive semidefiniteness (Fig. 5) -------------------------------------

def test_psd_boundary_at_ideal_sound_speed():
    # det of the (4,9) block at k = (pi, pi) is zero at kappa = 0.05 when cs2 = 1/3, tau = 1
    kx = ky = np.pi
    e05 = th.min_eig_block49(th.Model(kappa=0.05, kT=1.0), kx, ky)
    assert abs(e05) < 1e-12
    assert th.min_eig_block49(th.Model(kappa=0.06, kT=1.0), kx, ky) < -1e-3
    assert th.min_eig_block49(th.Model(kappa=0.01, kT=1.0), kx, ky) > 1.0
    # eigenvalue routine agrees with a dense solve of the closed form
    m = th.Model(kappa=0.03, cs2=0.2, kT=1.0, tau_s=0.7)
    for kx, ky in _ks():
        X = m.Xi_closed(kx, ky)
        e = np.linalg.eigvalsh(X[np.ix_([3, 8], [3, 8])]).min()
        np.testing.assert_allclose(th.min_eig_block49(m, kx, ky), e, atol=1e-12)


def test_cholesky_psd():
    for n in [2, 6]:
        for rank in range(1, n + 1):
            B = RNG.normal(size=(n, rank))
            X = B @ B.T
            L = th.cholesky_psd(X)
            assert np.allclose(np.triu(L, 1), 0)
            np.testing.assert_allclose(L @ L.T, X, atol=1e-10 * np.abs(X).max())
            if rank == n:
                np.testing.assert_allclose(L, np.linalg.cholesky(X), atol=1e-10)
    with pytest.raises(ValueError):
        th.cholesky_psd(np.array([[1.0, 0.0], [0.0, -1.0]]))


@pytest.mark.parametrize("m", list(_models()))
def test_noise_factor_reproduces_Xi0(m):
    L = th.noise_factor(m.Xi_zero())
    np.testing.assert_allclose(L @ L.T, m.Xi_zero(), atol=1e-14 * max(1.0, np.abs(m.Xi_zero()).max()))
