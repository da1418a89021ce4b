"""Pins of the oracle's noise (Sec. IV of arXiv:1009.0254) and of the equilibrium
statistics it produces (Sec. V A, the equilibration ratios of Figs. 3 and 4)."""
import numpy as np
import pytest

import oracle
from oracle import theory as th


def _xi_samples(model, mode, nx, ny, steps, seed=11):
    L0 = None
    out = []
    for t in range(steps):
        out.append(oracle.noise_fields(model, mode, nx, ny, seed, t, L0))
    return np.array(out)                                  # (steps, 9, ny, nx)


@pytest.mark.parametrize("mode", [oracle.NOISE_LW, oracle.NOISE_DIAG])
def test_uncorrelated_noise_covariance(mode):
    # Sec. IV: xi = L nu with L L^T = Xi(0) (LW) or diag Xi(0) (ideal-gas-like, DIAG);
    # c_s != sigma_s so that Xi_49(0) != 0
    m = th.Model(rho0=1.0, cs2=0.2 ** 2, kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.0, tau_ghost=1.2)
    X0 = m.Xi_zero()
    target = X0 if mode == oracle.NOISE_LW else np.diag(np.diag(X0))
    assert abs(X0[3, 8]) > 0.1 * np.sqrt(X0[3, 3] * X0[8, 8])
    xi = _xi_samples(m, mode, 32, 32, 20)
    v = xi.transpose(1, 0, 2, 3).reshape(9, -1)
    Nn = v.shape[1]
    C = v @ v.T / Nn
    assert np.all(C[:3] == 0) and np.all(C[:, :3] == 0)       # no noise on rho, j
    C, target = C[3:, 3:], target[3:, 3:]
    sig = np.sqrt((np.outer(np.diag(target), np.diag(target)) + target ** 2) / Nn)
    assert np.all(np.abs(C - target) <= 5 * sig)
    # spatially white: neighbour correlation vanishes
    nb = (xi * np.roll(xi, 1, axis=3)).mean(axis=(0, 2, 3))
    assert np.all(np.abs(nb[3:]) <= 5 * np.diag(target) / np.sqrt(Nn))


def test_hermitian_eta_field():
    nx, ny = 8, 6
    e1, e2 = oracle.eta_field(nx, ny, seed=3, step=9)
    conj = oracle._fft_conj_index(nx, ny)
    for e in (e1, e2):
        flat = e.ravel()
        np.testing.assert_array_equal(flat[conj.ravel()], np.conj(flat))
        selfc = conj.ravel() == np.arange(nx * ny)
        assert np.all(flat[selfc].imag == 0)
    # unit variance over many draws
    acc = np.zeros((ny, nx))
    for t in range(400):
        e1, _ = oracle.eta_field(nx, ny, seed=3, step=t)
        acc += np.abs(e1) ** 2
    assert np.all(np.abs(acc / 400 - 1) < 5 * np.sqrt(2 / 400))


def test_full_noise_is_L_eta_in_k_space():
    # the transform back and the forward transform of Sec. III are inverse: the
    # spectrum of the real-space noise field is exactly L(k) eta(k)
    m = th.Model(rho0=1.0, cs2=1 / 3, kappa=0.03, kT=1e-4, tau_s=0.8)
    nx, ny = 16, 8
    x4, x9 = oracle.xi49_full(m, nx, ny, seed=4, step=2)
    e1, e2 = oracle.eta_field(nx, ny, seed=4, step=2)
    KX, KY = th.lattice_k(nx, ny)
    L44, L49, L94, L99 = oracle.block49_factor(m, KX, KY)
    assert np.all(L49 == 0)
    np.testing.assert_allclose(oracle.unitary_ft(x4), L44 * e1, atol=1e-14)
    np.testing.assert_allclose(oracle.unitary_ft(x9), L94 * e1 + L99 * e2, atol=1e-14)
    # L L^T reproduces the (4,9) block of Eq. (noise-yeo) at every k
    for (j, i) in [(0, 0), (3, 5), (4, 8), (7, 15)]:
        X = m.Xi_closed(KX[j, i], KY[j, i])
        Lm = np.array([[L44[j, i], 0], [L94[j, i], L99[j, i]]])
        np.testing.assert_allclose(Lm @ Lm.T, X[np.ix_([3, 8], [3, 8])], atol=1e-18)


def test_full_noise_spectrum_statistics():
    m = th.Model(rho0=1.0, cs2=0.25 ** 2, kappa=0.05, kT=1e-4, tau_s=1.0)
    nx = ny = 16
    KX, KY = th.lattice_k(nx, ny)
    steps = 300
    P44 = np.zeros((ny, nx)); P99 = np.zeros((ny, nx)); P49 = np.zeros((ny, nx))
    for t in range(steps):
        x4, x9 = oracle.xi49_full(m, nx, ny, seed=8, step=t)
        a, b = oracle.unitary_ft(x4), oracle.unitary_ft(x9)
        P44 += np.abs(a) ** 2; P99 += np.abs(b) ** 2; P49 += (a * np.conj(b)).real
    X = np.array([[m.Xi_closed(KX[j, i], KY[j, i]) for i in range(nx)] for j in range(ny)])
    # aggregate in 4 shells of k^2; each entry is an average of steps*count draws
    k2 = th.k2_lattice(KX, KY)
    edges = np.quantile(k2, [0, 0.25, 0.5, 0.75, 1.0])
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (k2 >= lo) & (k2 <= hi)
        nS = sel.sum() * steps
        for P, ab in [(P44, (3, 3)), (P99, (8, 8))]:
            ratio = P[sel].sum() / (steps * X[sel][:, ab[0], ab[1]].sum())
            assert abs(ratio - 1) < 5 * np.sqrt(2.0 / nS)
        c = P49[sel].sum() / steps
        ref = X[sel][:, 3, 8].sum()
        sd = np.sqrt((X[sel][:, 3, 3] * X[sel][:, 8, 8]).sum() / steps)
        assert abs(c - ref) < 5 * sd


def _equilibration_ratios(lat, burn, samples, every, G_of_k):
    nx, ny = lat.nx, lat.ny
    KX, KY = th.lattice_k(nx, ny)
    lat.step(burn)
    acc = np.zeros((9, ny, nx))
    for _ in range(samples):
        lat.step(every)
        dm = lat.moments() - lat.model.mbar()[:, None, None]
        acc += np.abs(np.array([oracle.unitary_ft(dm[a]) for a in range(9)])) ** 2
    acc /= samples
    G = np.array([[np.diag(G_of_k(KX[j, i], KY[j, i])).real for i in range(nx)] for j in range(ny)])
    ratio = acc / G.transpose(2, 0, 1)
    keep = np.ones((ny, nx), bool)
    keep[0, 0] = False                   # k = 0: frozen by conservation
    keep[0, nx // 2] = False             # staggered momentum invariants (see theory tests)
    keep[ny // 2, 0] = False
    return ratio, keep


@pytest.mark.slow
def test_full_noise_equilibrates_every_mode():
    # Sec. V A: with the correlated noise of Eq. (noise-yeo) every mode equilibrates,
    # <|dm_a(k)|^2> / G_aa(k) = 1 (Fig. 3); kappa = 0.08, c_s = 0.265, tau = 1
    lat = oracle.Lattice(12, 12, rho0=1.0, cs2=0.265 ** 2, seed=77)
    lat.set_params(kT=1e-6, kappa=0.08, tau_s=1.0, tau_b=1.0, tau_ghost=1.0, noise_mode=oracle.NOISE_FULL)
    ratio, keep = _equilibration_ratios(lat, burn=400, samples=1500, every=2, G_of_k=lat.model.G_closed)
    for a in range(9):
        r = ratio[a][keep]
        assert abs(r.mean() - 1) < 0.04, (a, r.mean())


@pytest.mark.slow
def test_long_wavelength_noise_matches_its_own_stationary_theory():
    # LW noise (Eq. noise-matrix-k0 used at every k): the stationary spectrum is the
    # solution of G = M G M^H + A(-k) Xi(0) A(-k)^H; it tends to G(k) as k -> 0
    m0 = th.Model(rho0=1.0, cs2=0.15 ** 2, kappa=0.03, kT=1e-6, tau_s=1.0, tau_b=1.0, tau_ghost=1.0)
    lat = oracle.Lattice(12, 12, rho0=1.0, cs2=0.15 ** 2, seed=78)
    lat.set_params(kT=1e-6, kappa=0.03, tau_s=1.0, tau_b=1.0, tau_ghost=1.0, noise_mode=oracle.NOISE_LW)
    X0 = m0.Xi_zero()

    def G_lw(kx, ky):
        if kx == 0 and ky == 0:
            return m0.G_closed(0.0, 0.0)
        if np.abs(np.linalg.eigvals(m0.M(kx, ky))).max() > 1 - 1e-9:
            return m0.G_closed(kx, ky)
        return th.lyapunov_G(m0, kx, ky, X0)

    ratio, keep = _equilibration_ratios(lat, burn=400, samples=1500, every=2, G_of_k=G_lw)
    for a in range(9):
        r = ratio[a][keep]
        assert abs(r.mean() - 1) < 0.04, (a, r.mean())


@pytest.mark.parametrize("cs2,kappa", [(1 / 3, 0.03), (0.25 ** 2, 0.05), (0.265 ** 2, 0.08)])
def test_eigen_factor_reproduces_the_noise_matrix(cs2, kappa):
    # Sec. IV: L = S diag(sqrt(e)) with S the eigenvectors is the alternative to Cholesky;
    # either must satisfy L L^T = Xi, at k = 0 (9x9) and for the (4,9) block at every k
    m = th.Model(rho0=1.0, cs2=cs2, kappa=kappa, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    X0 = m.Xi_zero()
    for factor in ("cholesky", "eigen"):
        L = th.noise_factor(X0, factor)
        np.testing.assert_allclose(L @ L.T, X0, atol=1e-14 * np.abs(X0).max(), rtol=0)
    Le = th.noise_factor(X0, "eigen")
    assert Le[3, 8] != 0.0 or X0[3, 8] == 0.0          # not triangular when Xi49 != 0
    nx, ny = 16, 8
    KX, KY = th.lattice_k(nx, ny)
    l11, l12, l21, l22 = oracle.block49_factor(m, KX, KY, "eigen")
    for (j, i) in [(0, 0), (3, 5), (4, 8), (7, 15), (2, 3)]:
        X = m.Xi_closed(KX[j, i], KY[j, i])[np.ix_([3, 8], [3, 8])]
        Lm = np.array([[l11[j, i], l12[j, i]], [l21[j, i], l22[j, i]]])
        np.testing.assert_allclose(Lm @ Lm.T, X, atol=1e-14 * np.abs(X).max())
        # the columns of L are eigenvectors scaled by sqrt(eigenvalues), largest first
        e = np.linalg.eigvalsh(X)
        np.testing.assert_allclose(np.sort(np.sum(Lm * Lm, axis=0)), np.sort(e), atol=1e-14 * np.abs(X).max())
        assert np.sum(Lm[:, 0] ** 2) >= np.sum(Lm[:, 1] ** 2) - 1e-20


def test_eigen_factor_lw_noise_statistics():
    # the realisations differ from Cholesky but the covariance of xi is the same Xi(0)
    m = th.Model(rho0=1.0, cs2=0.15 ** 2, kappa=0.03, kT=1e-4, tau_s=1.0)
    nx = ny = 64
    acc = np.zeros((9, 9))
    steps = 40
    for t in range(steps):
        xi = oracle.noise_fields(m, oracle.NOISE_LW, nx, ny, seed=5, step=t, factor="eigen").reshape(9, -1)
        acc += xi @ xi.T
    C = acc / (steps * nx * ny)
    X0 = m.Xi_zero()
    ns = steps * nx * ny
    for a in range(3, 9):
        for b in range(3, 9):
            sd = np.sqrt((X0[a, a] * X0[b, b] + X0[a, b] ** 2) / ns)
            assert abs(C[a, b] - X0[a, b]) < 5 * sd + 1e-30, (a, b)


# --- correlated noise built in real space (2 x 2 stencil, oracle.xi49_stencil) -----------

STENCIL_MODELS = [
    th.Model(rho0=1.0, cs2=1 / 3, kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9),
    th.Model(rho0=0.9, cs2=0.265 ** 2, kappa=0.08, kT=1e-7, tau_s=1.0, tau_b=1.0, tau_ghost=1.0),
    th.Model(rho0=1.2, cs2=0.2 ** 2, kappa=0.02, kT=1e-4, tau_s=0.7, tau_b=1.3, tau_ghost=0.8),
]


@pytest.mark.parametrize("m", STENCIL_MODELS)
@pytest.mark.parametrize("factor", ["cholesky", "eigen"])
@pytest.mark.parametrize("nx,ny", [(12, 10), (16, 16), (7, 5)])
def test_stencil_noise_has_the_noise_matrix_at_every_k(m, factor, nx, ny):
    # The construction is linear in the white fields: xi = K * nu.  Its impulse responses
    # give the transfer function K(k) = sum_d K(d) e^{i k.d}, and the covariance of xi(k)
    # for unit white nu is sum over the 8 inputs of K K^H.  It must equal the (4,9) block
    # of the printed Eq. (noise-yeo) at every wavevector of the lattice, any size.
    Ls = oracle.stencil_factors(m, factor)
    n = nx * ny
    cov = np.zeros((ny, nx, 2, 2), dtype=complex)
    for f in range(4):
        for c in range(2):
            nu = np.zeros((4, 2, ny, nx))
            nu[f, c, 0, 0] = 1.0
            resp = oracle.stencil_combine(nu, Ls)                  # (2, ny, nx)
            K = np.fft.ifft2(resp, axes=(1, 2)) * n               # sum_r resp(r) e^{+i k.r}
            cov += np.einsum("iyx,jyx->yxij", K, np.conj(K))
    KX, KY = th.lattice_k(nx, ny)
    for j in range(ny):
        for i in range(nx):
            X = m.Xi_closed(KX[j, i], KY[j, i])[np.ix_([3, 8], [3, 8])]
            np.testing.assert_allclose(cov[j, i], X, rtol=0, atol=1e-13 * np.abs(X).max())


def test_stencil_noise_is_local_and_uses_four_independent_fields():
    # xi(r) depends on the draws of r, r - e_x, r - e_y, r - e_x - e_y only, and every
    # field enters (dropping one changes the result)
    m = STENCIL_MODELS[0]
    nx, ny = 9, 7
    nu = oracle.stencil_fields(nx, ny, seed=5, step=3)
    Ls = oracle.stencil_factors(m)
    base = oracle.stencil_combine(nu, Ls)
    q = (4, 3)                                                  # (y, x) of a perturbed node
    pert = nu.copy()
    pert[:, :, q[0], q[1]] += 1.0
    diff = np.abs(oracle.stencil_combine(pert, Ls) - base).max(axis=0)
    changed = set(zip(*np.nonzero(diff > 1e-15)))
    assert changed == {(4, 3), (4, 4), (5, 3), (5, 4)}          # r = q, q + e_x, q + e_y, q + e_x + e_y
    for f in range(4):
        drop = nu.copy()
        drop[f] = 0.0
        assert np.abs(oracle.stencil_combine(drop, Ls) - base).max() > 1e-8
    # the sampled-site version agrees with the field
    sites = np.array([0, 5, nx - 1, nx * (ny - 1), nx * ny - 1, 31])
    x4, x9 = oracle.xi49_stencil(m, nx, ny, seed=5, step=3)
    at = oracle.xi49_stencil_at(m, nx, ny, 5, 3, sites)
    np.testing.assert_allclose(at[:, 0], x4.ravel()[sites], atol=1e-15)
    np.testing.assert_allclose(at[:, 1], x9.ravel()[sites], atol=1e-15)


def test_stencil_noise_spectrum_statistics():
    # the draws behind the construction are the stated ones: the sampled spectrum of the
    # generated fields matches Xi(k) in every k^2 shell, like the Fourier construction's
    m = th.Model(rho0=1.0, cs2=0.25 ** 2, kappa=0.05, kT=1e-4, tau_s=1.0)
    nx, ny = 16, 12
    KX, KY = th.lattice_k(nx, ny)
    steps = 300
    P44 = np.zeros((ny, nx)); P99 = np.zeros((ny, nx)); P49 = np.zeros((ny, nx))
    for t in range(steps):
        x4, x9 = oracle.xi49_stencil(m, nx, ny, seed=8, step=t)
        a, b = oracle.unitary_ft(x4), oracle.unitary_ft(x9)
        P44 += np.abs(a) ** 2; P99 += np.abs(b) ** 2; P49 += (a * np.conj(b)).real
    X = np.array([[m.Xi_closed(KX[j, i], KY[j, i]) for i in range(nx)] for j in range(ny)])
    k2 = th.k2_lattice(KX, KY)
    edges = np.quantile(k2, [0, 0.25, 0.5, 0.75, 1.0])
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (k2 >= lo) & (k2 <= hi)
        nS = sel.sum() * steps
        for P, ab in [(P44, (3, 3)), (P99, (8, 8))]:
            ratio = P[sel].sum() / (steps * X[sel][:, ab[0], ab[1]].sum())
            assert abs(ratio - 1) < 5 * np.sqrt(2.0 / nS)
        c = P49[sel].sum() / steps
        ref = X[sel][:, 3, 8].sum()
        sd = np.sqrt((X[sel][:, 3, 3] * X[sel][:, 8, 8]).sum() / steps)
        assert abs(c - ref) < 5 * sd


def test_stencil_noise_needs_psd_at_both_ends_of_the_k2_range():
    # kappa = 0.06 at cs2 = 1/3: Xi is not positive semidefinite at large k^2
    m = th.Model(rho0=1.0, cs2=1 / 3, kappa=0.06, kT=1e-4, tau_s=1.0)
    with pytest.raises(ValueError):
        oracle.stencil_factors(m)


@pytest.mark.slow
def test_stencil_noise_equilibrates_every_mode():
    # Sec. V A with the real-space construction on a lattice whose sides are not powers of
    # two: every mode equilibrates, <|dm_a(k)|^2> / G_aa(k) = 1 (Fig. 3 parameters)
    lat = oracle.Lattice(12, 10, rho0=1.0, cs2=0.265 ** 2, seed=79)
    lat.set_params(kT=1e-6, kappa=0.08, tau_s=1.0, tau_b=1.0, tau_ghost=1.0, noise_mode=oracle.NOISE_FULL_RS)
    ratio, keep = _equilibration_ratios(lat, burn=400, samples=1500, every=2, G_of_k=lat.model.G_closed)
    for a in range(9):
        r = ratio[a][keep]
        assert abs(r.mean() - 1) < 0.04, (a, r.mean())
