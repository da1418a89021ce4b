"""Pins of the oracle's deterministic step (oracle/lbref.c): linear dynamics against the
propagator of Eq. (lb-lang-ft), the equilibrium against the pressure tensor of
Eq. (press-ten), conservation (Table I), and internal consistency."""
import numpy as np
import pytest

import oracle
from oracle import theory as th

RNG = np.random.default_rng(7)

MODELS = [
    th.Model(rho0=1.0, cs2=1 / 3, kappa=0.01, kT=0.0, tau_s=1.0, tau_b=1.0, tau_ghost=1.0),
    th.Model(rho0=1.0, cs2=1 / 3, kappa=0.02, kT=0.0, tau_s=0.8, tau_b=1.1, tau_ghost=0.9),
    th.Model(rho0=0.9, cs2=0.265 ** 2, kappa=0.08, kT=0.0, tau_s=1.0, tau_b=1.0, tau_ghost=1.0),
    th.Model(rho0=1.2, cs2=0.15 ** 2, kappa=0.03, kT=0.0, tau_s=0.6, tau_b=1.4, tau_ghost=0.7),
]


def _plane_wave_state(m, nx, ny, mx, my, v, eps):
    kx, ky = 2 * np.pi * mx / nx, 2 * np.pi * my / ny
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ph = np.exp(-1j * (kx * X + ky * Y))
    dm = np.real(eps * v[:, None, None] * ph[None])
    f = m.fbar()[:, None, None] + np.einsum("ia,ayx->iyx", th.TINV, dm)
    return f, ph, kx, ky


@pytest.mark.parametrize("m", MODELS)
def test_rest_state_is_a_fixed_point(m):
    f = np.broadcast_to(m.fbar()[:, None, None], (9, 6, 10)).copy()
    g = oracle.step(f, m)
    np.testing.assert_allclose(g, f, atol=1e-15)


@pytest.mark.parametrize("m", MODELS)
@pytest.mark.parametrize("mx,my", [(1, 0), (3, -2), (5, 4), (8, 6)])
def test_small_amplitude_dynamics_follow_the_propagator(m, mx, my):
    # kT = 0: a small plane wave evolves as dm(k, t) = M(k)^t dm(k, 0), Eq. (lb-lang-ft),
    # with Omega of Eq. (coll-op-yeo) and A of Eq. (lb-adv); nonlinear terms are O(eps^2)
    nx, ny = 16, 12
    v = RNG.normal(size=9) + 1j * RNG.normal(size=9)
    eps = 1e-7
    f, ph, kx, ky = _plane_wave_state(m, nx, ny, mx, my, v, eps)
    M = m.M(kx, ky)
    vt = v.copy()
    for _ in range(15):
        f = oracle.step(f, m)
        vt = M @ vt
    dm = np.einsum("ai,iyx->ayx", th.T, f - m.fbar()[:, None, None])
    pred = np.real(eps * vt[:, None, None] * ph[None])
    assert np.abs(dm - pred).max() < 1e-5 * eps


def _lattice_gradient(rho):
    gx = np.zeros_like(rho)
    gy = np.zeros_like(rho)
    for i in range(1, 9):
        cx, cy = th.C[i]
        nb = np.roll(rho, shift=(-cy, -cx), axis=(0, 1))
        gx += 3 * th.W[i] * cx * nb
        gy += 3 * th.W[i] * cy * nb
    return gx, gy


@pytest.mark.parametrize("m", MODELS)
def test_relaxed_second_moment_is_the_pressure_tensor(m):
    # with every tau = 1 (lambda = -1) the collision sets m_a = m_a^eq for a >= 4, so the
    # post-collision second moment is P^th + rho u u, Eq. (press-ten) with p0 = cs2 rho
    mm = th.Model(m.rho0, m.cs2, m.kappa, 0.0, 1.0, 1.0, 1.0)
    nx, ny = 12, 10
    f = mm.fbar()[:, None, None] * (1 + 0.05 * RNG.normal(size=(9, ny, nx)))
    sites = np.arange(nx * ny)
    fs = oracle.collide_sites(f, mm, sites)                      # (n, 9)
    rho = f.sum(axis=0)
    jx = np.einsum("i,iyx->yx", th.C[:, 0].astype(float), f)
    jy = np.einsum("i,iyx->yx", th.C[:, 1].astype(float), f)
    lap = th.laplacian_stencil(rho)
    gx, gy = _lattice_gradient(rho)
    p0 = mm.cs2 * rho
    iso = p0 - mm.kappa * rho * lap - 0.5 * mm.kappa * (gx * gx + gy * gy)
    Pxx = iso + mm.kappa * gx * gx + jx * jx / rho
    Pyy = iso + mm.kappa * gy * gy + jy * jy / rho
    Pxy = mm.kappa * gx * gy + jx * jy / rho
    cx = th.C[:, 0].astype(float)
    cy = th.C[:, 1].astype(float)
    np.testing.assert_allclose(fs @ (cx * cx), Pxx.ravel(), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(fs @ (cy * cy), Pyy.ravel(), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(fs @ (cx * cy), Pxy.ravel(), rtol=1e-12, atol=1e-14)
    # conserved moments untouched, vector ghosts relaxed to 0
    np.testing.assert_allclose(fs.sum(axis=1), rho.ravel(), rtol=1e-14)
    np.testing.assert_allclose(fs @ th.T[6], 0.0, atol=1e-14)
    np.testing.assert_allclose(fs @ th.T[7], 0.0, atol=1e-14)


def test_collide_sites_matches_full_step():
    m = th.Model(1.0, 1 / 3, 0.02, 1e-4, 0.8, 1.0, 1.0)
    nx, ny = 9, 7
    f = m.fbar()[:, None, None] * (1 + 0.02 * RNG.normal(size=(9, ny, nx)))
    xi = 1e-3 * RNG.normal(size=(9, ny, nx))
    xi[:3] = 0
    g = oracle.step(f, m, xi)
    sites = np.arange(nx * ny)
    fs = oracle.collide_sites(f, m, sites, xi.reshape(9, -1).T)
    # stream by hand: f_i(r + c_i) = f*_i(r)
    h = np.empty_like(f)
    for i in range(9):
        h[i] = np.roll(fs[:, i].reshape(ny, nx), shift=(th.C[i, 1], th.C[i, 0]), axis=(0, 1))
    np.testing.assert_allclose(g, h, atol=1e-15)


@pytest.mark.parametrize("mode", [oracle.NOISE_LW, oracle.NOISE_FULL, oracle.NOISE_DIAG])
def test_noise_conserves_mass_and_momentum(mode):
    lat = oracle.Lattice(12, 8, rho0=1.0, seed=5)
    lat.set_params(kT=1e-3, kappa=0.02, tau_s=0.8, tau_b=1.0, tau_ghost=1.0, noise_mode=mode)
    m0 = lat.moments().sum(axis=(1, 2))
    lat.step(40)
    m1 = lat.moments().sum(axis=(1, 2))
    np.testing.assert_allclose(m1[:3], m0[:3], atol=1e-12)
    assert np.abs(lat.f - lat.model.fbar()[:, None, None]).max() > 1e-3   # noise did act


def _gradient_swapped_diagonals(rho):
    """The gradient with the density neighbours at (1, 1) and (-1, 1) exchanged: the
    mistake of a mis-wired diagonal in a kernel's density ring (the Laplacian, symmetric
    in the four diagonals, does not see it)."""
    gx = np.zeros_like(rho)
    gy = np.zeros_like(rho)
    for i in range(1, 9):
        cx, cy = th.C[i]
        sx, sy = th.C[{5: 6, 6: 5}.get(i, i)]
        nb = np.roll(rho, shift=(-sy, -sx), axis=(0, 1))
        gx += 3 * th.W[i] * cx * nb
        gy += 3 * th.W[i] * cy * nb
    return gx, gy


@pytest.mark.parametrize("case", ["ideal", "nonideal"])
def test_nonlinear_parity_state_resolves_the_second_order_terms(case):
    # The state of the GPU nonlinear parity tests (tests/nonlinear_case.py): each
    # second-order term of the Table II equilibrium, and a swap of two diagonal density
    # neighbours, moves the post-collision populations by >= 100 x their tolerance.
    import nonlinear_case as nl
    m = nl.model(case)
    nx, ny = 64, 48
    f = nl.state(case, nx, ny, seed=101)
    tol = nl.tolerance(f)
    rho = f.sum(axis=0)
    drho = rho - m.rho0
    jx = np.einsum("i,iyx->yx", th.C[:, 0].astype(float), f)
    jy = np.einsum("i,iyx->yx", th.C[:, 1].astype(float), f)
    lap = th.laplacian_stencil(rho)
    gx, gy = _lattice_gradient(rho)
    k = m.kappa

    def dfstar(dm):
        # change of f* = T^-1 (m + lambda (m - m^eq)) caused by a change dm of m^eq
        return np.einsum("ia,ayx->iyx", th.TINV, -m.lam[:, None, None] * dm)

    def moments(**kw):
        dm = np.zeros((9, ny, nx))
        for a, v in kw.items():
            dm[int(a[1:])] = v
        return dm

    # the contribution map against the oracle itself: the whole kappa dependence of f*
    sites = np.arange(nx * ny)
    m0 = th.Model(m.rho0, m.cs2, 0.0, m.kT, m.tau_s, m.tau_b, m.tau_ghost)
    got = (oracle.collide_sites(f, m, sites) - oracle.collide_sites(f, m0, sites)).T.reshape(9, ny, nx)
    want = dfstar(moments(m3=-6 * k * rho * lap, m4=k * (gx * gx - gy * gy), m5=k * gx * gy,
                          m8=6 * k * rho * lap - 3 * k * (gx * gx + gy * gy)))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)

    sgx, sgy = _gradient_swapped_diagonals(rho)
    terms = {
        "rho u u": moments(m3=3 * (jx * jx + jy * jy) / rho, m4=(jx * jx - jy * jy) / rho, m5=jx * jy / rho),
        "kappa grad grad (shear)": moments(m4=k * (gx * gx - gy * gy), m5=k * gx * gy),
        "-3 kappa |grad rho|^2 (m9)": moments(m8=-3 * k * (gx * gx + gy * gy)),
        "kappa drho lap rho": moments(m3=-6 * k * drho * lap, m8=6 * k * drho * lap),
        "diagonals swapped": moments(m4=k * ((sgx * sgx - sgy * sgy) - (gx * gx - gy * gy)), m5=k * (sgx * sgy - gx * gy),
                                     m8=-3 * k * ((sgx * sgx + sgy * sgy) - (gx * gx + gy * gy))),
    }
    for name, dm in terms.items():
        size = np.abs(dfstar(dm)).max()
        print("%s %s: %.2e = %.0f x tolerance %.2e" % (case, name, size, size / tol, tol))
        assert size >= 100 * tol, (name, size, tol)


def test_the_diverging_request_of_the_watchdog_test_diverges():
    # tests/nonlinear_case.py DIVERGING: the oracle's own FP64 run of it leaves the finite
    # numbers, so the served run of the same request must be reported LB_ENONFINITE
    import nonlinear_case as nl
    d = nl.DIVERGING
    m = nl.diverging_model()
    f = nl.diverging_state()
    assert np.isfinite(oracle.step(f, m)).all()          # a sane start
    with np.errstate(all="ignore"):
        for _ in range(d["steps"]):
            f = oracle.step(f, m)
    assert not np.isfinite(f).all()
    assert not np.isfinite(f.sum())
