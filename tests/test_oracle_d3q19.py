"""Pins of the D3Q19 oracle (oracle/d3q19.py), the paper's model carried to three dimensions
(Sec. IV: the noise derivation holds on any DdQn lattice).  Each test checks the oracle
against something other than itself: the lattice's isotropy, the second moment against the
pressure tensor of Eq. (press-ten), the independent D2Q9 C core on fields that are uniform
along one axis, Navier-Stokes shear and sound modes, closed forms of Xi(0) derived by hand,
and equipartition of the ideal fluctuating gas."""
import numpy as np
import pytest

import oracle
from oracle import d3q19 as d3
from oracle import theory as th
from paper_1009_0254_gb300 import synth

S2 = 1.0 / 3.0


def test_lattice_weights_are_isotropic_to_fourth_order():
    C, W = d3.C.astype(float), d3.W
    assert len({tuple(c) for c in d3.C}) == 19
    assert (d3.C[d3.OPP] == -d3.C).all()
    assert abs(W.sum() - 1) < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia->a", W, C), 0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", W, C, C), S2 * np.eye(3), atol=1e-16)
    d = np.eye(3)
    iso4 = S2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d))
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic,id->abcd", W, C, C, C, C), iso4, atol=1e-16)
    # odd moments vanish
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", W, C, C, C), 0, atol=1e-16)


def test_basis_is_weighted_orthogonal_and_spans_the_hydrodynamic_moments():
    G = (d3.T * d3.W) @ d3.T.T
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-15
    np.testing.assert_allclose(d3.T @ d3.TINV, np.eye(19), atol=1e-14)
    # the normalisers of the mode table, evaluated by hand from the polynomials
    want = [1, 1 / 3, 1 / 3, 1 / 3, 2 / 3, 4 / 3, 4 / 9, 1 / 9, 1 / 9, 1 / 9, 2 / 3, 2 / 3, 2 / 3,
            2 / 9, 2 / 9, 2 / 9, 2, 4 / 3, 4 / 9]
    np.testing.assert_allclose(d3.N, want, rtol=1e-14)
    # the second-moment tensor of any population vector follows from m0 and m4..m9
    rng = np.random.default_rng(0)
    f = rng.random(19)
    m = d3.T @ f
    Pi = np.einsum("i,ia,ib->ab", f, d3.C.astype(float), d3.C.astype(float))
    tr = m[0] + m[4]
    pxx = (m[5] + tr) / 3
    pyy = (tr - pxx + m[6]) / 2
    pzz = (tr - pxx - m[6]) / 2
    np.testing.assert_allclose([pxx, pyy, pzz, m[7], m[8], m[9]],
                               [Pi[0, 0], Pi[1, 1], Pi[2, 2], Pi[0, 1], Pi[1, 2], Pi[2, 0]], rtol=1e-14)


def _wave(n, k):
    return 2 * np.pi * k / n


def test_density_stencils_approach_the_derivatives():
    # a plane wave of long wavelength: the stencils' Laplacian and gradient agree with the
    # analytic derivatives up to the O(k^4) and O(k^3) truncation of Appendix B's stencils
    nx, ny, nz = 32, 16, 24
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kx, ky, kz = _wave(nx, 1), _wave(ny, 1), _wave(nz, 1)
    ph = kx * x + ky * y + kz * z
    rho = 1.0 + 0.1 * np.sin(ph)
    lap, grad = d3.density_stencils(rho)
    k2 = kx * kx + ky * ky + kz * kz
    np.testing.assert_allclose(lap, -k2 * 0.1 * np.sin(ph), atol=0.1 * k2 * k2 / 3)
    for g, kk in zip(grad, (kx, ky, kz)):
        np.testing.assert_allclose(g, kk * 0.1 * np.cos(ph), atol=0.1 * k2 ** 1.5 / 2)


def test_equilibrium_carries_the_pressure_tensor():
    # sum_i f^eq_i c_a c_b = P^th_ab + rho u_a u_b with P^th of Eq. (press-ten), p0 = cs2 rho;
    # the first moments are rho and j; the third moment is sigma_s^2 (j_a d_bc + perms)
    rng = np.random.default_rng(1)
    shape = (5, 4, 6)
    rho = 1.0 + 0.2 * rng.random(shape)
    j = 0.05 * rng.standard_normal((3,) + shape)
    lap = rng.standard_normal(shape)
    grad = 0.3 * rng.standard_normal((3,) + shape)
    cs2, kappa = 0.21, 0.07
    m = d3.equilibrium_moments(rho, j, lap, grad, cs2, kappa)
    f = np.einsum("ia,a...->i...", d3.TINV, m)
    C = d3.C.astype(float)
    np.testing.assert_allclose(f.sum(axis=0), rho, rtol=1e-14)
    np.testing.assert_allclose(np.einsum("ia,i...->a...", C, f), j, atol=1e-15)
    u = j / rho
    g2 = (grad ** 2).sum(axis=0)
    P2 = np.einsum("ia,ib,i...->ab...", C, C, f)
    for a in range(3):
        for b in range(3):
            want = rho * u[a] * u[b] + kappa * grad[a] * grad[b]
            if a == b:
                want = want + cs2 * rho - kappa * rho * lap - 0.5 * kappa * g2
            np.testing.assert_allclose(P2[a, b], want, atol=1e-14)
    P3 = np.einsum("ia,ib,ic,i...->abc...", C, C, C, f)
    d = np.eye(3)
    want3 = S2 * (np.einsum("a...,bc->abc...", j, d) + np.einsum("b...,ac->abc...", j, d)
                  + np.einsum("c...,ab->abc...", j, d))
    np.testing.assert_allclose(P3, want3, atol=1e-14)


@pytest.mark.parametrize("cs2,kappa", [(S2, 0.0), (0.2, 0.05), (0.1, 0.01)])
def test_rest_state_is_a_fixed_point(cs2, kappa):
    # the pressure cs2 rho0 sits on the moving populations (w_i 3 cs2 rho0) and the rest
    # population takes the remainder; that state is left unchanged by a step
    m = d3.Model(rho0=0.9, cs2=cs2, kappa=kappa, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    fb = m.fbar()
    np.testing.assert_allclose(fb[1:], d3.W[1:] * 3 * cs2 * 0.9, rtol=1e-14)
    assert abs(fb.sum() - 0.9) < 1e-15
    f = np.broadcast_to(fb[:, None, None, None], (19, 3, 4, 5)).copy()
    np.testing.assert_allclose(d3.step(f, m), f, atol=1e-15)


def _project(f3, axes):
    """Populations of a 3-D state uniform along the third axis, summed onto the D2Q9
    velocities of the plane spanned by `axes` (x', y'), as an array [9, n_y', n_x']."""
    drop = ({0, 1, 2} - set(axes)).pop()
    sl = [slice(None)] * 4
    sl[3 - drop] = 0                       # array axes: 1 = z, 2 = y, 3 = x
    plane = f3[tuple(sl)]                  # [19, a, b] with the two remaining array axes
    rem = [ax for ax in (2, 1, 0) if ax != drop]      # spatial axes in array order (z, y, x)
    # order the plane as [y', x']
    if rem[0] != axes[1]:
        plane = np.transpose(plane, (0, 2, 1))
    out = np.zeros((9,) + plane.shape[1:])
    for i, c in enumerate(d3.C):
        k = [n for n in range(9) if th.C[n, 0] == c[axes[0]] and th.C[n, 1] == c[axes[1]]][0]
        out[k] += plane[i]
    return out


@pytest.mark.parametrize("axes", [(0, 1), (1, 2), (2, 0)])
def test_field_uniform_along_an_axis_evolves_as_the_d2q9_model(axes):
    # at tau_s = tau_b = tau_ghost a state uniform along one axis and mirror-symmetric
    # along it is a D2Q9 state of the other two: the D3Q19 oracle must then follow the
    # independent D2Q9 C core (Table II, Appendix B) step for step, nonlinear terms included
    n = {0: 12, 1: 10, 2: 9}
    drop = ({0, 1, 2} - set(axes)).pop()
    shape3 = [n[2], n[1], n[0]]            # (nz, ny, nx)
    shape3[2 - drop] = 1
    cs2, kappa, tau = 0.25, 0.05, 0.85
    m3 = d3.Model(rho0=1.0, cs2=cs2, kappa=kappa, tau_s=tau, tau_b=tau, tau_ghost=tau)
    m2 = th.Model(rho0=1.0, cs2=cs2, kappa=kappa, tau_s=tau, tau_b=tau, tau_ghost=tau)
    pert = synth.gaussian_field((19,) + tuple(shape3), seed=5 + drop, scale=0.05)
    # mirror-symmetric along the dropped axis, so that its velocity stays zero (a D2Q9
    # state has no third component)
    flip = d3.C.copy()
    flip[:, drop] *= -1
    mirror = [int(np.where((d3.C == c).all(axis=1))[0][0]) for c in flip]
    pert = 0.5 * (pert + pert[mirror])
    f3 = m3.fbar()[:, None, None, None] * (1.0 + pert)
    f2 = _project(f3, axes)
    for _ in range(12):
        f3 = d3.step(f3, m3)
        f2 = oracle.step(f2, m2)
        np.testing.assert_allclose(_project(f3, axes), f2, rtol=0, atol=2e-14)
    # the nonlinear and gradient terms were exercised
    r2 = f2.sum(axis=0)
    assert r2.std() > 1e-3


def test_mass_and_momentum_are_conserved_with_noise():
    L = d3.Lattice(6, 5, 4, rho0=1.0, cs2=0.2, seed=3)
    L.set_params(1e-4, 0.03, 0.8, 1.1, 0.9, d3.NOISE_LW)
    m0 = L.moments()[:4].sum(axis=(1, 2, 3))
    L.step(30)
    m1 = L.moments()[:4].sum(axis=(1, 2, 3))
    np.testing.assert_allclose(m1, m0, atol=1e-12)
    assert np.abs(L.f - L.model.fbar()[:, None, None, None]).max() > 1e-4     # the noise acted


def _fit_decay(a, t0, t1):
    t = np.arange(t0, t1)
    return -np.polyfit(t, np.log(np.abs(a[t0:t1])), 1)[0]


@pytest.mark.parametrize("tau_s", [0.7, 1.3])
def test_shear_wave_decays_at_the_shear_viscosity(tau_s):
    # u_x(z) = U sin(k z): j_x(k) decays as exp(-nu k^2 t) with nu = sigma_s^2 (tau_s - 1/2)
    nz = 64
    k = 2 * np.pi / nz
    m = d3.Model(rho0=1.0, cs2=0.25, kappa=0.02, tau_s=tau_s, tau_b=1.1, tau_ghost=0.9)
    z = np.arange(nz)
    rho = np.ones((nz, 1, 1))
    j = np.zeros((3, nz, 1, 1))
    j[0] = 1e-4 * np.sin(k * z)[:, None, None]
    lap, grad = d3.density_stencils(rho)
    f = np.einsum("ia,a...->i...", d3.TINV, d3.equilibrium_moments(rho, j, lap, grad, m.cs2, m.kappa))
    amp = []
    for _ in range(400):
        jx = np.einsum("i,i...->...", d3.C[:, 0].astype(float), f)[:, 0, 0]
        amp.append((jx * np.sin(k * z)).sum() * 2 / nz)
        f = d3.step(f, m)
    rate = _fit_decay(np.array(amp), 20, 400)
    nu = S2 * (tau_s - 0.5)
    print("shear: rate %.6e  nu k^2 %.6e" % (rate, nu * k * k))
    assert abs(rate / (nu * k * k) - 1) < 5e-3


@pytest.mark.parametrize("cs2,tau_b", [(0.25, 1.1), (0.15, 0.7)])
def test_sound_wave_speed_and_damping(cs2, tau_b):
    # a standing density wave along x: frequency c_s k and damping Gamma k^2 with
    # Gamma = (4 eta / 3 + zeta) / (2 rho0), eta = rho0 sigma_s^2 (tau_s - 1/2) and the bulk
    # viscosity of this model in three dimensions, zeta = rho0 (tau_b - 1/2)(5 sigma_s^2 -
    # 3 c_s^2) / 3 (Chapman-Enskog; its D2Q9 form is Eq. bulkv-yeo at kappa = 0)
    from scipy.optimize import curve_fit
    nx = 64
    k = 2 * np.pi / nx
    tau_s = 0.8
    m = d3.Model(rho0=1.0, cs2=cs2, kappa=0.0, tau_s=tau_s, tau_b=tau_b, tau_ghost=0.9)
    x = np.arange(nx)
    rho = (1.0 + 1e-4 * np.cos(k * x))[None, None, :]
    j = np.zeros((3, 1, 1, nx))
    lap, grad = d3.density_stencils(rho)
    f = np.einsum("ia,a...->i...", d3.TINV, d3.equilibrium_moments(rho, j, lap, grad, m.cs2, m.kappa))
    amp = []
    steps = 700
    for _ in range(steps):
        r = f.sum(axis=0)[0, 0]
        amp.append(((r - 1.0) * np.cos(k * x)).sum() * 2 / nx)
        f = d3.step(f, m)
    t = np.arange(steps, dtype=float)
    a = np.array(amp)
    fun = lambda tt, A, g, w, p: A * np.exp(-g * tt) * np.cos(w * tt + p)
    sel = t >= 30
    p, _ = curve_fit(fun, t[sel], a[sel], p0=[1e-4, 1e-3, np.sqrt(cs2) * k, 0.0])
    eta = S2 * (tau_s - 0.5)
    zeta = (tau_b - 0.5) * (5 * S2 - 3 * cs2) / 3
    gamma = (4 * eta / 3 + zeta) / 2 * k * k
    w = np.sqrt(cs2 * k * k - gamma ** 2)          # damped oscillator of the linear theory
    print("sound: omega %.6e (theory %.6e), damping %.6e (theory %.6e)" % (abs(p[2]), w, p[1], gamma))
    assert abs(abs(p[2]) / w - 1) < 2e-3
    assert abs(p[1] / gamma - 1) < 2e-2


@pytest.mark.parametrize("cs2", [S2, 0.25, 0.12, 0.3])
def test_noise_matrix_has_the_closed_form(cs2):
    # Xi(0) by hand: with y4 = e4 - d rho, y16 = e16 + d rho (d = 3 (cs2 - sigma_s^2)) the
    # collision is diagonal, and the ansatz covariances of y are rho0 kT (5 - 9 cs2),
    # 9 rho0 kT (1 - cs2) and 3 rho0 kT (3 cs2 - 1); every other non-conserved mode has
    # N_a rho0 kT / sigma_s^2.  Stationarity then gives Xi = -Y lambda (2 + lambda) on the
    # diagonal and -Y_{4,16} (lambda_b + lambda_g + lambda_b lambda_g) between 4 and 16.
    rho0, kT = 0.95, 2e-4
    lb, ls, lg = -1 / 1.1, -1 / 0.8, -1 / 0.9
    m = d3.Model(rho0=rho0, cs2=cs2, kappa=0.04, kT=kT, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    X = m.Xi_zero()
    til = lambda l: l * (2 + l)
    want = np.zeros((19, 19))
    lam = [lb] + [ls] * 5 + [lg] * 9
    for a in range(4, 19):
        want[a, a] = -(rho0 * kT / S2) * d3.N[a] * til(lam[a - 4])
    want[4, 4] = -rho0 * kT * (5 - 9 * cs2) * til(lb)
    want[16, 16] = -9 * rho0 * kT * (1 - cs2) * til(lg)
    want[4, 16] = want[16, 4] = -3 * rho0 * kT * (3 * cs2 - 1) * (lb + lg + lb * lg)
    np.testing.assert_allclose(X, want, rtol=1e-13, atol=1e-13 * kT)
    L = m.noise_factor()
    np.testing.assert_allclose(L @ L.T, X, atol=1e-14 * kT)


def test_noise_counters():
    # tag 4 and tag 5 draws: unit normals, independent of each other
    nu = d3.noise_normals(16, 16, 16, seed=11, step_index=7)
    assert np.all(nu[:4] == 0)
    v = nu[4:].reshape(15, -1)
    assert np.abs(v.mean(axis=1)).max() < 5 / np.sqrt(v.shape[1])
    assert np.abs(v.var(axis=1) - 1).max() < 6 * np.sqrt(2 / v.shape[1])
    c = np.corrcoef(v)
    assert np.abs(c - np.eye(15)).max() < 5 / np.sqrt(v.shape[1])
    # the first eight come from the tag-4 draw: the same as the C core's normals
    a = oracle.normals(np.arange(16 ** 3, dtype=np.uint32), 11, 7, 4)
    np.testing.assert_array_equal(nu[4:12].reshape(8, -1), a.T)


def test_ideal_fluctuating_gas_is_in_equipartition():
    # cs2 = sigma_s^2, kappa = 0: the uncorrelated noise of Xi(0) is exact at every k (the
    # ideal fluctuating lattice gas), so each node has <dm_a^2> = N_a rho0 kT / sigma_s^2
    # for the non-conserved modes, and the conserved rho, j have that variance less their
    # k = 0 share (1/n).  Replicas give independent samples for the z-scores.
    rho0, kT = 1.0, 1e-4
    nx = ny = nz = 4
    n = nx * ny * nz
    R, steps, burn = 6, 600, 100
    acc = []
    for r in range(R):
        L = d3.Lattice(nx, ny, nz, rho0=rho0, cs2=S2, seed=100 + r)
        L.set_params(kT, 0.0, 0.8, 1.1, 0.9, d3.NOISE_LW)
        L.step(burn)
        s = np.zeros(19)
        cnt = 0
        for t in range(steps):
            L.step(1)
            if t % 5 == 0:
                dm = L.moments() - L.model.mbar()[:, None, None, None]
                s += (dm.reshape(19, -1) ** 2).mean(axis=1)
                cnt += 1
        acc.append(s / cnt)
    acc = np.array(acc)                     # (R, 19)
    want = d3.N * rho0 * kT / S2
    want[:4] *= (1 - 1 / n)
    mean = acc.mean(axis=0)
    sd = acc.std(axis=0, ddof=1) / np.sqrt(R)
    z = (mean - want) / np.maximum(sd, 1e-30)
    print("equipartition ratios", np.round(mean / want, 3))
    assert np.abs(mean / want - 1).max() < 0.05
    assert np.abs(z).max() < 4.0


# --- correlated noise Xi(k) (Sec. III C, Eq. noise-matrix) ---------------------------------

@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (np.pi, 0.0, 0.0), (np.pi, np.pi, 0.0), (np.pi, np.pi, np.pi),
                               (0.3, 1.1, -2.0), (2.0, 2.5, 0.7)])
def test_noise_matrix_at_k_is_the_long_wavelength_form_at_cs2_k(k):
    # the FDT of Eq. (noise-matrix) with advection A(k) and the k-dependent ansatz against the
    # hand-derived Xi(0) closed forms evaluated at c_s^2(k) = cs2 + rho0 kappa s(k)
    m = d3.Model(rho0=0.9, cs2=0.25, kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    X = d3.Xi_k(m, *k)
    s = float(d3.lattice_s(*k))
    m2 = d3.Model(rho0=0.9, cs2=0.25 + 0.9 * 0.03 * s, kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    np.testing.assert_allclose(X, m2.Xi_zero(), rtol=1e-12, atol=1e-13 * 1e-4)
    assert np.abs(X[:4]).max() < 1e-18


def test_lattice_symbol_at_the_corners_and_its_small_k_limit():
    # s(k) = k^2 + O(k^4) (Appendix B's stencil is isotropic) and the corner values 0, 4, 16/3, 4
    k = np.array([0.01, -0.02, 0.015])
    assert abs(float(d3.lattice_s(*k)) / (k @ k) - 1) < 1e-3
    for kk, want in [((0, 0, 0), 0.0), ((np.pi, 0, 0), 4.0), ((0, np.pi, np.pi), 16 / 3), ((np.pi,) * 3, 4.0)]:
        assert abs(float(d3.lattice_s(*kk)) - want) < 1e-12


def test_real_space_construction_reproduces_Xi_k_at_every_wavevector():
    # transfer function of the 2x2x2 box: sum_abc L L^T |(1/8) sum_d a^dx b^dy c^dz e^{-i k.d}|^2
    # must equal the (4,16) block of Xi(k) from the FDT at every k of a 6 x 5 x 4 lattice
    m = d3.Model(rho0=1.0, cs2=0.2, kappa=0.04, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    Ls = d3.rs_factors(m)
    for mz in range(4):
        for my in range(5):
            for mx in range(6):
                k = (2 * np.pi * mx / 6, 2 * np.pi * my / 5, 2 * np.pi * mz / 4)
                got = np.zeros((2, 2))
                for w, (a, b, c) in enumerate(d3.CORNERS):
                    t = sum((a ** dx) * (b ** dy) * (c ** dz) * np.exp(-1j * (k[0] * dx + k[1] * dy + k[2] * dz))
                            for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)) / 8.0
                    got += abs(t) ** 2 * (Ls[w] @ Ls[w].T)
                X = d3.Xi_k(m, *k)
                want = np.array([[X[4, 4], X[4, 16]], [X[16, 4], X[16, 16]]])
                np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-18)


def test_real_space_fields_have_the_Xi_k_spectrum():
    # sampled: the generated (xi_4, xi_16) fields' spectral covariance at a few k against Xi(k)
    m = d3.Model(rho0=1.0, cs2=0.2, kappa=0.04, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    n = 6
    Ls = d3.rs_factors(m)
    acc = np.zeros((2, 2, n, n, n), dtype=complex)
    draws = 400
    for t in range(draws):
        xi = d3.xi416_rs(m, n, n, n, seed=9, step_index=t, Ls=Ls)
        xk = np.fft.fftn(xi, axes=(1, 2, 3)) / np.sqrt(n ** 3)
        acc += np.einsum("a...,b...->ab...", xk, np.conj(xk))
    acc /= draws
    for (mz, my, mx) in [(0, 0, 1), (0, 3, 3), (3, 3, 3), (1, 2, 5), (0, 0, 0)]:
        k = (2 * np.pi * mx / n, 2 * np.pi * my / n, 2 * np.pi * mz / n)
        X = d3.Xi_k(m, *k)
        want = np.array([[X[4, 4], X[4, 16]], [X[16, 4], X[16, 16]]])
        got = acc[:, :, mz, my, mx].real
        sd = np.sqrt((np.abs(np.diag(want))[:, None] * np.abs(np.diag(want))[None, :] + want ** 2) / draws)
        assert np.abs(got - want).max() < 5 * sd.max(), (k, got, want)


def _spectra(L, n):
    m = L.moments()
    drho = np.fft.fftn(m[0] - L.model.rho0) / np.sqrt(n ** 3)
    j = [np.fft.fftn(m[a]) / np.sqrt(n ** 3) for a in (1, 2, 3)]
    return np.abs(drho) ** 2, sum(np.abs(x) ** 2 for x in j) / 3


@pytest.mark.parametrize("mode", ["rs", "lw"])
def test_correlated_noise_equilibrates_every_wavevector(mode):
    # Sec. V A in three dimensions: with Xi(k) the density spectrum is the Ornstein-Zernike
    # S(k) = rho0 kT / c_s^2(k) and the momentum spectrum rho0 kT at every k; with the
    # long-wavelength Xi(0) alone the largest wavevectors stay out of equipartition
    n, R, steps, burn = 4, 4, 500, 80
    cs2, kappa, kT = 0.2, 0.04, 1e-4       # Xi(k) positive semidefinite up to s = 16/3
    S_acc = np.zeros((n, n, n))
    J_acc = np.zeros((n, n, n))
    cnt = 0
    for r in range(R):
        L = d3.Lattice(n, n, n, cs2=cs2, seed=300 + r)
        L.set_params(kT, kappa, 0.8, 1.1, 0.9, d3.NOISE_FULL_RS if mode == "rs" else d3.NOISE_LW)
        L.step(burn)
        for t in range(steps):
            L.step(1)
            if t % 2 == 0:
                s_, j_ = _spectra(L, n)
                S_acc += s_
                J_acc += j_
                cnt += 1
    S_acc /= cnt
    J_acc /= cnt
    k1 = 2 * np.pi * np.fft.fftfreq(n)
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")       # arrays [z, y, x]
    s = d3.lattice_s(KX, KY, KZ)
    S_th = 1.0 * kT / (cs2 + kappa * s)
    ratio_S = (S_acc / S_th).ravel()[1:]
    # j_a at k = pi e_a is the staggered-momentum invariant (next test): those three never
    # equilibrate, as (pi, 0) and (0, pi) on D2Q9
    keep = np.ones((n, n, n), bool)
    keep[0, 0, 0] = keep[0, 0, n // 2] = keep[0, n // 2, 0] = keep[n // 2, 0, 0] = False
    ratio_J = (J_acc / kT)[keep]
    print(mode, "S ratio range %.3f..%.3f, J ratio range %.3f..%.3f" % (ratio_S.min(), ratio_S.max(),
                                                                        ratio_J.min(), ratio_J.max()))
    if mode == "rs":
        assert np.abs(ratio_S - 1).max() < 0.12 and np.abs(ratio_J - 1).max() < 0.12
        assert abs(ratio_S.mean() - 1) < 0.02 and abs(ratio_J.mean() - 1) < 0.02
    else:
        assert np.abs(ratio_S - 1).max() > 0.2          # the long-wavelength noise misses large k


def test_staggered_momentum_is_an_invariant_of_the_noisy_step():
    # sum_r (-1)^x j_x(r) (and its y, z analogues): streaming multiplies every population with
    # c_x = +-1 by -1 at k = (pi, 0, 0), the collision conserves j and the noise has no
    # momentum component, so the staggered momentum only changes sign each step
    n = 4
    L = d3.Lattice(n, n, n, cs2=0.2, seed=4)
    L.set_params(1e-4, 0.04, 0.8, 1.1, 0.9, d3.NOISE_FULL_RS)
    L.f = L.f * (1.0 + synth.gaussian_field(L.f.shape, seed=2, scale=0.01))
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    def stag():
        m = L.moments()
        return np.array([((-1.0) ** x * m[1]).sum(), ((-1.0) ** y * m[2]).sum(), ((-1.0) ** z * m[3]).sum()])
    s0 = stag()
    assert np.abs(s0).min() > 1e-4
    for t in range(1, 6):
        L.step(1)
        np.testing.assert_allclose(stag(), (-1) ** t * s0, atol=1e-14)
