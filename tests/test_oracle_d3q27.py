"""Pins of the D3Q27 oracle (oracle/d3q27.py): the lattice's isotropy, the product basis
(orthogonality, its norms, the D2Q9 basis of Table I as its c_z-independent members), the
second and third moments of the equilibrium against Eq. (press-ten), the rest state, exact
agreement with the independent D2Q9 C core on fields uniform along an axis, Navier-Stokes
shear and sound, the ansatz covariance as a rank-one update of a diagonal, the ideal-gas
noise in closed form, the fluctuation-dissipation balance of Xi(0) by simulation of the
k = 0 dynamics, equipartition of the ideal fluctuating gas; for the correlated noise Xi(k):
the FDT with advection equal to Xi(0) at c_s^2(k), the Laplacian symbol against the stencil,
the real-space construction's transfer function and sampled spectrum equal to Xi(k), and
equipartition at every wavevector (which Xi(0) alone misses)."""
import numpy as np
import pytest

import oracle
from oracle import d3q27 as d
from oracle import theory as th
from paper_1009_0254_gb300 import synth

S2 = 1.0 / 3.0


def test_lattice_is_the_product_of_d1q3_and_isotropic_to_fourth_order():
    C, W = d.C.astype(float), d.W
    assert len({tuple(c) for c in d.C}) == 27 and (d.C[d.OPP] == -d.C).all()
    assert abs(W.sum() - 1) < 1e-15
    np.testing.assert_allclose(sorted(set(np.round(W, 15))), sorted({8 / 27, 2 / 27, 1 / 54, 1 / 216}))
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", W, C, C), S2 * np.eye(3), atol=1e-16)
    dd = np.eye(3)
    iso4 = S2 ** 2 * (np.einsum("ab,cd->abcd", dd, dd) + np.einsum("ac,bd->abcd", dd, dd)
                      + np.einsum("ad,bc->abcd", dd, dd))
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic,id->abcd", W, C, C, C, C), iso4, atol=1e-16)


def test_product_basis_is_orthogonal_and_contains_the_d2q9_basis():
    G = (d.T * d.W) @ d.T.T
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-15
    n1 = [1.0, 1 / 3, 2.0]                          # D1Q3 norms of 1, c, 3c^2 - 1
    np.testing.assert_allclose(d.N, [n1[a] * n1[b] * n1[c] for a, b, c in d.MODES], rtol=1e-14)
    # Table I's polynomials on the c_z = 0 velocities are the (a, b, 0) product modes
    sel = d.C[:, 2] == 0
    cx, cy = d.C[sel, 0].astype(float), d.C[sel, 1].astype(float)
    c2 = cx * cx + cy * cy
    row = lambda m: d.T[d.IDX[m]][sel]
    np.testing.assert_allclose(3 * c2 - 2, row((2, 0, 0)) + row((0, 2, 0)))
    np.testing.assert_allclose(2 * cx * cx - c2, (row((2, 0, 0)) - row((0, 2, 0))) / 3)
    np.testing.assert_allclose(cx * cy, row((1, 1, 0)))
    np.testing.assert_allclose((3 * c2 - 4) * cx, row((1, 2, 0)))
    np.testing.assert_allclose((3 * c2 - 4) * cy, row((2, 1, 0)))
    np.testing.assert_allclose(9 * c2 * c2 - 15 * c2 + 2, 2 * row((2, 2, 0)))


def test_relaxation_rates_on_the_bulk_and_traceless_modes():
    L = d.relaxation_matrix(0.8, 1.1, 0.9)
    v = np.zeros(27)
    for k in d.SECOND_DIAG:
        v[k] = 1.0
    np.testing.assert_allclose(L @ v, -v / 1.1, atol=1e-15)            # bulk: p_2x + p_2y + p_2z
    w = np.zeros(27)
    w[d.SECOND_DIAG[0]], w[d.SECOND_DIAG[1]] = 1.0, -1.0
    np.testing.assert_allclose(L @ w, -w / 0.8, atol=1e-15)            # traceless
    assert L[d.IDX[(1, 1, 0)], d.IDX[(1, 1, 0)]] == -1 / 0.8
    assert L[d.IDX[(2, 1, 1)], d.IDX[(2, 1, 1)]] == -1 / 0.9
    assert np.all(L[d.CONSERVED] == 0)


def test_equilibrium_carries_the_pressure_tensor():
    rng = np.random.default_rng(1)
    shape = (4, 3, 5)
    rho = 1.0 + 0.2 * rng.random(shape)
    j = 0.05 * rng.standard_normal((3,) + shape)
    lap = rng.standard_normal(shape)
    grad = 0.3 * rng.standard_normal((3,) + shape)
    cs2, kappa = 0.21, 0.07
    f = np.einsum("ia,a...->i...", d.TINV, d.equilibrium_moments(rho, j, lap, grad, cs2, kappa))
    C = d.C.astype(float)
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
    dd = np.eye(3)
    want3 = S2 * (np.einsum("a...,bc->abc...", j, dd) + np.einsum("b...,ac->abc...", j, dd)
                  + np.einsum("c...,ab->abc...", j, dd))
    np.testing.assert_allclose(P3, want3, atol=1e-14)


@pytest.mark.parametrize("cs2", [S2, 0.2, 0.1])
def test_rest_state_is_a_fixed_point(cs2):
    m = d.Model(rho0=0.9, cs2=cs2, kappa=0.05, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    fb = m.fbar()
    np.testing.assert_allclose(fb[1:], d.W[1:] * 3 * cs2 * 0.9, rtol=1e-13)
    assert abs(fb.sum() - 0.9) < 1e-15
    f = np.broadcast_to(fb[:, None, None, None], (27, 3, 4, 5)).copy()
    np.testing.assert_allclose(d.step(f, m), f, atol=1e-15)


def _project(f3, axes):
    drop = ({0, 1, 2} - set(axes)).pop()
    sl = [slice(None)] * 4
    sl[3 - drop] = 0
    plane = f3[tuple(sl)]
    rem = [ax for ax in (2, 1, 0) if ax != drop]
    if rem[0] != axes[1]:
        plane = np.transpose(plane, (0, 2, 1))
    out = np.zeros((9,) + plane.shape[1:])
    for i, c in enumerate(d.C):
        k = [n for n in range(9) if th.C[n, 0] == c[axes[0]] and th.C[n, 1] == c[axes[1]]][0]
        out[k] += plane[i]
    return out


@pytest.mark.parametrize("axes", [(0, 1), (1, 2), (2, 0)])
def test_field_uniform_along_an_axis_evolves_as_the_d2q9_model(axes):
    # equal relaxation times, a state uniform and mirror-symmetric along the dropped axis:
    # the D3Q27 oracle follows the independent D2Q9 C core (Table II) step for step
    n = {0: 12, 1: 10, 2: 9}
    drop = ({0, 1, 2} - set(axes)).pop()
    shape3 = [n[2], n[1], n[0]]
    shape3[2 - drop] = 1
    cs2, kappa, tau = 0.25, 0.05, 0.85
    m3 = d.Model(1.0, cs2, kappa, 0.0, tau, tau, tau)
    m2 = th.Model(rho0=1.0, cs2=cs2, kappa=kappa, tau_s=tau, tau_b=tau, tau_ghost=tau)
    pert = synth.gaussian_field((27,) + tuple(shape3), seed=9 + drop, scale=0.05)
    flip = d.C.copy()
    flip[:, drop] *= -1
    mirror = [int(np.where((d.C == c).all(axis=1))[0][0]) for c in flip]
    pert = 0.5 * (pert + pert[mirror])
    f3 = m3.fbar()[:, None, None, None] * (1.0 + pert)
    f2 = _project(f3, axes)
    for _ in range(12):
        f3 = d.step(f3, m3)
        f2 = oracle.step(f2, m2)
        np.testing.assert_allclose(_project(f3, axes), f2, rtol=0, atol=2e-14)
    assert f2.sum(axis=0).std() > 1e-3


def test_mass_and_momentum_are_conserved_with_noise():
    L = d.Lattice(5, 4, 3, cs2=0.2, seed=3)
    L.set_params(1e-4, 0.03, 0.8, 1.1, 0.9, d.NOISE_LW)
    c = [d.IDX[(0, 0, 0)], d.IDX[(1, 0, 0)], d.IDX[(0, 1, 0)], d.IDX[(0, 0, 1)]]
    m0 = L.moments()[c].sum(axis=(1, 2, 3))
    L.step(20)
    np.testing.assert_allclose(L.moments()[c].sum(axis=(1, 2, 3)), m0, atol=1e-12)


@pytest.mark.parametrize("tau_s", [0.7, 1.3])
def test_shear_wave_decays_at_the_shear_viscosity(tau_s):
    nz = 64
    k = 2 * np.pi / nz
    m = d.Model(1.0, 0.25, 0.02, 0.0, tau_s, 1.1, 0.9)
    z = np.arange(nz)
    rho = np.ones((nz, 1, 1))
    j = np.zeros((3, nz, 1, 1))
    j[0] = 1e-4 * np.sin(k * z)[:, None, None]
    lap, grad = d.density_stencils(rho)
    f = np.einsum("ia,a...->i...", d.TINV, d.equilibrium_moments(rho, j, lap, grad, m.cs2, m.kappa))
    amp = []
    for _ in range(400):
        jx = np.einsum("i,i...->...", d.C[:, 0].astype(float), f)[:, 0, 0]
        amp.append((jx * np.sin(k * z)).sum() * 2 / nz)
        f = d.step(f, m)
    t = np.arange(20, 400)
    rate = -np.polyfit(t, np.log(np.abs(np.array(amp)[20:400])), 1)[0]
    nu = S2 * (tau_s - 0.5)
    assert abs(rate / (nu * k * k) - 1) < 5e-3


@pytest.mark.parametrize("cs2,tau_b", [(0.25, 1.1), (0.15, 0.7)])
def test_sound_wave_speed_and_damping(cs2, tau_b):
    # Gamma = (4 eta / 3 + zeta) / (2 rho0), zeta = rho0 (tau_b - 1/2)(5 sigma_s^2 - 3 cs2) / 3
    from scipy.optimize import curve_fit
    nx = 64
    k = 2 * np.pi / nx
    tau_s = 0.8
    m = d.Model(1.0, cs2, 0.0, 0.0, tau_s, tau_b, 0.9)
    x = np.arange(nx)
    rho = (1.0 + 1e-4 * np.cos(k * x))[None, None, :]
    j = np.zeros((3, 1, 1, nx))
    lap, grad = d.density_stencils(rho)
    f = np.einsum("ia,a...->i...", d.TINV, d.equilibrium_moments(rho, j, lap, grad, m.cs2, m.kappa))
    amp = []
    for _ in range(700):
        r = f.sum(axis=0)[0, 0]
        amp.append(((r - 1.0) * np.cos(k * x)).sum() * 2 / nx)
        f = d.step(f, m)
    t = np.arange(700, dtype=float)
    fun = lambda tt, A, g, w, p: A * np.exp(-g * tt) * np.cos(w * tt + p)
    sel = t >= 30
    p, _ = curve_fit(fun, t[sel], np.array(amp)[sel], p0=[1e-4, 1e-3, np.sqrt(cs2) * k, 0.0])
    gamma = (4 * S2 * (tau_s - 0.5) / 3 + (tau_b - 0.5) * (5 * S2 - 3 * cs2) / 3) / 2 * k * k
    w = np.sqrt(cs2 * k * k - gamma ** 2)
    assert abs(abs(p[2]) / w - 1) < 2e-3
    assert abs(p[1] / gamma - 1) < 2e-2


@pytest.mark.parametrize("cs2", [S2, 0.25, 0.12])
def test_ansatz_covariance_is_a_rank_one_update_of_a_diagonal(cs2):
    # fbar_i = 3 cs2 rho0 w_i + rho0 (1 - 3 cs2) delta_i0, so
    # (S / rho0) T diag(fbar) T^T = S [3 cs2 diag(N) + (1 - 3 cs2) t0 t0^T], t0 the modes at c = 0
    rho0, kT = 0.9, 1e-4
    m = d.Model(rho0, cs2, 0.03, kT, 0.8, 1.1, 0.9)
    S = rho0 * kT / cs2
    t0 = d.T[:, 0]
    want = S * (3 * cs2 * np.diag(d.N) + (1 - 3 * cs2) * np.outer(t0, t0))
    np.testing.assert_allclose(m.G0(), want, rtol=1e-12, atol=1e-18)


def test_ideal_gas_noise_in_closed_form():
    # cs2 = sigma_s^2: G = N rho0 kT / sigma_s^2 (diagonal), Omega = Lambda, so
    # Xi = -(rho0 kT / sigma_s^2) N_a lambda (2 + lambda) mode by mode, with the p_2 block
    # lambda~_s I + (lambda~_b - lambda~_s) / 3 (1 1^T) (N = 2 each)
    rho0, kT = 1.0, 1e-4
    m = d.Model(rho0, S2, 0.0, kT, 0.8, 1.1, 0.9)
    til = lambda l: l * (2 + l)
    lb, ls, lg = -1 / 1.1, -1 / 0.8, -1 / 0.9
    Tt = rho0 * kT / S2
    want = np.zeros((27, 27))
    for k in range(27):
        if k not in d.CONSERVED:
            want[k, k] = -Tt * d.N[k] * til(lg)
    for k in d.SECOND_OFF:
        want[k, k] = -Tt * d.N[k] * til(ls)
    for a in d.SECOND_DIAG:
        for b in d.SECOND_DIAG:
            want[a, b] = -Tt * 2 * ((til(lb) - til(ls)) / 3 + (til(ls) if a == b else 0.0))
    np.testing.assert_allclose(m.Xi_zero(), want, rtol=1e-12, atol=1e-13 * kT)


@pytest.mark.parametrize("cs2", [0.25, 0.12])
def test_single_node_dynamics_reaches_the_conditional_ansatz_covariance(cs2):
    # On a 1x1x1 periodic lattice streaming is the identity, rho and j are fixed and the
    # collision is linear: m -> m + Omega (m - mbar) + xi exactly.  The stationary
    # covariance of the non-conserved modes must be the ansatz G(0) conditioned on the fixed
    # density, G_nn - G_n0 G_0n / G_00: the fluctuation-dissipation balance of Xi(0), checked
    # by simulation instead of algebra.
    kT = 1e-6
    L = d.Lattice(1, 1, 1, cs2=cs2, seed=17)
    L.set_params(kT, 0.04, 0.8, 1.1, 0.9, d.NOISE_LW)
    mbar = L.model.mbar()
    L.step(50)
    nc = d.NONCONSERVED
    steps = 16000
    acc = np.zeros((len(nc), len(nc)))
    samples = []
    for _ in range(steps):
        L.step(1)
        v = (L.moments()[:, 0, 0, 0] - mbar)[nc]
        acc += np.outer(v, v)
        samples.append(v)
    Cs = acc / steps
    G = L.model.G0()
    Gc = G[np.ix_(nc, nc)] - np.outer(G[nc, 0], G[0, nc]) / G[0, 0]
    # standard error of each diagonal entry from batch means (batches of 200 steps)
    s = np.array(samples) ** 2
    bm = s.reshape(80, 200, -1).mean(axis=1)
    se = bm.std(axis=0, ddof=1) / np.sqrt(80)
    z = (np.diag(Cs) - np.diag(Gc)) / se
    print("k = 0 variance ratios", np.round(np.diag(Cs) / np.diag(Gc), 3), "max |z| %.2f" % np.abs(z).max())
    assert np.abs(z).max() < 4.5
    # the coupled entries (bulk, fourth- and sixth-order ghosts) too
    k4 = [nc.index(k) for k in d.SECOND_DIAG + d.FOURTH_PAIR + [d.SIXTH]]
    sub = np.abs(Cs[np.ix_(k4, k4)] - Gc[np.ix_(k4, k4)]).max() / np.abs(Gc[np.ix_(k4, k4)]).max()
    assert sub < 0.08


def test_ideal_fluctuating_gas_is_in_equipartition():
    rho0, kT = 1.0, 1e-4
    nx = ny = nz = 3
    n = nx * ny * nz
    R, steps = 6, 300
    acc = []
    for r in range(R):
        L = d.Lattice(nx, ny, nz, rho0=rho0, cs2=S2, seed=200 + r)
        L.set_params(kT, 0.0, 0.8, 1.1, 0.9, d.NOISE_LW)
        L.step(60)
        s = np.zeros(27)
        cnt = 0
        for t in range(steps):
            L.step(1)
            if t % 3 == 0:
                dm = L.moments() - L.model.mbar()[:, None, None, None]
                s += (dm.reshape(27, -1) ** 2).mean(axis=1)
                cnt += 1
        acc.append(s / cnt)
    acc = np.array(acc)
    want = d.N * rho0 * kT / S2
    want[d.CONSERVED] *= 1 - 1 / n
    mean = acc.mean(axis=0)
    sd = acc.std(axis=0, ddof=1) / np.sqrt(R)
    print("D3Q27 equipartition ratios", np.round(mean / want, 3))
    assert np.abs(mean / want - 1).max() < 0.06
    assert np.abs((mean - want) / sd).max() < 5.0


# --- correlated noise Xi(k) (Sec. III C, Eq. noise-matrix) ---------------------------------

@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (np.pi, 0.0, 0.0), (np.pi, np.pi, 0.0), (np.pi, np.pi, np.pi),
                               (0.3, 1.1, -2.0), (2.0, 2.5, 0.7)])
def test_noise_matrix_at_k_is_the_long_wavelength_form_at_cs2_k(k):
    # the FDT of Eq. (noise-matrix) with advection A(k) and the k-dependent ansatz against
    # Xi(0) of a homogeneous system at c_s^2(k) = cs2 + rho0 kappa s(k)
    m = d.Model(rho0=0.9, cs2=0.25, kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    X = d.Xi_k(m, *k)
    s = float(d.lattice_s(*k))
    m2 = d.Model(rho0=0.9, cs2=0.25 + 0.9 * 0.03 * s, kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    np.testing.assert_allclose(X, m2.Xi_zero(), rtol=1e-12, atol=1e-13 * 1e-4)
    assert np.abs(X[d.CONSERVED]).max() < 1e-18


def test_lattice_symbol_is_the_stencils_and_has_its_corner_values():
    # s(k) = k^2 + O(k^4); the corner values 0, 4, 16/3, 52/9; and s is what the oracle's
    # Laplacian stencil does to a plane wave on a periodic lattice
    k = np.array([0.01, -0.02, 0.015])
    assert abs(float(d.lattice_s(*k)) / (k @ k) - 1) < 1e-3
    for kk, want in [((0, 0, 0), 0.0), ((np.pi, 0, 0), 4.0), ((0, np.pi, np.pi), 16 / 3), ((np.pi,) * 3, 52 / 9)]:
        assert abs(float(d.lattice_s(*kk)) - want) < 1e-12
    n = (6, 5, 4)
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    for m in [(1, 0, 0), (2, 3, 1), (3, 2, 2)]:
        kv = [2 * np.pi * m[a] / n[a] for a in range(3)]
        wave = np.cos(kv[0] * x + kv[1] * y + kv[2] * z)
        lap, _ = d.density_stencils(wave)
        np.testing.assert_allclose(-lap, float(d.lattice_s(*kv)) * wave, atol=1e-12)


def _transfer(k, w, d3=d):
    """|(1/8) sum_d (+-1)^d e^{-i k.d}|^2 of corner w: the spectrum of its box-filtered field."""
    a, b, c = d3.CORNERS[w]
    t = sum((a ** dx) * (b ** dy) * (c ** dz) * np.exp(-1j * (k[0] * dx + k[1] * dy + k[2] * dz))
            for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)) / 8.0
    return abs(t) ** 2


def test_real_space_construction_reproduces_Xi_k_at_every_wavevector():
    # the white part C plus the two box-filtered scalar fields along p and q: their spectral
    # covariance C + sum_w |t_w(k)|^2 (a_p,w^2 p p^T + a_q,w^2 q q^T) must equal the coupled
    # block of Xi(k) from the FDT at every k of a 6 x 5 x 4 lattice
    m = d.Model(rho0=1.0, cs2=0.2, kappa=0.04, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    Lw, p, q = d.rs_split(m)
    ap, aq = d.rs_weights()
    C = Lw @ Lw.T
    for mz in range(4):
        for my in range(5):
            for mx in range(6):
                k = (2 * np.pi * mx / 6, 2 * np.pi * my / 5, 2 * np.pi * mz / 4)
                got = C.copy()
                for w in range(8):
                    tw = _transfer(k, w)
                    got += tw * (ap[w] ** 2 * np.outer(p, p) + aq[w] ** 2 * np.outer(q, q))
                want = d.Xi_k(m, *k)[np.ix_(d.COUPLED, d.COUPLED)]
                np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-18)


def test_corner_amplitudes_interpolate_s_and_its_complement():
    # the corner transfers are the multilinear interpolation weights: they sum to one and,
    # weighted by the corner values of s, give s(k) itself at any k
    ap, aq = d.rs_weights()
    S = d.s_max()
    assert abs(S - 52 / 9) < 1e-12
    np.testing.assert_allclose(sorted(set(np.round(ap ** 2, 12))), [0, 4, 16 / 3, 52 / 9], atol=1e-12)
    for k in [(0.3, -1.2, 2.2), (np.pi, 0.4, 0.0), (1.0, 2.0, 3.0)]:
        tw = np.array([_transfer(k, w) for w in range(8)])
        assert abs(tw.sum() - 1) < 1e-14
        assert abs(tw @ ap ** 2 - float(d.lattice_s(*k))) < 1e-12
        assert abs(tw @ aq ** 2 - (S - float(d.lattice_s(*k)))) < 1e-12


@pytest.mark.parametrize("cs2,kappa,tb,tg", [(0.2, 0.04, 1.1, 0.9), (1 / 3, 0.01, 1.1, 0.9), (0.2, 0.04, 0.6, 1.5),
                                             (0.1, 0.06, 0.6, 0.9), (0.3, 0.02, 2.0, 1.5)])
def test_split_of_the_slope_has_rank_two_and_a_white_part_exactly_where_Xi_is_psd(cs2, kappa, tb, tg):
    # D = (X(S) - X0) / S has one positive and one negative eigenvalue (the slope of Xi(0) in
    # c_s^2 has rank two); D = p p^T - q q^T; C = X0 - S q q^T is positive semidefinite; and
    # C + S p p^T is X at k = (pi, pi, pi).  The cases with tau_b = 0.6 are ones where the
    # split along the eigenvectors of D itself leaves C indefinite: the whitened split does not
    m = d.Model(rho0=1.0, cs2=cs2, kappa=kappa, kT=1e-4, tau_s=0.8, tau_b=tb, tau_ghost=tg)
    S = d.s_max()
    X0 = d.Xi_k(m, 0, 0, 0)[np.ix_(d.COUPLED, d.COUPLED)]
    XS = d.Xi_k(m, np.pi, np.pi, np.pi)[np.ix_(d.COUPLED, d.COUPLED)]
    D = (XS - X0) / S
    ev = np.linalg.eigvalsh(D)
    big = np.abs(ev) > 1e-9 * np.abs(ev).max()
    assert big.sum() == 2 and ev[0] < 0 < ev[-1]
    Lw, p, q = d.rs_split(m)
    np.testing.assert_allclose(np.outer(p, p) - np.outer(q, q), D, rtol=0, atol=1e-12 * np.abs(D).max())
    C = Lw @ Lw.T
    np.testing.assert_allclose(C, X0 - S * np.outer(q, q), rtol=0, atol=1e-12 * np.abs(X0).max())
    np.testing.assert_allclose(C + S * np.outer(p, p), XS, rtol=0, atol=1e-12 * np.abs(X0).max())
    for v in (p, q):
        big = np.abs(v) >= 0.5 * np.abs(v).max()
        assert v[np.argmax(big)] > 0
    if tb == 0.6:
        w, E = np.linalg.eigh(D)
        qe = np.sqrt(-w[0]) * E[:, 0]
        assert np.linalg.eigvalsh(X0 - S * np.outer(qe, qe)).min() < 0


def test_split_refuses_where_Xi_is_indefinite_at_the_far_corner():
    # c_s^2(k) = 0.3 + 0.06 * 52/9 at k = (pi, pi, pi): the coupled block is indefinite there
    m = d.Model(rho0=1.0, cs2=0.3, kappa=0.06, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    XS = d.Xi_k(m, np.pi, np.pi, np.pi)[np.ix_(d.COUPLED, d.COUPLED)]
    assert np.linalg.eigvalsh(XS).min() < 0
    with pytest.raises(ValueError):
        d.rs_split(m)


def test_correlated_noise_at_zero_kappa_is_the_long_wavelength_noise():
    # kappa = 0: no slope, p = q = 0, and the white part's factor is that of Xi(0): the
    # correlated mode steps exactly as the long-wavelength mode
    m = d.Model(rho0=1.0, cs2=0.2, kappa=0.0, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    Lw, p, q = d.rs_split(m)
    assert not p.any() and not q.any()
    a = d.Lattice(5, 4, 3, cs2=0.2, seed=11)
    b = d.Lattice(5, 4, 3, cs2=0.2, seed=11)
    a.set_params(1e-4, 0.0, 0.8, 1.1, 0.9, d.NOISE_FULL_RS)
    b.set_params(1e-4, 0.0, 0.8, 1.1, 0.9, d.NOISE_LW)
    a.step(3)
    b.step(3)
    np.testing.assert_allclose(a.f, b.f, rtol=0, atol=1e-15)
    assert np.abs(a.f - d.Lattice(5, 4, 3, cs2=0.2).f).max() > 1e-4


def test_real_space_fields_have_the_Xi_k_spectrum():
    # sampled: the coupled modes' noise of the lattice (the white part through the
    # long-wavelength normals plus p phi_p + q phi_q) against Xi(k) at a few k
    m = d.Model(rho0=1.0, cs2=0.2, kappa=0.04, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    n = 6
    split = d.rs_split(m)
    L = d.rs_noise_factor(m, split)
    nodes = np.arange(n ** 3, dtype=np.uint32).reshape(n, n, n)
    acc = np.zeros((7, 7, n, n, n), dtype=complex)
    draws = 300
    for t in range(draws):
        xi = d.noise_lw_nodes(m, nodes, 9, t, L)[d.COUPLED] + d.xi_coupled_rs(m, n, n, n, 9, t, split)
        xk = np.fft.fftn(xi, axes=(1, 2, 3)) / np.sqrt(n ** 3)
        acc += np.einsum("a...,b...->ab...", xk, np.conj(xk))
    acc /= draws
    for (mz, my, mx) in [(0, 0, 1), (0, 3, 3), (3, 3, 3), (1, 2, 5), (0, 0, 0)]:
        k = (2 * np.pi * mx / n, 2 * np.pi * my / n, 2 * np.pi * mz / n)
        want = d.Xi_k(m, *k)[np.ix_(d.COUPLED, d.COUPLED)]
        got = acc[:, :, mz, my, mx].real
        sd = np.sqrt((np.abs(np.diag(want))[:, None] * np.abs(np.diag(want))[None, :] + want ** 2) / draws)
        assert np.abs(got - want).max() < 5 * sd.max(), (k, np.abs(got - want).max(), sd.max())


def _spectra(L, n):
    m = L.moments()
    drho = np.fft.fftn(m[d.IDX[(0, 0, 0)]] - L.model.rho0) / np.sqrt(n ** 3)
    j = [np.fft.fftn(m[d.IDX[c]]) / np.sqrt(n ** 3) for c in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    return np.abs(drho) ** 2, sum(np.abs(x) ** 2 for x in j) / 3


@pytest.mark.parametrize("mode", ["rs", "lw"])
def test_correlated_noise_equilibrates_every_wavevector(mode):
    # Sec. V A on D3Q27: with Xi(k) the density spectrum is the Ornstein-Zernike
    # S(k) = rho0 kT / c_s^2(k) and the momentum spectrum rho0 kT at every k (the staggered
    # momenta at k = pi e_a excepted, an invariant as on D3Q19); with Xi(0) alone the largest
    # wavevectors stay out of equipartition
    n, R, steps, burn = 4, 6, 500, 80
    cs2, kappa, kT = 0.2, 0.04, 1e-4
    S_acc = np.zeros((n, n, n))
    J_acc = np.zeros((n, n, n))
    cnt = 0
    for r in range(R):
        L = d.Lattice(n, n, n, cs2=cs2, seed=400 + r)
        L.set_params(kT, kappa, 0.8, 1.1, 0.9, d.NOISE_FULL_RS if mode == "rs" else d.NOISE_LW)
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
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    S_th = kT / (cs2 + kappa * d.lattice_s(KX, KY, KZ))
    ratio_S = (S_acc / S_th).ravel()[1:]
    keep = np.ones((n, n, n), bool)
    keep[0, 0, 0] = keep[0, 0, n // 2] = keep[0, n // 2, 0] = keep[n // 2, 0, 0] = False
    ratio_J = (J_acc / kT)[keep]
    print(mode, "S ratio range %.3f..%.3f, J ratio range %.3f..%.3f" % (ratio_S.min(), ratio_S.max(),
                                                                        ratio_J.min(), ratio_J.max()))
    if mode == "rs":
        assert np.abs(ratio_S - 1).max() < 0.12 and np.abs(ratio_J - 1).max() < 0.12
        assert abs(ratio_S.mean() - 1) < 0.02 and abs(ratio_J.mean() - 1) < 0.02
    else:
        assert np.abs(ratio_S - 1).max() > 0.2
