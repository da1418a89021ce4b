"""Pins of the 3-D oracles' two-phase model (Sec. II A; Sec. IV and Sec. V B): the Landau
double-well bulk pressure in the D3Q19 and D3Q27 equilibria (fixed points at every uniform
density; on fields uniform and mirror-symmetric along an axis, step-for-step agreement with
the independent D2Q9 C core and its double well), the structure of Xi(0) the local noise
relies on (rho times an affine function of c_s^2), and the noise at the local density
(the uniform noise at uniform density, Xi(0) of the local state as its covariance)."""
import numpy as np
import pytest

import oracle
from oracle import d3q19, d3q27
from oracle import theory as th
from paper_1009_0254_gb300 import synth

WELL = th.DoubleWell(0.04, 0.5, 1.0)
LATTICES = [d3q19, d3q27]


def _model(mod, rho, eos=WELL, **kw):
    return mod.Model(rho0=rho, cs2=eos.cs2(rho), p0_rest=eos.p0(rho), **kw)


@pytest.mark.parametrize("mod", LATTICES, ids=["d3q19", "d3q27"])
def test_uniform_states_are_fixed_points_of_the_double_well_collision(mod):
    # a uniform state at rest with the equilibrium of its own density (bulk pressure p0(rho)
    # of the double well) is left unchanged by a step, at the coexisting densities, inside
    # the spinodal region and above; with p0 = cs2 rho instead it is not
    for rho in (WELL.rhoV, WELL.rhoL, 0.5 * (WELL.rhoV + WELL.rhoL), 1.2):
        m = _model(mod, rho, kappa=0.05, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
        f = np.broadcast_to(m.rest()[:, None, None, None], (mod.Q, 3, 4, 5)).copy()
        np.testing.assert_allclose(mod.step(f, m, eos=WELL), f, atol=1e-15)
        if abs(WELL.p0(rho) - WELL.cs2(rho) * rho) > 1e-6:
            assert np.abs(mod.step(f, m) - f).max() > 1e-6


def _project(mod, f3, drop):
    """Populations of a 3-D state uniform along axis `drop`, summed onto the D2Q9 velocities
    of the other two axes (in increasing order), as [9, n_y', n_x']."""
    axes = [a for a in (0, 1, 2) if a != drop]
    sl = [slice(None)] * 4
    sl[3 - drop] = 0
    plane = f3[tuple(sl)]
    out = np.zeros((9,) + plane.shape[1:])
    for i, c in enumerate(mod.C):
        k = [n for n in range(9) if th.C[n, 0] == c[axes[0]] and th.C[n, 1] == c[axes[1]]][0]
        out[k] += plane[i]
    return out


@pytest.mark.parametrize("mod,drop", [(d3q19, 2), (d3q19, 0), (d3q27, 2), (d3q27, 1)],
                         ids=["d3q19-z", "d3q19-x", "d3q27-z", "d3q27-y"])
def test_double_well_field_uniform_along_an_axis_evolves_as_the_d2q9_model(mod, drop):
    # equal relaxation times, a liquid-side state (rho0 = 1, c_s^2 = 0.02) uniform and
    # mirror-symmetric along the dropped axis: the 3-D oracle with the double well follows
    # the independent D2Q9 C core with its own double-well bulk pressure step for step
    n = {0: 10, 1: 9, 2: 8}
    shape3 = [n[2], n[1], n[0]]
    shape3[2 - drop] = 1
    kappa, tau, rho0 = 0.05, 0.85, 1.0
    m3 = _model(mod, rho0, kappa=kappa, tau_s=tau, tau_b=tau, tau_ghost=tau)
    m2 = th.Model(rho0=rho0, cs2=WELL.cs2(rho0), kappa=kappa, tau_s=tau, tau_b=tau, tau_ghost=tau,
                  p0_rest=WELL.p0(rho0))
    pert = synth.gaussian_field((mod.Q,) + tuple(shape3), seed=21 + drop, scale=0.05)
    flip = mod.C.copy()
    flip[:, drop] *= -1
    mirror = [int(np.where((mod.C == c).all(axis=1))[0][0]) for c in flip]
    pert = 0.5 * (pert + pert[mirror])
    f3 = m3.rest()[:, None, None, None] * (1.0 + pert)
    f2 = _project(mod, f3, drop)
    for _ in range(10):
        f3 = mod.step(f3, m3, eos=WELL)
        f2 = oracle.step(f2, m2, eos=WELL)
        np.testing.assert_allclose(_project(mod, f3, drop), f2, rtol=0, atol=2e-14)
    r = f2.sum(axis=0)
    assert r.std() > 1e-3
    # the quartic terms of p0 mattered: the linear p0 = c_s^2(rho0) rho drifts apart
    g2 = _project(mod, m3.rest()[:, None, None, None] * (1.0 + pert), drop)
    for _ in range(10):
        g2 = oracle.step(g2, m2)
    assert np.abs(g2 - f2).max() > 1e-6


@pytest.mark.parametrize("mod", LATTICES, ids=["d3q19", "d3q27"])
def test_xi_zero_is_rho_times_an_affine_function_of_cs2(mod):
    # the library evaluates the local Xi(0) as rho (A + B c_s^2): pin that structure, and that
    # B vanishes outside the coupled block (the other modes scale with rho alone)
    kw = dict(kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    c1, c2 = 0.2, 0.45
    X1 = mod.Model(1.0, c1, **kw).Xi_zero()
    X2 = mod.Model(1.0, c2, **kw).Xi_zero()
    B = (X2 - X1) / (c2 - c1)
    A = X1 - B * c1
    for rho, c in [(0.7, 0.05), (1.3, 0.3), (0.9, -0.2), (1.0, 0.55)]:
        X = mod.Model(rho, c, **kw).Xi_zero()
        np.testing.assert_allclose(X, rho * (A + B * c), rtol=0, atol=1e-12 * np.abs(X).max())
    coupled = mod.COUPLED
    mask = np.ones_like(B, dtype=bool)
    mask[np.ix_(coupled, coupled)] = False
    assert np.abs(B[mask]).max() < 1e-12 * np.abs(B).max()
    assert np.abs(B[np.ix_(coupled, coupled)]).max() > 1e-6


@pytest.mark.parametrize("mod", LATTICES, ids=["d3q19", "d3q27"])
def test_local_factor_reproduces_xi0_and_clamps_indefinite_blocks(mod):
    kw = dict(kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    nc = [a for a in range(mod.Q) if np.abs(mod.Model(1.0, 0.3, **kw).Xi_zero()[a]).max() > 0]
    for rho, c in [(1.0, 1 / 3), (0.8, 0.05), (1.2, 0.4)]:
        X = mod.Model(rho, c, **kw).Xi_zero()
        L = mod.local_factor(X, mod.COUPLED) if mod is d3q19 else mod.local_factor(X)
        np.testing.assert_allclose((L @ L.T)[np.ix_(nc, nc)], X[np.ix_(nc, nc)], rtol=0,
                                   atol=1e-12 * np.abs(X).max())
    # with these relaxation times the coupled block is indefinite for c_s^2 above about 0.5
    # (and positive semidefinite in the spinodal region, c_s^2 < 0): there the factor stays
    # finite, a clamped pivot leaves its column zero, and the other modes are unchanged
    X = mod.Model(0.7, 0.8, **kw).Xi_zero()
    Bx = X[np.ix_(mod.COUPLED, mod.COUPLED)]
    assert np.linalg.eigvalsh(Bx).min() < -1e-6 * np.abs(Bx).max()
    L = mod.local_factor(X, mod.COUPLED) if mod is d3q19 else mod.local_factor(X)
    assert np.all(np.isfinite(L))
    Bk = L[np.ix_(mod.COUPLED, mod.COUPLED)]
    zero = np.diag(Bk) == 0
    assert zero.any() and np.all(Bk[:, zero] == 0)
    other = [a for a in nc if a not in mod.COUPLED]
    np.testing.assert_allclose(np.diag(L)[other] ** 2, np.diag(X)[other], rtol=1e-13)


@pytest.mark.parametrize("mod", LATTICES, ids=["d3q19", "d3q27"])
def test_local_noise_at_uniform_density_is_the_uniform_noise(mod):
    # Sec. IV: at a uniform density the local noise is the long-wavelength noise of Xi(0),
    # draw for draw
    for cs2, rho0 in [(1 / 3, 1.0), (0.2, 0.9)]:
        m = mod.Model(rho0, cs2, kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
        nx, ny, nz = 4, 3, 2
        rho = np.full((nz, ny, nx), rho0)
        a = mod.noise_lw_local(m, rho, cs2, seed=9, step_index=4)
        nodes = np.arange(nx * ny * nz, dtype=np.uint32).reshape(nz, ny, nx)
        b = mod.noise_lw_nodes(m, nodes, 9, 4)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-13 * np.abs(b).max())


def test_local_noise_covariance_follows_the_density_field():
    # a fixed inhomogeneous density (a double-well interface along x): the sample covariance
    # of the D3Q19 local noise at each node over many steps is Xi(0) at that node's density
    # and c_s^2
    m = d3q19.Model(0.75, WELL.cs2(0.75), kappa=0.03, kT=1e-4, tau_s=0.8, tau_b=1.1, tau_ghost=0.9)
    nx = 12
    x = np.arange(nx)
    rho = (0.75 + 0.25 * np.tanh((x - 6) / 2.0))[None, None, :].copy()
    c2 = WELL.cs2(rho)
    steps = 2500
    acc = np.zeros((19, 19, nx))
    for t in range(steps):
        xi = d3q19.noise_lw_local(m, rho, c2, seed=2, step_index=t)[:, 0, 0, :]
        acc += np.einsum("ax,bx->abx", xi, xi)
    C = acc / steps
    ok = 0
    for k in range(nx):
        X = d3q19.Model(rho[0, 0, k], c2[0, 0, k], m.kappa, m.kT, m.tau_s, m.tau_b, m.tau_ghost).Xi_zero()
        x44, x416, x1616 = X[4, 4], X[4, 16], X[16, 16]
        if not (x44 >= 0 and x1616 >= 0 and x44 * x1616 >= x416 * x416):
            continue
        ok += 1
        for a, b in [(4, 4), (16, 16), (4, 16), (5, 5), (10, 10), (18, 18)]:
            sd = np.sqrt((abs(C[a, a, k] * C[b, b, k]) + X[a, b] ** 2) / steps)
            assert abs(C[a, b, k] - X[a, b]) < 5 * sd, (k, a, b)
    assert ok >= 6
    assert np.all(C[:4] == 0)
