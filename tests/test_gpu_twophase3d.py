"""The two-phase model on the 3-D lattices (include/lbfluct3d.h: lb3_set_eos, LB_NOISE_LW_LOCAL)
against the FP64 oracles (oracle/d3q19.py, oracle/d3q27.py): element by element on liquid
slabs in vapour with the Landau double well, without noise, with the noise at the local
density and, on a liquid-side lattice, with the long-wavelength and the correlated noise; the
re-basing of the
stored state by lb3_set_eos; the local noise against the uniform one at uniform density; the
error paths; and a flat interface relaxing to the tanh profile of width xi of Eq.
(interf-width)."""
import numpy as np
import pytest

import paper_1009_0254_gb300 as lbf
from oracle import d3q19, d3q27
from oracle import theory as th
from paper_1009_0254_gb300 import synth

pytestmark = pytest.mark.gpu
WELL = th.DoubleWell(0.04, 0.5, 1.0)
PARAMS = (1e-4, 0.03, 0.8, 1.1, 0.9)       # kT, kappa, tau_s, tau_b, tau_ghost
TOL, TOL64 = 1e-5, 1e-12
ORACLE = {19: d3q19, 27: d3q27}
MODES = {lbf.LB_NOISE_OFF: 0, lbf.LB_NOISE_LW: 1, lbf.LB_NOISE_LW_LOCAL: 5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0254_gb300 import build
    build.build()
    lbf.load()


def _slab(mod, nx, ny, nz, seed, amp=0.01):
    """A liquid slab in vapour along x (two tanh interfaces of width 2) at rest, each node in
    the rest state of its own density, times (1 + a small perturbation)."""
    x = np.arange(nx)
    d = np.minimum(x - nx / 4.0, 3.0 * nx / 4.0 - x)
    rho = 0.5 * (WELL.rhoL + WELL.rhoV) + 0.5 * (WELL.rhoL - WELL.rhoV) * np.tanh(d / 2.0)
    rest = np.stack([mod.Model(r, WELL.cs2(r), p0_rest=WELL.p0(r)).rest() for r in rho], axis=1)   # [Q, nx]
    pert = synth.gaussian_field((mod.Q, nz, ny, nx), seed=seed, scale=amp)
    return rest[:, None, None, :] * (1.0 + pert)


def _pair(lattice, nx, ny, nz, mode, precision, rho0=0.75, seed=7, state=None):
    mod = ORACLE[lattice]
    g = lbf.Lattice3(nx, ny, nz, seed=seed, rho0=rho0, cs2=1.0 / 3.0, precision=precision, lattice=lattice)
    g.set_eos(lbf.LB_EOS_DOUBLE_WELL, WELL.beta, WELL.rhoV, WELL.rhoL)
    g.set_params(*PARAMS, mode)
    o = mod.Lattice(nx, ny, nz, rho0=rho0, seed=seed, eos=WELL)
    o.set_params(*PARAMS, MODES[mode])
    f0 = _slab(mod, nx, ny, nz, seed + 100) if state is None else state
    g.set_populations(f0, t=0)
    o.f = f0.copy()
    return g, o, f0


@pytest.mark.parametrize("lattice", [19, 27])
@pytest.mark.parametrize("nx,ny,nz", [(32, 6, 4), (21, 5, 3), (7, 3, 2)])
@pytest.mark.parametrize("mode", [lbf.LB_NOISE_OFF, lbf.LB_NOISE_LW_LOCAL])
@pytest.mark.parametrize("precision", [lbf.LB_FP32, lbf.LB_FP64])
def test_double_well_slab_follows_the_oracle(lattice, nx, ny, nz, mode, precision):
    g, o, f0 = _pair(lattice, nx, ny, nz, mode, precision)
    g.step(4)
    o.step(4)
    err = np.abs(g.populations() - o.f).max()
    tol = TOL if precision == lbf.LB_FP32 else TOL64
    print("D3Q%d %s %dx%dx%d mode %d: %.2e" % (lattice, "FP32" if precision == lbf.LB_FP32 else "FP64",
                                             nx, ny, nz, mode, err))
    assert err <= tol
    # the interfaces moved the state: the double well's terms acted
    assert np.abs(o.f - f0).max() > 100 * tol
    if mode == lbf.LB_NOISE_LW_LOCAL:
        q = ORACLE[lattice].Lattice(nx, ny, nz, rho0=0.75, seed=7, eos=WELL)
        q.set_params(*PARAMS, 0)
        q.f = f0.copy()
        q.step(4)
        assert np.abs(q.f - o.f).max() > 100 * tol          # the local noise acted


@pytest.mark.parametrize("lattice", [19, 27])
def test_liquid_side_lattice_with_the_uniform_noise(lattice):
    # rho0 = 1 (the liquid density; c_s^2 = 0.02 > 0): the long-wavelength noise of the linear
    # theory about rho0, with the double well's bulk pressure in every node's equilibrium
    mod = ORACLE[lattice]
    nx, ny, nz = 24, 5, 4
    m = mod.Model(1.0, WELL.cs2(1.0), p0_rest=WELL.p0(1.0))
    f0 = m.rest()[:, None, None, None] * (1.0 + synth.gaussian_field((mod.Q, nz, ny, nx), seed=4, scale=0.02))
    g, o, _ = _pair(lattice, nx, ny, nz, lbf.LB_NOISE_LW, lbf.LB_FP32, rho0=1.0, state=f0)
    g.step(5)
    o.step(5)
    assert np.abs(g.populations() - o.f).max() <= TOL


@pytest.mark.parametrize("lattice", [19, 27])
@pytest.mark.parametrize("precision", [lbf.LB_FP32, lbf.LB_FP64])
def test_set_eos_keeps_the_state_and_rebases_it(lattice, precision):
    mod = ORACLE[lattice]
    nx, ny, nz = 12, 5, 3
    g = lbf.Lattice3(nx, ny, nz, seed=3, rho0=0.8, cs2=0.25, precision=precision, lattice=lattice)
    f0 = _slab(mod, nx, ny, nz, 11)
    g.set_populations(f0, t=0)
    tol = 1e-6 if precision == lbf.LB_FP32 else 1e-14
    g.set_eos(lbf.LB_EOS_DOUBLE_WELL, WELL.beta, WELL.rhoV, WELL.rhoL)
    assert np.abs(g.populations() - f0).max() <= tol
    g.set_eos(lbf.LB_EOS_LINEAR)
    assert np.abs(g.populations() - f0).max() <= tol
    # a uniform rest state of the double well is a fixed point of the step
    g.set_eos(lbf.LB_EOS_DOUBLE_WELL, WELL.beta, WELL.rhoV, WELL.rhoL)
    g.set_params(0.0, 0.05, 0.8, 1.1, 0.9, lbf.LB_NOISE_OFF)
    rest = mod.Model(0.8, WELL.cs2(0.8), p0_rest=WELL.p0(0.8)).rest()
    fr = np.broadcast_to(rest[:, None, None, None], f0.shape).copy()
    g.set_populations(fr, t=0)
    g.step(3)
    assert np.abs(g.populations() - fr).max() <= (1e-6 if precision == lbf.LB_FP32 else 1e-14)


@pytest.mark.parametrize("lattice", [19, 27])
def test_local_noise_at_uniform_density_is_the_uniform_noise(lattice):
    # one step from an exactly uniform state: the local noise (factored on the GPU at the
    # node's density) and the long-wavelength noise (factored on the host) draw the same numbers
    nx, ny, nz = 16, 6, 4
    mod = ORACLE[lattice]
    out = {}
    for mode in (lbf.LB_NOISE_LW, lbf.LB_NOISE_LW_LOCAL):
        g = lbf.Lattice3(nx, ny, nz, seed=21, rho0=1.0, cs2=0.25, lattice=lattice)
        g.set_params(*PARAMS, mode)
        fr = np.broadcast_to(mod.Model(1.0, 0.25).fbar()[:, None, None, None], (mod.Q, nz, ny, nx)).copy()
        g.set_populations(fr, t=5)
        g.step(1)
        out[mode] = g.populations()
    d = np.abs(out[lbf.LB_NOISE_LW] - out[lbf.LB_NOISE_LW_LOCAL]).max()
    assert d <= 1e-7
    assert np.abs(out[lbf.LB_NOISE_LW] - fr).max() > 1e-4


@pytest.mark.parametrize("lattice", [19, 27])
def test_two_phase_error_paths(lattice):
    g = lbf.Lattice3(8, 8, 8, rho0=0.75, lattice=lattice)
    for args in [(lbf.LB_EOS_DOUBLE_WELL, -1.0, 0.5, 1.0), (lbf.LB_EOS_DOUBLE_WELL, 0.04, 1.0, 0.5), (7, 0, 0, 0)]:
        with pytest.raises(lbf.LBError) as e:
            g.set_eos(*args)
        assert e.value.code == lbf.LB_EINVAL
    g.set_eos(lbf.LB_EOS_DOUBLE_WELL, WELL.beta, WELL.rhoV, WELL.rhoL)
    # rho0 = 0.75 lies in the spinodal region: the uniform noise modes are refused ...
    with pytest.raises(lbf.LBError) as e:
        g.set_params(*PARAMS, lbf.LB_NOISE_LW)
    assert e.value.code == lbf.LB_ENOTPSD
    # ... the local noise is not
    g.set_params(*PARAMS, lbf.LB_NOISE_LW_LOCAL)
    g.step(2)
    # parameters that the new linear theory refuses come back as lb3_set_eos's error
    h = lbf.Lattice3(8, 8, 8, rho0=0.75, lattice=lattice)
    h.set_params(*PARAMS, lbf.LB_NOISE_LW)
    with pytest.raises(lbf.LBError) as e:
        h.set_eos(lbf.LB_EOS_DOUBLE_WELL, WELL.beta, WELL.rhoV, WELL.rhoL)
    assert e.value.code == lbf.LB_ENOTPSD
    with pytest.raises(lbf.LBError):
        h.step(1)


@pytest.mark.parametrize("lattice", [19, 27])
def test_flat_interface_relaxes_to_the_tanh_profile_of_width_xi(lattice):
    # a liquid slab with sharp edges, noise off, 128 x 4 x 4: the stationary profile is
    # rho(x) = (rhoL + rhoV)/2 + (rhoL - rhoV)/2 tanh(2 x / xi) with xi of Eq. (interf-width)
    # (the lattice shortens it by a relative O(1/xi^2)) and the bulk at the coexisting densities
    from scipy.optimize import curve_fit
    mod = ORACLE[lattice]
    nx, ny, nz, kappa = 128, 4, 4, 0.03
    g = lbf.Lattice3(nx, ny, nz, seed=1, rho0=0.75, lattice=lattice)
    g.set_eos(lbf.LB_EOS_DOUBLE_WELL, WELL.beta, WELL.rhoV, WELL.rhoL)
    g.set_params(0.0, kappa, 1.0, 1.0, 1.0, lbf.LB_NOISE_OFF)
    x = np.arange(nx)
    prof = np.where((x >= 32) & (x < 96), WELL.rhoL, WELL.rhoV)
    rest = np.stack([mod.Model(r, WELL.cs2(r), p0_rest=WELL.p0(r)).rest() for r in prof], axis=1)
    f0 = np.broadcast_to(rest[:, None, None, :], (mod.Q, nz, ny, nx)).copy()
    g.set_populations(f0, t=0)
    mass0 = g.sums()[0]
    g.step(10000)
    f = g.populations()
    rho = f.sum(axis=0)
    assert np.abs(rho - rho[:1, :1, :]).max() < 1e-5          # flat: no y or z dependence
    assert abs(g.sums()[0] - mass0) < 1e-6 * mass0
    xi = WELL.width(kappa)
    fun = lambda xx, x0, w, a, b: a + b * np.tanh(2 * (xx - x0) / w)
    p, _ = curve_fit(fun, x[16:64].astype(float), rho[0, 0, 16:64],
                     p0=[32, xi, 0.5 * (WELL.rhoL + WELL.rhoV), 0.5 * (WELL.rhoL - WELL.rhoV)])
    print("D3Q%d xi: Eq. (interf-width) %.4f, stationary profile %.4f" % (lattice, xi, p[1]))
    assert abs(p[1] / xi - 1) < 0.7 / xi ** 2
    assert abs(rho[0, 0, 64] - WELL.rhoL) < 1e-3 and abs(rho[0, 0, 0] - WELL.rhoV) < 1e-3


@pytest.mark.parametrize("lattice", [19, 27])
def test_correlated_noise_on_a_double_well_lattice(lattice):
    # rho0 = 1 (the liquid density, c_s^2 = 0.02): the correlated noise Xi(k) of the linear
    # theory about rho0 (c_s^2(k) = 0.02 + rho0 kappa s(k)) with the double well's bulk pressure
    # in every node's equilibrium
    mod = ORACLE[lattice]
    nx, ny, nz = 21, 6, 5
    params = (1e-4, 0.04, 0.8, 1.1, 0.9)
    m = mod.Model(1.0, WELL.cs2(1.0), p0_rest=WELL.p0(1.0))
    f0 = m.rest()[:, None, None, None] * (1.0 + synth.gaussian_field((mod.Q, nz, ny, nx), seed=6, scale=0.02))
    g = lbf.Lattice3(nx, ny, nz, seed=9, rho0=1.0, lattice=lattice)
    g.set_eos(lbf.LB_EOS_DOUBLE_WELL, WELL.beta, WELL.rhoV, WELL.rhoL)
    g.set_params(*params, lbf.LB_NOISE_FULL_RS)
    o = mod.Lattice(nx, ny, nz, rho0=1.0, seed=9, eos=WELL)
    o.set_params(*params, mod.NOISE_FULL_RS)
    g.set_populations(f0, t=0)
    o.f = f0.copy()
    g.step(5)
    o.step(5)
    err = np.abs(g.populations() - o.f).max()
    print("D3Q%d RS double well: %.2e" % (lattice, err))
    assert err <= TOL
