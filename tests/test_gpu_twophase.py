"""Two-phase runs on the GPU against the FP64 oracle: the Landau double-well equation of
state of Sec. II A (lb_set_eos) and the uncorrelated noise at the local density and sound
speed (LB_NOISE_LW_LOCAL, Sec. IV / Sec. V B), on a liquid slab in its vapour."""
import numpy as np
import pytest

import oracle
import paper_1009_0254_gb300 as lbf
from oracle import theory as th
from paper_1009_0254_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5              # the FP32 population bar
TOL64 = 1e-12

EOS = th.DoubleWell(0.04, 0.5, 1.0)            # the capillary parameters of Sec. V B
KAPPA = 0.03


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0254_gb300 import build
    build.build()
    lbf.load()


def slab(nx, ny, seed, amp=0.01, eos=EOS, width=4.9):
    """A liquid slab across x in [nx/4, 3nx/4) with tanh edges, each node at the rest
    equilibrium of its own density (p0 of the double well), plus a seeded perturbation."""
    x = np.arange(nx)
    mid, half = 0.5 * (eos.rhoL + eos.rhoV), 0.5 * (eos.rhoL - eos.rhoV)
    prof = mid + half * (np.tanh(2 * (x - nx / 4) / width) - np.tanh(2 * (x - 3 * nx / 4) / width)) - half
    f = np.zeros((9, ny, nx))
    for i, r in enumerate(prof):
        f[:, :, i] = th.Model(rho0=r, cs2=eos.cs2(r), p0_rest=eos.p0(r)).rest()[:, None]
    return f * (1.0 + synth.gaussian_field((9, ny, nx), seed=seed, scale=amp))


def _pair(nx, ny, seed, params, mode, precision=lbf.LB_FP32, rho0=0.75, eos=EOS):
    g = lbf.Lattice(nx, ny, seed=seed, rho0=rho0, precision=precision)
    g.set_eos(lbf.LB_EOS_DOUBLE_WELL, eos.beta, eos.rhoV, eos.rhoL)
    g.set_params(*params, mode)
    o = oracle.Lattice(nx, ny, rho0=rho0, seed=seed, eos=eos)
    o.set_params(*params, mode)
    f0 = slab(nx, ny, seed=100 + nx + ny)
    g.set_populations(f0, t=0)
    o.f = f0.copy()
    return g, o


@pytest.fixture(params=["tma", "simple", "sweep"])
def kernel(request, monkeypatch):
    monkeypatch.setenv("LBFLUCT_STEP_KERNEL", request.param)
    monkeypatch.delenv("LBFLUCT_TMA_TILE", raising=False)
    return request.param


@pytest.mark.parametrize("nx,ny,mode", [(64, 32, "off"), (64, 32, "local"), (100, 36, "local"), (33, 17, "off"),
                                        (130, 9, "local")])
def test_double_well_slab_follows_oracle(nx, ny, mode, kernel):
    m = {"off": lbf.LB_NOISE_OFF, "local": lbf.LB_NOISE_LW_LOCAL}[mode]
    g, o = _pair(nx, ny, 7, (1e-6, KAPPA, 1.0, 1.0, 1.0), m)
    g.step(50)
    o.step(50)
    err = np.abs(g.populations() - o.f).max()
    print("%s %s %dx%d: %.2e" % (kernel, mode, nx, ny, err))
    assert err <= TOL, err
    if m != lbf.LB_NOISE_OFF:
        q = oracle.Lattice(nx, ny, rho0=0.75, seed=7, eos=EOS)
        q.set_params(1e-6, KAPPA, 1.0, 1.0, 1.0, oracle.NOISE_OFF)
        q.f = slab(nx, ny, seed=100 + nx + ny)
        q.step(50)
        assert np.abs(q.f - o.f).max() > 100 * TOL          # the noise acted


@pytest.mark.parametrize("tile", range(5))
def test_local_noise_every_tile_shape(tile, monkeypatch):
    # the local-density noise with p0 = cs2 rho runs on the TMA kernels: every tile shape,
    # on a state whose density varies by tens of percent from node to node
    monkeypatch.setenv("LBFLUCT_STEP_KERNEL", "tma")
    monkeypatch.setenv("LBFLUCT_TMA_TILE", str(tile))
    nx, ny = 100, 36
    params = (1e-5, 0.02, 0.8, 1.1, 0.9)
    g = lbf.Lattice(nx, ny, seed=3, cs2=0.2 ** 2)
    o = oracle.Lattice(nx, ny, seed=3, cs2=0.2 ** 2)
    g.set_params(*params, lbf.LB_NOISE_LW_LOCAL)
    o.set_params(*params, oracle.NOISE_LW_LOCAL)
    f0 = o.model.fbar()[:, None, None] * (1.0 + synth.clipped_gaussian_field((9, ny, nx), 31, 0.2, 3.5))
    g.set_populations(f0, t=0)
    o.f = f0.copy()
    g.step(20)
    o.step(20)
    assert np.abs(g.populations() - o.f).max() <= TOL


@pytest.mark.parametrize("mode", [lbf.LB_NOISE_OFF, lbf.LB_NOISE_LW_LOCAL])
def test_double_well_fp64_to_rounding(mode):
    g, o = _pair(64, 32, 5, (1e-6, KAPPA, 0.8, 1.1, 0.9), mode, precision=lbf.LB_FP64)
    g.step(100)
    o.step(100)
    err = np.abs(g.populations() - o.f).max()
    print("FP64 double well: %.2e" % err)
    assert err <= TOL64


def test_set_eos_keeps_the_populations_and_conserves_mass():
    nx, ny = 48, 16
    g = lbf.Lattice(nx, ny, seed=2, rho0=0.75)
    f0 = slab(nx, ny, seed=4)
    g.set_populations(f0, t=0)
    g.set_eos(lbf.LB_EOS_DOUBLE_WELL, EOS.beta, EOS.rhoV, EOS.rhoL)
    np.testing.assert_allclose(g.populations(), f0, rtol=0, atol=1e-7)      # FP32 storage of deviations
    g.set_params(1e-6, KAPPA, 1.0, 1.0, 1.0, lbf.LB_NOISE_LW_LOCAL)
    s0 = g.sums()
    g.step(500)
    s1 = g.sums()
    np.testing.assert_allclose(s1, s0, rtol=0, atol=1e-3)
    g.set_eos(lbf.LB_EOS_LINEAR)
    with pytest.raises(lbf.LBError) as e:
        g.set_eos(lbf.LB_EOS_DOUBLE_WELL, -1.0, 0.5, 1.0)
    assert e.value.code == lbf.LB_EINVAL
    # the spinodal density has c_s^2 < 0: modes built on the linear theory about rho0 refuse
    h = lbf.Lattice(16, 16, seed=1, rho0=0.75)
    h.set_eos(lbf.LB_EOS_DOUBLE_WELL, EOS.beta, EOS.rhoV, EOS.rhoL)
    with pytest.raises(lbf.LBError):
        h.set_params(1e-6, KAPPA, 1.0, 1.0, 1.0, lbf.LB_NOISE_LW)
    h.set_params(1e-6, KAPPA, 1.0, 1.0, 1.0, lbf.LB_NOISE_LW_LOCAL)


@pytest.mark.parametrize("cs2", [1 / 3, 0.15 ** 2])
def test_local_noise_at_uniform_density_is_the_uniform_noise(cs2):
    # Sec. IV: at uniform density the local noise is the long-wavelength noise of Xi(0);
    # the GPU's per-node factors (FP32) follow the host's FP64 ones to rounding
    a = lbf.Lattice(64, 32, seed=8, cs2=cs2)
    b = lbf.Lattice(64, 32, seed=8, cs2=cs2)
    a.set_params(1e-4, 0.02, 0.8, 1.1, 0.9, lbf.LB_NOISE_LW)
    b.set_params(1e-4, 0.02, 0.8, 1.1, 0.9, lbf.LB_NOISE_LW_LOCAL)
    a.step(1)
    b.step(1)
    assert np.abs(a.populations() - b.populations()).max() < 1e-8
    o = oracle.Lattice(64, 32, seed=8, cs2=cs2)
    o.set_params(1e-4, 0.02, 0.8, 1.1, 0.9, oracle.NOISE_LW_LOCAL)
    a.step(59)
    b.step(59)
    o.step(60)
    assert np.abs(b.populations() - o.f).max() <= TOL


def test_flat_interface_on_the_gpu_relaxes_to_the_oracle_profile():
    # the interface pin of the oracle (tanh of width xi, Eq. interf-width) on the GPU:
    # 10^4 deterministic steps from a sharp slab, same stationary profile as the oracle
    nx, ny = 128, 2
    x = np.arange(nx)
    prof = np.where((x >= 32) & (x < 96), EOS.rhoL, EOS.rhoV)
    f0 = np.zeros((9, ny, nx))
    for i, r in enumerate(prof):
        f0[:, :, i] = th.Model(rho0=r, cs2=EOS.cs2(r), p0_rest=EOS.p0(r)).rest()[:, None]
    g = lbf.Lattice(nx, ny, seed=1, rho0=0.75, precision=lbf.LB_FP64)
    g.set_eos(lbf.LB_EOS_DOUBLE_WELL, EOS.beta, EOS.rhoV, EOS.rhoL)
    g.set_params(0.0, KAPPA, 1.0, 1.0, 1.0, lbf.LB_NOISE_OFF)
    g.set_populations(f0, t=0)
    g.step(10000)
    o = oracle.Lattice(nx, ny, rho0=0.75, seed=1, eos=EOS)
    o.set_params(0.0, KAPPA, 1.0, 1.0, 1.0, oracle.NOISE_OFF)
    o.f = f0.copy()
    o.step(10000)
    rg = g.populations().sum(axis=0)[0]
    ro = o.f.sum(axis=0)[0]
    assert np.abs(rg - ro).max() < 1e-10
    assert abs(rg[64] - EOS.rhoL) < 1e-3 and abs(rg[0] - EOS.rhoV) < 1e-3
