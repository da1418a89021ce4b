"""FP64 storage and arithmetic on the GPU (LB_FP64) against the FP64 oracle: the same
trajectory to rounding, for every noise mode, ragged sizes, a non-ideal sound speed and the
config-1 lattice over 1000 steps."""
import numpy as np
import pytest

import oracle
import paper_1009_0254_gb300 as lbf
from paper_1009_0254_gb300 import synth

pytestmark = pytest.mark.gpu
TOL64 = 1e-12       # FP64 on both sides: only the order of rounding differs

MODES = {"off": lbf.LB_NOISE_OFF, "lw": lbf.LB_NOISE_LW, "full": lbf.LB_NOISE_FULL, "diag": lbf.LB_NOISE_DIAG,
         "rs": lbf.LB_NOISE_FULL_RS}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0254_gb300 import build
    build.build()
    lbf.load()


def _pair(nx, ny, seed, rho0, cs2, params, mode, scale, factor=None):
    g = lbf.Lattice(nx, ny, seed=seed, rho0=rho0, cs2=cs2, precision=lbf.LB_FP64)
    o = oracle.Lattice(nx, ny, rho0=rho0, cs2=cs2, seed=seed)
    if factor == "eigen":
        g.set_noise_factor(lbf.LB_FACTOR_EIGEN)
    g.set_params(*params, mode)
    o.set_params(*params, mode, factor=factor)
    if scale > 0:
        pert = synth.gaussian_field((9, ny, nx), seed=3000 + nx + ny, scale=scale)
        f0 = o.model.fbar()[:, None, None] * (1.0 + pert)
        o.f = f0.copy()
        g.set_populations(f0, t=0)
    return g, o


@pytest.mark.parametrize("nx,ny,mode", [(64, 32, "full"), (64, 32, "lw"), (33, 17, "lw"), (40, 24, "diag"),
                                        (37, 5, "off"), (2, 2, "lw"), (16, 128, "full"), (8, 2, "full"),
                                        (64, 32, "rs"), (33, 17, "rs"), (2, 2, "rs"), (70, 9, "rs")])
def test_fp64_follows_oracle_to_rounding(nx, ny, mode):
    g, o = _pair(nx, ny, 5, 1.0, 1 / 3, (2e-4, 0.02, 0.8, 1.1, 0.9), MODES[mode], 0.01)
    g.step(100)
    o.step(100)
    err = np.abs(g.populations() - o.f).max()
    assert err <= TOL64, err


@pytest.mark.parametrize("mode", ["full", "lw", "rs"])
def test_fp64_nonideal_and_eigen_factor(mode):
    g, o = _pair(64, 32, 9, 0.9, 0.265 ** 2, (1e-5, 0.08, 1.0, 1.1, 0.9), MODES[mode], 0.005, factor="eigen")
    g.step(80)
    o.step(80)
    assert np.abs(g.populations() - o.f).max() <= TOL64


def test_fp64_config1_1000_steps():
    # 64^2, rho0 = 1, kappa = 0.01, tau = 1, kT = 1e-4, cs2 = 1/3, seed 42, rest start,
    # correlated (full FDT) noise: the plain FP64 run of the first configuration
    g, o = _pair(64, 64, 42, 1.0, 1 / 3, (1e-4, 0.01, 1.0, 1.0, 1.0), lbf.LB_NOISE_FULL, 0.0)
    g.step(1000)
    o.step(1000)
    err = np.abs(g.populations() - o.f).max()
    print("FP64 config 1, 1000 steps: max |f - f_oracle| = %.3e" % err)
    assert err <= 10 * TOL64
    s = g.sums()
    # both conserve mass and momentum to FP64 rounding (the oracle, which stores full
    # populations, drifts by ~3e-13 of the mass over the 1000 steps)
    np.testing.assert_allclose(s, o.moments()[:3].sum(axis=(1, 2)), rtol=0, atol=1e-12 * 64 * 64)
    assert abs(s[0] - 64 * 64) < 1e-12 * 64 * 64


def test_fp64_moments_spectra_and_limits():
    g, o = _pair(32, 32, 2, 1.0, 1 / 3, (1e-4, 0.02, 0.8, 1.0, 1.0), lbf.LB_NOISE_LW, 0.01)
    g.set_sampling(1, 16)
    g.step(3)
    acc = np.zeros((3, 16))
    for _ in range(3):
        o.step(1)
        S, L, T, cnt = oracle.spectra_sample(o.f, 1.0, 16)
        acc += np.array([S, L, T])
    m, _ = g.moments()
    np.testing.assert_allclose(m, o.moments(), atol=1e-12)
    Sg, Lg, Tg, cg, ns = g.structure_factor()
    den = np.where(cnt > 0, cnt * 3, 1)
    for got, ref in zip([Sg, Lg, Tg], acc / den):
        np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-12)     # FP32 transforms
    # correlated noise with FP64 storage is limited to ny <= 4096
    big = lbf.Lattice(16, 8192, seed=1, precision=lbf.LB_FP64)
    with pytest.raises(lbf.LBError) as e:
        big.set_params(1e-4, 0.01, 1.0, 1.0, 1.0, lbf.LB_NOISE_FULL)
    assert e.value.code == lbf.LB_EINVAL


def test_fp64_config1_1000_steps_real_space_correlated_noise():
    # the first configuration with the correlated noise built in real space (the same
    # covariance Xi(k) as the k-space construction)
    g, o = _pair(64, 64, 42, 1.0, 1 / 3, (1e-4, 0.01, 1.0, 1.0, 1.0), lbf.LB_NOISE_FULL_RS, 0.0)
    g.step(1000)
    o.step(1000)
    err = np.abs(g.populations() - o.f).max()
    print("FP64 config 1 (real-space correlated noise), 1000 steps: max |f - f_oracle| = %.3e" % err)
    assert err <= 10 * TOL64
