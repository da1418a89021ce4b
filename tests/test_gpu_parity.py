"""GPU path against the FP64 oracle through the C ABI (element by element, same seeded
inputs, same Philox counters).  Tolerance: max |f_gpu - f_oracle| <= 1e-5 after 100
steps in FP32 storage (the bar the workload sets for populations)."""
import numpy as np
import pytest

import oracle
import paper_1009_0254_gb300 as lbf
from oracle import theory as th
from paper_1009_0254_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5

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


def _pair(nx, ny, seed, rho0, cs2, params, mode, init_scale):
    """A GPU lattice and an oracle lattice with identical state and parameters."""
    g = lbf.Lattice(nx, ny, seed=seed, rho0=rho0, cs2=cs2)
    o = oracle.Lattice(nx, ny, rho0=rho0, cs2=cs2, seed=seed)
    g.set_params(*params, mode)
    o.set_params(*params, mode)
    if init_scale > 0:
        pert = synth.gaussian_field((9, ny, nx), seed=1000 + nx * 7 + ny, scale=init_scale)
        f0 = o.model.fbar()[:, None, None] * (1.0 + pert)
        o.f = f0.copy()
        g.set_populations(f0, t=0)
    return g, o


CONFIG1 = (1e-4, 0.01, 1.0, 1.0, 1.0)   # kT, kappa, tau_s, tau_b, tau_ghost


@pytest.fixture(params=["tma", "simple", "sweep", "sweep6"])
def kernel(request, monkeypatch):
    """Every step kernel: TMA-staged persistent (default), plain, warp-autonomous sweep."""
    monkeypatch.setenv("LBFLUCT_STEP_KERNEL", request.param)
    return request.param


@pytest.mark.parametrize("mode", ["full", "lw", "diag", "off", "rs"])
def test_parity_64x64_config1(mode, kernel):
    # 64^2, rho0 = 1, kappa = 0.01, tau = 1, kT = 1e-4, cs2 = 1/3, seed 42, start at rest
    scale = 0.01 if mode == "off" else 0.0
    g, o = _pair(64, 64, 42, 1.0, 1 / 3, CONFIG1, MODES[mode], scale)
    g.step(100)
    o.step(100)
    assert g.t == 100
    err = np.abs(g.populations() - o.f).max()
    assert err <= TOL, err
    if mode != "off":
        assert np.abs(o.f - o.model.fbar()[:, None, None]).max() > 100 * TOL   # noise acted


@pytest.mark.parametrize("nx,ny,mode", [(6, 10, "lw"), (33, 17, "lw"), (100, 36, "diag"), (2, 2, "lw"),
                                        (37, 5, "off"), (64, 32, "full"), (16, 128, "full"), (2, 8, "full"),
                                        (300, 20, "lw"), (129, 9, "diag"), (256, 8, "full"), (512, 2, "full"),
                                        (1024, 4, "full"), (6, 10, "rs"), (33, 17, "rs"), (2, 2, "rs"),
                                        (100, 36, "rs"), (129, 9, "rs"), (1024, 4, "rs"), (3, 70, "rs")])
def test_parity_ragged_and_small_lattices(nx, ny, mode, kernel):
    g, o = _pair(nx, ny, 7, 1.0, 1 / 3, (2e-4, 0.02, 0.8, 1.0, 1.0), MODES[mode], 0.01)
    g.step(60)
    o.step(60)
    err = np.abs(g.populations() - o.f).max()
    assert err <= TOL, err


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("nx,ny,mode", [(100, 36, "lw"), (70, 50, "off"), (128, 64, "full"), (100, 36, "rs"),
                                        (130, 70, "rs")])
def test_parity_every_tile_shape(tile, nx, ny, mode, monkeypatch):
    # each TMA tile shape (32x16, 32x32, 64x8, 64x16, 32x16 on 128 threads) on ragged edges
    monkeypatch.setenv("LBFLUCT_STEP_KERNEL", "tma")
    monkeypatch.setenv("LBFLUCT_TMA_TILE", str(tile))
    g, o = _pair(nx, ny, 11, 1.0, 1 / 3, (2e-4, 0.02, 0.8, 1.0, 1.0), MODES[mode], 0.01)
    g.step(40)
    o.step(40)
    assert np.abs(g.populations() - o.f).max() <= TOL


def test_parity_across_noise_mode_changes(monkeypatch):
    # the default tile shape follows the noise mode; switching modes mid-run re-encodes the
    # tensor maps and the trajectory stays the oracle's
    monkeypatch.setenv("LBFLUCT_STEP_KERNEL", "tma")
    monkeypatch.delenv("LBFLUCT_TMA_TILE", raising=False)
    params = (2e-4, 0.02, 0.8, 1.0, 1.0)
    g, o = _pair(128, 64, 13, 1.0, 1 / 3, params, MODES["lw"], 0.01)
    for mode in ["lw", "full", "off", "rs", "lw", "diag", "full", "rs"]:
        g.set_params(*params, MODES[mode])
        o.set_params(*params, MODES[mode])
        g.step(15)
        o.step(15)
        assert np.abs(g.populations() - o.f).max() <= TOL, mode


@pytest.mark.parametrize("mode", ["lw", "full", "rs"])
def test_parity_nonideal_sound_speed(mode, kernel):
    # cs != sigma_s: rest populations differ from w_i rho0 and Xi_49(0) != 0
    g, o = _pair(32, 32, 9, 0.9, 0.265 ** 2, (1e-5, 0.08, 1.0, 1.1, 0.9), MODES[mode], 0.005)
    g.step(100)
    o.step(100)
    err = np.abs(g.populations() - o.f).max()
    assert err <= TOL, err


def test_moments_and_sums_match_oracle():
    g, o = _pair(40, 24, 3, 1.1, 1 / 3, (1e-4, 0.02, 0.8, 1.0, 1.0), lbf.LB_NOISE_LW, 0.01)
    g.step(10)
    o.step(10)
    m, s = g.moments()
    mo = o.moments()
    np.testing.assert_allclose(m, mo, atol=4 * TOL)
    # the device FP64 reduction equals the sum of the device's own FP64 moments ...
    np.testing.assert_allclose(s, m[:3].sum(axis=(1, 2)), rtol=1e-13, atol=1e-13)
    # ... and the oracle's sums up to the FP32 rounding of n stored nodes (~1e-7 each)
    n = 40 * 24
    np.testing.assert_allclose(s, mo[:3].sum(axis=(1, 2)), rtol=0, atol=30 * 1e-7 * np.sqrt(n))


def test_full_size_sampled_parity_and_conservation(kernel):
    # the roofline workload's size (4096^2), one step from a seeded random state in each
    # noise mode, compared on sampled nodes (corners and edges included)
    nx = ny = 4096
    params = (1e-4, 0.01, 0.8, 1.0, 1.0)
    m = th.Model(1.0, 1 / 3, 0.01, 1e-4, 0.8, 1.0, 1.0)
    pert = synth.gaussian_field((9, ny, nx), seed=5, scale=0.01)
    f0 = m.fbar()[:, None, None] * (1.0 + pert)
    del pert
    nodes = synth.sample_nodes(nx, ny, 2000, seed=6)
    g = lbf.Lattice(nx, ny, seed=42)
    for mode in ["lw", "full", "rs"]:
        g.set_params(*params, MODES[mode])
        g.set_populations(f0, t=123)
        s0 = g.sums()
        g.step(1)
        fg = g.populations().reshape(9, -1)[:, nodes].T
        fo = oracle.step_sampled(f0, m, MODES[mode], 42, 123, nodes)
        err = np.abs(fg - fo).max()
        assert err <= TOL, (mode, err)
        g.step(99)
        s1 = g.sums()
        assert abs(s1[0] - s0[0]) < 1e-7 * nx * ny
        assert np.all(np.abs(s1[1:] - s0[1:]) < 1e-7 * nx * ny)


@pytest.mark.parametrize("mode", ["full", "lw", "rs"])
def test_parity_64x64_config1_1000_steps(mode):
    # the same configuration over its full 1000 steps (default step kernel): the FP32
    # path stays within the population bar of the FP64 oracle, and both conserve mass
    g, o = _pair(64, 64, 42, 1.0, 1 / 3, CONFIG1, MODES[mode], 0.0)
    g.step(1000)
    o.step(1000)
    fg = g.populations()
    err = np.abs(fg - o.f).max()
    # conserved sums: the FP32 rounding of 9 n stored deviations per step (relative 2^-24
    # each, independent) adds up as a random walk over nodes and steps
    dmax = np.abs(o.f - o.model.fbar()[:, None, None]).max()
    walk = np.sqrt(9 * 64 * 64 * 1000) * 2.0 ** -24 * dmax
    ds = np.abs(g.sums() - o.moments()[:3].sum(axis=(1, 2))).max()
    print("1000 steps %s: max |f - f_oracle| = %.3e, sums diff %.3e (walk %.3e)" % (mode, err, ds, walk))
    assert err <= TOL, err
    assert ds <= 10 * walk, (ds, walk)


@pytest.mark.parametrize("mode,cs2,kappa", [("lw", 0.15 ** 2, 0.03), ("lw", 1 / 3, 0.01), ("full", 1 / 3, 0.03),
                                           ("diag", 0.25 ** 2, 0.02), ("rs", 0.265 ** 2, 0.08), ("rs", 1 / 3, 0.03)])
def test_parity_eigen_noise_factor(mode, cs2, kappa):
    # Sec. IV: the eigen-decomposition factor of the noise matrix instead of Cholesky
    params = (1e-4, kappa, 1.0, 1.1, 0.9)
    g = lbf.Lattice(64, 32, seed=13, cs2=cs2)
    o = oracle.Lattice(64, 32, cs2=cs2, seed=13)
    g.set_noise_factor(lbf.LB_FACTOR_EIGEN)
    g.set_params(*params, MODES[mode])
    o.set_params(*params, MODES[mode], factor="eigen")
    pert = synth.gaussian_field((9, 32, 64), seed=77, scale=0.005)
    f0 = o.model.fbar()[:, None, None] * (1.0 + pert)
    o.f = f0.copy()
    g.set_populations(f0, t=0)
    g.step(60)
    o.step(60)
    err = np.abs(g.populations() - o.f).max()
    assert err <= TOL, err
    # and the realisation really differs from the Cholesky one where Xi49 != 0
    if mode == "lw" and cs2 != 1 / 3:
        c = oracle.Lattice(64, 32, cs2=cs2, seed=13)
        c.set_params(*params, MODES[mode])
        c.f = f0.copy()
        c.step(60)
        assert np.abs(c.f - o.f).max() > 100 * TOL


def test_reproducible_and_resumable(kernel):
    a = lbf.Lattice(64, 64, seed=11)
    b = lbf.Lattice(64, 64, seed=11)
    for L in (a, b):
        L.set_params(1e-4, 0.01, 0.8, 1.0, 1.0, lbf.LB_NOISE_FULL)
    a.step(100)
    b.step(50)
    ck = b.populations()
    c = lbf.Lattice(64, 64, seed=11)
    c.set_params(1e-4, 0.01, 0.8, 1.0, 1.0, lbf.LB_NOISE_FULL)
    c.set_populations(ck, t=50)
    c.step(50)
    b.step(50)
    pa, pb, pc = a.populations(), b.populations(), c.populations()
    assert np.array_equal(pa, pb)          # bitwise: same seed, same counters
    assert np.array_equal(pa, pc)          # resumed from a checkpoint
    d = lbf.Lattice(64, 64, seed=12)
    d.set_params(1e-4, 0.01, 0.8, 1.0, 1.0, lbf.LB_NOISE_FULL)
    d.step(100)
    assert not np.array_equal(pa, d.populations())


@pytest.mark.parametrize("nx,ny,nb", [(64, 32, 24), (256, 128, 64), (2, 8, 4), (8, 2, 4), (128, 512, 300)])
def test_spectra_match_oracle(nx, ny, nb):
    # half-plane binning: rows with and without a mirror row, lanes beyond nx/2, several
    # warp units per row, more bins than wavevectors in some
    g, o = _pair(nx, ny, 21, 1.0, 1 / 3, (1e-4, 0.02, 0.8, 1.0, 1.0), lbf.LB_NOISE_LW, 0.01)
    g.set_sampling(1, nb)
    g.step(3)
    o_acc = np.zeros((3, nb))
    for _ in range(3):
        o.step(1)
        S, L, T, cnt = oracle.spectra_sample(o.f, o.model.rho0, nb)
        o_acc += np.array([S, L, T])
    Sg, Lg, Tg, cg, ns = g.structure_factor()
    assert ns == 3
    np.testing.assert_array_equal(cg, cnt)
    den = np.where(cnt > 0, cnt * 3, 1)
    for got, ref in zip([Sg, Lg, Tg], o_acc / den):
        np.testing.assert_allclose(got, ref, rtol=1e-4, atol=1e-12)


def test_api_errors():
    L = lbf.Lattice(16, 16)
    with pytest.raises(lbf.LBError) as e:
        L.step(1)
    assert e.value.code == lbf.LB_ESTATE
    with pytest.raises(lbf.LBError) as e:
        L.set_params(1e-4, 0.01, 0.5, 1.0, 1.0, lbf.LB_NOISE_LW)
    assert e.value.code == lbf.LB_EINVAL
    with pytest.raises(lbf.LBError) as e:
        L.set_params(1e-4, 0.06, 1.0, 1.0, 1.0, lbf.LB_NOISE_FULL)
    assert e.value.code == lbf.LB_ENOTPSD
    odd = lbf.Lattice(12, 16)
    with pytest.raises(lbf.LBError):
        odd.set_params(1e-4, 0.01, 1.0, 1.0, 1.0, lbf.LB_NOISE_FULL)
    with pytest.raises(lbf.LBError):
        odd.set_sampling(10, 8)
    L.set_params(0.05, 0.01, 1.0, 1.0, 1.0, lbf.LB_NOISE_LW)
    assert lbf.lb_warnings(L.ctx) & lbf.LB_WARN_LOW_MACH
    with pytest.raises(lbf.LBError):
        lbf.Lattice(1, 16)


def test_kernel_timing_samples_every_kth_launch():
    L = lbf.Lattice(32, 32)
    L.set_params(1e-4, 0.01, 1.0, 1.0, 1.0, lbf.LB_NOISE_LW)
    with pytest.raises(lbf.LBError) as e:
        lbf.lb_set_kernel_timing(L.ctx, -1)
    assert e.value.code == lbf.LB_EINVAL
    lbf.lb_set_kernel_timing(L.ctx, 3)
    L.step(10)                                     # launches 0, 3, 6, 9 are timed
    ms, k = lbf.lb_kernel_time(L.ctx)
    assert k == 4 and ms > 0
    lbf.lb_set_kernel_timing(L.ctx, 1)
    L.step(5)
    assert lbf.lb_kernel_time(L.ctx)[1] == 5
    lbf.lb_set_kernel_timing(L.ctx, 0)
    L.step(2)
    assert lbf.lb_kernel_time(L.ctx)[1] == 0
