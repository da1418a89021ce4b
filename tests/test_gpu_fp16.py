"""FP16 deviation storage (populations kept as (f_i - fbar_i)/w_i in FP16, arithmetic in
FP32) against the FP64 oracle: per-step rounding, conservation and the equilibrium
statistics of Sec. V A."""
import numpy as np
import pytest

import oracle
import paper_1009_0254_gb300 as lbf
from oracle import theory as th
from paper_1009_0254_gb300 import synth

pytestmark = pytest.mark.gpu
HALF_ULP = 2.0 ** -11            # relative rounding unit of FP16 (round to nearest)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0254_gb300 import build
    build.build()
    lbf.load()


@pytest.fixture(params=["tma", "simple", "sweep", "sweep6"])
def kernel(request, monkeypatch):
    monkeypatch.setenv("LBFLUCT_STEP_KERNEL", request.param)
    return request.param


@pytest.mark.parametrize("nx,ny,mode", [(64, 64, lbf.LB_NOISE_FULL), (33, 17, lbf.LB_NOISE_LW),
                                        (100, 36, lbf.LB_NOISE_DIAG), (100, 36, lbf.LB_NOISE_FULL_RS),
                                        (64, 64, lbf.LB_NOISE_FULL_RS)])
def test_fp16_follows_oracle_within_rounding(nx, ny, mode, kernel):
    # Each step rounds every stored g_i = df_i / w_i to FP16 (error <= 2^-11 |g_i|); the step
    # itself is a contraction on every non-conserved mode, so after N steps the population
    # error is bounded by N * 2^-11 * max|g| * max w_i, with max|g| taken along the oracle's
    # own trajectory.
    params = (2e-4, 0.02, 0.8, 1.0, 1.0)
    g = lbf.Lattice(nx, ny, seed=5, precision=lbf.LB_FP16DEV)
    o = oracle.Lattice(nx, ny, seed=5)
    g.set_params(*params, mode)
    o.set_params(*params, mode)
    f0 = o.model.fbar()[:, None, None] * (1.0 + synth.gaussian_field((9, ny, nx), seed=17, scale=0.01))
    o.f = f0.copy()
    g.set_populations(f0, t=0)
    nsteps = 20
    gmax = 0.0
    for _ in range(nsteps):
        gmax = max(gmax, np.abs((o.f - o.model.fbar()[:, None, None]) / th.W[:, None, None]).max())
        o.step(1)
    g.step(nsteps)
    err = np.abs(g.populations() - o.f).max()
    bound = nsteps * HALF_ULP * gmax * th.W.max()
    assert err <= bound, (err, bound)
    assert err > 1e-9          # FP16 storage really is in use


def test_fp16_mass_drift_is_rounding_sized():
    n = 128
    L = lbf.Lattice(n, n, seed=8, precision=lbf.LB_FP16DEV)
    L.set_params(1e-4, 0.01, 0.8, 1.0, 1.0, lbf.LB_NOISE_LW)
    s0 = L.sums()
    L.step(1000)
    s1 = L.sums()
    # per node per step the rounding error of the mass is ~ sum_i w_i 2^-11 |g_i| ~ 1e-6;
    # independent roundings add as a random walk over nodes and steps
    sigma_g = np.sqrt(3 * 1e-4)
    walk = np.sqrt(n * n * 1000) * HALF_ULP * sigma_g
    assert abs(s1[0] - s0[0]) < 10 * walk, (s1[0] - s0[0], walk)
    assert np.all(np.abs(s1[1:] - s0[1:]) < 10 * walk)


@pytest.mark.slow
def test_fp16_equilibrates_every_mode():
    # the Fig. 3 set-up of Sec. V A with FP16 storage: every mode's equilibration ratio,
    # averaged over the wavevectors, within 3 standard errors of 1 (R independent lattices;
    # tests/equilibration.py), every radial bin within the family-wise bound
    import equilibration as eq
    R, nx, ny, nb = 16, 128, 128, 8
    cs2 = 0.265 ** 2
    m = th.Model(1.0, cs2, 0.08, 1e-5, 1.0, 1.0, 1.0)
    lats = []
    for r in range(R):
        L = lbf.Lattice(nx, ny, seed=2012 + 7919 * r, rho0=1.0, cs2=cs2, precision=lbf.LB_FP16DEV)
        L.set_params(1e-5, 0.08, 1.0, 1.0, 1.0, lbf.LB_NOISE_FULL)
        L.step(12000)
        lats.append(L)
    sp = eq.ModeSpectra(R, nx, ny, m)
    for _ in range(200):
        for r, L in enumerate(lats):
            L.step(40)
            lbf.lb_get_populations(L.ctx, sp.f[r], lbf.LB_DEVICE)
        sp.add()
    ratio = sp.mean() / eq.diag_theory(nx, ny, m.G_closed)[None]
    keep = eq.kept_wavevectors(nx, ny)
    bins, _ = eq.radial_bins(nx, ny, nb)
    zfw = eq.family_z(9 * nb)
    for a in range(9):
        mean, se, z = eq.replica_z(ratio[:, a][:, keep].mean(axis=1))
        print("FP16 Fig. 3 mode %d: ratio %.5f +- %.5f (z = %+.2f)" % (a + 1, mean, se, z))
        assert abs(z) <= 3.0, (a, mean, se, z)
        for b in range(nb):
            sel = keep & (bins == b)
            mb, sb, zb = eq.replica_z(ratio[:, a][:, sel].mean(axis=1))
            assert abs(zb) <= zfw, (a, b, mb, sb, zb)
    for L in lats:
        L.close()
