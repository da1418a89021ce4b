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
                                        (100, 36, lbf.LB_NOISE_DIAG)])
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
    # the Fig. 3 set-up of Sec. V A with FP16 storage: every equilibration ratio stays at 1
    cs2 = 0.265 ** 2
    nx = ny = 128
    L = lbf.Lattice(nx, ny, seed=2012, rho0=1.0, cs2=cs2, precision=lbf.LB_FP16DEV)
    L.set_params(1e-5, 0.08, 1.0, 1.0, 1.0, lbf.LB_NOISE_FULL)
    m = th.Model(1.0, cs2, 0.08, 1e-5, 1.0, 1.0, 1.0)
    KX, KY = th.lattice_k(nx, ny)
    L.step(12000)
    acc = np.zeros((9, ny, nx))
    mbar = m.mbar()[:, None, None]
    for _ in range(300):
        L.step(40)
        mm, _ = L.moments()
        acc += np.abs(np.fft.ifft2(mm - mbar, axes=(1, 2)) * nx) ** 2
    acc /= 300
    G = np.array([[np.diag(m.G_closed(KX[j, i], KY[j, i])) for i in range(nx)] for j in range(ny)]).transpose(2, 0, 1)
    keep = np.ones((ny, nx), bool)
    keep[0, 0] = keep[0, nx // 2] = keep[ny // 2, 0] = False
    for a in range(9):
        r = (acc[a] / G[a])[keep].mean()
        assert abs(r - 1) < 0.03, (a, r)
