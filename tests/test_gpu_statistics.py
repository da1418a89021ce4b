"""Statistics of the GPU path against the paper's theory (Sec. V A): equilibration ratios
<|dm_a(k)|^2> / G_aa(k) of every mode (Figs. 3 and 4) and the device-accumulated spectra
against Eqs. (struct-fact) and (momtm-fluct)."""
import numpy as np
import pytest

import oracle
import paper_1009_0254_gb300 as lbf
from oracle import theory as th

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0254_gb300 import build
    build.build()
    lbf.load()


def _ratios(L, model, burn, samples, every, G_of_k):
    nx, ny = L.nx, L.ny
    KX, KY = th.lattice_k(nx, ny)
    L.step(burn)
    acc = np.zeros((9, ny, nx))
    mbar = model.mbar()[:, None, None]
    for _ in range(samples):
        L.step(every)
        m, _ = L.moments()
        dm = m - mbar
        acc += np.abs(np.fft.ifft2(dm, axes=(1, 2)) * np.sqrt(nx * ny)) ** 2
    acc /= samples
    G = np.empty((9, ny, nx))
    for j in range(ny):
        for i in range(nx):
            G[:, j, i] = np.diag(G_of_k(KX[j, i], KY[j, i])).real
    keep = np.ones((ny, nx), bool)
    keep[0, 0] = keep[0, nx // 2] = keep[ny // 2, 0] = False
    return acc / G, keep, KX, KY


def _radial(ratio, keep, KX, KY, nb=8):
    kw = np.sqrt(np.minimum(KX, 2 * np.pi - KX) ** 2 + np.minimum(KY, 2 * np.pi - KY) ** 2)
    edges = np.linspace(0, kw.max() + 1e-9, nb + 1)
    out = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = keep & (kw >= lo) & (kw < hi)
        out.append(ratio[sel].mean() if sel.any() else 1.0)
    return np.array(out)


@pytest.mark.slow
def test_correlated_noise_equilibrates_every_mode_fig3():
    # Fig. 3 set-up: 128^2, kappa = 0.08, c_s = 0.265, tau = 1, T = 1e-7, 400 snapshots
    cs2 = 0.265 ** 2
    L = lbf.Lattice(128, 128, seed=2010, rho0=1.0, cs2=cs2)
    L.set_params(1e-7, 0.08, 1.0, 1.0, 1.0, lbf.LB_NOISE_FULL)
    m = th.Model(1.0, cs2, 0.08, 1e-7, 1.0, 1.0, 1.0)
    ratio, keep, KX, KY = _ratios(L, m, burn=12000, samples=400, every=40, G_of_k=m.G_closed)
    for a in range(9):
        mean = ratio[a][keep].mean()
        assert abs(mean - 1) < 0.03, (a, mean)
        rad = _radial(ratio[a], keep, KX, KY)
        assert np.all(np.abs(rad[1:] - 1) < 0.1), (a, rad)


@pytest.mark.slow
def test_uncorrelated_noise_fig4_setup():
    # Fig. 4 set-up: kappa = 0.03, c_s = 0.15, tau = 1, long-wavelength noise.
    # (1) Every mode follows the exact stationary theory of this noise: the solution of
    #     G = M G M^H + A(-k) Xi(0) A(-k)^H (stationarity of Eq. lb-lang-ft).
    # (2) In the hydrodynamic range k <~ 0.8 the errors against G(k) of Eq. (g-mat-yeo)
    #     are negligible (Sec. V A).  At larger k that theory itself puts the density
    #     ratio up to ~1.2 (along the diagonal), above the paper's "< 10 %" for this figure;
    #     the test records the measured value without asserting the paper's bound.
    cs2 = 0.15 ** 2
    nx = ny = 64
    L = lbf.Lattice(nx, ny, seed=2011, rho0=1.0, cs2=cs2)
    L.set_params(1e-7, 0.03, 1.0, 1.0, 1.0, lbf.LB_NOISE_LW)
    m = th.Model(1.0, cs2, 0.03, 1e-7, 1.0, 1.0, 1.0)
    ratio, keep, KX, KY = _ratios(L, m, burn=8000, samples=400, every=40, G_of_k=m.G_closed)
    X0 = m.Xi_zero()
    Glw = np.empty((9, ny, nx))
    Gc = np.empty((9, ny, nx))
    for j in range(ny):
        for i in range(nx):
            kx, ky = KX[j, i], KY[j, i]
            Gc[:, j, i] = np.diag(m.G_closed(kx, ky))
            Glw[:, j, i] = Gc[:, j, i] if not keep[j, i] else np.diag(th.lyapunov_G(m, kx, ky, X0)).real
    r2 = ratio * Gc / Glw
    for a in range(9):
        assert abs(r2[a][keep].mean() - 1) < 0.03, (a, r2[a][keep].mean())
        rad = _radial(r2[a], keep, KX, KY)
        assert np.all(np.abs(rad[1:] - 1) < 0.1), (a, rad)
    kw = np.sqrt(np.minimum(KX, 2 * np.pi - KX) ** 2 + np.minimum(KY, 2 * np.pi - KY) ** 2)
    hydro = keep & (kw <= 0.8)
    for a in range(9):
        assert abs(ratio[a][hydro].mean() - 1) < 0.05, (a, ratio[a][hydro].mean())
    print("Fig. 4 set-up: density ratio vs G(k) in the outermost radial bin = %.3f"
          % _radial(ratio[0], keep, KX, KY)[-1])


@pytest.mark.slow
def test_device_structure_factor_against_ornstein_zernike():
    # Eq. (struct-fact) with the lattice k^2 (Appendix B) and Eq. (momtm-fluct)
    nx = ny = 128
    nb = 16
    kT, kappa = 1e-6, 0.05
    L = lbf.Lattice(nx, ny, seed=77)
    L.set_params(kT, kappa, 1.0, 1.0, 1.0, lbf.LB_NOISE_FULL)
    L.step(12000)
    L.set_sampling(20, nb)
    L.step(8000)
    S, Jl, Jt, cnt, ns = L.structure_factor()
    assert ns == 400
    m = th.Model(1.0, 1 / 3, kappa, kT, 1.0, 1.0, 1.0)
    b, KXw, KYw, _ = oracle.k_bins(nx, ny, nb)
    Sth = m.S_k(KXw, KYw)
    keep = b >= 0
    keep[0, nx // 2] = keep[ny // 2, 0] = False
    for k in range(1, nb):
        sel = keep & (b == k)
        if sel.sum() < 50:
            continue
        th_mean = Sth[sel].mean()
        assert abs(S[k] / th_mean - 1) < 0.08, (k, S[k], th_mean)
        assert abs(Jl[k] / kT - 1) < 0.08, (k, Jl[k])
        assert abs(Jt[k] / kT - 1) < 0.08, (k, Jt[k])
