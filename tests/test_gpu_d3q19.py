"""The D3Q19 step on the GPU (include/lbfluct3d.h) against the FP64 oracle (oracle/d3q19.py):
element by element on whole lattices (exact tiles, ragged tails, degenerate one-node axes),
with and without the uncorrelated noise of Xi(0), in FP32 (the population bar) and FP64
(to rounding, which resolves the kappa |grad rho|^2 terms at large amplitude); sampled
nodes of one step at the benchmark size; conservation; the ABI's error paths; and
equipartition of the ideal fluctuating gas with replica z-scores."""
import numpy as np
import pytest

import oracle
import paper_1009_0254_gb300 as lbf
from waves3d import wave_state_box
from oracle import d3q19 as d3
from paper_1009_0254_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5        # FP32 storage of deviations: the population bar
TOL64 = 1e-12
S2 = 1.0 / 3.0
PARAMS = (1e-4, 0.04, 0.8, 1.1, 0.9)       # kT, kappa, tau_s, tau_b, tau_ghost


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0254_gb300 import build
    build.build()
    lbf.load()


def _state(nx, ny, nz, m, seed, amp=0.01, clip=None):
    shape = (19, nz, ny, nx)
    if clip is None:
        pert = synth.gaussian_field(shape, seed=seed, scale=amp)
    else:
        pert = synth.clipped_gaussian_field(shape, seed, amp, clip)
    return m.fbar()[:, None, None, None] * (1.0 + pert)


def _pair(nx, ny, nz, mode, precision=lbf.LB_FP32, cs2=0.25, rho0=1.0, seed=7, amp=0.01, clip=None,
          params=PARAMS):
    g = lbf.Lattice3(nx, ny, nz, seed=seed, rho0=rho0, cs2=cs2, precision=precision)
    g.set_params(*params, mode)
    o = d3.Lattice(nx, ny, nz, rho0=rho0, cs2=cs2, seed=seed)
    o.set_params(*params, {lbf.LB_NOISE_OFF: d3.NOISE_OFF, lbf.LB_NOISE_LW: d3.NOISE_LW}[mode])
    f0 = _state(nx, ny, nz, o.model, seed + 100, amp, clip)
    g.set_populations(f0, t=0)
    o.f = f0.copy()
    return g, o


SIZES = [(32, 8, 4), (37, 11, 5), (64, 16, 9), (5, 3, 2), (1, 1, 8), (40, 1, 3), (3, 17, 1)]


# the staged kernel staging by TMA or by copies, with three or two raw slots, and the plain
# kernel (FP64 and the correlated noise take the variants their configuration offers)
KERNELS3 = {"tma3": ("staged", "tma", "3"), "tma2": ("staged", "tma", "2"), "copy3": ("staged", "copy", "3"),
            "copy2": ("staged", "copy", "2"), "plain": ("plain", "copy", "3")}


@pytest.fixture(params=list(KERNELS3))
def kernel3(request, monkeypatch):
    kernel, stage, slots = KERNELS3[request.param]
    monkeypatch.setenv("LBFLUCT3_KERNEL", kernel)
    monkeypatch.setenv("LBFLUCT3_STAGE", stage)
    monkeypatch.setenv("LBFLUCT3_SLOTS", slots)
    return request.param


@pytest.mark.parametrize("nx,ny,nz", SIZES)
@pytest.mark.parametrize("mode", [lbf.LB_NOISE_OFF, lbf.LB_NOISE_LW])
def test_fp32_step_follows_the_oracle(nx, ny, nz, mode, kernel3):
    g, o = _pair(nx, ny, nz, mode)
    g.step(6)
    o.step(6)
    err = np.abs(g.populations() - o.f).max()
    print("D3Q19 FP32 %s %dx%dx%d mode %d: %.2e" % (kernel3, nx, ny, nz, mode, err))
    assert err <= TOL
    if mode == lbf.LB_NOISE_LW:
        q = d3.Lattice(nx, ny, nz, rho0=1.0, cs2=0.25, seed=7)
        q.set_params(*PARAMS, d3.NOISE_OFF)
        q.f = _state(nx, ny, nz, q.model, 107)
        q.step(6)
        assert np.abs(q.f - o.f).max() > 100 * TOL          # the noise acted


@pytest.mark.parametrize("nx,ny,nz", [(32, 8, 4), (37, 11, 5), (6, 5, 7)])
@pytest.mark.parametrize("mode", [lbf.LB_NOISE_OFF, lbf.LB_NOISE_LW])
def test_fp64_step_to_rounding_at_large_amplitude(nx, ny, nz, mode, kernel3):
    # 25 % perturbations (clipped at 3.5 sigma): kappa (grad rho)^2 and rho u u are ~1e-3 per
    # step here, far above the 1e-12 bar, so a dropped or mis-wired term fails
    g, o = _pair(nx, ny, nz, mode, precision=lbf.LB_FP64, amp=0.25, clip=3.5,
                 params=(1e-4, 0.08, 0.8, 1.1, 0.9))
    g.step(4)
    o.step(4)
    err = np.abs(g.populations() - o.f).max()
    print("D3Q19 FP64 %s %dx%dx%d mode %d: %.2e" % (kernel3, nx, ny, nz, mode, err))
    assert err <= TOL64
    # the same run without the kappa terms differs by far more than the bar
    q = d3.Lattice(nx, ny, nz, rho0=1.0, cs2=0.25, seed=7)
    q.set_params(1e-4, 0.0, 0.8, 1.1, 0.9, d3.NOISE_OFF if mode == lbf.LB_NOISE_OFF else d3.NOISE_LW)
    q.f = _state(nx, ny, nz, q.model, 107, 0.25, 3.5)
    q.step(4)
    assert np.abs(q.f - o.f).max() > 1e3 * TOL64


def test_fp32_nonlinear_terms_at_large_amplitude(kernel3):
    # the FP32 kernel on the 25 % state: the bar is the FP32 rounding of the step's terms
    g, o = _pair(37, 11, 5, lbf.LB_NOISE_LW, amp=0.25, clip=3.5, params=(1e-4, 0.08, 0.8, 1.1, 0.9))
    g.step(3)
    o.step(3)
    err = np.abs(g.populations() - o.f).max()
    print("D3Q19 FP32 nonlinear %s: %.2e" % (kernel3, err))
    assert err <= 2e-6


WAVES = np.random.default_rng(12)
KVEC = WAVES.integers(0, 256, size=(19, 3, 3))          # per population: three integer wavevectors
PHASE = WAVES.uniform(0, 2 * np.pi, size=(19, 3))


def _wave_state(fbar, n, z, y, x, amp, xp=np):
    """fbar_i (1 + amp sum_w sin(2 pi k_iw . r / n + phi_iw)) at the given coordinates (numpy
    or torch arrays), periodic on the n^3 box: a state both sides can evaluate anywhere."""
    out = []
    for i in range(19):
        s = 0.0
        for w in range(3):
            kx, ky, kz = (int(v) for v in KVEC[i, w])
            s = s + xp.sin((2 * np.pi / n) * ((kx * x + ky * y + kz * z) % n) + float(PHASE[i, w]))
        out.append(fbar[i] * (1.0 + amp * s))
    return out


def _patch_step(m, n, centre, seed, t, L, amp):
    """Oracle value of one step at node `centre`: a 5x5x5 periodic neighbourhood (the step at
    a node depends on nodes within two lattice units), stepped with the noise of the
    neighbourhood's global node indices."""
    z0, y0, x0 = centre
    zs = (np.arange(z0 - 2, z0 + 3)) % n
    ys = (np.arange(y0 - 2, y0 + 3)) % n
    xs = (np.arange(x0 - 2, x0 + 3)) % n
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    sub = np.array(_wave_state(m.fbar(), n, Z, Y, X, amp))
    nodes = (Z * n + Y) * n + X
    xi = d3.noise_lw_nodes(m, nodes, seed, t, L)
    return d3.step(sub, m, xi)[:, 2, 2, 2]


def test_sampled_nodes_at_the_benchmark_size():
    # 256^3, FP32, uncorrelated noise: the launch configuration the benchmark times; one step
    # from a state of plane waves (built on the device), checked on sampled nodes
    import torch
    n, amp = 256, 0.01
    m = d3.Model(rho0=1.0, cs2=0.25, kappa=PARAMS[1], kT=PARAMS[0], tau_s=PARAMS[2], tau_b=PARAMS[3],
                 tau_ghost=PARAMS[4])
    g = lbf.Lattice3(n, n, n, seed=5, rho0=1.0, cs2=0.25)
    g.set_params(*PARAMS, lbf.LB_NOISE_LW)
    dev = torch.empty((19, n, n, n), dtype=torch.float64, device="cuda")
    r = torch.arange(n, device="cuda", dtype=torch.float64)          # integer-valued coordinates
    Z, Y, X = torch.meshgrid(r, r, r, indexing="ij")
    for i, plane in enumerate(_wave_state(m.fbar(), n, Z, Y, X, amp, xp=torch)):
        dev[i] = plane
    del Z, Y, X
    lbf.lb3_set_populations(g.ctx, dev, lbf.LB_DEVICE, 11)
    g.step(1)
    lbf.lb3_get_populations(g.ctx, dev, lbf.LB_DEVICE)
    torch.cuda.synchronize()
    L = m.noise_factor()
    rng = np.random.default_rng(0)
    picks = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 5), (n - 1, 0, 31), (128, 128, 0), (7, 8, 255)]
    picks += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(20)]
    err = 0.0
    for c in picks:
        got = dev[:, c[0], c[1], c[2]].cpu().numpy()
        err = max(err, np.abs(got - _patch_step(m, n, c, 5, 11, L, amp)).max())
    print("256^3 sampled: %.2e" % err)
    assert err <= TOL
    del dev, g
    torch.cuda.empty_cache()


def test_mass_and_momentum_are_conserved():
    g = lbf.Lattice3(24, 20, 16, seed=3, rho0=1.0, cs2=0.2, precision=lbf.LB_FP64)
    g.set_params(1e-4, 0.03, 0.8, 1.1, 0.9, lbf.LB_NOISE_LW)
    o = d3.Model(rho0=1.0, cs2=0.2)
    g.set_populations(_state(24, 20, 16, o, 9, 0.02), t=0)
    s0 = g.sums()
    g.step(300)
    s1 = g.sums()
    np.testing.assert_allclose(s1, s0, rtol=0, atol=1e-10)


def test_error_paths():
    with pytest.raises(lbf.LBError) as e:
        lbf.Lattice3(8, 8, 8, precision=lbf.LB_FP16DEV)
    assert e.value.code == lbf.LB_EINVAL
    with pytest.raises(lbf.LBError):
        lbf.Lattice3(0, 8, 8)
    g = lbf.Lattice3(8, 8, 8, cs2=0.6)
    with pytest.raises(lbf.LBError) as e:
        g.step(1)
    assert e.value.code == lbf.LB_ESTATE
    with pytest.raises(lbf.LBError) as e:
        g.set_params(1e-4, 0.0, 1.0, 1.0, 1.0, lbf.LB_NOISE_LW)      # cs2 > 5/9: Xi(0) indefinite
    assert e.value.code == lbf.LB_ENOTPSD
    g.set_params(1e-4, 0.0, 1.0, 1.0, 1.0, lbf.LB_NOISE_OFF)
    for bad in [(1e-4, 0.0, 0.5, 1.0, 1.0, 0), (1e-4, -0.1, 1.0, 1.0, 1.0, 0), (1e-4, 0.0, 1.0, 1.0, 1.0, 2)]:
        with pytest.raises(lbf.LBError) as e:
            g.set_params(*bad)
        assert e.value.code == lbf.LB_EINVAL


def test_ideal_fluctuating_gas_is_in_equipartition():
    # cs2 = sigma_s^2, kappa = 0: every mode has <dm_a^2> = N_a rho0 kT / sigma_s^2 per node
    # (the conserved rho and j less the k = 0 share 1/n); independent replicas give the
    # z-scores, held to a Bonferroni family bound over the 19 modes (Student t, R - 1 dof)
    from scipy.stats import t as student
    rho0, kT = 1.0, 1e-4
    nx = ny = nz = 12
    n = nx * ny * nz
    R, samples, every, burn = 32, 60, 25, 200
    mbar = d3.Model(rho0, S2).mbar()[:, None, None, None]
    acc = np.zeros((R, 19))
    for r in range(R):
        g = lbf.Lattice3(nx, ny, nz, seed=1000 + r, rho0=rho0, cs2=S2)
        g.set_params(kT, 0.0, 0.8, 1.1, 0.9, lbf.LB_NOISE_LW)
        g.step(burn)
        for _ in range(samples):
            g.step(every)
            dm = np.einsum("ai,i...->a...", d3.T, g.populations()) - mbar
            acc[r] += (dm.reshape(19, -1) ** 2).mean(axis=1)
        acc[r] /= samples
    want = d3.N * rho0 * kT / S2
    want[:4] *= 1 - 1 / n
    mean = acc.mean(axis=0)
    sd = acc.std(axis=0, ddof=1) / np.sqrt(R)
    z = (mean - want) / sd
    bound = float(student.isf(0.01 / (2 * 19), R - 1))
    print("GPU equipartition ratios", np.round(mean / want, 4), "max |z| %.2f (bound %.2f)" % (np.abs(z).max(), bound))
    assert np.abs(z).max() < bound


# --- correlated noise Xi(k), built in real space (LB_NOISE_FULL_RS) ---------------------------

RS_PARAMS = (1e-4, 0.04, 0.8, 1.1, 0.9)


def _pair_rs(nx, ny, nz, precision=lbf.LB_FP32, amp=0.01, clip=None, params=RS_PARAMS, seed=7):
    g = lbf.Lattice3(nx, ny, nz, seed=seed, cs2=0.2, precision=precision)
    g.set_params(*params, lbf.LB_NOISE_FULL_RS)
    o = d3.Lattice(nx, ny, nz, cs2=0.2, seed=seed)
    o.set_params(*params, d3.NOISE_FULL_RS)
    f0 = _state(nx, ny, nz, o.model, seed + 100, amp, clip)
    g.set_populations(f0, t=0)
    o.f = f0.copy()
    return g, o


@pytest.mark.parametrize("nx,ny,nz", [(32, 8, 4), (37, 11, 5), (64, 16, 9), (5, 3, 2), (1, 1, 8), (40, 1, 3),
                                      (3, 17, 1), (33, 9, 2)])
def test_fp32_correlated_noise_follows_the_oracle(nx, ny, nz, kernel3):
    g, o = _pair_rs(nx, ny, nz)
    g.step(6)
    o.step(6)
    err = np.abs(g.populations() - o.f).max()
    print("D3Q19 FP32 RS %s %dx%dx%d: %.2e" % (kernel3, nx, ny, nz, err))
    assert err <= TOL
    q = d3.Lattice(nx, ny, nz, cs2=0.2, seed=7)
    q.set_params(*RS_PARAMS, d3.NOISE_LW)
    q.f = _state(nx, ny, nz, q.model, 107)
    q.step(6)
    assert np.abs(q.f - o.f).max() > 10 * TOL           # the correlated part acted


@pytest.mark.parametrize("nx,ny,nz", [(32, 8, 4), (37, 11, 5), (6, 5, 7)])
def test_fp64_correlated_noise_to_rounding(nx, ny, nz, kernel3):
    g, o = _pair_rs(nx, ny, nz, precision=lbf.LB_FP64, amp=0.25, clip=3.5, params=(1e-4, 0.04, 0.8, 1.1, 0.9))
    g.step(4)
    o.step(4)
    err = np.abs(g.populations() - o.f).max()
    print("D3Q19 FP64 RS %s %dx%dx%d: %.2e" % (kernel3, nx, ny, nz, err))
    assert err <= TOL64


def test_correlated_noise_refuses_an_indefinite_Xi():
    g = lbf.Lattice3(8, 8, 8, cs2=0.3)
    # c_s^2(k) = 0.3 + 0.06 * 16/3 = 0.62 > 5/9 at s = 16/3
    with pytest.raises(lbf.LBError) as e:
        g.set_params(1e-4, 0.06, 0.8, 1.1, 0.9, lbf.LB_NOISE_FULL_RS)
    assert e.value.code == lbf.LB_ENOTPSD
    g.set_params(1e-4, 0.06, 0.8, 1.1, 0.9, lbf.LB_NOISE_LW)           # Xi(0) alone is fine


def _patch_step_rs(m, n, centre, seed, t, L, Ls, amp):
    """One oracle step at `centre` with the correlated noise: the 6x6x6 neighbourhood from
    centre - 3 .. centre + 2 holds every node the box sums of the 3x3x3 collisions need."""
    z0, y0, x0 = centre
    zs, ys, xs = ((np.arange(c - 3, c + 3)) % n for c in (z0, y0, x0))
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    nodes = (Z * n + Y) * n + X
    sub = np.array(_wave_state(m.fbar(), n, Z, Y, X, amp))
    xi = d3.noise_lw_nodes(m, nodes, seed, t, L)
    g = np.concatenate([oracle.normals(nodes.ravel().astype(np.uint32), seed, t, tg) for tg in d3.TAG_RS], axis=1)
    nu = g.T.reshape(8, 2, 6, 6, 6)
    v = np.einsum("wab,wb...->wa...", Ls, nu)
    xi416 = np.zeros((2, 6, 6, 6))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                h = sum((d3.CORNERS[w][0] ** dx) * (d3.CORNERS[w][1] ** dy) * (d3.CORNERS[w][2] ** dz) * v[w]
                        for w in range(8)) / 8.0
                xi416 += np.roll(h, shift=(dz, dy, dx), axis=(1, 2, 3))     # exact away from the low faces
    xi[4], xi[16] = xi416[0], xi416[1]
    return d3.step(sub, m, xi)[:, 3, 3, 3]


def test_correlated_noise_sampled_at_the_benchmark_size():
    import torch
    n, amp = 256, 0.01
    kT, kappa, ts, tb, tg = RS_PARAMS
    m = d3.Model(1.0, 0.2, kappa, kT, ts, tb, tg)
    g = lbf.Lattice3(n, n, n, seed=5, cs2=0.2)
    g.set_params(*RS_PARAMS, lbf.LB_NOISE_FULL_RS)
    dev = torch.empty((19, n, n, n), dtype=torch.float64, device="cuda")
    r = torch.arange(n, device="cuda", dtype=torch.float64)
    Z, Y, X = torch.meshgrid(r, r, r, indexing="ij")
    for i, plane in enumerate(_wave_state(m.fbar(), n, Z, Y, X, amp, xp=torch)):
        dev[i] = plane
    del Z, Y, X
    lbf.lb3_set_populations(g.ctx, dev, lbf.LB_DEVICE, 9)
    g.step(1)
    lbf.lb3_get_populations(g.ctx, dev, lbf.LB_DEVICE)
    torch.cuda.synchronize()
    L, Ls = m.noise_factor(), d3.rs_factors(m)
    rng = np.random.default_rng(3)
    picks = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 5), (n - 1, 0, 31), (128, 128, 0), (7, 8, n - 1)]
    picks += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(16)]
    err = 0.0
    for c in picks:
        got = dev[:, c[0], c[1], c[2]].cpu().numpy()
        err = max(err, np.abs(got - _patch_step_rs(m, n, c, 5, 9, L, Ls, amp)).max())
    print("RS 256^3 sampled: %.2e" % err)
    assert err <= TOL
    del dev, g
    torch.cuda.empty_cache()


def test_correlated_noise_equilibrates_every_wavevector_on_the_gpu():
    # Sec. V A in three dimensions on the GPU: S(k) = rho0 kT / c_s^2(k) and <|j(k)|^2> = rho0 kT
    # at every k of a 12^3 lattice, binned by s(k), replicas for the standard errors, a
    # Bonferroni bound over the bins (Student t); the staggered-momentum invariants excluded
    from scipy.stats import t as student
    n, R, samples, every, burn = 12, 16, 40, 20, 300
    cs2, kappa, kT = 0.2, 0.04, 1e-4
    k1 = 2 * np.pi * np.fft.fftfreq(n)
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    s = d3.lattice_s(KX, KY, KZ)
    edges = np.linspace(0, 16 / 3 + 1e-9, 9)
    b = np.digitize(s, edges) - 1
    keep = np.ones((n, n, n), bool)
    keep[0, 0, 0] = False
    keepj = keep.copy()
    keepj[0, 0, n // 2] = keepj[0, n // 2, 0] = keepj[n // 2, 0, 0] = False
    S_th = kT / (cs2 + kappa * s)
    accS = np.zeros((R, 8))
    accJ = np.zeros((R, 8))
    for r in range(R):
        g = lbf.Lattice3(n, n, n, seed=500 + r, cs2=cs2)
        g.set_params(kT, kappa, 0.8, 1.1, 0.9, lbf.LB_NOISE_FULL_RS)
        g.step(burn)
        S = np.zeros((n, n, n))
        J = np.zeros((n, n, n))
        for _ in range(samples):
            g.step(every)
            m = np.einsum("ai,i...->a...", d3.T, g.populations())
            S += np.abs(np.fft.fftn(m[0] - 1.0)) ** 2 / n ** 3
            J += sum(np.abs(np.fft.fftn(m[a])) ** 2 for a in (1, 2, 3)) / (3 * n ** 3)
        for q in range(8):
            accS[r, q] = (S / samples / S_th)[keep & (b == q)].mean()
            accJ[r, q] = (J / samples / kT)[keepj & (b == q)].mean()
    bound = float(student.isf(0.01 / (2 * 16), R - 1))
    for name, acc in (("S", accS), ("J", accJ)):
        mean = acc.mean(axis=0)
        se = acc.std(axis=0, ddof=1) / np.sqrt(R)
        z = (mean - 1) / se
        print("RS GPU %s ratios by s bin" % name, np.round(mean, 4), "max |z| %.2f (bound %.2f)" % (np.abs(z).max(), bound))
        assert np.abs(z).max() < bound


def test_lattice_with_64_bit_plane_offsets_sampled():
    # 1024 x 1024 x 216 nodes: 19 planes hold more than 2^32 elements, so the step takes its
    # 64-bit offsets; one step from a plane-wave state checked on sampled nodes, several in the
    # last planes (offsets above 2^32)
    import torch
    nx, ny, nz, amp = 1024, 1024, 216, 0.01
    assert 19 * nx * ny * nz >= 2 ** 32
    m = d3.Model(1.0, 0.25, PARAMS[1], PARAMS[0], PARAMS[2], PARAMS[3], PARAMS[4])
    g = lbf.Lattice3(nx, ny, nz, seed=5, cs2=0.25)
    g.set_params(*PARAMS, lbf.LB_NOISE_LW)
    dev = torch.empty((19, nz, ny, nx), dtype=torch.float64, device="cuda")
    for z0 in range(0, nz, 24):
        zz = torch.arange(z0, min(z0 + 24, nz), device="cuda", dtype=torch.float64)
        yy = torch.arange(ny, device="cuda", dtype=torch.float64)
        xx = torch.arange(nx, device="cuda", dtype=torch.float64)
        Z, Y, X = torch.meshgrid(zz, yy, xx, indexing="ij")
        for i, plane in enumerate(wave_state_box(m.fbar(), (nx, ny, nz), Z, Y, X, amp, xp=torch)):
            dev[i, z0:z0 + Z.shape[0]] = plane
        del Z, Y, X
    lbf.lb3_set_populations(g.ctx, dev, lbf.LB_DEVICE, 2)
    g.step(1)
    lbf.lb3_get_populations(g.ctx, dev, lbf.LB_DEVICE)
    torch.cuda.synchronize()
    L = m.noise_factor()
    rng = np.random.default_rng(5)
    picks = [(nz - 1, ny - 1, nx - 1), (nz - 1, 0, 0), (nz - 2, 517, 1023), (0, 0, 0), (108, 512, 511)]
    picks += [(int(rng.integers(nz - 20, nz)), int(rng.integers(0, ny)), int(rng.integers(0, nx))) for _ in range(8)]
    err = 0.0
    for c in picks:
        zc, yc, xc = c
        zs, ys, xs = (np.arange(c0 - 2, c0 + 3) % nn for c0, nn in ((zc, nz), (yc, ny), (xc, nx)))
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        sub = np.array(wave_state_box(m.fbar(), (nx, ny, nz), Z, Y, X, amp))
        nodes = (Z * ny + Y) * nx + X
        want = d3.step(sub, m, d3.noise_lw_nodes(m, nodes, 5, 2, L))[:, 2, 2, 2]
        err = max(err, np.abs(dev[:, zc, yc, xc].cpu().numpy() - want).max())
    print("1024x1024x216 sampled: %.2e" % err)
    assert err <= TOL
    del dev, g
    torch.cuda.empty_cache()
