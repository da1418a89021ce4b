"""Nonlinear parity: every step kernel against the FP64 oracle on a large-amplitude
deterministic state (tests/nonlinear_case.py) at a tolerance on the scale of FP32
rounding, 2e-6 max|f|.  At that state the second-order terms of the Table II equilibrium
(rho u u, kappa grad rho grad rho, -3 kappa |grad rho|^2, kappa drho lap rho) and a swap
of two diagonal density neighbours each move f* by 100x the tolerance or more
(test_oracle_step.py::test_nonlinear_parity_state_resolves_the_second_order_terms), so a
kernel whose density ring, gradient or equilibrium is wrong fails here even where the
1e-5 population bar of the fluctuating tests would not see it.

Covered: the TMA kernel in each of its five tile shapes, the plain and sweep kernels, the
4096^2 roofline size on sampled nodes, FP16 storage (to one FP16 unit in the last place
against the oracle rounded the same way), the batched engine in each of its seven tile
shapes and the served engine."""
import numpy as np
import pytest

import nonlinear_case as nl
import oracle
import paper_1009_0254_gb300 as lbf
from oracle import theory as th
from paper_1009_0254_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [(64, 64), (100, 36), (33, 17), (130, 9)]
# (tile_x, tile_y, threads) of the batched kernel's shapes 0..6, in the library's order
BATCH_TILES = [(32, 16, 256), (32, 16, 128), (32, 8, 256), (32, 8, 128), (64, 8, 256), (64, 16, 512), (32, 32, 512)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0254_gb300 import build
    build.build()
    lbf.load()


def _oracle(case, f0, steps):
    rho0, cs2, p = nl.CASES[case]
    nx, ny = f0.shape[2], f0.shape[1]
    o = oracle.Lattice(nx, ny, rho0=rho0, cs2=cs2, seed=1)
    o.set_params(*p, oracle.NOISE_OFF)
    o.f = f0.copy()
    o.step(steps)
    return o.f


KERNELS = [("tma", t) for t in range(5)] + [("simple", None), ("sweep", None), ("sweep6", None)]


@pytest.mark.parametrize("kernel,tile", KERNELS)
@pytest.mark.parametrize("case", ["ideal", "nonideal"])
def test_single_lattice_kernels_resolve_the_nonlinear_terms(kernel, tile, case, monkeypatch):
    monkeypatch.setenv("LBFLUCT_STEP_KERNEL", kernel)
    if tile is None:
        monkeypatch.delenv("LBFLUCT_TMA_TILE", raising=False)
    else:
        monkeypatch.setenv("LBFLUCT_TMA_TILE", str(tile))
    rho0, cs2, p = nl.CASES[case]
    for k, (nx, ny) in enumerate(SIZES):
        f0 = nl.state(case, nx, ny, seed=300 + k)
        g = lbf.Lattice(nx, ny, seed=1, rho0=rho0, cs2=cs2)
        g.set_params(*p, lbf.LB_NOISE_OFF)
        g.set_populations(f0, t=0)
        g.step(nl.STEPS)
        err = np.abs(g.populations() - _oracle(case, f0, nl.STEPS)).max()
        tol = nl.tolerance(f0)
        print("%s/%s %s %dx%d: max |f - f_oracle| = %.2e (tolerance %.2e)" % (kernel, tile, case, nx, ny, err, tol))
        assert err <= tol, (nx, ny, err, tol)
        g.close()


@pytest.mark.parametrize("kernel", ["tma", "simple", "sweep"])
def test_roofline_size_sampled_nonlinear_parity(kernel, monkeypatch):
    # 4096^2 (the benchmark's lattice), one step, compared on sampled nodes
    monkeypatch.setenv("LBFLUCT_STEP_KERNEL", kernel)
    monkeypatch.delenv("LBFLUCT_TMA_TILE", raising=False)
    nx = ny = 4096
    case = "ideal"
    rho0, cs2, p = nl.CASES[case]
    m = nl.model(case)
    f0 = nl.state(case, nx, ny, seed=7)
    nodes = synth.sample_nodes(nx, ny, 3000, seed=8)
    g = lbf.Lattice(nx, ny, seed=1, rho0=rho0, cs2=cs2)
    g.set_params(*p, lbf.LB_NOISE_OFF)
    g.set_populations(f0, t=0)
    g.step(1)
    fg = g.populations().reshape(9, -1)[:, nodes].T
    fo = oracle.step_sampled(f0, m, oracle.NOISE_OFF, 1, 0, nodes)
    err = np.abs(fg - fo).max()
    tol = nl.tolerance(f0)
    print("%s 4096^2 sampled: %.2e (tolerance %.2e)" % (kernel, err, tol))
    assert err <= tol, (err, tol)
    g.close()


def _fp16_code(f, fbar):
    """Stored FP16 words of populations f (g_i = (f_i - fbar_i) / w_i, rounded to nearest)."""
    g = (f - fbar[:, None, None]) / th.W[:, None, None]
    return g.astype(np.float16)


# FP32 arithmetic error of the collision in g units (intermediates of size up to ~1 at this
# state, a few dozen operations): below one FP16 unit in the last place for words of order
# one, above it for words near zero, where an FP16 unit is as small as 6e-8
G_ARITH = 4e-6


@pytest.mark.parametrize("kernel", ["tma", "simple", "sweep", "sweep6"])
@pytest.mark.parametrize("case", ["ideal", "nonideal"])
def test_fp16_storage_resolves_the_nonlinear_terms(kernel, case, monkeypatch):
    # FP16 storage keeps g_i = (f_i - fbar_i)/w_i in FP16.  Start from a state whose g_i are
    # FP16 numbers (stored exactly), take one step, and compare the stored words with the
    # oracle's result rounded to FP16 the same way: they may differ only where the FP32
    # arithmetic lands within its own rounding error (G_ARITH) of an FP16 rounding boundary,
    # i.e. by at most one unit in the last place plus G_ARITH, and rarely; a dropped
    # second-order term moves g by 1e-3 or more (over 250 x G_ARITH).
    monkeypatch.setenv("LBFLUCT_STEP_KERNEL", kernel)
    monkeypatch.delenv("LBFLUCT_TMA_TILE", raising=False)
    rho0, cs2, p = nl.CASES[case]
    m = nl.model(case)
    fbar = m.fbar()
    for k, (nx, ny) in enumerate(SIZES[:3]):
        f = nl.state(case, nx, ny, seed=500 + k)
        h = _fp16_code(f, fbar)
        f0 = fbar[:, None, None] + th.W[:, None, None] * h.astype(np.float64)
        g = lbf.Lattice(nx, ny, seed=1, rho0=rho0, cs2=cs2, precision=lbf.LB_FP16DEV)
        g.set_params(*p, lbf.LB_NOISE_OFF)
        g.set_populations(f0, t=0)
        assert np.array_equal(_fp16_code(g.populations(), fbar), h)      # stored exactly
        g.step(1)
        got = _fp16_code(g.populations(), fbar).astype(np.float64)
        want16 = _fp16_code(_oracle(case, f0, 1), fbar)
        want = want16.astype(np.float64)
        ulp = np.spacing(np.abs(want16)).astype(np.float64)
        d = np.abs(got - want)
        print("fp16 %s %s %dx%d: words that differ %d of %d, largest difference %.2e (%.1f units of the word)"
              % (kernel, case, nx, ny, (d > 0).sum(), d.size, d.max(), (d / ulp).max()))
        assert np.all(d <= ulp + G_ARITH), (d - ulp).max()
        assert (d == 0).mean() >= 0.99
        g.close()


@pytest.mark.parametrize("tile", range(7))
@pytest.mark.parametrize("case", ["ideal", "nonideal"])
def test_batched_engine_resolves_the_nonlinear_terms(tile, case, monkeypatch):
    monkeypatch.setenv("LBFLUCT_BATCH_TILE", str(tile))
    rho0, cs2, p = nl.CASES[case]
    sizes = SIZES + [(2, 2), (64, 64)]
    states = [nl.state(case, nx, ny, seed=700 + k) for k, (nx, ny) in enumerate(sizes)]
    ens = lbf.Ensemble(sizes, [1 + k for k in range(len(sizes))], rho0=rho0, cs2=cs2)
    assert tuple(lbf.lb_batch_tuning(ens.b)[:3]) == BATCH_TILES[tile]
    for r, f0 in enumerate(states):
        ens.set_params(r, *p, lbf.LB_NOISE_OFF)
        ens.set_populations(r, f0, t=0)
    ens.step(1)
    ens.step(nl.STEPS - 1, graph_steps=1)
    for r, f0 in enumerate(states):
        err = np.abs(ens.populations(r) - _oracle(case, f0, nl.STEPS)).max()
        assert err <= nl.tolerance(f0), (r, sizes[r], err)
    ens.close()


@pytest.mark.parametrize("case", ["ideal", "nonideal"])
def test_served_engine_resolves_the_nonlinear_terms(case):
    rho0, cs2, p = nl.CASES[case]
    kT, kappa, tau_s, tau_b, tau_g = p
    srv = lbf.Server(1 << 30, max_active=16, max_chunk_steps=2)     # the steps span chunks
    sizes = SIZES + [(2, 2)]
    ids, states = [], []
    for k, (nx, ny) in enumerate(sizes):
        f0 = nl.state(case, nx, ny, seed=900 + k)
        states.append(f0)
        ids.append(srv.submit(nx, ny, nl.STEPS, kT=kT, kappa=kappa, tau_s=tau_s, tau_b=tau_b, tau_ghost=tau_g,
                              noise_mode=lbf.LB_NOISE_OFF, seed=3, rho0=rho0, cs2=cs2, keep_state=True, init=f0))
    for i, (nx, ny), f0 in zip(ids, sizes, states):
        res = srv.wait(i, timeout_s=60)
        assert res.status == lbf.LB_OK
        f = srv.fetch(i, nx, ny)
        err = np.abs(f - _oracle(case, f0, nl.STEPS)).max()
        assert err <= nl.tolerance(f0), ((nx, ny), err)
    srv.close()
