"""Batched ensembles (lb_batch_*) on the GPU: every replica against the FP64 oracle, a
replica's trajectory independent of the batch it is stepped in, graph replay identical
to eager stepping, and per-replica spectra against the oracle."""
import numpy as np
import pytest

import oracle
import paper_1009_0254_gb300 as lbf
from oracle import theory as th
from paper_1009_0254_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0254_gb300 import build
    build.build()
    lbf.load()


# mixed sizes (powers of two, ragged, tiny), seeds, parameters and noise modes
MIX = [
    ((32, 32), 11, (1.0e-4, 0.01, 1.0, 1.0, 1.0), lbf.LB_NOISE_LW),
    ((64, 64), 12, (2.0e-4, 0.02, 0.8, 1.0, 1.0), lbf.LB_NOISE_LW),
    ((33, 17), 13, (5.0e-5, 0.00, 1.2, 0.9, 1.1), lbf.LB_NOISE_DIAG),
    ((32, 32), 14, (1.5e-4, 0.05, 0.7, 1.3, 1.0), lbf.LB_NOISE_LW),
    ((2, 2), 15, (1.0e-4, 0.01, 1.0, 1.0, 1.0), lbf.LB_NOISE_LW),
    ((100, 36), 16, (1.0e-4, 0.01, 1.0, 1.0, 1.0), lbf.LB_NOISE_OFF),
    ((64, 64), 17, (8.0e-5, 0.01, 0.9, 1.0, 0.8), lbf.LB_NOISE_LW),
    ((130, 9), 18, (1.0e-4, 0.03, 1.0, 1.0, 1.0), lbf.LB_NOISE_DIAG),
]


def _initial(nx, ny, params, rho0=1.0, cs2=1 / 3, seed=0):
    m = th.Model(rho0, cs2, params[1], params[0], params[2], params[3], params[4])
    pert = synth.gaussian_field((9, ny, nx), seed=2000 + seed, scale=0.01)
    return m.fbar()[:, None, None] * (1.0 + pert)


def _ensemble(entries, t0=0):
    ens = lbf.Ensemble([e[0] for e in entries], [e[1] for e in entries])
    for r, (size, seed, params, mode) in enumerate(entries):
        ens.set_params(r, *params, mode)
        ens.set_populations(r, _initial(*size, params, seed=seed), t=t0 + r)
    return ens


def test_every_replica_matches_oracle():
    ens = _ensemble(MIX)
    ens.step(13)                      # eager
    ens.step(47, graph_steps=10)      # 4 graph replays + 7 eager
    for r, (size, seed, params, mode) in enumerate(MIX):
        o = oracle.Lattice(*size, seed=seed)
        o.set_params(*params, mode)
        o.f = _initial(*size, params, seed=seed)
        o.t = r
        o.step(60)
        assert ens.t(r) == 60 + r
        err = np.abs(ens.populations(r) - o.f).max()
        assert err <= TOL, (r, size, err)
        if mode != lbf.LB_NOISE_OFF:
            assert np.abs(o.f - o.model.fbar()[:, None, None]).max() > 100 * TOL


def test_replica_alone_equals_replica_in_mix():
    mixed = _ensemble(MIX)
    mixed.step(40)
    for r in [0, 2, 4, 6]:
        alone = lbf.Ensemble([MIX[r][0]], [MIX[r][1]])
        alone.set_params(0, *MIX[r][2], MIX[r][3])
        alone.set_populations(0, _initial(*MIX[r][0], MIX[r][2], seed=MIX[r][1]), t=r)
        alone.step(40)
        assert np.array_equal(alone.populations(0), mixed.populations(r)), r


def test_replica_matches_single_lattice_path():
    # the batched kernel and the single-lattice kernel agree up to FP32 rounding order
    size, seed, params, mode = MIX[1]
    ens = _ensemble([MIX[1]])
    L = lbf.Lattice(*size, seed=seed)
    L.set_params(*params, mode)
    L.set_populations(_initial(*size, params, seed=seed), t=0)
    ens.step(50)
    L.step(50)
    assert np.abs(ens.populations(0) - L.populations()).max() <= 1e-6


def test_graph_replay_equals_eager_with_odd_graph_length():
    entries = [MIX[0], MIX[1], MIX[6]]
    a, b = _ensemble(entries), _ensemble(entries)
    for e in (a, b):
        e.set_sampling(7, 16)
    a.step(77)
    b.step(77, graph_steps=21)        # 3 replays of an odd-length graph + leftovers
    for r in range(len(entries)):
        assert np.array_equal(a.populations(r), b.populations(r)), r
        assert a.t(r) == b.t(r)
        sa, sb = a.structure_factor(r), b.structure_factor(r)
        assert sa[4] == sb[4] == 11
        for x, y in zip(sa[:3], sb[:3]):
            np.testing.assert_allclose(x, y, rtol=1e-12, atol=0)


def test_replica_spectra_match_oracle():
    entries = [MIX[0], ((64, 32), 31, (1e-4, 0.02, 0.8, 1.0, 1.0), lbf.LB_NOISE_LW), MIX[3]]
    nb = 16
    ens = _ensemble(entries)
    ens.set_sampling(1, nb)
    ens.step(3)
    for r, (size, seed, params, mode) in enumerate(entries):
        o = oracle.Lattice(*size, seed=seed)
        o.set_params(*params, mode)
        o.f = _initial(*size, params, seed=seed)
        o.t = r
        acc = np.zeros((3, nb))
        for _ in range(3):
            o.step(1)
            S, L, T, cnt = oracle.spectra_sample(o.f, o.model.rho0, nb)
            acc += np.array([S, L, T])
        Sg, Lg, Tg, cg, ns = ens.structure_factor(r)
        assert ns == 3
        np.testing.assert_array_equal(cg, cnt)
        den = np.where(cnt > 0, cnt * 3, 1)
        for got, ref in zip([Sg, Lg, Tg], acc / den):
            np.testing.assert_allclose(got, ref, rtol=1e-4, atol=1e-12)


def test_mass_and_momentum_conserved_per_replica():
    ens = _ensemble(MIX)
    s0 = [ens.sums(r) for r in range(len(MIX))]
    ens.step(100, graph_steps=25)
    for r, (size, *_rest) in enumerate(MIX):
        n = size[0] * size[1]
        s1 = ens.sums(r)
        np.testing.assert_allclose(s1, s0[r], rtol=0, atol=100 * 30 * 1e-7 * np.sqrt(n) + 1e-9)


def test_autotune_resets_to_rest_and_keeps_results():
    entries = [MIX[0], MIX[1], MIX[0][:1] + (21,) + MIX[0][2:]]
    ens = lbf.Ensemble([e[0] for e in entries], [e[1] for e in entries])
    for r, (_s, _seed, params, mode) in enumerate(entries):
        ens.set_params(r, *params, mode)
    ens.autotune(3)
    for r, (size, seed, params, mode) in enumerate(entries):
        assert ens.t(r) == 0
        m = th.Model(1.0, 1 / 3, params[1], params[0], params[2], params[3], params[4])
        np.testing.assert_allclose(ens.populations(r), np.broadcast_to(m.fbar()[:, None, None], (9,) + size[::-1]),
                                   rtol=0, atol=1e-7)
    ens.step(30, graph_steps=10)
    for r, (size, seed, params, mode) in enumerate(entries):
        o = oracle.Lattice(*size, seed=seed)
        o.set_params(*params, mode)
        o.step(30)
        assert np.abs(ens.populations(r) - o.f).max() <= TOL, r


def test_batch_api_errors():
    ens = lbf.Ensemble([(16, 16), (24, 8)], [1, 2])
    with pytest.raises(lbf.LBError) as e:
        ens.step(1)
    assert e.value.code == lbf.LB_ESTATE
    with pytest.raises(lbf.LBError) as e:
        ens.set_params(1, 1e-4, 0.01, 1.0, 1.0, 1.0, lbf.LB_NOISE_FULL)    # 24 x 8: not powers of two
    assert e.value.code == lbf.LB_EINVAL
    with pytest.raises(lbf.LBError) as e:
        ens.set_params(0, 1e-4, 0.01, 0.5, 1.0, 1.0, lbf.LB_NOISE_LW)
    assert e.value.code == lbf.LB_EINVAL
    with pytest.raises(lbf.LBError) as e:
        ens.set_params(2, 1e-4, 0.01, 1.0, 1.0, 1.0, lbf.LB_NOISE_LW)
    assert e.value.code == lbf.LB_EINVAL
    ens.set_params(-1, 1e-4, 0.01, 1.0, 1.0, 1.0, lbf.LB_NOISE_LW)
    with pytest.raises(lbf.LBError) as e:
        ens.set_sampling(10, 8)            # 24 is not a power of two
    assert e.value.code == lbf.LB_EINVAL
    with pytest.raises(lbf.LBError) as e:
        lbf.lb_batch_step_graph(ens.b, 10, 0)
    assert e.value.code == lbf.LB_EINVAL
    ens.step(5)
    assert ens.t(0) == 5 and ens.t(1) == 5
    assert lbf.lb_batch_launch_count(ens.b) == 5      # one persistent launch per step for both classes
    with pytest.raises(lbf.LBError):
        lbf.Ensemble([(1, 16)], [1])


FULL_MIX = [
    ((32, 32), 41, (1.0e-4, 0.01, 1.0, 1.0, 1.0), lbf.LB_NOISE_FULL),
    ((64, 32), 42, (2.0e-4, 0.03, 0.8, 1.1, 0.9), lbf.LB_NOISE_FULL),
    ((32, 32), 43, (1.5e-4, 0.02, 0.7, 1.0, 1.2), lbf.LB_NOISE_LW),
    ((16, 64), 44, (1.0e-4, 0.05, 1.0, 1.0, 1.0), lbf.LB_NOISE_FULL),
    ((33, 17), 45, (1.0e-4, 0.01, 1.0, 1.0, 1.0), lbf.LB_NOISE_DIAG),
    ((32, 32), 46, (8.0e-5, 0.04, 0.9, 1.0, 1.0), lbf.LB_NOISE_FULL),
]


def test_correlated_noise_replicas_match_oracle():
    ens = _ensemble(FULL_MIX)
    ens.step(11)
    ens.step(39, graph_steps=13)
    for r, (size, seed, params, mode) in enumerate(FULL_MIX):
        o = oracle.Lattice(*size, seed=seed)
        o.set_params(*params, mode)
        o.f = _initial(*size, params, seed=seed)
        o.t = r
        o.step(50)
        err = np.abs(ens.populations(r) - o.f).max()
        assert err <= TOL, (r, size, mode, err)


def test_correlated_replica_alone_equals_in_mix_and_single_path():
    mixed = _ensemble(FULL_MIX)
    mixed.step(30, graph_steps=10)
    size, seed, params, mode = FULL_MIX[1]
    alone = _ensemble([FULL_MIX[1]], t0=1)
    alone.step(30, graph_steps=10)
    assert np.array_equal(alone.populations(0), mixed.populations(1))
    L = lbf.Lattice(*size, seed=seed)
    L.set_params(*params, mode)
    L.set_populations(_initial(*size, params, seed=seed), t=1)
    L.step(30)
    assert np.abs(L.populations() - mixed.populations(1)).max() <= 1e-6


RS_MIX = [
    ((32, 32), 51, (1.0e-4, 0.01, 1.0, 1.0, 1.0), lbf.LB_NOISE_FULL_RS),
    ((33, 17), 52, (2.0e-4, 0.03, 0.8, 1.1, 0.9), lbf.LB_NOISE_FULL_RS),
    ((32, 32), 53, (1.5e-4, 0.02, 0.7, 1.0, 1.2), lbf.LB_NOISE_LW),
    ((100, 36), 54, (1.0e-4, 0.04, 1.0, 1.0, 1.0), lbf.LB_NOISE_FULL_RS),
    ((2, 2), 55, (1.0e-4, 0.01, 1.0, 1.0, 1.0), lbf.LB_NOISE_FULL_RS),
    ((64, 32), 56, (8.0e-5, 0.04, 0.9, 1.0, 1.0), lbf.LB_NOISE_FULL),
]


@pytest.mark.parametrize("tile", [0, 5, 6, 2])
def test_real_space_correlated_replicas_match_oracle(tile, monkeypatch):
    # correlated noise built in real space (LB_NOISE_FULL_RS) in a mix with the other modes,
    # lattices of any size; several tile shapes of the batched kernel
    monkeypatch.setenv("LBFLUCT_BATCH_TILE", str(tile))
    ens = _ensemble(RS_MIX)
    ens.step(11)
    ens.step(39, graph_steps=13)
    for r, (size, seed, params, mode) in enumerate(RS_MIX):
        o = oracle.Lattice(*size, seed=seed)
        o.set_params(*params, mode)
        o.f = _initial(*size, params, seed=seed)
        o.t = r
        o.step(50)
        err = np.abs(ens.populations(r) - o.f).max()
        assert err <= TOL, (r, size, mode, err)


def test_real_space_correlated_replica_alone_equals_in_mix_and_single_path():
    mixed = _ensemble(RS_MIX)
    mixed.step(30, graph_steps=10)
    size, seed, params, mode = RS_MIX[3]
    alone = _ensemble([RS_MIX[3]], t0=3)
    alone.step(30, graph_steps=10)
    assert np.array_equal(alone.populations(0), mixed.populations(3))
    L = lbf.Lattice(*size, seed=seed)
    L.set_params(*params, mode)
    L.set_populations(_initial(*size, params, seed=seed), t=3)
    L.step(30)
    assert np.abs(L.populations() - mixed.populations(3)).max() <= 1e-6
    # switching the mode off and on rebuilds the launches (lean step kernel without it)
    for r in range(len(RS_MIX)):
        mixed.set_params(r, *RS_MIX[r][2], lbf.LB_NOISE_LW)
    mixed.step(5, graph_steps=5)
    mixed.set_params(3, *params, mode)
    mixed.step(5, graph_steps=5)
    with pytest.raises(lbf.LBError) as e:
        mixed.set_params(0, *RS_MIX[0][2], lbf.LB_NOISE_LW_LOCAL)
    assert e.value.code == lbf.LB_EINVAL
