"""Precision study: FP32 and FP16-deviation storage (arithmetic FP32 either way) against
the FP64 oracle and the linear theory, correlated (full FDT) noise, kappa = 0.02.

* 256 x 256, kT in {1e-5, 1e-4}: the GPU and the oracle step the same trajectory (same
  seed, same noise); compared are the mass drift, the spatial variance of every moment
  (three snapshots) and the accumulated S(k), j_l, j_t spectra (every 10 steps).
* 2048 x 2048, 5000 steps, kT in {1e-5, 1e-4}: S(k) accumulated on the device against the
  Ornstein-Zernike S(k) of Eq. (struct-fact) on bins that equilibrate within the burn-in.

Each test prints its table (pytest -s)."""
import numpy as np
import pytest

import oracle
import paper_1009_0254_gb300 as lbf
from oracle import theory as th

pytestmark = pytest.mark.gpu

PREC = {"fp32": lbf.LB_FP32, "fp16": lbf.LB_FP16DEV}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0254_gb300 import build
    build.build()
    lbf.load()


def _moment_var(m, mbar):
    d = m - mbar[:, None, None]
    return (d * d).mean(axis=(1, 2))


@pytest.mark.parametrize("kT", [1e-5, 1e-4])
def test_storage_precision_against_fp64_oracle_256(kT):
    n, steps, every, nb, seed = 256, 300, 10, 48, 99
    params = (kT, 0.02, 1.0, 1.0, 1.0)
    model = th.Model(1.0, 1 / 3, 0.02, kT, 1.0, 1.0, 1.0)
    mbar = model.mbar()
    snaps = (100, 200, 300)

    # FP64 oracle
    o = oracle.Lattice(n, n, seed=seed)
    o.set_params(*params, lbf.LB_NOISE_FULL)
    mass0 = o.f.sum()
    acc = np.zeros((3, nb))
    var_o = []
    for t in range(1, steps + 1):
        o.step(1)
        if t % every == 0:
            S, L, T, cnt = oracle.spectra_sample(o.f, 1.0, nb)
            acc += np.array([S, L, T])
        if t in snaps:
            var_o.append(_moment_var(o.moments(), mbar))
    nsamp = steps // every
    den = np.where(cnt > 0, cnt * nsamp, 1)
    spec_o = acc / den
    var_o = np.mean(var_o, axis=0)
    drift_o = abs(o.f.sum() - mass0) / mass0

    rows = []
    for name, prec in PREC.items():
        g = lbf.Lattice(n, n, seed=seed, precision=prec)
        g.set_params(*params, lbf.LB_NOISE_FULL)
        g.set_sampling(every, nb)
        s0 = g.sums()
        var_g = []
        t = 0
        for ts in snaps:
            g.step(ts - t)
            t = ts
            m, _ = g.moments()
            var_g.append(_moment_var(m, mbar))
        var_g = np.mean(var_g, axis=0)
        Sg, Lg, Tg, cg, ns = g.structure_factor()
        assert ns == nsamp
        np.testing.assert_array_equal(cg, cnt)
        drift = abs(g.sums()[0] - s0[0]) / s0[0]
        var_err = np.abs(var_g - var_o) / var_o
        sel = cnt > 0
        spec_err = [np.abs(x[sel] - y[sel]).max() / y[sel].mean() for x, y in zip([Sg, Lg, Tg], spec_o)]
        rows.append((name, drift, var_err.max(), spec_err))
        g.close()

    print("\n256^2 FULL kT=%g, %d steps; FP64 oracle mass drift %.2e" % (kT, steps, drift_o))
    print("storage | mass drift | max moment-variance rel err | S(k) err | j_l err | j_t err")
    for name, drift, ve, se in rows:
        print("%s | %.2e | %.2e | %.2e | %.2e | %.2e" % (name, drift, ve, se[0], se[1], se[2]))
    fp32, fp16 = rows
    assert fp32[1] < 1e-9 and fp32[2] < 1e-4 and max(fp32[3]) < 1e-4
    assert fp16[1] < 1e-6 and fp16[2] < 0.05 and max(fp16[3]) < 0.05


@pytest.mark.parametrize("kT", [1e-5, 1e-4])
def test_storage_precision_against_theory_2048(kT):
    n, nb, burn, steps, every = 2048, 64, 2000, 3000, 100
    params = (kT, 0.02, 1.0, 1.0, 1.0)
    model = th.Model(1.0, 1 / 3, 0.02, kT, 1.0, 1.0, 1.0)
    b, KX, KY, kmag = oracle.k_bins(n, n, nb)
    sel = b >= 0
    cnt = np.bincount(b[sel], minlength=nb)
    S_th = np.bincount(b[sel], weights=model.S_k(KX, KY)[sel], minlength=nb) / np.maximum(cnt, 1)
    kc = (np.arange(nb) + 0.5) * np.pi * np.sqrt(2) / nb
    ok = (kc > 0.3) & (kc < np.pi) & (cnt > 1000)   # equilibrated within the burn-in, full bins
    rows = {}
    for name, prec in PREC.items():
        g = lbf.Lattice(n, n, seed=7, precision=prec)
        g.set_params(*params, lbf.LB_NOISE_FULL)
        s0 = g.sums()
        g.step(burn)
        g.set_sampling(every, nb)
        g.step(steps)
        S, _, _, c, ns = g.structure_factor()
        drift = abs(g.sums()[0] - s0[0]) / s0[0]
        rel = S[ok] / S_th[ok] - 1
        rows[name] = (drift, np.abs(rel).max(), rel.mean(), S)
        g.close()
    dS = np.abs(rows["fp16"][3][ok] - rows["fp32"][3][ok]) / rows["fp32"][3][ok]
    print("\n2048^2 FULL kT=%g, kappa=0.02, %d + %d steps, %d S(k) bins with |k| in (0.3, pi)" % (kT, burn, steps,
                                                                                               ok.sum()))
    print("storage | mass drift | max |S/S_theory - 1| | mean (S/S_theory - 1)")
    for name, (drift, mx, mean, _) in rows.items():
        print("%s | %.2e | %.2e | %+.2e" % (name, drift, mx, mean))
    print("fp16 vs fp32 S(k): max rel diff %.2e" % dS.max())
    for name, (drift, mx, mean, _) in rows.items():
        assert mx < 0.05, (name, mx)
        assert abs(mean) < 0.01, (name, mean)
    assert rows["fp32"][0] < 1e-9
    assert rows["fp16"][0] < 1e-5
