"""The request server (lb_server_*) on the GPU: served results against the FP64 oracle,
each result the same alone and in a mix of concurrent requests, admission within the HBM
budget, latency bookkeeping and request validation."""
import threading

import numpy as np
import pytest

import oracle
import paper_1009_0254_gb300 as lbf

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


def _oracle_run(nx, ny, steps, seed, kT, kappa, tau_s, tau_b, tau_g, mode, rho0=1.0, cs2=1 / 3):
    o = oracle.Lattice(nx, ny, rho0=rho0, cs2=cs2, seed=seed)
    o.set_params(kT, kappa, tau_s, tau_b, tau_g, mode)
    o.step(steps)
    return o


@pytest.mark.parametrize("nx,ny,mode", [(32, 32, lbf.LB_NOISE_LW), (70, 12, lbf.LB_NOISE_DIAG),
                                        (2, 2, lbf.LB_NOISE_LW), (64, 48, lbf.LB_NOISE_LW)])
def test_served_result_matches_oracle(nx, ny, mode):
    srv = lbf.Server(1 << 30, max_active=16, max_chunk_steps=37)
    p = dict(kT=1.5e-4, kappa=0.02, tau_s=0.8, tau_b=1.1, tau_ghost=0.9, noise_mode=mode, seed=77)
    i = srv.submit(nx, ny, 100, keep_state=True, **p)
    res = srv.wait(i, timeout_s=60)
    assert res.status == lbf.LB_OK and res.steps == 100
    f = srv.fetch(i, nx, ny)
    o = _oracle_run(nx, ny, 100, 77, 1.5e-4, 0.02, 0.8, 1.1, 0.9, mode)
    assert np.abs(f - o.f).max() <= TOL
    # the reported FP64 sums are those of the final state
    np.testing.assert_allclose(res.sums, o.moments()[:3].sum(axis=(1, 2)), rtol=0, atol=1e-6 * nx * ny)
    srv.close()


@pytest.mark.parametrize("nx,ny", [(32, 32), (64, 16), (8, 128), (256, 8)])
def test_served_correlated_noise_matches_oracle(nx, ny):
    # Sec. IV, Eq. (noise-yeo): k-space noise of modes 4 and 9 per served request
    srv = lbf.Server(1 << 30, max_active=16, max_chunk_steps=29)
    p = dict(kT=1.5e-4, kappa=0.03, tau_s=0.8, tau_b=1.1, tau_ghost=0.9, noise_mode=lbf.LB_NOISE_FULL, seed=31)
    i = srv.submit(nx, ny, 70, keep_state=True, **p)
    res = srv.wait(i, timeout_s=60)
    assert res.status == lbf.LB_OK
    f = srv.fetch(i, nx, ny)
    o = _oracle_run(nx, ny, 70, 31, 1.5e-4, 0.03, 0.8, 1.1, 0.9, lbf.LB_NOISE_FULL)
    assert np.abs(f - o.f).max() <= TOL
    srv.close()


def test_served_correlated_result_same_alone_and_in_the_mix():
    X = dict(nx=64, ny=32, steps=180, kT=1e-4, kappa=0.02, tau_s=0.9, seed=2024, noise_mode=lbf.LB_NOISE_FULL)
    alone = lbf.Server(1 << 30, max_active=8, max_chunk_steps=50)
    ia = alone.submit(keep_state=True, **X)
    alone.wait(ia, timeout_s=60)
    fa = alone.fetch(ia, 64, 32)
    alone.close()

    rng = np.random.default_rng(8)
    mix = lbf.Server(1 << 30, max_active=64, max_chunk_steps=17)
    reqs = _random_requests(rng, 30)
    for k, r in enumerate(reqs):
        if k % 2 == 0:
            r["noise_mode"] = lbf.LB_NOISE_FULL     # same and other sizes share noise launches
    for r in reqs[:15]:
        mix.submit(**r)
    ix = mix.submit(keep_state=True, **X)
    for r in reqs[15:]:
        mix.submit(**r)
    mix.wait(0, timeout_s=120)
    assert all(r.status == lbf.LB_OK for r in mix.poll())
    fm = mix.fetch(ix, 64, 32)
    assert np.array_equal(fa, fm)
    mix.close()

    # and the batched engine steps the same correlated trajectory
    ens = lbf.Ensemble([(64, 32)], [2024])
    ens.set_params(0, 1e-4, 0.02, 0.9, 1.0, 1.0, lbf.LB_NOISE_FULL)
    ens.step(180)
    assert np.abs(ens.populations(0) - fa).max() <= 1e-6


def test_nonideal_request_matches_oracle():
    srv = lbf.Server(1 << 30, max_active=4, max_chunk_steps=50)
    i = srv.submit(32, 32, 80, kT=1e-5, kappa=0.08, tau_s=1.0, tau_b=1.1, tau_ghost=0.9, seed=9, rho0=0.9,
                   cs2=0.265 ** 2, keep_state=True)
    srv.wait(i, timeout_s=60)
    f = srv.fetch(i, 32, 32)
    o = _oracle_run(32, 32, 80, 9, 1e-5, 0.08, 1.0, 1.1, 0.9, lbf.LB_NOISE_LW, rho0=0.9, cs2=0.265 ** 2)
    assert np.abs(f - o.f).max() <= TOL
    srv.close()


def _random_requests(rng, n):
    out = []
    for _ in range(n):
        L = int(rng.choice([16, 32, 64, 128]))
        out.append(dict(nx=L, ny=int(rng.choice([L, L // 2])), steps=int(rng.integers(20, 400)),
                        kT=float(rng.uniform(5e-5, 2e-4)), kappa=float(rng.uniform(0.005, 0.05)),
                        tau_s=float(rng.uniform(0.6, 1.5)), seed=int(rng.integers(1, 2 ** 62))))
    return out


def test_result_same_alone_and_in_the_mix():
    X = dict(nx=64, ny=64, steps=250, kT=1e-4, kappa=0.01, tau_s=0.8, seed=12345)
    alone = lbf.Server(1 << 30, max_active=8, max_chunk_steps=64)
    ia = alone.submit(keep_state=True, **X)
    alone.wait(ia, timeout_s=60)
    fa = alone.fetch(ia, 64, 64)
    alone.close()

    rng = np.random.default_rng(4)
    mix = lbf.Server(1 << 30, max_active=64, max_chunk_steps=23)
    ids = []
    reqs = _random_requests(rng, 40)
    for r in reqs[:20]:
        ids.append(mix.submit(**r))
    ix = mix.submit(keep_state=True, **X)               # arrives while others run
    for r in reqs[20:]:
        ids.append(mix.submit(**r))
    mix.wait(0, timeout_s=120)
    fm = mix.fetch(ix, 64, 64)
    assert np.array_equal(fa, fm)
    assert mix.stats().completed == 41
    mix.close()


def test_served_equals_batched_replica():
    # the served kernel and the batched ensemble kernel step the same trajectory (up to the
    # FP32 rounding order of two compilations of the same arithmetic)
    X = dict(kT=1e-4, kappa=0.01, tau_s=0.8, tau_b=1.0, tau_ghost=1.0)
    srv = lbf.Server(1 << 30, max_active=4, max_chunk_steps=50)
    i = srv.submit(64, 32, 120, seed=5, keep_state=True, **X)
    srv.wait(i, timeout_s=60)
    fs = srv.fetch(i, 64, 32)
    srv.close()
    ens = lbf.Ensemble([(64, 32)], [5])
    ens.set_params(0, X["kT"], X["kappa"], X["tau_s"], X["tau_b"], X["tau_ghost"], lbf.LB_NOISE_LW)
    ens.step(120)
    assert np.abs(ens.populations(0) - fs).max() <= 1e-6


def test_admission_stays_within_budget_and_everything_completes():
    b128 = lbf.lb_server_request_bytes(128, 128)
    budget = 3 * b128 + b128 // 2                      # three 128^2 lattices at a time
    srv = lbf.Server(budget, max_active=64, max_chunk_steps=40)
    ids = [srv.submit(128, 128, 150, seed=s) for s in range(1, 11)]
    ids += [srv.submit(32, 32, 60, seed=100 + s) for s in range(6)]   # small ones backfill
    srv.wait(0, timeout_s=120)
    st = srv.stats()
    assert st.completed == len(ids)
    assert st.bytes_peak <= budget
    assert st.bytes_in_use == 0
    res = {r.id: r for r in srv.poll()}
    assert set(res) == set(ids)
    for r in res.values():
        assert r.status == lbf.LB_OK
        assert r.t_submit <= r.t_admit <= r.t_complete
        n = r.nx * r.ny
        assert abs(r.sums[0] - n) <= 1e-4 * n          # mass of a lattice at rho0 = 1
        assert abs(r.sums[1]) <= 1e-4 * n and abs(r.sums[2]) <= 1e-4 * n
    assert st.node_updates == pytest.approx(10 * 150 * 128 * 128 + 6 * 60 * 32 * 32)
    srv.close()


def test_concurrent_submitters():
    srv = lbf.Server(1 << 31, max_active=128, max_chunk_steps=50)
    got, errs = [], []

    def client(k):
        try:
            rng = np.random.default_rng(100 + k)
            for r in _random_requests(rng, 15):
                got.append(srv.submit(**r))
        except Exception as e:      # pragma: no cover - reported below
            errs.append(e)

    th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs
    srv.wait(0, timeout_s=120)
    assert len(set(got)) == 60
    assert srv.stats().completed == 60
    srv.close()


def test_submit_validation():
    srv = lbf.Server(lbf.lb_server_request_bytes(64, 64), max_active=4)
    with pytest.raises(lbf.LBError) as e:
        srv.submit(48, 32, 10, noise_mode=lbf.LB_NOISE_FULL)     # 48 is not a power of two
    assert e.value.code == lbf.LB_EINVAL
    assert lbf.lb_server_request_bytes(64, 64, lbf.LB_NOISE_FULL) == \
        lbf.lb_server_request_bytes(64, 64) + 64 * 64 * 8
    with pytest.raises(lbf.LBError) as e:
        srv.submit(64, 64, 10, noise_mode=lbf.LB_NOISE_FULL)     # its noise field exceeds the budget
    assert e.value.code == lbf.LB_ENOMEM
    with pytest.raises(lbf.LBError) as e:
        srv.submit(32, 32, 10, tau_s=0.5)
    assert e.value.code == lbf.LB_EINVAL
    with pytest.raises(lbf.LBError) as e:
        srv.submit(32, 32, 0)
    assert e.value.code == lbf.LB_EINVAL
    with pytest.raises(lbf.LBError) as e:
        srv.submit(128, 128, 10)                   # alone larger than the budget
    assert e.value.code == lbf.LB_ENOMEM
    with pytest.raises(lbf.LBError):
        srv.fetch(12345, 4, 4)
    i = srv.submit(16, 16, 5)
    srv.wait(i, timeout_s=30)
    with pytest.raises(lbf.LBError):               # not kept
        srv.fetch(i, 16, 16)
    srv.close()


def test_cancel_queued_and_running_requests():
    b = lbf.lb_server_request_bytes(256, 256)
    srv = lbf.Server(b + b // 2, max_active=8, max_chunk_steps=20)     # one 256^2 at a time
    long_id = srv.submit(256, 256, 200000, seed=1)                     # runs for seconds
    queued = srv.submit(256, 256, 50, seed=2)                          # waits for the budget
    srv.cancel(queued)
    import time
    time.sleep(0.2)
    srv.cancel(long_id)
    r_long = srv.wait(long_id, timeout_s=30)
    r_q = srv.wait(queued, timeout_s=30)
    assert r_q.status == lbf.LB_ECANCELED and r_long.status == lbf.LB_ECANCELED
    after = srv.submit(64, 64, 30, seed=3)
    r = srv.wait(after, timeout_s=30)
    assert r.status == lbf.LB_OK
    st = srv.stats()
    assert st.bytes_in_use == 0 and st.completed == 3
    with pytest.raises(lbf.LBError):
        srv.cancel(after)                                              # already completed
    srv.close()


def test_injected_allocation_failures_leave_the_server_running():
    srv = lbf.Server(1 << 30, max_active=16, max_chunk_steps=50)
    lbf.lb_server_inject_alloc_failures(srv.srv, 2)
    ids = [srv.submit(32, 32, 40, seed=s) for s in range(1, 6)]
    srv.wait(0, timeout_s=60)
    res = {r.id: r for r in srv.poll()}
    status = [res[i].status for i in ids]
    assert status.count(lbf.LB_ENOMEM) == 2 and status.count(lbf.LB_OK) == 3
    assert srv.stats().bytes_in_use == 0
    srv.close()


def test_diverged_run_is_reported_not_finite():
    # tests/nonlinear_case.py DIVERGING: a request whose FP64 oracle run overflows
    # (test_oracle_step.py::test_the_diverging_request_of_the_watchdog_test_diverges)
    # completes with exactly LB_ENONFINITE, and the server goes on serving
    import nonlinear_case as nl
    d = nl.DIVERGING
    srv = lbf.Server(1 << 30, max_active=4, max_chunk_steps=64)
    i = srv.submit(d["n"], d["n"], d["steps"], kT=0.0, kappa=d["kappa"], tau_s=d["tau"], tau_b=d["tau"],
                   tau_ghost=d["tau"], noise_mode=lbf.LB_NOISE_OFF, seed=3, init=nl.diverging_state())
    r = srv.wait(i, timeout_s=60)
    assert r.status == lbf.LB_ENONFINITE
    assert not np.all(np.isfinite(r.sums))
    j = srv.submit(32, 32, 50, kT=1e-4, kappa=0.01, tau_s=0.8, seed=4)
    assert srv.wait(j, timeout_s=60).status == lbf.LB_OK
    srv.close()


def test_non_finite_initial_state_is_reported_not_finite():
    f = np.broadcast_to(np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None], (9, 8, 8)).copy()
    f[3, 2, 5] = np.nan
    srv = lbf.Server(1 << 30, max_active=4, max_chunk_steps=10)
    i = srv.submit(8, 8, 5, kT=1e-4, kappa=0.01, tau_s=0.8, seed=4, init=f)
    k = srv.submit(8, 8, 5, kT=1e-4, kappa=0.01, tau_s=0.8, seed=4)
    assert srv.wait(i, timeout_s=60).status == lbf.LB_ENONFINITE
    assert srv.wait(k, timeout_s=60).status == lbf.LB_OK
    srv.close()


def test_device_wait_gives_up_and_context_survives():
    rc, gave_up = lbf.lb_selftest_bounded_wait(0.05)
    assert rc == lbf.LB_ETIMEOUT and gave_up == 1
    L = lbf.Lattice(16, 16, seed=1)
    L.set_params(1e-4, 0.01, 1.0, 1.0, 1.0, lbf.LB_NOISE_LW)
    L.step(5)
    assert L.t == 5 and np.all(np.isfinite(L.populations()))


@pytest.mark.parametrize("nx,ny", [(32, 32), (33, 17), (100, 36)])
def test_served_real_space_correlated_noise_matches_oracle(nx, ny):
    srv = lbf.Server(1 << 30, max_active=16, max_chunk_steps=29)
    p = dict(kT=1.5e-4, kappa=0.03, tau_s=0.8, tau_b=1.1, tau_ghost=0.9, noise_mode=lbf.LB_NOISE_FULL_RS, seed=33)
    i = srv.submit(nx, ny, 70, keep_state=True, **p)
    res = srv.wait(i, timeout_s=60)
    assert res.status == lbf.LB_OK
    f = srv.fetch(i, nx, ny)
    o = _oracle_run(nx, ny, 70, 33, 1.5e-4, 0.03, 0.8, 1.1, 0.9, lbf.LB_NOISE_FULL_RS)
    assert np.abs(f - o.f).max() <= TOL
    with pytest.raises(lbf.LBError):
        srv.submit(nx, ny, 10, noise_mode=lbf.LB_NOISE_LW_LOCAL)
    srv.close()


def test_served_real_space_correlated_result_same_alone_and_in_the_mix():
    X = dict(nx=60, ny=36, steps=150, kT=1e-4, kappa=0.02, tau_s=0.9, seed=77, noise_mode=lbf.LB_NOISE_FULL_RS)
    alone = lbf.Server(1 << 30, max_active=8, max_chunk_steps=50)
    ia = alone.submit(keep_state=True, **X)
    alone.wait(ia, timeout_s=60)
    fa = alone.fetch(ia, 60, 36)
    alone.close()
    rng = np.random.default_rng(9)
    mix = lbf.Server(1 << 30, max_active=64, max_chunk_steps=17)
    reqs = _random_requests(rng, 24)
    for k, r in enumerate(reqs):
        r["noise_mode"] = [lbf.LB_NOISE_FULL_RS, lbf.LB_NOISE_LW, lbf.LB_NOISE_FULL][k % 3]
    for r in reqs[:12]:
        mix.submit(**r)
    ix = mix.submit(keep_state=True, **X)
    for r in reqs[12:]:
        mix.submit(**r)
    mix.wait(0, timeout_s=120)
    assert all(r.status == lbf.LB_OK for r in mix.poll())
    assert np.array_equal(fa, mix.fetch(ix, 60, 36))
    mix.close()


def test_admission_limit_on_large_requests():
    # lb_server_set_admission: two large lattices are not admitted together (the second waits
    # until the first has issued its last step), small ones pass; results are unchanged
    def run(limit):
        srv = lbf.Server(1 << 31, max_active=16, max_chunk_steps=25)
        if limit:
            lbf.lb_server_set_admission(srv.srv, 256 * 256, 1)
        big1 = srv.submit(256, 256, 300, seed=1, keep_state=True)
        big2 = srv.submit(256, 256, 300, seed=2, keep_state=True)
        small = srv.submit(32, 32, 300, seed=3, keep_state=True)
        r = [srv.wait(i, timeout_s=120) for i in (big1, big2, small)]
        f = [srv.fetch(i, n, n) for i, n in ((big1, 256), (big2, 256), (small, 32))]
        srv.close()
        return r, f
    r0, f0 = run(False)
    r1, f1 = run(True)
    for a, b in zip(f0, f1):
        assert np.array_equal(a, b)
    assert all(x.status == lbf.LB_OK for x in r1)
    # with the limit the second large lattice is admitted only after the first ran; the small
    # one ran alongside the first
    assert r1[1].t_admit >= r1[0].t_admit + 0.5 * (r1[0].t_complete - r1[0].t_admit)
    assert r1[2].t_admit <= r1[0].t_complete
    srv = lbf.Server(1 << 20)
    with pytest.raises(lbf.LBError) as e:
        lbf.lb_server_set_admission(srv.srv, 0, 1)
    assert e.value.code == lbf.LB_EINVAL
    srv.close()
