"""The C ABI without a GPU: the library loads, exports every entry point declared in
include/lbfluct.h and include/lbfluct3d.h, and its host-side FP64 theory agrees with the
oracle."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_1009_0254_gb300 as lbf
from oracle import theory as th

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1009_0254_gb300 import build
    build.build()
    return lbf.load()


def _declared():
    names = []
    for h in ("lbfluct.h", "lbfluct3d.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(lb3?_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "lb_create" in names and "lb_step" in names and "lb_structure_factor" in names
    assert "lb3_create" in names and "lb3_step" in names and "lb3_noise_matrix" in names
    for n in names:
        assert hasattr(lib, n), n


def test_workspace_size(lib):
    assert lbf.lb_workspace_bytes(1, 8) == 0
    assert lbf.lb_workspace_bytes(64, 64, 7) == 0
    b = lbf.lb_workspace_bytes(64, 64)
    assert b >= 2 * 9 * 64 * 64 * 4 + 2 * 64 * 64 * 8
    h = lbf.lb_workspace_bytes(64, 64, lbf.LB_FP16DEV)
    assert 2 * 9 * 64 * 64 * 2 + 2 * 64 * 64 * 8 <= h < b


@pytest.mark.parametrize("pars", [
    dict(rho0=1.0, cs2=1 / 3, kT=1e-4, kappa=0.01, tau_s=1.0, tau_b=1.0, tau_ghost=1.0),
    dict(rho0=1.0, cs2=1 / 3, kT=1e-4, kappa=0.05, tau_s=0.8, tau_b=1.0, tau_ghost=1.0),
    dict(rho0=0.8, cs2=0.265 ** 2, kT=1e-7, kappa=0.08, tau_s=1.0, tau_b=1.2, tau_ghost=0.9),
])
def test_library_noise_matrix_matches_oracle(lib, pars):
    m = th.Model(pars["rho0"], pars["cs2"], pars["kappa"], pars["kT"], pars["tau_s"], pars["tau_b"], pars["tau_ghost"])
    for kx, ky in [(0.0, 0.0), (np.pi, np.pi), (0.7, -2.1), (np.pi, 0.3)]:
        X = lbf.lb_noise_matrix(pars["rho0"], pars["cs2"], pars["kT"], pars["kappa"], pars["tau_s"],
                                pars["tau_b"], pars["tau_ghost"], kx, ky)
        np.testing.assert_allclose(X, m.Xi_closed(kx, ky), atol=1e-14 * np.abs(X).max())


def test_parameter_validation(lib):
    ok = dict(nx=64, ny=64, rho0=1.0, cs2=1 / 3, kT=1e-4, kappa=0.01, tau_s=0.8, tau_b=1.0, tau_ghost=1.0,
              noise_mode=lbf.LB_NOISE_FULL)
    assert lbf.lb_check_params(**ok) == lbf.LB_OK
    for bad in [dict(tau_s=0.5), dict(tau_b=0.4), dict(tau_ghost=0.5), dict(kT=-1.0), dict(kappa=-0.1),
                dict(noise_mode=7), dict(nx=1)]:
        assert lbf.lb_check_params(**{**ok, **bad}) == lbf.LB_EINVAL, bad
    # Sec. III C / Fig. 5: at cs2 = 1/3, tau = 1 the (4,9) block of Xi(k) is singular at
    # k = (pi, pi) for kappa = 0.05 and indefinite beyond
    edge = {**ok, "tau_s": 1.0, "kappa": 0.05}
    assert lbf.lb_check_params(**edge) == lbf.LB_OK
    assert lbf.lb_check_params(**{**edge, "kappa": 0.06}) == lbf.LB_ENOTPSD
    # an odd lattice does not contain (pi, pi): kappa slightly above 0.05 may still pass there
    assert th.min_eig_block49(th.Model(kappa=0.06, kT=1.0), np.pi, np.pi) < 0
    # the long-wavelength mode uses Xi(0) only
    assert lbf.lb_check_params(**{**edge, "kappa": 0.06, "noise_mode": lbf.LB_NOISE_LW}) == lbf.LB_OK
    # noise off needs no PSD check
    assert lbf.lb_check_params(**{**edge, "kappa": 0.5, "noise_mode": lbf.LB_NOISE_OFF}) == lbf.LB_OK


def test_psd_check_agrees_with_oracle_over_a_parameter_grid(lib):
    # recompute the allowed region of Fig. 5 (tau = 1) on a 32^2 lattice both ways
    nx = ny = 32
    KX, KY = th.lattice_k(nx, ny)
    for cs in [0.05, 0.15, 0.25, 0.35, 0.5]:
        for kappa in [0.0, 0.01, 0.03, 0.05, 0.08, 0.15]:
            m = th.Model(1.0, cs * cs, kappa, 1.0, 1.0, 1.0, 1.0)
            e = th.min_eig_block49(m, KX, KY).min()
            d44 = (m.Xi_closed(np.pi, np.pi)[3, 3], m.Xi_closed(0, 0)[3, 3])
            scale = max(abs(v) for v in d44)
            rc = lbf.lb_check_params(nx, ny, 1.0, cs * cs, 1.0, kappa, 1.0, 1.0, 1.0, lbf.LB_NOISE_FULL)
            if e < -1e-9 * scale:
                assert rc == lbf.LB_ENOTPSD, (cs, kappa, e)
            elif e > 1e-9 * scale:
                assert rc == lbf.LB_OK, (cs, kappa, e)


@pytest.mark.parametrize("cs2,tau", [(1 / 3, (1.0, 1.0, 1.0)), (0.2, (0.8, 1.1, 0.9)), (0.12, (1.3, 0.7, 1.05))])
def test_library_d3q19_noise_matrix_matches_oracle(lib, cs2, tau):
    # the library's closed-form Xi(0) against the oracle's FDT construction from the ansatz
    from oracle import d3q19 as d3
    m = d3.Model(rho0=0.9, cs2=cs2, kappa=0.03, kT=3e-5, tau_s=tau[0], tau_b=tau[1], tau_ghost=tau[2])
    X = lbf.lb3_noise_matrix(0.9, cs2, 3e-5, *tau)
    np.testing.assert_allclose(X, m.Xi_zero(), rtol=1e-12, atol=1e-13 * np.abs(X).max())


@pytest.mark.parametrize("cs2,tau", [(1 / 3, (1.0, 1.0, 1.0)), (0.2, (0.8, 1.1, 0.9)), (0.12, (1.3, 0.7, 1.05))])
def test_library_d3q27_noise_matrix_matches_oracle(lib, cs2, tau):
    # the library's rank-one ansatz route against the oracle's T diag(fbar) T^T and Omega
    from oracle import d3q27 as d
    m = d.Model(rho0=0.9, cs2=cs2, kappa=0.03, kT=3e-5, tau_s=tau[0], tau_b=tau[1], tau_ghost=tau[2])
    X = lbf.lb3_noise_matrix(0.9, cs2, 3e-5, *tau, lattice=lbf.LB_D3Q27)
    np.testing.assert_allclose(X, m.Xi_zero(), rtol=1e-12, atol=1e-13 * np.abs(X).max())
    with pytest.raises(lbf.LBError):
        lbf.lb3_noise_matrix(0.9, cs2, 3e-5, *tau, lattice=15)
