"""Python binding of liblbfluct.so, the GB300 fluctuating lattice Boltzmann library.

Argument marshalling only: every step runs in the library's CUDA kernels.  The
functions below carry the names of the C ABI (include/lbfluct.h) and raise
``LBError`` on a negative return code.  ``Lattice`` is a small convenience wrapper
that lets PyTorch own the device workspace and supply the stream.

There is no fallback: if the shared library is missing or cannot be loaded, every
call raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbfluct.so")

LB_OK, LB_EINVAL, LB_ENOTPSD, LB_ENOMEM, LB_ECUDA, LB_ETIMEOUT, LB_ESTATE = 0, -1, -2, -3, -4, -5, -6
LB_ENONFINITE, LB_ECANCELED = -7, -8
LB_FP32, LB_FP16DEV, LB_FP64 = 0, 1, 2
LB_NOISE_OFF, LB_NOISE_LW, LB_NOISE_FULL, LB_NOISE_DIAG, LB_NOISE_FULL_RS, LB_NOISE_LW_LOCAL = 0, 1, 2, 3, 4, 5
LB_EOS_LINEAR, LB_EOS_DOUBLE_WELL = 0, 1
LB_FACTOR_CHOLESKY, LB_FACTOR_EIGEN = 0, 1
LB_HOST, LB_DEVICE = 0, 1
LB_WARN_LOW_MACH = 1
LB_D3Q19, LB_D3Q27 = 19, 27

_lib = None


class lb_request(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("steps", ctypes.c_int64),
                ("rho0", ctypes.c_double), ("cs2", ctypes.c_double), ("kT", ctypes.c_double),
                ("kappa", ctypes.c_double), ("tau_s", ctypes.c_double), ("tau_b", ctypes.c_double),
                ("tau_ghost", ctypes.c_double), ("noise_mode", ctypes.c_int), ("keep_state", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("init", ctypes.POINTER(ctypes.c_double))]


class lb_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("state_kept", ctypes.c_int), ("steps", ctypes.c_int64), ("sums", ctypes.c_double * 3),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_complete", ctypes.c_double)]


class lb_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("steps_issued", ctypes.c_int64), ("bytes_in_use", ctypes.c_size_t),
                ("bytes_peak", ctypes.c_size_t), ("bytes_budget", ctypes.c_size_t),
                ("node_updates", ctypes.c_double), ("gpu_busy_s", ctypes.c_double),
                ("t_first_admit", ctypes.c_double), ("t_last_complete", ctypes.c_double)]


class LBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("lbfluct error %d: %s" % (code, msg))
        self.code = code


def load(path: str = LIB_PATH):
    """Load liblbfluct.so (built by paper_1009_0254_gb300/build.py) and declare its ABI."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("liblbfluct.so not found at %s: build it first (python -c 'import "
                           "__graft_entry__ as g; g.build()')" % path)
    L = ctypes.CDLL(path)
    vp, dp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
    c_int, c_i64, c_u64, c_dbl, c_sz = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t
    proto = {
        "lb_workspace_bytes": (c_sz, [c_int, c_int, c_int]),
        "lb_create": (c_int, [c_int, c_int, c_int, c_u64, c_dbl, c_dbl, vp, c_sz, ctypes.POINTER(vp)]),
        "lb_destroy": (c_int, [vp]),
        "lb_set_stream": (c_int, [vp, vp]),
        "lb_set_params": (c_int, [vp, c_dbl, c_dbl, c_dbl, c_dbl, c_dbl, c_int]),
        "lb_step": (c_int, [vp, c_i64]),
        "lb_set_noise_factor": (c_int, [vp, c_int]),
        "lb_set_eos": (c_int, [vp, c_int, c_dbl, c_dbl, c_dbl]),
        "lb_get_time": (c_int, [vp, i64p]),
        "lb_set_populations": (c_int, [vp, vp, c_int, c_i64]),
        "lb_get_populations": (c_int, [vp, vp, c_int]),
        "lb_moments": (c_int, [vp, vp, c_int, dp]),
        "lb_set_sampling": (c_int, [vp, c_int, c_int]),
        "lb_structure_factor": (c_int, [vp, c_int, dp, dp, dp, i64p, i64p]),
        "lb_warnings": (c_int, [vp]),
        "lb_last_error": (ctypes.c_char_p, [vp]),
        "lb_synchronize": (c_int, [vp]),
        "lb_set_kernel_timing": (c_int, [vp, c_int]),
        "lb_kernel_time": (c_int, [vp, dp, i64p]),
        "lb_launch_count": (c_int, [vp, i64p]),
        "lb_noise_matrix": (c_int, [c_dbl] * 9 + [dp]),
        "lb_check_params": (c_int, [c_int, c_int] + [c_dbl] * 7 + [c_int]),
        "lb_conserved_sums_static": (c_int, [vp, c_int, c_int, vp, vp]),
        "lb_batch_workspace_bytes": (c_sz, [c_int, vp, vp]),
        "lb_batch_create": (c_int, [c_int, vp, vp, vp, c_dbl, c_dbl, vp, c_sz, ctypes.POINTER(vp)]),
        "lb_batch_destroy": (c_int, [vp]),
        "lb_batch_set_stream": (c_int, [vp, vp]),
        "lb_batch_set_params": (c_int, [vp, c_int, c_dbl, c_dbl, c_dbl, c_dbl, c_dbl, c_int]),
        "lb_batch_autotune": (c_int, [vp, c_int]),
        "lb_batch_step": (c_int, [vp, c_i64]),
        "lb_batch_step_graph": (c_int, [vp, c_i64, c_i64]),
        "lb_batch_get_time": (c_int, [vp, c_int, i64p]),
        "lb_batch_set_populations": (c_int, [vp, c_int, vp, c_int, c_i64]),
        "lb_batch_get_populations": (c_int, [vp, c_int, vp, c_int]),
        "lb_batch_sums": (c_int, [vp, c_int, dp]),
        "lb_batch_set_sampling": (c_int, [vp, c_int, c_int]),
        "lb_batch_structure_factor": (c_int, [vp, c_int, c_int, dp, dp, dp, i64p, i64p]),
        "lb_batch_launch_count": (c_int, [vp, i64p]),
        "lb_batch_tuning": (c_int, [vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int), dp]),
        "lb_batch_last_error": (ctypes.c_char_p, [vp]),
        "lb_server_request_bytes": (c_sz, [c_int, c_int, c_int]),
        "lb_server_create": (c_int, [c_sz, c_int, c_int, ctypes.POINTER(vp)]),
        "lb_server_submit": (c_int, [vp, ctypes.POINTER(lb_request), i64p]),
        "lb_server_poll": (c_int, [vp, ctypes.POINTER(lb_result), c_int, ctypes.POINTER(c_int)]),
        "lb_server_wait": (c_int, [vp, c_i64, c_dbl, ctypes.POINTER(lb_result)]),
        "lb_server_fetch_populations": (c_int, [vp, c_i64, vp]),
        "lb_server_get_stats": (c_int, [vp, ctypes.POINTER(lb_server_stats)]),
        "lb_server_destroy": (c_int, [vp]),
        "lb_server_cancel": (c_int, [vp, c_i64]),
        "lb_server_inject_alloc_failures": (c_int, [vp, c_int]),
        "lb_server_set_admission": (c_int, [vp, c_i64, c_int]),
        "lb_selftest_bounded_wait": (c_int, [c_dbl, ctypes.POINTER(c_int)]),
        "lb_server_last_error": (ctypes.c_char_p, [vp]),
        "lb3_workspace_bytes": (c_sz, [c_int, c_int, c_int, c_int, c_int]),
        "lb3_create": (c_int, [c_int, c_int, c_int, c_int, c_int, c_u64, c_dbl, c_dbl, ctypes.POINTER(vp)]),
        "lb3_destroy": (c_int, [vp]),
        "lb3_set_stream": (c_int, [vp, vp]),
        "lb3_set_params": (c_int, [vp, c_dbl, c_dbl, c_dbl, c_dbl, c_dbl, c_int]),
        "lb3_set_eos": (c_int, [vp, c_int, c_dbl, c_dbl, c_dbl]),
        "lb3_step": (c_int, [vp, c_i64]),
        "lb3_get_time": (c_int, [vp, i64p]),
        "lb3_set_populations": (c_int, [vp, vp, c_int, c_i64]),
        "lb3_get_populations": (c_int, [vp, vp, c_int]),
        "lb3_sums": (c_int, [vp, dp]),
        "lb3_set_kernel_timing": (c_int, [vp, c_int]),
        "lb3_kernel_time": (c_int, [vp, dp, i64p]),
        "lb3_launch_count": (c_int, [vp, i64p]),
        "lb3_synchronize": (c_int, [vp]),
        "lb3_last_error": (ctypes.c_char_p, [vp]),
        "lb3_noise_matrix": (c_int, [c_int] + [c_dbl] * 6 + [dp]),
    }
    for name, (res, args) in proto.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc, ctx=None):
    if rc < 0:
        msg = load().lb_last_error(ctx)
        raise LBError(rc, msg.decode() if msg else "")
    return rc


def _bcheck(rc, b=None):
    if rc < 0:
        msg = load().lb_batch_last_error(b)
        raise LBError(rc, msg.decode() if msg else "")
    return rc


def _ptr(a):
    """Device or host address of a torch tensor or numpy array (plain int passes through)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()          # torch.Tensor


def _dptr(a):
    return ctypes.cast(_ptr(a), ctypes.POINTER(ctypes.c_double)) if a is not None else None


# --- the ABI, one Python function per C entry point ---------------------------------------

def lb_workspace_bytes(nx, ny, precision=LB_FP32):
    return load().lb_workspace_bytes(nx, ny, precision)


def lb_create(nx, ny, precision=LB_FP32, seed=42, rho0=1.0, cs2=1.0 / 3.0, workspace=None, workspace_bytes=0):
    out = ctypes.c_void_p()
    _check(load().lb_create(nx, ny, precision, seed, rho0, cs2, _ptr(workspace), workspace_bytes,
                            ctypes.byref(out)))
    return out.value


def lb_destroy(ctx):
    return _check(load().lb_destroy(ctx))


def lb_set_stream(ctx, stream):
    return _check(load().lb_set_stream(ctx, stream), ctx)


def lb_set_params(ctx, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode):
    return _check(load().lb_set_params(ctx, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode), ctx)


def lb_set_eos(ctx, eos, beta=0.0, rhoV=0.0, rhoL=0.0):
    return _check(load().lb_set_eos(ctx, eos, float(beta), float(rhoV), float(rhoL)), ctx)


def lb_set_noise_factor(ctx, factor):
    return _check(load().lb_set_noise_factor(ctx, factor), ctx)


def lb_step(ctx, nsteps):
    return _check(load().lb_step(ctx, nsteps), ctx)


def lb_get_time(ctx):
    t = ctypes.c_int64()
    _check(load().lb_get_time(ctx, ctypes.byref(t)), ctx)
    return t.value


def lb_set_populations(ctx, f, loc, t):
    return _check(load().lb_set_populations(ctx, _ptr(f), loc, t), ctx)


def lb_get_populations(ctx, f, loc):
    return _check(load().lb_get_populations(ctx, _ptr(f), loc), ctx)


def lb_moments(ctx, m, loc, sums):
    return _check(load().lb_moments(ctx, _ptr(m), loc, _dptr(sums)), ctx)


def lb_set_sampling(ctx, every, nbins):
    return _check(load().lb_set_sampling(ctx, every, nbins), ctx)


def lb_structure_factor(ctx, nbins, S_rho, S_jl, S_jt, counts, nsamples):
    i64 = lambda a: ctypes.cast(_ptr(a), ctypes.POINTER(ctypes.c_int64)) if a is not None else None
    return _check(load().lb_structure_factor(ctx, nbins, _dptr(S_rho), _dptr(S_jl), _dptr(S_jt), i64(counts),
                                             i64(nsamples)), ctx)


def lb_warnings(ctx):
    return load().lb_warnings(ctx)


def lb_last_error(ctx=None):
    m = load().lb_last_error(ctx)
    return m.decode() if m else ""


def lb_synchronize(ctx):
    return _check(load().lb_synchronize(ctx), ctx)


def lb_set_kernel_timing(ctx, on):
    return _check(load().lb_set_kernel_timing(ctx, int(on)), ctx)


def lb_kernel_time(ctx):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().lb_kernel_time(ctx, ctypes.byref(ms), ctypes.byref(n)), ctx)
    return ms.value, n.value


def lb_launch_count(ctx):
    n = ctypes.c_int64()
    _check(load().lb_launch_count(ctx, ctypes.byref(n)), ctx)
    return n.value


LB_STATIC_MAX_ROWS = 16384


def lb_conserved_sums_static(f, nx, ny, sums, stream=None):
    """Allocation-free FP64 conserved sums of caller-owned device populations (f, FP64,
    9*nx*ny) into the caller's device buffer sums (3 doubles), on `stream` (a cudaStream_t
    handle or None).  Returns without waiting for the GPU."""
    return _check(load().lb_conserved_sums_static(_ptr(f), nx, ny, _ptr(sums), stream))


def lb_noise_matrix(rho0, cs2, kT, kappa, tau_s, tau_b, tau_ghost, kx, ky):
    xi = np.zeros(81)
    _check(load().lb_noise_matrix(rho0, cs2, kT, kappa, tau_s, tau_b, tau_ghost, kx, ky, _dptr(xi)))
    return xi.reshape(9, 9)


def lb_check_params(nx, ny, rho0, cs2, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode):
    return load().lb_check_params(nx, ny, rho0, cs2, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode)


# --- batched ensembles -----------------------------------------------------------------------

def _i32(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32))


def lb_batch_workspace_bytes(nx, ny):
    nx, ny = _i32(nx), _i32(ny)
    return load().lb_batch_workspace_bytes(len(nx), nx.ctypes.data, ny.ctypes.data)


def lb_batch_create(nx, ny, seeds, rho0=1.0, cs2=1.0 / 3.0, workspace=None, workspace_bytes=0):
    nx, ny = _i32(nx), _i32(ny)
    sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    if not (len(nx) == len(ny) == len(sd)):
        raise LBError(LB_EINVAL, "nx, ny and seeds must have one entry per replica")
    out = ctypes.c_void_p()
    _bcheck(load().lb_batch_create(len(nx), nx.ctypes.data, ny.ctypes.data, sd.ctypes.data, rho0, cs2,
                                   _ptr(workspace), workspace_bytes, ctypes.byref(out)))
    return out.value


def lb_batch_destroy(b):
    return _bcheck(load().lb_batch_destroy(b))


def lb_batch_set_stream(b, stream):
    return _bcheck(load().lb_batch_set_stream(b, stream), b)


def lb_batch_set_params(b, replica, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode):
    return _bcheck(load().lb_batch_set_params(b, replica, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode), b)


def lb_batch_autotune(b, steps):
    return _bcheck(load().lb_batch_autotune(b, steps), b)


def lb_batch_step(b, nsteps):
    return _bcheck(load().lb_batch_step(b, nsteps), b)


def lb_batch_step_graph(b, nsteps, steps_per_graph):
    return _bcheck(load().lb_batch_step_graph(b, nsteps, steps_per_graph), b)


def lb_batch_get_time(b, replica):
    t = ctypes.c_int64()
    _bcheck(load().lb_batch_get_time(b, replica, ctypes.byref(t)), b)
    return t.value


def lb_batch_set_populations(b, replica, f, loc, t):
    return _bcheck(load().lb_batch_set_populations(b, replica, _ptr(f), loc, t), b)


def lb_batch_get_populations(b, replica, f, loc):
    return _bcheck(load().lb_batch_get_populations(b, replica, _ptr(f), loc), b)


def lb_batch_sums(b, replica, sums):
    return _bcheck(load().lb_batch_sums(b, replica, _dptr(sums)), b)


def lb_batch_set_sampling(b, every, nbins):
    return _bcheck(load().lb_batch_set_sampling(b, every, nbins), b)


def lb_batch_structure_factor(b, replica, nbins, S_rho, S_jl, S_jt, counts, nsamples):
    i64 = lambda a: ctypes.cast(_ptr(a), ctypes.POINTER(ctypes.c_int64)) if a is not None else None
    return _bcheck(load().lb_batch_structure_factor(b, replica, nbins, _dptr(S_rho), _dptr(S_jl), _dptr(S_jt),
                                                    i64(counts), i64(nsamples)), b)


def lb_batch_launch_count(b):
    n = ctypes.c_int64()
    _bcheck(load().lb_batch_launch_count(b, ctypes.byref(n)), b)
    return n.value


def lb_batch_tuning(b):
    """(tile_x, tile_y, threads, ms_per_step) of the step kernel in use."""
    tx, ty, nt, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _bcheck(load().lb_batch_tuning(b, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(nt), ctypes.byref(ms)), b)
    return tx.value, ty.value, nt.value, ms.value


def lb_batch_last_error(b=None):
    m = load().lb_batch_last_error(b)
    return m.decode() if m else ""


# --- request server --------------------------------------------------------------------------

def _scheck(rc, srv=None):
    if rc < 0:
        msg = load().lb_server_last_error(srv)
        raise LBError(rc, msg.decode() if msg else "")
    return rc


def lb_server_request_bytes(nx, ny, noise_mode=LB_NOISE_LW):
    return load().lb_server_request_bytes(nx, ny, noise_mode)


def lb_server_create(hbm_budget_bytes, max_active=4096, max_chunk_steps=500):
    out = ctypes.c_void_p()
    _scheck(load().lb_server_create(int(hbm_budget_bytes), max_active, max_chunk_steps, ctypes.byref(out)))
    return out.value


def lb_server_submit(srv, req):
    i = ctypes.c_int64()
    _scheck(load().lb_server_submit(srv, ctypes.byref(req), ctypes.byref(i)), None)
    return i.value


def lb_server_poll(srv, max_results=1024):
    buf = (lb_result * max_results)()
    n = ctypes.c_int()
    _scheck(load().lb_server_poll(srv, buf, max_results, ctypes.byref(n)), srv)
    return [buf[i] for i in range(n.value)]


def lb_server_wait(srv, id=0, timeout_s=-1.0):
    res = lb_result()
    _scheck(load().lb_server_wait(srv, id, timeout_s, ctypes.byref(res)), srv)
    return res if id > 0 else None


def lb_server_fetch_populations(srv, id, f):
    return _scheck(load().lb_server_fetch_populations(srv, id, _ptr(f)), srv)


def lb_server_get_stats(srv):
    st = lb_server_stats()
    _scheck(load().lb_server_get_stats(srv, ctypes.byref(st)), srv)
    return st


def lb_server_cancel(srv, id):
    return _scheck(load().lb_server_cancel(srv, id), srv)


def lb_server_set_admission(srv, large_nodes, max_large):
    return _scheck(load().lb_server_set_admission(srv, int(large_nodes), int(max_large)), srv)


def lb_server_inject_alloc_failures(srv, count):
    return _scheck(load().lb_server_inject_alloc_failures(srv, count), srv)


def lb_selftest_bounded_wait(limit_s):
    """Runs the device-side timeout self-test; returns (return code, gave_up flag)."""
    g = ctypes.c_int()
    rc = load().lb_selftest_bounded_wait(limit_s, ctypes.byref(g))
    return rc, g.value


def lb_server_destroy(srv):
    return _scheck(load().lb_server_destroy(srv))


def lb_server_last_error(srv=None):
    m = load().lb_server_last_error(srv)
    return m.decode() if m else ""


# --- convenience wrappers ------------------------------------------------------------------

class Lattice:
    """One lattice on the current CUDA device.  PyTorch allocates the workspace and
    provides the stream (torch.cuda.current_stream() at construction, unless given)."""

    def __init__(self, nx, ny, seed=42, rho0=1.0, cs2=1.0 / 3.0, stream=None, precision=LB_FP32):
        import torch
        self.nx, self.ny = int(nx), int(ny)
        nbytes = lb_workspace_bytes(self.nx, self.ny, precision)
        if nbytes == 0:
            raise LBError(LB_EINVAL, "invalid lattice size %dx%d or precision" % (nx, ny))
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self._ws.data_ptr()
        aligned = (base + 255) & ~255
        self.ctx = lb_create(self.nx, self.ny, precision, seed, rho0, cs2, aligned, nbytes)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        lb_set_stream(self.ctx, self.stream.cuda_stream)
        self.nbins = 0

    def close(self):
        if getattr(self, "ctx", None):
            lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode):
        lb_set_params(self.ctx, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode)

    def set_eos(self, eos, beta=0.0, rhoV=0.0, rhoL=0.0):
        lb_set_eos(self.ctx, eos, beta, rhoV, rhoL)

    def set_noise_factor(self, factor):
        lb_set_noise_factor(self.ctx, factor)

    def step(self, n=1):
        lb_step(self.ctx, n)

    @property
    def t(self):
        return lb_get_time(self.ctx)

    def set_populations(self, f, t=0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx)
        lb_set_populations(self.ctx, f, LB_HOST, t)

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        lb_get_populations(self.ctx, f, LB_HOST)
        return f

    def moments(self):
        m = np.empty((9, self.ny, self.nx))
        s = np.zeros(3)
        lb_moments(self.ctx, m, LB_HOST, s)
        return m, s

    def sums(self):
        s = np.zeros(3)
        lb_moments(self.ctx, None, LB_HOST, s)
        return s

    def set_sampling(self, every, nbins):
        lb_set_sampling(self.ctx, every, nbins)
        self.nbins = nbins

    def structure_factor(self):
        nb = self.nbins
        S, L, Tt = np.zeros(nb), np.zeros(nb), np.zeros(nb)
        cnt = np.zeros(nb, dtype=np.int64)
        ns = np.zeros(1, dtype=np.int64)
        lb_structure_factor(self.ctx, nb, S, L, Tt, cnt, ns)
        return S, L, Tt, cnt, int(ns[0])


class Ensemble:
    """Many independent lattices stepped together on the current CUDA device (workspace
    owned by PyTorch, stream as for ``Lattice``).  ``sizes`` is a list of (nx, ny)."""

    def __init__(self, sizes, seeds, rho0=1.0, cs2=1.0 / 3.0, stream=None):
        import torch
        self.sizes = [(int(a), int(b)) for a, b in sizes]
        nx = [a for a, _ in self.sizes]
        ny = [b for _, b in self.sizes]
        nbytes = lb_batch_workspace_bytes(nx, ny)
        if nbytes == 0:
            raise LBError(LB_EINVAL, "invalid lattice sizes")
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        aligned = (self._ws.data_ptr() + 255) & ~255
        self.b = lb_batch_create(nx, ny, seeds, rho0, cs2, aligned, nbytes)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        lb_batch_set_stream(self.b, self.stream.cuda_stream)
        self.nbins = 0

    def __len__(self):
        return len(self.sizes)

    def close(self):
        if getattr(self, "b", None):
            lb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, replica, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode):
        lb_batch_set_params(self.b, replica, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode)

    def autotune(self, steps=10):
        lb_batch_autotune(self.b, steps)

    def step(self, n=1, graph_steps=0):
        if graph_steps > 0:
            lb_batch_step_graph(self.b, n, graph_steps)
        else:
            lb_batch_step(self.b, n)

    def t(self, replica):
        return lb_batch_get_time(self.b, replica)

    def set_populations(self, replica, f, t=0):
        nx, ny = self.sizes[replica]
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (9, ny, nx)
        lb_batch_set_populations(self.b, replica, f, LB_HOST, t)

    def populations(self, replica):
        nx, ny = self.sizes[replica]
        f = np.empty((9, ny, nx))
        lb_batch_get_populations(self.b, replica, f, LB_HOST)
        return f

    def sums(self, replica):
        s = np.zeros(3)
        lb_batch_sums(self.b, replica, s)
        return s

    def set_sampling(self, every, nbins):
        lb_batch_set_sampling(self.b, every, nbins)
        self.nbins = nbins

    def structure_factor(self, replica):
        nb = self.nbins
        S, L, Tt = np.zeros(nb), np.zeros(nb), np.zeros(nb)
        cnt = np.zeros(nb, dtype=np.int64)
        ns = np.zeros(1, dtype=np.int64)
        lb_batch_structure_factor(self.b, replica, nb, S, L, Tt, cnt, ns)
        return S, L, Tt, cnt, int(ns[0])


class Server:
    """The request server on the current CUDA device (see lb_server_* in lbfluct.h)."""

    def __init__(self, hbm_budget_bytes, max_active=4096, max_chunk_steps=500):
        self.srv = lb_server_create(hbm_budget_bytes, max_active, max_chunk_steps)

    def submit(self, nx, ny, steps, kT=1e-4, kappa=0.01, tau_s=1.0, tau_b=1.0, tau_ghost=1.0,
               noise_mode=LB_NOISE_LW, seed=42, rho0=1.0, cs2=1.0 / 3.0, keep_state=False, init=None):
        """init: optional FP64 pre-collision populations [9, ny, nx] to start from (else rest)."""
        r = lb_request(nx=int(nx), ny=int(ny), steps=int(steps), rho0=rho0, cs2=cs2, kT=kT, kappa=kappa,
                       tau_s=tau_s, tau_b=tau_b, tau_ghost=tau_ghost, noise_mode=noise_mode,
                       keep_state=int(bool(keep_state)), seed=int(seed))
        if init is not None:
            f = np.ascontiguousarray(init, dtype=np.float64)
            if f.shape != (9, int(ny), int(nx)):
                raise ValueError("init must have shape (9, ny, nx)")
            r.init = f.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            return lb_server_submit(self.srv, r)       # copied before the call returns; f alive here
        return lb_server_submit(self.srv, r)

    def wait(self, id=0, timeout_s=-1.0):
        return lb_server_wait(self.srv, id, timeout_s)

    def poll(self, max_results=1024):
        return lb_server_poll(self.srv, max_results)

    def fetch(self, id, nx, ny):
        f = np.empty((9, ny, nx))
        lb_server_fetch_populations(self.srv, id, f)
        return f

    def stats(self):
        return lb_server_get_stats(self.srv)

    def cancel(self, id):
        lb_server_cancel(self.srv, id)

    def close(self):
        if getattr(self, "srv", None):
            lb_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- D3Q19 lattice (include/lbfluct3d.h) ---------------------------------------------------

def _check3(rc, ctx=None):
    if rc < 0:
        msg = load().lb3_last_error(ctx)
        raise LBError(rc, msg.decode() if msg else "")
    return rc


def lb3_workspace_bytes(nx, ny, nz, lattice=LB_D3Q19, precision=LB_FP32):
    return load().lb3_workspace_bytes(nx, ny, nz, lattice, precision)


def lb3_create(nx, ny, nz, lattice=LB_D3Q19, precision=LB_FP32, seed=42, rho0=1.0, cs2=1.0 / 3.0):
    out = ctypes.c_void_p()
    _check3(load().lb3_create(nx, ny, nz, lattice, precision, seed, rho0, cs2, ctypes.byref(out)))
    return out.value


def lb3_destroy(ctx):
    return _check3(load().lb3_destroy(ctx))


def lb3_set_stream(ctx, stream):
    return _check3(load().lb3_set_stream(ctx, stream), ctx)


def lb3_set_params(ctx, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode):
    return _check3(load().lb3_set_params(ctx, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode), ctx)


def lb3_set_eos(ctx, eos, beta=0.0, rhoV=0.0, rhoL=0.0):
    return _check3(load().lb3_set_eos(ctx, eos, float(beta), float(rhoV), float(rhoL)), ctx)


def lb3_step(ctx, nsteps):
    return _check3(load().lb3_step(ctx, nsteps), ctx)


def lb3_get_time(ctx):
    t = ctypes.c_int64()
    _check3(load().lb3_get_time(ctx, ctypes.byref(t)), ctx)
    return t.value


def lb3_set_populations(ctx, f, loc, t):
    return _check3(load().lb3_set_populations(ctx, _ptr(f), loc, t), ctx)


def lb3_get_populations(ctx, f, loc):
    return _check3(load().lb3_get_populations(ctx, _ptr(f), loc), ctx)


def lb3_sums(ctx, sums):
    return _check3(load().lb3_sums(ctx, _dptr(sums)), ctx)


def lb3_set_kernel_timing(ctx, every):
    return _check3(load().lb3_set_kernel_timing(ctx, every), ctx)


def lb3_kernel_time(ctx):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check3(load().lb3_kernel_time(ctx, ctypes.byref(ms), ctypes.byref(n)), ctx)
    return ms.value, n.value


def lb3_launch_count(ctx):
    n = ctypes.c_int64()
    _check3(load().lb3_launch_count(ctx, ctypes.byref(n)), ctx)
    return n.value


def lb3_synchronize(ctx):
    return _check3(load().lb3_synchronize(ctx), ctx)


def lb3_noise_matrix(rho0, cs2, kT, tau_s, tau_b, tau_ghost, lattice=LB_D3Q19):
    X = np.zeros((lattice, lattice))
    _check3(load().lb3_noise_matrix(lattice, rho0, cs2, kT, tau_s, tau_b, tau_ghost, _dptr(X)))
    return X


class Lattice3:
    """One periodic D3Q19 or D3Q27 lattice on the current CUDA device; its work runs on the
    given stream (torch.cuda.current_stream() at construction, unless given)."""

    def __init__(self, nx, ny, nz, seed=42, rho0=1.0, cs2=1.0 / 3.0, stream=None, precision=LB_FP32,
                 lattice=LB_D3Q19):
        import torch
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.q = int(lattice)
        self.ctx = lb3_create(self.nx, self.ny, self.nz, lattice, precision, seed, rho0, cs2)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        lb3_set_stream(self.ctx, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "ctx", None):
            lb3_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode):
        lb3_set_params(self.ctx, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode)

    def set_eos(self, eos, beta=0.0, rhoV=0.0, rhoL=0.0):
        lb3_set_eos(self.ctx, eos, beta, rhoV, rhoL)

    def step(self, n=1):
        lb3_step(self.ctx, n)

    @property
    def t(self):
        return lb3_get_time(self.ctx)

    def set_populations(self, f, t=0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (self.q, self.nz, self.ny, self.nx)
        lb3_set_populations(self.ctx, f, LB_HOST, t)

    def populations(self):
        f = np.empty((self.q, self.nz, self.ny, self.nx))
        lb3_get_populations(self.ctx, f, LB_HOST)
        return f

    def sums(self):
        s = np.zeros(4)
        lb3_sums(self.ctx, s)
        return s
