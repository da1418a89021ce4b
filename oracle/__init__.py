"""FP64 CPU oracle for the fluctuating D2Q9 lattice Boltzmann step of arXiv:1009.0254.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers.  The product library never imports this
package and shares no code with it: the C core (``lbref.c``) does the per-site
collision and streaming in plain loops, and this module builds the noise of Sec. IV
and the statistics used by the paper's Results section with numpy.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against the
paper's printed matrices, closed forms, the linear theory or brute force (see the
tests named in each docstring).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import theory
from .theory import C, N, SIGMA_S2, T, TINV, W, Model

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbref.so")
_lib = None

NOISE_OFF, NOISE_LW, NOISE_FULL, NOISE_DIAG, NOISE_FULL_RS, NOISE_LW_LOCAL = 0, 1, 2, 3, 4, 5
TAG_NODE, TAG_KSPACE, TAG_STENCIL = 0, 2, 3


def build(force: bool = False) -> str:
    """Compile the C core with gcc into oracle/_build/liblbref.so."""
    src = os.path.join(_HERE, "lbref.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.oracle_tables.argtypes = [dp, dp, dp, ctypes.POINTER(ctypes.c_int)]
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_normals.argtypes = [ctypes.c_int64, u32p, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_uint32, dp]
        L.oracle_step.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        L.oracle_collide_sites.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_int64), dp, dp, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


# --- random numbers ------------------------------------------------------------

def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (Salmon et al., SC'11) of the C core."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib().oracle_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
    return out


def normals(index, seed: int, step: int, tag: int) -> np.ndarray:
    """Eight unit normals per counter index (one Box-Muller pair per Philox output word):
    shape (len(index), 8)."""
    idx = np.ascontiguousarray(np.asarray(index, dtype=np.uint32))
    out = np.zeros((idx.size, 8))
    lib().oracle_normals(idx.size, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                         ctypes.c_uint64(seed), ctypes.c_uint64(step), ctypes.c_uint32(tag), _dp(out))
    return out


# --- noise of Sec. IV ------------------------------------------------------------

def _fft_conj_index(nx, ny):
    """Linear index of -k for every k = (mx, my), array [my, mx]."""
    mx = np.arange(nx)
    my = np.arange(ny)
    MX, MY = np.meshgrid(mx, my, indexing="xy")
    return ((ny - MY) % ny) * nx + (nx - MX) % nx


def eta_field(nx, ny, seed, step):
    """Two independent Hermitian unit Gaussian fields eta_1(k), eta_2(k), arrays [my, mx].

    Every pair (k, -k) shares one draw owned by the lower linear index my*nx + mx
    (tag 2): eta = (n0 + i n1)/sqrt(2), (n2 + i n3)/sqrt(2) at the owner and the
    conjugate at its partner; at self-conjugate k only the real parts n0, n2 are
    used, so <|eta(k)|^2> = 1 everywhere."""
    n = nx * ny
    lin = np.arange(n).reshape(ny, nx)
    conj = _fft_conj_index(nx, ny)
    owner = np.minimum(lin, conj)
    g = normals(np.arange(n, dtype=np.uint32), seed, step, TAG_KSPACE)   # draw for every index
    go = g[owner.ravel()].reshape(ny, nx, 8)
    selfc = lin == conj
    is_owner = lin == owner
    e1 = np.where(selfc, go[..., 0] + 0j, (go[..., 0] + 1j * go[..., 1]) / np.sqrt(2))
    e2 = np.where(selfc, go[..., 2] + 0j, (go[..., 2] + 1j * go[..., 3]) / np.sqrt(2))
    e1 = np.where(is_owner | selfc, e1, np.conj(e1))
    e2 = np.where(is_owner | selfc, e2, np.conj(e2))
    return e1, e2


def block49_factor(model: Model, kx, ky, factor: str = "cholesky"):
    """Factor (L44, L49, L94, L99) of the (4,9) block of Xi(k), Eq. (noise-yeo), vectorised
    over k: Cholesky (L49 = 0; zero pivots clamped to 0, Sec. IV: Xi is only PSD) or the
    eigen-decomposition factor S diag(sqrt(e))."""
    c2k = model.cs2_k(kx, ky)
    lb, le = model.lam[3], model.lam[8]
    pref = -(model.rho0 * model.kT / SIGMA_S2)
    x44 = pref * N[3] * (2 - 3 * c2k) * lb * (2 + lb)
    x49 = pref * 12 * (c2k - SIGMA_S2) * (lb + le + lb * le)
    x99 = pref * N[8] * (5 / 4 - 3 / 4 * c2k) * le * (2 + le)
    scale = np.maximum(np.abs(x44), np.abs(x99)) + 1e-300
    if np.any(x44 < -1e-9 * scale) or np.any(x99 < -1e-9 * scale):
        raise ValueError("Xi(k) is not positive semidefinite on this grid")
    if factor == "eigen":
        return theory.eigen_factor_2x2(x44, x49, x99)
    L44 = np.sqrt(np.maximum(x44, 0.0))
    L94 = np.where(L44 > 0, x49 / np.where(L44 > 0, L44, 1.0), 0.0)
    rem = x99 - L94 * L94
    if np.any(rem < -1e-9 * scale):
        raise ValueError("Xi(k) is not positive semidefinite on this grid")
    L99 = np.sqrt(np.maximum(rem, 0.0))
    return L44, np.zeros_like(L44), L94, L99


def xi49_full(model: Model, nx, ny, seed, step, factor: str = "cholesky"):
    """Spatially correlated noise of modes 4 and 9 (Sec. IV, last paragraph): in k-space
    xi(k) = L(k) eta(k) with L L^T the (4,9) block of Xi(k), Eq. (noise-yeo), then one
    transform back to the lattice with the unitary convention of Sec. III:
    a(r) = n^-1/2 sum_k exp(-i k.r) a(k).  Returns real fields xi4[y, x], xi9[y, x]."""
    KX, KY = theory.lattice_k(nx, ny)
    L44, L49, L94, L99 = block49_factor(model, KX, KY, factor)
    e1, e2 = eta_field(nx, ny, seed, step)
    x4k = L44 * e1 + L49 * e2
    x9k = L94 * e1 + L99 * e2
    n = nx * ny
    # numpy's forward fft2 computes sum_k a(k) exp(-2 pi i (mx x/nx + my y/ny))
    x4 = np.fft.fft2(x4k) / np.sqrt(n)
    x9 = np.fft.fft2(x9k) / np.sqrt(n)
    return x4.real, x9.real


# --- correlated noise built in real space ------------------------------------------------
#
# Every k-dependent entry of Xi(k), Eq. (noise-yeo), depends on k only through the lattice
# k^2 = s(k) of Appendix B, and affinely: Xi_(4,9)(k) = A + B s(k), s in [0, 16/3].  With
# cx = cos kx, cy = cos ky, s = (10 - 4 cx - 4 cy - 2 cx cy) / 3, and the four products
# P_ab(k) = (1 + a e^{i kx})(1 + b e^{i ky}) (a, b = +-1) have |P_ab|^2 = 4 (1 + a cx)(1 + b cy),
#   (1/16) [ |P_++|^2 + |P_+-|^2 + |P_-+|^2 + |P_--|^2 ]              = 1,
#   (1/16) [ 4 (|P_+-|^2 + |P_-+|^2) + (16/3) |P_--|^2 ]               = s(k),
# so Xi(k) = (1/16) [ Xi(s=0) |P_++|^2 + Xi(s=4) (|P_+-|^2 + |P_-+|^2) + Xi(s=16/3) |P_--|^2 ].
# Four independent white 2-vector fields nu_ab, each multiplied by a factor L_ab of Xi at its
# s and filtered by the 2 x 2 stencil P_ab, add up to a field whose covariance is Xi(k) at
# every k: the same Gaussian field the Fourier construction of Sec. IV gives (it exists when
# Xi is positive semidefinite at s = 0 and s = 16/3, hence on the whole range), built from
# one 2 x 2 box of nodes, on a lattice of any size.

# wavevectors where the lattice k^2 takes the values 0, 4 and 16/3
STENCIL_K = {"++": (0.0, 0.0), "+-": (2 * np.pi / 3, np.pi / 2), "-+": (2 * np.pi / 3, np.pi / 2),
             "--": (np.pi, np.pi)}
STENCIL_SIGNS = {"++": (1, 1), "+-": (1, -1), "-+": (-1, 1), "--": (-1, -1)}
STENCIL_ORDER = ("++", "+-", "-+", "--")


def stencil_factors(model: Model, factor: str = "cholesky"):
    """Factors L_ab (2 x 2, rows/columns modes 4 and 9) of the four fields: L L^T is the
    (4,9) block of Xi of Eq. (noise-yeo) at s = 0, 4, 4 and 16/3."""
    out = []
    for ab in STENCIL_ORDER:
        kx, ky = STENCIL_K[ab]
        l11, l12, l21, l22 = block49_factor(model, np.array(kx), np.array(ky), factor)
        out.append(np.array([[float(l11), float(l12)], [float(l21), float(l22)]]))
    return out


def stencil_combine(nu, Ls):
    """xi_(4,9)(r) = 1/4 sum_ab sum_{dx,dy in {0,1}} a^dx b^dy L_ab nu_ab(r - dx e_x - dy e_y)
    (periodic), from nu[ab, component, y, x] (ab in STENCIL_ORDER); returns (2, ny, nx)."""
    out = np.zeros(nu.shape[1:])
    for idx, ab in enumerate(STENCIL_ORDER):
        a, b = STENCIL_SIGNS[ab]
        g = np.einsum("cd,dyx->cyx", Ls[idx], nu[idx])
        for dx in (0, 1):
            for dy in (0, 1):
                out += (a ** dx) * (b ** dy) * np.roll(g, shift=(dy, dx), axis=(1, 2))
    return out / 4.0


def stencil_fields(nx, ny, seed, step):
    """The four white fields nu_ab (shape (4, 2, ny, nx)): one draw per node (tag 3), the
    Box-Muller pair of output word w gives the two components of field w."""
    g = normals(np.arange(nx * ny, dtype=np.uint32), seed, step, TAG_STENCIL)      # (n, 8)
    return g.T.reshape(4, 2, ny, nx)


def xi49_stencil(model: Model, nx, ny, seed, step, factor: str = "cholesky"):
    """Correlated noise of modes 4 and 9 with covariance Xi(k) built in real space (see
    above).  Returns real fields xi4[y, x], xi9[y, x]."""
    x = stencil_combine(stencil_fields(nx, ny, seed, step), stencil_factors(model, factor))
    return x[0], x[1]


def xi49_stencil_at(model: Model, nx, ny, seed, step, sites, factor: str = "cholesky"):
    """The same at the listed linear sites only (draws at the 2 x 2 box below-left of each
    site): returns (len(sites), 2)."""
    sites = np.asarray(sites, dtype=np.int64)
    x = sites % nx
    y = sites // nx
    Ls = stencil_factors(model, factor)
    out = np.zeros((sites.size, 2))
    for dx in (0, 1):
        for dy in (0, 1):
            q = ((y - dy) % ny) * nx + (x - dx) % nx
            nu = normals(q.astype(np.uint32), seed, step, TAG_STENCIL).reshape(-1, 4, 2)
            for idx, ab in enumerate(STENCIL_ORDER):
                a, b = STENCIL_SIGNS[ab]
                out += (a ** dx) * (b ** dy) * (nu[:, idx, :] @ Ls[idx].T)
    return out / 4.0


def noise_fields(model: Model, mode: int, nx, ny, seed, step, L0=None, factor: str = "cholesky"):
    """xi[a, y, x] for one step (Sec. IV).

    LW:   xi = L nu with L L^T = Xi(0) (lower-right 6x6 Cholesky); one draw per node
          (tag 0): nu_5..8 from its words 0, 1 and (nu_4, nu_9) from word 2; spatially
          uncorrelated.
    DIAG: as LW with the off-diagonal Xi_49 dropped ("ideal gas-like" noise, Sec. IV).
    FULL: modes 5..8 as LW (their variances do not depend on k); modes 4, 9 from
          xi49_full().
    FULL_RS: as FULL with modes 4, 9 from xi49_stencil() (the same covariance Xi(k))."""
    n = nx * ny
    xi = np.zeros((9, ny, nx))
    if mode == NOISE_OFF or model.kT == 0.0:
        return xi
    idx = np.arange(n, dtype=np.uint32)
    g0 = normals(idx, seed, step, TAG_NODE)
    nu = np.zeros((9, n))
    nu[4:8] = g0[:, 0:4].T
    if mode in (NOISE_LW, NOISE_DIAG):
        nu[3] = g0[:, 4]
        nu[8] = g0[:, 5]
    if L0 is None:
        X0 = model.Xi_zero()
        if mode == NOISE_DIAG:
            X0 = np.diag(np.diag(X0))
        L0 = theory.noise_factor(X0, factor)
    xi_flat = L0 @ nu
    xi[:] = xi_flat.reshape(9, ny, nx)
    if mode == NOISE_FULL:
        x4, x9 = xi49_full(model, nx, ny, seed, step, factor)
        xi[3] = x4
        xi[8] = x9
    elif mode == NOISE_FULL_RS:
        x4, x9 = xi49_stencil(model, nx, ny, seed, step, factor)
        xi[3] = x4
        xi[8] = x9
    return xi


# --- the step -----------------------------------------------------------------------

def params_vector(model: Model, eos=None) -> np.ndarray:
    """{rho0, cs2, kappa, lambda_1..9, eos, beta, rhoV, rhoL} for the C core (eos 0: p0 = cs2
    rho; 1: the double well `eos`, a theory.DoubleWell)."""
    tail = [0.0, 0.0, 0.0, 0.0] if eos is None else [1.0, eos.beta, eos.rhoV, eos.rhoL]
    return np.concatenate([[model.rho0, model.cs2, model.kappa], model.lam, tail]).astype(np.float64)


def step(f: np.ndarray, model: Model, xi=None, eos=None) -> np.ndarray:
    """One step of Eq. (fluct-lin-lbe) on a periodic lattice: f[9, ny, nx] pre-collision
    populations in, next pre-collision populations out (FP64).  eos: None for p0 = cs2 rho,
    else a theory.DoubleWell."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, ny, nx = f.shape
    out = np.empty_like(f)
    par = params_vector(model, eos)
    xi_c = None if xi is None else np.ascontiguousarray(xi, dtype=np.float64)
    lib().oracle_step(nx, ny, _dp(f), _dp(out), _dp(par), _dp(xi_c))
    return out


def collide_sites(f: np.ndarray, model: Model, sites: np.ndarray, xi_sites=None, eos=None) -> np.ndarray:
    """Post-collision populations f*_i at the given linear sites, shape (len(sites), 9)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, ny, nx = f.shape
    s = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.zeros((s.size, 9))
    par = params_vector(model, eos)
    xs = None if xi_sites is None else np.ascontiguousarray(xi_sites, dtype=np.float64)
    lib().oracle_collide_sites(nx, ny, _dp(f), s.size, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               _dp(par), _dp(xs), _dp(out))
    return out


# --- uncorrelated noise at the local density (inhomogeneous systems) ------------------------

def xi_zero_local(model: Model, rho, c2):
    """Entries of Xi(0), Eq. (noise-yeo) at k = 0, with the density rho0 and the sound speed
    squared c_s^2 replaced by local values rho, c2 (arrays): the uncorrelated noise of an
    inhomogeneous system (Sec. IV, and Sec. V B: local density and sound speed in the
    real-space noise variance).  Returns x44, x49, x99, x55, x66, x77 (= x88)."""
    lb, ls, lq, le = model.lam[3], model.lam[4], model.lam[6], model.lam[8]
    til = lambda l: l * (2 + l)
    til_be = lb + le + lb * le
    pref = -(np.asarray(rho) * model.kT / SIGMA_S2)
    return (pref * N[3] * (2 - 3 * c2) * til(lb), pref * 12 * (c2 - SIGMA_S2) * til_be,
            pref * N[8] * (5 / 4 - 3 / 4 * c2) * til(le), pref * N[4] * til(ls), pref * N[5] * til(ls),
            pref * N[6] * til(lq))


def local_noise_fields(model: Model, rho, c2, seed, step):
    """xi[a, y, x] of the uncorrelated noise at the local density: at every node the (4,9)
    block of xi_zero_local is factored by Cholesky (a negative pivot, where the local block is
    not positive semidefinite, is clamped to zero), the other modes take the square roots of
    their variances; the unit normals are the long-wavelength mode's (tag 0)."""
    ny, nx = rho.shape
    n = nx * ny
    g0 = normals(np.arange(n, dtype=np.uint32), seed, step, TAG_NODE)
    x44, x49, x99, x55, x66, x77 = xi_zero_local(model, rho.ravel(), np.broadcast_to(c2, rho.shape).ravel())
    L44 = np.sqrt(np.maximum(x44, 0.0))
    L94 = np.where(L44 > 0, x49 / np.where(L44 > 0, L44, 1.0), 0.0)
    L99 = np.sqrt(np.maximum(x99 - L94 * L94, 0.0))
    xi = np.zeros((9, n))
    xi[3] = L44 * g0[:, 4]
    xi[8] = L94 * g0[:, 4] + L99 * g0[:, 5]
    xi[4] = np.sqrt(np.maximum(x55, 0.0)) * g0[:, 0]
    xi[5] = np.sqrt(np.maximum(x66, 0.0)) * g0[:, 1]
    xi[6] = np.sqrt(np.maximum(x77, 0.0)) * g0[:, 2]
    xi[7] = np.sqrt(np.maximum(x77, 0.0)) * g0[:, 3]
    return xi.reshape(9, ny, nx)


class Lattice:
    """A periodic nx x ny lattice stepped by the oracle (FP64), noise per Sec. IV.

    ``f`` holds pre-collision populations f[i, y, x]; ``t`` is the index of the next
    collision, which keys its random numbers.  ``eos`` (a theory.DoubleWell) replaces the
    linearised p0 = cs2 rho by the double well's bulk pressure; the linear theory about rho0
    (noise covariance, rest state) then takes c_s^2(rho0) and p0(rho0)."""

    def __init__(self, nx, ny, rho0=1.0, cs2=SIGMA_S2, seed=42, eos=None):
        self.nx, self.ny = int(nx), int(ny)
        self.seed = int(seed)
        self.eos = eos
        if eos is None:
            self.model = Model(rho0=rho0, cs2=cs2)
        else:
            self.model = Model(rho0=rho0, cs2=eos.cs2(rho0), p0_rest=eos.p0(rho0))
        self.mode = NOISE_OFF
        self.t = 0
        rest = self.model.fbar() if eos is None else self.model.rest()
        self.f = np.broadcast_to(rest[:, None, None], (9, ny, nx)).copy()
        self._L0 = None
        self.factor = "cholesky"

    def set_params(self, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode, factor=None):
        """factor: "cholesky" (default) or "eigen", the factorisation of the noise matrix
        (Sec. IV); None keeps the current one."""
        if factor is not None:
            self.factor = factor
        m = Model(self.model.rho0, self.model.cs2, kappa, kT, tau_s, tau_b, tau_ghost, p0_rest=self.model.p0_rest)
        fb_old = self.model.fbar()
        self.model = m
        self.mode = int(noise_mode)
        X0 = m.Xi_zero()
        if self.mode == NOISE_DIAG:
            X0 = np.diag(np.diag(X0))
        self._L0 = theory.noise_factor(X0, self.factor)
        del fb_old

    def local_sound_speed2(self, rho):
        """c_s^2 at density rho: rho d2f0/drho2 of the double well, else the constant cs2."""
        return self.eos.cs2(rho) if self.eos is not None else np.full_like(rho, self.model.cs2)

    def noise(self, t=None):
        t = self.t if t is None else t
        if self.mode == NOISE_LW_LOCAL:
            rho = self.f.sum(axis=0)         # the density the collision at time t sees
            return local_noise_fields(self.model, rho, self.local_sound_speed2(rho), self.seed, t)
        return noise_fields(self.model, self.mode, self.nx, self.ny, self.seed, t, self._L0, self.factor)

    def step(self, nsteps=1):
        for _ in range(int(nsteps)):
            xi = None
            if self.mode != NOISE_OFF and self.model.kT > 0:
                xi = self.noise()
            self.f = step(self.f, self.model, xi, self.eos)
            self.t += 1
        return self

    def moments(self) -> np.ndarray:
        """m_a(r) = sum_i T_ai f_i(r), shape (9, ny, nx)."""
        return np.einsum("ai,iyx->ayx", T, self.f)


# --- statistics of the Results section ------------------------------------------------

def unitary_ft(a: np.ndarray) -> np.ndarray:
    """a(k) = n^-1/2 sum_r exp(+i k.r) a(r) (Sec. III, notation), array [my, mx]."""
    n = a.size
    return np.fft.ifft2(a) * np.sqrt(n)


def k_bins(nx, ny, nbins):
    """Radial bin of every wavevector: |k| with components wrapped to (-pi, pi], bin width
    pi sqrt(2)/nbins, k = 0 excluded (bin -1).  Decided in FP64."""
    mx = np.arange(nx)
    my = np.arange(ny)
    mxw = np.where(mx > nx // 2, mx - nx, mx)
    myw = np.where(my > ny // 2, my - ny, my)
    KXw, KYw = np.meshgrid(2.0 * np.pi * mxw / nx, 2.0 * np.pi * myw / ny, indexing="xy")
    kmag = np.sqrt(KXw * KXw + KYw * KYw)
    width = np.pi * np.sqrt(2.0) / nbins
    b = np.floor(kmag / width).astype(np.int64)
    b = np.minimum(b, nbins - 1)
    b[0, 0] = -1
    return b, KXw, KYw, kmag


def spectra_sample(f: np.ndarray, rho0: float, nbins: int):
    """Per-bin sums of |drho(k)|^2, |j_l(k)|^2, |j_t(k)|^2 and the bin counts for one state
    (Eqs. struct-fact and momtm-fluct are the theories they estimate)."""
    _, ny, nx = f.shape
    rho = f.sum(axis=0)
    jx = np.einsum("i,iyx->yx", C[:, 0].astype(float), f)
    jy = np.einsum("i,iyx->yx", C[:, 1].astype(float), f)
    rk = unitary_ft(rho - rho0)
    jxk = unitary_ft(jx)
    jyk = unitary_ft(jy)
    b, KXw, KYw, kmag = k_bins(nx, ny, nbins)
    kk = np.where(kmag > 0, kmag, 1.0)
    jl = (KXw * jxk + KYw * jyk) / kk
    jt = (-KYw * jxk + KXw * jyk) / kk
    sel = b >= 0
    Srho = np.bincount(b[sel], weights=np.abs(rk[sel]) ** 2, minlength=nbins)
    Sjl = np.bincount(b[sel], weights=np.abs(jl[sel]) ** 2, minlength=nbins)
    Sjt = np.bincount(b[sel], weights=np.abs(jt[sel]) ** 2, minlength=nbins)
    cnt = np.bincount(b[sel], minlength=nbins)
    return Srho, Sjl, Sjt, cnt


def noise_at_sites(model: Model, mode: int, nx, ny, seed, step, sites, L0=None, xi49=None,
                   factor: str = "cholesky"):
    """xi[k, a] at the listed linear sites (same draws as noise_fields); for the
    correlated mode the (4, 9) fields over the whole lattice may be passed in xi49."""
    sites = np.asarray(sites, dtype=np.int64)
    xi = np.zeros((sites.size, 9))
    if mode == NOISE_OFF or model.kT == 0.0:
        return xi
    if L0 is None:
        X0 = model.Xi_zero()
        if mode == NOISE_DIAG:
            X0 = np.diag(np.diag(X0))
        L0 = theory.noise_factor(X0)
    idx = sites.astype(np.uint32)
    nu = np.zeros((9, sites.size))
    g0 = normals(idx, seed, step, TAG_NODE)
    nu[4:8] = g0[:, 0:4].T
    if mode in (NOISE_LW, NOISE_DIAG):
        nu[3] = g0[:, 4]
        nu[8] = g0[:, 5]
    xi[:] = (L0 @ nu).T
    if mode == NOISE_FULL:
        if xi49 is None:
            xi49 = xi49_full(model, nx, ny, seed, step, factor)
        x4, x9 = xi49
        xi[:, 3] = x4.ravel()[sites]
        xi[:, 8] = x9.ravel()[sites]
    elif mode == NOISE_FULL_RS:
        x49 = xi49_stencil_at(model, nx, ny, seed, step, sites, factor)
        xi[:, 3] = x49[:, 0]
        xi[:, 8] = x49[:, 1]
    return xi


def step_sampled(f: np.ndarray, model: Model, mode: int, seed: int, step: int, nodes, L0=None, xi49=None,
                 factor: str = "cholesky"):
    """Pre-collision populations f_i(r, t+1) = f*_i(r - c_i, t) at the listed nodes only,
    shape (len(nodes), 9); the collisions run at the nine source sites of each node."""
    _, ny, nx = f.shape
    nodes = np.asarray(nodes, dtype=np.int64)
    x = nodes % nx
    y = nodes // nx
    src = np.stack([((y - C[i, 1]) % ny) * nx + (x - C[i, 0]) % nx for i in range(9)], axis=1)
    sites, inv = np.unique(src.ravel(), return_inverse=True)
    xi = noise_at_sites(model, mode, nx, ny, seed, step, sites, L0, xi49, factor)
    fs = collide_sites(f, model, sites, xi)
    inv = inv.reshape(src.shape)
    return np.stack([fs[inv[:, i], i] for i in range(9)], axis=1)
