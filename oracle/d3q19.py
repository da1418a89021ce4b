"""FP64 CPU oracle of the fluctuating non-ideal model on the D3Q19 lattice.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers; the product library shares no code with it.

Sec. IV of Gross, Adhikari, Cates & Varnik (arXiv:1009.0254) states that the derivation of
the noise from the lattice fluctuation-dissipation theorem holds on any DdQn lattice.  This
module carries the D2Q9 model of the paper to D3Q19 with the same steps:

  * the weighted-orthogonal basis of Duenweg, Schiller & Ladd, Phys. Rev. E 76, 036704
    (2007), Table I (the D3Q19 modes); the D2Q9 basis of Table I of the paper is the
    two-dimensional member of that family;
  * the fluctuating collision of Eq. (fluct-lin-lbe) in moment space and the streaming of
    Eq. (gen-lbe), on a periodic box;
  * equilibrium moments that carry the pressure tensor of Eq. (press-ten) with
    p0 = cs2 rho (the linearised equation of state), Galilean corrections and forcing
    omitted as in the D2Q9 model;
  * the long-wavelength noise Xi(0) of Eq. (noise-matrix-k0), built from the equilibrium
    correlations of the ansatz Eq. (f-correl-yeo) and the linearised collision operator,
    then factored by Cholesky (Sec. IV).

Readings where the paper is silent (also listed in the design notes):
  * the second-order moments are the trace and the traceless part of P^th + rho u u
    (Eq. press-ten), so sum_i f^eq_i c_ia c_ib = P^th_ab + rho u_a u_b;
  * the ghost equilibria are zero except the isotropic fourth-order ghost,
    e16^eq = -3 (p0 - sigma_s^2 rho - kappa rho lap rho) - (9/2) kappa |grad rho|^2,
    the one isotropic choice for which a field that is uniform along one axis evolves,
    at equal relaxation times, exactly as the paper's D2Q9 model (Table II);
  * one bulk rate lambda_b for mode 4, one shear rate lambda_s for modes 5..9 and one
    ghost rate for modes 10..18;
  * the Laplacian and the gradient are the isotropic stencils of Appendix B written with
    the D3Q19 weights.

Indices: velocities and moments are array positions 0..18; f[i, z, y, x].
Random numbers: two Philox4x32-10 draws per node and step with counter (node, t mod 2^32,
t div 2^32, tag), node = (z ny + y) nx + x; tag 4 gives nu_4..nu_11, tag 5 gives
nu_12..nu_18 (its last normal unused), each word one Box-Muller pair as for D2Q9.

Two-phase model (Sec. II A; Sec. IV and Sec. V B): with a double-well ``eos``
(theory.DoubleWell) the second moments carry p0(rho) = rho f0'(rho) - f0(rho) of the Landau
free energy instead of cs2 rho, the uniform rest state is the equilibrium at rho0 with
p0(rho0), and the linear theory about rho0 (the noise of the homogeneous modes) takes
c_s^2 = rho0 f0''(rho0).  NOISE_LW_LOCAL draws the long-wavelength normals and scales them
at every node by the factor of Xi(0) of a homogeneous system at that node's density and
sound speed c_s^2(rho(r)) (the double well's, else cs2): Cholesky of the (4,16) block with a
negative pivot clamped to zero, where the local block is not positive semidefinite.

Correlated noise (Sec. III C, Eq. noise-matrix at every k): with the ansatz the advection
drops out of the fluctuation-dissipation relation (A(k) G(k) A(-k)^T = G(k), the phases of
a diagonal matrix cancel), so Xi(k) is the long-wavelength form at c_s^2(k) = cs2 + rho0
kappa s(k), s the Laplacian symbol; only the (4,16) block depends on k, affinely in s.  s is
multilinear in (cos kx, cos ky, cos kz), so Xi(k) is the multilinear interpolation of its
values at the eight corners k in {0, pi}^3 (s = 0, 4, 16/3, 4 for 0..3 components at pi):
eight white 2-vector fields nu_abc per node (a, b, c = +-1; + for k = 0), each times the
Cholesky factor of the (4,16) block at its corner, combined as
h_d(r) = (1/8) sum_abc a^dx b^dy c^dz L_abc nu_abc(r) and summed over the 2x2x2 box,
xi(r) = sum_d h_d(r - d), give (xi_4, xi_16) with covariance Xi(k) at every k.  Their draws:
tags 10 and 11, word w of the pair -> corner w = 4 ia + 2 ib + ic (sign +1 for index 0).
"""
from __future__ import annotations

import numpy as np

from . import normals
from .theory import cholesky_psd

SIGMA_S2 = 1.0 / 3.0
TAG_A, TAG_B = 4, 5


def _velocities() -> np.ndarray:
    """Rest, the six faces (+x, -x, +y, -y, +z, -z), then the twelve edges in the (x,y),
    (y,z), (z,x) planes with signs (++, +-, -+, --)."""
    c = [(0, 0, 0)]
    for a in range(3):
        for s in (1, -1):
            v = [0, 0, 0]
            v[a] = s
            c.append(tuple(v))
    for a, b in ((0, 1), (1, 2), (2, 0)):
        for s in (1, -1):
            for t in (1, -1):
                v = [0, 0, 0]
                v[a], v[b] = s, t
                c.append(tuple(v))
    return np.array(c, dtype=np.int64)


#: D3Q19 velocities c_i.
C = _velocities()
#: Weights 1/3 (rest), 1/18 (faces), 1/36 (edges).
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
Q = 19
#: opposite direction: C[OPP[i]] = -C[i]
OPP = np.array([int(np.where((C == -C[i]).all(axis=1))[0][0]) for i in range(Q)])


def basis_T() -> np.ndarray:
    """The nineteen mode polynomials (Duenweg, Schiller & Ladd 2007, Table I) on C:
    rho; j; the bulk mode c^2 - 1; five shear modes; six third-order ghosts; three
    fourth-order ghosts."""
    cx, cy, cz = (C[:, k].astype(np.float64) for k in range(3))
    c2 = cx * cx + cy * cy + cz * cz
    rows = [
        np.ones(Q), cx, cy, cz,                          # 0: rho, 1..3: j
        c2 - 1,                                          # 4: bulk
        3 * cx * cx - c2, cy * cy - cz * cz,             # 5, 6: shear, diagonal
        cx * cy, cy * cz, cz * cx,                       # 7..9: shear, off-diagonal
        (3 * c2 - 5) * cx, (3 * c2 - 5) * cy, (3 * c2 - 5) * cz,        # 10..12
        (cy * cy - cz * cz) * cx, (cz * cz - cx * cx) * cy, (cx * cx - cy * cy) * cz,  # 13..15
        3 * c2 * c2 - 6 * c2 + 1,                        # 16: isotropic fourth order
        (2 * c2 - 3) * (3 * cx * cx - c2), (2 * c2 - 3) * (cy * cy - cz * cz),    # 17, 18
    ]
    return np.array(rows)


T = basis_T()
#: N_a = sum_i w_i T_ai^2 (the scalar product of Eq. scalar-prod with the D3Q19 weights).
N = (T * T * W[None, :]).sum(axis=1)
#: (T^-1)_ia = w_i T_ai / N_a.
TINV = (W[:, None] * T.T) / N[None, :]


def lambdas(tau_s: float, tau_b: float, tau_ghost: float) -> np.ndarray:
    """lambda_a = -1/tau: 0 for the conserved modes, bulk, five shear, nine ghosts."""
    return np.array([0.0] * 4 + [-1.0 / tau_b] + [-1.0 / tau_s] * 5 + [-1.0 / tau_ghost] * 9)


class Model:
    """One homogeneous run on D3Q19: rho0, cs2 (p0 = cs2 rho, or the c_s^2 of the linear
    theory about rho0), kappa, kT, relaxation times; p0_rest the bulk pressure of the uniform
    rest state (cs2 rho0 unless given: p0(rho0) of a double well)."""

    def __init__(self, rho0=1.0, cs2=SIGMA_S2, kappa=0.0, kT=0.0, tau_s=1.0, tau_b=1.0, tau_ghost=1.0,
                 p0_rest=None):
        self.rho0, self.cs2, self.kappa, self.kT = float(rho0), float(cs2), float(kappa), float(kT)
        self.p0_rest = self.cs2 * self.rho0 if p0_rest is None else float(p0_rest)
        self.tau_s, self.tau_b, self.tau_ghost = float(tau_s), float(tau_b), float(tau_ghost)
        self.lam = lambdas(tau_s, tau_b, tau_ghost)

    def d(self) -> float:
        """Weight of the pressure deviation in the rest moments: 3 (cs2 - sigma_s^2)."""
        return 3.0 * (self.cs2 - SIGMA_S2)

    def mbar(self) -> np.ndarray:
        """Rest moments: rho0, e4 = d rho0, e16 = -d rho0 (the equilibrium at u = 0 and
        uniform density), the rest zero."""
        m = np.zeros(Q)
        m[0] = self.rho0
        m[4] = self.d() * self.rho0
        m[16] = -self.d() * self.rho0
        return m

    def fbar(self) -> np.ndarray:
        return TINV @ self.mbar()

    def rest(self) -> np.ndarray:
        """Populations of the uniform rest state at rho0: the equilibrium at u = 0 with bulk
        pressure p0_rest, e4 = 3 p0 - rho0 and e16 = -e4 (fbar() for p0 = cs2 rho)."""
        m = np.zeros(Q)
        m[0] = self.rho0
        m[4] = 3.0 * (self.p0_rest - SIGMA_S2 * self.rho0)
        m[16] = -m[4]
        return TINV @ m

    def Omega0(self) -> np.ndarray:
        """Linearised collision operator at k = 0 (the analogue of Eq. coll-op-yeo): mode a
        relaxes at lambda_a towards its equilibrium, which for e4 and e16 follows the
        density through p0 = cs2 rho."""
        O = np.diag(self.lam)
        O[4, 0] = -self.lam[4] * self.d()
        O[16, 0] = self.lam[16] * self.d()
        return O

    def G0(self) -> np.ndarray:
        """Equal-time mode correlations of the ansatz <df_i df_j> = (S/rho0) fbar_i delta_ij,
        Eq. (f-correl-yeo), at k = 0 with S = rho0 kT / cs2 (Eq. struct-fact)."""
        S = self.rho0 * self.kT / self.cs2
        return (S / self.rho0) * (T @ np.diag(self.fbar()) @ T.T)

    def Xi_zero(self) -> np.ndarray:
        """Xi(0) = -G Omega^T - Omega G - Omega G Omega^T, Eq. (noise-matrix-k0)."""
        G, O = self.G0(), self.Omega0()
        return -G @ O.T - O @ G - O @ G @ O.T

    def noise_factor(self) -> np.ndarray:
        """19x19 L with L L^T = Xi(0): Cholesky of the block of the non-conserved modes
        4..18 (Sec. IV), rows 0..3 zero."""
        L = np.zeros((Q, Q))
        L[4:, 4:] = cholesky_psd(self.Xi_zero()[4:, 4:])
        return L


# --- the step -------------------------------------------------------------------------

def _shift(a: np.ndarray, c) -> np.ndarray:
    """b(r) = a(r + c) on the periodic box, a[z, y, x]."""
    return np.roll(a, shift=(-int(c[2]), -int(c[1]), -int(c[0])), axis=(0, 1, 2))


def density_stencils(rho: np.ndarray):
    """Laplacian sum_{i != 0} w_i [rho(r + c_i) + rho(r - c_i) - 2 rho(r)] / sigma_s^2 and the
    gradient 3 sum_i w_i c_i rho(r + c_i) (Appendix B's isotropic stencils, D3Q19 weights)."""
    lap = np.zeros_like(rho)
    grad = np.zeros((3,) + rho.shape)
    for i in range(1, Q):
        ri = _shift(rho, C[i])
        lap += W[i] * (ri + _shift(rho, C[OPP[i]]) - 2.0 * rho) / SIGMA_S2
        for k in range(3):
            grad[k] += 3.0 * W[i] * C[i, k] * ri
    return lap, grad


def equilibrium_moments(rho, j, lap, grad, cs2, kappa, p0=None) -> np.ndarray:
    """m^eq[a, ...] for each node: rho, j, then the second-order moments of
    P^th_ab + rho u_a u_b with P^th of Eq. (press-ten) for the bulk pressure p0 (cs2 rho
    unless given),
        P^th_ab = (p0 - kappa rho lap rho - kappa |grad rho|^2 / 2) delta_ab
                  + kappa d_a rho d_b rho,
    and the fourth-order ghost e16 of the module's reading; the other ghosts zero."""
    u = j / rho
    if p0 is None:
        p0 = cs2 * rho
    P = np.zeros((3, 3) + rho.shape)
    g2 = (grad * grad).sum(axis=0)
    piso = p0 - kappa * rho * lap - 0.5 * kappa * g2
    for a in range(3):
        for b in range(3):
            P[a, b] = rho * u[a] * u[b] + kappa * grad[a] * grad[b]
        P[a, a] = P[a, a] + piso
    m = np.zeros((Q,) + rho.shape)
    m[0] = rho
    m[1:4] = j
    m[4] = P[0, 0] + P[1, 1] + P[2, 2] - rho
    m[5] = 2 * P[0, 0] - P[1, 1] - P[2, 2]
    m[6] = P[1, 1] - P[2, 2]
    m[7], m[8], m[9] = P[0, 1], P[1, 2], P[2, 0]
    m[16] = -3.0 * (p0 - SIGMA_S2 * rho - kappa * rho * lap) - 4.5 * kappa * g2
    return m


def collide(f: np.ndarray, model: Model, xi=None, eos=None) -> np.ndarray:
    """Post-collision populations f*_i = (T^-1 m*)_i with
    m*_a = m_a + lambda_a (m_a - m^eq_a) + xi_a, Eq. (fluct-lin-lbe); eos: a double well
    whose p0(rho) replaces cs2 rho in the equilibrium."""
    m = np.einsum("ai,i...->a...", T, f)
    rho = m[0]
    lap, grad = density_stencils(rho)
    p0 = None if eos is None else eos.p0(rho)
    meq = equilibrium_moments(rho, m[1:4], lap, grad, model.cs2, model.kappa, p0)
    ms = m + model.lam[:, None, None, None] * (m - meq)
    if xi is not None:
        ms = ms + xi
    return np.einsum("ia,a...->i...", TINV, ms)


def stream(fs: np.ndarray) -> np.ndarray:
    """f_i(r + c_i, t + 1) = f*_i(r, t), Eq. (gen-lbe), periodic."""
    out = np.empty_like(fs)
    for i in range(Q):
        out[i] = np.roll(fs[i], shift=(int(C[i, 2]), int(C[i, 1]), int(C[i, 0])), axis=(0, 1, 2))
    return out


def step(f: np.ndarray, model: Model, xi=None, eos=None) -> np.ndarray:
    return stream(collide(f, model, xi, eos))


# --- noise of Sec. IV -------------------------------------------------------------------

def noise_normals(nx, ny, nz, seed: int, step_index: int) -> np.ndarray:
    """nu[a, z, y, x] for a = 4..18 (rows 0..3 zero): the counter layout of the module
    docstring."""
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.uint32)
    ga = normals(idx, seed, step_index, TAG_A)
    gb = normals(idx, seed, step_index, TAG_B)
    nu = np.zeros((Q, n))
    nu[4:12] = ga.T
    nu[12:19] = gb[:, :7].T
    return nu.reshape(Q, nz, ny, nx)


def noise_lw_nodes(model: Model, nodes: np.ndarray, seed: int, step_index: int, L=None) -> np.ndarray:
    """xi[a, ...] = L nu at the given global node indices (any shape): the draws of
    noise_normals() for those nodes."""
    if L is None:
        L = model.noise_factor()
    idx = np.ascontiguousarray(nodes, dtype=np.uint32).ravel()
    ga = normals(idx, seed, step_index, TAG_A)
    gb = normals(idx, seed, step_index, TAG_B)
    nu = np.zeros((Q, idx.size))
    nu[4:12] = ga.T
    nu[12:19] = gb[:, :7].T
    return (L @ nu).reshape((Q,) + np.shape(nodes))


def noise_lw(model: Model, nx, ny, nz, seed: int, step_index: int, L=None) -> np.ndarray:
    """xi = L nu with L L^T = Xi(0), independently at every node."""
    if L is None:
        L = model.noise_factor()
    nu = noise_normals(nx, ny, nz, seed, step_index)
    return np.einsum("ab,b...->a...", L, nu)


def local_factor(X: np.ndarray, coupled) -> np.ndarray:
    """Q x Q factor of one node's Xi(0) for the local noise: Cholesky of the coupled block
    (in mode order) in which a pivot below zero is clamped to zero and a zero pivot leaves
    its column zero; the square roots of the other non-conserved modes' variances."""
    L = np.zeros((Q, Q))
    n = len(coupled)
    B = np.zeros((n, n))
    for j in range(n):
        s = X[coupled[j], coupled[j]] - np.dot(B[j, :j], B[j, :j])
        B[j, j] = np.sqrt(max(s, 0.0))
        for i in range(j + 1, n):
            t = X[coupled[i], coupled[j]] - np.dot(B[i, :j], B[j, :j])
            B[i, j] = t / B[j, j] if B[j, j] > 0 else 0.0
    L[np.ix_(coupled, coupled)] = B
    for a in range(4, Q):
        if a not in coupled:
            L[a, a] = np.sqrt(max(X[a, a], 0.0))
    return L


COUPLED = [4, 16]


def noise_lw_local(model: Model, rho: np.ndarray, c2, seed: int, step_index: int) -> np.ndarray:
    """xi[a, z, y, x] of NOISE_LW_LOCAL: the long-wavelength normals, at every node times the
    local factor of Xi(0) of a homogeneous system at that node's density rho(r) and sound
    speed c2(r) (the model's kappa, kT and relaxation times)."""
    nz, ny, nx = rho.shape
    nu = noise_normals(nx, ny, nz, seed, step_index).reshape(Q, -1)
    r = rho.ravel()
    c = np.broadcast_to(np.asarray(c2, dtype=np.float64), rho.shape).ravel()
    xi = np.zeros((Q, r.size))
    for n in range(r.size):
        X = Model(r[n], c[n], model.kappa, model.kT, model.tau_s, model.tau_b, model.tau_ghost).Xi_zero()
        xi[:, n] = local_factor(X, COUPLED) @ nu[:, n]
    return xi.reshape(Q, nz, ny, nx)


# --- correlated noise (Sec. III C, Eq. noise-matrix) ------------------------------------------

TAG_RS = (10, 11)


def lattice_s(kx, ky, kz):
    """Symbol of the Laplacian stencil: -lap e^{ik.r} = s(k) e^{ik.r},
    s = 6 sum_{i != 0} w_i (1 - cos k.c_i)."""
    kv = np.stack(np.broadcast_arrays(np.asarray(kx, float), np.asarray(ky, float), np.asarray(kz, float)), axis=-1)
    return 6.0 * sum(W[i] * (1.0 - np.cos(kv @ C[i].astype(float))) for i in range(1, Q))


def Xi_k(model: Model, kx, ky, kz) -> np.ndarray:
    """Xi(k) = A(k) G(k) A(-k)^T - (1 + Omega(k)) G(k) (1 + Omega(k))^T, Eq. (noise-matrix), with
    G(k) the ansatz (S(k)/rho0) T diag(fbar(k)) T^T and the density dependence of the
    equilibrium through c_s^2(k) = cs2 + rho0 kappa s(k) (Eq. sound-speed-k)."""
    c2k = model.cs2 + model.rho0 * model.kappa * float(lattice_s(kx, ky, kz))
    dk = 3.0 * (c2k - SIGMA_S2)
    mb = np.zeros(Q)
    mb[0] = model.rho0
    mb[4], mb[16] = dk * model.rho0, -dk * model.rho0
    G = (model.kT / c2k) * (T @ np.diag(TINV @ mb) @ T.T)
    O = np.diag(model.lam).astype(complex)
    O[4, 0] = -model.lam[4] * dk
    O[16, 0] = model.lam[16] * dk
    ph = np.exp(-1j * (C.astype(float) @ np.array([kx, ky, kz], dtype=float)))
    A = T @ np.diag(ph) @ TINV
    Am = T @ np.diag(np.conj(ph)) @ TINV
    IO = np.eye(Q) + O
    X = A @ G @ Am.T - IO @ G @ IO.T
    return X.real


CORNERS = [(1 if (w >> 2) & 1 == 0 else -1, 1 if (w >> 1) & 1 == 0 else -1, 1 if w & 1 == 0 else -1)
           for w in range(8)]


def rs_factors(model: Model) -> np.ndarray:
    """2x2 Cholesky factors of the (4,16) block of Xi at the eight corners (sign +1: k = 0)."""
    out = np.zeros((8, 2, 2))
    for w, (a, b, c) in enumerate(CORNERS):
        k = [0.0 if v > 0 else np.pi for v in (a, b, c)]
        X = Xi_k(model, *k)
        out[w] = cholesky_psd(np.array([[X[4, 4], X[4, 16]], [X[16, 4], X[16, 16]]]))
    return out


def rs_fields(nx, ny, nz, seed: int, step_index: int) -> np.ndarray:
    """nu[w, 2, z, y, x]: the white 2-vector of corner w at every node."""
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.uint32)
    g = np.concatenate([normals(idx, seed, step_index, t) for t in TAG_RS], axis=1)     # (n, 16)
    return g.T.reshape(8, 2, nz, ny, nx)


def xi416_rs(model: Model, nx, ny, nz, seed: int, step_index: int, Ls=None) -> np.ndarray:
    """(xi_4, xi_16)[2, z, y, x] of the real-space construction (module docstring)."""
    if Ls is None:
        Ls = rs_factors(model)
    nu = rs_fields(nx, ny, nz, seed, step_index)
    v = np.einsum("wab,wb...->wa...", Ls, nu)                 # L_abc nu_abc
    out = np.zeros((2, nz, ny, nx))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                h = sum((CORNERS[w][0] ** dx) * (CORNERS[w][1] ** dy) * (CORNERS[w][2] ** dz) * v[w]
                        for w in range(8)) / 8.0
                out += np.roll(h, shift=(dz, dy, dx), axis=(1, 2, 3))      # h_d(r - d)
    return out


NOISE_OFF, NOISE_LW, NOISE_FULL_RS, NOISE_LW_LOCAL = 0, 1, 4, 5


class Lattice:
    """A periodic nx x ny x nz D3Q19 lattice: f[19, nz, ny, nx] pre-collision populations,
    t the index of the next collision (it keys the random numbers).  Noise: NOISE_LW (Xi(0)),
    NOISE_FULL_RS (Xi(k), the (4,16) block built in real space, the other modes as LW) or
    NOISE_LW_LOCAL (Xi(0) at each node's density and sound speed).  ``eos`` (a
    theory.DoubleWell) replaces p0 = cs2 rho by the double well's bulk pressure; the rest
    state and the linear theory about rho0 then take p0(rho0) and c_s^2(rho0)."""

    def __init__(self, nx, ny, nz, rho0=1.0, cs2=SIGMA_S2, seed=42, eos=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.seed = int(seed)
        self.eos = eos
        if eos is None:
            self.model = Model(rho0=rho0, cs2=cs2)
        else:
            self.model = Model(rho0=rho0, cs2=eos.cs2(rho0), p0_rest=eos.p0(rho0))
        self.mode = NOISE_OFF
        self.t = 0
        self.f = np.broadcast_to(self.model.rest()[:, None, None, None], (Q, nz, ny, nx)).copy()
        self._L = None
        self._Ls = None

    def set_params(self, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode):
        m = self.model
        self.model = Model(m.rho0, m.cs2, kappa, kT, tau_s, tau_b, tau_ghost, m.p0_rest)
        self.mode = int(noise_mode)
        noisy = self.mode in (NOISE_LW, NOISE_FULL_RS) and kT > 0
        self._L = self.model.noise_factor() if noisy else None
        self._Ls = rs_factors(self.model) if (noisy and self.mode == NOISE_FULL_RS) else None

    def noise(self, t=None):
        t = self.t if t is None else t
        xi = noise_lw(self.model, self.nx, self.ny, self.nz, self.seed, t, self._L)
        if self._Ls is not None:
            xi[[4, 16]] = xi416_rs(self.model, self.nx, self.ny, self.nz, self.seed, t, self._Ls)
        return xi

    def step(self, nsteps=1):
        for _ in range(int(nsteps)):
            xi = None
            if self._L is not None:
                xi = self.noise()
            elif self.mode == NOISE_LW_LOCAL and self.model.kT > 0:
                rho = self.f.sum(axis=0)
                c2 = self.model.cs2 if self.eos is None else self.eos.cs2(rho)
                xi = noise_lw_local(self.model, rho, c2, self.seed, self.t)
            self.f = step(self.f, self.model, xi, self.eos)
            self.t += 1
        return self

    def moments(self) -> np.ndarray:
        return np.einsum("ai,i...->a...", T, self.f)
