"""FP64 CPU oracle of the fluctuating non-ideal model on the D3Q27 lattice.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers; the product library shares no code with it.

Sec. IV of Gross, Adhikari, Cates & Varnik (arXiv:1009.0254) states that the noise
derivation holds on any DdQn lattice.  This module carries the D2Q9 model of the paper to
D3Q27 with the steps of ``oracle.d3q19``:

  * the basis: products p_a(c_x) p_b(c_y) p_c(c_z) of the polynomials p_0 = 1, p_1 = c,
    p_2 = 3c^2 - 1, orthogonal under the D1Q3 weights (2/3, 1/6, 1/6) whose products are the
    D3Q27 weights; the c_z-independent members (p_a(c_x) p_b(c_y)) span the D2Q9 basis of
    the paper's Table I (e = p_2x + p_2y, p_ww = (p_2x - p_2y)/3, q_x = p_1x p_2y, eps =
    2 p_2x p_2y, ...), so the paper's basis is the two-dimensional member of this family;
  * the fluctuating collision of Eq. (fluct-lin-lbe): the bulk mode p_2x + p_2y + p_2z
    relaxes at lambda_b, the traceless second-order modes at lambda_s, all higher modes
    at one ghost rate;
  * the pressure tensor of Eq. (press-ten) with p0 = cs2 rho in the second moments;
  * the long-wavelength noise Xi(0) of Eq. (noise-matrix-k0) from the ansatz Eq.
    (f-correl-yeo), factored by Cholesky (Sec. IV).

Readings where the paper is silent (also listed in the design notes):
  * second moments: sum_i f^eq_i c_ia c_ib = P^th_ab + rho u_a u_b (as for D3Q19);
  * ghost equilibria are those of the equilibrium that carries the pressure on the moving
    velocities (w_i [3 p + 3 c.j + (9/2)(rho uu + kappa grad rho grad rho):cc
    - (3/2)(rho u^2 + kappa |grad rho|^2)], the remainder at rest), except the three
    fourth-order modes p_2a p_2b (a != b), which take Table II's correction:
    m^eq(p_2a p_2b) = -3 (p0 - rho/3 - kappa rho lap rho) - (3/2) kappa |grad rho|^2, so that
    a field uniform and mirror-symmetric along one axis evolves, at equal relaxation times,
    as the D2Q9 model of Table II; the sixth-order mode has
    m^eq(p_2x p_2y p_2z) = 3 (p0 - rho/3 - kappa rho lap rho) - (3/2) kappa |grad rho|^2 and
    every other ghost equilibrium is zero;
  * the Laplacian and gradient are Appendix B's isotropic stencils with the D3Q27 weights.

Two-phase model (Sec. II A; Sec. IV and Sec. V B), as ``oracle.d3q19``: a double-well
``eos`` puts p0(rho) of the Landau free energy in the second moments and the ghost
equilibria, the rest state takes p0(rho0) and the linear theory c_s^2(rho0); NOISE_LW_LOCAL
scales the long-wavelength normals at every node by the factor of Xi(0) at that node's
density and sound speed (Cholesky of the seven coupled modes with negative pivots clamped
to zero, square roots of the other variances).

Correlated noise (Sec. III C, Eq. noise-matrix at every k), as ``oracle.d3q19``: with the
ansatz the advection drops out of the fluctuation-dissipation relation, so Xi(k) is Xi(0) at
c_s^2(k) = cs2 + rho0 kappa s(k), s the symbol of the D3Q27 Laplacian,
s = 6 (1 - prod_a (2 + cos k_a) / 3), which is multilinear in the three cosines; Xi(0) is
affine in c_s^2 and only its seven coupled modes depend on it: their block is
X(k) = X0 + s(k) D, X0 the block at k = 0 and D its slope (rho0 kappa times the slope of
Xi(0) in c_s^2), of rank two with one positive and one negative eigenvalue.  With S = 52/9
the largest s (k = (pi, pi, pi)) and D = p p^T - q q^T,

    X(k) = C + s(k) p p^T + (S - s(k)) q q^T,    C = X0 - S q q^T,

so the coupled noise is C^(1/2) nu (white) plus p phi_p + q phi_q, two scalar fields whose
spectra s(k) and S - s(k) are, like s, multilinear in the cosines: the multilinear
interpolation of their corner values (s = 0, 4, 16/3, 52/9 at 0..3 components at pi).  A
field with corner values sigma_w is built from eight white scalar fields nu_w per node
(w = 4 ia + 2 ib + ic, a set bit for a component at pi) as h_d = (1/8) sum_w
(-1)^{popcount(w & d)} sqrt(sigma_w) nu_w, summed over the 2x2x2 box: phi(r) = sum_d h_d(r - d).
Of the splits p, q of D the one that whitens X0 (eigenvectors of L0^-1 D L0^-T, X0 = L0 L0^T)
makes C positive semidefinite exactly when X at k = (pi, pi, pi) is, which with X0 positive
definite is the condition for Xi(k) at every k.  The white part uses the long-wavelength
normals of the coupled modes (their factor becomes that of C); the other modes keep the
long-wavelength noise.  Draws: tags 12 and 13, word w (in tag order) gives the pair
(nu_w of phi_p, nu_w of phi_q) of corner w.

Indices: velocity i = 9 ix + 3 iy + iz with c = (v[ix], v[iy], v[iz]), v = (0, 1, -1); mode
a = 9 ax + 3 ay + az for p_ax(c_x) p_ay(c_y) p_az(c_z).  f[i, z, y, x].
Random numbers: three Philox4x32-10 draws per node and step with counter (node, t mod 2^32,
t div 2^32, tag), node = (z ny + y) nx + x, tags 6, 7, 8; their 24 normals in order go to the
23 non-conserved modes in increasing mode index (the last normal unused).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import normals
from .theory import cholesky_psd

SIGMA_S2 = 1.0 / 3.0
Q = 27
TAGS = (6, 7, 8)
_V = (0, 1, -1)

#: velocities c_i, i = 9 ix + 3 iy + iz
C = np.array([(_V[a], _V[b], _V[c]) for a, b, c in itertools.product(range(3), repeat=3)], dtype=np.int64)
_W1 = {0: 2 / 3, 1: 1 / 6, -1: 1 / 6}
#: weights: products of the D1Q3 weights (8/27, 2/27, 1/54, 1/216)
W = np.array([_W1[int(a)] * _W1[int(b)] * _W1[int(c)] for a, b, c in C])
OPP = np.array([int(np.where((C == -C[i]).all(axis=1))[0][0]) for i in range(Q)])
#: mode labels (ax, ay, az)
MODES = list(itertools.product(range(3), repeat=3))
IDX = {m: k for k, m in enumerate(MODES)}
CONSERVED = [IDX[(0, 0, 0)], IDX[(1, 0, 0)], IDX[(0, 1, 0)], IDX[(0, 0, 1)]]
SECOND_DIAG = [IDX[(2, 0, 0)], IDX[(0, 2, 0)], IDX[(0, 0, 2)]]
SECOND_OFF = [IDX[(1, 1, 0)], IDX[(0, 1, 1)], IDX[(1, 0, 1)]]
FOURTH_PAIR = [IDX[(2, 2, 0)], IDX[(0, 2, 2)], IDX[(2, 0, 2)]]
SIXTH = IDX[(2, 2, 2)]
NONCONSERVED = [k for k in range(Q) if k not in CONSERVED]


def _p(a, c):
    c = c.astype(np.float64)
    return np.ones_like(c) if a == 0 else (c if a == 1 else 3 * c * c - 1)


def basis_T() -> np.ndarray:
    """T_ai = p_ax(c_ix) p_ay(c_iy) p_az(c_iz)."""
    return np.array([_p(a, C[:, 0]) * _p(b, C[:, 1]) * _p(c, C[:, 2]) for a, b, c in MODES])


T = basis_T()
N = (T * T * W[None, :]).sum(axis=1)
TINV = (W[:, None] * T.T) / N[None, :]


def relaxation_matrix(tau_s, tau_b, tau_ghost) -> np.ndarray:
    """Lambda with m* = m + Lambda (m - m^eq) + xi: lambda_b on the bulk direction (1, 1, 1)/3
    of the three p_2a modes, lambda_s on its traceless complement and on p_1a p_1b, the ghost
    rate on every mode above second order, zero on the conserved modes."""
    lb, ls, lg = -1.0 / tau_b, -1.0 / tau_s, -1.0 / tau_ghost
    L = np.zeros((Q, Q))
    for k in range(Q):
        if k in CONSERVED:
            continue
        L[k, k] = lg
    for k in SECOND_OFF:
        L[k, k] = ls
    for a in SECOND_DIAG:
        for b in SECOND_DIAG:
            L[a, b] = (lb - ls) / 3.0 + (ls if a == b else 0.0)
    return L


class Model:
    """One homogeneous run on D3Q27: rho0, cs2 (p0 = cs2 rho, or the c_s^2 of the linear
    theory about rho0), kappa, kT, relaxation times; p0_rest the bulk pressure of the uniform
    rest state (cs2 rho0 unless given)."""

    def __init__(self, rho0=1.0, cs2=SIGMA_S2, kappa=0.0, kT=0.0, tau_s=1.0, tau_b=1.0, tau_ghost=1.0,
                 p0_rest=None):
        self.rho0, self.cs2, self.kappa, self.kT = float(rho0), float(cs2), float(kappa), float(kT)
        self.p0_rest = self.cs2 * self.rho0 if p0_rest is None else float(p0_rest)
        self.tau_s, self.tau_b, self.tau_ghost = float(tau_s), float(tau_b), float(tau_ghost)
        self.Lam = relaxation_matrix(tau_s, tau_b, tau_ghost)

    def d(self) -> float:
        return 3.0 * (self.cs2 - SIGMA_S2)

    def mbar(self) -> np.ndarray:
        """Rest moments: the equilibrium at u = 0 and uniform rho0."""
        m = np.zeros(Q)
        m[IDX[(0, 0, 0)]] = self.rho0
        d = self.d() * self.rho0
        for k in SECOND_DIAG:
            m[k] = d
        for k in FOURTH_PAIR:
            m[k] = -d
        m[SIXTH] = d
        return m

    def fbar(self) -> np.ndarray:
        return TINV @ self.mbar()

    def rest(self) -> np.ndarray:
        """Populations of the uniform rest state at rho0 with bulk pressure p0_rest (fbar()
        for p0 = cs2 rho)."""
        m = np.zeros(Q)
        m[IDX[(0, 0, 0)]] = self.rho0
        d = 3.0 * (self.p0_rest - SIGMA_S2 * self.rho0)
        for k in SECOND_DIAG:
            m[k] = d
        for k in FOURTH_PAIR:
            m[k] = -d
        m[SIXTH] = d
        return TINV @ m

    def J0(self) -> np.ndarray:
        """d m^eq / d m at the rest state (only the density column is non-zero beyond the
        conserved modes)."""
        J = np.zeros((Q, Q))
        for k in CONSERVED:
            J[k, k] = 1.0
        d = self.d()
        for k in SECOND_DIAG:
            J[k, 0] = d
        for k in FOURTH_PAIR:
            J[k, 0] = -d
        J[SIXTH, 0] = d
        return J

    def Omega0(self) -> np.ndarray:
        """Linearised collision at k = 0: Omega = Lambda (I - J0)."""
        return self.Lam @ (np.eye(Q) - self.J0())

    def G0(self) -> np.ndarray:
        """(S/rho0) T diag(fbar) T^T with S = rho0 kT / cs2 (Eqs. f-correl-yeo, struct-fact)."""
        S = self.rho0 * self.kT / self.cs2
        return (S / self.rho0) * (T @ np.diag(self.fbar()) @ T.T)

    def Xi_zero(self) -> np.ndarray:
        """Xi(0) = -G Omega^T - Omega G - Omega G Omega^T, Eq. (noise-matrix-k0)."""
        G, O = self.G0(), self.Omega0()
        return -G @ O.T - O @ G - O @ G @ O.T

    def noise_factor(self) -> np.ndarray:
        """27 x 27 L, L L^T = Xi(0): Cholesky of the non-conserved block in mode order."""
        L = np.zeros((Q, Q))
        nc = NONCONSERVED
        L[np.ix_(nc, nc)] = cholesky_psd(self.Xi_zero()[np.ix_(nc, nc)])
        return L


# --- the step -------------------------------------------------------------------------------

def _shift(a, c):
    return np.roll(a, shift=(-int(c[2]), -int(c[1]), -int(c[0])), axis=(0, 1, 2))


def density_stencils(rho):
    """Appendix B's Laplacian and the isotropic gradient with the D3Q27 weights."""
    lap = np.zeros_like(rho)
    grad = np.zeros((3,) + rho.shape)
    for i in range(1, Q):
        ri = _shift(rho, C[i])
        lap += W[i] * (ri + _shift(rho, C[OPP[i]]) - 2.0 * rho) / SIGMA_S2
        for k in range(3):
            grad[k] += 3.0 * W[i] * C[i, k] * ri
    return lap, grad


def equilibrium_moments(rho, j, lap, grad, cs2, kappa, p0=None) -> np.ndarray:
    """m^eq[a, ...]: rho, j, the second-order modes of P^th + rho u u (Eq. press-ten with
    the bulk pressure p0, cs2 rho unless given), and the fourth- and sixth-order ghosts of
    the module's reading."""
    u = j / rho
    if p0 is None:
        p0 = cs2 * rho
    g2 = (grad * grad).sum(axis=0)
    piso = p0 - kappa * rho * lap - 0.5 * kappa * g2
    Pi = np.zeros((3, 3) + rho.shape)
    for a in range(3):
        for b in range(3):
            Pi[a, b] = rho * u[a] * u[b] + kappa * grad[a] * grad[b]
        Pi[a, a] = Pi[a, a] + piso
    iso = p0 - SIGMA_S2 * rho - kappa * rho * lap
    m = np.zeros((Q,) + rho.shape)
    m[IDX[(0, 0, 0)]] = rho
    m[IDX[(1, 0, 0)]], m[IDX[(0, 1, 0)]], m[IDX[(0, 0, 1)]] = j[0], j[1], j[2]
    for a, k in enumerate(SECOND_DIAG):               # sum_i f_i (3 c_a^2 - 1) = 3 Pi_aa - rho
        m[k] = 3.0 * Pi[a, a] - rho
    m[IDX[(1, 1, 0)]], m[IDX[(0, 1, 1)]], m[IDX[(1, 0, 1)]] = Pi[0, 1], Pi[1, 2], Pi[0, 2]
    for k in FOURTH_PAIR:
        m[k] = -3.0 * iso - 1.5 * kappa * g2
    m[SIXTH] = 3.0 * iso - 1.5 * kappa * g2
    return m


def collide(f, model: Model, xi=None, eos=None):
    m = np.einsum("ai,i...->a...", T, f)
    rho = m[0]
    lap, grad = density_stencils(rho)
    j = np.array([m[IDX[(1, 0, 0)]], m[IDX[(0, 1, 0)]], m[IDX[(0, 0, 1)]]])
    p0 = None if eos is None else eos.p0(rho)
    meq = equilibrium_moments(rho, j, lap, grad, model.cs2, model.kappa, p0)
    ms = m + np.einsum("ab,b...->a...", model.Lam, m - meq)
    if xi is not None:
        ms = ms + xi
    return np.einsum("ia,a...->i...", TINV, ms)


def stream(fs):
    out = np.empty_like(fs)
    for i in range(Q):
        out[i] = np.roll(fs[i], shift=(int(C[i, 2]), int(C[i, 1]), int(C[i, 0])), axis=(0, 1, 2))
    return out


def step(f, model: Model, xi=None, eos=None):
    return stream(collide(f, model, xi, eos))


# --- noise of Sec. IV ---------------------------------------------------------------------

def noise_lw_nodes(model: Model, nodes, seed: int, step_index: int, L=None) -> np.ndarray:
    """xi[a, ...] = L nu at the given global node indices."""
    if L is None:
        L = model.noise_factor()
    idx = np.ascontiguousarray(nodes, dtype=np.uint32).ravel()
    g = np.concatenate([normals(idx, seed, step_index, t) for t in TAGS], axis=1)     # (n, 24)
    nu = np.zeros((Q, idx.size))
    nu[NONCONSERVED] = g[:, :len(NONCONSERVED)].T
    return (L @ nu).reshape((Q,) + np.shape(nodes))


# the modes whose Xi(0) entries couple (p_2z, p_2y, p_2y p_2z, p_2x, p_2x p_2z, p_2x p_2y,
# p_2x p_2y p_2z), in mode order
COUPLED = [IDX[(0, 0, 2)], IDX[(0, 2, 0)], IDX[(0, 2, 2)], IDX[(2, 0, 0)], IDX[(2, 0, 2)], IDX[(2, 2, 0)],
           IDX[(2, 2, 2)]]


def local_factor(X: np.ndarray) -> np.ndarray:
    """Q x Q factor of one node's Xi(0) for the local noise: Cholesky of the coupled block in
    mode order with a pivot below zero clamped to zero (a zero pivot leaves its column zero),
    the square roots of the other non-conserved variances."""
    L = np.zeros((Q, Q))
    n = len(COUPLED)
    B = np.zeros((n, n))
    for j in range(n):
        s = X[COUPLED[j], COUPLED[j]] - np.dot(B[j, :j], B[j, :j])
        B[j, j] = np.sqrt(max(s, 0.0))
        for i in range(j + 1, n):
            t = X[COUPLED[i], COUPLED[j]] - np.dot(B[i, :j], B[j, :j])
            B[i, j] = t / B[j, j] if B[j, j] > 0 else 0.0
    L[np.ix_(COUPLED, COUPLED)] = B
    for a in NONCONSERVED:
        if a not in COUPLED:
            L[a, a] = np.sqrt(max(X[a, a], 0.0))
    return L


def noise_lw_local(model: Model, rho: np.ndarray, c2, seed: int, step_index: int) -> np.ndarray:
    """xi[a, z, y, x] of NOISE_LW_LOCAL: the long-wavelength normals, at every node times the
    local factor of Xi(0) of a homogeneous system at that node's density and sound speed."""
    nz, ny, nx = rho.shape
    n = rho.size
    idx = np.arange(n, dtype=np.uint32)
    g = np.concatenate([normals(idx, seed, step_index, t) for t in TAGS], axis=1)
    nu = np.zeros((Q, n))
    nu[NONCONSERVED] = g[:, :len(NONCONSERVED)].T
    r = rho.ravel()
    c = np.broadcast_to(np.asarray(c2, dtype=np.float64), rho.shape).ravel()
    xi = np.zeros((Q, n))
    for k in range(n):
        X = Model(r[k], c[k], model.kappa, model.kT, model.tau_s, model.tau_b, model.tau_ghost).Xi_zero()
        xi[:, k] = local_factor(X) @ nu[:, k]
    return xi.reshape(Q, nz, ny, nx)


# --- correlated noise (Sec. III C, Eq. noise-matrix) ------------------------------------------

TAG_RS = (12, 13)


def lattice_s(kx, ky, kz):
    """Symbol of the D3Q27 Laplacian stencil: -lap e^{ik.r} = s(k) e^{ik.r},
    s = 6 sum_{i != 0} w_i (1 - cos k.c_i)."""
    kv = np.stack(np.broadcast_arrays(np.asarray(kx, float), np.asarray(ky, float), np.asarray(kz, float)), axis=-1)
    return 6.0 * sum(W[i] * (1.0 - np.cos(kv @ C[i].astype(float))) for i in range(1, Q))


def Xi_k(model: Model, kx, ky, kz) -> np.ndarray:
    """Xi(k) = A(k) G(k) A(-k)^T - (1 + Omega(k)) G(k) (1 + Omega(k))^T, Eq. (noise-matrix), with
    G(k) and Omega(k) = Lambda (I - J(k)) those of a homogeneous system at
    c_s^2(k) = cs2 + rho0 kappa s(k) (Eq. sound-speed-k)."""
    c2k = model.cs2 + model.rho0 * model.kappa * float(lattice_s(kx, ky, kz))
    mk = Model(model.rho0, c2k, model.kappa, model.kT, model.tau_s, model.tau_b, model.tau_ghost)
    G = mk.G0()
    O = mk.Omega0()
    ph = np.exp(-1j * (C.astype(float) @ np.array([kx, ky, kz], dtype=float)))
    A = T @ np.diag(ph) @ TINV
    Am = T @ np.diag(np.conj(ph)) @ TINV
    IO = np.eye(Q) + O
    X = A @ G @ Am.T - IO @ G @ IO.T
    return X.real


CORNERS = [(1 if (w >> 2) & 1 == 0 else -1, 1 if (w >> 1) & 1 == 0 else -1, 1 if w & 1 == 0 else -1)
           for w in range(8)]


def s_max() -> float:
    """The largest value of s(k): at k = (pi, pi, pi)."""
    return float(lattice_s(np.pi, np.pi, np.pi))


def _positive_convention(v: np.ndarray) -> np.ndarray:
    """v with the sign that makes its first component of magnitude at least half its
    largest positive (the split's vectors are defined up to sign)."""
    big = np.abs(v) >= 0.5 * np.abs(v).max()
    return -v if v[np.argmax(big)] < 0 else v


def rs_split(model: Model):
    """(Lw, p, q): the rank-two split of the coupled block of Xi(k) = X0 + s(k) D (module
    docstring).  Lw is the Cholesky factor of the white part C = X0 - S q q^T; p and q the
    vectors of D = p p^T - q q^T that whiten X0: with X0 = L0 L0^T and
    L0^-1 D L0^-T = mu+ y+ y+^T + mu- y- y-^T, p = sqrt(mu+) L0 y+ and q = sqrt(-mu-) L0 y-, so
    C = L0 (I - S |mu-| y- y-^T) L0^T.  Raises when X0 is not positive definite, when D has
    more than one eigenvalue of either sign, or when C is not positive semidefinite (X at
    k = (pi, pi, pi) is not)."""
    S = s_max()
    X0 = Xi_k(model, 0.0, 0.0, 0.0)[np.ix_(COUPLED, COUPLED)]
    XS = Xi_k(model, np.pi, np.pi, np.pi)[np.ix_(COUPLED, COUPLED)]
    D = (XS - X0) / S
    L0 = np.linalg.cholesky(X0)
    Y = np.linalg.solve(L0, np.linalg.solve(L0, D).T)         # L0^-1 D L0^-T (symmetric)
    Y = 0.5 * (Y + Y.T)
    mu, E = np.linalg.eigh(Y)
    # Y is relative to X0: eigenvalues below 1e-9 in magnitude are rounding (kappa = 0: none)
    if np.sum(mu > 1e-9) > 1 or np.sum(mu < -1e-9) > 1:
        raise ValueError("the slope of the coupled block is not of rank two with one eigenvalue of each sign")
    mp = mu[-1] if mu[-1] > 1e-9 else 0.0
    mm = mu[0] if mu[0] < -1e-9 else 0.0
    p = _positive_convention(np.sqrt(mp) * (L0 @ E[:, -1])) if mp > 0 else np.zeros(7)
    q = _positive_convention(np.sqrt(-mm) * (L0 @ E[:, 0])) if mm < 0 else np.zeros(7)
    if 1.0 - S * (-mm) < -1e-9:
        raise ValueError("Xi(k) is not positive semidefinite at k = (pi, pi, pi)")
    C = X0 - S * np.outer(q, q)
    return cholesky_psd(0.5 * (C + C.T)), p, q


def rs_weights():
    """(a_p, a_q)[w]: sqrt(s) and sqrt(S - s) at corner w, the amplitudes that give phi_p and
    phi_q the spectra s(k) and S - s(k)."""
    S = s_max()
    sw = np.array([float(lattice_s(*[0.0 if v > 0 else np.pi for v in CORNERS[w]])) for w in range(8)])
    return np.sqrt(np.maximum(sw, 0.0)), np.sqrt(np.maximum(S - sw, 0.0))


def rs_fields(nx, ny, nz, seed: int, step_index: int) -> np.ndarray:
    """nu[w, 2, z, y, x]: the white pair (phi_p's, phi_q's) of corner w at every node."""
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.uint32)
    g = np.concatenate([normals(idx, seed, step_index, t) for t in TAG_RS], axis=1)     # (n, 16)
    return g.T.reshape(8, 2, nz, ny, nx)


def rs_scalar_fields(nx, ny, nz, seed: int, step_index: int) -> np.ndarray:
    """(phi_p, phi_q)[2, z, y, x]: the two box-filtered scalar fields."""
    nu = rs_fields(nx, ny, nz, seed, step_index)
    ap, aq = rs_weights()
    v = np.stack([ap[:, None, None, None] * nu[:, 0], aq[:, None, None, None] * nu[:, 1]], axis=1)
    out = np.zeros((2, nz, ny, nx))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                h = sum((CORNERS[w][0] ** dx) * (CORNERS[w][1] ** dy) * (CORNERS[w][2] ** dz) * v[w]
                        for w in range(8)) / 8.0
                out += np.roll(h, shift=(dz, dy, dx), axis=(1, 2, 3))      # h_d(r - d)
    return out


def xi_coupled_rs(model: Model, nx, ny, nz, seed: int, step_index: int, split=None) -> np.ndarray:
    """xi[7, z, y, x]: the k-dependent part p phi_p + q phi_q of the coupled modes' noise (in
    COUPLED order); the white part is the long-wavelength noise with rs_noise_factor."""
    _, p, q = rs_split(model) if split is None else split
    phi = rs_scalar_fields(nx, ny, nz, seed, step_index)
    return p[:, None, None, None] * phi[0] + q[:, None, None, None] * phi[1]


def rs_noise_factor(model: Model, split=None) -> np.ndarray:
    """Q x Q factor of the white part of the correlated noise: the long-wavelength factor with
    its coupled block replaced by the factor of C."""
    Lw = (rs_split(model) if split is None else split)[0]
    L = model.noise_factor()
    L[np.ix_(COUPLED, COUPLED)] = Lw
    return L


NOISE_OFF, NOISE_LW, NOISE_FULL_RS, NOISE_LW_LOCAL = 0, 1, 4, 5


class Lattice:
    """A periodic nx x ny x nz D3Q27 lattice: f[27, nz, ny, nx] pre-collision populations.
    ``eos`` (a theory.DoubleWell) as for oracle.d3q19.Lattice."""

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
        self._split = None

    def set_params(self, kT, kappa, tau_s, tau_b, tau_ghost, noise_mode):
        m = self.model
        self.model = Model(m.rho0, m.cs2, kappa, kT, tau_s, tau_b, tau_ghost, m.p0_rest)
        self.mode = int(noise_mode)
        noisy = self.mode in (NOISE_LW, NOISE_FULL_RS) and kT > 0
        self._split = rs_split(self.model) if (noisy and self.mode == NOISE_FULL_RS) else None
        if not noisy:
            self._L = None
        elif self._split is not None:
            self._L = rs_noise_factor(self.model, self._split)
        else:
            self._L = self.model.noise_factor()

    def step(self, nsteps=1):
        n = self.nx * self.ny * self.nz
        nodes = np.arange(n, dtype=np.uint32).reshape(self.nz, self.ny, self.nx)
        for _ in range(int(nsteps)):
            xi = None
            if self._L is not None:
                xi = noise_lw_nodes(self.model, nodes, self.seed, self.t, self._L)
                if self._split is not None:
                    xi[COUPLED] += xi_coupled_rs(self.model, self.nx, self.ny, self.nz, self.seed, self.t,
                                                 self._split)
            elif self.mode == NOISE_LW_LOCAL and self.model.kT > 0:
                rho = self.f.sum(axis=0)
                c2 = self.model.cs2 if self.eos is None else self.eos.cs2(rho)
                xi = noise_lw_local(self.model, rho, c2, self.seed, self.t)
            self.f = step(self.f, self.model, xi, self.eos)
            self.t += 1
        return self

    def moments(self):
        return np.einsum("ai,i...->a...", T, self.f)
