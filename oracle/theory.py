"""Linear theory of the fluctuating D2Q9 modified-equilibrium model, in FP64 numpy.

TEST INFRASTRUCTURE ONLY.  This module belongs to the oracle: only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it.
It shares no code with the CUDA library and the library never imports it.

Every function restates one passage of Gross, Adhikari, Cates & Varnik,
"Thermal fluctuations in the lattice Boltzmann method for non-ideal fluids"
(arXiv:1009.0254), named in its docstring.  Indices: velocities i = 1..9 and
moments a = 1..9 of the paper are array positions 0..8 here.

Readings where the paper is silent (also listed in the design notes):
  * the equation of state is linearised as p0(rho) = cs2 * rho, so the rest
    state's moment m4 is d(0) rho0 (Appendix A uses exactly this reference state);
  * lambda_e of Eq. (noise-yeo) is the bulk eigenvalue lambda_b of Table I;
  * one ghost relaxation time sets lambda_q and lambda_eps.
"""
from __future__ import annotations

import numpy as np

# --- lattice constants -------------------------------------------------------

#: D2Q9 velocities in the column order of the printed basis matrix, Eq. (Tmat).
C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1],
              [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.int64)
#: Weights w_1 = 4/9, w_2..5 = 1/9, w_6..9 = 1/36 (Sec. III A).
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
#: sigma_s^2 = 1/3, the ideal lattice-gas sound speed squared (Sec. III, notation).
SIGMA_S2 = 1.0 / 3.0


def basis_T() -> np.ndarray:
    """Basis vectors T_ai from the polynomials of Table I evaluated on the velocities."""
    cx = C[:, 0].astype(np.float64)
    cy = C[:, 1].astype(np.float64)
    c2 = cx * cx + cy * cy
    rows = [
        np.ones(9),                 # 1: rho
        cx,                         # 2: j_x
        cy,                         # 3: j_y
        3 * c2 - 2,                 # 4: e (bulk stress)
        2 * cx * cx - c2,           # 5: p_ww (shear)
        cx * cy,                    # 6: p_xy (shear)
        (3 * c2 - 4) * cx,          # 7: q_x (ghost)
        (3 * c2 - 4) * cy,          # 8: q_y (ghost)
        9 * c2 * c2 - 15 * c2 + 2,  # 9: eps (ghost)
    ]
    return np.array(rows)


T = basis_T()
#: Lengths N_a = sum_i w_i T_ai^2, Eq. (scalar-prod).
N = (T * T * W[None, :]).sum(axis=1)
#: Inverse transform (T^-1)_ia = w_i T_ai / N_a (Sec. III A, below Eq. scalar-prod).
TINV = (W[:, None] * T.T) / N[None, :]


def lambdas(tau_s: float, tau_b: float, tau_ghost: float) -> np.ndarray:
    """Eigenvalues lambda_a = -1/tau_a of the collision operator (Table I; Sec. III A)."""
    lb, ls, lg = -1.0 / tau_b, -1.0 / tau_s, -1.0 / tau_ghost
    return np.array([0.0, 0.0, 0.0, lb, ls, ls, lg, lg, lg])


# --- lattice Fourier transforms (Appendix B) --------------------------------

def laplacian_stencil(a: np.ndarray) -> np.ndarray:
    """Discrete Laplacian of Appendix B on a periodic field a[y, x]:
    sum over the eight moving directions of w_i [a(r+c_i) + a(r-c_i) - 2 a(r)] / sigma_s^2."""
    out = np.zeros_like(a)
    for i in range(1, 9):
        cx, cy = C[i]
        plus = np.roll(a, shift=(-cy, -cx), axis=(0, 1))   # a(r + c_i)
        minus = np.roll(a, shift=(cy, cx), axis=(0, 1))    # a(r - c_i)
        out += W[i] * (plus + minus - 2 * a)
    return out / SIGMA_S2


def k2_lattice(kx, ky):
    """Minus the Fourier symbol of the Appendix B Laplacian; replaces k^2 in S and c_s^2(k)."""
    kx = np.asarray(kx, dtype=np.float64)
    ky = np.asarray(ky, dtype=np.float64)
    sym = (4 / 9 * (np.cos(kx) + np.cos(ky)) + 2 / 9 * np.cos(kx) * np.cos(ky) - 10 / 9) / SIGMA_S2
    return -sym


class DoubleWell:
    """Landau double-well bulk free energy f0 = beta (rho - rhoV)^2 (rho - rhoL)^2 (Sec. II A,
    Eq. f0-bulk), its bulk pressure p0 = rho df0/drho - f0, sound speed squared
    c_s^2 = dp0/drho = rho d2f0/drho2, and the flat-interface results of Eqs. (interf-width)
    and (surf-tension)."""

    def __init__(self, beta, rhoV, rhoL):
        self.beta, self.rhoV, self.rhoL = float(beta), float(rhoV), float(rhoL)

    def f0(self, rho):
        return self.beta * (rho - self.rhoV) ** 2 * (rho - self.rhoL) ** 2

    def df0(self, rho):
        a, b = rho - self.rhoV, rho - self.rhoL
        return 2 * self.beta * a * b * (a + b)

    def d2f0(self, rho):
        a, b = rho - self.rhoV, rho - self.rhoL
        return 2 * self.beta * (a * a + 4 * a * b + b * b)

    def p0(self, rho):
        return rho * self.df0(rho) - self.f0(rho)

    def cs2(self, rho):
        return rho * self.d2f0(rho)

    def width(self, kappa):
        """Interface width xi = sqrt(8 kappa / beta) / (rhoL - rhoV), Eq. (interf-width)."""
        return np.sqrt(8 * kappa / self.beta) / (self.rhoL - self.rhoV)

    def surface_tension(self, kappa):
        """sigma = (rhoL - rhoV)^3 sqrt(2 kappa beta) / 6, Eq. (surf-tension)."""
        return (self.rhoL - self.rhoV) ** 3 * np.sqrt(2 * kappa * self.beta) / 6


class Model:
    """Parameters of one homogeneous run: rho0, cs2, kappa, kT and the relaxation times.
    p0_rest is the bulk pressure of the uniform rest state at rho0 (cs2 rho0 for the
    linearised equation of state; p0(rho0) of a double well, whose fluctuations about rho0
    have cs2 = c_s^2(rho0))."""

    def __init__(self, rho0=1.0, cs2=SIGMA_S2, kappa=0.0, kT=0.0,
                 tau_s=1.0, tau_b=1.0, tau_ghost=1.0, p0_rest=None):
        self.rho0 = float(rho0)
        self.p0_rest = float(cs2) * float(rho0) if p0_rest is None else float(p0_rest)
        self.cs2 = float(cs2)
        self.kappa = float(kappa)
        self.kT = float(kT)
        self.tau_s, self.tau_b, self.tau_ghost = float(tau_s), float(tau_b), float(tau_ghost)
        self.lam = lambdas(tau_s, tau_b, tau_ghost)

    # Eq. (sound-speed-k) with the lattice k^2 of Appendix B
    def cs2_k(self, kx, ky):
        return self.cs2 + self.rho0 * self.kappa * k2_lattice(kx, ky)

    def d_k(self, kx, ky):
        """d(k) = 6 [c_s^2(k) - sigma_s^2], Eq. (eq-mom-yeo)."""
        return 6.0 * (self.cs2_k(kx, ky) - SIGMA_S2)

    def S_k(self, kx, ky):
        """Ornstein-Zernike structure factor rho0 kT / (c_s^2 + rho0 kappa k^2), Eq. (struct-fact)."""
        return self.rho0 * self.kT / self.cs2_k(kx, ky)

    # --- rest state ---------------------------------------------------------
    def mbar(self, kx=0.0, ky=0.0) -> np.ndarray:
        """Reference moments {rho0,0,0,d rho0,0,0,0,0,-d rho0} (Appendix A, last subsection)."""
        d = float(self.d_k(kx, ky))
        m = np.zeros(9)
        m[0] = self.rho0
        m[3] = d * self.rho0
        m[8] = -d * self.rho0
        return m

    def fbar(self, kx=0.0, ky=0.0) -> np.ndarray:
        """Rest populations fbar_i = (T^-1 mbar)_i; at k = 0 the uniform rest state of the run
        for the linearised equation of state."""
        return TINV @ self.mbar(kx, ky)

    def rest(self) -> np.ndarray:
        """Populations of the uniform rest state at rho0: Table II at u = 0, grad rho = 0,
        m4 = -m9 = 6 (p0(rho0) - sigma_s^2 rho0), through T^-1."""
        m = np.zeros(9)
        m[0] = self.rho0
        m[3] = 6 * (self.p0_rest - SIGMA_S2 * self.rho0)
        m[8] = -m[3]
        return TINV @ m

    # --- linearised collision and advection (Sec. III B, C) ------------------
    def Omega(self, kx, ky) -> np.ndarray:
        """Linearised collision operator, Eq. (coll-op-yeo)."""
        d = float(self.d_k(kx, ky))
        lb, ls, lq, le = self.lam[3], self.lam[4], self.lam[6], self.lam[8]
        O = np.zeros((9, 9))
        O[3, 3] = lb
        O[3, 0] = -lb * d
        O[4, 4] = ls
        O[5, 5] = ls
        O[6, 6] = lq
        O[7, 7] = lq
        O[8, 8] = le
        O[8, 0] = le * d
        return O

    @staticmethod
    def A(kx, ky) -> np.ndarray:
        """Moment-space advection A_ab(k) = T_aj exp(-i k.c_j) (T^-1)_jb, Eq. (lb-adv)."""
        ph = np.exp(-1j * (kx * C[:, 0] + ky * C[:, 1]))
        return T @ np.diag(ph) @ TINV

    def M(self, kx, ky) -> np.ndarray:
        """One-step propagator of Eq. (lb-lang-ft): dm(k,t+1) = A(-k)(I+Omega) dm(k,t) + A(-k) xi."""
        return self.A(-kx, -ky) @ (np.eye(9) + self.Omega(kx, ky))

    # --- equilibrium correlations and noise (Sec. III B, C) -------------------
    def G_closed(self, kx, ky) -> np.ndarray:
        """Equal-time mode correlations as printed, Eq. (g-mat-yeo)."""
        S = float(self.S_k(kx, ky))
        d = float(self.d_k(kx, ky))
        Tt = self.rho0 * self.kT / SIGMA_S2
        G = np.zeros((9, 9))
        G[0, 0] = S
        G[0, 3] = G[3, 0] = S * d
        G[0, 8] = G[8, 0] = -S * d
        G[1, 1] = G[2, 2] = Tt * SIGMA_S2
        G[3, 3] = N[3] * S
        G[3, 8] = G[8, 3] = 2 * S * d
        G[4, 4] = N[4] * Tt
        G[5, 5] = N[5] * Tt
        G[6, 6] = N[6] * Tt
        G[7, 7] = N[7] * Tt
        G[8, 8] = N[8] * (S + 3 * Tt) / 4
        return G

    def G_ansatz(self, kx, ky) -> np.ndarray:
        """G from the ansatz <df_i df_j> = (S/rho0) fbar_i(k) delta_ij, Eq. (f-correl-yeo),
        transformed with T as in Eq. (g-correl)."""
        S = float(self.S_k(kx, ky))
        fb = self.fbar(kx, ky)
        return (S / self.rho0) * (T @ np.diag(fb) @ T.T)

    def Xi_closed(self, kx, ky) -> np.ndarray:
        """Noise covariance as printed, Eq. (noise-yeo)."""
        c2k = float(self.cs2_k(kx, ky))
        lb, ls, lq, le = self.lam[3], self.lam[4], self.lam[6], self.lam[8]
        til = lambda l: l * (2 + l)                      # tilde lambda_a = lambda_a (2 + lambda_a)
        til_ee = lb + le + lb * le                       # tilde lambda_{e eps}
        X = np.zeros((9, 9))
        X[3, 3] = N[3] * (2 - 3 * c2k) * til(lb)
        X[3, 8] = X[8, 3] = 12 * (c2k - SIGMA_S2) * til_ee
        X[4, 4] = N[4] * til(ls)
        X[5, 5] = N[5] * til(ls)
        X[6, 6] = N[6] * til(lq)
        X[7, 7] = N[7] * til(lq)
        X[8, 8] = N[8] * (5 / 4 - 3 / 4 * c2k) * til(le)
        return -(self.rho0 * self.kT / SIGMA_S2) * X

    def Xi_fdt(self, kx, ky, G=None) -> np.ndarray:
        """Noise covariance from the LB fluctuation-dissipation theorem, Eq. (noise-matrix):
        Xi = A(k) G A(-k)^T - (I + Omega) G (I + Omega)^T."""
        if G is None:
            G = self.G_closed(kx, ky)
        A = self.A(kx, ky)
        Am = self.A(-kx, -ky)
        IO = np.eye(9) + self.Omega(kx, ky)
        X = A @ G @ Am.T - IO @ G @ IO.T
        return X.real if np.abs(X.imag).max() < 1e-12 * max(1.0, np.abs(X).max()) else X

    def Xi_zero(self) -> np.ndarray:
        """Long-wavelength noise Xi(0) = -G Omega^T - Omega G - Omega G Omega^T, Eq. (noise-matrix-k0)."""
        G = self.G_closed(0.0, 0.0)
        O = self.Omega(0.0, 0.0)
        return -G @ O.T - O @ G - O @ G @ O.T

    # --- hydrodynamic limit (Sec. II C, Eq. bulkv-yeo, Appendix C) ------------
    def shear_viscosity(self):
        """eta = rho0 sigma_s^2 (tau_s - 1/2) (text after Eq. bulkv-yeo)."""
        return self.rho0 * SIGMA_S2 * (self.tau_s - 0.5)

    def bulk_viscosity(self, kx, ky):
        """zeta(k) = rho0 sigma_s^2 (tau_b - 1/2) [2 - c_s^2(k)/sigma_s^2], Eq. (bulkv-yeo)."""
        return self.rho0 * SIGMA_S2 * (self.tau_b - 0.5) * (2 - self.cs2_k(kx, ky) / SIGMA_S2)


# --- noise factorisation (Sec. IV) -------------------------------------------

def cholesky_psd(X: np.ndarray, rel_tol: float = 1e-12) -> np.ndarray:
    """Lower-triangular L with L L^T = X for a positive-semidefinite X (Sec. IV: the
    Cholesky factorisation is done on the lower-right (n-d-1) block of Xi, modes 4..9).

    Plain Cholesky-Banachiewicz; a pivot that is zero up to ``rel_tol`` (relative to the
    largest diagonal entry) is clamped to 0 and its column left zero.  Raises if X has a
    clearly negative pivot (not PSD)."""
    n = X.shape[0]
    L = np.zeros_like(X, dtype=np.float64)
    scale = max(float(np.max(np.abs(np.diag(X)))), 1e-300)
    for j in range(n):
        s = X[j, j] - np.dot(L[j, :j], L[j, :j])
        if s <= rel_tol * scale:
            if s < -1e-9 * scale:
                raise ValueError("matrix is not positive semidefinite (pivot %g)" % s)
            continue
        L[j, j] = np.sqrt(s)
        for i in range(j + 1, n):
            L[i, j] = (X[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    return L


def eigen_factor_2x2(a, b, c):
    """Factor L = S diag(sqrt(e1), sqrt(e2)) of the symmetric PSD block [[a, b], [b, c]]
    (Sec. IV, the eigen-decomposition alternative to Cholesky): e1 >= e2 its eigenvalues,
    S = [[cos t, -sin t], [sin t, cos t]] their eigenvectors, t in [0, pi) with
    tan 2t = 2b / (a - c), i.e. t = atan2(2b, a - c) / 2 shifted by pi when negative (the
    first eigenvector's y component is >= 0; this keeps L continuous where b changes sign
    while a < c, the case of the (4,9) block of this model).  Returns (L11, L12, L21, L22);
    vectorised; a negative e2 that is zero up to rounding is clamped to 0."""
    a, b, c = np.asarray(a, float), np.asarray(b, float), np.asarray(c, float)
    half = 0.5 * (a + c)
    rad = np.sqrt(0.25 * (a - c) ** 2 + b * b)
    e1, e2 = half + rad, half - rad
    scale = np.maximum(np.abs(a), np.abs(c)) + 1e-300
    if np.any(e2 < -1e-9 * scale):
        raise ValueError("matrix is not positive semidefinite")
    t = 0.5 * np.arctan2(2.0 * b, a - c)
    t = np.where(t < 0, t + np.pi, t)
    r1, r2 = np.sqrt(np.maximum(e1, 0.0)), np.sqrt(np.maximum(e2, 0.0))
    return np.cos(t) * r1, -np.sin(t) * r2, np.sin(t) * r1, np.cos(t) * r2


def noise_factor(Xi: np.ndarray, factor: str = "cholesky") -> np.ndarray:
    """9x9 factor L with xi = L nu and L L^T = Xi for a PSD noise matrix whose conserved
    rows vanish (Sec. IV); rows/columns 1..3 are zero.  factor = "cholesky": Cholesky of
    the lower-right 6x6 block (modes 4..9); "eigen": the eigen-decomposition factor
    S diag(sqrt(e)) of every block of that matrix (the (4,9) block is the only one that is
    not diagonal in this model)."""
    L = np.zeros((9, 9))
    if factor == "cholesky":
        L[3:, 3:] = cholesky_psd(Xi[3:, 3:])
        return L
    if factor != "eigen":
        raise ValueError("unknown factor %r" % factor)
    off = Xi[3:, 3:] - np.diag(np.diag(Xi[3:, 3:]))
    off[0, 5] = off[5, 0] = 0.0
    if np.any(np.abs(off) > 1e-12 * (np.abs(Xi).max() + 1e-300)):
        raise ValueError("the eigen factor expects only the (4,9) block to be coupled")
    for a in (4, 5, 6, 7):
        L[a, a] = np.sqrt(max(Xi[a, a], 0.0))
    l11, l12, l21, l22 = eigen_factor_2x2(Xi[3, 3], Xi[3, 8], Xi[8, 8])
    L[3, 3], L[3, 8], L[8, 3], L[8, 8] = float(l11), float(l12), float(l21), float(l22)
    return L


def min_eig_block49(model: Model, kx, ky):
    """Smallest eigenvalue of the k-dependent (4,9) block of Xi(k) (the other entries are
    constant).  Vectorised over arrays of k."""
    c2k = model.cs2_k(kx, ky)
    lb, le = model.lam[3], model.lam[8]
    pref = -(model.rho0 * model.kT / SIGMA_S2)
    a = pref * N[3] * (2 - 3 * c2k) * lb * (2 + lb)
    b = pref * 12 * (c2k - SIGMA_S2) * (lb + le + lb * le)
    c = pref * N[8] * (5 / 4 - 3 / 4 * c2k) * le * (2 + le)
    tr = a + c
    disc = np.sqrt(np.maximum((a - c) ** 2 + 4 * b * b, 0.0))
    return 0.5 * (tr - disc)


def lattice_k(nx: int, ny: int):
    """Wavevector grid k = 2 pi (mx/nx, my/ny), arrays indexed [my, mx]."""
    kx = 2 * np.pi * np.arange(nx) / nx
    ky = 2 * np.pi * np.arange(ny) / ny
    return np.meshgrid(kx, ky, indexing="xy")


def lyapunov_G(model: Model, kx, ky, Xi_k: np.ndarray) -> np.ndarray:
    """Stationary G of dm(t+1) = M dm(t) + A(-k) xi with <xi xi^H> = Xi_k:
    solves G = M G M^H + A(-k) Xi_k A(-k)^H (stationarity of Eq. lb-lang-ft)."""
    from scipy.linalg import solve_discrete_lyapunov
    M = model.M(kx, ky)
    Am = model.A(-kx, -ky)
    Q = Am @ Xi_k @ Am.conj().T
    G = solve_discrete_lyapunov(M, Q)
    return G
