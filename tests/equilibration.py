"""Replica statistics of the equilibration tests (Sec. V A).

The paper's measure of thermalisation is the equilibration ratio <|dm_a(k)|^2> / G_aa(k)
of every mode a.  Here it is estimated from R independent replicas (own Philox seeds):
each replica gives its own time average after a burn-in, and the spread of the R values
gives the standard error of their mean, so the tests can ask for agreement within a
stated number of standard errors instead of a fixed tolerance.  The moment spectra are
formed on the device with PyTorch from the FP64 populations the library returns (test
analysis only; the path under test is the library's step)."""
import numpy as np

from oracle import theory as th


def family_z(count, alpha=0.01):
    """Two-sided normal quantile that keeps the chance of any of `count` independent
    correct estimates failing below alpha (Bonferroni)."""
    from scipy.stats import norm
    return float(norm.isf(alpha / (2.0 * count)))


class ModeSpectra:
    """Accumulates, per replica, <|dm_a(k)|^2> with the unitary transform of Sec. III and
    dm = m - mbar (mbar the rest moments), from device FP64 populations."""

    def __init__(self, R, nx, ny, model):
        import torch
        self.torch = torch
        self.R, self.nx, self.ny = R, nx, ny
        self.T = torch.tensor(th.T, dtype=torch.float64, device="cuda")
        self.mbar = torch.tensor(model.mbar(), dtype=torch.float64, device="cuda")[None, :, None, None]
        self.f = torch.empty((R, 9, ny, nx), dtype=torch.float64, device="cuda")
        self.acc = torch.zeros((R, 9, ny, nx), dtype=torch.float64, device="cuda")
        self.samples = 0

    def add(self):
        """Call after self.f holds the current populations of every replica."""
        torch = self.torch
        m = torch.einsum("ai,riyx->rayx", self.T, self.f) - self.mbar
        self.acc += torch.abs(torch.fft.fft2(m)) ** 2 / (self.nx * self.ny)
        self.samples += 1

    def mean(self):
        return (self.acc / self.samples).cpu().numpy()


def kept_wavevectors(nx, ny):
    """Every wavevector but k = 0 (conserved) and the two staggered-momentum invariants
    (pi, 0) and (0, pi) of D2Q9 that never equilibrate (reading R12)."""
    keep = np.ones((ny, nx), bool)
    keep[0, 0] = keep[0, nx // 2] = keep[ny // 2, 0] = False
    return keep


def diag_theory(nx, ny, G_of_k):
    """G_aa(k) on the lattice's wavevectors, shape (9, ny, nx)."""
    KX, KY = th.lattice_k(nx, ny)
    G = np.empty((9, ny, nx))
    for j in range(ny):
        for i in range(nx):
            G[:, j, i] = np.diag(G_of_k(KX[j, i], KY[j, i])).real
    return G


def radial_bins(nx, ny, nb):
    """Radial bin (0 .. nb-1) of every wavevector, |k| with components wrapped to
    (-pi, pi], nb equal bins up to the largest |k|."""
    KX, KY = th.lattice_k(nx, ny)
    kw = np.sqrt(np.minimum(KX, 2 * np.pi - KX) ** 2 + np.minimum(KY, 2 * np.pi - KY) ** 2)
    edges = np.linspace(0, kw.max() + 1e-9, nb + 1)
    return np.clip(np.searchsorted(edges, kw, side="right") - 1, 0, nb - 1), kw


def replica_z(values, target=1.0):
    """Mean over replicas (axis 0), its standard error from the replica spread, and the
    z-score of (mean - target)."""
    v = np.asarray(values, dtype=float)
    R = v.shape[0]
    mean = v.mean(axis=0)
    se = v.std(axis=0, ddof=1) / np.sqrt(R)
    return mean, se, (mean - target) / se
