"""Plane-wave population states of a 3-D box that both the device (torch) and the host (numpy)
can evaluate anywhere: the seeded inputs of the large-lattice sampled tests."""
import numpy as np


def wave_state_box(fbar, dims, z, y, x, amp, xp=np, q=19, seed=21):
    """fbar_i (1 + amp sum_w sin(2 pi (kx x / nx + ky y / ny + kz z / nz) + phi)) on an
    nx x ny x nz box (integer wavevectors per axis)."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    kv = rng.integers(0, 64, size=(q, 3, 3))
    ph = rng.uniform(0, 2 * np.pi, size=(q, 3))
    out = []
    for i in range(q):
        s = 0.0
        for w in range(3):
            kx, ky, kz = (int(v) for v in kv[i, w])
            arg = (2 * np.pi) * (((kx * x) % nx) / nx + ((ky * y) % ny) / ny + ((kz * z) % nz) / nz)
            s = s + xp.sin(arg + float(ph[i, w]))
        out.append(fbar[i] * (1.0 + amp * s))
    return out
