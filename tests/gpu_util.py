"""Shared helpers of the GPU parity tests (test code only)."""
import numpy as np

C19 = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
                (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)])
OPP = np.array([0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17])
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def random_state(mask, amp, seed):
    """Unshifted populations f = w (1 + amp * noise) at fluid nodes, w at solids."""
    rng = np.random.default_rng(seed)
    f = W[:, None, None, None] * (1 + amp * rng.standard_normal((19,) + mask.shape))
    f[:, mask == 1] = W[:, None]
    return f


def dev_err(a, b, w=W):
    """max |a - b| relative to the largest deviation of b from rest."""
    wb = w.reshape((19,) + (1,) * (b.ndim - 1))
    return np.abs(a - b).max() / max(np.abs(b - wb).max(), 1e-300)


def sample_nodes(mask, count, seed):
    """Random fluid node indices of a mask [Lz, Ly, Lx]."""
    rng = np.random.default_rng(seed)
    flat = np.flatnonzero(mask.reshape(-1) == 0)
    return np.sort(rng.choice(flat, size=min(count, flat.size), replace=False))


def upstream_nodes(mask, nodes):
    """Node index of x - c_i for every node and direction: [len(nodes), 19]."""
    Lz, Ly, Lx = mask.shape
    x = nodes % Lx
    y = (nodes // Lx) % Ly
    z = nodes // (Lx * Ly)
    xs = (x[:, None] - C19[None, :, 0]) % Lx
    ys = (y[:, None] - C19[None, :, 1]) % Ly
    zs = (z[:, None] - C19[None, :, 2]) % Lz
    return xs + Lx * (ys + Ly * zs)
