"""Independent numpy checks used to pin the oracle (no code shared with it).

`image_distances` finds the true minimum-image distance by enumerating lattice images
directly (no rounding sequence), which is what the oracle's reduction must reproduce.
"""
from __future__ import annotations

import itertools

import numpy as np


def box_matrix(b) -> np.ndarray:
    Lx, Ly, Lz, xy, xz, yz = np.asarray(b.params() if hasattr(b, "params") else b, np.float64)
    return np.array([[Lx, xy * Ly, xz * Lz], [0.0, Ly, yz * Lz], [0.0, 0.0, Lz]])


def image_distances(b, xi: np.ndarray, xj: np.ndarray, reach: int = 2) -> np.ndarray:
    """min over lattice vectors n (|n_k| <= reach) of |x_j - x_i + M n|, all pairs (i, j)."""
    M = box_matrix(b)
    xi = np.asarray(xi, np.float64)
    xj = np.asarray(xj, np.float64)
    d = xj[None, :, :] - xi[:, None, :]
    # bring every displacement into the primary cell first, then try nearby images
    s = d @ np.linalg.inv(M).T
    d = (s - np.round(s)) @ M.T
    best = np.full(d.shape[:2], np.inf)
    for n in itertools.product(range(-reach, reach + 1), repeat=3):
        shift = M @ np.array(n, np.float64)
        best = np.minimum(best, np.linalg.norm(d + shift, axis=-1))
    return best


def legendre_p(l: int, x) -> np.ndarray:
    c = np.zeros(l + 1)
    c[l] = 1.0
    return np.polynomial.legendre.legval(x, c)


def q_from_bonds(bonds: np.ndarray, l: int) -> float:
    """q_l of one particle from its bond vectors via the addition theorem (numpy)."""
    u = bonds / np.linalg.norm(bonds, axis=1, keepdims=True)
    S = legendre_p(l, np.clip(u @ u.T, -1.0, 1.0)).sum()
    return float(np.sqrt(max(S, 0.0)) / len(u))


def nl_sets(offsets, pj):
    return [set(pj[offsets[i]:offsets[i + 1]].tolist()) for i in range(len(offsets) - 1)]


def image_vectors_2d(b, xi: np.ndarray, xj: np.ndarray, reach: int = 2) -> np.ndarray:
    """Nearest-image vectors x_j - x_i + a1 n1 + a2 n2 (|n_k| <= reach) of a 2D box
    (Lz = 0), all pairs (i, j), shape (len(xi), len(xj), 2), by enumerating images."""
    Lx, Ly, _, xy, _, _ = np.asarray(b.params() if hasattr(b, "params") else b, np.float64)
    M = np.array([[Lx, xy * Ly], [0.0, Ly]])
    xi = np.asarray(xi, np.float64)[:, :2]
    xj = np.asarray(xj, np.float64)[:, :2]
    d = xj[None, :, :] - xi[:, None, :]
    s = d @ np.linalg.inv(M).T
    d = (s - np.round(s)) @ M.T
    best = np.full(d.shape[:2], np.inf)
    vec = np.zeros_like(d)
    for n in itertools.product(range(-reach, reach + 1), repeat=2):
        c = d + M @ np.array(n, np.float64)
        r = np.linalg.norm(c, axis=-1)
        better = r < best
        best = np.where(better, r, best)
        vec[better] = c[better]
    return vec
