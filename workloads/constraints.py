"""Mechanical support conditions as per-DOF masks (input description).

A mask is a uint8 array of length 3 * n_nodes, DOF index = 3 * node + component,
node = (k * (ny+1) + j) * (nx+1) + i; nonzero = displacement held at zero.
"""
from __future__ import annotations

import numpy as np


def _nid(p, i, j, k):
    return (k * (p.ny + 1) + j) * (p.nx + 1) + i


def clamped_bottom(p) -> np.ndarray:
    """Every node of the z = 0 face fixed in x, y and z."""
    m = np.zeros((p.nz + 1, p.ny + 1, p.nx + 1, 3), np.uint8)
    m[0] = 1
    return m.reshape(-1)


def kinematic_mount(p) -> np.ndarray:
    """Minimum constraint of Sec. III-B: the bottom-face centre node fixed in
    x, y, z; the node on the bottom face's right edge (x = max) with the
    centre's y fixed in y and z; the node on the bottom face's top edge
    (y = max) with the centre's x fixed in z. The centre node is
    (nx//2, ny//2, 0)."""
    m = np.zeros(3 * p.n_nodes, np.uint8)
    ic, jc = p.nx // 2, p.ny // 2
    c0 = _nid(p, ic, jc, 0)
    c1 = _nid(p, p.nx, jc, 0)
    c2 = _nid(p, ic, p.ny, 0)
    m[3 * c0:3 * c0 + 3] = 1
    m[3 * c1 + 1] = m[3 * c1 + 2] = 1
    m[3 * c2 + 2] = 1
    return m


def from_node_bits(bits: np.ndarray) -> np.ndarray:
    """uint8 per node with bit c set for a fixed component c -> DOF mask."""
    b = np.asarray(bits, np.uint8).reshape(-1)
    return np.stack([(b >> c) & 1 for c in range(3)], axis=1).astype(np.uint8).reshape(-1)


def to_node_bits(mask: np.ndarray) -> np.ndarray:
    m = np.asarray(mask, np.uint8).reshape(-1, 3)
    return (m[:, 0] | (m[:, 1] << 1) | (m[:, 2] << 2)).astype(np.uint8)
