"""The library's packed per-macro vector layout, restated for the tests.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Layout (a property of the library interface, written here from its
definition): a vector of a P1 (P2) space at level l holds, for every macro in
order, all lattice points of resolution N = 2^l (N = 2^(l+1)) in the order
k slowest, then j, i fastest -- including the points on the macro's faces,
edges and vertices, which are therefore stored once per macro that contains
them.  A vector-valued field stores 3 components per point (component
fastest), and a batch of nrhs right-hand sides stores the batch index
fastest of all.
"""
from __future__ import annotations

import numpy as np

from .assemble import Space


def to_packed(space: Space, xg: np.ndarray, ncomp: int = 1, nrhs: int = 1) -> np.ndarray:
    """Global (oracle-numbered) vector -> packed library layout, every copy filled."""
    xg = np.asarray(xg).reshape(space.ndof, ncomp, nrhs)
    return xg[space.gid.reshape(-1)].reshape(-1)


def from_packed(space: Space, xp: np.ndarray, ncomp: int = 1, nrhs: int = 1) -> np.ndarray:
    """Packed library layout -> global vector, taking the copy in the lowest-numbered macro."""
    xp = np.asarray(xp).reshape(-1, ncomp, nrhs)
    flat = space.gid.reshape(-1)
    _, first = np.unique(flat, return_index=True)      # first occurrence = lowest macro
    out = xp[first]
    return out.reshape(-1) if (ncomp == 1 and nrhs == 1) else out.reshape(space.ndof * ncomp * nrhs)


def copies_spread(space: Space, xp: np.ndarray, ncomp: int = 1, nrhs: int = 1) -> float:
    """Largest difference between copies of the same DoF in a packed vector."""
    xp = np.asarray(xp, dtype=np.float64).reshape(-1, ncomp * nrhs)
    flat = space.gid.reshape(-1)
    lo = np.full((space.ndof, ncomp * nrhs), np.inf)
    hi = np.full((space.ndof, ncomp * nrhs), -np.inf)
    np.minimum.at(lo, flat, xp)
    np.maximum.at(hi, flat, xp)
    return float(np.max(hi - lo)) if len(flat) else 0.0


def n1_to_packed(space, xg: np.ndarray) -> np.ndarray:
    """Global N1 vector -> packed (doubled-lattice) layout in macro-local orientation."""
    from .mesh import lattice_size
    P = lattice_size(2 * space.n)
    out = np.zeros((space.mesh.nmacro, P))
    out[:, space.edge_pos] = space.local_sign * np.asarray(xg)[space.gid]
    return out.reshape(-1)


def n1_from_packed(space, xp: np.ndarray) -> np.ndarray:
    """Packed N1 vector -> global vector, from the copy in the lowest-numbered macro."""
    from .mesh import lattice_size
    P = lattice_size(2 * space.n)
    xp = np.asarray(xp, dtype=np.float64).reshape(space.mesh.nmacro, P)[:, space.edge_pos]
    vals = space.local_sign * xp
    flat = space.gid.reshape(-1)
    _, first = np.unique(flat, return_index=True)
    return vals.reshape(-1)[first]


def n1_copies_spread(space, xp: np.ndarray) -> float:
    """Largest difference between the copies (global orientation) of a shared edge."""
    from .mesh import lattice_size
    P = lattice_size(2 * space.n)
    vals = (space.local_sign * np.asarray(xp, dtype=np.float64).reshape(space.mesh.nmacro, P)[:, space.edge_pos])
    flat, v = space.gid.reshape(-1), vals.reshape(-1)
    lo = np.full(space.ndof, np.inf)
    hi = np.full(space.ndof, -np.inf)
    np.minimum.at(lo, flat, v)
    np.maximum.at(hi, flat, v)
    return float(np.max(hi - lo))
